"""The package's smoke entry point (one small run of the hot path checked
against the oracle) passes on the GPU."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    pytest.importorskip("torch")
    import __graft_entry__ as g
    g.smoke()
