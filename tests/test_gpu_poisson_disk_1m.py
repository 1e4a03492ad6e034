"""The operator workload on 1,000,000 scattered nodes: Poisson-disk points in
the unit square (one collocated set), batched weights of d/dx, d/dy and the
Laplacian for (n, m, q) = (28, 7, 3) (38 x 38 systems) and (28, 7, 4)
(43 x 43 systems), applied to f = sin(8 pi x + 4 pi y) cos(6 pi y) as FP64 and
FP32 ELL SpMVs.  Sampled stencils and weights against the oracle (computed row
by row), sampled SpMV rows against FP64 sums, and the truncation error against
the analytic derivatives over the interior.  Its bounds come from the oracle's
errors at 10,000 and 40,000 points (first derivatives converge like h^3 for
q = 3, the Laplacian like h^2), extrapolated to 1,000,000 points (h five
times smaller than at 40,000) with a margin of about ten."""
import numpy as np
import pytest

from oracle import rbffd_oracle as O
from paper_2206_06495_gb300 import nodesets as ns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_PTS = 1_000_000
SAMPLES = 64


@pytest.fixture(scope="module")
def R():
    from paper_2206_06495_gb300 import build
    build.build()
    from paper_2206_06495_gb300 import rbffd
    return rbffd


@pytest.fixture(scope="module")
def pts():
    return ns.poisson_disk(N_PTS, 1)


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("q", [3, 4])
def test_weights_spmv_and_truncation_error(R, pts, q):
    x, y = pts
    n = x.size
    ctx = R.Context(28, 7, q)
    X, Y = _d(x), _d(y)
    idx, w, bad = R.build_weights(ctx, X, Y, X, Y, R.OP_DX | R.OP_DY | R.OP_LAP)
    assert bad == -1
    rng = np.random.default_rng(10 + q)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, SAMPLES, replace=False)]))
    ti = torch.as_tensor(rows, device="cuda")
    got_idx = idx[:, ti].T.cpu().numpy().astype(np.int64)
    ref_idx = O.knn(x[rows], y[rows], x, y, 28, chunk=8)
    assert np.array_equal(got_idx, ref_idx)
    ops = (O.OP_DX, O.OP_DY, O.OP_LAP)
    _, W = O.build_weights(x[rows], y[rows], x, y, 28, 7, q, ops, idx=ref_idx)
    for o, op in enumerate(ops):
        got = w[o][:, ti].T.cpu().numpy()
        rel = np.abs(got - W[op]).max(1) / np.abs(W[op]).max(1)
        assert rel.max() < 1e-10, (q, op, rel.max())

    f, fx, fy, lap = ns.wave_test_function(x, y)
    F64, F32 = _d(f), _d(f).float()
    # away from the walls, where stencils turn one-sided
    inner = (x > 0.02) & (x < 0.98) & (y > 0.02) & (y < 0.98)
    for o, exact, bound in ((0, fx, 1e-5), (1, fy, 1e-5), (2, lap, 3e-4)):
        y64 = R.apply_op(ctx, idx, w[o], n, n, F64).cpu().numpy()
        err = np.abs(y64 - exact)[inner].max() / np.abs(exact).max()
        assert err < bound, (q, o, err)
        # sampled rows: FP64 sums, and the FP32 SpMV to its rounding level
        ww = w[o][:, ti].T.double().cpu().numpy()
        ref = (ww * f[got_idx]).sum(1)
        scale = (np.abs(ww) * np.abs(f[got_idx])).sum(1)
        assert (np.abs(y64[rows] - ref) / scale).max() < 1e-13
        y32 = R.apply_op(ctx, idx, w[o].float(), n, n, F32).double().cpu().numpy()
        assert (np.abs(y32[rows] - ref) / scale).max() < 2e-6
