"""rbffd_build_weights_noalloc: the allocation-free variant of the stencil and
weight build, for callers that may not allocate GPU memory.  It must return
what rbffd_build_weights returns, call after call, although every call reuses
the same fixed device array (this file is collected last on purpose)."""
import ctypes as C

import numpy as np
import pytest

from paper_2206_06495_gb300 import nodesets as ns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    from paper_2206_06495_gb300 import build
    build.build()
    from paper_2206_06495_gb300 import rbffd
    return rbffd


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _noalloc(R, params, ax, ay, bx, by, mask):
    na = ax.numel()
    ld = R.round_up(na)
    nops = len(R.ops_of(mask))
    idx = torch.full((params.n, ld), -7, dtype=torch.int32, device="cuda")
    w = torch.full((nops, params.n, ld), np.nan, dtype=torch.float64, device="cuda")
    bad = C.c_int64(123)
    torch.cuda.synchronize()
    rc = R.lib().rbffd_build_weights_noalloc(C.byref(params), R._ptr(ax), R._ptr(ay), na,
                                             R._ptr(bx), R._ptr(by), bx.numel(), mask,
                                             R._ptr(idx), R._ptr(w), ld, C.byref(bad),
                                             R._stream())
    return rc, idx, w, bad.value


def _check_same(R, ctx, params, ax, ay, bx, by, mask):
    rc, idx, w, bad = _noalloc(R, params, ax, ay, bx, by, mask)
    assert rc == R.OK and bad == -1
    ref_idx, ref_w, ref_bad = R.build_weights(ctx, ax, ay, bx, by, mask)
    assert ref_bad == -1
    na = ax.numel()
    assert torch.equal(idx[:, :na], ref_idx[:, :na])
    a, b = w[:, :, :na], ref_w[:, :, :na]
    rel = ((a - b).abs().amax(dim=1) / b.abs().amax(dim=1)).max().item()
    assert rel < 1e-12, rel


def test_noalloc_matches_allocating_build_on_consecutive_calls(R):
    params = R.Params(28, 7, 3)
    ctx = R.Context(28, 7, 3)
    mask = R.OP_DX | R.OP_DY | R.OP_LAP
    a = ns.jittered_cavity(17, 11)
    b = ns.jittered_cavity(41, 12)
    # call 1: V-values -> P-nodes on a small set; call 2: V -> V on a larger
    # one, over scratch that still holds call 1's buckets; call 3 repeats call 1
    _check_same(R, ctx, params, _d(a.px), _d(a.py), _d(a.vx), _d(a.vy), mask)
    _check_same(R, ctx, params, _d(b.vx), _d(b.vy), _d(b.vx), _d(b.vy), mask)
    _check_same(R, ctx, params, _d(a.px), _d(a.py), _d(a.vx), _d(a.vy), mask)


def test_noalloc_other_parameters(R):
    params = R.Params(21, 5, 2)
    ctx = R.Context(21, 5, 2)
    a = ns.jittered_cavity(23, 13)
    _check_same(R, ctx, params, _d(a.vx), _d(a.vy), _d(a.px), _d(a.py), R.OP_INTERP | R.OP_LAP)


def test_noalloc_rejects_sizes_beyond_its_scratch(R):
    n_beta = 65537
    x = _d(np.random.default_rng(0).random(n_beta))
    y = _d(np.random.default_rng(1).random(n_beta))
    rc, idx, w, bad = _noalloc(R, R.Params(28, 7, 3), x[:100].contiguous(), y[:100].contiguous(),
                               x, y, R.OP_DX)
    assert rc == R.ERR_INVALID_ARG
    assert (idx == -7).all()  # nothing was written
