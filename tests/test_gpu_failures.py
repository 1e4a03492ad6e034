"""Error codes of rbffd_step through the C ABI (include/rbffd.h), and the
Kim & Moin modes other than the default, against the oracle.

Failures are made on the host: an iteration cap too small to converge, wall
data with a NaN, and a staged-copy wait told to give up at once through the
test hook rbffd_debug_set_wait_limit (the kernels then wait, bounded, for
their own copies and report through the solve's error flag).  Nothing here
traps, faults or hangs the GPU."""
import numpy as np
import pytest

from oracle import rbffd_oracle as O
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


def _setup(R, n=16, precision=None, **kw):
    ctx = R.Context(28, 7, 3)
    nd = ns.jittered_cavity(n, 0)
    prec = R.PREC_FP64 if precision is None else precision
    flow = R.flow_from_nodes(ctx, nd, Re=100.0, dt=2e-3, precision=prec, tol=1e-12, **kw)
    gu, gv = O.lid_bc(nd)
    return ctx, nd, flow, _d(gu), _d(gv)


def test_iteration_cap_returns_not_converged_with_stats(R):
    """max_iter = 1: a solve of the step cannot reach 1e-12 (the viscous one,
    or, when its extrapolated guess lets it converge in one iteration, the
    pressure one), the call returns RBFFD_ERR_NOT_CONVERGED with the
    statistics filled, and the state keeps the last completed step."""
    ctx, nd, flow, gu, gv = _setup(R)
    st = R.State.zeros(flow)
    R.step(ctx, flow, st, gu, gv, 2)
    u2 = st.u.clone()
    flow.max_iter = 1
    with pytest.raises(R.RbffdError) as e:
        R.step(ctx, flow, st, gu, gv, 1)
    assert e.value.code == R.ERR_NOT_CONVERGED
    stats = e.value.stats
    assert stats["steps"] == 0 and stats["helm_iters"] >= 1
    if stats["poisson_iters"] == 0:  # the viscous solve stopped the step
        assert stats["helm_relres"] > 1e-12
    else:
        assert stats["helm_relres"] <= 1e-12 and stats["poisson_relres"] > 1e-12
    assert st.j == 2 and torch.equal(st.u, u2)
    flow.max_iter = 20000
    R.step(ctx, flow, st, gu, gv, 1)
    assert st.j == 3


def test_nonfinite_wall_data_returns_nonfinite(R):
    ctx, nd, flow, gu, gv = _setup(R)
    st = R.State.zeros(flow)
    bad = gu.clone()
    wall = int(np.nonzero(nd.v_boundary)[0][3])
    bad[wall] = float("nan")
    with pytest.raises(R.RbffdError) as e:
        R.step(ctx, flow, st, bad, gv, 1)
    assert e.value.code == R.ERR_NONFINITE


def test_staged_copy_wait_that_gives_up_reports_and_recovers(R):
    """With the first wait limited to zero polls every staged SpMV tile is
    given up: the step returns RBFFD_ERR_CUDA naming the bounded wait, and
    after the default limit is restored the same context steps normally and
    matches a fresh run bit for bit.  MIXED precision: its FP32 Krylov SpMVs
    stage their tiles (the FP64 ones load directly)."""
    ctx, nd, flow, gu, gv = _setup(R, precision=R.PREC_MIXED)
    st = R.State.zeros(flow)
    R.debug_set_wait_limit(ctx, 0)
    try:
        with pytest.raises(R.RbffdError) as e:
            R.step(ctx, flow, st, gu, gv, 1)
    finally:
        R.debug_set_wait_limit(ctx, -1)
    assert e.value.code == R.ERR_CUDA and "bounded wait" in str(e.value)
    assert st.j == 0
    st = R.State.zeros(flow)
    R.step(ctx, flow, st, gu, gv, 3)
    ctx2, _, flow2, _, _ = _setup(R, precision=R.PREC_MIXED)
    st2 = R.State.zeros(flow2)
    R.step(ctx2, flow2, st2, gu, gv, 3)
    assert torch.equal(st.u, st2.u) and torch.equal(st.pt, st2.pt)


@pytest.mark.parametrize("km_mode", [0, 1])
def test_kim_moin_modes_match_oracle(R, km_mode):
    """The wall value of u** without the pressure term (0) and with its
    tangential component only (1): 20 steps on a 20 x 20 cavity in FP64
    against the oracle with the same mode (velocities 1e-9, p~ 1e-8)."""
    ctx = R.Context(28, 7, 3)
    nd = ns.jittered_cavity(20, 0)
    flow = R.flow_from_nodes(ctx, nd, Re=100.0, dt=2e-3, precision=R.PREC_FP64, tol=1e-12,
                             km_mode=km_mode)
    st = R.State.zeros(flow)
    gu, gv = O.lid_bc(nd)
    R.step(ctx, flow, st, _d(gu), _d(gv), 20)
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3, km_mode=km_mode)
    s = fs.initial_state()
    for _ in range(20):
        s = fs.step(s, gu, gv)
    assert np.abs(st.u.cpu().numpy() - s.u).max() < 1e-9
    assert np.abs(st.v.cpu().numpy() - s.v).max() < 1e-9
    assert np.abs(st.pt.cpu().numpy() - s.pt).max() < 1e-8 * np.abs(s.pt).max()
