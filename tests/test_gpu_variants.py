"""The step's variants through the C ABI against the oracle: the exactly
projecting step (projection = RBFFD_PROJ_EXACT: pressure operator
D^(P,V) G0, discretely divergence-free velocity) and Kim & Moin's
Crank-Nicolson right side (cn_form = RBFFD_CN_KIM_MOIN)."""
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


def _oracle(nd, steps, Re, dt, **kw):
    fs = O.FractionalStep(nd, Re=Re, dt=dt, **kw)
    gu, gv = O.lid_bc(nd)
    st = fs.initial_state()
    for _ in range(steps):
        st = fs.step(st, gu, gv)
    return fs, st


def _gpu(R, nd, steps, Re, dt, precision, **kw):
    ctx = R.Context(28, 7, 3)
    flow = R.flow_from_nodes(ctx, nd, Re=Re, dt=dt, precision=precision,
                             tol=1e-12 if precision == R.PREC_FP64 else 1e-11, **kw)
    st = R.State.zeros(flow)
    gu, gv = O.lid_bc(nd)
    stats = R.step(ctx, flow, st, _d(gu), _d(gv), steps)
    return ctx, flow, st, stats


def _check(st, ref, tol_u, tol_p):
    du = max(np.abs(st.u.cpu().numpy() - ref.u).max(), np.abs(st.v.cpu().numpy() - ref.v).max())
    assert du < tol_u, du
    for name, got, want in (("pt", st.pt, ref.pt), ("p", st.p, ref.p)):
        err = np.abs(got.cpu().numpy() - want).max() / np.abs(want).max()
        assert err < tol_p, (name, err)


@pytest.mark.parametrize("precision,tol_u,tol_p", [(0, 1e-9, 1e-8), (1, 1e-6, 1e-5)])
def test_exact_projection_matches_oracle_and_is_divergence_free(R, precision, tol_u, tol_p):
    """20 x 20 cavity, Re 100, dt 2e-3, 100 steps with the composed pressure
    operator: every field against the oracle's exact projection, the wall flux
    against the oracle's, and D^(P,V) u_{j+1} (applied by rbffd_apply_op)
    zero at every P-node to the solve's tolerance."""
    nd = ns.jittered_cavity(20, 0)
    fs, ref = _oracle(nd, 100, 100.0, 2e-3, projection="exact")
    ctx, flow, st, stats = _gpu(R, nd, 100, 100.0, 2e-3, precision, projection=R.PROJ_EXACT)
    _check(st, ref, tol_u, tol_p)
    assert abs(stats["wall_flux"] - ref.lam) < 1e3 * tol_u * max(abs(ref.lam), 1e-3)
    t = flow.tensors
    div = (R.apply_op(ctx, t["pv_idx"], t["pv_dx"], nd.M, nd.N, st.u)
           + R.apply_op(ctx, t["pv_idx"], t["pv_dy"], nd.M, nd.N, st.v)).cpu().numpy()
    ref_div = fs.ops.pv_x @ st.u.cpu().numpy() + fs.ops.pv_y @ st.v.cpu().numpy()
    scale = np.abs(fs.ops.pv_x).sum(1).max()
    assert np.abs(div).max() < 1e-8 * scale, np.abs(div).max()
    assert np.abs(ref_div).max() < 1e-8 * scale


_exact150 = {}


@pytest.mark.parametrize("precision,tol_u,tol_p", [(0, 1e-8, 1e-8), (1, 1e-6, 1e-5)])
def test_exact_projection_multilevel_matches_oracle(R, precision, tol_u, tol_p):
    """150 x 150 cavity at the benchmark's Re 1e4 and dt 2e-4, 30 steps,
    preconditioned by the multigrid V-cycle (several levels) on the composed
    operator, in both precisions."""
    nd = ns.jittered_cavity(150, 5)
    if "ref" not in _exact150:
        _exact150["ref"] = _oracle(nd, 30, 1e4, 2e-4, projection="exact",
                                   viscous_solver="krylov")[1]
    _, _, st, _ = _gpu(R, nd, 30, 1e4, 2e-4, precision, projection=R.PROJ_EXACT)
    _check(st, _exact150["ref"], tol_u, tol_p)


@pytest.mark.parametrize("projection", ["paper", "exact"])
def test_kim_moin_crank_nicolson_matches_oracle(R, projection):
    """cn_form = Kim & Moin: right side u* + a D_Lap u_j; 20 steps on a 20 x 20
    cavity (Re 100, dt 2e-3) in FP64 for both projections."""
    nd = ns.jittered_cavity(20, 0)
    _, ref = _oracle(nd, 20, 100.0, 2e-3, projection=projection, cn_form="kim_moin")
    _, _, st, _ = _gpu(R, nd, 20, 100.0, 2e-3, R.PREC_FP64, cn_form=R.CN_KIM_MOIN,
                       projection=R.PROJ_EXACT if projection == "exact" else R.PROJ_PAPER)
    _check(st, ref, 1e-9, 1e-8)


def test_adjoint_refuses_the_variants(R):
    nd = ns.jittered_cavity(12, 0)
    ctx = R.Context(28, 7, 3)
    flow = R.flow_from_nodes(ctx, nd, Re=100.0, dt=2e-3, projection=R.PROJ_EXACT)
    st = R.State.zeros(flow)
    lam = R.Adjoint.zeros(flow)
    g = torch.zeros(nd.N, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RbffdError) as e:
        R.adjoint_step(ctx, flow, st, lam, g, g.clone())
    assert e.value.code == R.ERR_INVALID_ARG
