"""rbffd_ensemble_step through the C ABI: every member of a batched ensemble
of cavities (different Reynolds numbers and lid speeds, one node set, shared
operators) against its own oracle run of the paper's step."""
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


def _run(R, n, seed, Re, lid, steps, dt):
    nd = ns.jittered_cavity(n, seed)
    E = len(Re)
    ctx = R.Context(28, 7, 3)
    flow = R.flow_from_nodes(ctx, nd, Re=1.0, dt=dt, precision=R.PREC_MIXED, tol=1e-11,
                             inner_tol=5e-3)
    gu = np.zeros((nd.N, E))
    for e in range(E):
        gu[:, e] = O.lid_bc(nd, lid[e])[0]
    gu_d = torch.as_tensor(np.ascontiguousarray(gu.ravel()), device="cuda")
    gv_d = torch.zeros_like(gu_d)
    st = R.ensemble_zeros(flow, E)
    stats = R.ensemble_step(ctx, flow, Re, st, gu_d, gv_d, steps)
    out = {k: getattr(st, k).cpu().numpy().reshape(-1, E)
           for k in ("u", "v", "pt", "p", "cu_prev", "cv_prev")}
    ops = O.build_operators(nd)
    for e in range(E):
        fs = O.FractionalStep(nd, Re=Re[e], dt=dt, ops=ops)
        s = fs.initial_state()
        g = O.lid_bc(nd, lid[e])
        for _ in range(steps):
            s = fs.step(s, *g)
        du = max(np.abs(out["u"][:, e] - s.u).max(), np.abs(out["v"][:, e] - s.v).max())
        assert du < 1e-6 * max(1.0, lid[e]), (e, du)
        for k in ("pt", "p", "cu_prev", "cv_prev"):
            ref = getattr(s, k)
            err = np.abs(out[k][:, e] - ref).max() / np.abs(ref).max()
            assert err < 1e-5, (e, k, err)
    return stats


def test_ensemble_config0_members_match_oracle(R):
    """Four cavities on the config-0 node set (40 x 40, dt 2e-3), Re 100 to
    2,500 and lid speeds 0.5 to 1.2, 200 steps in one batched call; the
    multigrid hierarchy here is its dense coarsest level only."""
    stats = _run(R, 40, 0, [100.0, 400.0, 1000.0, 2500.0], [1.0, 0.8, 1.2, 0.5], 200, 2e-3)
    assert stats["steps"] == 200


def test_ensemble_multilevel_members_match_oracle(R):
    """Eight cavities on a 100 x 100 node set (the V-cycle has levels below its
    coarsest one), Re drawn from U[100, 5000] like the configured ensemble,
    lid speeds 1 + 0.05 N(0, 1), 40 steps of dt 2e-3."""
    rng = np.random.default_rng(4)
    Re = list(rng.uniform(100.0, 5000.0, 8))
    lid = list(1.0 + 0.05 * rng.standard_normal(8))
    _run(R, 100, 4, Re, lid, 40, 2e-3)


def test_ensemble_refuses_bad_member_counts(R):
    nd = ns.jittered_cavity(12, 0)
    ctx = R.Context(28, 7, 3)
    flow = R.flow_from_nodes(ctx, nd, Re=1.0, dt=2e-3)
    st = R.ensemble_zeros(flow, 3)
    g = torch.zeros(nd.N * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RbffdError) as e:
        R.ensemble_step(ctx, flow, [100.0, 200.0, 300.0], st, g, g.clone(), 1)
    assert e.value.code == R.ERR_INVALID_ARG
