"""The discrete adjoint on the GPU (rbffd_adjoint_step, the checkpointed
autograd rollout) against the oracle's adjoint and central differences."""
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


def _setup(R, n=12, Re=400.0, dt=2e-3, seed=0):
    nd = ns.jittered_cavity(n, 4)
    rng = np.random.default_rng(seed)
    lid = nd.v_wall == ns.WALL_TOP
    g0 = np.zeros(nd.N)
    g0[lid] = 1 + 0.05 * rng.standard_normal(lid.sum())
    u0 = np.zeros(nd.N)
    inner = ~nd.v_boundary
    u0[inner] = 0.01 * rng.standard_normal(inner.sum())
    ctx = R.Context()
    flow = R.flow_from_nodes(ctx, nd, Re=Re, dt=dt, tol=1e-13)
    fs = O.FractionalStep(nd, Re=Re, dt=dt)
    return nd, ctx, flow, fs, g0, u0


@pytest.mark.parametrize("j_start", [0, 3])
def test_adjoint_step_matches_oracle(R, j_start):
    nd, ctx, flow, fs, g0, u0 = _setup(R)
    st = fs.initial_state(u0, np.zeros(nd.N))
    for _ in range(j_start):
        st = fs.step(st, g0, np.zeros(nd.N))
    rng = np.random.default_rng(7)
    lam_np = O.AdjointState(rng.standard_normal(nd.N), rng.standard_normal(nd.N),
                            rng.standard_normal(nd.N), rng.standard_normal(nd.N),
                            rng.standard_normal(nd.M))
    ref, rgu, rgv = O.adjoint_step(fs, st, lam_np)
    fwd = R.State(_d(st.u), _d(st.v), _d(st.cu_prev), _d(st.cv_prev), _d(st.pt), _d(st.p), st.j)
    lam = R.Adjoint(_d(lam_np.u), _d(lam_np.v), _d(lam_np.cu_prev), _d(lam_np.cv_prev),
                    _d(lam_np.pt))
    gu = torch.zeros(nd.N, dtype=torch.float64, device="cuda")
    gv = torch.zeros_like(gu)
    R.adjoint_step(ctx, flow, fwd, lam, gu, gv)
    for name, got, want in (("u", lam.u, ref.u), ("v", lam.v, ref.v),
                            ("cu", lam.cu_prev, ref.cu_prev), ("cv", lam.cv_prev, ref.cv_prev),
                            ("pt", lam.pt, ref.pt), ("gu", gu, rgu), ("gv", gv, rgv)):
        g = got.cpu().numpy()
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(g - want).max() <= 1e-8 * scale, (name, np.abs(g - want).max(), scale)


def test_rollout_gradient_matches_oracle_and_central_differences(R):
    """J = 1/2 sum(u^2 + v^2) after 10 steps, checkpoints every 4 steps (a
    ragged last segment): gradient with respect to per-node lid velocity and
    to the initial velocity, against the oracle adjoint (1e-7) and central
    differences of the GPU forward solver (1e-4, the target tolerance)."""
    from paper_2206_06495_gb300.autograd import rollout
    nd, ctx, flow, fs, g0, u0 = _setup(R)
    steps = 10
    gu = _d(g0).requires_grad_(True)
    gv = torch.zeros(nd.N, dtype=torch.float64, device="cuda", requires_grad=True)
    u0t = _d(u0).requires_grad_(True)
    v0t = torch.zeros(nd.N, dtype=torch.float64, device="cuda", requires_grad=True)
    u, v = rollout(ctx, flow, gu, gv, u0t, v0t, steps, every=4)
    J = 0.5 * (u * u + v * v).sum()
    J.backward()
    # oracle adjoint of the same objective
    sts = [fs.initial_state(u0, np.zeros(nd.N))]
    for _ in range(steps):
        sts.append(fs.step(sts[-1], g0, np.zeros(nd.N)))
    lam = O.AdjointState(sts[-1].u.copy(), sts[-1].v.copy(), np.zeros(nd.N), np.zeros(nd.N),
                         np.zeros(nd.M))
    G = np.zeros(nd.N)
    for j in range(steps - 1, -1, -1):
        lam, lgu, _ = O.adjoint_step(fs, sts[j], lam)
        G += lgu
    lid = nd.v_wall == ns.WALL_TOP
    ggu = gu.grad.cpu().numpy()
    assert np.abs(ggu[lid] - G[lid]).max() <= 1e-7 * np.abs(G[lid]).max()
    inner = ~nd.v_boundary
    gu0 = u0t.grad.cpu().numpy()
    assert np.abs(gu0[inner] - lam.u[inner]).max() <= 1e-7 * np.abs(lam.u[inner]).max()

    def J_gpu(g, uu):
        st = R.State.zeros(flow)
        st.u.copy_(_d(uu))
        gut = _d(g)
        gvt = torch.zeros_like(gut)
        R.step(ctx, flow, st, gut, gvt, steps)
        return 0.5 * float((st.u * st.u).sum() + (st.v * st.v).sum())

    eps = 1e-6
    for k in np.nonzero(lid)[0][:3]:
        gp, gm = g0.copy(), g0.copy()
        gp[k] += eps
        gm[k] -= eps
        fd = (J_gpu(gp, u0) - J_gpu(gm, u0)) / (2 * eps)
        assert abs(ggu[k] - fd) <= 1e-4 * abs(fd), (k, ggu[k], fd)
    for k in np.nonzero(inner)[0][[3, 50]]:
        up, um = u0.copy(), u0.copy()
        up[k] += eps
        um[k] -= eps
        fd = (J_gpu(g0, up) - J_gpu(g0, um)) / (2 * eps)
        assert abs(gu0[k] - fd) <= 1e-4 * max(abs(fd), 1e-3), (k, gu0[k], fd)
