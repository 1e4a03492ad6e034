"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
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


@pytest.fixture(scope="module")
def ctx(R):
    return R.Context(28, 7, 3)


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


OPS = (O.OP_INTERP, O.OP_DX, O.OP_DY, O.OP_LAP)


def _pairs(nd):
    return {"vv": (nd.vx, nd.vy, nd.vx, nd.vy), "pv": (nd.px, nd.py, nd.vx, nd.vy),
            "pp": (nd.px, nd.py, nd.px, nd.py), "vp": (nd.vx, nd.vy, nd.px, nd.py)}


@pytest.mark.parametrize("n", [12, 23])
def test_knn_bit_exact(R, ctx, n):
    nd = ns.jittered_cavity(n, 3)
    for name, (ax, ay, bx, by) in _pairs(nd).items():
        idx, w, bad = R.build_weights(ctx, _d(ax), _d(ay), _d(bx), _d(by), R.OP_DX)
        assert bad == -1
        got = idx.cpu().numpy()[:, : ax.size].T
        ref = O.knn(ax, ay, bx, by, 28)
        assert np.array_equal(got, ref), name


def test_knn_exact_lattice_ties(R, ctx):
    """Exact lattice: the 28th neighbour sits in a 4-way tie, broken by index."""
    g = np.arange(9, dtype=float) * 0.125
    x, y = np.meshgrid(g, g, indexing="ij")
    x, y = x.ravel(), y.ravel()
    idx, _, _ = R.build_weights(ctx, _d(x), _d(y), _d(x), _d(y), R.OP_INTERP)
    assert np.array_equal(idx.cpu().numpy()[:, : x.size].T, O.knn(x, y, x, y, 28))


@pytest.mark.parametrize("q", [3, 4])
def test_weights_match_oracle(R, q):
    ctx = R.Context(28, 7, q)
    nd = ns.jittered_cavity(17, 4)
    mask = R.OP_INTERP | R.OP_DX | R.OP_DY | R.OP_LAP
    for name, (ax, ay, bx, by) in _pairs(nd).items():
        idx, w, bad = R.build_weights(ctx, _d(ax), _d(ay), _d(bx), _d(by), mask)
        assert bad == -1
        n = ax.size
        gi = idx.cpu().numpy()[:, :n].T.astype(np.int64)
        _, W = O.build_weights(ax, ay, bx, by, 28, 7, q, OPS, idx=gi)
        wg = w.cpu().numpy()[:, :, :n]
        for o, op in enumerate(OPS):
            ref = W[op]
            got = wg[o].T
            rel = np.abs(got - ref).max(1) / np.abs(ref).max(1)
            assert rel.max() < 1e-10, (name, op, rel.max())


def test_weights_other_params(R):
    """A runtime-sized stencil (n = 21, m = 5, q = 2) and plain RBF-FD (q = -1)."""
    nd = ns.jittered_cavity(12, 5)
    for (n, m, q) in ((21, 5, 2), (15, 3, -1)):
        ctx = R.Context(n, m, q)
        idx, w, bad = R.build_weights(ctx, _d(nd.px), _d(nd.py), _d(nd.vx), _d(nd.vy),
                                      R.OP_DX | R.OP_LAP)
        gi = idx.cpu().numpy()[:, : nd.M].T.astype(np.int64)
        assert np.array_equal(gi, O.knn(nd.px, nd.py, nd.vx, nd.vy, n))
        _, W = O.build_weights(nd.px, nd.py, nd.vx, nd.vy, n, m, q, (O.OP_DX, O.OP_LAP), idx=gi)
        for o, op in enumerate((O.OP_DX, O.OP_LAP)):
            got = w.cpu().numpy()[o][:, : nd.M].T
            rel = np.abs(got - W[op]).max(1) / np.abs(W[op]).max(1)
            assert rel.max() < 1e-9, (n, m, q, op, rel.max())


@pytest.mark.parametrize("n", [15, 20, 37])
def test_masked_one_sided_stencils_match_oracle(R, ctx, n):
    """Boundary P-nodes: slot 0 = the node, then its 27 nearest interior P-nodes."""
    nd = ns.jittered_cavity(n, 8)
    bnd = np.nonzero(nd.p_boundary)[0]
    rows = _d(bnd.astype(np.int32))
    idx, w, bad = R.build_weights_masked(ctx, _d(nd.px[bnd]), _d(nd.py[bnd]), _d(nd.px),
                                         _d(nd.py), R.OP_DX | R.OP_DY,
                                         beta_mask=_d((~nd.p_boundary).astype(np.uint8)),
                                         alpha_self=rows)
    assert bad == -1
    gi = idx.cpu().numpy()[:, : bnd.size].T.astype(np.int64)
    ref = O.knn(nd.px[bnd], nd.py[bnd], nd.px, nd.py, 28, beta_mask=~nd.p_boundary,
                alpha_self=bnd)
    assert np.array_equal(gi, ref)
    _, W = O.build_weights(nd.px[bnd], nd.py[bnd], nd.px, nd.py, 28, 7, 3, (O.OP_DX, O.OP_DY),
                           idx=ref)
    for o, op in enumerate((O.OP_DX, O.OP_DY)):
        got = w[o].cpu().numpy()[:, : bnd.size].T
        assert (np.abs(got - W[op]).max(1) / np.abs(W[op]).max(1)).max() < 1e-10


def test_masked_rejects_too_few_candidates(R, ctx):
    nd = ns.jittered_cavity(6, 9)  # 36 P-nodes, 16 interior
    bnd = np.nonzero(nd.p_boundary)[0]
    with pytest.raises(R.RbffdError) as e:
        R.build_weights_masked(ctx, _d(nd.px[bnd]), _d(nd.py[bnd]), _d(nd.px), _d(nd.py),
                               R.OP_DX, beta_mask=_d((~nd.p_boundary).astype(np.uint8)),
                               alpha_self=_d(bnd.astype(np.int32)))
    assert e.value.code == R.ERR_INVALID_ARG


def test_singular_stencil_reported(R, ctx):
    """Duplicate beta-nodes make the systems that contain both singular."""
    nd = ns.jittered_cavity(10, 6)
    bx = np.concatenate([nd.px, nd.px[:3]])
    by = np.concatenate([nd.py, nd.py[:3]])
    idx, w, bad = R.build_weights(ctx, _d(nd.px), _d(nd.py), _d(bx), _d(by), R.OP_DX)
    assert bad == 0


def test_invalid_args_rejected(R, ctx):
    x = _d(np.zeros(10))
    with pytest.raises(R.RbffdError) as e:
        R.build_weights(ctx, x, x, x, x, R.OP_DX)  # 28 > 10 beta-nodes
    assert e.value.code == R.ERR_INVALID_ARG
    with pytest.raises(R.RbffdError):
        R.Context(28, 6, 3)  # even exponent


def test_empty_inputs_are_no_ops(R, ctx):
    """No alpha-nodes and no operator rows: the calls succeed and touch nothing."""
    rng = np.random.default_rng(4)
    e = _d(np.zeros(0))
    bx, by = _d(rng.random(40)), _d(rng.random(40))
    idx, w, bad = R.build_weights(ctx, e, e, bx, by, R.OP_DX | R.OP_LAP)
    assert bad == -1 and tuple(w.shape) == (2, 28, 32)
    idx.fill_(0)
    w.fill_(1.0)
    y = R.apply_op(ctx, idx, w[0], 0, 40, _d(np.ones(40)))
    assert y.numel() == 0
    # a zero-row operator leaves an existing output alone
    y = _d(np.full(3, 7.0))
    R.apply_op(ctx, idx, w[0], 0, 40, _d(np.ones(40)), y, alpha=2.0, beta=0.5)
    assert (y.cpu().numpy() == 7.0).all()


@pytest.mark.parametrize("wdt", ["f64", "f32"])
def test_apply_op_matches_csr(R, ctx, wdt):
    nd = ns.jittered_cavity(33, 7)
    idx, w, _ = R.build_weights(ctx, _d(nd.vx), _d(nd.vy), _d(nd.px), _d(nd.py),
                                R.OP_DX | R.OP_LAP)
    gi = idx.cpu().numpy()[:, : nd.N].T.astype(np.int64)
    f, *_ = ns.wave_test_function(nd.px, nd.py)
    for o in range(2):
        wt = w[o] if wdt == "f64" else w[o].float()
        D = O.csr(gi, wt.cpu().numpy()[:, : nd.N].T.astype(np.float64), nd.M)
        ref = D @ f
        x = _d(f) if wdt == "f64" else _d(f).float()
        y0 = torch.ones(nd.N, dtype=x.dtype, device="cuda")
        y = R.apply_op(ctx, idx, wt, nd.N, nd.M, x, y0.clone(), alpha=2.0, beta=-0.5)
        got = y.double().cpu().numpy()
        tol = 1e-12 if wdt == "f64" else 2e-6
        scale = np.abs(D).sum(1).A.ravel() * np.abs(f).max()
        assert (np.abs(got - (2.0 * ref - 0.5)) / scale).max() < tol


def _run_cavity(R, ctx, n, steps, precision, Re=100.0, dt=2e-3):
    nd = ns.jittered_cavity(n, 0)
    flow = R.flow_from_nodes(ctx, nd, Re=Re, dt=dt, precision=precision,
                             tol=1e-12 if precision == R.PREC_FP64 else 1e-11)
    st = R.State.zeros(flow)
    gu, gv = O.lid_bc(nd)
    stats = R.step(ctx, flow, st, _d(gu), _d(gv), steps)
    return nd, flow, st, stats


def test_step_fp64_matches_oracle_short(R, ctx):
    nd, flow, st, stats = _run_cavity(R, ctx, 20, 20, R.PREC_FP64)
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3)
    s = fs.initial_state()
    gu, gv = O.lid_bc(nd)
    for _ in range(20):
        s = fs.step(s, gu, gv)
    assert np.abs(st.u.cpu().numpy() - s.u).max() < 1e-9
    assert np.abs(st.v.cpu().numpy() - s.v).max() < 1e-9
    assert np.abs(st.pt.cpu().numpy() - s.pt).max() < 1e-8 * np.abs(s.pt).max()
    assert np.abs(st.p.cpu().numpy() - s.p).max() < 1e-8 * np.abs(s.p).max()
    assert np.abs(st.cu_prev.cpu().numpy() - s.cu_prev).max() < 1e-8


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_step_config0_500_steps(R, ctx, precision, tol):
    """Lid-driven cavity Re 100, 40 x 40 jittered P-lattice, dt 2e-3, 500 steps."""
    nd, flow, st, stats = _run_cavity(R, ctx, 40, 500, precision)
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3)
    s = fs.initial_state()
    gu, gv = O.lid_bc(nd)
    for _ in range(500):
        s = fs.step(s, gu, gv)
    du = np.abs(st.u.cpu().numpy() - s.u).max()
    dv = np.abs(st.v.cpu().numpy() - s.v).max()
    assert du < tol and dv < tol, (du, dv, stats)
    # the other fields of the state, relative to their size: the FP64 path to
    # 1e-8 throughout.  Mixed precision: the convective terms C_{j-1} are
    # products of FP32-weight derivative stencils, each of the k = 28 weights
    # rounded by 2^-24, so they are good to about k 2^-24 = 1.7e-6 of their
    # scale; they and the pressures (which that rounding reaches through the
    # divergence, undamped by the pressure solve) are held to 1e-5
    ptol = tol if precision == 0 else 1e-5
    for name, got, ref, t in (("pt", st.pt, s.pt, ptol), ("p", st.p, s.p, ptol),
                              ("cu_prev", st.cu_prev, s.cu_prev, ptol),
                              ("cv_prev", st.cv_prev, s.cv_prev, ptol)):
        err = np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < t, (name, err)


def test_apply_op_autotuned_shape_is_a_candidate_and_result_independent(R):
    """rbffd_apply_op picks its launch shape by timing candidates on first use;
    every shape adds each row's terms in the same order, so two contexts (which
    may pick different shapes) return identical bits."""
    nd = ns.jittered_cavity(60, 7)
    outs = []
    for _ in range(2):
        ctx = R.Context(28, 7, 3)
        idx, w, _ = R.build_weights(ctx, _d(nd.vx), _d(nd.vy), _d(nd.vx), _d(nd.vy), R.OP_LAP)
        f, *_ = ns.wave_test_function(nd.vx, nd.vy)
        for wdt, x in ((w[0], _d(f)), (w[0].float(), _d(f).float())):
            y = R.apply_op(ctx, idx, wdt, nd.N, nd.N, x)
            t, b = R.apply_op_shape(ctx, idx, wdt, nd.N, nd.N, x.dtype)
            assert (t, b) in {(128, 4), (128, 8), (128, 16), (256, 2), (256, 4), (256, 8),
                              (512, 2), (512, 4)}
            outs.append(y.cpu().numpy())
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])
