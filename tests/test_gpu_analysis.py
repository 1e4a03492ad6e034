"""Accuracy-analysis kernels through the C ABI against the oracle: condition
numbers of the local systems, the modified wavenumber of Eq. 2d_mw, the
per-node relative error of Eq. relative_error and the (n, m, q) sweep built
on them (Section 4)."""
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


@pytest.mark.parametrize("nmq", [(28, 7, 3), (28, 7, 4), (21, 5, 2), (15, 3, -1)])
def test_condition_numbers_match_oracle(R, nmq):
    """Every stencil of a 20 x 20 cavity's V->V and P->V families: within
    1e-7 relative of the oracle's dense inverse (cond ~ 1e6: the inverse's
    entries carry about cond * 1e-16 of rounding)."""
    nd = ns.jittered_cavity(20, 0)
    ctx = R.Context(*nmq)
    for ax, ay, bx, by in ((nd.vx, nd.vy, nd.vx, nd.vy), (nd.px, nd.py, nd.vx, nd.vy)):
        idx, _, bad = R.build_weights(ctx, _d(ax), _d(ay), _d(bx), _d(by), R.OP_DX)
        assert bad == -1
        c = R.stencil_condition(ctx, _d(ax), _d(ay), _d(bx), _d(by), idx).cpu().numpy()
        gi = idx.cpu().numpy()[:, : ax.size].T.astype(np.int64)
        ref = O.stencil_condition(ax, ay, bx, by, gi, nmq[1], nmq[2])
        assert np.abs(c / ref - 1).max() < 1e-7


@pytest.mark.parametrize("theta", [0.0, 0.4, np.pi / 4, 1.2])
def test_modified_wavenumber_matches_oracle(R, theta):
    """k*/k~ of (kx D_x + ky D_y)/k~ and k*^2/k~^2 of D_Lap at k~ dr = sqrt(2)
    (the paper's reference point) and at k~ dr = 0.5, both grid pairs."""
    nd = ns.jittered_cavity(24, 1)
    ctx = R.Context(28, 7, 3)
    for ax, ay, bx, by in ((nd.vx, nd.vy, nd.vx, nd.vy), (nd.px, nd.py, nd.vx, nd.vy)):
        idx, w, _ = R.build_weights(ctx, _d(ax), _d(ay), _d(bx), _d(by),
                                    R.OP_DX | R.OP_DY | R.OP_LAP)
        gi = idx.cpu().numpy()[:, : ax.size].T.astype(np.int64)
        W = [w[o].cpu().numpy()[:, : ax.size].T for o in range(3)]
        dr = O.local_spacing(bx, by).mean()
        for ktdr in (np.sqrt(2.0), 0.5):
            kt = ktdr / dr
            kx, ky = kt * np.cos(theta), kt * np.sin(theta)
            k1, k2 = R.modified_wavenumber(ctx, idx, w[0], w[1], _d(ax), _d(ay), _d(bx), _d(by),
                                           kx, ky, idx, w[2])
            r1, r2 = O.modified_wavenumber_local(W[0], W[1], gi, ax, ay, bx, by, kx, ky, W[2])
            assert np.abs(k1.cpu().numpy() - r1).max() < 1e-9
            assert np.abs(k2.cpu().numpy() - r2).max() < 1e-9
            # the oracle's global-phase form of Eq. 2d_mw agrees too
            g = O.modified_wavenumber(W[0], W[1], gi, ax, ay, bx, by, kx, ky) / kt
            assert np.abs(k1.cpu().numpy() - g).max() < 1e-7


@pytest.mark.parametrize("op", ["dx", "dy", "lap", "interp"])
def test_stencil_error_matches_oracle(R, op):
    """Per-node relative error of every operator on the node-scaled test
    function, with dr from each stencil (collocated V-set) and with dr given
    (P <- V), and the device-reduced mean."""
    ops = {"dx": (R.OP_DX, O.OP_DX), "dy": (R.OP_DY, O.OP_DY), "lap": (R.OP_LAP, O.OP_LAP),
           "interp": (R.OP_INTERP, O.OP_INTERP)}
    bit, oop = ops[op]
    nd = ns.jittered_cavity(30, 2)
    ctx = R.Context(28, 7, 3)
    for ax, ay, bx, by, given in ((nd.vx, nd.vy, nd.vx, nd.vy, False),
                                  (nd.px, nd.py, nd.vx, nd.vy, True)):
        idx, w, _ = R.build_weights(ctx, _d(ax), _d(ay), _d(bx), _d(by), bit)
        dr = O.local_spacing(ax, ay)
        err, mean = R.stencil_error(ctx, idx, w[0], bit, _d(ax), _d(ay), _d(bx), _d(by),
                                    _d(dr) if given else None)
        gi = idx.cpu().numpy()[:, : ax.size].T.astype(np.int64)
        W = w[0].cpu().numpy()[:, : ax.size].T
        ref = O.stencil_error(W, gi, ax, ay, bx, by, oop, dr)
        assert np.abs(err.cpu().numpy() - ref).max() < 1e-9
        assert abs(float(mean) - ref.mean()) < 1e-11


def test_parameter_sweep_matches_oracle_and_paper_trends(R):
    """The GPU sweep over (n, m, q) reproduces the oracle's mean errors and the
    trends the paper bases its choice on (Section 4.1-4.2)."""
    from paper_2206_06495_gb300.sweep import parameter_sweep
    nd = ns.jittered_cavity(40, 0)
    x, y = nd.vx, nd.vy
    inner = (x > 0.2) & (x < 0.8) & (y > 0.2) & (y < 0.8)
    ax, ay = x[inner], y[inner]
    dr = O.local_spacing(x, y)[inner]
    triples = [(28, 3, 3), (28, 5, 3), (28, 7, 1), (28, 7, 3), (28, 7, 4), (21, 7, 3), (35, 7, 3)]
    rows = parameter_sweep(_d(ax), _d(ay), _d(x), _d(y), triples, R.OP_DX | R.OP_LAP, _d(dr),
                           condition=True)
    E = {}
    for r in rows:
        t = (r["n"], r["m"], r["q"])
        idx, W = O.build_weights(ax, ay, x, y, *t, (O.OP_DX, O.OP_LAP))
        for key, op in (("dx", O.OP_DX), ("lap", O.OP_LAP)):
            ref = O.stencil_error(W[op], idx, ax, ay, x, y, op, dr).mean()
            assert abs(float(r["E_" + key]) - ref) < 1e-10 * max(1.0, ref), (t, key)
        E[t] = float(r["E_dx"])
        assert r["bad_node"] == -1 and torch.isfinite(r["cond"]).all()
    assert E[(28, 3, 3)] > E[(28, 5, 3)] > E[(28, 7, 3)]
    assert E[(21, 7, 3)] > E[(28, 7, 3)] > E[(35, 7, 3)]
    assert E[(28, 7, 1)] > E[(28, 7, 3)] and E[(28, 7, 4)] >= E[(28, 7, 3)]
