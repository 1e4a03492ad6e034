"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a special case that reduces to a simpler textbook problem, a
convergence rate, a brute-force count, or a bound the paper prints.
"""
import os

import numpy as np
import pytest

from oracle import rbffd_oracle as O
from paper_2206_06495_gb300 import nodesets as ns

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def cavity20():
    return ns.jittered_cavity(20, 0)


@pytest.fixture(scope="module")
def ops20(cavity20):
    return O.build_operators(cavity20)


def test_parameters_and_monomial_count():
    g = _golden("parameters.txt")
    assert len(O.monomial_exponents(int(g["q"]))) == g["n_monomials_q3"]
    assert len(O.monomial_exponents(int(g["q_variant"]))) == g["n_monomials_q4"]
    # graded lexicographic order, reading R2
    assert O.monomial_exponents(2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]


# ---------------------------------------------------------------- stencils
def test_knn_exact_lattice_shells():
    """On a perfect unit lattice the shells around an interior node hold
    1, 4, 4, 4, 8, 4, 4 nodes at d^2 = 0, 1, 2, 4, 5, 8, 9; the 28 nearest are
    the 25 nodes with d^2 <= 8 plus the 3 lowest-index nodes at d^2 = 9."""
    n = 11
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = ii.ravel().astype(float)
    y = jj.ravel().astype(float)
    c = 5 * n + 5
    idx = O.knn(x[[c]], y[[c]], x, y, 28)[0]
    d2 = (x[idx] - x[c]) ** 2 + (y[idx] - y[c]) ** 2
    assert idx[0] == c
    assert np.all(np.diff(d2) >= 0)
    assert np.count_nonzero(d2 <= 8) == 25
    ring9 = np.nonzero((x - x[c]) ** 2 + (y - y[c]) ** 2 == 9)[0]
    assert sorted(idx[d2 == 9]) == sorted(ring9)[:3]


def test_knn_brute_force_small_random():
    """Against a direct enumeration of all pairs on a tiny set."""
    rng = np.random.default_rng(5)
    x, y = rng.random(60), rng.random(60)
    qx, qy = rng.random(7), rng.random(7)
    idx = O.knn(qx, qy, x, y, 9)
    for i in range(7):
        pairs = sorted(((x[j] - qx[i]) ** 2 + (y[j] - qy[i]) ** 2, j) for j in range(60))
        assert list(idx[i]) == [j for _, j in pairs[:9]]


def test_knn_tree_path_equals_brute_force():
    """The k-d tree candidate path of the oracle's k-NN gives exactly the
    brute-force stencils: random points, a masked candidate set, one-sided
    stencils (alpha_self) and an exact lattice full of distance ties."""
    rng = np.random.default_rng(11)
    bx, by = rng.random(2500), rng.random(2500)
    ax, ay = rng.random(600), rng.random(600)
    for k in (28, 9):
        assert np.array_equal(O.knn(ax, ay, bx, by, k, method="tree"),
                              O.knn(ax, ay, bx, by, k, method="brute"))
    mask = rng.random(2500) < 0.5
    assert np.array_equal(O.knn(ax, ay, bx, by, 28, beta_mask=mask, method="tree"),
                          O.knn(ax, ay, bx, by, 28, beta_mask=mask, method="brute"))
    selfi = np.arange(40)
    mask2 = np.ones(2500, bool)
    mask2[:40] = False
    assert np.array_equal(
        O.knn(bx[:40], by[:40], bx, by, 28, beta_mask=mask2, alpha_self=selfi, method="tree"),
        O.knn(bx[:40], by[:40], bx, by, 28, beta_mask=mask2, alpha_self=selfi, method="brute"))
    n = 25
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x, y = ii.ravel() * 0.1, jj.ravel() * 0.1
    assert np.array_equal(O.knn(x, y, x, y, 28, method="tree"), O.knn(x, y, x, y, 28, method="brute"))


# ---------------------------------------------------------------- weights
@pytest.mark.parametrize("q", [3, 4])
def test_polynomial_exactness_all_grids(cavity20, q):
    """P1: every operator reproduces derivatives of all monomials of degree
    <= q exactly (vanishing-moment conditions, Section 2.1)."""
    nd = cavity20
    pairs = {"vv": (nd.vx, nd.vy, nd.vx, nd.vy), "pv": (nd.px, nd.py, nd.vx, nd.vy),
             "pp": (nd.px, nd.py, nd.px, nd.py), "vp": (nd.vx, nd.vy, nd.px, nd.py)}
    for name, (ax, ay, bx, by) in pairs.items():
        idx, W = O.build_weights(ax, ay, bx, by, 28, 7, q, O.ALL_OPS)
        for a, b in O.monomial_exponents(q):
            f = bx ** a * by ** b
            ex = {
                O.OP_INTERP: ax ** a * ay ** b,
                O.OP_DX: a * ax ** max(a - 1, 0) * ay ** b,
                O.OP_DY: b * ax ** a * ay ** max(b - 1, 0),
                O.OP_LAP: a * (a - 1) * ax ** max(a - 2, 0) * ay ** b
                + b * (b - 1) * ax ** a * ay ** max(b - 2, 0),
            }
            for op in O.ALL_OPS:
                got = (W[op] * f[idx]).sum(1)
                scale = 1.0 / nd.h ** (2 if op == O.OP_LAP else 1)
                assert np.abs(got - ex[op]).max() < 1e-8 * scale, (name, op, a, b)


def test_exactness_stops_at_degree_q(cavity20):
    """The reproduction is not accidental: degree q+1 is not exact."""
    nd = cavity20
    idx, W = O.build_weights(nd.vx, nd.vy, nd.vx, nd.vy, 28, 7, 3, (O.OP_DX,))
    f = nd.vx ** 4
    err = np.abs((W[O.OP_DX] * f[idx]).sum(1) - 4 * nd.vx ** 3).max()
    assert err > 1e-6


def test_weight_sum_identities(ops20):
    """Sum of weights: 0 for derivatives, and sum w_j x_j = 1 for d/dx."""
    for D in (ops20.vv_x, ops20.vv_lap, ops20.pv_y, ops20.pp_lap, ops20.vp_x):
        assert np.abs(D.sum(1)).max() < 1e-8 / 0.05 ** 2


def test_interpolation_is_lagrange_on_collocated(cavity20):
    """An interpolant through the stencil reproduces the data at the stencil
    nodes, so collocated interpolation weights are the unit vector e_0."""
    nd = cavity20
    idx, W = O.build_weights(nd.px, nd.py, nd.px, nd.py, 28, 7, 3, (O.OP_INTERP,))
    e0 = np.zeros(28)
    e0[0] = 1.0
    assert np.abs(W[O.OP_INTERP] - e0).max() < 1e-9


def test_unisolvent_special_case_is_polynomial_interpolation():
    """P2: with n equal to the number of monomials the vanishing-moment rows
    alone fix w (P^T w = L P); the RBF block drops out.  Checked against the
    transposed Vandermonde system solved on its own."""
    rng = np.random.default_rng(3)
    q = 3
    mono = O.monomial_exponents(q)
    X = rng.uniform(-1, 1, (len(mono), 2))
    c = np.array([0.1, -0.2])
    w, _ = O.stencil_weights(c, X, 7, q, (O.OP_DX, O.OP_LAP))
    Xl = X - c
    V = np.array([[xl ** a * yl ** b for a, b in mono] for xl, yl in Xl])
    rhs_dx = np.array([1.0 if ab == (1, 0) else 0.0 for ab in mono])
    rhs_lap = np.array([2.0 if ab in ((2, 0), (0, 2)) else 0.0 for ab in mono])
    assert np.allclose(w[O.OP_DX], np.linalg.solve(V.T, rhs_dx), rtol=1e-8, atol=1e-8)
    assert np.allclose(w[O.OP_LAP], np.linalg.solve(V.T, rhs_lap), rtol=1e-8, atol=1e-8)


def test_scale_translation_invariance():
    """P3: weights of a translated and scaled stencil scale like the operator."""
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (28, 2))
    c = np.zeros(2)
    w1, _ = O.stencil_weights(c, X, 7, 3, (O.OP_DX, O.OP_LAP))
    s, t = 3.7e-3, np.array([12.5, -4.0])
    w2, _ = O.stencil_weights(c * s + t, X * s + t, 7, 3, (O.OP_DX, O.OP_LAP))
    assert np.abs(w2[O.OP_DX] * s - w1[O.OP_DX]).max() < 1e-10 * np.abs(w1[O.OP_DX]).max()
    assert np.abs(w2[O.OP_LAP] * s * s - w1[O.OP_LAP]).max() < 1e-10 * np.abs(w1[O.OP_LAP]).max()


def test_truncation_error_converges_for_wave_function():
    """P4: error of D_x and D_Lap on f = sin(8 pi x + 4 pi y) cos(6 pi y)
    falls under refinement at a high order (q sets the order)."""
    errs = {"dx": [], "lap": []}
    hs = []
    for n in (33, 65, 129):
        nd = ns.jittered_cavity(n, 1)
        x, y = nd.px, nd.py
        inner = (x > 0.2) & (x < 0.8) & (y > 0.2) & (y < 0.8)
        ax, ay = x[inner], y[inner]
        idx, W = O.build_weights(ax, ay, x, y, 28, 7, 3, (O.OP_DX, O.OP_LAP))
        f, fx, fy, lap = ns.wave_test_function(x, y)
        _, efx, _, elap = ns.wave_test_function(ax, ay)
        # mean error over max |L f|, the form of Eq. relative_error
        errs["dx"].append(np.abs((W[O.OP_DX] * f[idx]).sum(1) - efx).mean() / np.abs(efx).max())
        errs["lap"].append(np.abs((W[O.OP_LAP] * f[idx]).sum(1) - elap).mean() / np.abs(elap).max())
    # q = 3: first derivatives O(h^3), second derivatives O(h^2)
    for key, lo in (("dx", 2.6), ("lap", 1.8)):
        e = np.array(errs[key])
        rate = np.log(e[0] / e[-1]) / np.log(4.0)
        assert np.all(e[1:] < e[:-1]) and rate > lo, (key, e, rate)


def test_modified_wavenumber_within_paper_bound():
    """P5 with the paper's printed bound: at k~ Delta r = sqrt(2) the radial
    modified wavenumber of the 28-point (7, 3) operators deviates from k~ by
    at most 1.5 % over wave angles (Section 6), on the collocated grids.
    Delta r: mean distance to the 6 nearest same-grid nodes (reading R10).
    The paper's bound is read over its grid-wide diagram, so the node mean is
    held to it; single stencils of these jittered lattices (rougher than the
    paper's mesh) spread wider, and the 90th percentile over nodes is held
    to twice the bound so that no stencil family can hide in the mean."""
    bound = _golden("mw_deviation_bounds.txt")["all_angles_bound"]
    nd = ns.jittered_cavity(40, 0)
    h = nd.h
    for ax, ay in ((nd.vx, nd.vy), (nd.px, nd.py)):
        idx, W = O.build_weights(ax, ay, ax, ay, 28, 7, 3, (O.OP_DX, O.OP_DY, O.OP_LAP))
        dr = O.local_spacing(ax, ay).mean()
        inner = (ax > 5 * h) & (ax < 1 - 5 * h) & (ay > 5 * h) & (ay < 1 - 5 * h)
        for th in np.linspace(0, np.pi / 2, 5):
            kt = np.sqrt(2.0) / dr
            kx, ky = kt * np.cos(th), kt * np.sin(th)
            ks = O.modified_wavenumber(W[O.OP_DX], W[O.OP_DY], idx, ax, ay, ax, ay, kx, ky)
            d1 = np.abs(ks[inner].real / kt - 1)
            assert d1.mean() < bound and np.percentile(d1, 90) < 2 * bound
            ph = np.exp(1j * (kx * ax + ky * ay))
            k2 = -(W[O.OP_LAP] * ph[idx]).sum(1) * np.conj(ph)
            d2 = np.abs(k2[inner].real / kt ** 2 - 1)
            assert d2.mean() < bound and np.percentile(d2, 90) < 2 * bound
        # and the spectral limit: k*/k~ -> 1 as k~ Delta r -> 0
        kt = 0.05 / dr
        ks = O.modified_wavenumber(W[O.OP_DX], W[O.OP_DY], idx, ax, ay, ax, ay, kt, 0.0)
        assert np.abs(ks[inner] / kt - 1).max() < 1e-5


# ------------------------------------------- parameter study (Section 4)
@pytest.fixture(scope="module")
def sweep_nodes():
    nd = ns.jittered_cavity(40, 0)
    x, y = nd.vx, nd.vy
    inner = (x > 0.2) & (x < 0.8) & (y > 0.2) & (y < 0.8)
    return x, y, inner, O.local_spacing(x, y)


def _mean_error(sweep_nodes, n, m, q, op):
    x, y, inner, dr = sweep_nodes
    idx, W = O.build_weights(x[inner], y[inner], x, y, n, m, q, (op,))
    return O.stencil_error(W[op], idx, x[inner], y[inner], x, y, op, dr[inner]).mean()


def test_test_function_derivatives_against_finite_differences():
    """The closed forms of L g (Eq. test) against central differences of g."""
    rng = np.random.default_rng(2)
    x, y = rng.random(50), rng.random(50)
    dr, eps = 0.07, 1e-5
    g = lambda a, b: np.cos(a / dr) * np.cos(b / dr)  # noqa: E731
    fd = {O.OP_DX: (g(x + eps, y) - g(x - eps, y)) / (2 * eps),
          O.OP_DY: (g(x, y + eps) - g(x, y - eps)) / (2 * eps),
          O.OP_LAP: (g(x + eps, y) + g(x - eps, y) + g(x, y + eps) + g(x, y - eps)
                     - 4 * g(x, y)) / eps ** 2,
          O.OP_INTERP: g(x, y)}
    for op, ref in fd.items():
        val, scale = O.test_function_derivative(x, y, dr, op)
        assert np.abs(val - ref).max() < 1e-4 * scale, op
        assert np.abs(val).max() <= scale * (1 + 1e-12)


def test_parameter_study_trends(sweep_nodes):
    """Section 4.1-4.2 on a jittered lattice: the relative error E of D_x
    falls as the PHS exponent grows from 3 to 7 and as the stencil grows, and
    for n = 28, m = 7 it falls from q = 1 to q = 3 while q = 4 brings no gain
    (the paper's reasons for (n, m, q) = (28, 7, 3))."""
    e = {t: _mean_error(sweep_nodes, *t, O.OP_DX)
         for t in ((28, 3, 3), (28, 5, 3), (28, 7, 3), (28, 7, 1), (28, 7, 4), (21, 7, 3),
                   (35, 7, 3))}
    assert e[(28, 3, 3)] > e[(28, 5, 3)] > e[(28, 7, 3)], e
    assert e[(21, 7, 3)] > e[(28, 7, 3)] > e[(35, 7, 3)], e
    assert e[(28, 7, 1)] > 1.2 * e[(28, 7, 3)] and e[(28, 7, 4)] >= e[(28, 7, 3)], e


def test_condition_number_definition_and_invariance(sweep_nodes):
    """The oracle's 1-norm condition number equals the definition written
    out with a plain Gauss-Jordan inverse on a small stencil, is unchanged by
    shifting and scaling the nodes (R1), and grows with the PHS exponent m
    (Section 4.2: m = 11 is numerically unstable)."""
    x, y, inner, _ = sweep_nodes
    idx = O.knn(x[:3], y[:3], x, y, 6)
    c = O.stencil_condition(x[:3], y[:3], x, y, idx, 3, 1)
    for i in range(3):
        X = np.stack([x[idx[i]] - x[i], y[idx[i]] - y[i]], -1)
        X = X / np.sqrt((X ** 2).sum(1).max())
        A = O.augmented_matrix(X, 3, 1).tolist()
        S = len(A)
        aug = [row[:] + [1.0 if r == c2 else 0.0 for c2 in range(S)] for r, row in enumerate(A)]
        for col in range(S):
            piv = max(range(col, S), key=lambda r: abs(aug[r][col]))
            aug[col], aug[piv] = aug[piv], aug[col]
            pv = aug[col][col]
            aug[col] = [v / pv for v in aug[col]]
            for r in range(S):
                if r != col:
                    f = aug[r][col]
                    aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
        inv_norm = max(sum(abs(aug[r][S + c2]) for r in range(S)) for c2 in range(S))
        a_norm = max(sum(abs(A[r][c2]) for r in range(S)) for c2 in range(S))
        assert abs(c[i] / (a_norm * inv_norm) - 1) < 1e-9
    sel = np.nonzero(inner)[0][:200]
    idx = O.knn(x[sel], y[sel], x, y, 28)
    c1 = O.stencil_condition(x[sel], y[sel], x, y, idx, 7, 3)
    c2 = O.stencil_condition(x[sel] * 1e-3 + 5, y[sel] * 1e-3 - 2, x * 1e-3 + 5, y * 1e-3 - 2,
                             idx, 7, 3)
    assert np.abs(c1 / c2 - 1).max() < 1e-8
    med = [np.median(O.stencil_condition(x[sel], y[sel], x, y, idx, m, 3)) for m in (3, 5, 7, 9)]
    assert med[0] < med[1] < med[2] < med[3], med


# ---------------------------------------------------------------- the step
def _tg(x, y, t, Re):
    e = np.exp(-2 * t / Re)
    return (-np.cos(x) * np.sin(y) * e, np.sin(x) * np.cos(y) * e,
            -0.25 * (np.cos(2 * x) + np.cos(2 * y)) * e * e)


def _tg_run(n, dt, T, Re=10.0, km_mode=2, ops=None, nd=None):
    nd = ns.jittered_cavity(n, 0, length=np.pi) if nd is None else nd
    fs = O.FractionalStep(nd, Re=Re, dt=dt, km_mode=km_mode, ops=ops)
    u0, v0, _ = _tg(nd.vx, nd.vy, 0.0, Re)
    st = fs.initial_state(u0, v0)
    steps = int(round(T / dt))
    for j in range(steps):
        gu, gv, _ = _tg(nd.vx, nd.vy, (j + 1) * dt, Re)
        st = fs.step(st, gu, gv)
    return nd, st, steps * dt


def test_taylor_green_spatial_convergence():
    """P6: the decaying Taylor-Green vortex on [0, pi]^2 with its exact wall
    data.  Velocity and mean-free pressure errors fall at high order."""
    Re = 10.0
    eu, ep = [], []
    for n in (9, 17, 33):
        nd, st, T = _tg_run(n, 0.005, 0.25, Re)
        ue, ve, _ = _tg(nd.vx, nd.vy, T, Re)
        _, _, pe = _tg(nd.px, nd.py, T, Re)
        eu.append(max(np.abs(st.u - ue).max(), np.abs(st.v - ve).max()))
        ep.append(np.abs((st.p - st.p.mean()) - (pe - pe.mean())).max())
    eu, ep = np.array(eu), np.array(ep)
    assert eu[-1] < 1e-4
    assert np.all(np.log2(eu[:-1] / eu[1:]) > 2.5), eu
    assert ep[-1] < 1e-3 and np.all(ep[1:] < ep[:-1]), ep


TIME_DTS = (0.01, 0.005, 0.0025, 0.00125)
_time_cache = {}


def tg_time_errors(n, km_mode=2):
    """Velocity errors at T = 0.2 (Re 10) for the steps TIME_DTS against a
    run with dt = 1.5625e-4 on the same nodes (the time-discretisation error
    alone).  Cached per (n, km_mode, oracle step function)."""
    key = (n, km_mode, O.FractionalStep.step, O.FractionalStep.intermediate)
    if key not in _time_cache:
        nd = ns.jittered_cavity(n, 0, length=np.pi)
        ops = O.build_operators(nd)
        ref = _tg_run(n, 0.00015625, 0.2, km_mode=km_mode, ops=ops, nd=nd)[1]
        errs = []
        for dt in TIME_DTS:
            st = _tg_run(n, dt, 0.2, km_mode=km_mode, ops=ops, nd=nd)[1]
            errs.append(max(np.abs(st.u - ref.u).max(), np.abs(st.v - ref.v).max()))
        _time_cache[key] = np.array(errs)
    return _time_cache[key]


def first_order_coefficient(errs):
    """A of err = A dt + B dt^2 through the two smallest steps."""
    d1, d2 = TIME_DTS[-2], TIME_DTS[-1]
    e1, e2 = errs[-2], errs[-1]
    B = (e1 - 2 * e2) / (d1 * d1 - 2 * d2 * d2)
    return (e1 - B * d1 * d1) / d1


def test_taylor_green_time_order():
    """App. D: the three-stage step is second order in time.  On a 33 x 33
    node set the observed order over dt = 1e-2 ... 1.25e-3 is at least 1.8 on
    every halving (1.87, 1.88, 1.87 when pinned).  Dropping the Kim & Moin
    wall term makes it first order."""
    e = tg_time_errors(33)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 1.8), (e, order)
    assert e[0] < 5e-5, e


def test_first_order_time_term_is_a_projection_defect():
    """Reading of App. D: the printed scheme projects with D^(P,P)_Lap, which
    differs from D^(P,V) D^(V,P) by the truncation error, so each projection
    leaves a divergence of order dt times that difference and the scheme
    carries an O(dt) term.  Its coefficient A (err = A dt + B dt^2) falls at
    a high power of h (3.3e-4, 7.9e-5, 4.1e-5 on 25^2, 33^2, 41^2 when
    pinned), so the order on the smallest steps rises toward 2 under
    refinement (1.54, 1.87, 1.93)."""
    errs = {n: tg_time_errors(n) for n in (25, 33, 41)}
    A = [first_order_coefficient(errs[n]) for n in (25, 33, 41)]
    assert A[1] < A[0] / 3 and A[2] < A[1] / 1.5, A
    last = [np.log2(errs[n][-2] / errs[n][-1]) for n in (25, 33, 41)]
    assert last[0] < last[1] < last[2], last


def test_kim_moin_modes_agree_and_dropping_the_term_is_first_order():
    """R5: the wall value of u** with both components of dt D^(V,P) p~_j (the
    printed formula, km_mode 2) and with the tangential component only
    (km_mode 1) agree to the spatial truncation level, because the normal
    component vanishes with the Neumann pressure condition; without the term
    (km_mode 0) the wall carries an O(dt) slip and the time error is first
    order and far larger."""
    e2, e1 = tg_time_errors(33, 2), tg_time_errors(33, 1)
    assert np.all(np.abs(e1 - e2) < 0.1 * e2), (e1, e2)
    e0 = tg_time_errors(33, 0)
    assert np.all(e0 > 20 * e2), (e0, e2)
    assert np.all(np.log2(e0[:-1] / e0[1:]) < 1.2), e0


def test_projection_reduces_divergence():
    """P7 / R13: on the smooth Taylor-Green flow the correction removes most of
    the divergence of the intermediate field, increasingly so under refinement
    (the projection is not exact because D^(P,P)_Lap differs from
    D^(P,V) D^(V,P))."""
    Re, dt = 10.0, 0.005
    ratios = []
    for n in (17, 33):
        nd = ns.jittered_cavity(n, 0, length=np.pi)
        fs = O.FractionalStep(nd, Re=Re, dt=dt)
        u0, v0, _ = _tg(nd.vx, nd.vy, 0.0, Re)
        st = fs.initial_state(u0, v0)
        for j in range(5):
            gu, gv, _ = _tg(nd.vx, nd.vy, (j + 1) * dt, Re)
            st = fs.step(st, gu, gv)
        gu, gv, _ = _tg(nd.vx, nd.vy, 6 * dt, Re)
        _, _, uss, vss, F = fs.intermediate(st, gu, gv)
        st2 = fs.step(st, gu, gv)
        inner = ~nd.p_boundary
        div = fs.ops.pv_x @ st2.u + fs.ops.pv_y @ st2.v
        ratios.append(np.linalg.norm(div[inner]) / np.linalg.norm(F[inner]))
    assert ratios[0] < 0.2 and ratios[1] < 0.5 * ratios[0], ratios


# ------------------------------------------- exactly projecting variant (f1)
def _two_mode(x, y, t, Re, eps=0.5):
    """Taylor-Green modes of wavenumber 1 and 2, each decaying at its own
    viscous rate.  Their sum is not a Navier-Stokes solution (the modes
    interact through the convective term, which is not a gradient here); it
    serves as a smooth initial field and smooth wall data for the time
    refinement, against a fine-step run on the same nodes."""
    e1, e2 = np.exp(-2 * t / Re), np.exp(-8 * t / Re)
    return (-np.cos(x) * np.sin(y) * e1 - eps * np.cos(2 * x) * np.sin(2 * y) * e2,
            np.sin(x) * np.cos(y) * e1 + eps * np.sin(2 * x) * np.cos(2 * y) * e2)


def two_mode_time_errors(n=17, **kw):
    nd = ns.jittered_cavity(n, 0, length=np.pi)
    ops = O.build_operators(nd)

    def run(dt, T=0.2, Re=10.0):
        fs = O.FractionalStep(nd, Re=Re, dt=dt, ops=ops, **kw)
        st = fs.initial_state(*_two_mode(nd.vx, nd.vy, 0.0, Re))
        for j in range(int(round(T / dt))):
            st = fs.step(st, *_two_mode(nd.vx, nd.vy, (j + 1) * dt, Re))
        return st
    ref = run(0.00015625)
    errs = []
    for dt in TIME_DTS:
        st = run(dt)
        errs.append(max(np.abs(st.u - ref.u).max(), np.abs(st.v - ref.v).max()))
    return np.array(errs)


def test_exact_projection_is_divergence_free(cavity20, ops20):
    """f1: with the composed operator D^(P,V) G0 the corrected velocity is
    discretely divergence-free at every P-node (to solver rounding), on the
    lid-driven cavity over 100 steps.  The uniform wall-normal velocity that
    takes up the one component no gradient can remove stays below 1 % of the
    lid speed (it settles near 0.3 %: the lid corners, where the wall data
    jump, dominate it; on Taylor-Green it is 4e-7 at 33^2)."""
    nd = cavity20
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3, ops=ops20, projection="exact")
    gu, gv = O.lid_bc(nd)
    st = fs.initial_state()
    for _ in range(100):
        st = fs.step(st, gu, gv)
        div = ops20.pv_x @ st.u + ops20.pv_y @ st.v
        assert np.abs(div).max() < 1e-11, np.abs(div).max()
        assert abs(st.lam) < 1e-2, st.lam
    inner = ~nd.v_boundary
    assert np.abs(st.u).max() <= 1.0 + 1e-9 and np.isfinite(st.u[inner]).all()


def test_exact_projection_taylor_green_space_and_time():
    """f1 on Taylor-Green: velocity error falls at high order in space
    (9^2, 17^2, 33^2) and the step is second order in time from 17^2 on
    (orders >= 1.9 per halving; the paper's projection is first order there,
    see test_first_order_time_term_is_a_projection_defect)."""
    eu = []
    for n in (9, 17, 33):
        nd = ns.jittered_cavity(n, 0, length=np.pi)
        fs = O.FractionalStep(nd, Re=10.0, dt=0.005, projection="exact")
        u0, v0, _ = _tg(nd.vx, nd.vy, 0.0, 10.0)
        st = fs.initial_state(u0, v0)
        for j in range(50):
            gu, gv, _ = _tg(nd.vx, nd.vy, (j + 1) * 0.005, 10.0)
            st = fs.step(st, gu, gv)
        ue, ve, _ = _tg(nd.vx, nd.vy, 0.25, 10.0)
        eu.append(max(np.abs(st.u - ue).max(), np.abs(st.v - ve).max()))
    eu = np.array(eu)
    assert eu[-1] < 1e-5 and np.all(np.log2(eu[:-1] / eu[1:]) > 2.5), eu
    nd = ns.jittered_cavity(17, 0, length=np.pi)
    ops = O.build_operators(nd)

    def run(dt):
        fs = O.FractionalStep(nd, Re=10.0, dt=dt, ops=ops, projection="exact")
        st = fs.initial_state(*_tg(nd.vx, nd.vy, 0.0, 10.0)[:2])
        for j in range(int(round(0.2 / dt))):
            st = fs.step(st, *_tg(nd.vx, nd.vy, (j + 1) * dt, 10.0)[:2])
        return st
    ref = run(0.00015625)
    e = np.array([np.abs(run(dt).u - ref.u).max() for dt in TIME_DTS])
    assert np.all(np.log2(e[:-1] / e[1:]) >= 1.9), e


def test_exact_projection_with_kim_moin_crank_nicolson_is_second_order():
    """R14: with the exact projection the remaining first-order term of the
    step is the printed Crank-Nicolson form (Eq. u_ss applies I + a D_Lap to
    u*, which holds the convective update).  On a flow whose convective term
    is not a gradient, Kim & Moin's form (right side u* + a D_Lap u_j) gives
    order >= 1.9 on every halving (2.02, 2.02, 2.03 when pinned), the printed
    form below 1.3 (1.09, 1.08, 1.12).  This also pins the Adams-Bashforth
    history, which Taylor-Green cannot."""
    e = two_mode_time_errors(17, projection="exact", cn_form="kim_moin")
    assert np.all(np.log2(e[:-1] / e[1:]) >= 1.9), e
    e = two_mode_time_errors(17, projection="exact", cn_form="printed")
    assert np.all(np.log2(e[:-1] / e[1:]) < 1.3), e


def test_bordered_poisson_compatible_rhs_has_zero_multiplier(ops20, cavity20):
    """R4: for a right side in the range of L the multiplier vanishes and the
    solution is the generating field minus its mean."""
    nd = cavity20
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3, ops=ops20)
    p = np.cos(3 * nd.px) * np.sin(2 * nd.py) + nd.px ** 2
    A = fs.Pb.tocsr()
    M = nd.M
    b = A[:M, :M] @ p
    sol = fs.P_lu.solve(np.concatenate([b, [0.0]]))
    assert abs(sol[-1]) < 1e-8
    assert np.abs(sol[:-1] - (p - p.mean())).max() < 1e-8


def test_helmholtz_boundary_rows_are_identity(ops20, cavity20):
    nd = cavity20
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3, ops=ops20)
    H = fs.H.tocsr()
    b = np.nonzero(nd.v_boundary)[0]
    for i in b[:20]:
        row = H.getrow(i).toarray().ravel()
        e = np.zeros(nd.N)
        e[i] = 1.0
        assert np.array_equal(row, e)


def test_viscous_krylov_solve_matches_lu(cavity20, ops20):
    """P8: the oracle's iterative viscous solve (for large node sets) and the
    LU factorisation of the paper give the same steps (Re 1e4, dt 2e-4)."""
    nd = cavity20
    gu, gv = O.lid_bc(nd)
    outs = []
    for solver in ("lu", "krylov"):
        fs = O.FractionalStep(nd, Re=1e4, dt=2e-4, ops=ops20, viscous_solver=solver)
        st = fs.initial_state()
        for _ in range(10):
            st = fs.step(st, gu, gv)
        outs.append(st)
    assert np.abs(outs[0].u - outs[1].u).max() < 1e-12
    assert np.abs(outs[0].pt - outs[1].pt).max() < 1e-10 * np.abs(outs[0].pt).max()


def test_cavity_runs_stably_and_keeps_wall_data(cavity20, ops20):
    """Config-0-like cavity (Re 100, dt 2e-3) stays bounded; wall nodes hold
    the lid and no-slip data exactly (reading R6)."""
    nd = cavity20
    fs = O.FractionalStep(nd, Re=100.0, dt=2e-3, ops=ops20)
    st = fs.initial_state()
    gu, gv = O.lid_bc(nd)
    for _ in range(150):
        st = fs.step(st, gu, gv)
    assert np.isfinite(st.u).all() and np.abs(st.u).max() <= 1.0 + 1e-9
    vb = nd.v_boundary
    assert np.array_equal(st.u[vb], gu[vb]) and np.array_equal(st.v[vb], gv[vb])
    assert abs(st.pt.mean()) < 1e-12


# ---------------------------------------------------------------- adjoint
def _adj_setup(km_mode=2, seed=0):
    nd = ns.jittered_cavity(12, 4)
    fs = O.FractionalStep(nd, Re=400.0, dt=2e-3, km_mode=km_mode)
    rng = np.random.default_rng(seed)
    lid = nd.v_wall == ns.WALL_TOP
    g0 = np.zeros(nd.N)
    g0[lid] = 1 + 0.05 * rng.standard_normal(lid.sum())
    u0 = np.zeros(nd.N)
    inner = ~nd.v_boundary
    u0[inner] = 0.01 * rng.standard_normal(inner.sum())
    return nd, fs, g0, u0


def _adj_run(fs, nd, gu, u0, steps):
    st = fs.initial_state(u0, np.zeros(nd.N))
    sts = [st]
    for _ in range(steps):
        st = fs.step(st, gu, np.zeros(nd.N))
        sts.append(st)
    return sts


@pytest.mark.parametrize("km_mode", [2, 1])
def test_adjoint_matches_central_differences(km_mode):
    """P9: gradients of J = 1/2 sum(u^2 + v^2) after 8 steps with respect to
    per-node lid velocity and to the initial velocity, from the discrete
    adjoint, against central differences of the forward solver (eps 1e-6)."""
    nd, fs, g0, u0 = _adj_setup(km_mode)
    steps = 8
    sts = _adj_run(fs, nd, g0, u0, steps)
    lam = O.AdjointState(sts[-1].u.copy(), sts[-1].v.copy(), np.zeros(nd.N), np.zeros(nd.N),
                         np.zeros(nd.M))
    G = np.zeros(nd.N)
    for j in range(steps - 1, -1, -1):
        lam, lgu, _ = O.adjoint_step(fs, sts[j], lam)
        G += lgu
    eps = 1e-6
    lid = np.nonzero(nd.v_wall == ns.WALL_TOP)[0][:3]
    inner = np.nonzero(~nd.v_boundary)[0][[0, 7, 40]]
    for k in lid:
        gp, gm = g0.copy(), g0.copy()
        gp[k] += eps
        gm[k] -= eps
        fd = (O.kinetic_energy(_adj_run(fs, nd, gp, u0, steps)[-1])
              - O.kinetic_energy(_adj_run(fs, nd, gm, u0, steps)[-1])) / (2 * eps)
        assert abs(G[k] - fd) <= 1e-6 * abs(fd), (k, G[k], fd)
    for k in inner:
        up, um = u0.copy(), u0.copy()
        up[k] += eps
        um[k] -= eps
        fd = (O.kinetic_energy(_adj_run(fs, nd, g0, up, steps)[-1])
              - O.kinetic_energy(_adj_run(fs, nd, g0, um, steps)[-1])) / (2 * eps)
        assert abs(lam.u[k] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, lam.u[k], fd)


def test_adjoint_dot_product_identity():
    """<J_step dx, y> = <dx, J_step^T y> for the linearised step: perturb the
    input state along a random direction, compare the change of a random
    linear functional of the output with the adjoint's prediction."""
    nd, fs, g0, u0 = _adj_setup(seed=3)
    sts = _adj_run(fs, nd, g0, u0, 3)
    st = sts[2]
    rng = np.random.default_rng(9)
    du = rng.standard_normal(nd.N) * (~nd.v_boundary)
    dpt = rng.standard_normal(nd.M)
    yu, yv = rng.standard_normal(nd.N), rng.standard_normal(nd.N)
    ypt = rng.standard_normal(nd.M)

    def functional(s):
        out = fs.step(s, g0, np.zeros(nd.N))
        return yu @ out.u + yv @ out.v + ypt @ out.pt

    eps = 1e-6
    sp_ = O.FlowState(st.u + eps * du, st.v, st.cu_prev, st.cv_prev, st.pt + eps * dpt, st.p,
                      0.0, st.j)
    sm_ = O.FlowState(st.u - eps * du, st.v, st.cu_prev, st.cv_prev, st.pt - eps * dpt, st.p,
                      0.0, st.j)
    fd = (functional(sp_) - functional(sm_)) / (2 * eps)
    lam, _, _ = O.adjoint_step(fs, st, O.AdjointState(yu, yv, np.zeros(nd.N), np.zeros(nd.N), ypt))
    pred = lam.u @ du + lam.pt @ dpt
    assert abs(pred - fd) <= 1e-6 * abs(fd), (pred, fd)
