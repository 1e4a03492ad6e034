"""Pins of the oracle's open-flow step (R17) and of the cylinder-wake
quantities of Section 5.2, each against something other than the oracle's own
formulas: closed-form forces of polynomial fields (the stencils reproduce
polynomials to degree q = 3, Simpson's rule integrates their low trigonometric
degree exactly), exact Navier-Stokes solutions that satisfy every boundary
condition of the wake domain, a lift signal of known frequency, and
polynomial reproduction of the boundary rows."""
import numpy as np
import pytest

from oracle import rbffd_oracle as O
from paper_2206_06495_gb300 import nodesets as ns

R_CYL = 0.5
SMALL = dict(h_wall=0.06, h_wake=0.08, h_far=0.5, x0=-3.0, x1=6.0, y0=-3.0, y1=3.0)


@pytest.fixture(scope="module")
def wake():
    nd = ns.cylinder_wake(**SMALL)
    return nd, O.build_operators(nd)


def channel(h):
    return ns.cylinder_wake(radius=0.0, h_wall=h, h_wake=h, h_far=h, x0=0.0, x1=8.0, y0=-4.0,
                            y1=4.0)


def test_paper_sized_layout():
    """The default layout has about the paper's node counts (M = 18,647 and
    N = 55,671, Section 5.2), N/M close to 3, every boundary segment as an
    edge (the generator checks), an even number of cylinder nodes equally
    spaced in angle, and unit outward normals on every boundary node."""
    nd = ns.cylinder_wake()
    assert abs(nd.M - 18647) < 0.06 * 18647 and abs(nd.N - 55671) < 0.06 * 55671
    assert 2.9 < nd.N / nd.M < 3.05
    cyl = nd.p_wall == ns.WALL_CYLINDER
    th = np.sort(np.mod(np.arctan2(nd.py[cyl], nd.px[cyl]), 2 * np.pi))
    assert cyl.sum() % 2 == 0
    assert np.allclose(np.diff(th), 2 * np.pi / cyl.sum(), rtol=1e-9)
    assert np.allclose(np.hypot(nd.px[cyl], nd.py[cyl]), R_CYL, rtol=1e-12)
    for nx, ny, b in ((nd.p_nx, nd.p_ny, nd.p_boundary), (nd.v_nx, nd.v_ny, nd.v_boundary)):
        assert np.allclose(np.hypot(nx[b], ny[b]), 1.0)
    # cylinder normals point out of the fluid, into the body
    assert np.all(nd.p_nx[cyl] * nd.px[cyl] + nd.p_ny[cyl] * nd.py[cyl] < 0)


@pytest.mark.parametrize("field", ["p=x", "p=y", "u=y^2", "v=x^2"])
def test_forces_of_polynomial_fields(wake, field):
    """Closed forms of F = integral of (-p I + (grad U + grad U^T)/Re) n over
    the circle r = R, n = (cos t, sin t), C = F / (1/2 D):
    p = x: F = (-pi R^2, 0); p = y: (0, -pi R^2);
    u = y^2 (v = p = 0): traction_x = 2 y n_y / Re, F = (2 pi R^2 / Re, 0);
    v = x^2: traction_y = 2 x n_x / Re, F = (0, 2 pi R^2 / Re)."""
    nd, ops = wake
    Re = 100.0
    z, zp = np.zeros(nd.N), np.zeros(nd.M)
    u, v, p, want = {
        "p=x": (z, z, nd.px.copy(), (-np.pi * R_CYL, 0.0)),
        "p=y": (z, z, nd.py.copy(), (0.0, -np.pi * R_CYL)),
        "u=y^2": (nd.vy ** 2, z, zp, (2 * np.pi * R_CYL / Re, 0.0)),
        "v=x^2": (z, nd.vx ** 2, zp, (0.0, 2 * np.pi * R_CYL / Re)),
    }[field]
    cd, cl = O.cylinder_forces(nd, ops, u, v, p, Re)
    scale = max(abs(want[0]), abs(want[1]))
    assert abs(cd - want[0]) < 1e-11 * scale and abs(cl - want[1]) < 1e-11 * scale


def test_simpson_rule_is_exact_for_low_trigonometric_degree():
    """Composite Simpson's rule on a periodic grid of n points integrates
    cos(m t) exactly (2 pi for m = 0, else 0) for m < n/2, and a smooth
    periodic function to near machine precision."""
    n = 40
    t = 2 * np.pi * np.arange(n) / n
    for m in range(n // 2):
        want = 2 * np.pi if m == 0 else 0.0
        assert abs(O.simpson_periodic(np.cos(m * t), 2 * np.pi) - want) < 1e-12
    # exp(cos t) integrates to 2 pi I_0(1)
    from scipy.special import i0
    assert abs(O.simpson_periodic(np.exp(np.cos(t)), 2 * np.pi) - 2 * np.pi * i0(1.0)) < 1e-12


def test_strouhal_of_a_known_frequency():
    t = np.arange(0.0, 60.0, 0.005)
    cl = 0.34 * np.sin(2 * np.pi * 0.171 * t + 0.3) + 0.02
    assert abs(O.strouhal(t, cl) - 0.171) < 1e-6
    assert abs(O.strouhal(t, cl, diameter=2.0) - 0.342) < 2e-6


def test_neumann_velocity_rows_reproduce_cubics(wake):
    """The one-sided Neumann V-rows give n.grad f exactly for polynomials up
    to degree q = 3."""
    nd, _ = wake
    bu, bv, _, _, _ = O.wake_conditions(nd)
    rows = np.nonzero((bu == O.BC_NEUMANN) | (bv == O.BC_NEUMANN))[0]
    VN = O.neumann_rows(nd, rows)
    x, y = nd.vx, nd.vy
    for f, fx, fy in ((x ** 3 - 2 * x * y, 3 * x ** 2 - 2 * y, -2 * x),
                      (y ** 3 + x * y ** 2, y ** 2, 3 * y ** 2 + 2 * x * y)):
        got = (VN @ f)[rows]
        want = nd.v_nx[rows] * fx[rows] + nd.v_ny[rows] * fy[rows]
        assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()


def test_open_pressure_rows(wake):
    """Rows of the open-flow pressure matrix on a cubic f: Laplacian inside,
    n.grad f on the Neumann rows, f itself on the Dirichlet (outlet) rows;
    the outlet's corners are Neumann rows."""
    nd, ops = wake
    bu, bv, bp, gu, gv = O.wake_conditions(nd)
    fs = O.OpenFlowStep(nd, 100.0, 0.005, bu, bv, bp, ops=ops)
    x, y = nd.px, nd.py
    f = x ** 3 + x * y ** 2 - 2 * y
    fx, fy, lap = 3 * x ** 2 + y ** 2, 2 * x * y - 2, 6 * x + 2 * x
    Lf = fs.L @ f
    inn, neu, dirichlet = bp == O.BC_INTERIOR, bp == O.BC_NEUMANN, bp == O.BC_DIRICHLET
    sc = np.abs(lap).max()
    assert np.abs(Lf[inn] - lap[inn]).max() < 1e-7 * sc
    assert np.abs(Lf[neu] - (nd.p_nx * fx + nd.p_ny * fy)[neu]).max() < 1e-8 * np.abs(fx).max()
    assert np.array_equal(Lf[dirichlet], f[dirichlet])
    corners = (nd.p_wall == ns.WALL_OUTFLOW) & ((y == -3.0) | (y == 3.0))
    assert corners.sum() == 2 and np.all(bp[corners] == O.BC_NEUMANN)
    assert dirichlet.sum() == (nd.p_wall == ns.WALL_OUTFLOW).sum() - 2


def test_uniform_channel_flow_is_steady():
    """u = 1, v = 0, p = 0 solves Navier-Stokes in the channel with every
    boundary condition of the wake domain; the step keeps it to rounding over
    200 steps (with Dirichlet pressure rows at the outlet's corners too, a
    corner mode grew by 1.66 per step, R17)."""
    nd = channel(0.1)
    bu, bv, bp, gu, gv = O.wake_conditions(nd)
    fs = O.OpenFlowStep(nd, 100.0, 0.01, bu, bv, bp)
    st = fs.initial_state(np.ones(nd.N), np.zeros(nd.N))
    for _ in range(200):
        st = fs.step(st, gu, gv)
    assert np.abs(st.u - 1.0).max() < 1e-10 and np.abs(st.v).max() < 1e-10
    assert np.abs(st.pt).max() < 1e-9


def test_decaying_shear_mode_converges():
    """u = 1 + eps exp(-k^2 t / Re) cos(k y), v = 0, p = const with
    k = pi / 4 is an exact solution (u.grad u = 0) that meets the symmetry
    sides (v = 0, du/dy = 0 at y = +-4), the stress-free outlet (du/dx =
    dv/dx = 0, p = 0) and takes its inflow data from the solution.  At
    Re = 10 and t = 2 the error is at truncation level and falls when h and
    dt are halved (8.7e-6 and 1.2e-6 when pinned)."""
    Re, eps, k = 10.0, 0.1, np.pi / 4

    def exact(y, t):
        return 1.0 + eps * np.exp(-k * k * t / Re) * np.cos(k * y)

    errs = []
    for h, dt in ((0.2, 0.01), (0.1, 0.005)):
        nd = channel(h)
        bu, bv, bp, _, gv = O.wake_conditions(nd)
        fs = O.OpenFlowStep(nd, Re, dt, bu, bv, bp)
        st = fs.initial_state(exact(nd.vy, 0.0), np.zeros(nd.N))
        n = int(round(2.0 / dt))
        inflow = nd.v_wall == ns.WALL_INFLOW
        for j in range(n):
            st = fs.step(st, np.where(inflow, exact(nd.vy, (j + 1) * dt), 0.0), gv)
        errs.append(max(np.abs(st.u - exact(nd.vy, 2.0)).max(), np.abs(st.v).max()))
    assert errs[0] < 2e-5 and errs[1] < errs[0] / 4, errs


def test_cylinder_start_is_bounded_and_drag_is_physical(wake):
    """Impulsive start past the cylinder at Re = 100 (dt = 0.005, 200 steps):
    the speed stays below twice the free stream and the drag coefficient of
    the early transient lies between the steady value near 1.4 and the
    impulsive-start peak (1.5 < C_D < 2.5), the lift near zero."""
    nd, ops = wake
    bu, bv, bp, gu, gv = O.wake_conditions(nd)
    fs = O.OpenFlowStep(nd, 100.0, 0.005, bu, bv, bp, ops=ops)
    st = fs.initial_state(np.where(bu == O.BC_DIRICHLET, gu, 1.0), np.zeros(nd.N))
    for _ in range(200):
        st = fs.step(st, gu, gv)
    assert np.abs(np.hypot(st.u, st.v)).max() < 2.0
    cd, cl = O.cylinder_forces(nd, ops, st.u, st.v, st.p, 100.0)
    assert 1.5 < cd < 2.5 and abs(cl) < 0.05, (cd, cl)
