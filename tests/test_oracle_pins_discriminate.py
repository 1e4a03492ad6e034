"""The pins catch plausible mistakes: each test plants one in the oracle (on
the CPU, through monkeypatching) and checks that a pin then fails."""
import numpy as np
import pytest

from oracle import rbffd_oracle as O
from tests import test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_wrong_laplacian_of_phs_is_caught(monkeypatch):
    """m(m-1) r^(m-2) (the 1-D second derivative) instead of m^2 r^(m-2)."""
    orig = O._op_rhs_rbf

    def bad(op, X, m):
        if op == O.OP_LAP:
            r = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
            return m * (m - 1) * r ** (m - 2)
        return orig(op, X, m)

    monkeypatch.setattr(O, "_op_rhs_rbf", bad)
    assert _fails(pins.test_modified_wavenumber_within_paper_bound)


def test_wrong_sign_of_rbf_derivative_is_caught(monkeypatch):
    orig = O._op_rhs_rbf

    def bad(op, X, m):
        if op == O.OP_DX:
            return -orig(op, X, m)
        return orig(op, X, m)

    monkeypatch.setattr(O, "_op_rhs_rbf", bad)
    assert _fails(pins.test_modified_wavenumber_within_paper_bound)


def test_transposed_polynomial_block_is_caught(monkeypatch):
    """Swapping x and y in the monomials of the P block."""
    orig = O.augmented_matrix

    def bad(X, m, q):
        return orig(X[..., ::-1], m, q) * 0 + _mix(X, m, q, orig)

    def _mix(X, m, q, f):
        A = f(X, m, q)
        n = X.shape[-2]
        Xs = X[..., ::-1]
        B = f(Xs, m, q)
        A[..., :n, n:] = B[..., :n, n:]
        A[..., n:, :n] = B[..., n:, :n]
        return A

    monkeypatch.setattr(O, "augmented_matrix", bad)
    assert _fails(pins.test_polynomial_exactness_all_grids, pins.ns.jittered_cavity(20, 0), 3)


@pytest.mark.parametrize("mistake", ["convection_sign", "drop_ab2", "pressure_sign"])
def test_step_mistakes_are_caught_by_taylor_green(monkeypatch, mistake):
    if mistake == "convection_sign":
        orig = O.FractionalStep.convection
        monkeypatch.setattr(O.FractionalStep, "convection",
                            lambda self, u, v, q: -orig(self, u, v, q))
    elif mistake == "drop_ab2":
        orig = O.FractionalStep.convection
        monkeypatch.setattr(O.FractionalStep, "convection",
                            lambda self, u, v, q: 0.0 * orig(self, u, v, q))
    else:
        orig_init = O.FractionalStep.__init__

        def init(self, *a, **k):
            orig_init(self, *a, **k)
            self.ops.vp_x = -self.ops.vp_x
            self.ops.vp_y = -self.ops.vp_y
        monkeypatch.setattr(O.FractionalStep, "__init__", init)
    with np.errstate(all="ignore"):
        assert _fails(pins.test_taylor_green_spatial_convergence)


@pytest.fixture
def fresh_time_cache():
    pins._time_cache.clear()
    yield
    pins._time_cache.clear()


def test_dropped_kim_moin_term_is_caught(monkeypatch, fresh_time_cache):
    """Dropping the Kim & Moin wall term of u** (end of Section 3) leaves an
    O(dt) slip at the walls: the App. D time-order pin must fail."""
    orig_init = O.FractionalStep.__init__

    def init(self, *a, **k):
        orig_init(self, *a, **k)
        self.km_mode = 0
    monkeypatch.setattr(O.FractionalStep, "__init__", init)
    assert _fails(pins.test_taylor_green_time_order)


def test_euler_convection_is_caught_by_the_two_mode_pin(monkeypatch):
    """Forward Euler for the convective term (C_{j-1} = C_j at every step)
    instead of the Adams-Bashforth history makes the exactly projecting,
    Kim & Moin Crank-Nicolson step first order on the two-mode flow."""
    orig = O.FractionalStep.intermediate

    def euler(self, st, gu, gv):
        return orig(self, O.FlowState(st.u, st.v, st.cu_prev, st.cv_prev, st.pt, st.p,
                                      st.lam, 0), gu, gv)
    monkeypatch.setattr(O.FractionalStep, "intermediate", euler)
    assert _fails(pins.test_exact_projection_with_kim_moin_crank_nicolson_is_second_order)


def test_wrong_sign_of_pressure_increment_is_caught(monkeypatch):
    """The exact projection's predictor with +dt G0 p~_j instead of -dt G0 p~_j."""
    orig_init = O.FractionalStep.__init__

    def init(self, *a, **k):
        orig_init(self, *a, **k)
        if self.projection == "exact":
            self.G0x, self.G0y = -self.G0x, -self.G0y
    monkeypatch.setattr(O.FractionalStep, "__init__", init)
    with np.errstate(all="ignore"):
        assert _fails(pins.test_exact_projection_taylor_green_space_and_time)


def _planted(monkeypatch, fn_name, old, new):
    """Replace `old` by `new` in the source of oracle function `fn_name` and
    install the result in the oracle module (one planted mistake)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(O, fn_name)))
    assert src.count(old) == 1, (fn_name, old)
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), f"<planted {fn_name}>", "exec"), ns)
    monkeypatch.setattr(O, fn_name, ns[fn_name])


@pytest.mark.parametrize("old,new,field", [
    ("(uy + vx) * nx", "uy * nx", "v=x^2"),        # grad U^T dropped from the stress
    ("-pc * nx", "pc * nx", "p=x"),                 # pressure traction with the wrong sign
    ("return 2.0 * fx / d, 2.0 * fy / d", "return fx / d, fy / d", "u=y^2"),  # C = F / D
])
def test_force_mistakes_are_caught(monkeypatch, old, new, field):
    from paper_2206_06495_gb300 import nodesets as ns
    from tests import test_oracle_pins_wake as wp
    nd = ns.cylinder_wake(**wp.SMALL)
    wake = (nd, O.build_operators(nd))
    _planted(monkeypatch, "cylinder_forces", old, new)
    assert _fails(wp.test_forces_of_polynomial_fields, wake, field)


def test_tangential_derivative_in_neumann_rows_is_caught(monkeypatch):
    """Neumann V-rows built from D_x alone instead of n_x D_x + n_y D_y."""
    from paper_2206_06495_gb300 import nodesets as ns
    from tests import test_oracle_pins_wake as wp
    nd = ns.cylinder_wake(**wp.SMALL)
    _planted(monkeypatch, "neumann_rows", "nodes.v_nx[rows, None] * w[OP_DX] + "
             "nodes.v_ny[rows, None] * w[OP_DY]", "w[OP_DX]")
    assert _fails(wp.test_neumann_velocity_rows_reproduce_cubics, (nd, None))
