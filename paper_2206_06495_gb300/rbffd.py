"""Python binding of librbffd (include/rbffd.h): argument marshalling only.

Every entry point keeps the C name without the `rbffd_` prefix and forwards
torch CUDA tensors as raw device pointers on torch's current stream.  All
arithmetic happens in the CUDA library; there is no fallback: if the library
is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbffd.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_SINGULAR_STENCIL = -2
ERR_NOT_CONVERGED = -3
ERR_NONFINITE = -4
ERR_CUDA = -5
ERR_OOM = -6

OP_INTERP, OP_DX, OP_DY, OP_LAP = 1, 2, 4, 8
F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
PROJ_PAPER, PROJ_EXACT = 0, 1
BC_DIRICHLET, BC_NEUMANN = 1, 2  # rbffd_flow.v_bcu / v_bcv
PBC_DIRICHLET = 2                # rbffd_flow.p_bc: p~ = 0 row
CN_PRINTED, CN_KIM_MOIN = 0, 1

_ERRNAMES = {ERR_INVALID_ARG: "INVALID_ARG", ERR_SINGULAR_STENCIL: "SINGULAR_STENCIL",
             ERR_NOT_CONVERGED: "NOT_CONVERGED", ERR_NONFINITE: "NONFINITE",
             ERR_CUDA: "CUDA", ERR_OOM: "OOM"}


class RbffdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rbffd error {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("q", C.c_int32)]


class Ell(C.Structure):
    _fields_ = [("idx", C.c_void_p), ("w", C.c_void_p), ("n_rows", C.c_int64),
                ("n_cols", C.c_int64), ("ld", C.c_int64), ("n", C.c_int32),
                ("w_dtype", C.c_int32)]


class FlowC(C.Structure):
    _fields_ = [("N", C.c_int64), ("M", C.c_int64), ("ld_v", C.c_int64), ("ld_p", C.c_int64),
                ("vv_idx", C.c_void_p), ("vv_dx", C.c_void_p), ("vv_dy", C.c_void_p),
                ("vv_lap", C.c_void_p),
                ("pv_idx", C.c_void_p), ("pv_dx", C.c_void_p), ("pv_dy", C.c_void_p),
                ("pp_idx", C.c_void_p), ("pp_dx", C.c_void_p), ("pp_dy", C.c_void_p),
                ("pp_lap", C.c_void_p),
                ("vp_idx", C.c_void_p), ("vp_dx", C.c_void_p), ("vp_dy", C.c_void_p),
                ("v_bc", C.c_void_p), ("v_nx", C.c_void_p), ("v_ny", C.c_void_p),
                ("p_bc", C.c_void_p), ("p_nx", C.c_void_p), ("p_ny", C.c_void_p),
                ("nb_p", C.c_int64), ("ld_b", C.c_int64), ("pn_rows", C.c_void_p),
                ("pn_idx", C.c_void_p), ("pn_dx", C.c_void_p), ("pn_dy", C.c_void_p),
                ("Re", C.c_double), ("dt", C.c_double), ("precision", C.c_int32),
                ("precond", C.c_int32),
                ("tol", C.c_double), ("inner_tol", C.c_double), ("max_iter", C.c_int32),
                ("km_mode", C.c_int32), ("overwrite_bc", C.c_int32), ("profile", C.c_int32),
                ("p_edges", C.c_void_p), ("n_edges", C.c_int64), ("p_x", C.c_void_p),
                ("p_y", C.c_void_p), ("projection", C.c_int32), ("cn_form", C.c_int32),
                ("v_bcu", C.c_void_p), ("v_bcv", C.c_void_p), ("nb_v", C.c_int64),
                ("ld_vb", C.c_int64), ("vn_rows", C.c_void_p), ("vn_idx", C.c_void_p),
                ("vn_dx", C.c_void_p), ("vn_dy", C.c_void_p)]


class StateC(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("cu_prev", C.c_void_p),
                ("cv_prev", C.c_void_p), ("pt", C.c_void_p), ("p", C.c_void_p),
                ("j", C.c_int64)]


class AdjointC(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("cu_prev", C.c_void_p),
                ("cv_prev", C.c_void_p), ("pt", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("helm_iters", C.c_int64), ("poisson_iters", C.c_int64),
                ("refinements", C.c_int64), ("helm_relres", C.c_double),
                ("poisson_relres", C.c_double), ("launches", C.c_int64),
                ("spmv_launches", C.c_int64), ("spmv_ms", C.c_double),
                ("spmv_batch_launches", C.c_int64), ("spmv_batch_ms", C.c_double),
                ("wall_flux", C.c_double), ("vspmv_batch_launches", C.c_int64),
                ("vspmv_batch_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# exported symbols and their prototypes (kept in step with include/rbffd.h)
PROTOTYPES = {
    "rbffd_version": (C.c_int, []),
    "rbffd_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Params)]),
    "rbffd_destroy": (C.c_int, [C.c_void_p]),
    "rbffd_last_error": (C.c_char_p, [C.c_void_p]),
    "rbffd_build_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_void_p, C.c_int64, C.c_uint32,
                                      C.c_void_p, C.c_void_p, C.c_int64,
                                      C.POINTER(C.c_int64), C.c_void_p]),
    "rbffd_build_weights_masked": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                             C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                             C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "rbffd_build_weights_noalloc": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p,
                                              C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.c_uint32, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.POINTER(C.c_int64), C.c_void_p]),
    "rbffd_probe_fma": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                  C.c_void_p]),
    "rbffd_debug_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "rbffd_ensemble_step": (C.c_int, [C.c_void_p, C.POINTER(FlowC), C.c_int32,
                                      C.POINTER(C.c_double), C.POINTER(StateC), C.c_void_p,
                                      C.c_void_p, C.c_int32, C.POINTER(Stats), C.c_void_p]),
    "rbffd_stencil_condition": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_int64, C.c_void_p, C.c_void_p]),
    "rbffd_modified_wavenumber": (C.c_int, [C.c_void_p, C.POINTER(Ell), C.POINTER(Ell),
                                            C.POINTER(Ell), C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_stencil_error": (C.c_int, [C.c_void_p, C.POINTER(Ell), C.c_uint32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_apply_op": (C.c_int, [C.c_void_p, C.POINTER(Ell), C.c_void_p, C.c_void_p,
                                 C.c_double, C.c_double, C.c_int32, C.c_void_p]),
    "rbffd_apply_op_shape": (C.c_int, [C.c_void_p, C.POINTER(Ell), C.c_int32,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "rbffd_step": (C.c_int, [C.c_void_p, C.POINTER(FlowC), C.POINTER(StateC), C.c_void_p,
                             C.c_void_p, C.c_int32, C.POINTER(Stats), C.c_void_p]),
    "rbffd_adjoint_step": (C.c_int, [C.c_void_p, C.POINTER(FlowC), C.POINTER(StateC),
                                     C.POINTER(AdjointC), C.c_void_p, C.c_void_p,
                                     C.POINTER(Stats), C.c_void_p]),
    "rbffd_cylinder_forces": (C.c_int, [C.c_void_p, C.POINTER(FlowC), C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                        C.c_double, C.c_double, C.c_double,
                                        C.POINTER(C.c_double), C.c_void_p]),
}


def lib():
    """The loaded librbffd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2206_06495_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("rbffd needs a CUDA device; no CPU fallback exists")
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("rbffd arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("rbffd arrays must be contiguous")
    return C.c_void_p(t.data_ptr())


def round_up(a: int, b: int = 32) -> int:
    return (a + b - 1) // b * b


class Context:
    """rbffd_create / rbffd_destroy around stencil parameters (n, m, q)."""

    def __init__(self, n: int = 28, m: int = 7, q: int = 3):
        _torch()
        self.n, self.m, self.q = n, m, q
        h = C.c_void_p()
        rc = lib().rbffd_create(C.byref(h), C.byref(Params(n, m, q)))
        if rc != OK:
            raise RbffdError(rc, f"rbffd_create(n={n}, m={m}, q={q}) failed")
        self.handle = h

    def check(self, rc: int):
        if rc != OK:
            msg = lib().rbffd_last_error(self.handle)
            raise RbffdError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            lib().rbffd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ops_of(mask: int) -> list[int]:
    return [b for b in (OP_INTERP, OP_DX, OP_DY, OP_LAP) if mask & b]


def build_weights(ctx: Context, ax, ay, bx, by, op_mask: int, ld: int | None = None):
    """rbffd_build_weights.  Returns (idx int32 [n, ld], w float64 [nops, n, ld], bad_node)."""
    torch = _torch()
    na = ax.numel()
    ld = round_up(max(na, 1)) if ld is None else ld
    nops = len(ops_of(op_mask))
    idx = torch.empty((ctx.n, ld), dtype=torch.int32, device=ax.device)
    w = torch.empty((nops, ctx.n, ld), dtype=torch.float64, device=ax.device)
    bad = C.c_int64(-1)
    rc = lib().rbffd_build_weights(ctx.handle, _ptr(ax), _ptr(ay), na, _ptr(bx), _ptr(by),
                                   bx.numel(), op_mask, _ptr(idx), _ptr(w), ld, C.byref(bad),
                                   _stream())
    if rc == ERR_SINGULAR_STENCIL:
        return idx, w, int(bad.value)
    ctx.check(rc)
    return idx, w, -1


def build_weights_masked(ctx: Context, ax, ay, bx, by, op_mask: int, beta_mask=None,
                         alpha_self=None, ld: int | None = None):
    """rbffd_build_weights_masked (see build_weights); beta_mask uint8 [n_beta],
    alpha_self int32 [n_alpha], either may be None."""
    torch = _torch()
    na = ax.numel()
    ld = round_up(max(na, 1)) if ld is None else ld
    nops = len(ops_of(op_mask))
    idx = torch.empty((ctx.n, ld), dtype=torch.int32, device=ax.device)
    w = torch.empty((nops, ctx.n, ld), dtype=torch.float64, device=ax.device)
    bad = C.c_int64(-1)
    rc = lib().rbffd_build_weights_masked(ctx.handle, _ptr(ax), _ptr(ay), na, _ptr(bx), _ptr(by),
                                          bx.numel(), _ptr(beta_mask), _ptr(alpha_self), op_mask,
                                          _ptr(idx), _ptr(w), ld, C.byref(bad), _stream())
    if rc == ERR_SINGULAR_STENCIL:
        return idx, w, int(bad.value)
    ctx.check(rc)
    return idx, w, -1


def apply_op(ctx: Context, idx, w, n_rows: int, n_cols: int, x, y=None, alpha: float = 1.0,
             beta: float = 0.0):
    """rbffd_apply_op: y = alpha * D x + beta * y.  w: [n, ld] float64 or float32."""
    torch = _torch()
    if y is None:
        y = torch.zeros(n_rows, dtype=x.dtype, device=x.device)
    D = Ell(idx=_ptr(idx).value, w=_ptr(w).value, n_rows=n_rows, n_cols=n_cols,
            ld=idx.shape[1], n=idx.shape[0], w_dtype=F64 if w.dtype == torch.float64 else F32)
    xy = F64 if x.dtype == torch.float64 else F32
    ctx.check(lib().rbffd_apply_op(ctx.handle, C.byref(D), _ptr(x), _ptr(y), alpha, beta, xy,
                                   _stream()))
    return y


def apply_op_shape(ctx: Context, idx, w, n_rows: int, n_cols: int, x_dtype) -> tuple[int, int]:
    """rbffd_apply_op_shape: (threads per block, blocks per SM) of the SpMV launch."""
    torch = _torch()
    D = Ell(idx=_ptr(idx).value, w=_ptr(w).value, n_rows=n_rows, n_cols=n_cols,
            ld=idx.shape[1], n=idx.shape[0], w_dtype=F64 if w.dtype == torch.float64 else F32)
    t, b = C.c_int32(0), C.c_int32(0)
    ctx.check(lib().rbffd_apply_op_shape(ctx.handle, C.byref(D),
                                         F64 if x_dtype == torch.float64 else F32,
                                         C.byref(t), C.byref(b)))
    return t.value, b.value


@dataclass
class Flow:
    """Device tensors of one staggered flow problem plus its rbffd_flow struct."""
    N: int
    M: int
    tensors: dict
    Re: float
    dt: float
    precision: int = PREC_FP64
    tol: float = 1e-12
    inner_tol: float = 5e-3
    max_iter: int = 20000
    km_mode: int = 2
    overwrite_bc: int = 1
    profile: int = 0
    precond: int = 1
    projection: int = PROJ_PAPER
    cn_form: int = CN_PRINTED
    _c: FlowC = field(default=None, repr=False)

    def cstruct(self) -> FlowC:
        t = self.tensors
        p = lambda k: _ptr(t[k]).value  # noqa: E731
        return FlowC(N=self.N, M=self.M, ld_v=t["vv_idx"].shape[1], ld_p=t["pp_idx"].shape[1],
                     vv_idx=p("vv_idx"), vv_dx=p("vv_dx"), vv_dy=p("vv_dy"), vv_lap=p("vv_lap"),
                     pv_idx=p("pv_idx"), pv_dx=p("pv_dx"), pv_dy=p("pv_dy"),
                     pp_idx=p("pp_idx"), pp_dx=p("pp_dx"), pp_dy=p("pp_dy"), pp_lap=p("pp_lap"),
                     vp_idx=p("vp_idx"), vp_dx=p("vp_dx"), vp_dy=p("vp_dy"),
                     v_bc=p("v_bc"), v_nx=p("v_nx"), v_ny=p("v_ny"),
                     p_bc=p("p_bc"), p_nx=p("p_nx"), p_ny=p("p_ny"),
                     nb_p=t["pn_rows"].numel(), ld_b=t["pn_idx"].shape[1],
                     pn_rows=p("pn_rows"), pn_idx=p("pn_idx"), pn_dx=p("pn_dx"), pn_dy=p("pn_dy"),
                     Re=self.Re, dt=self.dt, precision=self.precision, tol=self.tol,
                     inner_tol=self.inner_tol, max_iter=self.max_iter, km_mode=self.km_mode,
                     overwrite_bc=self.overwrite_bc, profile=self.profile,
                     precond=self.precond,
                     p_edges=p("p_edges") if "p_edges" in t else None,
                     n_edges=t["p_edges"].shape[0] if "p_edges" in t else 0,
                     p_x=p("px") if "px" in t else None, p_y=p("py") if "py" in t else None,
                     projection=self.projection, cn_form=self.cn_form,
                     v_bcu=p("v_bcu") if "v_bcu" in t else None,
                     v_bcv=p("v_bcv") if "v_bcv" in t else None,
                     nb_v=t["vn_rows"].numel() if "vn_rows" in t else 0,
                     ld_vb=t["vn_idx"].shape[1] if "vn_idx" in t else 0,
                     vn_rows=p("vn_rows") if "vn_rows" in t else None,
                     vn_idx=p("vn_idx") if "vn_idx" in t else None,
                     vn_dx=p("vn_dx") if "vn_dx" in t else None,
                     vn_dy=p("vn_dy") if "vn_dy" in t else None)


def flow_from_nodes(ctx: Context, nodes, Re: float, dt: float, device="cuda", **kw) -> Flow:
    """Build the four operator families of Section 4 on the GPU (four calls of
    rbffd_build_weights) and the boundary tables of a staggered node set."""
    torch = _torch()
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)  # noqa: E731
    px, py, vx, vy = d(nodes.px), d(nodes.py), d(nodes.vx), d(nodes.vy)
    N, M = nodes.N, nodes.M
    ld_v, ld_p = round_up(N), round_up(M)
    t = {}
    i, w, bad = build_weights(ctx, vx, vy, vx, vy, OP_DX | OP_DY | OP_LAP, ld_v)
    if bad >= 0:
        raise RbffdError(ERR_SINGULAR_STENCIL, f"V->V stencil {bad}")
    t["vv_idx"], t["vv_dx"], t["vv_dy"], t["vv_lap"] = i, w[0], w[1], w[2]
    i, w, bad = build_weights(ctx, px, py, vx, vy, OP_DX | OP_DY, ld_p)
    if bad >= 0:
        raise RbffdError(ERR_SINGULAR_STENCIL, f"V->P stencil {bad}")
    t["pv_idx"], t["pv_dx"], t["pv_dy"] = i, w[0], w[1]
    i, w, bad = build_weights(ctx, px, py, px, py, OP_DX | OP_DY | OP_LAP, ld_p)
    if bad >= 0:
        raise RbffdError(ERR_SINGULAR_STENCIL, f"P->P stencil {bad}")
    t["pp_idx"], t["pp_dx"], t["pp_dy"], t["pp_lap"] = i, w[0], w[1], w[2]
    i, w, bad = build_weights(ctx, vx, vy, px, py, OP_DX | OP_DY, ld_v)
    if bad >= 0:
        raise RbffdError(ERR_SINGULAR_STENCIL, f"P->V stencil {bad}")
    t["vp_idx"], t["vp_dx"], t["vp_dy"] = i, w[0], w[1]
    # one-sided Neumann stencils of boundary P-nodes: the node, then its
    # nearest interior P-nodes
    bnd = np.nonzero(nodes.p_boundary)[0]
    rows = d(bnd.astype(np.int32))
    interior = d((~nodes.p_boundary).astype(np.uint8))
    i, w, bad = build_weights_masked(ctx, px[rows.long()], py[rows.long()], px, py,
                                     OP_DX | OP_DY, beta_mask=interior, alpha_self=rows)
    if bad >= 0:
        raise RbffdError(ERR_SINGULAR_STENCIL, f"Neumann stencil {bad}")
    t["pn_rows"], t["pn_idx"], t["pn_dx"], t["pn_dy"] = rows, i, w[0].contiguous(), w[1].contiguous()
    t["v_bc"] = d(nodes.v_boundary.astype(np.uint8))
    t["v_nx"], t["v_ny"] = d(nodes.v_nx), d(nodes.v_ny)
    t["p_bc"] = d(nodes.p_boundary.astype(np.uint8))
    t["p_nx"], t["p_ny"] = d(nodes.p_nx), d(nodes.p_ny)
    t["px"], t["py"], t["vx"], t["vy"] = px, py, vx, vy
    t["p_edges"] = d(np.asarray(nodes.edges, dtype=np.int32))
    return Flow(N=N, M=M, tensors=t, Re=Re, dt=dt, **kw)


@dataclass
class State:
    u: object
    v: object
    cu_prev: object
    cv_prev: object
    pt: object
    p: object
    j: int = 0

    @staticmethod
    def zeros(flow: Flow, device="cuda"):
        torch = _torch()
        z = lambda n: torch.zeros(n, dtype=torch.float64, device=device)  # noqa: E731
        return State(z(flow.N), z(flow.N), z(flow.N), z(flow.N), z(flow.M), z(flow.M), 0)


def step(ctx: Context, flow: Flow, state: State, gu, gv, n_steps: int = 1) -> dict:
    """rbffd_step: advance `state` in place by n_steps; returns the statistics.
    On failure the raised RbffdError carries them as `.stats`."""
    fc = flow.cstruct()
    sc = StateC(u=_ptr(state.u).value, v=_ptr(state.v).value, cu_prev=_ptr(state.cu_prev).value,
                cv_prev=_ptr(state.cv_prev).value, pt=_ptr(state.pt).value,
                p=_ptr(state.p).value, j=state.j)
    st = Stats()
    rc = lib().rbffd_step(ctx.handle, C.byref(fc), C.byref(sc), _ptr(gu), _ptr(gv), n_steps,
                          C.byref(st), _stream())
    state.j = sc.j
    try:
        ctx.check(rc)
    except RbffdError as e:
        e.stats = st.as_dict()
        raise
    return st.as_dict()


def _ell(idx, w, n_rows: int, n_cols: int) -> Ell:
    torch = _torch()
    return Ell(idx=_ptr(idx).value, w=_ptr(w).value, n_rows=n_rows, n_cols=n_cols,
               ld=idx.shape[1], n=idx.shape[0], w_dtype=F64 if w.dtype == torch.float64 else F32)


def stencil_condition(ctx: Context, ax, ay, bx, by, idx):
    """rbffd_stencil_condition: 1-norm condition number of every stencil's
    local system (float64 [n_alpha])."""
    torch = _torch()
    na = ax.numel()
    cond = torch.empty(na, dtype=torch.float64, device=ax.device)
    ctx.check(lib().rbffd_stencil_condition(ctx.handle, _ptr(ax), _ptr(ay), na, _ptr(bx),
                                            _ptr(by), bx.numel(), _ptr(idx), idx.shape[1],
                                            _ptr(cond), _stream()))
    return cond


def modified_wavenumber(ctx: Context, idx, wx, wy, ax, ay, bx, by, kx: float, ky: float,
                        idx_lap=None, w_lap=None):
    """rbffd_modified_wavenumber: (k*/k~, k*^2/k~^2 or None) as complex128 tensors."""
    torch = _torch()
    n = ax.numel()
    Dx, Dy = _ell(idx, wx, n, bx.numel()), _ell(idx, wy, n, bx.numel())
    Dl = _ell(idx_lap, w_lap, n, bx.numel()) if w_lap is not None else None
    k1 = torch.empty(2 * n, dtype=torch.float64, device=ax.device)
    k2 = torch.empty(2 * n, dtype=torch.float64, device=ax.device) if Dl else None
    ctx.check(lib().rbffd_modified_wavenumber(
        ctx.handle, C.byref(Dx), C.byref(Dy), C.byref(Dl) if Dl else None, _ptr(ax), _ptr(ay),
        _ptr(bx), _ptr(by), kx, ky, _ptr(k1), _ptr(k2), _stream()))
    as_c = lambda t: torch.view_as_complex(t.view(n, 2))  # noqa: E731
    return as_c(k1), (as_c(k2) if k2 is not None else None)


def stencil_error(ctx: Context, idx, w, op: int, ax, ay, bx, by, dr=None):
    """rbffd_stencil_error: (per-node relative error, its mean as a 0-d tensor)."""
    torch = _torch()
    n = ax.numel()
    D = _ell(idx, w, n, bx.numel())
    err = torch.empty(n, dtype=torch.float64, device=ax.device)
    mean = torch.zeros((), dtype=torch.float64, device=ax.device)
    ctx.check(lib().rbffd_stencil_error(ctx.handle, C.byref(D), op, _ptr(ax), _ptr(ay),
                                        _ptr(bx), _ptr(by), _ptr(dr), _ptr(err), _ptr(mean),
                                        _stream()))
    return err, mean


def ensemble_zeros(flow: Flow, n_members: int, device="cuda") -> State:
    """A member-contiguous ensemble state at rest ([N * E] and [M * E] arrays)."""
    torch = _torch()
    z = lambda n: torch.zeros(n * n_members, dtype=torch.float64, device=device)  # noqa: E731
    return State(z(flow.N), z(flow.N), z(flow.N), z(flow.N), z(flow.M), z(flow.M), 0)


def ensemble_step(ctx: Context, flow: Flow, Re, state: State, gu, gv, n_steps: int = 1) -> dict:
    """rbffd_ensemble_step: E = len(Re) members, member-contiguous state and
    wall data (entry (i, e) at [i * E + e]); advances state in place."""
    E = len(Re)
    re = (C.c_double * E)(*[float(r) for r in Re])
    fc = flow.cstruct()
    sc = _state_c(state)
    st = Stats()
    rc = lib().rbffd_ensemble_step(ctx.handle, C.byref(fc), E, re, C.byref(sc), _ptr(gu),
                                   _ptr(gv), n_steps, C.byref(st), _stream())
    state.j = sc.j
    try:
        ctx.check(rc)
    except RbffdError as e:
        e.stats = st.as_dict()
        raise
    return st.as_dict()


def debug_set_wait_limit(ctx: Context, polls: int) -> None:
    """rbffd_debug_set_wait_limit (test hook): polls of the first staged-copy
    wait; 0 gives up at once, a negative value restores the default."""
    ctx.check(lib().rbffd_debug_set_wait_limit(ctx.handle, polls))


@dataclass
class Adjoint:
    """Adjoint variables of a State (dJ/du, dJ/dv, dJ/dC_{j-1}, dJ/dp~)."""
    u: object
    v: object
    cu_prev: object
    cv_prev: object
    pt: object

    @staticmethod
    def zeros(flow: Flow, device="cuda"):
        torch = _torch()
        z = lambda n: torch.zeros(n, dtype=torch.float64, device=device)  # noqa: E731
        return Adjoint(z(flow.N), z(flow.N), z(flow.N), z(flow.N), z(flow.M))


def _state_c(state: State) -> StateC:
    return StateC(u=_ptr(state.u).value, v=_ptr(state.v).value,
                  cu_prev=_ptr(state.cu_prev).value, cv_prev=_ptr(state.cv_prev).value,
                  pt=_ptr(state.pt).value, p=_ptr(state.p).value, j=state.j)


def adjoint_step(ctx: Context, flow: Flow, fwd: State, lam: Adjoint, grad_gu, grad_gv) -> dict:
    """rbffd_adjoint_step: lam (adjoints of step j+1) -> adjoints of step j, in
    place; the step's wall-data adjoint is added to grad_gu, grad_gv."""
    fc = flow.cstruct()
    sc = _state_c(fwd)
    ac = AdjointC(u=_ptr(lam.u).value, v=_ptr(lam.v).value, cu_prev=_ptr(lam.cu_prev).value,
                  cv_prev=_ptr(lam.cv_prev).value, pt=_ptr(lam.pt).value)
    st = Stats()
    ctx.check(lib().rbffd_adjoint_step(ctx.handle, C.byref(fc), C.byref(sc), C.byref(ac),
                                       _ptr(grad_gu), _ptr(grad_gv), C.byref(st), _stream()))
    return st.as_dict()


def probe_fma(ctx: Context, dtype: int = F64, iters: int = 4096) -> float:
    """rbffd_probe_fma: measured FMA throughput in GFLOP/s."""
    g = C.c_double(0.0)
    ctx.check(lib().rbffd_probe_fma(ctx.handle, dtype, iters, C.byref(g), _stream()))
    return g.value


def version() -> int:
    return lib().rbffd_version()


def cylinder_forces(ctx: Context, flow: Flow, state: State, rows, radius: float, Re: float,
                    cx: float = 0.0, cy: float = 0.0):
    """rbffd_cylinder_forces: (C_D, C_L) of the circular body whose surface
    P-nodes are `rows` (int32 device tensor, increasing angle, even count)."""
    out = (C.c_double * 2)()
    fc = flow.cstruct()
    ctx.check(lib().rbffd_cylinder_forces(ctx.handle, C.byref(fc), _ptr(state.u), _ptr(state.v),
                                          _ptr(state.p), _ptr(rows), rows.numel(), cx, cy,
                                          radius, Re, out, _stream()))
    return float(out[0]), float(out[1])
