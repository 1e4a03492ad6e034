"""Plain FP64 CPU oracle for the RBF-FD staggered-node Navier-Stokes hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module: only the tests, the package's smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA path.

Every function restates a step of the paper (Chu & Schmidt, "RBF-FD
discretization of the Navier-Stokes equations on scattered but staggered
nodes") in the plainest form that numpy/scipy allow:

  * stencils: the n nearest beta-nodes of each alpha-node (Section 2.2),
    brute force, ties broken by node index;
  * weights: one dense solve of the augmented PHS+poly saddle system per
    stencil (Section 2.1, Eq. rbf_poly_compact), LU with partial pivoting
    (numpy.linalg.solve);
  * operators: CSR matrices D_L^(alpha,beta) (Section 2.2);
  * the fractional step (Section 3): AB2 convection, Crank-Nicolson viscous
    solve, divergence, pressure Poisson, pressure, velocity correction, with
    the Kim & Moin intermediate-velocity boundary values.  The implicit
    matrices are LU-factorised once, as in the paper (end of Section 3).

Readings of points the paper leaves open:
  R1 local coordinates: shift by the stencil centre, scale by the largest
     centre-to-node distance s; weights of first derivatives are divided by s
     and of the Laplacian by s^2 afterwards.
  R2 monomials in graded lexicographic order 1, x, y, x^2, xy, y^2, ...
  R3 k-NN ties: sort by (squared distance, index); squared distance is
     dx*dx + dy*dy with each operation rounded (no fused multiply-add).
  R4 pressure Poisson: boundary P-rows are replaced by a homogeneous Neumann
     row n_x D_x + n_y D_y whose stencil is the boundary node itself followed
     by its n-1 nearest interior P-nodes (a one-sided stencil that does not
     lean on the other wall nodes, which carry no normal information); the
     constant null space is removed by bordering
     [L e; 1^T 0][p; lam] = [b; 0], where e is 1 on boundary P-rows and 0 on
     interior rows: every interior row is Eq. pressure_Poisson exactly, and
     the multiplier absorbs the incompatibility of the non-symmetric L as a
     uniform normal derivative on the Neumann rows.  (With e on the interior
     rows instead, each projection leaves a uniform interior divergence
     lam*dt that the next right side carries again, so it accumulates over
     the run; on the boundary rows it does not.)  The result is the
     mean-zero pressure correction.
  R5 boundary V-rows of the Crank-Nicolson solve are identity rows whose
     right-hand side is the Kim & Moin value of the end of Section 3: the
     wall data g_{j+1} plus dt D^(VP) p~_j, both components as printed
     (km_mode 2, the default).  km_mode 1 adds only the component along the
     wall tangent (the normal one vanishes for the continuous problem under
     the Neumann pressure condition), km_mode 0 adds nothing.
  R6 after the velocity correction, boundary V-nodes are overwritten with
     g_{j+1} (switchable).
  R7 AB2 at the first step uses C_{-1} = C_0; the flow starts from rest with
     p~_0 = 0.
  R17 open flows (Section 5.2, flow past a cylinder): each boundary V-node
     carries a Dirichlet or a homogeneous Neumann condition per velocity
     component, each boundary P-node a homogeneous Neumann or a Dirichlet
     (p~ = 0) condition.  The stress-free outlet is read as du/dn = dv/dn = 0
     for the intermediate velocity and p~ = 0 for the pressure correction
     (the outlet rows of the pressure system make it nonsingular: no
     bordering); the outlet's two corner P-nodes keep the side walls'
     Neumann row.  (With p~ = 0 there too, a mode localised at the corner,
     where the slip side meets the outlet, grew by 1.66 per step at dt 0.01
     on a uniform channel flow, an exact solution; with the Neumann corner
     rows the flow stays at rounding level.)  Neumann V-rows are n_x D_x + n_y D_y on a one-sided stencil,
     the node itself followed by its n-1 nearest interior V-nodes (as R4).
     Dirichlet V-rows take the Kim & Moin value of R5; after the correction
     only Dirichlet components are overwritten with the data.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

OP_INTERP, OP_DX, OP_DY, OP_LAP = "interp", "dx", "dy", "lap"
ALL_OPS = (OP_INTERP, OP_DX, OP_DY, OP_LAP)


# --------------------------------------------------------------------------
# Stencils (Section 2.2: row i uses the n nearest beta-nodes of alpha-node i)
# --------------------------------------------------------------------------
def knn(ax, ay, bx, by, k: int, chunk: int = 256, beta_mask=None, alpha_self=None,
        method: str = "auto") -> np.ndarray:
    """Indices of the k nearest beta-nodes of every alpha-node, nearest first.

    The definition is brute force over all beta-nodes with the ordering key
    (d^2, index), d^2 = dx*dx + dy*dy evaluated one rounded operation at a
    time (R3).  For large sets ("auto" above 4e7 node pairs, or "tree") a k-d
    tree proposes k + 12 candidates per alpha-node; those are ordered by the
    same key, and a row is kept only when its k-th key is below every key the
    tree did not return (checked against the farthest candidate with a
    relative margin of 1e-12); the other rows fall back to brute force.  The
    result is identical to the brute-force one.
    beta_mask: only beta-nodes with a nonzero mask are candidates.
    alpha_self: beta index of each alpha-node; when given, slot 0 is that
    node and the other k-1 slots are the nearest masked beta-nodes.
    Returns int64 [n_alpha, k].
    """
    ax = np.asarray(ax, np.float64)
    ay = np.asarray(ay, np.float64)
    bx = np.asarray(bx, np.float64)
    by = np.asarray(by, np.float64)
    nb = bx.size
    kk = k - (1 if alpha_self is not None else 0)
    allowed = np.ones(nb, bool) if beta_mask is None else np.asarray(beta_mask) != 0
    if kk > int(allowed.sum()):
        raise ValueError("stencil size exceeds the number of beta-nodes")
    out = np.empty((ax.size, k), np.int64)
    if alpha_self is not None:
        out[:, 0] = np.asarray(alpha_self)
        if kk > 0:
            out[:, 1:] = knn(ax, ay, bx, by, kk, chunk, beta_mask, None, method)
        return out
    if method == "tree" or (method == "auto" and ax.size * nb > 4e7):
        return _knn_tree(ax, ay, bx, by, k, allowed, chunk)
    return _knn_brute(ax, ay, bx, by, k, allowed, chunk)


def _knn_brute(ax, ay, bx, by, k, allowed, chunk=256):
    """Brute-force k nearest: every beta-node's key, the k smallest kept."""
    nb = bx.size
    out = np.empty((ax.size, k), np.int64)
    cols = np.arange(nb)
    for s in range(0, ax.size, chunk):
        dx = bx[None, :] - ax[s:s + chunk, None]
        dy = by[None, :] - ay[s:s + chunk, None]
        d2 = dx * dx + dy * dy
        d2[:, ~allowed] = np.inf
        for r in range(d2.shape[0]):
            row = d2[r]
            kth = np.partition(row, k - 1)[k - 1]
            cand = np.nonzero(row <= kth)[0]
            order = np.lexsort((cols[cand], row[cand]))[:k]
            out[s + r] = cand[order]
    return out


def _knn_tree(ax, ay, bx, by, k, allowed, chunk=256):
    """k nearest from k-d tree candidates, exact under the (d^2, index) key."""
    from scipy.spatial import cKDTree
    cand_ids = np.nonzero(allowed)[0]
    kq = min(k + 12, cand_ids.size)
    tree = cKDTree(np.stack([bx[cand_ids], by[cand_ids]], -1))
    _, nn = tree.query(np.stack([ax, ay], -1), k=kq)
    nn = cand_ids[np.asarray(nn).reshape(ax.size, kq)]
    dx = bx[nn] - ax[:, None]
    dy = by[nn] - ay[:, None]
    d2 = dx * dx + dy * dy
    order = np.lexsort((nn, d2), axis=-1)
    nn = np.take_along_axis(nn, order, -1)
    d2 = np.take_along_axis(d2, order, -1)
    out = nn[:, :k].copy()
    if kq < cand_ids.size:
        # every beta-node the tree left out is at least as far as its farthest
        # candidate; a row is exact when its k-th key is strictly closer
        bad = np.nonzero(~(d2[:, k - 1] < d2[:, -1] * (1.0 - 1e-12)))[0]
        if bad.size:
            out[bad] = _knn_brute(ax[bad], ay[bad], bx, by, k, allowed, chunk)
    return out


# --------------------------------------------------------------------------
# Local weights (Section 2.1)
# --------------------------------------------------------------------------
def monomial_exponents(q: int) -> list[tuple[int, int]]:
    """(a, b) of x^a y^b for all monomials of degree <= q, graded lex (R2).

    There are (q+1)(q+2)/2 of them (Eq. Lf_PHS); q = -1 means none.
    """
    return [(d - b, b) for d in range(q + 1) for b in range(d + 1)]


def _phs(r, m):
    """phi(r) = r^m, m odd (Section 2.1)."""
    return r ** m


def _op_rhs_rbf(op, X, m):
    """L phi(||x - x_j||) at the stencil centre x = 0 (right side of Eq. w_local)."""
    r = np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2)
    if op == OP_INTERP:
        return _phs(r, m)
    # d/dx r^m = m r^(m-2) (x - x_j); at x = 0 this is -m r^(m-2) x_j
    if op == OP_DX:
        return -m * r ** (m - 2) * X[..., 0]
    if op == OP_DY:
        return -m * r ** (m - 2) * X[..., 1]
    # 2-D Laplacian of r^m: m(m-1) r^(m-2) + (1/r) m r^(m-1) = m^2 r^(m-2)
    if op == OP_LAP:
        return m * m * r ** (m - 2)
    raise ValueError(op)


def _op_rhs_poly(op, q):
    """L P_i at the stencil centre x = 0 (the vanishing-moment right side)."""
    out = []
    for a, b in monomial_exponents(q):
        if op == OP_INTERP:
            v = 1.0 if (a, b) == (0, 0) else 0.0
        elif op == OP_DX:
            v = 1.0 if (a, b) == (1, 0) else 0.0
        elif op == OP_DY:
            v = 1.0 if (a, b) == (0, 1) else 0.0
        elif op == OP_LAP:
            v = 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0
        else:
            raise ValueError(op)
        out.append(v)
    return np.array(out)


def augmented_matrix(X: np.ndarray, m: int, q: int) -> np.ndarray:
    """A_aug = [[A, P], [P^T, 0]] of Eq. rbf_poly_compact for stencil nodes X.

    X: [..., n, 2] local (shifted, scaled) coordinates.
    A_ij = phi(||x_i - x_j||) (Eq. A), P_ji = P_i(x_j).
    """
    n = X.shape[-2]
    mono = monomial_exponents(q)
    S = n + len(mono)
    batch = X.shape[:-2]
    Aaug = np.zeros(batch + (S, S))
    diff = X[..., :, None, :] - X[..., None, :, :]
    r = np.sqrt(diff[..., 0] ** 2 + diff[..., 1] ** 2)
    Aaug[..., :n, :n] = _phs(r, m)
    for i, (a, b) in enumerate(mono):
        col = X[..., 0] ** a * X[..., 1] ** b
        Aaug[..., :n, n + i] = col
        Aaug[..., n + i, :n] = col
    return Aaug


def stencil_weights(center, nodes, m: int, q: int, ops=(OP_DX, OP_DY, OP_LAP)):
    """Weights w (Eq. Lf) of each operator for one or many stencils.

    center: [..., 2]; nodes: [..., n, 2] (global coordinates).
    Returns {op: [..., n]} and the per-stencil scale s.
    Steps: shift to the centre and divide by s = max ||x_j - x_0|| (R1);
    assemble A_aug (Eq. rbf_poly_compact); solve A_aug [w; c] = [L phi; L P]
    by LU with partial pivoting; keep w; undo the scaling.
    """
    center = np.asarray(center, np.float64)
    nodes = np.asarray(nodes, np.float64)
    n = nodes.shape[-2]
    X = nodes - center[..., None, :]
    s = np.sqrt((X[..., 0] ** 2 + X[..., 1] ** 2).max(-1))
    X = X / s[..., None, None]
    Aaug = augmented_matrix(X, m, q)
    rhs = []
    for op in ops:
        top = _op_rhs_rbf(op, X, m)
        bot = np.broadcast_to(_op_rhs_poly(op, q), X.shape[:-2] + (Aaug.shape[-1] - n,))
        rhs.append(np.concatenate([top, bot], -1))
    B = np.stack(rhs, -1)  # [..., S, nops]
    sol = np.linalg.solve(Aaug, B)
    out = {}
    for j, op in enumerate(ops):
        w = sol[..., :n, j]
        if op in (OP_DX, OP_DY):
            w = w / s[..., None]
        elif op == OP_LAP:
            w = w / (s[..., None] ** 2)
        out[op] = w
    return out, s


def build_weights(ax, ay, bx, by, k: int, m: int = 7, q: int = 3,
                  ops=(OP_DX, OP_DY, OP_LAP), chunk: int = 4096, idx=None):
    """Stencils and weights of D_L^(alpha,beta) for every alpha-node.

    Returns (idx [n_alpha, k] int64, {op: w [n_alpha, k] float64}).
    """
    ax = np.asarray(ax, np.float64)
    ay = np.asarray(ay, np.float64)
    bx = np.asarray(bx, np.float64)
    by = np.asarray(by, np.float64)
    if idx is None:
        idx = knn(ax, ay, bx, by, k)
    W = {op: np.empty(idx.shape) for op in ops}
    for s0 in range(0, ax.size, chunk):
        sl = slice(s0, s0 + chunk)
        c = np.stack([ax[sl], ay[sl]], -1)
        X = np.stack([bx[idx[sl]], by[idx[sl]]], -1)
        w, _ = stencil_weights(c, X, m, q, ops)
        for op in ops:
            W[op][sl] = w[op]
    return idx, W


def csr(idx: np.ndarray, w: np.ndarray, n_cols: int) -> sp.csr_matrix:
    """The sparse matrix D with D[i, idx[i, s]] = w[i, s] (Section 2.2)."""
    n_rows, k = idx.shape
    indptr = np.arange(0, n_rows * k + 1, k)
    return sp.csr_matrix((w.ravel(), idx.ravel(), indptr), shape=(n_rows, n_cols))


# --------------------------------------------------------------------------
# Accuracy measures (Section 4)
# --------------------------------------------------------------------------
def local_spacing(x, y, n_adj: int = 6) -> np.ndarray:
    """Delta r_j: mean distance from node j to its n_adj nearest other nodes
    of the same set (reading of Section 3's 'locally averaged distance')."""
    idx = knn(x, y, x, y, n_adj + 1)
    d = np.hypot(x[idx[:, 1:]] - x[:, None], y[idx[:, 1:]] - y[:, None])
    return d.mean(1)


def modified_wavenumber(w_dx, w_dy, idx, ax, ay, bx, by, kx, ky):
    """Radial modified wavenumber k* of Eq. 2d_mw at every alpha-node.

    delta_r = (kx D_x + ky D_y)/k~ applied to exp(i k~ r~), r~ = (kx x + ky y)/k~,
    then multiplied by -i exp(-i k~ r~(x_0)).
    """
    kt = np.hypot(kx, ky)
    phase_b = np.exp(1j * (kx * bx + ky * by))
    phase_a = np.exp(-1j * (kx * ax + ky * ay))
    d_r = (kx * w_dx + ky * w_dy) / kt
    return (-1j * (d_r * phase_b[idx]).sum(1) * phase_a)


def test_function_derivative(x, y, dr, op):
    """L g at (x, y) for the test function g = cos(x/dr) cos(y/dr) of
    Section 4 (Eq. test), with max |L g| over the plane (reading R11):
    returns (L g, max |L g|)."""
    cx, sx = np.cos(x / dr), np.sin(x / dr)
    cy, sy = np.cos(y / dr), np.sin(y / dr)
    if op == OP_DX:
        return -sx * cy / dr, 1.0 / dr
    if op == OP_DY:
        return -cx * sy / dr, 1.0 / dr
    if op == OP_LAP:
        return -2.0 * cx * cy / dr ** 2, 2.0 / dr ** 2
    return cx * cy, 1.0


def stencil_error(w, idx, ax, ay, bx, by, op, dr) -> np.ndarray:
    """Per-node relative error of Eq. relative_error: for alpha-node i and its
    own test function g_i = cos(x/dr_i) cos(y/dr_i) (Eq. test, dr_i the local
    spacing), |sum_s w_is g_i(x_j) - L g_i(x_i)| / max |L g_i|.  The paper's E
    is the mean over the nodes."""
    dr = np.asarray(dr, np.float64)
    g = np.cos(bx[idx] / dr[:, None]) * np.cos(by[idx] / dr[:, None])
    exact, scale = test_function_derivative(ax, ay, dr, op)
    return np.abs((w * g).sum(1) - exact) / scale


def stencil_condition(ax, ay, bx, by, idx, m: int, q: int) -> np.ndarray:
    """1-norm condition number ||A_aug||_1 ||A_aug^-1||_1 of every stencil's
    augmented matrix (Eq. rbf_poly_compact) in the local coordinates of R1,
    the matrix the weight solve factors (Section 4.2 discusses these numbers
    for the parameter choice).  Exact: numpy's dense inverse per stencil."""
    ax = np.asarray(ax, np.float64)
    ay = np.asarray(ay, np.float64)
    out = np.empty(idx.shape[0])
    for s0 in range(0, idx.shape[0], 2048):
        sl = slice(s0, s0 + 2048)
        X = np.stack([bx[idx[sl]] - ax[sl, None], by[idx[sl]] - ay[sl, None]], -1)
        sc = np.sqrt((X[..., 0] ** 2 + X[..., 1] ** 2).max(-1))
        A = augmented_matrix(X / sc[:, None, None], m, q)
        out[sl] = np.linalg.cond(A, 1)
    return out


def modified_wavenumber_local(w_dx, w_dy, idx, ax, ay, bx, by, kx, ky, w_lap=None):
    """Normalised modified wavenumbers k*/k~ (Eq. 2d_mw) of the first
    derivative along the wave direction and, when w_lap is given, k*^2/k~^2
    of the Laplacian, at every alpha-node; the phase of each stencil node is
    taken relative to the alpha-node, exp(i k.(x_j - x_0)), which equals
    exp(i k.x_j) exp(-i k.x_0)."""
    kt = np.hypot(kx, ky)
    ph = np.exp(1j * (kx * (bx[idx] - ax[:, None]) + ky * (by[idx] - ay[:, None])))
    k1 = -1j * ((kx * w_dx + ky * w_dy) / kt * ph).sum(1) / kt
    k2 = None if w_lap is None else -(w_lap * ph).sum(1) / (kt * kt)
    return k1, k2


# --------------------------------------------------------------------------
# The fractional-step Navier-Stokes solver (Section 3)
# --------------------------------------------------------------------------
@dataclass
class Operators:
    """The seven differentiation matrices of Section 4 plus P->P first
    derivatives for the Neumann rows of reading R4."""
    vv_x: sp.csr_matrix
    vv_y: sp.csr_matrix
    vv_lap: sp.csr_matrix
    pv_x: sp.csr_matrix  # D^(P,V): V-values -> P-nodes
    pv_y: sp.csr_matrix
    pp_lap: sp.csr_matrix
    pp_x: sp.csr_matrix
    pp_y: sp.csr_matrix
    vp_x: sp.csr_matrix  # D^(V,P): P-values -> V-nodes
    vp_y: sp.csr_matrix
    pn_x: sp.csr_matrix  # P -> boundary P-nodes, one-sided Neumann stencils (R4)
    pn_y: sp.csr_matrix
    raw: dict


def build_operators(nodes, k: int = 28, m: int = 7, q: int = 3) -> Operators:
    """All operators of Section 4 for a staggered node set."""
    px, py, vx, vy = nodes.px, nodes.py, nodes.vx, nodes.vy
    M, N = px.size, vx.size
    i_vv, w_vv = build_weights(vx, vy, vx, vy, k, m, q, (OP_DX, OP_DY, OP_LAP))
    i_pv, w_pv = build_weights(px, py, vx, vy, k, m, q, (OP_DX, OP_DY))
    i_pp, w_pp = build_weights(px, py, px, py, k, m, q, (OP_DX, OP_DY, OP_LAP))
    i_vp, w_vp = build_weights(vx, vy, px, py, k, m, q, (OP_DX, OP_DY))
    bnd = np.nonzero(nodes.p_boundary)[0]
    i_pn = knn(px[bnd], py[bnd], px, py, k, beta_mask=~nodes.p_boundary, alpha_self=bnd)
    _, w_pn = build_weights(px[bnd], py[bnd], px, py, k, m, q, (OP_DX, OP_DY), idx=i_pn)
    rows = np.repeat(bnd, k)
    pn_x = sp.csr_matrix((w_pn[OP_DX].ravel(), (rows, i_pn.ravel())), shape=(M, M))
    pn_y = sp.csr_matrix((w_pn[OP_DY].ravel(), (rows, i_pn.ravel())), shape=(M, M))
    raw = {"vv": (i_vv, w_vv), "pv": (i_pv, w_pv), "pp": (i_pp, w_pp), "vp": (i_vp, w_vp),
           "pn": (bnd, i_pn, w_pn)}
    return Operators(
        vv_x=csr(i_vv, w_vv[OP_DX], N), vv_y=csr(i_vv, w_vv[OP_DY], N),
        vv_lap=csr(i_vv, w_vv[OP_LAP], N),
        pv_x=csr(i_pv, w_pv[OP_DX], N), pv_y=csr(i_pv, w_pv[OP_DY], N),
        pp_lap=csr(i_pp, w_pp[OP_LAP], M), pp_x=csr(i_pp, w_pp[OP_DX], M),
        pp_y=csr(i_pp, w_pp[OP_DY], M),
        vp_x=csr(i_vp, w_vp[OP_DX], M), vp_y=csr(i_vp, w_vp[OP_DY], M),
        pn_x=pn_x, pn_y=pn_y, raw=raw)


def poisson_matrix(ops: Operators, p_boundary, p_nx, p_ny) -> sp.csr_matrix:
    """Bordered pressure matrix [[L, e], [1^T, 0]] of reading R4.

    L = D^(P,P)_Lap (Eq. pressure_Poisson) with every boundary P-row replaced
    by n_x D_x + n_y D_y on the one-sided Neumann stencil of that node (R4);
    e = indicator of the boundary P-rows.
    """
    M = ops.pp_lap.shape[0]
    bnd = sp.diags(p_boundary.astype(float))
    inn = sp.diags((~p_boundary).astype(float))
    L = inn @ ops.pp_lap + bnd @ (sp.diags(p_nx) @ ops.pn_x + sp.diags(p_ny) @ ops.pn_y)
    e = sp.csr_matrix(p_boundary.astype(float)[:, None])
    one = sp.csr_matrix(np.ones((1, M)))
    return sp.bmat([[L, e], [one, None]], format="csc")


def exact_projection_matrices(ops: Operators, v_boundary, v_nx, v_ny):
    """G0 = D^(V,P) with zero wall rows (x and y), the wall normal field w,
    and the bordered matrix [[D^(P,V) G0, D^(P,V) w], [1^T, 0]] of the
    exactly projecting variant (see FractionalStep)."""
    inner = sp.diags((~v_boundary).astype(float))
    G0x = (inner @ ops.vp_x).tocsr()
    G0y = (inner @ ops.vp_y).tocsr()
    L = (ops.pv_x @ G0x + ops.pv_y @ G0y).tocsr()
    w_x = np.where(v_boundary, v_nx, 0.0)
    w_y = np.where(v_boundary, v_ny, 0.0)
    e = ops.pv_x @ w_x + ops.pv_y @ w_y
    M = L.shape[0]
    B = sp.bmat([[L, sp.csr_matrix(e[:, None])], [sp.csr_matrix(np.ones((1, M))), None]],
                format="csc")
    return G0x, G0y, w_x, w_y, B


def helmholtz_matrix(ops: Operators, v_boundary, a: float) -> sp.csr_matrix:
    """I - a D^(V,V)_Lap (Eq. u_ss, a = dt/(2 Re)) with identity boundary rows (R5)."""
    N = ops.vv_lap.shape[0]
    inn = sp.diags((~v_boundary).astype(float))
    return (sp.identity(N) - a * (inn @ ops.vv_lap)).tocsc()


@dataclass
class FlowState:
    u: np.ndarray
    v: np.ndarray
    cu_prev: np.ndarray  # C_{j-1}(u)
    cv_prev: np.ndarray
    pt: np.ndarray       # pressure correction p~_j
    p: np.ndarray        # pressure p_j
    lam: float = 0.0     # bordering multiplier of the last Poisson solve
    j: int = 0


class FractionalStep:
    """Three-stage semi-implicit step of Section 3 on a staggered node set."""

    def __init__(self, nodes, Re: float, dt: float, k: int = 28, m: int = 7,
                 q: int = 3, ops: Operators | None = None, overwrite_bc: bool = True,
                 km_mode: int = 2, viscous_solver: str = "lu", projection: str = "paper",
                 cn_form: str = "printed"):
        """viscous_solver: "lu" factorises I - a D_Lap once, as the paper does
        (end of Section 3); "krylov" solves it at every step with BiCGSTAB to a
        relative residual of 1e-14 instead (a library routine; for node sets
        whose LU fill-in is too large: I - a D_Lap is close to I there).

        projection: "paper" is Section 3's step (pressure Poisson with
        D^(P,P)_Lap, Kim & Moin wall values).  "exact" projects with the
        composed operator D^(P,V) G0, where G0 is D^(V,P) with its wall rows
        set to zero, so the corrected velocity is discretely divergence-free
        at every P-node (the variant the paper's D^(P,P)_Lap approximates):
          u** : (I - a D_Lap) u** = RHS - dt G0 p~_j inside, u** = g_{j+1} on
                the walls (the pressure increment form, which needs no Kim &
                Moin wall term: the projection leaves wall values alone);
          phi : D^(P,V) G0 phi + mu e = F / dt, 1^T phi = 0, with
                e = D^(P,V) w and w the outward wall normal at wall V-nodes;
          u_{j+1} = u** - dt G0 phi - mu dt w,  p~_{j+1} = p~_j + phi,
          p_{j+1} = p~_{j+1} - a D^(P,P)_Lap phi.
        D^(P,V) and G0 are not adjoint, so no gradient can remove one
        component of the divergence; the multiplier mu takes it up as a
        uniform normal velocity mu dt through the walls (FlowState.lam holds
        mu dt), which keeps D^(P,V) u_{j+1} = 0 on every row.

        cn_form: "printed" is Eq. u_ss, (I - a D_Lap) u** = (I + a D_Lap) u*;
        "kim_moin" is the Crank-Nicolson form of Kim & Moin, whose right side
        is u* + a D_Lap u_j (the printed form adds (dt^2/2Re) D_Lap of the
        convective update, an O(dt) term)."""
        if km_mode not in (0, 1, 2):
            raise ValueError("km_mode is 0, 1 or 2")
        if viscous_solver not in ("lu", "krylov"):
            raise ValueError("viscous_solver is 'lu' or 'krylov'")
        if projection not in ("paper", "exact"):
            raise ValueError("projection is 'paper' or 'exact'")
        if cn_form not in ("printed", "kim_moin"):
            raise ValueError("cn_form is 'printed' or 'kim_moin'")
        self.nodes = nodes
        self.km_mode = km_mode
        self.viscous_solver = viscous_solver
        self.projection = projection
        self.cn_form = cn_form
        self.Re = float(Re)
        self.dt = float(dt)
        self.a = self.dt / (2.0 * self.Re)
        self.ops = ops if ops is not None else build_operators(nodes, k, m, q)
        self.vb = nodes.v_boundary
        self.pb = nodes.p_boundary
        # unit tangent (-n_y, n_x) of the wall at boundary V-nodes (R5)
        self.tx = -nodes.v_ny
        self.ty = nodes.v_nx
        self.overwrite_bc = overwrite_bc
        self.H = helmholtz_matrix(self.ops, self.vb, self.a)
        if projection == "exact":
            self.G0x, self.G0y, self.w_x, self.w_y, self.Pb = exact_projection_matrices(
                self.ops, self.vb, nodes.v_nx, nodes.v_ny)
        else:
            self.Pb = poisson_matrix(self.ops, self.pb, nodes.p_nx, nodes.p_ny)
        self.H_lu = spla.splu(self.H) if viscous_solver == "lu" else None
        self.P_lu = spla.splu(self.Pb)
        self._HT_lu = None
        self._PT_lu = None

    @property
    def HT_lu(self):
        if self._HT_lu is None:
            self._HT_lu = spla.splu(self.H.T.tocsc())
        return self._HT_lu

    @property
    def PT_lu(self):
        if self._PT_lu is None:
            self._PT_lu = spla.splu(self.Pb.T.tocsc())
        return self._PT_lu

    def initial_state(self, u0=None, v0=None) -> FlowState:
        N, M = self.nodes.N, self.nodes.M
        u = np.zeros(N) if u0 is None else np.array(u0, np.float64)
        v = np.zeros(N) if v0 is None else np.array(v0, np.float64)
        return FlowState(u=u, v=v, cu_prev=np.zeros(N), cv_prev=np.zeros(N),
                         pt=np.zeros(M), p=np.zeros(M))

    def convection(self, u, v, qv):
        """C(q) = -[u o (D_x q) + v o (D_y q)] on the V-grid (Section 3, stage 1)."""
        return -(u * (self.ops.vv_x @ qv) + v * (self.ops.vv_y @ qv))

    def step(self, st: FlowState, gu, gv) -> FlowState:
        """Advance from step j to j+1.  gu, gv: boundary values g_{j+1} at
        every V-node (only the boundary entries are used)."""
        o, dt, a, vb = self.ops, self.dt, self.a, self.vb
        cu, cv, uss, vss, F = self.intermediate(st, gu, gv)
        if self.projection == "exact":
            sol = self.P_lu.solve(np.concatenate([F / dt, [0.0]]))
            phi, mu = sol[:-1], sol[-1]
            un = uss - dt * (self.G0x @ phi) - mu * dt * self.w_x
            vn = vss - dt * (self.G0y @ phi) - mu * dt * self.w_y
            pt = st.pt + phi
            p = pt - a * (o.pp_lap @ phi)
            return FlowState(u=un, v=vn, cu_prev=cu, cv_prev=cv, pt=pt, p=p,
                             lam=float(mu * dt), j=st.j + 1)
        # stage 3: pressure Poisson, pressure, correction
        b = np.where(self.pb, 0.0, F / dt)
        sol = self.P_lu.solve(np.concatenate([b, [0.0]]))
        pt, lam = sol[:-1], sol[-1]
        p = pt - a * (o.pp_lap @ pt)
        un = uss - dt * (o.vp_x @ pt)
        vn = vss - dt * (o.vp_y @ pt)
        if self.overwrite_bc:
            un[vb] = gu[vb]
            vn[vb] = gv[vb]
        return FlowState(u=un, v=vn, cu_prev=cu, cv_prev=cv, pt=pt, p=p,
                         lam=float(lam), j=st.j + 1)

    def intermediate(self, st: FlowState, gu, gv):
        """Stages 1-2 and the divergence of stage 3: C_j(u), C_j(v), u**, v**
        and F_{j+1} = D^(P,V)_x u** + D^(P,V)_y v** (Eq. divergence)."""
        o, dt, a, vb = self.ops, self.dt, self.a, self.vb
        # stage 1: Adams-Bashforth convection
        cu = self.convection(st.u, st.v, st.u)
        cv = self.convection(st.u, st.v, st.v)
        cu_prev = cu if st.j == 0 else st.cu_prev
        cv_prev = cv if st.j == 0 else st.cv_prev
        us = st.u + dt * (1.5 * cu - 0.5 * cu_prev)
        vs = st.v + dt * (1.5 * cv - 0.5 * cv_prev)
        # stage 2: Crank-Nicolson viscous step, Kim & Moin boundary values
        if self.cn_form == "printed":  # Eq. u_ss
            ru = us + a * (o.vv_lap @ us)
            rv = vs + a * (o.vv_lap @ vs)
        else:
            ru = us + a * (o.vv_lap @ st.u)
            rv = vs + a * (o.vv_lap @ st.v)
        if self.projection == "exact":  # pressure increment form, plain wall data
            ru -= dt * (self.G0x @ st.pt)
            rv -= dt * (self.G0y @ st.pt)
            ru[vb] = gu[vb]
            rv[vb] = gv[vb]
            uss = self.solve_viscous(ru)
            vss = self.solve_viscous(rv)
            return cu, cv, uss, vss, o.pv_x @ uss + o.pv_y @ vss
        # Kim & Moin: u** = u_{j+1} + dt D^(V,P) p~_j on the wall (R5)
        gpx = o.vp_x @ st.pt
        gpy = o.vp_y @ st.pt
        if self.km_mode == 1:  # the component along the wall tangent only
            gt = self.tx * gpx + self.ty * gpy
            gpx, gpy = gt * self.tx, gt * self.ty
        elif self.km_mode == 0:
            gpx, gpy = 0.0 * gpx, 0.0 * gpy
        ru[vb] = gu[vb] + dt * gpx[vb]
        rv[vb] = gv[vb] + dt * gpy[vb]
        uss = self.solve_viscous(ru)
        vss = self.solve_viscous(rv)
        F = o.pv_x @ uss + o.pv_y @ vss
        return cu, cv, uss, vss, F

    def solve_viscous(self, r):
        """(I - a D^(V,V)_Lap) x = r with identity wall rows (Eq. u_ss)."""
        if self.H_lu is not None:
            return self.H_lu.solve(r)
        x, info = spla.bicgstab(self.H, r, x0=r.copy(), rtol=1e-14, atol=0.0, maxiter=2000)
        if info != 0:
            raise RuntimeError(f"viscous BiCGSTAB did not converge (info {info})")
        return x


@dataclass
class AdjointState:
    """Adjoint variables of a FlowState: dJ/du, dJ/dv, dJ/dC_{j-1}(u),
    dJ/dC_{j-1}(v), dJ/dp~ (the pressure p is not fed back, so it has none)."""
    u: np.ndarray
    v: np.ndarray
    cu_prev: np.ndarray
    cv_prev: np.ndarray
    pt: np.ndarray


def adjoint_step(fs: "FractionalStep", st_in: FlowState, lam: AdjointState,
                 km_mode: int | None = None):
    """Reverse-mode derivative of one step of FractionalStep.step.

    st_in: the forward state the step started from (step j); lam: adjoints of
    the step's outputs.  Returns (adjoints of the inputs, dJ/dgu, dJ/dgv) where
    gu, gv are the wall data of the step.  Every transpose is the explicit
    transpose of the oracle's CSR matrix; the transposed solves use the LU
    factors of H^T and of the bordered matrix's transpose.
    """
    if fs.projection != "paper" or fs.cn_form != "printed":
        raise NotImplementedError("the adjoint follows the paper's step (Section 3) only")
    o, dt, a = fs.ops, fs.dt, fs.a
    km_mode = fs.km_mode if km_mode is None else km_mode
    w = fs.vb
    inner = ~w
    N = st_in.u.size
    lgu = np.zeros(N)
    lgv = np.zeros(N)
    lun = lam.u.copy()
    lvn = lam.v.copy()
    if fs.overwrite_bc:
        lgu[w] += lun[w]
        lgv[w] += lvn[w]
        lun[w] = 0.0
        lvn[w] = 0.0
    # correction u_{j+1} = u** - dt G_x p~
    luss = lun.copy()
    lvss = lvn.copy()
    lpt = lam.pt - dt * (o.vp_x.T @ lun + o.vp_y.T @ lvn)
    # pressure solve: [p~; lam] = B^-1 [b; 0], b = F/dt inside, 0 on boundary rows
    z = fs.PT_lu.solve(np.concatenate([lpt, [0.0]]))[:-1]
    lF = np.where(fs.pb, 0.0, z / dt)
    luss += o.pv_x.T @ lF
    lvss += o.pv_y.T @ lF
    # Crank-Nicolson solves u** = H^-1 r_u
    lru = fs.HT_lu.solve(luss)
    lrv = fs.HT_lu.solve(lvss)
    lgu[w] += lru[w]
    lgv[w] += lrv[w]
    lpt_in = np.zeros_like(lam.pt)
    if km_mode == 1:
        mu = np.where(w, fs.tx * lru + fs.ty * lrv, 0.0) * dt
        lpt_in += o.vp_x.T @ (fs.tx * mu) + o.vp_y.T @ (fs.ty * mu)
    elif km_mode == 2:
        lpt_in += dt * (o.vp_x.T @ np.where(w, lru, 0.0) + o.vp_y.T @ np.where(w, lrv, 0.0))
    lri = np.where(inner, lru, 0.0)
    lrvi = np.where(inner, lrv, 0.0)
    lus = lri + a * (o.vv_lap.T @ lri)
    lvs = lrvi + a * (o.vv_lap.T @ lrvi)
    # Adams-Bashforth combination u* = u + dt (3/2 C_j - 1/2 C_{j-1})
    lu = lus.copy()
    lv = lvs.copy()
    lcu = 1.5 * dt * lus + lam.cu_prev
    lcv = 1.5 * dt * lvs + lam.cv_prev
    if st_in.j == 0:
        lcu += -0.5 * dt * lus
        lcv += -0.5 * dt * lvs
        lcup = np.zeros(N)
        lcvp = np.zeros(N)
    else:
        lcup = -0.5 * dt * lus
        lcvp = -0.5 * dt * lvs
    # convection C(q) = -[u o D_x q + v o D_y q]
    u, v = st_in.u, st_in.v
    dxu, dyu = o.vv_x @ u, o.vv_y @ u
    dxv, dyv = o.vv_x @ v, o.vv_y @ v
    lu += -(dxu * lcu) - o.vv_x.T @ (u * lcu) - o.vv_y.T @ (v * lcu) - dxv * lcv
    lv += -(dyu * lcu) - dyv * lcv - o.vv_x.T @ (u * lcv) - o.vv_y.T @ (v * lcv)
    return AdjointState(u=lu, v=lv, cu_prev=lcup, cv_prev=lcvp, pt=lpt_in), lgu, lgv


def kinetic_energy(st: FlowState) -> float:
    """J = 1/2 sum over V-nodes of u^2 + v^2 (unweighted)."""
    return 0.5 * float(st.u @ st.u + st.v @ st.v)


def lid_bc(nodes, lid_u=1.0):
    """Cavity boundary data: u = lid_u on the top wall, u = v = 0 elsewhere
    (Section 5.1).  lid_u may be a scalar or a per-V-node array."""
    from paper_2206_06495_gb300.nodesets import WALL_TOP
    from_top = nodes.v_wall == WALL_TOP
    gu = np.zeros(nodes.N)
    gu[from_top] = (np.broadcast_to(lid_u, (nodes.N,)))[from_top]
    gv = np.zeros(nodes.N)
    return gu, gv


# --------------------------------------------------------------------------
# Open flows: the cylinder wake of Section 5.2
BC_INTERIOR = 0
BC_DIRICHLET = 1
BC_NEUMANN = 2


def wake_conditions(nodes, u_inf: float = 1.0):
    """Boundary conditions of the cylinder wake (Section 5.2) on a
    nodesets.cylinder_wake node set: uniform inflow u = u_inf, v = 0;
    symmetry sides v = 0, du/dn = 0; no slip on the cylinder; the stress-free
    outlet as du/dn = dv/dn = 0 and p~ = 0 (R17).  Returns bc_u, bc_v (per
    V-node), bc_p (per P-node) and the Dirichlet data gu, gv."""
    from paper_2206_06495_gb300.nodesets import (WALL_CYLINDER, WALL_INFLOW, WALL_OUTFLOW,
                                                 WALL_SIDE)
    vw, pw = nodes.v_wall, nodes.p_wall
    bc_u = np.zeros(nodes.N, np.int8)
    bc_v = np.zeros(nodes.N, np.int8)
    bc_p = np.zeros(nodes.M, np.int8)
    bc_u[(vw == WALL_INFLOW) | (vw == WALL_CYLINDER)] = BC_DIRICHLET
    bc_u[(vw == WALL_SIDE) | (vw == WALL_OUTFLOW)] = BC_NEUMANN
    bc_v[(vw == WALL_INFLOW) | (vw == WALL_CYLINDER) | (vw == WALL_SIDE)] = BC_DIRICHLET
    bc_v[vw == WALL_OUTFLOW] = BC_NEUMANN
    bc_p[(pw == WALL_INFLOW) | (pw == WALL_SIDE) | (pw == WALL_CYLINDER)] = BC_NEUMANN
    bc_p[pw == WALL_OUTFLOW] = BC_DIRICHLET
    # the outlet's two corner nodes take the side walls' Neumann row (R17)
    y0, y1 = nodes.meta["domain"][2], nodes.meta["domain"][3]
    bc_p[(pw == WALL_OUTFLOW) & ((nodes.py == y0) | (nodes.py == y1))] = BC_NEUMANN
    gu = np.where(vw == WALL_INFLOW, u_inf, 0.0)
    gv = np.zeros(nodes.N)
    return bc_u, bc_v, bc_p, gu, gv


def neumann_rows(nodes, rows, k: int = 28, m: int = 7, q: int = 3) -> sp.csr_matrix:
    """n_x D_x + n_y D_y at the boundary V-nodes `rows` on one-sided stencils
    (the node itself, then its k-1 nearest interior V-nodes; R17), as an
    N x N matrix with those rows only."""
    N = nodes.N
    rows = np.asarray(rows, np.int64)
    if rows.size == 0:
        return sp.csr_matrix((N, N))
    vx, vy = nodes.vx, nodes.vy
    idx = knn(vx[rows], vy[rows], vx, vy, k, beta_mask=~nodes.v_boundary, alpha_self=rows)
    _, w = build_weights(vx[rows], vy[rows], vx, vy, k, m, q, (OP_DX, OP_DY), idx=idx)
    vals = nodes.v_nx[rows, None] * w[OP_DX] + nodes.v_ny[rows, None] * w[OP_DY]
    return sp.csr_matrix((vals.ravel(), (np.repeat(rows, k), idx.ravel())), shape=(N, N))


class OpenFlowStep:
    """Section 3's fractional step with per-component boundary conditions
    (R17), for open flows such as the cylinder wake of Section 5.2.

    Viscous step, for each component c in (u, v): interior rows
    (I - a D_Lap) c** = RHS (printed Crank-Nicolson form, or Kim & Moin's
    with cn_form="kim_moin"); Dirichlet rows c** = g_{j+1} + dt D^(V,P)_c p~_j
    (Kim & Moin, R5; km_mode 0 drops the pressure term); Neumann rows
    n.grad c** = 0.  Pressure: interior rows D^(P,P)_Lap p~ = F/dt, Neumann
    rows n.grad p~ = 0 (R4's one-sided rows), Dirichlet rows p~ = 0; the
    system is nonsingular when any Dirichlet row is present.  Then
    p = p~ - a D^(P,P)_Lap p~ and c_{j+1} = c** - dt D^(V,P)_c p~, with
    Dirichlet components overwritten by g_{j+1}."""

    def __init__(self, nodes, Re: float, dt: float, bc_u, bc_v, bc_p, k: int = 28,
                 m: int = 7, q: int = 3, ops: Operators | None = None, km_mode: int = 2,
                 cn_form: str = "printed", convective=None, u_conv: float = 1.0):
        if km_mode not in (0, 1, 2):
            raise ValueError("km_mode is 0, 1 or 2")
        if cn_form not in ("printed", "kim_moin"):
            raise ValueError("cn_form is 'printed' or 'kim_moin'")
        self.nodes = nodes
        self.Re, self.dt = float(Re), float(dt)
        self.a = self.dt / (2.0 * self.Re)
        self.km_mode, self.cn_form = km_mode, cn_form
        self.bc_u = np.asarray(bc_u, np.int8)
        self.bc_v = np.asarray(bc_v, np.int8)
        self.bc_p = np.asarray(bc_p, np.int8)
        # convective outflow nodes: Dirichlet rows whose data follow
        # dc/dt + u_conv dc/dn = 0 (explicit, one-sided normal derivative)
        self.conv = (np.zeros(nodes.N, bool) if convective is None
                     else np.asarray(convective, bool))
        self.u_conv = float(u_conv)
        if (self.conv & ((self.bc_u != BC_DIRICHLET) | (self.bc_v != BC_DIRICHLET))).any():
            raise ValueError("convective outflow nodes carry Dirichlet rows")
        if not (nodes.v_boundary[self.bc_u != BC_INTERIOR].all()
                and nodes.v_boundary[self.bc_v != BC_INTERIOR].all()
                and nodes.p_boundary[self.bc_p != BC_INTERIOR].all()):
            raise ValueError("boundary conditions on interior nodes")
        if (nodes.v_boundary & ((self.bc_u == BC_INTERIOR) | (self.bc_v == BC_INTERIOR))).any():
            raise ValueError("a boundary V-node without a condition")
        self.ops = ops if ops is not None else build_operators(nodes, k, m, q)
        o, N, M = self.ops, nodes.N, nodes.M
        nrows = np.nonzero((self.bc_u == BC_NEUMANN) | (self.bc_v == BC_NEUMANN)
                           | self.conv)[0]
        self.VN = neumann_rows(nodes, nrows, k, m, q)
        self.H_u = self._viscous_matrix(self.bc_u)
        self.H_v = self._viscous_matrix(self.bc_v)
        inn = sp.diags((self.bc_p == BC_INTERIOR).astype(float))
        neu = sp.diags((self.bc_p == BC_NEUMANN).astype(float))
        dirichlet = sp.diags((self.bc_p == BC_DIRICHLET).astype(float))
        self.L = (inn @ o.pp_lap
                  + neu @ (sp.diags(nodes.p_nx) @ o.pn_x + sp.diags(nodes.p_ny) @ o.pn_y)
                  + dirichlet).tocsc()
        self.Hu_lu = spla.splu(self.H_u)
        self.Hv_lu = spla.splu(self.H_v)
        self.L_lu = spla.splu(self.L)

    def _viscous_matrix(self, bc):
        N = self.nodes.N
        inn = sp.diags((bc == BC_INTERIOR).astype(float))
        dirichlet = sp.diags((bc == BC_DIRICHLET).astype(float))
        neu = sp.diags((bc == BC_NEUMANN).astype(float))
        return (inn @ (sp.identity(N) - self.a * self.ops.vv_lap) + dirichlet
                + neu @ self.VN).tocsc()

    def initial_state(self, u0=None, v0=None) -> FlowState:
        N, M = self.nodes.N, self.nodes.M
        u = np.zeros(N) if u0 is None else np.array(u0, np.float64)
        v = np.zeros(N) if v0 is None else np.array(v0, np.float64)
        return FlowState(u=u, v=v, cu_prev=np.zeros(N), cv_prev=np.zeros(N),
                         pt=np.zeros(M), p=np.zeros(M))

    def step(self, st: FlowState, gu, gv) -> FlowState:
        o, dt, a = self.ops, self.dt, self.a
        cu = -(st.u * (o.vv_x @ st.u) + st.v * (o.vv_y @ st.u))
        cv = -(st.u * (o.vv_x @ st.v) + st.v * (o.vv_y @ st.v))
        cu_prev = cu if st.j == 0 else st.cu_prev
        cv_prev = cv if st.j == 0 else st.cv_prev
        us = st.u + dt * (1.5 * cu - 0.5 * cu_prev)
        vs = st.v + dt * (1.5 * cv - 0.5 * cv_prev)
        if self.cn_form == "printed":
            ru = us + a * (o.vv_lap @ us)
            rv = vs + a * (o.vv_lap @ vs)
        else:
            ru = us + a * (o.vv_lap @ st.u)
            rv = vs + a * (o.vv_lap @ st.v)
        kp = 0.0 if self.km_mode == 0 else 1.0
        gpx = kp * (o.vp_x @ st.pt)
        gpy = kp * (o.vp_y @ st.pt)
        if self.km_mode == 1:  # the component along the wall tangent only (R5)
            tx, ty = -self.nodes.v_ny, self.nodes.v_nx
            gt = tx * gpx + ty * gpy
            gpx, gpy = gt * tx, gt * ty
        du, dv = self.bc_u == BC_DIRICHLET, self.bc_v == BC_DIRICHLET
        if self.conv.any():  # outflow data from the convective condition
            cvn = self.conv
            gu = np.where(cvn, st.u - dt * self.u_conv * (self.VN @ st.u), gu)
            gv = np.where(cvn, st.v - dt * self.u_conv * (self.VN @ st.v), gv)
        ru[du] = gu[du] + dt * gpx[du]
        rv[dv] = gv[dv] + dt * gpy[dv]
        ru[self.bc_u == BC_NEUMANN] = 0.0
        rv[self.bc_v == BC_NEUMANN] = 0.0
        uss = self.Hu_lu.solve(ru)
        vss = self.Hv_lu.solve(rv)
        F = o.pv_x @ uss + o.pv_y @ vss
        b = np.where(self.bc_p == BC_INTERIOR, F / dt, 0.0)
        pt = self.L_lu.solve(b)
        p = pt - a * (o.pp_lap @ pt)
        un = uss - dt * (o.vp_x @ pt)
        vn = vss - dt * (o.vp_y @ pt)
        un[du] = gu[du]
        vn[dv] = gv[dv]
        return FlowState(u=un, v=vn, cu_prev=cu, cv_prev=cv, pt=pt, p=p, lam=0.0, j=st.j + 1)


def simpson_periodic(f, period: float) -> float:
    """Composite Simpson's rule for a periodic function sampled at an even
    number n of equally spaced points f_0 .. f_{n-1} over one period (f_n =
    f_0): h/3 (2 f_0 + 4 f_1 + 2 f_2 + ... + 4 f_{n-1})."""
    f = np.asarray(f, np.float64)
    n = f.size
    if n < 2 or n % 2:
        raise ValueError("Simpson's rule needs an even number of intervals")
    w = np.where(np.arange(n) % 2 == 1, 4.0, 2.0)
    return float((period / n) / 3.0 * (w @ f))


def cylinder_forces(nodes, ops: Operators, u, v, p, Re: float):
    """Drag and lift coefficients (Section 5.2): the force of the fluid on
    the cylinder, F = integral over the surface of sigma n, with
    sigma = -p I + (grad U + grad U^T) / Re and n the unit normal pointing
    from the cylinder into the fluid, by Simpson's rule in the angle over the
    cylinder's P-nodes (equally spaced in angle, an even count), with the
    velocity gradient taken there by D^(P,V); C = F / (1/2 rho U^2 D) with
    rho = U = 1 and D = 2 radius.  Returns (C_D, C_L)."""
    from paper_2206_06495_gb300.nodesets import WALL_CYLINDER
    cyl = np.nonzero(nodes.p_wall == WALL_CYLINDER)[0]
    x, y = nodes.px[cyl], nodes.py[cyl]
    th = np.mod(np.arctan2(y, x), 2.0 * np.pi)
    order = np.argsort(th)
    cyl, x, y, th = cyl[order], x[order], y[order], th[order]
    radius = float(np.mean(np.hypot(x, y)))
    nx, ny = np.cos(th), np.sin(th)
    ux, uy = (ops.pv_x @ u)[cyl], (ops.pv_y @ u)[cyl]
    vx, vy = (ops.pv_x @ v)[cyl], (ops.pv_y @ v)[cyl]
    pc = np.asarray(p)[cyl]
    tx = -pc * nx + (2.0 * ux * nx + (uy + vx) * ny) / Re
    ty = -pc * ny + ((uy + vx) * nx + 2.0 * vy * ny) / Re
    fx = simpson_periodic(tx * radius, 2.0 * np.pi)
    fy = simpson_periodic(ty * radius, 2.0 * np.pi)
    d = 2.0 * radius
    return 2.0 * fx / d, 2.0 * fy / d


def strouhal(t, cl, diameter: float = 1.0, u_inf: float = 1.0) -> float:
    """St = f D / U of a lift signal: f from the mean spacing of the upward
    zero crossings of cl - mean(cl), located by linear interpolation."""
    t = np.asarray(t, np.float64)
    c = np.asarray(cl, np.float64) - np.mean(cl)
    up = np.nonzero((c[:-1] < 0.0) & (c[1:] >= 0.0))[0]
    if up.size < 2:
        raise ValueError("fewer than two upward zero crossings")
    tc = t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])
    period = (tc[-1] - tc[0]) / (tc.size - 1)
    return diameter / (period * u_inf)
