"""Seeded synthetic node sets shaped like the paper's workloads.

This module is the one piece shared by the CUDA path, the CPU oracle, the
tests and the benchmark.  It only places points and tags boundaries; it holds
none of the method's arithmetic (no RBF, no weights, no operators, no time
stepping).

Layouts follow Section 3 of the paper: the pressure nodes (P-grid) are the
vertices of a triangular mesh and the velocity nodes (V-grid) are the
midpoints of its edges, so N/M is about 3.  The paper meshes with DistMesh;
here the triangulation is a jittered Cartesian lattice with one seeded
diagonal per cell, which gives the same vertex/edge-midpoint structure.

All node sets are returned in Morton (Z-curve) order so that the k nearest
neighbours of a node sit close to it in memory.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Wall tags for boundary V-nodes and P-nodes of the unit-square cavity.
WALL_NONE = 0
WALL_BOTTOM = 1
WALL_RIGHT = 2
WALL_TOP = 3  # the moving lid (Section 5.1)
WALL_LEFT = 4
WALL_CORNER = 5
# Boundary tags of the open cylinder-wake domain (Section 5.2).
WALL_INFLOW = 6    # x = x0: uniform inflow
WALL_OUTFLOW = 7   # x = x1: stress-free outlet
WALL_SIDE = 8      # y = y0 and y = y1: symmetry (slip) walls
WALL_CYLINDER = 9  # the cylinder surface


def morton_order(x: np.ndarray, y: np.ndarray, bits: int = 20) -> np.ndarray:
    """Permutation that sorts points along a Z-order curve of their bounding box."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.size == 0:
        return np.zeros(0, np.int64)
    lo_x, hi_x = x.min(), x.max()
    lo_y, hi_y = y.min(), y.max()
    span = max(hi_x - lo_x, hi_y - lo_y, 1e-300)
    scale = (1 << bits) - 1
    qx = np.clip(((x - lo_x) / span * scale).astype(np.int64), 0, scale).astype(np.uint64)
    qy = np.clip(((y - lo_y) / span * scale).astype(np.int64), 0, scale).astype(np.uint64)

    def spread(v):
        v = v & np.uint64(0x00000000FFFFFFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
        return v

    code = spread(qx) | (spread(qy) << np.uint64(1))
    return np.argsort(code, kind="stable")


@dataclass
class StaggeredNodes:
    """A staggered P/V node pair with boundary tags.

    px, py      P-node coordinates, float64 [M]
    p_wall      wall tag per P-node (WALL_*), int8 [M]; nonzero = boundary
    p_nx, p_ny  outward unit normal at boundary P-nodes (corners: bisector), 0 inside
    vx, vy      V-node coordinates (edge midpoints), float64 [N]
    v_wall      wall tag per V-node, int8 [N]; nonzero = node lies on a wall
    v_nx, v_ny  outward unit normal of the wall at boundary V-nodes, 0 inside
    edges       the two P-node endpoints of the edge each V-node sits on, int64 [N, 2]
    h           nominal lattice spacing
    """

    px: np.ndarray
    py: np.ndarray
    p_wall: np.ndarray
    p_nx: np.ndarray
    p_ny: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    v_wall: np.ndarray
    v_nx: np.ndarray
    v_ny: np.ndarray
    edges: np.ndarray
    h: float
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.px.size)

    @property
    def N(self) -> int:
        return int(self.vx.size)

    @property
    def p_boundary(self) -> np.ndarray:
        return self.p_wall != WALL_NONE

    @property
    def v_boundary(self) -> np.ndarray:
        return self.v_wall != WALL_NONE


def jittered_cavity(n: int, seed: int = 0, jitter: float = 0.25,
                    length: float = 1.0) -> StaggeredNodes:
    """Staggered nodes for a square cavity [0, length]^2.

    P-nodes: an n x n lattice (spacing h = length/(n-1)) jittered by
    U(-jitter*h, +jitter*h); wall nodes move only along their wall and the
    four corners stay fixed.  Each lattice cell is cut into two triangles by
    one diagonal whose direction is drawn per cell.  V-nodes: the midpoints of
    all triangle edges; a V-node is a wall node when both endpoints of its
    edge lie on the same wall, so it sits exactly on that wall.
    """
    if n < 3:
        raise ValueError("need at least a 3 x 3 lattice")
    rng = np.random.default_rng(seed)
    h = length / (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    x = ii * h
    y = jj * h
    dx = rng.uniform(-jitter * h, jitter * h, ii.size)
    dy = rng.uniform(-jitter * h, jitter * h, ii.size)
    on_left = ii == 0
    on_right = ii == n - 1
    on_bottom = jj == 0
    on_top = jj == n - 1
    on_x_wall = on_left | on_right
    on_y_wall = on_bottom | on_top
    dx = np.where(on_x_wall, 0.0, dx)  # vertical walls: move along y only
    dy = np.where(on_y_wall, 0.0, dy)  # horizontal walls: move along x only
    x = x + dx
    y = y + dy
    # wall coordinates exactly on the walls, whatever (n-1)*h rounds to
    x[on_left] = 0.0
    x[on_right] = length
    y[on_bottom] = 0.0
    y[on_top] = length
    corner = on_x_wall & on_y_wall
    wall = np.zeros(ii.size, np.int8)
    wall[on_bottom] = WALL_BOTTOM
    wall[on_top] = WALL_TOP
    wall[on_left] = WALL_LEFT
    wall[on_right] = WALL_RIGHT
    wall[corner] = WALL_CORNER
    nx = np.zeros(ii.size)
    ny = np.zeros(ii.size)
    nx[on_left] = -1.0
    nx[on_right] = 1.0
    ny[on_bottom] = -1.0
    ny[on_top] = 1.0
    nrm = np.hypot(nx, ny)
    nz = nrm > 0
    nx[nz] /= nrm[nz]
    ny[nz] /= nrm[nz]

    lin = lambda a, b: a * n + b  # noqa: E731  lattice (i, j) -> flat id
    ci, cj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    ci = ci.ravel()
    cj = cj.ravel()
    # horizontal edges along every lattice row, including the top row
    hi_, hj_ = np.meshgrid(np.arange(n - 1), np.arange(n), indexing="ij")
    horiz = np.stack([lin(hi_.ravel(), hj_.ravel()), lin(hi_.ravel() + 1, hj_.ravel())], 1)
    vi_, vj_ = np.meshgrid(np.arange(n), np.arange(n - 1), indexing="ij")
    vert = np.stack([lin(vi_.ravel(), vj_.ravel()), lin(vi_.ravel(), vj_.ravel() + 1)], 1)
    flip = rng.integers(0, 2, ci.size).astype(bool)
    diag = np.where(flip[:, None],
                    np.stack([lin(ci + 1, cj), lin(ci, cj + 1)], 1),
                    np.stack([lin(ci, cj), lin(ci + 1, cj + 1)], 1))
    edges = np.concatenate([horiz, vert, diag], 0).astype(np.int64)

    # Morton-order the P-nodes and relabel the edge endpoints.
    perm = morton_order(x, y)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    x, y, wall, nx, ny = x[perm], y[perm], wall[perm], nx[perm], ny[perm]
    edges = inv[edges]
    edges.sort(axis=1)

    a, b = edges[:, 0], edges[:, 1]
    vx = 0.5 * (x[a] + x[b])
    vy = 0.5 * (y[a] + y[b])

    v_wall = np.zeros(edges.shape[0], np.int8)
    ya, yb = y[a], y[b]
    xa, xb = x[a], x[b]
    lo, hi = 0.0, length
    both_bottom = (ya == lo) & (yb == lo)
    both_top = (ya == hi) & (yb == hi)
    both_left = (xa == lo) & (xb == lo)
    both_right = (xa == hi) & (xb == hi)
    v_wall[both_bottom] = WALL_BOTTOM
    v_wall[both_right] = WALL_RIGHT
    v_wall[both_top] = WALL_TOP
    v_wall[both_left] = WALL_LEFT

    v_nx = np.zeros(edges.shape[0])
    v_ny = np.zeros(edges.shape[0])
    v_ny[both_bottom] = -1.0
    v_nx[both_right] = 1.0
    v_ny[both_top] = 1.0
    v_nx[both_left] = -1.0

    vperm = morton_order(vx, vy)
    vx, vy, v_wall, edges = vx[vperm], vy[vperm], v_wall[vperm], edges[vperm]
    v_nx, v_ny = v_nx[vperm], v_ny[vperm]
    return StaggeredNodes(px=x, py=y, p_wall=wall, p_nx=nx, p_ny=ny,
                          vx=vx, vy=vy, v_wall=v_wall, v_nx=v_nx, v_ny=v_ny,
                          edges=edges, h=h,
                          meta={"kind": "jittered_cavity", "n": n, "seed": seed,
                                "jitter": jitter, "length": length})


def wake_spacing(x, y, h_wall: float, h_wake: float, h_far: float, radius: float,
                 growth: float):
    """Target node spacing of the cylinder-wake layout: h_wall on the cylinder,
    growing by `growth` per unit distance from it; h_wake on the wake
    centreline (x > 0), growing by `growth` per unit |y| and by 3 % per unit x;
    never above h_far."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    r = np.hypot(x, y)
    h_c = h_wall + growth * np.maximum(r - radius, 0.0)
    h_w = np.where(x > 0.0, h_wake * (1.0 + 0.03 * x) + growth * np.abs(y), np.inf)
    return np.minimum(np.minimum(h_c, h_w), h_far)


def _edge_nodes(a, b, hfun):
    """Points from a to b (both included) spaced by the local target spacing,
    stretched uniformly so that the last one lands on b."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    length = float(np.hypot(*(b - a)))
    s = [0.0]
    while s[-1] < length:
        q = a + (b - a) * (s[-1] / length)
        s.append(s[-1] + float(hfun(q[0:1], q[1:2])[0]))
    s = np.array(s)
    if s.size > 2 and s[-1] - length > 0.5 * (s[-1] - s[-2]):
        s = s[:-1]  # the last step overshoots by more than half: drop it
    t = s / s[-1]  # graded positions, stretched so the last lands on b
    t[-1] = 1.0
    return a[0] + (b[0] - a[0]) * t, a[1] + (b[1] - a[1]) * t


def cylinder_wake(h_wall: float = 0.03, h_wake: float = 0.04, h_far: float = 0.3,
                  x0: float = -8.0, x1: float = 24.0, y0: float = -8.0, y1: float = 8.0,
                  radius: float = 0.5, growth: float = 0.14, seed: int = 3,
                  jitter: float = 0.25, rings: int = 6) -> StaggeredNodes:
    """Staggered nodes for flow past a cylinder (Section 5.2): the rectangle
    [x0, x1] x [y0, y1] outside the circle of `radius` about the origin
    (radius 0: no cylinder, a plain channel), graded by wake_spacing.

    P-nodes: boundary nodes on the circle (an even count, uniform in angle,
    the first at angle 0) and on the four sides (spaced by the local target
    spacing, corners included once); `rings` layers of nodes on circles
    about the cylinder, each sqrt(3)/2 of the local spacing further out,
    uniform in angle at the local spacing and turned by half a spacing from
    the layer below (near-equilateral triangles along the curved wall);
    outside them, one node per leaf of a quadtree refined until each leaf is
    no larger than the target spacing at its centre, placed at the leaf
    centre jittered by U(+-jitter * leaf side), and dropped where it comes
    closer than 0.6 of the local spacing to a boundary or to the last ring.  The P-nodes are triangulated (Delaunay, with a ring of
    ghost points outside the rectangle so that the sides stay straight;
    triangles inside the cylinder, touching a ghost, or joining two
    non-adjacent circle nodes are dropped).  V-nodes: the midpoints of the
    triangle edges.  A node on x = x0 is an inflow node (corners too), on
    x = x1 an outflow node (corners too), on y = y0 or y1 a side node, on the
    circle a cylinder node; a V-node is a boundary node when both endpoints of
    its edge lie on the same boundary.  Normals point out of the fluid (into
    the cylinder on its surface)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)

    def hfun(x, y):
        return wake_spacing(x, y, h_wall, h_wake, h_far, radius, growth)

    # boundary P-nodes
    bx, by, btag = [], [], []
    nc = 0
    if radius > 0.0:
        nc = max(8, 4 * int(round(2.0 * np.pi * radius / h_wall / 4.0)))
        th = 2.0 * np.pi * np.arange(nc) / nc
        bx.append(radius * np.cos(th))
        by.append(radius * np.sin(th))
        btag.append(np.full(nc, WALL_CYLINDER, np.int8))
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    for c in range(4):
        a, b = corners[c], corners[(c + 1) % 4]
        ex, ey = _edge_nodes(a, b, hfun)
        ex, ey = ex[:-1], ey[:-1]  # each corner once, as the start of its side
        tag = np.full(ex.size, WALL_SIDE, np.int8)
        tag[ex == x0] = WALL_INFLOW
        tag[ex == x1] = WALL_OUTFLOW
        bx.append(ex)
        by.append(ey)
        btag.append(tag)
    bx = np.concatenate(bx)
    by = np.concatenate(by)
    btag = np.concatenate(btag)

    # interior P-nodes: quadtree leaves no larger than the local spacing
    n0x = int(np.ceil((x1 - x0) / h_far))
    n0y = int(np.ceil((y1 - y0) / h_far))
    sx0, sy0 = (x1 - x0) / n0x, (y1 - y0) / n0y
    gx, gy = np.meshgrid(np.arange(n0x), np.arange(n0y), indexing="ij")
    cx = x0 + (gx.ravel() + 0.5) * sx0
    cy = y0 + (gy.ravel() + 0.5) * sy0
    sx = np.full(cx.size, sx0)
    sy = np.full(cy.size, sy0)
    leaves_x, leaves_y, leaves_sx, leaves_sy = [], [], [], []
    while cx.size:
        split = np.maximum(sx, sy) > hfun(cx, cy)
        leaves_x.append(cx[~split])
        leaves_y.append(cy[~split])
        leaves_sx.append(sx[~split])
        leaves_sy.append(sy[~split])
        cx, cy, sx, sy = cx[split], cy[split], sx[split] / 2, sy[split] / 2
        cx = np.concatenate([cx - sx / 2, cx + sx / 2, cx - sx / 2, cx + sx / 2])
        cy = np.concatenate([cy - sy / 2, cy - sy / 2, cy + sy / 2, cy + sy / 2])
        sx = np.tile(sx, 4)
        sy = np.tile(sy, 4)
    lx = np.concatenate(leaves_x)
    ly = np.concatenate(leaves_y)
    lsx = np.concatenate(leaves_sx)
    lsy = np.concatenate(leaves_sy)
    ix = lx + rng.uniform(-jitter, jitter, lx.size) * lsx
    iy = ly + rng.uniform(-jitter, jitter, ly.size) * lsy
    # ring layers about the cylinder
    rx, ry = [], []
    r_last = radius
    if radius > 0.0:
        n_prev = nc
        for layer in range(1, rings + 1):
            h_r = float(hfun(np.array([r_last]), np.array([0.0]))[0])
            r_k = r_last + 0.5 * np.sqrt(3.0) * h_r
            n_k = max(n_prev, 2 * int(round(np.pi * r_k / h_r)))
            th = 2.0 * np.pi * (np.arange(n_k) + 0.5 * (layer % 2)) / n_k
            px_k, py_k = r_k * np.cos(th), r_k * np.sin(th)
            ok = (px_k > x0) & (px_k < x1) & (py_k > y0) & (py_k < y1)
            rx.append(px_k[ok])
            ry.append(py_k[ok])
            r_last, n_prev = r_k, n_k
    rx = np.concatenate(rx) if rx else np.zeros(0)
    ry = np.concatenate(ry) if ry else np.zeros(0)
    hloc = hfun(ix, iy)
    # the margin takes the larger of the node's own spacing and the boundary
    # spacing at its projection, so no node enters the diametral circle of a
    # boundary segment (which would cut that segment out of the mesh)
    keep = (ix - x0 > 0.6 * np.maximum(hloc, hfun(np.full_like(iy, x0), iy))) & \
        (x1 - ix > 0.6 * np.maximum(hloc, hfun(np.full_like(iy, x1), iy))) & \
        (iy - y0 > 0.6 * np.maximum(hloc, hfun(ix, np.full_like(ix, y0)))) & \
        (y1 - iy > 0.6 * np.maximum(hloc, hfun(ix, np.full_like(ix, y1))))
    if radius > 0.0:
        r_i = np.maximum(np.hypot(ix, iy), 1e-300)
        h_proj = hfun(r_last * ix / r_i, r_last * iy / r_i)
        keep &= r_i - r_last > 0.6 * np.maximum(hloc, h_proj)
    ix, iy = np.concatenate([rx, ix[keep]]), np.concatenate([ry, iy[keep]])

    x = np.concatenate([bx, ix])
    y = np.concatenate([by, iy])
    wall = np.concatenate([btag, np.zeros(ix.size, np.int8)])
    nb = bx.size

    # ghost ring outside the rectangle, then Delaunay
    side = btag != WALL_CYLINDER
    hb = hfun(bx[side], by[side])
    gxs = np.clip(bx[side], x0, x1) + np.where(bx[side] == x0, -hb, np.where(bx[side] == x1, hb, 0))
    gys = np.clip(by[side], y0, y1) + np.where(by[side] == y0, -hb, np.where(by[side] == y1, hb, 0))
    ghost_x = np.concatenate([gxs, [x0 - h_far, x1 + h_far, x1 + h_far, x0 - h_far]])
    ghost_y = np.concatenate([gys, [y0 - h_far, y0 - h_far, y1 + h_far, y1 + h_far]])
    allx = np.concatenate([x, ghost_x])
    ally = np.concatenate([y, ghost_y])
    tri = Delaunay(np.stack([allx, ally], 1)).simplices
    n_real = x.size
    ok = (tri < n_real).all(1)
    tri = tri[ok]
    if radius > 0.0:
        cxm = x[tri].mean(1)
        cym = y[tri].mean(1)
        ok = np.hypot(cxm, cym) >= radius
        for e0, e1 in ((0, 1), (1, 2), (2, 0)):
            a_, b_ = tri[:, e0], tri[:, e1]
            both = (a_ < nc) & (b_ < nc)
            gap = np.abs(a_ - b_)
            ok &= ~(both & (gap != 1) & (gap != nc - 1))
        tri = tri[ok]
    used = np.zeros(n_real, bool)
    used[tri.ravel()] = True
    if not used[:nb].all():
        raise ValueError("a boundary node was left out of the triangulation")
    remap = -np.ones(n_real, np.int64)
    remap[used] = np.arange(used.sum())
    x, y, wall = x[used], y[used], wall[used]
    tri = remap[tri]
    edges = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 0)
    edges.sort(axis=1)
    edges = np.unique(edges, axis=0)

    nx = np.zeros(x.size)
    ny = np.zeros(x.size)
    nx[wall == WALL_INFLOW] = -1.0
    nx[wall == WALL_OUTFLOW] = 1.0
    sd = wall == WALL_SIDE
    ny[sd] = np.where(y[sd] == y0, -1.0, 1.0)
    cyl = wall == WALL_CYLINDER
    if radius > 0.0:
        nx[cyl] = -x[cyl] / radius
        ny[cyl] = -y[cyl] / radius

    perm = morton_order(x, y)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    x, y, wall, nx, ny = x[perm], y[perm], wall[perm], nx[perm], ny[perm]
    edges = inv[edges]
    edges.sort(axis=1)

    a, b = edges[:, 0], edges[:, 1]
    vx = 0.5 * (x[a] + x[b])
    vy = 0.5 * (y[a] + y[b])
    wa, wb = wall[a], wall[b]
    v_wall = np.zeros(edges.shape[0], np.int8)
    on_in = (x[a] == x0) & (x[b] == x0)
    on_out = (x[a] == x1) & (x[b] == x1)
    on_side = ((y[a] == y0) & (y[b] == y0)) | ((y[a] == y1) & (y[b] == y1))
    on_cyl = (wa == WALL_CYLINDER) & (wb == WALL_CYLINDER)
    v_wall[on_side] = WALL_SIDE
    v_wall[on_in] = WALL_INFLOW
    v_wall[on_out] = WALL_OUTFLOW
    v_wall[on_cyl] = WALL_CYLINDER
    v_nx = np.zeros(edges.shape[0])
    v_ny = np.zeros(edges.shape[0])
    v_nx[on_in] = -1.0
    v_nx[on_out] = 1.0
    v_ny[on_side] = np.where(vy[on_side] == y0, -1.0, 1.0)
    if radius > 0.0:
        rv = np.hypot(vx[on_cyl], vy[on_cyl])
        v_nx[on_cyl] = -vx[on_cyl] / rv
        v_ny[on_cyl] = -vy[on_cyl] / rv

    # every boundary segment is an edge: a closed boundary of k nodes has k
    # segments, each open side of k nodes k - 1
    n_bseg = int((v_wall != WALL_NONE).sum())
    n_side = [int(((x == x0)).sum()), int(((x == x1)).sum()), int(((y == y0)).sum()),
              int(((y == y1)).sum())]
    if n_bseg != sum(n_side) - 4 + nc:
        raise ValueError("a boundary segment is missing from the triangulation")

    vperm = morton_order(vx, vy)
    vx, vy, v_wall, edges = vx[vperm], vy[vperm], v_wall[vperm], edges[vperm]
    v_nx, v_ny = v_nx[vperm], v_ny[vperm]
    return StaggeredNodes(px=x, py=y, p_wall=wall, p_nx=nx, p_ny=ny,
                          vx=vx, vy=vy, v_wall=v_wall, v_nx=v_nx, v_ny=v_ny,
                          edges=edges, h=h_wall,
                          meta={"kind": "cylinder_wake", "radius": radius,
                                "domain": (x0, x1, y0, y1), "h_wall": h_wall,
                                "h_wake": h_wake, "h_far": h_far, "growth": growth,
                                "seed": seed, "n_cylinder": nc})


def poisson_disk(count: int, seed: int = 1, rounds: int = 24) -> tuple[np.ndarray, np.ndarray]:
    """`count` blue-noise points in [0,1]^2 with a minimum spacing (Poisson disk).

    Parallel dart throwing on a background grid of cell side r/sqrt(2), so a
    cell holds at most one point.  Cells are visited in 9 phases (i mod 3,
    j mod 3); cells of one phase are at least two cell sides apart, so the
    darts of one phase cannot conflict with each other and each phase is one
    vectorised step.  The radius is chosen so that a bit more than `count`
    points are placed; a seeded subset of exactly `count` is returned, in
    Morton order.
    """
    rng = np.random.default_rng(seed)
    # maximal Poisson-disk sets in 2-D reach a density of about 0.70 / r^2
    r = np.sqrt(0.66 / (count * 1.04))
    while True:
        cell = r / np.sqrt(2.0)
        g = int(np.ceil(1.0 / cell))
        occ = -np.ones((g + 4, g + 4), np.int64)  # padded by 2 cells
        n_pts = 0
        gi, gj = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
        gi = gi.ravel()
        gj = gj.ravel()
        allx = np.zeros(0)
        ally = np.zeros(0)
        for _ in range(rounds):
            for phase in range(9):
                sel = ((gi % 3) == phase // 3) & ((gj % 3) == phase % 3)
                ci, cj = gi[sel], gj[sel]
                empty = occ[ci + 2, cj + 2] < 0
                ci, cj = ci[empty], cj[empty]
                if ci.size == 0:
                    continue
                cx = (ci + rng.random(ci.size)) * cell
                cy = (cj + rng.random(cj.size)) * cell
                inside = (cx < 1.0) & (cy < 1.0)
                ci, cj, cx, cy = ci[inside], cj[inside], cx[inside], cy[inside]
                ok = np.ones(ci.size, bool)
                for di in range(-2, 3):
                    for dj in range(-2, 3):
                        nb = occ[ci + 2 + di, cj + 2 + dj]
                        has = nb >= 0
                        if not has.any():
                            continue
                        d2 = np.full(ci.size, np.inf)
                        d2[has] = (allx[nb[has]] - cx[has]) ** 2 + (ally[nb[has]] - cy[has]) ** 2
                        ok &= d2 >= r * r
                ci, cj, cx, cy = ci[ok], cj[ok], cx[ok], cy[ok]
                ids = n_pts + np.arange(ci.size)
                occ[ci + 2, cj + 2] = ids
                allx = np.concatenate([allx, cx])
                ally = np.concatenate([ally, cy])
                n_pts += ci.size
        if n_pts >= count:
            break
        r *= 0.97
    keep = np.sort(rng.choice(n_pts, count, replace=False))
    px, py = allx[keep], ally[keep]
    perm = morton_order(px, py)
    return px[perm], py[perm]


def wave_test_function(x: np.ndarray, y: np.ndarray):
    """f = sin(8 pi x + 4 pi y) cos(6 pi y) and its exact x-, y-derivatives and Laplacian.

    This is the input field of the 1M-node operator workload; the derivatives
    are the analytic values the discrete operators are measured against.
    """
    a = 8 * np.pi * x + 4 * np.pi * y
    b = 6 * np.pi * y
    f = np.sin(a) * np.cos(b)
    fx = 8 * np.pi * np.cos(a) * np.cos(b)
    fy = 4 * np.pi * np.cos(a) * np.cos(b) - 6 * np.pi * np.sin(a) * np.sin(b)
    lap = -(64 + 16 + 36) * np.pi ** 2 * np.sin(a) * np.cos(b) \
        - 2 * (4 * np.pi) * (6 * np.pi) * np.cos(a) * np.sin(b)
    return f, fx, fy, lap
