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
