"""Flow past a cylinder (Section 5.2) on the GPU: the flow description of a
nodesets.cylinder_wake node set, its wall data, and the quantities the paper
reports (drag and lift coefficients, Strouhal number).

Boundary conditions, per component: uniform inflow u = u_inf, v = 0
(Dirichlet); symmetry sides v = 0 (Dirichlet), du/dn = 0 (Neumann); no slip on
the cylinder (Dirichlet); the stress-free outlet as du/dn = dv/dn = 0
(Neumann) with p~ = 0 (Dirichlet pressure rows), the outlet's two corner
P-nodes keeping the sides' Neumann pressure row.  Neumann velocity rows use
one-sided stencils (the node, then its nearest interior V-nodes), as the
Neumann pressure rows do.  Everything here prepares arguments for the C ABI or
post-processes its scalar results; the step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import nodesets as ns
from . import rbffd as R


def wake_flow(ctx: R.Context, nodes, Re: float, dt: float, device="cuda", **kw) -> R.Flow:
    """rbffd_flow of a cylinder_wake node set with the boundary conditions of
    Section 5.2 (see the module docstring)."""
    import torch
    if nodes.meta.get("kind") != "cylinder_wake":
        raise ValueError("wake_flow needs a nodesets.cylinder_wake node set")
    flow = R.flow_from_nodes(ctx, nodes, Re=Re, dt=dt, device=device, **kw)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)  # noqa: E731
    vw, pw = nodes.v_wall, nodes.p_wall
    bcu = np.zeros(nodes.N, np.uint8)
    bcv = np.zeros(nodes.N, np.uint8)
    bcu[(vw == ns.WALL_INFLOW) | (vw == ns.WALL_CYLINDER)] = R.BC_DIRICHLET
    bcu[(vw == ns.WALL_SIDE) | (vw == ns.WALL_OUTFLOW)] = R.BC_NEUMANN
    bcv[(vw == ns.WALL_INFLOW) | (vw == ns.WALL_CYLINDER) | (vw == ns.WALL_SIDE)] = R.BC_DIRICHLET
    bcv[vw == ns.WALL_OUTFLOW] = R.BC_NEUMANN
    y0, y1 = nodes.meta["domain"][2], nodes.meta["domain"][3]
    pbc = nodes.p_boundary.astype(np.uint8)
    outlet = (pw == ns.WALL_OUTFLOW) & (nodes.py != y0) & (nodes.py != y1)
    pbc[outlet] = R.PBC_DIRICHLET
    t = flow.tensors
    t["v_bcu"], t["v_bcv"], t["p_bc"] = d(bcu), d(bcv), d(pbc)
    neu = np.nonzero((bcu == R.BC_NEUMANN) | (bcv == R.BC_NEUMANN))[0].astype(np.int32)
    rows = d(neu)
    vx, vy = t["vx"], t["vy"]
    interior = d((~nodes.v_boundary).astype(np.uint8))
    idx, w, bad = R.build_weights_masked(ctx, vx[rows.long()], vy[rows.long()], vx, vy,
                                         R.OP_DX | R.OP_DY, beta_mask=interior, alpha_self=rows)
    if bad >= 0:
        raise R.RbffdError(R.ERR_SINGULAR_STENCIL, f"Neumann V-stencil {bad}")
    t["vn_rows"], t["vn_idx"] = rows, idx
    t["vn_dx"], t["vn_dy"] = w[0].contiguous(), w[1].contiguous()
    return flow


def wake_data(nodes, u_inf: float = 1.0, device="cuda"):
    """Dirichlet wall data (gu, gv) at the V-nodes: u_inf on the inflow, 0
    elsewhere (only the Dirichlet entries are read)."""
    import torch
    gu = np.where(nodes.v_wall == ns.WALL_INFLOW, u_inf, 0.0)
    return (torch.as_tensor(gu, device=device),
            torch.zeros(nodes.N, dtype=torch.float64, device=device))


def surface_rows(nodes, device="cuda"):
    """The cylinder's surface P-nodes in increasing angle (int32 device
    tensor) and the radius."""
    import torch
    cyl = np.nonzero(nodes.p_wall == ns.WALL_CYLINDER)[0]
    th = np.mod(np.arctan2(nodes.py[cyl], nodes.px[cyl]), 2.0 * np.pi)
    rows = cyl[np.argsort(th)].astype(np.int32)
    return torch.as_tensor(rows, device=device), float(nodes.meta["radius"])


def forces(ctx: R.Context, flow: R.Flow, state: R.State, nodes, rows=None):
    """(C_D, C_L) of the cylinder (rbffd_cylinder_forces)."""
    if rows is None:
        rows, _ = surface_rows(nodes, device=state.u.device)
    return R.cylinder_forces(ctx, flow, state, rows, float(nodes.meta["radius"]), flow.Re)


def strouhal(t, cl, diameter: float = 1.0, u_inf: float = 1.0) -> float:
    """St = f D / U of a lift history: f from the mean spacing of the upward
    zero crossings of cl - mean(cl) (linear interpolation between samples)."""
    t = np.asarray(t, np.float64)
    c = np.asarray(cl, np.float64) - np.mean(cl)
    up = np.nonzero((c[:-1] < 0.0) & (c[1:] >= 0.0))[0]
    if up.size < 2:
        raise ValueError("fewer than two upward zero crossings")
    tc = t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])
    return diameter / ((tc[-1] - tc[0]) / (tc.size - 1) * u_inf)
