"""The (n, m, q) parameter study of the paper (Section 4.1-4.2, App. B) on the
GPU: for every stencil-size / PHS-exponent / polynomial-degree triple, the
batched weight build (rbffd_build_weights), the per-node relative error of
Eq. relative_error on the test function of Eq. test (rbffd_stencil_error,
which also reduces the node mean on the device) and, optionally, the
condition numbers of the local systems (rbffd_stencil_condition).  Host code
here only sequences those calls; every number comes from the CUDA library.
"""
from __future__ import annotations

from . import rbffd as R

_OP_NAMES = {R.OP_INTERP: "interp", R.OP_DX: "dx", R.OP_DY: "dy", R.OP_LAP: "lap"}


def parameter_sweep(ax, ay, bx, by, triples, op_mask: int = R.OP_DX | R.OP_LAP, dr=None,
                    condition: bool = False):
    """One entry per (n, m, q): {"n", "m", "q", "bad_node", "E_<op>" (0-d device
    tensor: the mean relative error), "err_<op>" (per-node errors) and, with
    condition=True, "cond" (per-node 1-norm condition numbers)}.  ax, ay:
    alpha-nodes; bx, by: beta-nodes (torch CUDA float64).  dr: per-alpha-node
    spacing, or None for a collocated set (the mean distance to the 6 nearest
    nodes, taken from each stencil; needs n >= 7)."""
    out = []
    for n, m, q in triples:
        ctx = R.Context(n, m, q)
        try:
            idx, w, bad = R.build_weights(ctx, ax, ay, bx, by, op_mask)
            entry = {"n": n, "m": m, "q": q, "bad_node": bad}
            for o, op in enumerate(R.ops_of(op_mask)):
                err, mean = R.stencil_error(ctx, idx, w[o], op, ax, ay, bx, by, dr)
                entry["E_" + _OP_NAMES[op]] = mean
                entry["err_" + _OP_NAMES[op]] = err
            if condition:
                entry["cond"] = R.stencil_condition(ctx, ax, ay, bx, by, idx)
            out.append(entry)
        finally:
            ctx.close()
    return out
