"""torch.autograd access to the fractional step and its discrete adjoint.

`rollout(...)` advances a flow n steps from an initial velocity with fixed
wall data and returns the final velocity; its backward pass walks the steps in
reverse with rbffd_adjoint_step.  Forward states are checkpointed every
`every` steps and the states inside a segment are recomputed from its
checkpoint when the backward pass reaches it, so memory holds
n/every + every states instead of n.  All arithmetic runs in librbffd.
"""
from __future__ import annotations

import torch

from . import rbffd as R


def _copy_state(s: R.State) -> R.State:
    return R.State(s.u.clone(), s.v.clone(), s.cu_prev.clone(), s.cv_prev.clone(), s.pt.clone(),
                   s.p.clone(), s.j)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, gu, gv, u0, v0, rb, flow, n_steps, every):
        st = R.State.zeros(flow)
        st.u.copy_(u0)
        st.v.copy_(v0)
        gu_c, gv_c = gu.detach().contiguous(), gv.detach().contiguous()
        checkpoints = {0: _copy_state(st)}
        for j in range(n_steps):
            R.step(rb, flow, st, gu_c, gv_c, 1)
            if (j + 1) % every == 0 and j + 1 < n_steps:
                checkpoints[j + 1] = _copy_state(st)
        fctx.rb, fctx.flow, fctx.n, fctx.every = rb, flow, n_steps, every
        fctx.checkpoints = checkpoints
        fctx.save_for_backward(gu_c, gv_c)
        return st.u.clone(), st.v.clone()

    @staticmethod
    def backward(fctx, gout_u, gout_v):
        gu, gv = fctx.saved_tensors
        rb, flow, n, every = fctx.rb, fctx.flow, fctx.n, fctx.every
        lam = R.Adjoint.zeros(flow)
        lam.u.copy_(gout_u)
        lam.v.copy_(gout_v)
        grad_gu = torch.zeros_like(gu)
        grad_gv = torch.zeros_like(gv)
        starts = sorted(fctx.checkpoints)
        for c in reversed(starts):
            end = min(c + every, n)
            st = _copy_state(fctx.checkpoints[c])
            states = [_copy_state(st)]
            for _ in range(c, end - 1):  # recompute the segment's forward states
                R.step(rb, flow, st, gu, gv, 1)
                states.append(_copy_state(st))
            for s in reversed(states):
                R.adjoint_step(rb, flow, s, lam, grad_gu, grad_gv)
        return grad_gu, grad_gv, lam.u, lam.v, None, None, None, None


def rollout(rb: R.Context, flow: R.Flow, gu, gv, u0, v0, n_steps: int, every: int = 20):
    """Final (u, v) after n_steps from (u0, v0) with wall data (gu, gv);
    differentiable with respect to gu, gv, u0 and v0."""
    return _Rollout.apply(gu, gv, u0, v0, rb, flow, n_steps, every)
