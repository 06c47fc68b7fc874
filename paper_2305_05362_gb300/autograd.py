"""Differentiable RAM steps on top of the C ABI.

RamSegment runs k steps forward with ram_step (donor residual) and, in backward,
recomputes the k forward states from its saved input and walks back through them
with ram_step_adjoint, accumulating the gradient of the residual velocity.  With
the limiter off the step is linear in Q (Sec. 3 with Eq. 6) and the backward pass
is its exact transpose; with the limiter on (a plan built with adjoint=True) each
step is linearised at its own input, the limiter branches frozen where that input
puts them, which is the gradient wherever the step is differentiable.
rollout() chains segments, so memory holds one checkpoint per segment
(checkpoint-and-recompute every k steps).
"""
from __future__ import annotations

import torch

from . import ram


class RamSegment(torch.autograd.Function):
    """k RAM steps as one differentiable operation (inputs: q, dv)."""

    @staticmethod
    def forward(ctx, q, dv, plan, v0, dt, nsub, k):
        ctx.plan, ctx.v0, ctx.dt, ctx.nsub, ctx.k = plan, v0, dt, nsub, k
        q = q.contiguous()
        ctx.save_for_backward(q, dv)
        cur = q
        for _ in range(k):
            nxt = torch.empty_like(cur)
            ram.step(plan, cur, nxt, v0, dt, dv=dv, scheme=ram.DONOR, nsub=nsub)
            cur = nxt
        return cur

    @staticmethod
    def backward(ctx, g):
        q, dv = ctx.saved_tensors
        plan, v0, dt, nsub, k = ctx.plan, ctx.v0, ctx.dt, ctx.nsub, ctx.k
        states = [q]
        for _ in range(k - 1):
            nxt = torch.empty_like(q)
            ram.step(plan, states[-1], nxt, v0, dt, dv=dv, scheme=ram.DONOR, nsub=nsub)
            states.append(nxt)
        g = g.contiguous()
        g_dv = None
        if dv is not None and ctx.needs_input_grad[1]:
            g_dv = torch.zeros_like(dv)
        for i in reversed(range(k)):
            gin = torch.empty_like(g)
            ram.step_adjoint(plan, states[i], g, gin, v0, dt, dv=dv, g_dv=g_dv, nsub=nsub)
            g = gin
        return g, g_dv, None, None, None, None, None


def rollout(plan, q0, v0, dt: float, steps: int, dv=None, nsub=None,
            checkpoint_every: int = 20):
    """Advance q0 by `steps` RAM steps, differentiable with respect to q0 and dv.
    The plan needs adjoint=True when its limiter is on, and when it has rows with
    their own mesh and dv is given."""
    q = q0
    done = 0
    while done < steps:
        k = min(checkpoint_every, steps - done)
        q = RamSegment.apply(q, dv, plan, v0, dt, nsub, k)
        done += k
    return q
