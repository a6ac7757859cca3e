"""torch.autograd wrapper of the advection step and a checkpointed rollout.

``advect(T_old, u_old, mesh, dt, n_sub, u_new=None)`` is differentiable in
T_old and in the velocity: the forward pass is ``elm_advect`` and the
backward pass ``elm_advect_adjoint`` (transpose interpolation and the
velocity sensitivity through the RK stages).  All tensors are in the mesh's
storage layout; gradients are gathered on each node's owner slot.

``rollout`` runs many steps and keeps activations only at segment
boundaries (every ``checkpoint_every`` steps); the steps inside a segment are
recomputed during the backward pass.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint


class Advect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T_old, u_old, u_new, mesh, dt, n_sub):
        steady = u_new is None
        mesh.set_velocity(u_old, None if steady else u_new)
        T_new = mesh.advect(T_old.contiguous(), dt, n_sub)
        ctx.mesh, ctx.dt, ctx.n_sub, ctx.steady = mesh, float(dt), int(n_sub), steady
        ctx.save_for_backward(T_old, u_old, u_old if steady else u_new)
        return T_new

    @staticmethod
    def backward(ctx, gT_new):
        T_old, u_old, u_new = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_velocity(u_old, None if ctx.steady else u_new)
        gT_old, gU_old, gU_new = mesh.advect_adjoint(T_old.contiguous(), gT_new.contiguous(), ctx.dt, ctx.n_sub,
                                                     split=not ctx.steady)
        return gT_old, gU_old, (None if ctx.steady else gU_new), None, None, None


def advect(T_old, u_old, mesh, dt, n_sub: int = 1, u_new=None):
    """One differentiable advection step (storage layout)."""
    return Advect.apply(T_old, u_old, u_new, mesh, dt, n_sub)


def rollout(T0, u, mesh, dt, steps: int, n_sub: int = 1, checkpoint_every: int = 10):
    """`steps` differentiable steps with a steady velocity u; activations are
    kept every `checkpoint_every` steps only (0 keeps every step)."""
    def segment(T, uu, k):
        for _ in range(k):
            T = advect(T, uu, mesh, dt, n_sub)
        return T

    T = T0
    done = 0
    while done < steps:
        k = min(checkpoint_every if checkpoint_every > 0 else steps, steps - done)
        if checkpoint_every > 0 and torch.is_grad_enabled():
            T = checkpoint(segment, T, u, k, use_reentrant=False)
        else:
            T = segment(T, u, k)
        done += k
    return T
