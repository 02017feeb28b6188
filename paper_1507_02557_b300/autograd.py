"""torch.autograd bridge: LSRK(5,4) propagation on a Mesh with a checkpointed discrete adjoint.

Argument marshalling only: the forward steps run through dg_step and the backward pass through
dg_adjoint_step (include/dg.h), one call per window of steps, last window first, each from the
checkpoint saved at the window's start.
"""
from __future__ import annotations

import torch


class Propagate(torch.autograd.Function):
    """q_n = S^n q_0: nsteps single-rate LSRK(5,4) steps of dt (0: the mesh's dt_min).

    Inputs: ``q0`` (device float32 [4, ndof]); ``c2`` (device float64, one entry per element in
    the dg_layout type order) stands for the mesh's own c^2 and receives dL/dc^2 (its values are
    not read: the mesh was built with its c^2); ``mesh`` (a dg.Mesh with nlevels = 1); ``every``
    the checkpoint interval.  Memory: one saved state per window."""

    @staticmethod
    def forward(ctx, q0, c2, mesh, nsteps, dt=0.0, every=20):
        q = q0.detach().contiguous()
        ckpts, lens = [], []
        mesh.set_state(q, on_device=True)
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            ck = torch.empty_like(q)
            mesh.get_state(ck, on_device=True)
            ckpts.append(ck)
            lens.append(n)
            mesh.step(n, dt)
            done += n
        out = torch.empty_like(q)
        mesh.get_state(out, on_device=True)
        ctx.save_for_backward(*ckpts)
        ctx.mesh, ctx.lens, ctx.dt, ctx.nc2 = mesh, lens, dt, c2.numel()
        return out

    @staticmethod
    def backward(ctx, gq):
        mesh = ctx.mesh
        lam = gq.detach().to(torch.float32).contiguous().clone()
        grad = None
        if ctx.needs_input_grad[1]:
            grad = torch.zeros(ctx.nc2, dtype=torch.float64, device=lam.device)
        for ck, n in zip(reversed(ctx.saved_tensors), reversed(ctx.lens)):
            mesh.set_state(ck, on_device=True)
            mesh.adjoint_step(n, lam, grad, ctx.dt)
        return lam, grad, None, None, None, None


def propagate(mesh, q0, c2, nsteps, dt=0.0, every=20):
    """Functional form of Propagate.apply."""
    return Propagate.apply(q0, c2, mesh, nsteps, dt, every)
