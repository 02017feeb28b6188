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


class Seismogram(torch.autograd.Function):
    """Receiver traces d[n, r]: p at the receivers after each of nsteps single-rate LSRK(5,4)
    steps of dt from q0 at time t0, on a Mesh with a point source and receivers set.

    Inputs: ``q0`` (device float32 [4, ndof]); ``c2`` (device float64, one per element in the
    dg_layout type order) and ``amp`` (device float64 [1]) stand for the mesh's c^2 and source
    amplitude and receive dL/dc^2 and dL/damp (their values are not read); ``every`` the
    checkpoint interval.  Backward: dg_adjoint_step per window, last first, with the window's
    rows of dL/dd as receiver forcing."""

    @staticmethod
    def forward(ctx, q0, c2, amp, mesh, nsteps, dt=0.0, t0=0.0, every=20):
        q = q0.detach().contiguous()
        mesh.set_state(q, on_device=True)
        out = torch.empty((nsteps, mesh.nrec), dtype=torch.float32, device=q.device)
        ckpts, starts, lens = [], [], []
        t = t0
        for n in range(nsteps):
            if n % every == 0:
                ck = torch.empty_like(q)
                mesh.get_state(ck, on_device=True)
                ckpts.append(ck)
                starts.append(t)
                lens.append(min(every, nsteps - n))
            t = mesh.step(1, dt, t)
            mesh.sample_receivers(out[n])
        ctx.save_for_backward(*ckpts)
        ctx.mesh, ctx.starts, ctx.lens, ctx.dt, ctx.nc2, ctx.every = mesh, starts, lens, dt, c2.numel(), every
        return out

    @staticmethod
    def backward(ctx, gd):
        mesh = ctx.mesh
        gd = gd.detach().to(torch.float32).contiguous()
        lam = torch.zeros_like(ctx.saved_tensors[0])
        grad_c2 = torch.zeros(ctx.nc2, dtype=torch.float64, device=lam.device) if ctx.needs_input_grad[1] else None
        grad_amp = torch.zeros(1, dtype=torch.float64, device=lam.device) if ctx.needs_input_grad[2] else None
        for w in range(len(ctx.lens) - 1, -1, -1):
            mesh.set_state(ctx.saved_tensors[w], on_device=True)
            rows = gd[w * ctx.every:w * ctx.every + ctx.lens[w]].contiguous()
            mesh.adjoint_step(ctx.lens[w], lam, grad_c2, ctx.dt, ctx.starts[w], rows, grad_amp)
        return lam, grad_c2, grad_amp, None, None, None, None, None


def seismogram(mesh, q0, c2, amp, nsteps, dt=0.0, t0=0.0, every=20):
    """Functional form of Seismogram.apply."""
    return Seismogram.apply(q0, c2, amp, mesh, nsteps, dt, t0, every)
