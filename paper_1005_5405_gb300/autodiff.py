"""Gradients through many cavity steps (bz_adjoint_step behind autograd).

J is any function of the final state h^M and of the time-averaged lid shear

    D_bar = (1/M) sum_{n=0}^{M-1} D_n,

with D_n the mean x-momentum flux through the lid of h^n (D of Sec. 5.2, as
bz_lid_shear computes it).  `rollout` returns (h^M, D_bar) as autograd
tensors whose gradients flow to the lid face speeds and to h^0.

The random sample sets of the steps are fixed (they depend on the seed and
the step number only), so each step is a smooth map and its adjoint is exact
up to rounding.  The forward pass keeps every `every`-th state (step
checkpointing); the backward pass replays one segment at a time from its
checkpoint, keeps that segment's states, and runs the adjoint steps of the
segment in reverse.  Memory: (M/every + every) states instead of M.
"""
from __future__ import annotations

import numpy as np
import torch


class Rollout(torch.autograd.Function):
    """(lid, h0) -> (h^M, D_bar) over `nsteps` steps of a Cavity handle."""

    @staticmethod
    def forward(ctx, lid, h0, cav, nsteps: int, step0: int, every: int):
        p = cav.p
        if nsteps < 1 or every < 1:
            raise ValueError("nsteps and every must be >= 1")
        lid_np = lid.detach().to(torch.float64).cpu().numpy().copy()
        if lid_np.shape != (p.nx,):
            raise ValueError(f"lid must have shape ({p.nx},)")
        cav.set_lid(0.0, p.lid_amp, p.lid_period, profile=lid_np)
        cav.set_state(h0.detach().to(cav.torch_dtype).contiguous(), step0)
        shear = torch.empty((nsteps, p.nx + 1), dtype=torch.float64, device=h0.device)
        ckpts = {}
        for n in range(nsteps):
            if n % every == 0:
                ckpts[n] = cav.get_state()[0].clone()
            cav.lid_shear(out=shear[n])
            cav.step(1)
        hM = cav.get_state()[0].clone()
        d_bar = float(np.mean(shear[:, p.nx].cpu().numpy()))
        ctx.cav, ctx.lid_np, ctx.ckpts = cav, lid_np, ckpts
        ctx.nsteps, ctx.step0, ctx.every = nsteps, step0, every
        ctx.lid_meta = (lid.dtype, lid.device)
        ctx.h0_meta = (h0.dtype, h0.device)
        return hM.to(h0.dtype), torch.tensor(d_bar, dtype=torch.float64, device=h0.device)

    @staticmethod
    def backward(ctx, g_h, g_d):
        cav, p = ctx.cav, ctx.cav.p
        M, K, s0 = ctx.nsteps, ctx.every, ctx.step0
        ref = ctx.ckpts[0]
        if g_h is None:
            lam = torch.zeros_like(ref)
        else:
            lam = g_h.detach().to(cav.torch_dtype).contiguous().clone()
        wD = float(g_d) / M if g_d is not None else 0.0
        grad_lid = torch.zeros(p.nx, dtype=torch.float64, device=ref.device)
        cav.set_lid(0.0, p.lid_amp, p.lid_period, profile=ctx.lid_np)
        for s in sorted(ctx.ckpts, reverse=True):
            e = min(s + K, M)
            states = [ctx.ckpts[s]]
            cav.set_state(ctx.ckpts[s], s0 + s)
            for _ in range(s + 1, e):
                cav.step(1)
                states.append(cav.get_state()[0].clone())
            for n in range(e - 1, s - 1, -1):
                cav.adjoint_step(s0 + n, states[n - s], lam, lam, grad_lid, wD)
        ldt, ldev = ctx.lid_meta
        hdt, hdev = ctx.h0_meta
        return grad_lid.to(dtype=ldt, device=ldev), lam.to(dtype=hdt, device=hdev), None, None, \
            None, None


def rollout(cav, lid, h0, nsteps: int, step0: int = 0, every: int = 50):
    """(h^M, D_bar) after `nsteps` steps of `cav` from h0 at step `step0`
    with lid face speeds `lid` ((nx,) tensor), differentiable in lid and h0.
    The handle's state and lid are overwritten (forward and backward)."""
    return Rollout.apply(lid, h0, cav, nsteps, step0, every)
