"""Gradients of a final-time objective through many split steps (torch.autograd).

``evolve(plan, psi0, gammas, t0)`` advances psi0 by len(gammas) TS2-GauSum
steps with per-step trap frequencies ``gammas`` ([nsteps][dim], float64) and
is differentiable with respect to both. The forward pass keeps one state
every ceil(sqrt(T)) steps; the backward pass recomputes the states of each
segment with ``fse_step`` and pulls the cotangent back with
``fse_step_adjoint``, last step first. Gradients follow torch's convention for
complex inputs, dJ/dRe + i dJ/dIm, which is the library's cotangent
convention.
"""
from __future__ import annotations

import math

import numpy as np
import torch


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, gammas, plan, t0):
        T = int(gammas.shape[0])
        seg = max(1, int(math.ceil(math.sqrt(T))))
        gam = gammas.detach().cpu().numpy().astype(np.float64)
        x = psi0.detach().clone().contiguous()
        ckpts = []
        dt = plan.params["dt"]
        for s0 in range(0, T, seg):
            ckpts.append(x.clone())
            n = min(seg, T - s0)
            plan.step(x, t0 + s0 * dt, n, gam[s0:s0 + n])
        ctx.plan, ctx.t0, ctx.seg, ctx.gam, ctx.ckpts = plan, t0, seg, gam, ckpts
        ctx.gdev = gammas.device
        ctx.gdtype = gammas.dtype
        return x

    @staticmethod
    def backward(ctx, g_out):
        plan, t0, seg, gam = ctx.plan, ctx.t0, ctx.seg, ctx.gam
        T = gam.shape[0]
        dt = plan.params["dt"]
        g = g_out.detach().clone().contiguous().to(plan.cdtype)
        dgam = np.zeros_like(gam)
        for si in range(len(ctx.ckpts) - 1, -1, -1):
            s0 = si * seg
            n = min(seg, T - s0)
            states = [ctx.ckpts[si]]
            x = ctx.ckpts[si].clone()
            for k in range(n - 1):
                plan.step(x, t0 + (s0 + k) * dt, 1, gam[s0 + k:s0 + k + 1])
                states.append(x.clone())
            for k in range(n - 1, -1, -1):
                dgam[s0 + k] = plan.adjoint(states[k], g, t0 + (s0 + k) * dt, gam[s0 + k], want_dgamma=True)[:plan.dim]
        ctx.ckpts = None
        return g, torch.as_tensor(dgam, dtype=ctx.gdtype, device=ctx.gdev), None, None


def evolve(plan, psi0: torch.Tensor, gammas: torch.Tensor, t0: float = 0.0) -> torch.Tensor:
    """Differentiable len(gammas) split steps of psi0 (device tensor of the plan's dtype)."""
    return _Evolve.apply(psi0, gammas, plan, t0)


def overlap_objective(psi: torch.Tensor, target: torch.Tensor, cell: float) -> torch.Tensor:
    """J = |<psi, target>|^2 with <f, g> = h^d sum f conj(g)."""
    c = cell * torch.sum(psi * torch.conj(target))
    return (c.real ** 2 + c.imag ** 2)
