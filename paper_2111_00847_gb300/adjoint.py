"""Reverse-mode gradients through the fused time steps.

``rollout(phi0, gravity, params, steps, every)`` runs ``steps`` steps of the
scheme from phi0 (u = 0, p = 0) under the body force (gx, gy) = gravity and
returns phi after the last step, as a differentiable PyTorch operation: its
backward pass runs the library's hand-written discrete adjoint
(lbm_adjoint_*), so any objective written in PyTorch on the returned phi gets
gradients with respect to phi0 (and through it, anything phi0 is built from)
and to gravity.

Checkpointing: the forward pass keeps a device snapshot of the state every
``every`` steps.  The backward pass walks the segments from the last to the
first; each segment is recomputed from its snapshot with the state after
every step kept (``every`` snapshots of work space), then swept in reverse by
the adjoint step.  Memory: (steps / every + every) states; time: one extra
forward pass plus the adjoint steps.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import LBM_PHI, Simulation


def _with_gravity(params, gx: float, gy: float):
    if hasattr(params, "with_"):
        return params.with_(gx=gx, gy=gy)
    p = copy.copy(params)
    p.gx, p.gy = gx, gy
    return p


class Rollout(torch.autograd.Function):
    """(phi0 [ny, nx] float64, gravity [2] float64) -> phi_N [ny, nx] float64."""

    @staticmethod
    def forward(ctx, phi0, gravity, params, steps, every):
        steps, every = int(steps), int(every)
        if steps < 1 or every < 1:
            raise ValueError("steps and every must be positive")
        g = gravity.detach().double().cpu().numpy()
        sim = Simulation(_with_gravity(params, float(g[0]), float(g[1])))
        sim.init_fields(phi0.detach().double().cpu().numpy())
        ckpts = [sim.snapshot(sim.new_state_buffer())]
        t = 0
        while t < steps:
            n = min(every, steps - t)
            sim.step(n)
            t += n
            if t < steps:
                ckpts.append(sim.snapshot(sim.new_state_buffer()))
        phiN = torch.from_numpy(sim.fields(LBM_PHI)).to(phi0.device)
        ctx.sim, ctx.ckpts, ctx.steps, ctx.every = sim, ckpts, steps, every
        ctx.devices = (phi0.device, gravity.device)
        return phiN

    @staticmethod
    def backward(ctx, grad_phiN):
        sim, ckpts, steps, K = ctx.sim, ctx.ckpts, ctx.steps, ctx.every
        sim.adjoint_seed(grad_phiN.detach().double().cpu().numpy())
        work = [sim.new_state_buffer() for _ in range(min(K, steps) - 1)]
        for c in reversed(range(len(ckpts))):
            t0 = c * K
            L = min(K, steps - t0)
            sim.restore(ckpts[c], t0)
            seg = [ckpts[c]]
            for j in range(1, L):
                sim.step(1)
                seg.append(sim.snapshot(work[j - 1]))
            for j in reversed(range(L)):
                sim.adjoint_step(seg[j])
        dphi0 = sim.adjoint_init(ckpts[0])
        dG = sim.adjoint_gravity()
        ctx.sim = ctx.ckpts = None
        sim.close()
        return (torch.from_numpy(dphi0).to(ctx.devices[0]),
                torch.from_numpy(dG).to(ctx.devices[1]), None, None, None)


def rollout(phi0: torch.Tensor, gravity: torch.Tensor, params, steps: int, every: int = 100) -> torch.Tensor:
    return Rollout.apply(phi0, gravity, params, steps, every)


def centroid_y(phi: torch.Tensor) -> torch.Tensor:
    """The phi-weighted vertical centroid, node centres at j + 1/2."""
    ny = phi.shape[0]
    y = torch.arange(ny, dtype=phi.dtype, device=phi.device).view(-1, 1) + 0.5
    return (phi * y).sum() / phi.sum()


def interface_phi0(amplitudes: torch.Tensor, nx: int, ny: int, width: float, phiA: float = 1.0,
                   phiB: float = 0.0) -> torch.Tensor:
    """Differentiable initial field of the RTI cases: phase A above
    y = ny/2 + sum_k a_k cos(2 pi k x / nx) with the tanh profile of width W
    (node centres at i + 1/2, j + 1/2)."""
    dt = amplitudes.dtype
    x = torch.arange(nx, dtype=dt, device=amplitudes.device) + 0.5
    y = torch.arange(ny, dtype=dt, device=amplitudes.device) + 0.5
    k = torch.arange(1, amplitudes.numel() + 1, dtype=dt, device=amplitudes.device)
    h = (amplitudes.view(-1, 1) * torch.cos(2.0 * np.pi * k.view(-1, 1) * x.view(1, -1) / nx)).sum(0)
    dist = y.view(-1, 1) - (0.5 * ny + h.view(1, -1))
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * torch.tanh(2.0 * dist / width)
