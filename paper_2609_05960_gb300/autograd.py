"""PyTorch autograd wrapper of the power walk.

``power_waveform(engine, window, bin_ps, load_ff, escale, lscale)`` returns
the waveform (W per bin, float64) as a differentiable function of every
gate's output load and every cell's internal-energy and leakage scale.  The
forward pass runs gtp_run_power; the backward pass runs the CUDA adjoint walk
(gtp_run_power_backward), which re-walks the events and gathers dL/dP per
bin.  Gradients come back as float32 (the walk's arithmetic type).
"""
from __future__ import annotations

import torch

from .gtpower import Engine


class _PowerWaveform(torch.autograd.Function):
    @staticmethod
    def forward(ctx, load_ff, escale, lscale, engine: Engine, window: int, bin_ps: int):
        engine.set_load(load_ff.detach().to(torch.float32).contiguous())
        engine.set_scales(escale.detach().to(torch.float32).cpu().numpy(),
                          lscale.detach().to(torch.float32).cpu().numpy())
        wave = engine.run_power(window, bin_ps)
        ctx.engine, ctx.window, ctx.bin_ps = engine, window, bin_ps
        ctx.like = (torch.empty(0, dtype=load_ff.dtype, device=load_ff.device),
                    torch.empty(0, dtype=escale.dtype, device=escale.device),
                    torch.empty(0, dtype=lscale.dtype, device=lscale.device))
        return wave

    @staticmethod
    def backward(ctx, grad_wave):
        dC, de, dl = ctx.engine.run_power_backward(ctx.window, ctx.bin_ps, grad_wave.to(torch.float32))
        lc, le, ll = ctx.like
        return dC.to(lc), de.to(le), dl.to(ll), None, None, None


def power_waveform(engine: Engine, window: int, bin_ps: int, load_ff: torch.Tensor, escale: torch.Tensor,
                   lscale: torch.Tensor) -> torch.Tensor:
    """Differentiable waveform; load_ff [n_gates] on the engine's device,
    escale / lscale [n_cells] (any device)."""
    return _PowerWaveform.apply(load_ff, escale, lscale, engine, window, bin_ps)


def peak_loss(P_w: torch.Tensor, tau_frac: float = 0.01) -> torch.Tensor:
    """sum_b P_b^2 + tau * log sum_b exp(P_b / tau) with P in mW and
    tau = tau_frac * mean(P) held constant (detached)."""
    P = P_w * 1e3
    tau = (tau_frac * P.mean()).detach()
    return (P * P).sum() + tau * torch.logsumexp(P / tau, dim=0)
