"""The density energy N = 1/2 sum_b A_b rho_b psi_b (Eq. 6) as a
torch.autograd.Function.

forward runs the scatter and the spectral solve (fftpl_energy); backward is
the field-gather kernel (fftpl_gather, mode "gather": the q.E of Eq. 7) or
the exact derivative of the binned energy (mode "adjoint"), scaled by the
incoming gradient.  Positions are float32 CUDA tensors of the problem's
movable cells.
"""
from __future__ import annotations

import torch

from . import fftpl as F

_MODES = {"gather": 0, "adjoint": 1}


class DensityEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, problem, mode="gather"):
        if mode not in _MODES:
            raise ValueError(f"mode must be one of {sorted(_MODES)}")
        x = x.detach().contiguous()
        y = y.detach().contiguous()
        N = F.fftpl_energy(problem.h, x, y)
        problem._energy_calls = getattr(problem, "_energy_calls", 0) + 1
        ctx.problem = problem
        ctx.mode = mode
        ctx.call = problem._energy_calls
        ctx.save_for_backward(x, y)
        return torch.tensor(N, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, grad_out):
        x, y = ctx.saved_tensors
        problem = ctx.problem
        if problem._energy_calls != ctx.call:
            # the handle's maps belong to a later evaluation: recompute them
            F.fftpl_energy(problem.h, x, y, sync=False)
            problem._energy_calls += 1
        gx = torch.empty_like(x)
        gy = torch.empty_like(y)
        F.fftpl_gather(problem.h, x, y, gx, gy, _MODES[ctx.mode])
        s = grad_out.to(torch.float32)
        return gx * s, gy * s, None, None


def density_energy(x, y, problem, mode="gather"):
    """N(x, y) with the hand-written backward (see DensityEnergy)."""
    return DensityEnergy.apply(x, y, problem, mode)
