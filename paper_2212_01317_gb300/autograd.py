"""The energy matching as a differentiable function of the block inverse
temperatures (argument marshalling over the C-ABI; every step runs in libmpr).

The calibration of Sec. 2.1 (applied per block in Sec. 2.2.2) matches the
calibration chains' mean specific block energy y_b = <E_b>/N_b to the
sample energy e_s,b. ``BlockEnergy.apply(beta, handle, ...)`` runs the
chains at ``beta`` (mpr_energy_moments) and returns y; its backward is the
library's vector-Jacobian-product kernel (mpr_energy_vjp), built on the
fluctuation identity d y_a / d beta_b = -Cov(E_a, E_b) / N_a with the
covariances measured by the same run. The Newton calibration built on the
same moments runs inside the library: mpr_calibrate with cal_method = 1.
"""
from __future__ import annotations

import torch

from . import mpr


class BlockEnergy(torch.autograd.Function):
    """y = BlockEnergy.apply(beta, handle, n_eq, n_meas, tag, restart).

    beta: float32 CUDA tensor [nblk] (> 0); handle: an mpr context; returns a
    float64 CUDA tensor [nblk]. The moments of the run stay in the context,
    so call backward before the next forward on the same context."""

    @staticmethod
    def forward(fctx, beta, handle, n_eq: int, n_meas: int, tag: int, restart: bool):
        b = beta.detach().to(torch.float32).contiguous()
        y = torch.empty(b.numel(), dtype=torch.float64, device=b.device)
        mpr.mpr_energy_moments(handle, b, n_eq, n_meas, tag, restart, mean_e=y)
        fctx.handle = handle
        fctx.beta_dtype = beta.dtype
        return y

    @staticmethod
    def backward(fctx, grad_y):
        g = grad_y.detach().to(torch.float64).contiguous()
        out = torch.empty_like(g)
        mpr.mpr_energy_vjp(fctx.handle, g, out)
        return out.to(fctx.beta_dtype), None, None, None, None, None


def block_moments(handle, beta, n_eq: int, n_meas: int, tag: int, restart: bool):
    """(y, Var(E_b), Cov right, Cov down) at beta, as float64 CUDA tensors."""
    b = beta.detach().to(torch.float32).contiguous()
    outs = [torch.empty(b.numel(), dtype=torch.float64, device=b.device) for _ in range(4)]
    mpr.mpr_energy_moments(handle, b, n_eq, n_meas, tag, restart, *outs)
    return outs
