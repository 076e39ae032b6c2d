"""torch.autograd wrapper of the adjoint: log|Psi| of every walker as a differentiable
function of the CI coefficients and the orbital coefficients.

Forward loads the parameters into the libmsd context (msd_set_params, which rebuilds the
state at the context's current positions) and returns log|Psi_w| for every walker; backward
is one msd_backward call with the incoming gradient as the walker weights.  The arithmetic of
both directions runs in the library's kernels; this module only moves tensors.
"""
from __future__ import annotations

import torch

from .msd import MSD


class LogPsi(torch.autograd.Function):
    """logabs [W] = log|Psi(R_w; c, B_up, B_dn)| at the context's current positions R.

    A restricted orbital set (one B for both spins) is passed as the same tensor twice;
    autograd then adds the two spin blocks of the gradient.
    """

    @staticmethod
    def forward(ctx, wf: MSD, ci: torch.Tensor, B_up: torch.Tensor, B_dn: torch.Tensor):
        wf.set_params(ci.detach().to("cpu", torch.float64).numpy(),
                      (B_up.detach().to("cpu", torch.float64).numpy(), B_dn.detach().to("cpu", torch.float64).numpy()))
        _, logabs, _ = wf.get_state()
        ctx.wf = wf
        ctx.devices = (ci.device, B_up.device, B_dn.device)
        ctx.dtypes = (ci.dtype, B_up.dtype, B_dn.dtype)
        return logabs.clone()

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        dci, (d_up, d_dn) = ctx.wf.backward(g.detach().to(ctx.wf.dev, torch.float64).contiguous())
        (dv0, dv1, dv2), (dt0, dt1, dt2) = ctx.devices, ctx.dtypes
        return None, dci.to(dv0, dt0), d_up.to(dv1, dt1), d_dn.to(dv2, dt2)


def log_psi(wf: MSD, ci: torch.Tensor, B_up: torch.Tensor, B_dn: torch.Tensor) -> torch.Tensor:
    """Differentiable log|Psi| per walker (see LogPsi)."""
    return LogPsi.apply(wf, ci, B_up, B_dn)
