"""Energy of the truncated ansatz as a differentiable torch function.

``SwcsEnergy.apply(theta, ctx, ops, n_keep, ckpt_every)`` returns
E(theta) = <psi|H|psi>/<psi|psi> for the gate sequence of Eq. 1 with top-N
truncation after every gate (Sec. II.B).  Its backward returns dE/dtheta from
the library's adjoint sweep (each truncation held as a fixed projector), so a
torch optimiser can drive the VQE step of ADAPT (Sec. II.C).  The forward
computes energy and gradient in one C-ABI call (swcs_energy_grad); backward
only scales the stored gradient.  No arithmetic of the method runs here.
"""
from __future__ import annotations

import numpy as np
import torch


class SwcsEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, ctx, ops, n_keep, ckpt_every=20):
        th = theta.detach().to("cpu", torch.float64).contiguous().numpy()
        e, d = ctx.energy_grad(np.asarray(ops), th, int(n_keep), int(ckpt_every))
        fctx.save_for_backward(torch.from_numpy(d).to(theta.device, theta.dtype))
        return torch.tensor(e, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(fctx, grad_out):
        (d,) = fctx.saved_tensors
        return grad_out * d, None, None, None, None


def energy(theta, ctx, ops, n_keep, ckpt_every=20):
    return SwcsEnergy.apply(theta, ctx, ops, n_keep, ckpt_every)
