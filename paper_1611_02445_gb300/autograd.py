"""torch.autograd.Function over the library's hand-written adjoint.

OutletFluxLoss.apply(g_field, tau, lattice, T, plane_x, ckpt_every) runs T fused steps
from the equilibrium at rest with the per-node x body force g_field (a float64 CUDA
tensor of the lattice's [nz, ny, nx] shape) and relaxation time tau (a 0-dim tensor),
and returns L = mean u_x over the non-solid nodes of the plane x = plane_x. When a
gradient is needed, the forward call runs lbm_adjoint (checkpoint every ckpt_every
steps, recompute, reverse sweep) and keeps dL/dg and dL/dtau for backward; otherwise
it only steps and evaluates L. All of it runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import lbm


class OutletFluxLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g_field, tau, lattice, T, plane_x, ckpt_every):
        if not (g_field.is_cuda and g_field.dtype == torch.float64 and g_field.is_contiguous()):
            raise ValueError("g_field must be a contiguous float64 CUDA tensor")
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        lattice.set_params(float(tau), (0.0, 0.0, 0.0), g_field)
        lattice.init_equilibrium(1.0)
        dg = torch.zeros_like(g_field) if need else None
        torch.cuda.current_stream().synchronize()
        L, dtau = lbm.lbm_adjoint(lattice.ctx, T, ckpt_every, plane_x, dg, need)
        if need:
            ctx.save_for_backward(dg, torch.tensor(dtau, dtype=torch.float64, device=g_field.device))
        return torch.tensor(L, dtype=torch.float64, device=g_field.device)

    @staticmethod
    def backward(ctx, grad_L):
        dg, dtau = ctx.saved_tensors
        return grad_L * dg, (grad_L * dtau).reshape(()), None, None, None, None


def outlet_flux_loss(g_field, tau, lattice, T, plane_x, ckpt_every=100):
    return OutletFluxLoss.apply(g_field, tau, lattice, T, plane_x, ckpt_every)
