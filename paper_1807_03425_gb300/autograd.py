"""torch.autograd.Function over the soft-min entry points of libsap.

``softmin(U, sap, tau)`` returns L(U) = -tau log sum_{i<j} exp(-r_ij/tau) as a
0-d FP64 tensor; its backward calls the library's backward kernels, which
recompute every pair rather than keeping per-pair weights from the forward.
U is a (k, n) FP64 tensor (CPU or CUDA) with orthonormal rows, the layout of
``Sap.set_basis``; the gradient has the same layout.  Both passes run on the
GPU behind the C ABI; nothing is computed in PyTorch.
"""
from __future__ import annotations

import torch


class SoftMinFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, sap, tau):
        Uc = U.detach().contiguous()
        sap.set_basis(Uc)
        L = sap.softmin_forward(tau)
        ctx.sap, ctx.tau, ctx.L = sap, float(tau), L
        ctx.save_for_backward(Uc)
        return torch.tensor(L, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_L):
        (Uc,) = ctx.saved_tensors
        sap = ctx.sap
        sap.set_basis(Uc)  # the handle may hold another basis by now
        G = torch.empty_like(Uc)
        sap.softmin_backward(ctx.tau, ctx.L, out=G)
        return grad_L * G, None, None


def softmin(U, sap, tau):
    """Soft-min objective of the handle's dataset at basis U (see module doc)."""
    return SoftMinFunction.apply(U, sap, tau)
