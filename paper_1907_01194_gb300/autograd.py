"""torch.autograd.Function wrappers of the library's adjoint kernels.

Energy.apply(X, h) returns E_h(X) (Eq. 3.7) as a 0-d float64 tensor; its backward
runs the gradient kernel (Eq. 3.12) on the saved X.  Gradient.apply(X, h)
returns nabla E_h(X); its backward runs the Hessian-vector kernel (Eq. 3.13),
which is the vector-Jacobian product because the real Hessian is symmetric.
Only X is saved: every FFT intermediate is recomputed by the kernels.

Complex convention: for a real loss L of a complex tensor X, PyTorch's gradient
is dL/dRe X + i dL/dIm X, which is the library's Euclidean gradient with respect
to Re<.,.> (Sec. 3, Taylor expansion of E_h).
"""
from __future__ import annotations

import torch


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, handle):
        X = X.contiguous()
        ctx.save_for_backward(X)
        ctx.handle = handle
        return torch.tensor(handle.energy(X), dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, gE):
        (X,) = ctx.saved_tensors
        G = torch.empty_like(X)
        ctx.handle.grad(X, G_euc=G, sync=False)
        return gE.to(G.real.dtype) * G, None


class Gradient(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, handle):
        X = X.contiguous()
        ctx.save_for_backward(X)
        ctx.handle = handle
        G = torch.empty_like(X)
        handle.grad(X, G_euc=G, sync=False)
        return G

    @staticmethod
    def backward(ctx, gG):
        (X,) = ctx.saved_tensors
        HZ = torch.empty_like(X)
        ctx.handle.hessvec(X, gG.contiguous(), HZ, sigma=0.0, riemannian=False)
        return HZ, None


def energy(X, handle):
    return Energy.apply(X, handle)


def gradient(X, handle):
    return Gradient.apply(X, handle)
