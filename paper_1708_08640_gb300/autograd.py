"""Differentiation form: the objective f of Eq. (7) as a ``torch.autograd.Function``.

forward(G, U_1..U_N, V_1..V_M) loads the parameters into the model and evaluates f on the
GPU (s3_loss); backward returns grad_out times the full gradient of f (s3_gradient: the
sum over all observed entries of Eq. (8), computed by the fused contribution kernels and
fixed-order segmented reductions; no per-entry Kronecker products are stored).
"""
from __future__ import annotations

import torch


class S3LossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, model, G, *factors):
        N = model.N
        U, V = list(factors[:N]), list(factors[N:])
        model.set_params(G.detach(), [u.detach() for u in U], [v.detach() for v in V])
        f, _ = model.loss()
        ctx.model = model
        ctx.save_for_backward(G, *factors)
        return torch.tensor(f, dtype=torch.float64, device=G.device)

    @staticmethod
    def backward(ctx, grad_out):
        model = ctx.model
        saved = ctx.saved_tensors
        N = model.N
        G, U, V = saved[0], list(saved[1:1 + N]), list(saved[1 + N:])
        model.set_params(G.detach(), [u.detach() for u in U], [v.detach() for v in V])
        dG, dU, dV = model.gradient()
        s = grad_out.to(torch.float32)
        return (None, dG * s, *[d * s for d in dU], *[d * s for d in dV])


def s3_loss(model, G, U, V):
    """f(G, U, V) with gradients w.r.t. every argument that requires them."""
    return S3LossFn.apply(model, G, *U, *V)
