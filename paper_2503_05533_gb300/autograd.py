"""dQ/dxi as a torch.autograd.Function (form 3 of the hot path).

Forward: KL synthesis of the coefficient from xi and the batched solve give
Q[s] (only Q is kept).  Backward: ``mlmc_adjoint_grad`` recomputes the
forward solution together with the adjoint solution A lambda = g in one
resident-solve launch, forms the element products and contracts them back onto
the KL terms (Problem 4.5 with the discrete adjoint of the P1 system).
"""
import torch

from . import capi as L


class MlmcQoI(torch.autograd.Function):
    """Q = G(u(xi)) per sample on the grid of ``level`` (n cells per side)."""

    @staticmethod
    def forward(fctx, xi, handle, level, n, prec, delta, max_iters):
        if not xi.is_cuda:
            raise ValueError("xi must be a CUDA tensor")
        xi = xi.detach().to(torch.float64).contiguous()
        S = xi.shape[0]
        # the same FP64 master field as the backward pass: FP64 contraction for the FP64 solve, the
        # tensor-core FP64 field for the mixed-precision solves
        field_prec = L.MLMC_FP64 if prec == L.MLMC_FP64 else L.MLMC_FP64TC
        a = torch.empty((S, (n + 1) * (n + 1)), dtype=torch.float64, device=xi.device)
        L.mlmc_synthesize_fields(handle, level, S, xi, a, field_prec)
        Q = torch.empty(S, dtype=torch.float64, device=xi.device)
        L.mlmc_level_solve(handle, n, S, a, L.MLMC_FP64, n, prec, L.MLMC_CG, delta, max_iters, None, Q)
        fctx.save_for_backward(xi)
        fctx.cfg = (handle, level, prec, delta, max_iters)
        return Q

    @staticmethod
    def backward(fctx, gQ):
        (xi,) = fctx.saved_tensors
        handle, level, prec, delta, max_iters = fctx.cfg
        S, K = xi.shape
        Q = torch.empty(S, dtype=torch.float64, device=xi.device)
        g = torch.empty((S, K), dtype=torch.float64, device=xi.device)
        L.mlmc_adjoint_grad(handle, level, S, xi, prec, delta, max_iters, Q, g)
        return gQ.to(torch.float64)[:, None] * g, None, None, None, None, None, None


def qoi(xi, handle, level, n, prec=L.MLMC_FP64, delta=1e-12, max_iters=100000):
    return MlmcQoI.apply(xi, handle, level, n, prec, delta, max_iters)
