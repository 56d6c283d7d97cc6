"""Differentiated form: T unrolled GoDec-BRP iterations at q = 0 as a torch.autograd.Function.

The forward pass runs the iterations on the GPU (``GoDec`` with q = 0) and keeps only the
supports Omega_1 .. Omega_{T-1} of S; the backward pass is ``godec_backward``, the
hand-written adjoint with those supports frozen (the selection is piecewise constant in
X), which recomputes the per-iteration factors itself.  Only X receives a gradient.
"""
import torch

from ._binding import GoDec, backward


class UnrolledGoDec(torch.autograd.Function):
    """L_T (m x n, dense) of T iterations of Algorithm 1 at q = 0 from S_0 = 0."""

    @staticmethod
    def forward(ctx, X, A1, r: int, k: int, T: int):
        g = GoDec(X, A1, r, k, 0, tol=0.0, max_iter=max(T, 1))
        try:
            supports = []
            for t in range(T):
                g.iterate(1)
                if t < T - 1:
                    supports.append(g.S()[0].clone())
            if g.info()["r_eff"] != r:
                raise RuntimeError("the rank test lowered r during the unrolled iterations; "
                                   "the differentiated form needs a fixed r")
            L = g.L_dense()
        finally:
            g.close()
        ctx.save_for_backward(X, A1, *supports)
        ctx.T = T
        return L

    @staticmethod
    def backward(ctx, gL):
        X, A1, *supports = ctx.saved_tensors
        dX = backward(X, A1, ctx.T, supports, gL=gL.contiguous().float())
        return dX, None, None, None, None


def unrolled_godec(X, A1, r: int, k: int, T: int):
    """L_T of T unrolled q = 0 iterations, differentiable with respect to X."""
    return UnrolledGoDec.apply(X, A1, r, k, T)
