"""torch.autograd.Function wrappers of the banded operators.

Each forward calls the CUDA forward kernel through the C ABI and each
backward calls the hand-written adjoint kernel (Alg. 2 for the Cholesky,
Alg. 4 for the subset inverse, the Table 1 compositions for solves and
products).  Tensors are the flat band / RHS pools of a ``batch.Layout``; the
``Plan`` fixes the batch.  Torch allocates outputs and zero cotangents only.
Outputs are zero-initialised: the kernels write only the entries of the
instances, so pool elements outside them (row padding, absent panel lanes)
read as 0 in reductions over whole pools.
"""
from __future__ import annotations

import torch

from . import binding as B


def _zeros_like_or(t, like):
    return torch.zeros_like(like) if t is None else t.contiguous()


class Cholesky(torch.autograd.Function):
    """(Q) -> (L, logdet): C of Sec. 4.1 with log det Q = 2 sum log L_jj."""

    @staticmethod
    def forward(ctx, plan, Q):
        lay = plan.layout
        L = torch.zeros_like(Q)
        logdet = torch.empty(lay.count, dtype=torch.float64, device=Q.device)
        info = torch.empty(lay.count, dtype=torch.int32, device=Q.device)
        B.banded_cholesky(plan.handle, Q.contiguous(), L, logdet, info)
        ctx.plan = plan
        ctx.save_for_backward(L)
        ctx.mark_non_differentiable(info)
        return L, logdet, info

    @staticmethod
    def backward(ctx, Lbar, ldbar, _info):
        (L,) = ctx.saved_tensors
        Lbar = _zeros_like_or(Lbar, L)
        ldbar = None if ldbar is None else ldbar.contiguous().to(torch.float64)
        Qbar = torch.zeros_like(L)
        B.banded_cholesky_vjp(ctx.plan.handle, L, Lbar, ldbar, Qbar, 0)
        return None, Qbar


class Solve(torch.autograd.Function):
    """(L, B) -> X with X = L^{-1} B (mode 0), L^{-T} B (1) or (L L^T)^{-1} B (2)."""

    @staticmethod
    def forward(ctx, plan, L, Bm, mode):
        X = torch.zeros_like(Bm)
        B.banded_solve(plan.handle, L.contiguous(), Bm.contiguous(), X, int(mode))
        ctx.plan, ctx.mode = plan, int(mode)
        ctx.save_for_backward(L, X)
        return X

    @staticmethod
    def backward(ctx, Xbar):
        L, X = ctx.saved_tensors
        Bbar = torch.zeros_like(X)
        Lbar = torch.zeros_like(L) if ctx.needs_input_grad[1] else None
        B.banded_solve_vjp(ctx.plan.handle, L, X, Xbar.contiguous(), ctx.mode, Bbar, Lbar, 0)
        return None, Lbar, Bbar, None


class SubsetInverse(torch.autograd.Function):
    """(L) -> S = band(Q^{-1}) with Q = L L^T (Alg. 3); backward Alg. 4."""

    @staticmethod
    def forward(ctx, plan, L):
        S = torch.zeros_like(L)
        B.banded_subset_inverse(plan.handle, L.contiguous(), S)
        ctx.plan = plan
        ctx.save_for_backward(L, S)
        return S

    @staticmethod
    def backward(ctx, Sbar):
        L, S = ctx.saved_tensors
        Lbar = torch.zeros_like(L)
        B.banded_subset_inverse_vjp(ctx.plan.handle, L, S, Sbar.contiguous(), Lbar, 0)
        return None, Lbar


class Product(torch.autograd.Function):
    """C = op(A) op(B) projected onto band (clo, cup) (Sec. 4.1); adjoints per Table 1."""

    @staticmethod
    def forward(ctx, plan, A, a_band, transA, Bm, b_band, transB, c_band):
        Cm = torch.zeros_like(A)
        B.banded_product(plan.handle, A.contiguous(), a_band[0], a_band[1], transA, Bm.contiguous(),
                         b_band[0], b_band[1], transB, Cm, c_band[0], c_band[1], 0)
        ctx.plan = plan
        ctx.args = (a_band, transA, b_band, transB, c_band)
        ctx.save_for_backward(A, Bm)
        return Cm

    @staticmethod
    def backward(ctx, Cbar):
        A, Bm = ctx.saved_tensors
        a_band, transA, b_band, transB, c_band = ctx.args
        Abar = torch.zeros_like(A) if ctx.needs_input_grad[1] else None
        Bbar = torch.zeros_like(Bm) if ctx.needs_input_grad[4] else None
        B.banded_product_vjp(ctx.plan.handle, A, a_band[0], a_band[1], transA, Bm, b_band[0], b_band[1], transB,
                             Cbar.contiguous(), c_band[0], c_band[1], Abar, Bbar, 0)
        return None, Abar, None, None, Bbar, None, None, None


class Matvec(torch.autograd.Function):
    """P = op(A) V for the plan's k columns (Sec. 4.1); adjoints per Table 1."""

    @staticmethod
    def forward(ctx, plan, A, a_band, transA, V):
        P = torch.zeros_like(V)
        B.banded_matvec(plan.handle, A.contiguous(), a_band[0], a_band[1], transA, V.contiguous(), P, 0)
        ctx.plan, ctx.args = plan, (a_band, transA)
        ctx.save_for_backward(A, V)
        return P

    @staticmethod
    def backward(ctx, Pbar):
        A, V = ctx.saved_tensors
        a_band, transA = ctx.args
        Pbar = Pbar.contiguous()
        Abar = Vbar = None
        if ctx.needs_input_grad[1]:
            # Abar = band_A(Pbar V^T) (or band_A(V Pbar^T) when transposed)
            Abar = torch.zeros_like(A)
            if transA:
                B.banded_outer(ctx.plan.handle, V, Pbar, Abar, a_band[0], a_band[1], 0)
            else:
                B.banded_outer(ctx.plan.handle, Pbar, V, Abar, a_band[0], a_band[1], 0)
        if ctx.needs_input_grad[4]:
            Vbar = torch.zeros_like(V)
            B.banded_matvec(ctx.plan.handle, A, a_band[0], a_band[1], 1 - transA, Pbar, Vbar, 0)
        return None, Abar, None, None, Vbar


class GMMStep(torch.autograd.Function):
    """Fused (Q, B) -> (X = Q^{-1} B, S = band(Q^{-1}), logdet, L), with the fused
    backward kernels for the cotangents of X, S and logdet."""

    @staticmethod
    def forward(ctx, plan, Q, Bm):
        lay = plan.layout
        L, S, X = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Bm)
        logdet = torch.empty(lay.count, dtype=torch.float64, device=Q.device)
        info = torch.empty(lay.count, dtype=torch.int32, device=Q.device)
        B.banded_gmm_forward(plan.handle, Q.contiguous(), Bm.contiguous(), L, X, S, logdet, info)
        ctx.plan = plan
        ctx.save_for_backward(L, X, S)
        ctx.mark_non_differentiable(L, info)
        return X, S, logdet, L, info

    @staticmethod
    def backward(ctx, Xbar, Sbar, ldbar, _Lbar, _info):
        L, X, S = ctx.saved_tensors
        Xbar = _zeros_like_or(Xbar, X)
        Sbar = _zeros_like_or(Sbar, S)
        ldbar = None if ldbar is None else ldbar.contiguous().to(torch.float64)
        Qbar, Bbar = torch.zeros_like(L), torch.zeros_like(X)
        B.banded_gmm_backward(ctx.plan.handle, L, X, S, Xbar, Sbar, ldbar, Qbar, Bbar)
        return None, Qbar, Bbar


def cholesky(plan, Q):
    return Cholesky.apply(plan, Q)


def solve(plan, L, Bm, mode):
    return Solve.apply(plan, L, Bm, mode)


def subset_inverse(plan, L):
    return SubsetInverse.apply(plan, L)


def product(plan, A, a_band, transA, Bm, b_band, transB, c_band):
    return Product.apply(plan, A, tuple(a_band), int(transA), Bm, tuple(b_band), int(transB), tuple(c_band))


def matvec(plan, A, a_band, transA, V):
    return Matvec.apply(plan, A, tuple(a_band), int(transA), V)


class GMMStepRecompute(torch.autograd.Function):
    """GMMStep that keeps no Cholesky factor between the forward and the backward:
    the forward writes L to a temporary that it drops, and the backward
    recomputes L from Q (one Cholesky sweep) before the fused backward kernels.
    What autograd holds per batch is Q, X and S instead of L, X and S plus the
    caller's Q -- one band pool less, for batches that are processed in chunks
    because their saved tensors would not fit in HBM.  Results are bitwise those
    of GMMStep (the same kernels recompute the same L)."""

    @staticmethod
    def forward(ctx, plan, Q, Bm):
        lay = plan.layout
        L, S, X = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Bm)
        logdet = torch.empty(lay.count, dtype=torch.float64, device=Q.device)
        info = torch.empty(lay.count, dtype=torch.int32, device=Q.device)
        Qc = Q.contiguous()
        B.banded_gmm_forward(plan.handle, Qc, Bm.contiguous(), L, X, S, logdet, info)
        del L
        ctx.plan = plan
        ctx.save_for_backward(Qc, X, S)
        ctx.mark_non_differentiable(info)
        return X, S, logdet, info

    @staticmethod
    def backward(ctx, Xbar, Sbar, ldbar, _info):
        Q, X, S = ctx.saved_tensors
        lay = ctx.plan.layout
        L = torch.zeros_like(Q)
        logdet = torch.empty(lay.count, dtype=torch.float64, device=Q.device)
        info = torch.empty(lay.count, dtype=torch.int32, device=Q.device)
        B.banded_cholesky(ctx.plan.handle, Q, L, logdet, info)
        Xbar = _zeros_like_or(Xbar, X)
        Sbar = _zeros_like_or(Sbar, S)
        ldbar = None if ldbar is None else ldbar.contiguous().to(torch.float64)
        Qbar, Bbar = torch.zeros_like(L), torch.zeros_like(X)
        B.banded_gmm_backward(ctx.plan.handle, L, X, S, Xbar, Sbar, ldbar, Qbar, Bbar)
        return None, Qbar, Bbar


def gmm_step(plan, Q, Bm, recompute_L=False):
    """(X, S, logdet, L, info) of the fused step; with recompute_L the factor is
    not kept for the backward (L is returned as None) and is recomputed there."""
    if recompute_L:
        X, S, logdet, info = GMMStepRecompute.apply(plan, Q, Bm)
        return X, S, logdet, None, info
    return GMMStep.apply(plan, Q, Bm)
