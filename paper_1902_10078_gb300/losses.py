"""Losses of the precision-parameterised Gaussian models, composed from the
banded operators (Sec. 3).  The operators and their adjoints run in the CUDA
kernels; torch only forms elementwise products and reductions of their
outputs (accumulated in FP64).

Trace over lower-band storage: for symmetric A, B stored by their lower band,
tr(A B) = sum_j A_jj B_jj + 2 sum_{d>=1} sum_j A[d, j] B[d, j], because each
stored off-diagonal entry stands for two entries of the full matrix.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import autograd as AG


def symmetric_weights(layout, device="cuda"):
    """Band pool with 1 on the diagonal row, 2 on the off-diagonal rows, 0 at corners/padding."""
    w = torch.zeros(layout.band_elems, dtype=torch.float64)
    for i in range(layout.count):
        n, l = layout.ns[i], layout.ls[i]
        v = layout.band_view(w, i)
        v[0, :n] = 1.0
        for d in range(1, min(l, n - 1) + 1):
            v[d, : n - d] = 2.0
    return w.to(device=device)


def chain_loss(plan, Q, b, W, wsym, recompute_L=False):
    """-1/2 b^T Q^{-1} b + 1/2 log det Q + 1/2 tr(band(Q^{-1}) W), summed over instances.

    Q, W: band pools (W symmetric with the bandwidth of Q); b: RHS pool (k = 1);
    wsym: symmetric_weights(layout).  Differentiable in Q (and b) through the
    fused GMM step kernels; recompute_L keeps no Cholesky factor for the
    backward (it is recomputed from Q there)."""
    X, S, logdet, _L, info = AG.gmm_step(plan, Q, b, recompute_L=recompute_L)
    quad = (b.to(torch.float64) * X.to(torch.float64)).sum()
    trace = (wsym * S.to(torch.float64) * W.to(torch.float64)).sum()
    return -0.5 * quad + 0.5 * logdet.sum() + 0.5 * trace, info


def diagonal_mask(layout, device="cuda"):
    """Band pool with True on the stored diagonal entries (d = 0, j < n) of every instance."""
    w = torch.zeros(layout.band_elems, dtype=torch.bool)
    for i in range(layout.count):
        layout.band_view(w, i)[0, :] = True
    return w.to(device=device)


# ---------------------------------------------------------------------------
# Matern-3/2 state-space prior (Sec. 2: the state (f, f') of each input,
# interleaved, gives a prior precision of lower bandwidth 3).  Textbook SDE
# with lambda = sqrt(3) / ell:
#   A(D) = exp(-lambda D) [[1 + lambda D, D], [-lambda^2 D, 1 - lambda D]],
#   Pinf = diag(s2, lambda^2 s2),  Sigma(D) = Pinf - A Pinf A^T,
# and Q_p = M^T M with M block lower-bidiagonal: M_00 = C_0^{-1},
# M_kk = C_k^{-1}, M_k,k-1 = -C_k^{-1} A_k, C = lower Cholesky factors of Pinf
# and Sigma(t_k - t_{k-1}).  With x = lambda D and q = exp(-2x):
#   Sigma_00 = s2 (1 - q (1 + 2x + 2x^2)),  Sigma_01 = 2 s2 lambda x^2 q,
#   Sigma_11 = s2 lambda^2 (1 - q (1 - 2x + 2x^2)),
# where the brackets come from Taylor series for x < 1/2 (the difference
# cancels at small gaps).  Built in FP64 torch (elementwise work on the n
# 2x2 blocks); the band operators then run in the layout's dtype.
# ---------------------------------------------------------------------------

_SERIES_X = 0.5
_SERIES_TERMS = 40


def _bracket_coeffs(c1):
    """Coefficients b_k of 1 - exp(-2x)(1 + c1 x + 2x^2) = sum_{k>=1} b_k x^k."""
    out = []
    for k in range(1, _SERIES_TERMS + 1):
        a = (-2.0) ** k / math.factorial(k) + c1 * (-2.0) ** (k - 1) / math.factorial(k - 1)
        if k >= 2:
            a += 2.0 * (-2.0) ** (k - 2) / math.factorial(k - 2)
        out.append(-a)
    return out


_B_PLUS = _bracket_coeffs(2.0)
_B_MINUS = _bracket_coeffs(-2.0)


def _bracket(x, coeffs, c1):
    direct = 1.0 - torch.exp(-2.0 * x) * (1.0 + c1 * x + 2.0 * x * x)
    xs = torch.clamp(x, max=_SERIES_X)
    acc = torch.zeros_like(xs)
    for b in reversed(coeffs):            # Horner: sum_k b_k xs^k
        acc = (acc + b) * xs
    return torch.where(x < _SERIES_X, acc, direct)


class MaternPrior:
    """Prior factor M of a batch of Matern-3/2 processes (instance i of the
    layout is process i, N_i = 2 n_i states), built for all processes at once
    on flat tensors: the inputs of every process concatenated, gaps and
    blocks computed elementwise, one scatter into the band pool.  Inputs and
    pool indices are uploaded once; `band(ells)` is differentiable in the
    (count,) FP64 lengthscales."""

    def __init__(self, layout, ts, s2, device="cuda"):
        self.layout, self.s2, self.device = layout, float(s2), device
        ns = [len(t) for t in ts]
        self.t = torch.as_tensor(np.concatenate([np.asarray(t, dtype=np.float64) for t in ts]), device=device)
        self.proc = torch.repeat_interleave(torch.arange(len(ts), device=device),
                                            torch.as_tensor(ns, device=device))
        G = self.t.shape[0]
        # gap g joins inputs g and g+1 when both belong to the same process
        self.same = self.proc[1:] == self.proc[:-1]
        first = torch.ones(G, dtype=torch.bool, device=device)
        first[1:] = ~self.same
        self.first = first
        flat = torch.arange(layout.band_elems, dtype=torch.int64)
        self.index = torch.cat([layout.band_view(flat, i) for i in range(layout.count)], dim=1).to(device)
        del flat
        assert self.index.shape == (4, 2 * G), "every instance must be a process with l = 3 and N = 2 n"
        self.N = float(2 * G)

    def band(self, ells):
        s2 = self.s2
        lam_in = math.sqrt(3.0) / ells[self.proc]                        # per input
        D = self.t[1:] - self.t[:-1]
        lam = lam_in[1:]                                                 # per gap (the later input's process)
        x = torch.where(self.same, lam * D, torch.ones_like(D))          # unused gaps get a harmless value
        Dm = torch.where(self.same, D, torch.zeros_like(D))
        e = torch.exp(-x)
        q = torch.exp(-2.0 * x)
        s00 = s2 * _bracket(x, _B_PLUS, 2.0)
        s01 = 2.0 * s2 * lam * x * x * q
        s11 = s2 * lam * lam * _bracket(x, _B_MINUS, -2.0)
        # lower Cholesky factor of each input's conditional covariance:
        # Pinf for the first input of a process, Sigma(gap before it) otherwise
        f = self.first
        pad = torch.zeros(1, dtype=D.dtype, device=D.device)
        g00 = torch.cat([pad, torch.sqrt(s00)])
        g10 = torch.cat([pad, s01 / torch.sqrt(s00)])
        g11 = torch.cat([pad, torch.sqrt(s11 - (s01 * s01) / s00)])
        one = torch.ones_like(lam_in)
        c00 = torch.where(f, math.sqrt(s2) * one, g00)
        c10 = torch.where(f, torch.zeros_like(lam_in), g10)
        c11 = torch.where(f, lam_in * math.sqrt(s2), g11)
        i00, i11 = 1.0 / c00, 1.0 / c11
        i10 = -c10 / (c00 * c11)
        # sub-diagonal block of the later input of gap g: -C^{-1} A(gap)
        a00, a01, a10, a11 = e * (1.0 + x), e * Dm, -e * lam * x, e * (1.0 - x)
        j00, j10, j11 = i00[1:], i10[1:], i11[1:]
        z = torch.zeros_like(D)
        o00 = torch.where(self.same, -(j00 * a00), z)
        o01 = torch.where(self.same, -(j00 * a01), z)
        o10 = torch.where(self.same, -(j10 * a00 + j11 * a10), z)
        o11 = torch.where(self.same, -(j10 * a01 + j11 * a11), z)
        G = self.t.shape[0]
        vals = torch.zeros((4, 2 * G), dtype=torch.float64, device=self.device)
        vals[0, 0::2] = i00
        vals[0, 1::2] = i11
        vals[1, 0::2] = i10
        # block (k, k-1): entry (2k + a, 2k - 2 + c) on diagonal 2 + a - c, column 2(k-1) + c
        vals[2, 0:2 * G - 2:2] = o00
        vals[1, 1:2 * G - 2:2] = o01
        vals[3, 0:2 * G - 2:2] = o10
        vals[2, 1:2 * G - 2:2] = o11
        pool = torch.zeros(self.layout.band_elems, dtype=torch.float64, device=self.device)
        pool = pool.index_put((self.index.reshape(-1),), vals.reshape(-1))
        return pool.to(self.layout.torch_dtype)


def matern_kl(plan, prior, ells, Lq, m, wsym, dmask):
    """sum_i KL(N(m_i, (Lq_i Lq_i^T)^{-1}) || N(0, Q_p,i^{-1})) (Eq. 5 / Alg. 7 with a
    zero prior mean), with Q_p = M^T M from `prior` (a MaternPrior):

      KL = 1/2 [ tr(Q_p band(Q_q^{-1})) + m^T Q_p m - N + log det Q_q - log det Q_p ],

    tr over lower storage (wsym), m^T Q_p m = |M m|^2 (matvec), log det Q_q =
    2 sum log Lq_ii and log det Q_p = 2 sum log M_ii (M is lower triangular).
    Differentiable in Lq, m and ells through the band operators' adjoints."""
    M = prior.band(ells)
    Qp = AG.product(plan, M, (3, 0), 1, M, (3, 0), 0, (3, 0))
    Sq = AG.subset_inverse(plan, Lq)
    trace = (wsym * Qp.to(torch.float64) * Sq.to(torch.float64)).sum()
    Mm = AG.matvec(plan, M, (3, 0), 0, m)
    quad = (Mm.to(torch.float64) ** 2).sum()
    one = torch.ones((), dtype=Lq.dtype, device=Lq.device)
    logq = 2.0 * torch.log(torch.where(dmask, Lq, one).abs().to(torch.float64)).sum()
    logp = 2.0 * torch.log(torch.where(dmask, M, one).abs().to(torch.float64)).sum()
    return 0.5 * (trace + quad - prior.N + logq - logp)
