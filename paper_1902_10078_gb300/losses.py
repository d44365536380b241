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


def chain_loss(plan, Q, b, W, wsym):
    """-1/2 b^T Q^{-1} b + 1/2 log det Q + 1/2 tr(band(Q^{-1}) W), summed over instances.

    Q, W: band pools (W symmetric with the bandwidth of Q); b: RHS pool (k = 1);
    wsym: symmetric_weights(layout).  Differentiable in Q (and b) through the
    fused GMM step kernels."""
    X, S, logdet, _L, info = AG.gmm_step(plan, Q, b)
    quad = (b.to(torch.float64) * X.to(torch.float64)).sum()
    trace = (wsym * S.to(torch.float64) * W.to(torch.float64)).sum()
    return -0.5 * quad + 0.5 * logdet.sum() + 0.5 * trace, info


def diagonal_mask(layout, device="cuda"):
    """Band pool with True on the stored diagonal entries (d = 0, j < n) of every instance."""
    w = torch.zeros(layout.band_elems, dtype=torch.bool)
    for i in range(layout.count):
        layout.band_view(w, i)[0, :] = True
    return w.to(device=device)


def band_index(layout, device="cuda"):
    """Flat pool index of every stored entry: per instance an (rows, n) int64 view."""
    idx = torch.arange(layout.band_elems, dtype=torch.int64)
    return [layout.band_view(idx, i) for i in range(layout.count)]


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


def matern_M_blocks(t, ell, s2):
    """Blocks of M for one process: diagonal C_k^{-1} (k = 0..n-1) and
    sub-diagonal -C_k^{-1} A_k (k = 1..n-1), as (n, 2, 2) and (n-1, 2, 2)
    FP64 tensors differentiable in ell (a 0-d tensor)."""
    lam = math.sqrt(3.0) / ell
    D = t[1:] - t[:-1]
    x = lam * D
    e = torch.exp(-x)
    q = torch.exp(-2.0 * x)
    s00 = s2 * _bracket(x, _B_PLUS, 2.0)
    s01 = 2.0 * s2 * lam * x * x * q
    s11 = s2 * lam * lam * _bracket(x, _B_MINUS, -2.0)
    # lower Cholesky factors: C_0 of Pinf, C_k of Sigma(D_k)
    c00 = torch.cat([torch.sqrt(s2 * torch.ones_like(lam)).reshape(1), torch.sqrt(s00)])
    c10 = torch.cat([torch.zeros(1, dtype=t.dtype, device=t.device), s01 / torch.sqrt(s00)])
    c11 = torch.cat([(lam * math.sqrt(s2)).reshape(1), torch.sqrt(s11 - (s01 * s01) / s00)])
    # inverses of the lower 2x2 factors
    i00, i11 = 1.0 / c00, 1.0 / c11
    i10 = -c10 / (c00 * c11)
    # -C_k^{-1} A_k for k >= 1, A_k = e [[1 + x, D], [-lam x, 1 - x]]
    a00, a01, a10, a11 = e * (1.0 + x), e * D, -e * lam * x, e * (1.0 - x)
    j00, j10, j11 = i00[1:], i10[1:], i11[1:]
    o00 = -(j00 * a00)
    o01 = -(j00 * a01)
    o10 = -(j10 * a00 + j11 * a10)
    o11 = -(j10 * a01 + j11 * a11)
    return (i00, i10, i11), (o00, o01, o10, o11)


def matern_M_band(layout, index, ts, ells, s2, device="cuda"):
    """Band pool (lower bandwidth 3) holding M of every process, differentiable in
    `ells` (a (count,) FP64 tensor).  Instance i is process i with N = 2 n_i."""
    vals, idxs = [], []
    for i in range(layout.count):
        t = torch.as_tensor(ts[i], dtype=torch.float64, device=device)
        (i00, i10, i11), (o00, o01, o10, o11) = matern_M_blocks(t, ells[i], s2)
        n = t.shape[0]
        N = 2 * n
        rows = torch.zeros((4, N), dtype=torch.float64, device=device)
        rows[0, 0::2] = i00
        rows[0, 1::2] = i11
        rows[1, 0::2] = i10
        # block (k, k-1) at rows 2k, 2k+1 and columns 2k-2, 2k-1: entry (2k+a, 2k-2+c) on diagonal 2+a-c
        rows[2, 0:N - 2:2] = o00                  # (a, c) = (0, 0)
        rows[1, 1:N - 2:2] = o01                  # (0, 1)
        rows[3, 0:N - 2:2] = o10                  # (1, 0)
        rows[2, 1:N - 2:2] = o11                  # (1, 1)
        vals.append(rows.reshape(-1))
        idxs.append(index[i].reshape(-1).to(device))
    pool = torch.zeros(layout.band_elems, dtype=torch.float64, device=device)
    pool = pool.index_put((torch.cat(idxs),), torch.cat(vals))
    return pool.to(layout.torch_dtype)


def matern_kl(plan, index, ts, ells, s2, Lq, m, wsym, dmask):
    """sum_i KL(N(m_i, (Lq_i Lq_i^T)^{-1}) || N(0, Q_p,i^{-1})) (Eq. 5 / Alg. 7 with a
    zero prior mean), with Q_p = M^T M built from (t_i, ell_i, s2):

      KL = 1/2 [ tr(Q_p band(Q_q^{-1})) + m^T Q_p m - N + log det Q_q - log det Q_p ],

    tr over lower storage (wsym), m^T Q_p m = |M m|^2 (matvec), log det Q_q =
    2 sum log Lq_ii and log det Q_p = 2 sum log M_ii (M is lower triangular).
    Differentiable in Lq, m and ells through the band operators' adjoints."""
    lay = plan.layout
    M = matern_M_band(lay, index, ts, ells, s2, device=Lq.device)
    Qp = AG.product(plan, M, (3, 0), 1, M, (3, 0), 0, (3, 0))
    Sq = AG.subset_inverse(plan, Lq)
    trace = (wsym * Qp.to(torch.float64) * Sq.to(torch.float64)).sum()
    Mm = AG.matvec(plan, M, (3, 0), 0, m)
    quad = (Mm.to(torch.float64) ** 2).sum()
    one = torch.ones((), dtype=Lq.dtype, device=Lq.device)
    logq = 2.0 * torch.log(torch.where(dmask, Lq, one).abs().to(torch.float64)).sum()
    logp = 2.0 * torch.log(torch.where(dmask, M, one).abs().to(torch.float64)).sum()
    N = float(sum(2 * len(t) for t in ts))
    return 0.5 * (trace + quad - N + logq - logp)
