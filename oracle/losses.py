"""Oracle compositions of the workload losses (test infrastructure only).

Built from the C oracle's operators; numpy does only elementwise work and
reductions.

* ``chain_loss``: for a single banded SPD precision Q (lower band, l),
  ``loss = -1/2 b^T Q^{-1} b + 1/2 log det Q + 1/2 tr(band(Q^{-1}) W)`` with W a
  symmetric band matrix of the same bandwidth, and its gradient with respect to
  the lower stored entries of Q, composed per Table 1, Alg. 2 and Alg. 4.
* ``matern_kl``: the KL term of Eq. 5 / Alg. 7 for a Matern-3/2 state-space
  prior and a banded variational posterior (mean m, precision L_q L_q^T).

Trace over lower band storage (reading of Eq. 5 and of the trace terms):
``tr(A B) = sum_d0 A_jj B_jj + 2 sum_{d>=1} A[d, j] B[d, j]`` for symmetric A, B
stored as lower bands, because each stored off-diagonal entry stands for two
entries of the full matrix.
"""
from __future__ import annotations

import math

import numpy as np

from . import (cholesky, cholesky_vjp, logdet, product, solve, solve_vjp, subset_inverse,
               subset_inverse_vjp)


def sym_weights(l1: int) -> np.ndarray:
    """Per-diagonal multiplicity of a symmetric lower-band entry: 1 on d=0, 2 above."""
    w = np.full((l1, 1), 2.0)
    w[0] = 1.0
    return w


def trace_sym(A: np.ndarray, B: np.ndarray) -> float:
    return float(np.sum(sym_weights(A.shape[0]) * A * B))


def chain_loss(Q, b, W, grad: bool = True):
    """Returns (loss, Qbar) with Qbar the stored-entry gradient (lower band)."""
    L, info = cholesky(Q)
    if info:
        raise ValueError(f"not SPD (info={info})")
    Y = solve(L, b, 0)
    X = solve(L, Y, 1)                               # X = Q^{-1} b
    S = subset_inverse(L)                            # band(Q^{-1})
    ld = logdet(L)
    loss = -0.5 * float(b @ X) + 0.5 * ld + 0.5 * trace_sym(S, W)
    if not grad:
        return loss, None
    Xbar = -0.5 * b
    Sbar = 0.5 * W * sym_weights(W.shape[0])
    ldbar = 0.5
    Lbar = subset_inverse_vjp(L, S, Sbar)            # Alg. 4
    Ybar, Lb1 = solve_vjp(L, 1, X, Xbar)             # X = L^{-T} Y   (Table 1)
    _bbar, Lb2 = solve_vjp(L, 0, Y, Ybar)            # Y = L^{-1} b   (Table 1)
    Lbar = Lbar + Lb1 + Lb2
    Lbar[0] += 2.0 * ldbar / L[0]                    # d(2 sum log L_ii)
    Qbar = cholesky_vjp(L, Lbar)                     # Alg. 2
    return loss, Qbar


# ---------------------------------------------------------------------------
# Matern-3/2 state-space prior (Sec. 2: state (f, f') interleaved gives lower
# bandwidth 3).  Textbook SDE: lambda = sqrt(3)/ell,
#   A(D) = exp(-lambda D) [[1 + lambda D, D], [-lambda^2 D, 1 - lambda D]]
#   Pinf = diag(s2, lambda^2 s2),  Sigma(D) = Pinf - A Pinf A^T.
# The precision of the stacked states x_0..x_{n-1} is M^T M with M block
# lower-bidiagonal: M_00 = C_0^{-1}, M_kk = C_k^{-1}, M_{k,k-1} = -C_k^{-1} A_k,
# where C_0 = chol(Pinf) and C_k = chol(Sigma(t_k - t_{k-1})).
#
# Sigma(D) written out with x = lambda D, q = exp(-2x):
#   Sigma_00 = s2 (1 - q (1 + 2x + 2x^2))
#   Sigma_01 = 2 s2 lambda x^2 q
#   Sigma_11 = s2 lambda^2 (1 - q (1 - 2x + 2x^2))
# For small x, 1 - q (1 + 2x + 2x^2) = 4/3 x^3 + O(x^4) cancels catastrophically
# when formed as a difference (the gaps of the workload reach x ~ 1e-5), so
# both brackets are summed from their Taylor series below x = 1/2.
# ---------------------------------------------------------------------------

_SERIES_X = 0.5
_SERIES_TERMS = 40


def one_minus_exp_poly(x, c1):
    """1 - exp(-2x) (1 + c1 x + 2 x^2), elementwise, for c1 = +2 or -2."""
    x = np.asarray(x, dtype=np.float64)
    direct = 1.0 - np.exp(-2.0 * x) * (1.0 + c1 * x + 2.0 * x * x)
    xs = np.minimum(x, _SERIES_X)
    # coefficient of x^k in exp(-2x) (1 + c1 x + 2 x^2):
    #   (-2)^k / k! + c1 (-2)^(k-1) / (k-1)! + 2 (-2)^(k-2) / (k-2)!
    ser = np.zeros_like(xs)
    xk = np.ones_like(xs)
    for k in range(1, _SERIES_TERMS + 1):
        xk = xk * xs
        a = (-2.0) ** k / math.factorial(k) + c1 * (-2.0) ** (k - 1) / math.factorial(k - 1)
        if k >= 2:
            a += 2.0 * (-2.0) ** (k - 2) / math.factorial(k - 2)
        ser = ser - a * xk
    return np.where(x < _SERIES_X, ser, direct)


def matern_transition(D, ell, s2):
    lam = math.sqrt(3.0) / ell
    D = np.asarray(D, dtype=np.float64)
    x = lam * D
    e = np.exp(-x)
    A = np.empty(D.shape + (2, 2))
    A[..., 0, 0] = e * (1.0 + x)
    A[..., 0, 1] = e * D
    A[..., 1, 0] = -e * lam * x
    A[..., 1, 1] = e * (1.0 - x)
    Pinf = np.array([[s2, 0.0], [0.0, lam * lam * s2]])
    Sig = np.empty(D.shape + (2, 2))
    Sig[..., 0, 0] = s2 * one_minus_exp_poly(x, 2.0)
    Sig[..., 0, 1] = Sig[..., 1, 0] = 2.0 * s2 * lam * x * x * np.exp(-2.0 * x)
    Sig[..., 1, 1] = s2 * lam * lam * one_minus_exp_poly(x, -2.0)
    return A, Sig, Pinf


def chol2(S):
    """Lower Cholesky of a stack of 2x2 SPD matrices."""
    c00 = np.sqrt(S[..., 0, 0])
    c10 = S[..., 1, 0] / c00
    c11 = np.sqrt(S[..., 1, 1] - c10 * c10)
    Cm = np.zeros(S.shape)
    Cm[..., 0, 0], Cm[..., 1, 0], Cm[..., 1, 1] = c00, c10, c11
    return Cm


def inv_lower2(Cm):
    Ci = np.zeros(Cm.shape)
    Ci[..., 0, 0] = 1.0 / Cm[..., 0, 0]
    Ci[..., 1, 1] = 1.0 / Cm[..., 1, 1]
    Ci[..., 1, 0] = -Cm[..., 1, 0] / (Cm[..., 0, 0] * Cm[..., 1, 1])
    return Ci


def matern_M_band(t, ell, s2):
    """M in general band storage with (lo, up) = (3, 0), size N = 2n."""
    n = t.shape[0]
    N = 2 * n
    D = np.diff(t)
    A, Sig, Pinf = matern_transition(D, ell, s2)
    Cs = np.concatenate([chol2(Pinf)[None], chol2(Sig)], axis=0)     # (n, 2, 2)
    Ci = inv_lower2(Cs)                                               # diagonal blocks
    Off = -(Ci[1:] @ A)                                               # sub-diagonal blocks
    M = np.zeros((4, N))
    # diagonal block k occupies rows/cols 2k, 2k+1 (lower triangular 2x2)
    M[0, 0::2] = Ci[:, 0, 0]
    M[0, 1::2] = Ci[:, 1, 1]
    M[1, 0::2] = Ci[:, 1, 0]
    # off-diagonal block for k >= 1: rows 2k, 2k+1; cols 2k-2, 2k-1
    k = np.arange(1, n)
    # entry (2k+a, 2k-2+c) -> diagonal index d = 2 + a - c, column 2k-2+c
    for a in range(2):
        for c in range(2):
            d = 2 + a - c
            M[d, 2 * k - 2 + c] = Off[:, a, c]
    return M


def matern_precision(t, ell, s2):
    M = matern_M_band(t, ell, s2)
    # Q_p = M^T M, projected to lower band 3 (it has exactly bandwidth 3)
    return product(M, 3, 0, 1, M, 3, 0, 0, 3, 0)


def matern_kl(t, ell, s2, Lq, m):
    """KL(N(m, (Lq Lq^T)^{-1}) || N(0, Q_p^{-1})), Eq. 5 / Alg. 7 with m_p = 0.

    The prior precision comes factored, Q_p = M^T M with M lower triangular, so
    the two terms of Alg. 7 that use a factor of Q_p take M:
    ||L_p^T (m_p - m_q)||^2 = m^T Q_p m = ||M m||^2 and log det Q_p =
    2 sum log |M_ii|.  (A Cholesky factor of Q_p itself loses all accuracy at
    the workload's smallest gaps, where Q_p reaches 1e15 and more.)"""
    from . import band_matvec
    M = matern_M_band(t, ell, s2)
    Qp = product(M, 3, 0, 1, M, 3, 0, 0, 3, 0)
    Sq = subset_inverse(Lq)
    N = Lq.shape[1]
    tr = trace_sym(Sq, Qp)
    v = band_matvec(M, 3, 0, 0, np.asarray(m, dtype=np.float64)[None])[0]
    quad = float(v @ v)
    logs = 2.0 * float(np.sum(np.log(Lq[0]))) - 2.0 * float(np.sum(np.log(np.abs(M[0]))))
    return 0.5 * (tr + logs + quad - N)
