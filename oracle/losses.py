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


# ---------------------------------------------------------------------------
# Reverse mode of the Matern KL (Eq. 5 / Alg. 7 with Q_p = M^T M), composed
# from the oracle's operator adjoints (Table 1 for the product and the
# band-vector product, Alg. 4 for the subset inverse) and the derivative of
# M with respect to the lengthscale taken analytically from the closed forms
# above.
# ---------------------------------------------------------------------------

def matern_M_band_dell(t, ell, s2):
    """(M, dM/d ell) in (lo, up) = (3, 0) band storage.

    With lam = sqrt(3)/ell, x = lam D, e = exp(-x), q = e^2 (D a gap):
      dA/dlam = e [[-D x, -D^2], [lam D (x - 2), -D (2 - x)]]
      dSigma_00/dlam = 4 s2 x^2 q D
      dSigma_01/dlam = 2 s2 x^2 q (3 - 2x)
      dSigma_11/dlam = s2 (2 lam f(x) + 4 lam x (1 - x)^2 q),
        f(x) = 1 - q (1 - 2x + 2x^2)  (the Sigma_11 bracket)
    (from f'(x) = 4 x^2 e^{-2x} and 4 (1 - x)^2 e^{-2x} for the two brackets),
    then the chain rule through the 2x2 Cholesky factor, its inverse and
    -C^{-1} A, and d lam / d ell = -lam / ell."""
    lam = math.sqrt(3.0) / ell
    t = np.asarray(t, dtype=np.float64)
    n = t.shape[0]
    D = np.diff(t)
    A, Sig, Pinf = matern_transition(D, ell, s2)
    x = lam * D
    e = np.exp(-x)
    q = e * e
    dA = np.empty(D.shape + (2, 2))
    dA[..., 0, 0] = -e * D * x
    dA[..., 0, 1] = -e * D * D
    dA[..., 1, 0] = e * lam * D * (x - 2.0)
    dA[..., 1, 1] = -e * D * (2.0 - x)
    dS00 = 4.0 * s2 * x * x * q * D
    dS01 = 2.0 * s2 * x * x * q * (3.0 - 2.0 * x)
    dS11 = s2 * (2.0 * lam * one_minus_exp_poly(x, -2.0) + 4.0 * lam * x * (1.0 - x) ** 2 * q)
    # Cholesky factors of Sigma and their derivatives
    c00 = np.sqrt(Sig[..., 0, 0])
    c10 = Sig[..., 1, 0] / c00
    c11 = np.sqrt(Sig[..., 1, 1] - c10 * c10)
    dc00 = dS00 / (2.0 * c00)
    dc10 = (dS01 - c10 * dc00) / c00
    dc11 = (dS11 - 2.0 * c10 * dc10) / (2.0 * c11)
    # the first block uses chol(Pinf) = diag(sqrt(s2), lam sqrt(s2))
    rs = math.sqrt(s2)
    C00 = np.concatenate([[rs], c00])
    C10 = np.concatenate([[0.0], c10])
    C11 = np.concatenate([[lam * rs], c11])
    dC00 = np.concatenate([[0.0], dc00])
    dC10 = np.concatenate([[0.0], dc10])
    dC11 = np.concatenate([[rs], dc11])
    # inverse of the lower 2x2 factor [[c00, 0], [c10, c11]] and its derivative
    I00, I11 = 1.0 / C00, 1.0 / C11
    I10 = -C10 / (C00 * C11)
    dI00, dI11 = -dC00 / (C00 * C00), -dC11 / (C11 * C11)
    dI10 = -(dC10 * C00 * C11 - C10 * (dC00 * C11 + C00 * dC11)) / (C00 * C11) ** 2
    Ci = np.zeros((n, 2, 2))
    dCi = np.zeros((n, 2, 2))
    Ci[:, 0, 0], Ci[:, 1, 0], Ci[:, 1, 1] = I00, I10, I11
    dCi[:, 0, 0], dCi[:, 1, 0], dCi[:, 1, 1] = dI00, dI10, dI11
    Off = -(Ci[1:] @ A)
    dOff = -(dCi[1:] @ A + Ci[1:] @ dA)

    def band_of(Cd, Od):
        M = np.zeros((4, 2 * n))
        M[0, 0::2] = Cd[:, 0, 0]
        M[0, 1::2] = Cd[:, 1, 1]
        M[1, 0::2] = Cd[:, 1, 0]
        k = np.arange(1, n)
        for a in range(2):
            for c in range(2):
                M[2 + a - c, 2 * k - 2 + c] = Od[:, a, c]
        return M
    M = band_of(Ci, Off)
    dM_dlam = band_of(dCi, dOff)
    return M, dM_dlam * (-lam / ell)


def matern_kl_grad(t, ell, s2, Lq, m):
    """KL of matern_kl and its gradients (KL, Lq_bar, m_bar, ell_bar).

    KL = 1/2 [tr(Q_p S_q) + |M m|^2 - N + 2 sum log Lq_ii - 2 sum log|M_ii|],
    Q_p = band_3(M^T M), S_q = band_3((Lq Lq^T)^{-1}):
      S_q bar  = 1/2 w Q_p   (w: 1 on the diagonal, 2 off it: trace over lower storage)
      Lq bar   = Alg. 4 adjoint of S_q with S_q bar, plus 1/Lq_ii on the diagonal
      Q_p bar  = 1/2 w S_q;  M bar from the product adjoint of M^T M (Table 1)
      v = M m:  m bar = M^T v, M bar += band_3(v m^T)  (band-vector adjoint, Table 1)
      M bar_ii -= 1/M_ii;    ell bar = sum M bar * dM/d ell."""
    from . import band_matvec, band_matvec_vjp, product_vjp
    M, dM = matern_M_band_dell(t, ell, s2)
    Lq = np.asarray(Lq, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    N = Lq.shape[1]
    w = sym_weights(4)
    Qp = product(M, 3, 0, 1, M, 3, 0, 0, 3, 0)
    Sq = subset_inverse(Lq)
    v = band_matvec(M, 3, 0, 0, m[None])[0]
    kl = 0.5 * (trace_sym(Sq, Qp) + float(v @ v) - N + 2.0 * float(np.sum(np.log(Lq[0])))
                - 2.0 * float(np.sum(np.log(np.abs(M[0])))))
    Lq_bar = subset_inverse_vjp(Lq, Sq, _zero_corners(0.5 * w * Qp))
    Lq_bar[0] += 1.0 / Lq[0]
    Qp_bar = _zero_corners(0.5 * w * Sq)
    Ma, Mb = product_vjp(M, 3, 0, 1, M, 3, 0, 0, Qp_bar, 3, 0)
    M_bar = Ma + Mb
    Mv_bar, m_bar = band_matvec_vjp(M, 3, 0, 0, m[None], v[None])
    M_bar = M_bar + Mv_bar
    M_bar[0] -= 1.0 / M[0]
    ell_bar = float(np.sum(_zero_corners(M_bar) * _zero_corners(dM)))
    return kl, _zero_corners(Lq_bar), m_bar[0], ell_bar


def _zero_corners(band):
    """Zero the undefined corners band[d, j], j + d >= n, of a lower band."""
    band = np.array(band, dtype=np.float64)
    n = band.shape[1]
    for d in range(1, band.shape[0]):
        band[d, max(n - d, 0):] = 0.0
    return band


# ---------------------------------------------------------------------------
# Inference compositions of Sec. 3 (marginal likelihood with partial
# observations, whitened log joint for HMC, state-space GP regression through
# natural parameters), from the oracle's operators.
# ---------------------------------------------------------------------------

def marginal_likelihood(Q, obs, y, tau2, logdet_prior=None):
    """log p(y | theta) for f ~ N(0, Q^{-1}) (lower band storage) observed at the
    node indices `obs` with Gaussian noise tau2 (Sec. 3.1, marginal-likelihood
    equation with E the 0/1 selection of the observed nodes):
      -n/2 log 2 pi - log|L| + log|L_Q| - n/2 log tau2 - y^T y / (2 tau2)
      + |L^{-1} E^T y|^2 / (2 tau2^2),   L L^T = Q + E^T E / tau2,  L_Q L_Q^T = Q.
    `logdet_prior` replaces 2 log|L_Q| when the prior precision comes factored."""
    Q = np.asarray(Q, dtype=np.float64)
    obs = np.asarray(obs, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    n = obs.shape[0]
    Qpost = Q.copy()
    Qpost[0, obs] += 1.0 / tau2
    L, info = cholesky(Qpost)
    if info:
        raise ValueError("posterior precision not SPD")
    if logdet_prior is None:
        LQ, info = cholesky(Q)
        if info:
            raise ValueError("prior precision not SPD")
        logdet_prior = logdet(LQ)
    ey = np.zeros(Q.shape[1])
    ey[obs] = y
    R = solve(L, ey, 0)
    return (-0.5 * n * math.log(2 * math.pi) - 0.5 * logdet(L) + 0.5 * logdet_prior - 0.5 * n * math.log(tau2)
            - float(y @ y) / (2 * tau2) + float(R @ R) / (2 * tau2 * tau2))


def whitened_log_joint(Q, v, obs, y, tau2):
    """log p(v) + sum_i log N(y_i; F_i, tau2) with F = L_Q^{-T} v (Sec. 3.2 and the
    log-likelihood pseudocode for HMC; the parameter prior log p(theta) is the
    caller's)."""
    L, info = cholesky(Q)
    if info:
        raise ValueError("precision not SPD")
    v = np.asarray(v, dtype=np.float64)
    F = solve(L, v, 1)
    obs = np.asarray(obs, dtype=np.int64)
    r = np.asarray(y, dtype=np.float64) - F[obs]
    N = v.shape[0]
    return (-0.5 * N * math.log(2 * math.pi) - 0.5 * float(v @ v)
            - 0.5 * obs.shape[0] * math.log(2 * math.pi * tau2) - float(r @ r) / (2 * tau2))


def ssm_gpr_log_marginal(t, ell, s2, y, tau2):
    """log p(y) of GP regression with a Matern-3/2 kernel through its state-space
    form (App. C, GP regression with banded matrices): the states (f, f') of
    the inputs t have prior precision Q_p = M^T M; y observes every f with
    noise tau2.  Natural parameters: Lambda_post = Q_p + H^T H / tau2,
    eta_post = H^T y / tau2 (zero prior mean), and
      log p(y) = -T/2 log(2 pi tau2) - y^T y / (2 tau2) + 1/2 log|Q_p|
                 - 1/2 log|Lambda_post| + 1/2 |C_post^{-1} eta_post|^2,
    the same expression as marginal_likelihood with E selecting the f states
    (log|Q_p| = 2 sum log|M_ii| from the factor)."""
    M = matern_M_band(np.asarray(t, dtype=np.float64), ell, s2)
    Qp = product(M, 3, 0, 1, M, 3, 0, 0, 3, 0)
    obs = 2 * np.arange(len(t))
    return marginal_likelihood(Qp, obs, y, tau2, logdet_prior=2.0 * float(np.sum(np.log(np.abs(M[0])))))
