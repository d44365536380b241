"""Pins of the FP64 oracle against things other than itself.

Each operator of the oracle is checked against at least one of: dense
LAPACK/numpy, scipy's banded LAPACK wrappers (same storage convention),
closed forms (the 1-D Laplacian), exact special cases (chol(L0 L0^T) = L0),
invariants that hold at any n (the Takahashi identity), central finite
differences, and dense PyTorch autograd on tiny problems.  A dropped term, a
flipped sign, a wrong index or a transposed operand in any oracle function
makes at least one of these fail.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import torch

from paper_1902_10078_gb300 import workloads as W

dense_sym = lambda b: W.dense_from_lower_band(b, symmetric=True)   # noqa: E731
dense_low = lambda b: W.dense_from_lower_band(b, symmetric=False)  # noqa: E731

SHAPES = [(1, 1), (2, 1), (5, 2), (17, 3), (40, 5), (33, 8), (12, 0), (9, 12)]


def spd(n, l, seed=0):
    return W.spd_band(W.rng_for(seed), n, max(l, 0)) if l > 0 else np.abs(W.rng_for(seed).normal(size=(1, n))) + 1.0


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --------------------------------------------------------------------------- C

@pytest.mark.parametrize("n,l", SHAPES)
def test_cholesky_matches_dense_lapack(oracle, n, l):
    Q = spd(n, l, seed=n * 31 + l)
    L, info = oracle.cholesky(Q)
    assert info == 0
    Ld = np.linalg.cholesky(dense_sym(Q))
    assert rel(dense_low(L), Ld) < 1e-13


@pytest.mark.parametrize("n,l", [(50, 1), (64, 3), (200, 7)])
def test_cholesky_matches_scipy_banded_layout(oracle, n, l):
    # scipy's lower band layout ab[i - j, j] is exactly the storage of Sec. 4.3
    Q = spd(n, l, seed=7)
    L, _ = oracle.cholesky(Q)
    ref = sla.cholesky_banded(Q, lower=True)
    assert rel(L, ref) < 1e-13


@pytest.mark.parametrize("l", [1, 2, 5])
def test_cholesky_of_exact_gram_returns_factor(oracle, l):
    rng = W.rng_for(3)
    L0 = W.random_lower_factor(rng, 300, l)
    Q = W.gram_band(L0)          # no shift: chol(L0 L0^T) = L0 (positive diagonal)
    L, info = oracle.cholesky(Q)
    assert info == 0
    assert rel(L, L0) < 1e-12


def laplacian(n):
    Q = np.zeros((2, n))
    Q[0] = 2.0
    Q[1, : n - 1] = -1.0
    return Q


def test_laplacian_closed_forms(oracle):
    # tridiag(-1, 2, -1): L_ii = sqrt((i+2)/(i+1)), L_{i+1,i} = -sqrt((i+1)/(i+2)),
    # det = n + 1, (Q^{-1})_{ij} = (min(i,j)+1) (n - max(i,j)) / (n + 1)   (0-based)
    n = 25
    Q = laplacian(n)
    L, info = oracle.cholesky(Q)
    assert info == 0
    i = np.arange(n)
    assert rel(L[0], np.sqrt((i + 2) / (i + 1))) < 1e-15
    assert rel(L[1, : n - 1], -np.sqrt((i[:-1] + 1) / (i[:-1] + 2))) < 1e-15
    assert abs(oracle.logdet(L) - math.log(n + 1)) < 1e-13
    S = oracle.subset_inverse(L)
    exact = np.zeros((2, n))
    exact[0] = (i + 1) * (n - i) / (n + 1)
    exact[1, : n - 1] = (i[:-1] + 1) * (n - i[:-1] - 1) / (n + 1)
    assert rel(S, exact) < 1e-13


@pytest.mark.parametrize("n,l", SHAPES)
def test_logdet_matches_slogdet(oracle, n, l):
    Q = spd(n, l, seed=11)
    L, _ = oracle.cholesky(Q)
    sign, ref = np.linalg.slogdet(dense_sym(Q))
    assert sign > 0
    assert abs(oracle.logdet(L) - ref) < 1e-11 * max(1.0, abs(ref))


def test_not_spd_reports_first_failing_row(oracle):
    n, l = 30, 2
    Q = spd(n, l, seed=5)
    Q[0, 17] = -5.0                      # breaks positive definiteness at row 17 at the latest
    Qd = dense_sym(Q)
    first = next(k for k in range(1, n + 1) if np.linalg.eigvalsh(Qd[:k, :k]).min() <= 0)
    L, info = oracle.cholesky(Q)
    assert info == first                 # 1-based order of the first non-PD leading minor
    assert np.all(np.isnan(L[0, info - 1:]))
    good = info - 1
    assert rel(dense_low(L)[:good, :good], np.linalg.cholesky(Qd[:good, :good])) < 1e-13


# --------------------------------------------------------------------------- S

@pytest.mark.parametrize("n,l", SHAPES)
@pytest.mark.parametrize("trans", [0, 1])
def test_solve_matches_dense_triangular(oracle, n, l, trans):
    Q = spd(n, l, seed=2)
    L, _ = oracle.cholesky(Q)
    B = W.rng_for(9).normal(size=(3, n))
    X = oracle.solve(L, B, trans)
    ref = sla.solve_triangular(dense_low(L), B.T, lower=True, trans=trans).T
    assert rel(X, ref) < 1e-12


@pytest.mark.parametrize("n,l", [(100, 1), (257, 4), (64, 7)])
def test_precision_solve_matches_solveh_banded(oracle, n, l):
    Q = spd(n, l, seed=4)
    L, _ = oracle.cholesky(Q)
    b = W.rng_for(1).normal(size=n)
    x = oracle.solve_precision(L, b)
    ref = sla.solveh_banded(Q, b, lower=True)
    assert rel(x, ref) < 1e-12


# --------------------------------------------------------------------------- I

@pytest.mark.parametrize("n,l", SHAPES)
def test_subset_inverse_matches_dense_inverse(oracle, n, l):
    Q = spd(n, l, seed=13)
    L, _ = oracle.cholesky(Q)
    S = oracle.subset_inverse(L)
    ref = W.lower_band_from_dense(np.linalg.inv(dense_sym(Q)), Q.shape[0] - 1)
    assert rel(S, ref) < 1e-12


@pytest.mark.parametrize("l", [1, 3, 7])
def test_takahashi_identity_at_large_n(oracle, l):
    # Sigma = L^{-T} L^{-1} gives L^T Sigma = L^{-1}: (L^T Sigma)_{ij} = delta_ij / L_ii for
    # 0 <= j - i <= l, using only band entries of Sigma; and diag(Q Sigma) = 1.
    n = 4000
    Q = spd(n, l, seed=17)
    L, _ = oracle.cholesky(Q)
    S = oracle.subset_inverse(L)

    def sig(i, j):
        i, j = np.maximum(i, j), np.minimum(i, j)
        return S[i - j, j]

    worst = 0.0
    for e in range(l + 1):                       # j = i + e
        i = np.arange(0, n - e)
        acc = np.zeros(i.shape)
        for d in range(l + 1):                   # t = i + d, L[t, i] = L[d, i]
            t = i + d
            ok = t < n
            acc[ok] += L[d, i[ok]] * sig(t[ok], i[ok] + e)
        target = (1.0 / L[0, i]) if e == 0 else np.zeros(i.shape)
        worst = max(worst, float(np.max(np.abs(acc - target))))
    assert worst < 1e-12
    diag = np.zeros(n)
    for d in range(-l, l + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        t = i + d
        q = Q[abs(d), np.minimum(i, t)]
        diag[i] += q * sig(t, i)
    assert np.max(np.abs(diag - 1.0)) < 1e-12


# --------------------------------------------------------------------------- P / O

def band_from_dense_general(M, lo, up):
    n = M.shape[0]
    out = np.zeros((lo + up + 1, n))
    for r in range(lo + up + 1):
        off = r - up                  # i - j
        j = np.arange(max(0, -off), min(n, n - off))
        out[r, j] = M[j + off, j]
    return out


def dense_from_general(Bm, lo, up, n):
    M = np.zeros((n, n))
    for r in range(lo + up + 1):
        off = r - up
        j = np.arange(max(0, -off), min(n, n - off))
        M[j + off, j] = Bm[r, j]
    return M


def rand_general(n, lo, up, seed):
    Bm = W.rng_for(seed).normal(size=(lo + up + 1, n))
    return band_from_dense_general(dense_from_general(Bm, lo, up, n), lo, up)


PROD_CASES = [
    (20, (2, 0), 0, (2, 0), 1, (2, 2)),       # L L^T, full band
    (20, (2, 0), 0, (2, 0), 1, (2, 0)),       # L L^T projected to its lower band
    (25, (3, 0), 1, (3, 0), 0, (3, 3)),       # M^T M
    (17, (1, 2), 0, (2, 1), 0, (3, 3)),
    (17, (1, 2), 1, (0, 3), 1, (1, 1)),       # narrower projection
    (9, (3, 1), 0, (2, 2), 1, (6, 2)),
]


@pytest.mark.parametrize("n,a,ta,b,tb,c", PROD_CASES)
def test_product_matches_dense(oracle, n, a, ta, b, tb, c):
    A = rand_general(n, *a, seed=1)
    B = rand_general(n, *b, seed=2)
    Ad = dense_from_general(A, *a, n)
    Bd = dense_from_general(B, *b, n)
    ref = (Ad.T if ta else Ad) @ (Bd.T if tb else Bd)
    Cm = oracle.product(A, *a, ta, B, *b, tb, *c)
    assert rel(Cm, band_from_dense_general(ref, *c)) < 1e-13


@pytest.mark.parametrize("n,a,ta,b,tb,c", PROD_CASES)
def test_product_vjp_matches_autograd(oracle, n, a, ta, b, tb, c):
    A = rand_general(n, *a, seed=3)
    B = rand_general(n, *b, seed=4)
    Cbar = rand_general(n, *c, seed=5)
    Abar, Bbar = oracle.product_vjp(A, *a, ta, B, *b, tb, Cbar, *c)
    At = torch.tensor(dense_from_general(A, *a, n), requires_grad=True)
    Bt = torch.tensor(dense_from_general(B, *b, n), requires_grad=True)
    P = (At.T if ta else At) @ (Bt.T if tb else Bt)
    (P * torch.tensor(dense_from_general(Cbar, *c, n))).sum().backward()
    assert rel(Abar, band_from_dense_general(At.grad.numpy(), *a)) < 1e-12
    assert rel(Bbar, band_from_dense_general(Bt.grad.numpy(), *b)) < 1e-12


@pytest.mark.parametrize("trans", [0, 1])
def test_band_matvec_and_vjp(oracle, trans):
    n, lo, up = 23, 2, 1
    A = rand_general(n, lo, up, seed=6)
    V = W.rng_for(7).normal(size=(2, n))
    Pb = W.rng_for(8).normal(size=(2, n))
    Ad = dense_from_general(A, lo, up, n)
    op = Ad.T if trans else Ad
    assert rel(oracle.band_matvec(A, lo, up, trans, V), (op @ V.T).T) < 1e-13
    Abar, Vbar = oracle.band_matvec_vjp(A, lo, up, trans, V, Pb)
    At = torch.tensor(Ad, requires_grad=True)
    Vt = torch.tensor(V, requires_grad=True)
    ((At.T if trans else At) @ Vt.T * torch.tensor(Pb.T)).sum().backward()
    assert rel(Abar, band_from_dense_general(At.grad.numpy(), lo, up)) < 1e-12
    assert rel(Vbar, Vt.grad.numpy()) < 1e-12


def test_outer_and_vjp(oracle):
    n, lo, up = 19, 3, 1
    M = W.rng_for(1).normal(size=(3, n))
    V = W.rng_for(2).normal(size=(3, n))
    O = oracle.outer(M, V, lo, up)
    assert rel(O, band_from_dense_general(M.T @ V, lo, up)) < 1e-14
    Ob = rand_general(n, lo, up, seed=9)
    Mbar, Vbar = oracle.outer_vjp(M, V, Ob, lo, up)
    Mt = torch.tensor(M, requires_grad=True)
    Vt = torch.tensor(V, requires_grad=True)
    (Mt.T @ Vt * torch.tensor(dense_from_general(Ob, lo, up, n))).sum().backward()
    assert rel(Mbar, Mt.grad.numpy()) < 1e-13
    assert rel(Vbar, Vt.grad.numpy()) < 1e-13


# --------------------------------------------------------------------------- adjoints

def sym_from_stored(x, n, l):
    """Dense symmetric torch matrix from lower stored entries x (shape (l+1, n))."""
    M = torch.zeros((n, n), dtype=torch.float64)
    for d in range(min(l + 1, n)):
        j = torch.arange(0, n - d)
        M = M.index_put((j + d, j), x[d, : n - d], accumulate=True)
        if d > 0:
            M = M.index_put((j, j + d), x[d, : n - d], accumulate=True)
    return M


def low_from_stored(x, n, l):
    M = torch.zeros((n, n), dtype=torch.float64)
    for d in range(min(l + 1, n)):
        j = torch.arange(0, n - d)
        M = M.index_put((j + d, j), x[d, : n - d], accumulate=True)
    return M


def stored_of(M, l):
    n = M.shape[0]
    out = torch.zeros((l + 1, n), dtype=M.dtype)
    for d in range(min(l + 1, n)):
        j = torch.arange(0, n - d)
        out[d, : n - d] = M[j + d, j]
    return out


@pytest.mark.parametrize("n,l", [(1, 1), (6, 1), (15, 2), (24, 3), (20, 7)])
def test_cholesky_vjp_matches_autograd(oracle, n, l):
    Q = spd(n, l, seed=21)
    L, _ = oracle.cholesky(Q)
    Lbar = W.zero_corners(W.rng_for(22).normal(size=Q.shape))
    Qbar = oracle.cholesky_vjp(L, Lbar)
    x = torch.tensor(Q, requires_grad=True)
    Lt = torch.linalg.cholesky(sym_from_stored(x, n, l))
    (stored_of(Lt, l) * torch.tensor(Lbar)).sum().backward()
    g = W.zero_corners(x.grad.numpy().copy())
    assert rel(Qbar, g) < 1e-11


@pytest.mark.parametrize("n,l", [(1, 1), (7, 1), (15, 2), (24, 3), (20, 7)])
def test_subset_inverse_vjp_matches_autograd(oracle, n, l):
    Q = spd(n, l, seed=31)
    L, _ = oracle.cholesky(Q)
    S = oracle.subset_inverse(L)
    Sbar = W.zero_corners(W.rng_for(32).normal(size=Q.shape))
    Lbar = oracle.subset_inverse_vjp(L, S, Sbar)
    x = torch.tensor(L, requires_grad=True)
    Lt = low_from_stored(x, n, l)
    Sig = torch.linalg.inv(Lt @ Lt.T)
    (stored_of(Sig, l) * torch.tensor(Sbar)).sum().backward()
    g = W.zero_corners(x.grad.numpy().copy())
    assert rel(Lbar, g) < 1e-10


def test_subset_inverse_vjp_central_fd(oracle):
    n, l = 40, 3
    Q = spd(n, l, seed=41)
    L, _ = oracle.cholesky(Q)
    Sbar = W.zero_corners(W.rng_for(42).normal(size=Q.shape))
    Lbar = oracle.subset_inverse_vjp(L, oracle.subset_inverse(L), Sbar)
    rng = W.rng_for(43)
    for _ in range(12):
        d, j = int(rng.integers(0, l + 1)), int(rng.integers(0, n))
        if j + d >= n:
            continue
        h = 1e-5 * max(1.0, abs(L[d, j]))
        Lp, Lm = L.copy(), L.copy()
        Lp[d, j] += h
        Lm[d, j] -= h
        fd = (np.sum(oracle.subset_inverse(Lp) * Sbar) - np.sum(oracle.subset_inverse(Lm) * Sbar)) / (2 * h)
        assert abs(fd - Lbar[d, j]) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("n,l", [(1, 1), (9, 2), (20, 4)])
def test_solve_vjp_matches_autograd(oracle, trans, n, l):
    Q = spd(n, l, seed=51)
    L, _ = oracle.cholesky(Q)
    V = W.rng_for(52).normal(size=(2, n))
    Sb = W.rng_for(53).normal(size=(2, n))
    S = oracle.solve(L, V, trans)
    Vbar, Lbar = oracle.solve_vjp(L, trans, S, Sb)
    x = torch.tensor(L, requires_grad=True)
    Vt = torch.tensor(V, requires_grad=True)
    Lt = low_from_stored(x, n, l)
    A = Lt.T if trans else Lt
    St = torch.linalg.solve_triangular(A, Vt.T, upper=bool(trans))
    (St.T * torch.tensor(Sb)).sum().backward()
    assert rel(Vbar, Vt.grad.numpy()) < 1e-11
    assert rel(Lbar, W.zero_corners(x.grad.numpy().copy())) < 1e-11


# --------------------------------------------------------------------------- losses

def test_chain_loss_matches_closed_form(oracle):
    from oracle.losses import chain_loss
    n, l = 120, 3
    rng = W.rng_for(61)
    Q = W.spd_band(rng, n, l)
    b = rng.normal(size=n)
    Wt = W.symmetric_band_weights(rng, n, l)
    loss, Qbar = chain_loss(Q, b, Wt)
    Qd, Wd = dense_sym(Q), dense_sym(Wt)
    Qi = np.linalg.inv(Qd)
    Sband = dense_sym(W.lower_band_from_dense(Qi, l))
    ref_loss = -0.5 * b @ Qi @ b + 0.5 * np.linalg.slogdet(Qd)[1] + 0.5 * np.trace(Sband @ Wd)
    assert abs(loss - ref_loss) < 1e-11 * max(1.0, abs(ref_loss))
    # G = 1/2 Q^-1 b b^T Q^-1 + 1/2 Q^-1 - 1/2 Q^-1 W Q^-1; stored-entry gradient G_ii, 2 G_ij
    x = Qi @ b
    G = 0.5 * np.outer(x, x) + 0.5 * Qi - 0.5 * Qi @ Wd @ Qi
    ref = W.lower_band_from_dense(G, l)
    ref[1:] *= 2.0
    assert rel(Qbar, W.zero_corners(ref)) < 1e-10


def test_chain_loss_central_fd(oracle):
    from oracle.losses import chain_loss
    n, l = 400, 3
    rng = W.rng_for(71)
    Q = W.spd_band(rng, n, l)
    b = rng.normal(size=n)
    Wt = W.symmetric_band_weights(rng, n, l)
    _, Qbar = chain_loss(Q, b, Wt)
    for _ in range(10):
        d, j = int(rng.integers(0, l + 1)), int(rng.integers(0, n - l))
        h = 1e-4 * max(1.0, abs(Q[d, j]))
        Qp, Qm = Q.copy(), Q.copy()
        Qp[d, j] += h
        Qm[d, j] -= h
        fd = (chain_loss(Qp, b, Wt, grad=False)[0] - chain_loss(Qm, b, Wt, grad=False)[0]) / (2 * h)
        assert abs(fd - Qbar[d, j]) < 1e-6 * max(1.0, abs(fd))


def test_batch_step_matches_dense_autograd(oracle):
    insts = [W.make_instance(n, l, 2, 100 + i) for i, (n, l) in enumerate([(9, 1), (14, 2), (20, 3), (11, 5)])]
    res, threads = oracle.batch_step(insts)
    assert threads >= 1
    for ins, r in zip(insts, res):
        n, l = ins.n, ins.l
        x = torch.tensor(ins.Q, requires_grad=True)
        Bt = torch.tensor(ins.B, requires_grad=True)
        Qd = sym_from_stored(x, n, l)
        X = torch.linalg.solve(Qd, Bt.T).T
        Sig = torch.linalg.inv(Qd)
        ld = torch.linalg.slogdet(Qd)[1]
        loss = (X * torch.tensor(ins.Xbar)).sum() + (stored_of(Sig, l) * torch.tensor(ins.Sbar)).sum() + ins.ldbar * ld
        loss.backward()
        assert r["info"] == 0
        assert rel(r["X"], X.detach().numpy()) < 1e-12
        assert rel(r["S"], W.zero_corners(stored_of(Sig, l).detach().numpy())) < 1e-12
        ldv = float(ld.detach())
        assert abs(r["logdet"] - ldv) < 1e-12 * max(1, abs(ldv))
        assert rel(r["Qbar"], W.zero_corners(x.grad.numpy().copy())) < 1e-10
        assert rel(r["Bbar"], Bt.grad.numpy()) < 1e-11


# --------------------------------------------------------------------------- Matern prior / KL

def matern_dense_cov(t, ell, s2):
    """Joint covariance of (f(t_0), f'(t_0), f(t_1), ...) from the Matern-3/2 kernel
    k(tau) = s2 (1 + lam |tau|) exp(-lam |tau|) and its derivatives."""
    lam = math.sqrt(3.0) / ell
    n = t.shape[0]
    K = np.zeros((2 * n, 2 * n))
    for a in range(n):
        for b in range(n):
            tau = t[a] - t[b]
            e = math.exp(-lam * abs(tau))
            kff = s2 * (1 + lam * abs(tau)) * e
            kfd = s2 * lam * lam * tau * e          # cov(f(t_a), f'(t_b))
            kdd = s2 * lam * lam * (1 - lam * abs(tau)) * e
            K[2 * a, 2 * b] = kff
            K[2 * a, 2 * b + 1] = kfd
            K[2 * a + 1, 2 * b] = -kfd                 # cov(f'(t_a), f(t_b))
            K[2 * a + 1, 2 * b + 1] = kdd
    return K


def test_matern_precision_matches_kernel_inverse(oracle):
    from oracle.losses import matern_precision
    rng = W.rng_for(81)
    n = 15
    t = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0, n - 1) + 0.05)])
    ell, s2 = 2.0, 1.3
    Qp = matern_precision(t, ell, s2)
    ref = np.linalg.inv(matern_dense_cov(t, ell, s2))
    assert np.max(np.abs(W.lower_band_from_dense(ref, 3) - Qp)) < 1e-9 * np.max(np.abs(ref))
    # and Q_p really is banded with lower bandwidth 3
    assert np.max(np.abs(np.tril(ref, -4))) < 1e-9 * np.max(np.abs(ref))


def test_matern_kl_matches_dense_gaussian_kl(oracle):
    from oracle.losses import matern_kl, matern_precision
    rng = W.rng_for(91)
    n = 12
    t = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0, n - 1) + 0.05)])
    ell, s2 = 1.5, 1.0
    N = 2 * n
    Lq = np.zeros((4, N))
    Lq[0] = 1.0 + 0.1 * rng.uniform(size=N)
    Lq[1:] = rng.normal(0.0, 0.05, (3, N))
    W.zero_corners(Lq)
    m = rng.normal(0.0, 0.1, N)
    kl = matern_kl(t, ell, s2, Lq, m)
    Qp = dense_sym(matern_precision(t, ell, s2))
    Lqd = dense_low(Lq)
    Sq = np.linalg.inv(Lqd @ Lqd.T)
    ref = 0.5 * (np.trace(Qp @ Sq) + m @ Qp @ m - N + np.linalg.slogdet(np.linalg.inv(Qp))[1]
                 - np.linalg.slogdet(Sq)[1])
    assert abs(kl - ref) < 1e-9 * max(1.0, abs(ref))


def test_matern_sigma_matches_definition_and_high_precision(oracle):
    """Sigma(D) = Pinf - A Pinf A^T: the closed form agrees with the matrix
    definition where the difference is well conditioned, and with a 50-digit
    evaluation of the definition at tiny gaps, where the plain difference
    cancels (relative error of the closed form <= 1e-13 everywhere)."""
    import mpmath
    from oracle.losses import matern_transition
    ell, s2 = 0.7, 1.3
    lam = math.sqrt(3.0) / ell
    D = np.array([1e-7, 3e-6, 1e-4, 2e-3, 0.05, 0.2, 0.28, 0.3, 0.5, 1.0, 4.0, 20.0])
    A, Sig, Pinf = matern_transition(D, ell, s2)
    plain = Pinf - A @ Pinf @ np.swapaxes(A, -1, -2)
    big = D * lam > 0.6
    assert np.max(np.abs(Sig[big] - plain[big]) / np.abs(plain[big]).max(axis=(1, 2), keepdims=True)) < 1e-13
    mpmath.mp.dps = 50
    for i, d in enumerate(D):
        L, dd = mpmath.mpf(lam), mpmath.mpf(float(d))
        e = mpmath.exp(-L * dd)
        Am = mpmath.matrix([[e * (1 + L * dd), e * dd], [-e * L * L * dd, e * (1 - L * dd)]])
        Pm = mpmath.matrix([[s2, 0], [0, L * L * s2]])
        Sm = Pm - Am * Pm * Am.T
        for a in range(2):
            for b in range(2):
                ref = float(Sm[a, b])
                assert abs(Sig[i, a, b] - ref) <= 1e-13 * abs(ref), (d, a, b, Sig[i, a, b], ref)


def test_matern_kl_at_tiny_gaps_matches_high_precision(oracle):
    """With a gap of 1e-6 the prior precision reaches ~1e17: the oracle KL
    (closed-form Sigma, factor M for the quadratic term and the log-det) still
    matches a 60-digit dense evaluation of the Gaussian KL."""
    import mpmath
    from oracle.losses import matern_kl
    mpmath.mp.dps = 60
    rng = W.rng_for(97)
    n = 6
    gaps = np.array([0.7, 1e-6, 1.3, 0.2, 2e-4])
    t = np.concatenate([[0.0], np.cumsum(gaps)])
    ell, s2 = 1.1, 1.0
    N = 2 * n
    Lq = np.zeros((4, N))
    Lq[0] = 1.0 + 0.1 * rng.uniform(size=N)
    Lq[1:] = rng.normal(0.0, 0.05, (3, N))
    W.zero_corners(Lq)
    m = rng.normal(0.0, 0.1, N)
    kl = matern_kl(t, ell, s2, Lq, m)
    lam = mpmath.sqrt(3) / ell
    K = mpmath.matrix(N, N)
    for a in range(n):
        for b in range(n):
            tau = mpmath.mpf(float(t[a])) - mpmath.mpf(float(t[b]))
            e = mpmath.exp(-lam * abs(tau))
            K[2 * a, 2 * b] = s2 * (1 + lam * abs(tau)) * e
            K[2 * a, 2 * b + 1] = s2 * lam * lam * tau * e
            K[2 * a + 1, 2 * b] = -s2 * lam * lam * tau * e
            K[2 * a + 1, 2 * b + 1] = s2 * lam * lam * (1 - lam * abs(tau)) * e
    Qp = mpmath.inverse(K)
    Ld = mpmath.matrix(N, N)
    for d in range(4):
        for j in range(N - d):
            Ld[j + d, j] = mpmath.mpf(float(Lq[d, j]))
    Qq = Ld * Ld.T
    Sq = mpmath.inverse(Qq)
    mv = mpmath.matrix([mpmath.mpf(float(x)) for x in m])
    tr = sum(Qp[i, j] * Sq[j, i] for i in range(N) for j in range(N))
    quad = (mv.T * Qp * mv)[0]
    ref = 0.5 * (tr + quad - N + mpmath.log(mpmath.det(Qq)) - mpmath.log(mpmath.det(Qp)))
    assert abs(kl - float(ref)) <= 1e-9 * abs(float(ref)), (kl, float(ref))


def _matern_kernel_cov_torch(t, ell, s2):
    """The joint (f, f') covariance of matern_dense_cov, as a torch function of ell
    (autograd pins the lengthscale gradient through the kernel, not the SDE)."""
    lam = math.sqrt(3.0) / ell
    tt = torch.tensor(t, dtype=torch.float64)
    tau = tt[:, None] - tt[None, :]
    a = tau.abs()
    e = torch.exp(-lam * a)
    n = t.shape[0]
    K = torch.zeros((2 * n, 2 * n), dtype=torch.float64)
    K[0::2, 0::2] = s2 * (1 + lam * a) * e
    K[0::2, 1::2] = s2 * lam * lam * tau * e
    K[1::2, 0::2] = -s2 * lam * lam * tau * e
    K[1::2, 1::2] = s2 * lam * lam * (1 - lam * a) * e
    return K


def test_matern_kl_grad_matches_dense_autograd(oracle):
    """The composed KL adjoint (product, band-vector and Alg. 4 adjoints, dM/d ell in
    closed form) against torch autograd of the dense Gaussian KL whose prior
    precision is the inverse of the kernel covariance."""
    from oracle.losses import matern_kl_grad
    rng = W.rng_for(93)
    n = 10
    t = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0, n - 1) + 0.05)])
    ell0, s2 = 1.7, 1.0
    N = 2 * n
    Lq = np.zeros((4, N))
    Lq[0] = 1.0 + 0.1 * rng.uniform(size=N)
    Lq[1:] = rng.normal(0.0, 0.05, (3, N))
    W.zero_corners(Lq)
    m = rng.normal(0.0, 0.1, N)
    kl, gL, gm, ge = matern_kl_grad(t, ell0, s2, Lq, m)
    ell = torch.tensor(ell0, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(Lq, requires_grad=True)
    mt = torch.tensor(m, requires_grad=True)
    K = _matern_kernel_cov_torch(t, ell, s2)
    Qp = torch.linalg.inv(K)
    Lt = low_from_stored(x, N, 3)
    Sq = torch.linalg.inv(Lt @ Lt.T)
    ref = 0.5 * (torch.trace(Qp @ Sq) + mt @ Qp @ mt - N + torch.logdet(Lt @ Lt.T) + torch.logdet(K))
    ref.backward()
    assert abs(kl - float(ref.detach())) < 1e-10 * abs(float(ref.detach()))
    assert abs(ge - float(ell.grad)) < 1e-8 * abs(float(ell.grad)), (ge, float(ell.grad))
    assert rel(gL, W.zero_corners(x.grad.numpy().copy())) < 1e-9
    assert rel(gm, mt.grad.numpy()) < 1e-9


def test_matern_kl_grad_at_tiny_gaps_matches_high_precision(oracle):
    """Gaps of 1e-6 and 2e-4 (the workload's smallest are of that order): the
    lengthscale gradient against a 60-digit central difference of the dense KL,
    and the m and Lq gradients against the 60-digit dense gradient formulas
    (m bar = Q_p m; Lq bar = -(Q_q^{-1} Q_p Q_q^{-1}) Lq + Lq^{-T} restricted to the band)."""
    import mpmath
    from oracle.losses import matern_kl_grad
    mpmath.mp.dps = 60
    rng = W.rng_for(97)
    n = 6
    gaps = np.array([0.7, 1e-6, 1.3, 0.2, 2e-4])
    t = np.concatenate([[0.0], np.cumsum(gaps)])
    ell0, s2 = 1.1, 1.0
    N = 2 * n
    Lq = np.zeros((4, N))
    Lq[0] = 1.0 + 0.1 * rng.uniform(size=N)
    Lq[1:] = rng.normal(0.0, 0.05, (3, N))
    W.zero_corners(Lq)
    m = rng.normal(0.0, 0.1, N)
    kl, gL, gm, ge = matern_kl_grad(t, ell0, s2, Lq, m)

    def prior_precision(ell):
        lam = mpmath.sqrt(3) / ell
        K = mpmath.matrix(N, N)
        for a in range(n):
            for b in range(n):
                tau = mpmath.mpf(float(t[a])) - mpmath.mpf(float(t[b]))
                e = mpmath.exp(-lam * abs(tau))
                K[2 * a, 2 * b] = s2 * (1 + lam * abs(tau)) * e
                K[2 * a, 2 * b + 1] = s2 * lam * lam * tau * e
                K[2 * a + 1, 2 * b] = -s2 * lam * lam * tau * e
                K[2 * a + 1, 2 * b + 1] = s2 * lam * lam * (1 - lam * abs(tau)) * e
        return mpmath.inverse(K)

    Ld = mpmath.matrix(N, N)
    for d in range(4):
        for j in range(N - d):
            Ld[j + d, j] = mpmath.mpf(float(Lq[d, j]))
    Sq = mpmath.inverse(Ld * Ld.T)
    mv = mpmath.matrix([mpmath.mpf(float(v)) for v in m])

    def kl_of(ell):
        Qp = prior_precision(ell)
        tr = sum(Qp[i, j] * Sq[j, i] for i in range(N) for j in range(N))
        return 0.5 * (tr + (mv.T * Qp * mv)[0] - N + mpmath.log(mpmath.det(Ld * Ld.T)) - mpmath.log(mpmath.det(Qp)))

    e0 = mpmath.mpf(ell0)
    h = mpmath.mpf("1e-25")
    ref_ge = float((kl_of(e0 + h) - kl_of(e0 - h)) / (2 * h))
    assert abs(ge - ref_ge) <= 1e-8 * abs(ref_ge), (ge, ref_ge)
    Qp = prior_precision(e0)
    ref_gm = np.array([float(v) for v in (Qp * mv)])
    assert rel(gm, ref_gm) < 1e-9
    G = -(Sq * Qp * Sq) * Ld + mpmath.inverse(Ld).T     # d KL / d L (dense), lower part is the stored gradient
    ref_gL = np.zeros_like(Lq)
    for d in range(4):
        for j in range(N - d):
            ref_gL[d, j] = float(G[j + d, j])
    assert rel(gL, ref_gL) < 1e-9


# --------------------------------------------------------------------------- Alg. 5 (banded RHS)

def _gdense(B, lo, up, n):
    M = np.zeros((n, n))
    for r in range(lo + up + 1):
        k = r - up
        for c in range(n):
            if 0 <= c + k < n:
                M[c + k, c] = B[r, c]
    return M


def _gband(M, lo, up):
    n = M.shape[0]
    B = np.zeros((lo + up + 1, n))
    for r in range(lo + up + 1):
        k = r - up
        for c in range(n):
            if 0 <= c + k < n:
                B[r, c] = M[c + k, c]
    return B


@pytest.mark.parametrize("trans,olo,oup", [(0, 2, 3), (0, 5, 4), (1, 1, 4), (1, 3, 6)])
@pytest.mark.parametrize("n,l", [(1, 2), (9, 2), (30, 4)])
def test_solve_band_matches_dense(oracle, n, l, trans, olo, oup):
    Q = spd(n, l, seed=61)
    L, _ = oracle.cholesky(Q)
    rlo, rup = 1, 3
    R = _gband(_gdense(W.rng_for(62).normal(size=(rlo + rup + 1, n)), rlo, rup, n), rlo, rup)
    O = oracle.solve_band(L, R, rlo, rup, trans, olo, oup)
    Ld = W.dense_from_lower_band(L, False)
    ref = np.linalg.solve(Ld.T if trans else Ld, _gdense(R, rlo, rup, n))
    assert rel(O, _gband(ref, olo, oup)) < 1e-13


@pytest.mark.parametrize("trans", [0, 1])
def test_solve_band_vjp_matches_autograd(oracle, trans):
    n, l = 14, 3
    rlo, rup = 2, 2
    olo, oup = (3, 2) if trans == 0 else (2, 4)
    Q = spd(n, l, seed=63)
    L, _ = oracle.cholesky(Q)
    rng = W.rng_for(64)
    R = _gband(_gdense(rng.normal(size=(rlo + rup + 1, n)), rlo, rup, n), rlo, rup)
    O = oracle.solve_band(L, R, rlo, rup, trans, olo, oup)
    Obar = _gband(_gdense(rng.normal(size=(olo + oup + 1, n)), olo, oup, n), olo, oup)
    Rbar, Lbar = oracle.solve_band_vjp(L, trans, O, olo, oup, Obar, rlo, rup)
    Lt = torch.tensor(W.dense_from_lower_band(L, False), requires_grad=True)
    Rt = torch.tensor(_gdense(R, rlo, rup, n), requires_grad=True)
    Od = torch.linalg.solve_triangular(Lt.T if trans else Lt, Rt, upper=bool(trans))
    (Od * torch.tensor(_gdense(Obar, olo, oup, n))).sum().backward()
    assert rel(Rbar, _gband(Rt.grad.numpy(), rlo, rup)) < 1e-12
    assert rel(Lbar, W.lower_band_from_dense(Lt.grad.numpy(), l)) < 1e-12


# --------------------------------------------------------------------------- Sec. 3 inference compositions

def test_marginal_likelihood_matches_dense_gaussian(oracle):
    from oracle.losses import marginal_likelihood
    n, l = 40, 3
    Q = spd(n, l, seed=71)
    rng = W.rng_for(72)
    obs = np.sort(rng.choice(n, size=15, replace=False))
    y = rng.normal(size=15)
    tau2 = 0.3
    got = marginal_likelihood(Q, obs, y, tau2)
    K = np.linalg.inv(W.dense_from_lower_band(Q, True))[np.ix_(obs, obs)] + tau2 * np.eye(15)
    ref = -0.5 * (15 * math.log(2 * math.pi) + np.linalg.slogdet(K)[1] + y @ np.linalg.solve(K, y))
    assert abs(got - ref) < 1e-10 * abs(ref)


def test_whitened_log_joint_matches_dense(oracle):
    from oracle.losses import whitened_log_joint
    n, l = 30, 2
    Q = spd(n, l, seed=73)
    rng = W.rng_for(74)
    v = rng.normal(size=n)
    obs = np.array([0, 3, 7, 8, 20, 29])
    y = rng.normal(size=obs.shape[0])
    tau2 = 0.5
    got = whitened_log_joint(Q, v, obs, y, tau2)
    Ld = np.linalg.cholesky(W.dense_from_lower_band(Q, True))
    F = np.linalg.solve(Ld.T, v)                 # F ~ N(0, Q^{-1}) when v ~ N(0, I)
    ref = (-0.5 * n * math.log(2 * math.pi) - 0.5 * v @ v
           + sum(-0.5 * math.log(2 * math.pi * tau2) - (y[i] - F[o]) ** 2 / (2 * tau2) for i, o in enumerate(obs)))
    assert abs(got - ref) < 1e-11 * abs(ref)


def test_ssm_gpr_matches_kernel_regression(oracle):
    """The state-space marginal likelihood equals the dense GP marginal likelihood
    with the Matern-3/2 kernel matrix of the inputs (an independent route)."""
    from oracle.losses import ssm_gpr_log_marginal
    rng = W.rng_for(75)
    n = 25
    t = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0, n - 1) + 0.01)])
    ell, s2, tau2 = 1.3, 0.8, 0.2
    y = rng.normal(size=n)
    got = ssm_gpr_log_marginal(t, ell, s2, y, tau2)
    lam = math.sqrt(3.0) / ell
    a = np.abs(t[:, None] - t[None, :])
    K = s2 * (1 + lam * a) * np.exp(-lam * a) + tau2 * np.eye(n)
    ref = -0.5 * (n * math.log(2 * math.pi) + np.linalg.slogdet(K)[1] + y @ np.linalg.solve(K, y))
    assert abs(got - ref) < 1e-9 * abs(ref)
