"""FP64 CPU oracle for the banded operators (arXiv 1902.10078).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The CUDA library never imports it.

The arithmetic lives in ``banded_oracle.c`` (Alg. 1-4 of App. B and the
Table 1 compositions, one instance per call).  This module only marshals
numpy arrays to it.  Band arrays use lower-band storage ``B[d, j] = M[j+d, j]``
(Sec. 4.3) unless a (lo, up) general band is stated; right-hand sides are
``(k, n)`` arrays, one row per column vector.

Parity: pinned by tests/test_oracle_pins.py against dense LAPACK/numpy,
scipy's banded routines, closed forms, invariants and central finite
differences (see those tests for which pin covers which function).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_i64 = C.c_int64
_int = C.c_int
_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_cholesky.restype = _int
        L.orc_cholesky.argtypes = [_i64, _int, _dp, _i64, _dp, _i64]
        L.orc_logdet.restype = C.c_double
        L.orc_logdet.argtypes = [_i64, _dp]
        L.orc_solve.restype = None
        L.orc_solve.argtypes = [_i64, _int, _dp, _i64, _int, _int, _dp, _i64, _dp, _i64]
        L.orc_subset_inverse.restype = None
        L.orc_subset_inverse.argtypes = [_i64, _int, _dp, _i64, _dp, _i64]
        L.orc_cholesky_vjp.restype = None
        L.orc_cholesky_vjp.argtypes = [_i64, _int, _dp, _i64, _dp, _i64, _dp, _i64]
        L.orc_subset_inverse_vjp.restype = None
        L.orc_subset_inverse_vjp.argtypes = [_i64, _int, _dp, _i64, _dp, _i64, _dp, _i64, _dp, _i64, _int]
        L.orc_product.restype = None
        L.orc_product.argtypes = [_i64, _dp, _i64, _int, _int, _int, _dp, _i64, _int, _int, _int,
                                  _dp, _i64, _int, _int]
        L.orc_band_matvec.restype = None
        L.orc_band_matvec.argtypes = [_i64, _dp, _i64, _int, _int, _int, _int, _dp, _i64, _dp, _i64]
        L.orc_outer.restype = None
        L.orc_outer.argtypes = [_i64, _int, _dp, _i64, _dp, _i64, _dp, _i64, _int, _int]
        L.orc_solve_vjp.restype = None
        L.orc_solve_vjp.argtypes = [_i64, _int, _dp, _i64, _int, _int, _dp, _i64, _dp, _i64,
                                    _dp, _i64, _dp, _i64]
        L.orc_product_vjp.restype = None
        L.orc_product_vjp.argtypes = [_i64, _dp, _i64, _int, _int, _int, _dp, _i64, _int, _int, _int,
                                      _dp, _i64, _int, _int, _dp, _i64, _dp, _i64]
        L.orc_band_matvec_vjp.restype = None
        L.orc_band_matvec_vjp.argtypes = [_i64, _dp, _i64, _int, _int, _int, _int, _dp, _i64,
                                          _dp, _i64, _dp, _i64, _dp, _i64]
        L.orc_outer_vjp.restype = None
        L.orc_outer_vjp.argtypes = [_i64, _int, _dp, _i64, _dp, _i64, _dp, _i64, _int, _int,
                                    _dp, _i64, _dp, _i64]
        L.orc_solve_band.restype = None
        L.orc_solve_band.argtypes = [_i64, _int, _dp, _i64, _int, _dp, _i64, _int, _int, _dp, _i64, _int, _int]
        L.orc_solve_band_vjp.restype = None
        L.orc_solve_band_vjp.argtypes = [_i64, _int, _dp, _i64, _int, _dp, _i64, _int, _int, _dp, _i64,
                                         _int, _int, _dp, _i64, _dp, _i64]
        L.orc_batch_step.restype = _int
        L.orc_batch_step.argtypes = [_int, C.c_void_p]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _null():
    return C.cast(None, _dp)


# ---------------------------------------------------------------------------
# Operators (Sec. 4.1 / App. B)
# ---------------------------------------------------------------------------

def cholesky(Q):
    """Alg. 1. Returns (L, info); info = first failing row + 1, or 0."""
    Q = _f64(Q)
    l, n = Q.shape[0] - 1, Q.shape[1]
    L = np.zeros_like(Q)
    info = lib().orc_cholesky(n, l, _p(Q), n, _p(L), n)
    return L, int(info)


def logdet(L):
    """log det(L L^T) = 2 sum log L_ii."""
    L = _f64(L)
    return float(lib().orc_logdet(L.shape[1], _p(L)))


def solve(L, B, trans: int):
    """trans=0: L^{-1} B; trans=1: L^{-T} B.  B is (k, n) or (n,)."""
    L = _f64(L)
    B = _f64(B)
    vec = B.ndim == 1
    B2 = B[None] if vec else B
    X = np.zeros_like(B2)
    n = L.shape[1]
    lib().orc_solve(n, L.shape[0] - 1, _p(L), n, int(trans), B2.shape[0], _p(B2), n, _p(X), n)
    return X[0] if vec else X


def solve_precision(L, B):
    """(L L^T)^{-1} B = L^{-T} (L^{-1} B)."""
    return solve(L, solve(L, B, 0), 1)


def subset_inverse(L):
    """Alg. 3: lower band of (L L^T)^{-1}."""
    L = _f64(L)
    S = np.zeros_like(L)
    n = L.shape[1]
    lib().orc_subset_inverse(n, L.shape[0] - 1, _p(L), n, _p(S), n)
    return S


def cholesky_vjp(L, Lbar):
    """Alg. 2: gradient w.r.t. the lower stored entries of Q."""
    L, Lbar = _f64(L), _f64(Lbar)
    Qbar = np.zeros_like(L)
    n = L.shape[1]
    lib().orc_cholesky_vjp(n, L.shape[0] - 1, _p(L), n, _p(Lbar), n, _p(Qbar), n)
    return Qbar


def subset_inverse_vjp(L, S, Sbar):
    """Alg. 4: gradient w.r.t. the stored entries of L."""
    L, S, Sbar = _f64(L), _f64(S), _f64(Sbar)
    Lbar = np.zeros_like(L)
    n = L.shape[1]
    lib().orc_subset_inverse_vjp(n, L.shape[0] - 1, _p(L), n, _p(S), n, _p(Sbar), n, _p(Lbar), n, 0)
    return Lbar


def product(A, alo, aup, transA, B, blo, bup, transB, clo, cup):
    """C = op(A) op(B) projected onto band (clo, cup); general band storage."""
    A, B = _f64(A), _f64(B)
    n = A.shape[1]
    Cm = np.zeros((clo + cup + 1, n))
    lib().orc_product(n, _p(A), n, alo, aup, int(transA), _p(B), n, blo, bup, int(transB),
                      _p(Cm), n, clo, cup)
    return Cm


def band_matvec(A, alo, aup, transA, V):
    A, V = _f64(A), _f64(V)
    vec = V.ndim == 1
    V2 = V[None] if vec else V
    n = A.shape[1]
    P = np.zeros_like(V2)
    lib().orc_band_matvec(n, _p(A), n, alo, aup, int(transA), V2.shape[0], _p(V2), n, _p(P), n)
    return P[0] if vec else P


def outer(M, V, clo, cup):
    """band_{clo,cup}(sum_r m_r v_r^T); M, V are (k, n) or (n,)."""
    M, V = _f64(M), _f64(V)
    M2 = M[None] if M.ndim == 1 else M
    V2 = V[None] if V.ndim == 1 else V
    n = M2.shape[1]
    Cm = np.zeros((clo + cup + 1, n))
    lib().orc_outer(n, M2.shape[0], _p(M2), n, _p(V2), n, _p(Cm), n, clo, cup)
    return Cm


def solve_band(L, R, rlo, rup, trans, olo, oup):
    """Alg. 5: band_{olo,oup}(L^{-1} R) (trans 0) or band_{olo,oup}(L^{-T} R) (trans 1);
    R and the result in general band storage."""
    L, R = _f64(L), _f64(R)
    n = L.shape[1]
    O = np.zeros((olo + oup + 1, n))
    lib().orc_solve_band(n, L.shape[0] - 1, _p(L), n, int(trans), _p(R), n, rlo, rup, _p(O), n, olo, oup)
    return O


# ---------------------------------------------------------------------------
# Table 1 compositions
# ---------------------------------------------------------------------------

def solve_band_vjp(L, trans, O, olo, oup, Obar, rlo, rup):
    """Table 1, solve matrix-matrix, for O = solve_band(...): returns (Rbar, Lbar)."""
    L, O, Obar = _f64(L), _f64(O), _f64(Obar)
    n = L.shape[1]
    l = L.shape[0] - 1
    Rbar = np.zeros((rlo + rup + 1, n))
    Lbar = np.zeros_like(L)
    lib().orc_solve_band_vjp(n, l, _p(L), n, int(trans), _p(O), n, olo, oup, _p(Obar), n, rlo, rup,
                             _p(Rbar), n, _p(Lbar), n)
    return Rbar, Lbar


def solve_vjp(L, trans, S, Sbar):
    """For S = L^{-1} V (trans 0) or L^{-T} V (trans 1): returns (Vbar, Lbar)."""
    L, S, Sbar = _f64(L), _f64(S), _f64(Sbar)
    vec = S.ndim == 1
    S2 = S[None] if vec else S
    Sb2 = Sbar[None] if vec else Sbar
    n = L.shape[1]
    Vbar = np.zeros_like(S2)
    Lbar = np.zeros_like(L)
    lib().orc_solve_vjp(n, L.shape[0] - 1, _p(L), n, int(trans), S2.shape[0], _p(S2), n, _p(Sb2), n,
                        _p(Vbar), n, _p(Lbar), n)
    return (Vbar[0] if vec else Vbar), Lbar


def product_vjp(A, alo, aup, transA, B, blo, bup, transB, Cbar, clo, cup):
    A, B, Cbar = _f64(A), _f64(B), _f64(Cbar)
    n = A.shape[1]
    Abar = np.zeros((alo + aup + 1, n))
    Bbar = np.zeros((blo + bup + 1, n))
    lib().orc_product_vjp(n, _p(A), n, alo, aup, int(transA), _p(B), n, blo, bup, int(transB),
                          _p(Cbar), n, clo, cup, _p(Abar), n, _p(Bbar), n)
    return Abar, Bbar


def band_matvec_vjp(A, alo, aup, transA, V, Pbar):
    A, V, Pbar = _f64(A), _f64(V), _f64(Pbar)
    vec = V.ndim == 1
    V2 = V[None] if vec else V
    P2 = Pbar[None] if vec else Pbar
    n = A.shape[1]
    Abar = np.zeros_like(A)
    Vbar = np.zeros_like(V2)
    lib().orc_band_matvec_vjp(n, _p(A), n, alo, aup, int(transA), V2.shape[0], _p(V2), n,
                              _p(P2), n, _p(Abar), n, _p(Vbar), n)
    return Abar, (Vbar[0] if vec else Vbar)


def outer_vjp(M, V, Obar, olo, oup):
    M, V, Obar = _f64(M), _f64(V), _f64(Obar)
    vec = M.ndim == 1
    M2 = M[None] if vec else M
    V2 = V[None] if vec else V
    n = M2.shape[1]
    Mbar = np.zeros_like(M2)
    Vbar = np.zeros_like(V2)
    lib().orc_outer_vjp(n, M2.shape[0], _p(M2), n, _p(V2), n, _p(Obar), n, olo, oup,
                        _p(Mbar), n, _p(Vbar), n)
    return (Mbar[0] if vec else Mbar), (Vbar[0] if vec else Vbar)


# ---------------------------------------------------------------------------
# The uneven-batch step (forward and backward of chol + solve + log det +
# subset inverse), run by the C oracle with OpenMP over instances.
# ---------------------------------------------------------------------------

class _StepIO(C.Structure):
    _fields_ = [("n", C.c_int64), ("l", C.c_int), ("k", C.c_int),
                ("Q", _dp), ("B", _dp), ("Xbar", _dp), ("Sbar", _dp), ("ldbar", C.c_double),
                ("L", _dp), ("X", _dp), ("S", _dp), ("Qbar", _dp), ("Bbar", _dp),
                ("logdet", _dp), ("info", C.POINTER(C.c_int))]


def batch_step(instances):
    """Runs the batch step for a list of workloads.Instance; returns (results, threads).

    Each result is a dict with L, logdet, info, X, S, Qbar, Bbar (float64)."""
    ios = (_StepIO * len(instances))()
    keep = []
    results = []
    for c, ins in enumerate(instances):
        Q, B, Xb, Sb = _f64(ins.Q), _f64(ins.B), _f64(ins.Xbar), _f64(ins.Sbar)
        k = B.shape[0]
        r = dict(L=np.zeros_like(Q), X=np.zeros_like(B), S=np.zeros_like(Q), Qbar=np.zeros_like(Q),
                 Bbar=np.zeros_like(B), logdet=np.zeros(1), info=np.zeros(1, dtype=np.int32))
        keep.append((Q, B, Xb, Sb))
        results.append(r)
        io = ios[c]
        io.n, io.l, io.k = ins.n, ins.l, k
        io.Q, io.B, io.Xbar, io.Sbar, io.ldbar = _p(Q), _p(B), _p(Xb), _p(Sb), float(ins.ldbar)
        io.L, io.X, io.S, io.Qbar, io.Bbar = _p(r["L"]), _p(r["X"]), _p(r["S"]), _p(r["Qbar"]), _p(r["Bbar"])
        io.logdet = _p(r["logdet"])
        io.info = r["info"].ctypes.data_as(C.POINTER(C.c_int))
    threads = lib().orc_batch_step(len(instances), C.cast(ios, C.c_void_p))
    for r in results:
        r["logdet"] = float(r["logdet"][0])
        r["info"] = int(r["info"][0])
    return results, int(threads)
