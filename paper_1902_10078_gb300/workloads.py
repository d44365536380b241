"""Seeded synthetic inputs for the banded-operator workloads.

This module is shared by the CUDA path, the tests and the oracle.  It holds
only input synthesis: random draws and the workload recipe that turns them
into a banded SPD precision.  It calls neither the CUDA library nor the
oracle, and implements none of the operators (Cholesky, solves, subset
inverse, adjoints).

Storage convention (Sec. 4.3): a lower-banded n x n matrix with lower
bandwidth l is held as an (l+1) x n array ``B`` with ``B[d, j] = M[j+d, j]``
(0-based reading of the paper's index formula).  Entries with ``j+d >= n``
are the undefined corners; generators set them to 0 (or to NaN on request,
for layout tests).

Recipe for an SPD precision with lower bandwidth l (the workload shape used
for all configurations): draw a lower-banded L0 with diagonal ``1+U(0,1)`` and
off-diagonals ``N(0, 0.3^2/l)``, then ``Q = band_l(L0 L0^T) + 1e-3 I``.  Since
L0 already has lower bandwidth l, ``L0 L0^T`` has bandwidth l and the band
truncation keeps every entry.

Seeds: instance ``i`` of a batch draws from ``numpy PCG64(base_seed + i)``
with base seed 1902; the draw order is fixed (L0 diagonal, L0
off-diagonals by diagonal index, RHS columns, then cotangents).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1902


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def zero_corners(band: np.ndarray, fill: float = 0.0) -> np.ndarray:
    """Set the undefined corner entries ``band[d, j]`` with ``j+d >= n``."""
    n = band.shape[1]
    for d in range(1, band.shape[0]):
        band[d, max(n - d, 0):] = fill
    return band


def random_lower_factor(rng: np.random.Generator, n: int, l: int) -> np.ndarray:
    """L0 in lower-band storage: diag 1+U(0,1), off-diagonal N(0, 0.3^2/l)."""
    L0 = np.zeros((l + 1, n))
    L0[0] = 1.0 + rng.uniform(0.0, 1.0, n)
    scale = 0.3 / math.sqrt(l) if l > 0 else 0.0
    for d in range(1, l + 1):
        L0[d] = rng.normal(0.0, 1.0, n) * scale
    return zero_corners(L0)


def gram_band(L0: np.ndarray) -> np.ndarray:
    """``band_l(L0 L0^T)`` for a lower-banded L0 (input synthesis only).

    Entry (j+d, j) is ``sum_t L0[j+d, t] L0[j, t]`` over ``t = j-e``,
    ``e = 0..l-d``; in storage ``L0[j+d, j-e] = L0s[d+e, j-e]`` and
    ``L0[j, j-e] = L0s[e, j-e]``.
    """
    l = L0.shape[0] - 1
    n = L0.shape[1]
    Q = np.zeros_like(L0)
    for d in range(l + 1):
        for e in range(l - d + 1):
            j = np.arange(e, n - d)
            Q[d, j] += L0[d + e, j - e] * L0[e, j - e]
    return Q


def spd_band(rng: np.random.Generator, n: int, l: int, shift: float = 1e-3) -> np.ndarray:
    """Q = band_l(L0 L0^T) + shift * I in lower-band storage, corners = 0."""
    Q = gram_band(random_lower_factor(rng, n, l))
    Q[0] += shift
    return zero_corners(Q)


@dataclass
class Instance:
    """One banded SPD system with its right-hand sides and cotangents."""
    n: int
    l: int
    Q: np.ndarray          # (l+1, n) lower band, float64
    B: np.ndarray          # (k, n) right-hand sides, one row per RHS column
    Xbar: np.ndarray       # (k, n) cotangent of X = Q^{-1} B
    Sbar: np.ndarray       # (l+1, n) cotangent of the stored entries of band(Q^{-1})
    ldbar: float           # cotangent of log det Q


def make_instance(n: int, l: int, k: int, seed: int, cotangents: bool = True) -> Instance:
    rng = rng_for(seed)
    Q = spd_band(rng, n, l)
    B = rng.normal(0.0, 1.0, (k, n))
    if cotangents:
        Xbar = rng.normal(0.0, 1.0, (k, n))
        Sbar = zero_corners(rng.normal(0.0, 1.0, (l + 1, n)))
    else:
        Xbar = np.zeros((k, n))
        Sbar = np.zeros((l + 1, n))
    return Instance(n=n, l=l, Q=Q, B=B, Xbar=Xbar, Sbar=Sbar, ldbar=0.5)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def single_config(n: int = 1000, l: int = 2, k: int = 1, seed: int = BASE_SEED) -> Instance:
    """A single plain instance (n=1000, l=2, one RHS by default)."""
    return make_instance(n, l, k, seed)


def batched_shapes(count: int = 4096, n_lo: int = 1000, n_hi: int = 65536,
                   ls=(1, 2, 3, 5, 7), seed: int = BASE_SEED):
    """Shapes of the uneven batch: n log-uniform in [n_lo, n_hi], l uniform in ``ls``.

    ``n = floor(exp(U(ln n_lo, ln n_hi)))`` clipped to [n_lo, n_hi].
    """
    rng = rng_for(seed + 10_000_000)
    u = rng.uniform(math.log(n_lo), math.log(n_hi), count)
    n = np.clip(np.floor(np.exp(u)).astype(np.int64), n_lo, n_hi)
    l = np.asarray(ls, dtype=np.int64)[rng.integers(0, len(ls), count)]
    return n, l


def batched_config(count: int = 4096, k: int = 4, n_lo: int = 1000, n_hi: int = 65536,
                   ls=(1, 2, 3, 5, 7), seed: int = BASE_SEED, cotangents: bool = True):
    """The uneven batch: instance i uses seed ``seed + i``."""
    ns, lsz = batched_shapes(count, n_lo, n_hi, ls, seed)
    return [make_instance(int(ns[i]), int(lsz[i]), k, seed + i, cotangents) for i in range(count)]


def symmetric_band_weights(rng: np.random.Generator, n: int, l: int) -> np.ndarray:
    """W: a symmetric banded matrix (lower bandwidth l) with N(0,1) stored entries."""
    return zero_corners(rng.normal(0.0, 1.0, (l + 1, n)))


def long_chain_config(n: int = 100_000, l: int = 3, seed: int = BASE_SEED):
    """Single long chain with the quadratic/log-det/trace loss: (Q, b, W)."""
    rng = rng_for(seed)
    Q = spd_band(rng, n, l)
    b = rng.normal(0.0, 1.0, n)
    W = symmetric_band_weights(rng, n, l)
    return Q, b, W


# ---------------------------------------------------------------------------
# Matern-3/2 state-space prior inputs (raw draws only; the prior precision is
# built by the loss code on each side from these draws).
# ---------------------------------------------------------------------------

@dataclass
class MaternProcess:
    t: np.ndarray            # (n,) sorted inputs, gaps ~ Exp(1)
    lengthscale: float       # U(0.5, 5)
    variance: float          # 1
    Lq: np.ndarray           # (4, 2n) lower band (l=3) near-identity variational factor
    m: np.ndarray            # (2n,) variational mean ~ N(0, 0.1^2)


def matern_process(n: int, seed: int) -> MaternProcess:
    rng = rng_for(seed)
    gaps = rng.exponential(1.0, n - 1)
    t = np.concatenate([[0.0], np.cumsum(gaps)])
    ell = float(rng.uniform(0.5, 5.0))
    N = 2 * n
    Lq = np.zeros((4, N))
    Lq[0] = 1.0 + 0.1 * rng.uniform(0.0, 1.0, N)
    for d in range(1, 4):
        Lq[d] = rng.normal(0.0, 0.01, N)
    zero_corners(Lq)
    m = rng.normal(0.0, 0.1, N)
    return MaternProcess(t=t, lengthscale=ell, variance=1.0, Lq=Lq, m=m)


def matern_batch(count: int = 256, n: int = 50_000, seed: int = BASE_SEED):
    return [matern_process(n, seed + i) for i in range(count)]


def dense_from_lower_band(band: np.ndarray, symmetric: bool) -> np.ndarray:
    """Dense matrix from lower-band storage (for small-n checks)."""
    l1, n = band.shape
    M = np.zeros((n, n))
    for d in range(min(l1, n)):
        j = np.arange(0, n - d)
        M[j + d, j] = band[d, : n - d]
        if symmetric and d > 0:
            M[j, j + d] = band[d, : n - d]
    return M


def lower_band_from_dense(M: np.ndarray, l: int) -> np.ndarray:
    n = M.shape[0]
    band = np.zeros((l + 1, n))
    for d in range(min(l + 1, n)):
        j = np.arange(0, n - d)
        band[d, : n - d] = M[j + d, j]
    return band


# ---------------------------------------------------------------------------
# Batch inputs in a pool layout (host side, parallel over instances)
# ---------------------------------------------------------------------------

def _fill_worker(args):
    """Draw the instances of one chunk: (slot, seed, n, l) -> FP32 band / RHS arrays."""
    jobs, k = args
    out = []
    for slot, seed, n, l in jobs:
        ins = make_instance(n, l, k, seed)
        out.append((slot, ins.Q.astype(np.float32), ins.Sbar.astype(np.float32), ins.B.astype(np.float32),
                    ins.Xbar.astype(np.float32)))
    return out


def fill_pools(lay, seeds, workers=1):
    """FP32 host pools Q, Sbar (band) and B, Xbar (RHS) of a batch in the
    arrangement of ``lay`` (a batch.Layout); instance ``slot`` of the layout
    draws ``make_instance(lay.ns[slot], lay.ls[slot], lay.k, seeds[slot])``, so
    a reordered layout keeps each instance's data by passing its seed along.
    ``workers`` > 1 uses a spawn pool (safe before or after CUDA use)."""
    import multiprocessing as mp
    pools = {"Q": np.zeros(lay.band_elems, np.float32), "Sbar": np.zeros(lay.band_elems, np.float32),
             "B": np.zeros(lay.rhs_elems, np.float32), "Xbar": np.zeros(lay.rhs_elems, np.float32)}
    items = [(s, int(seeds[s]), int(lay.ns[s]), int(lay.ls[s])) for s in range(lay.count)]
    chunks = max(1, min(workers * 4, lay.count))
    bounds = np.linspace(0, lay.count, chunks + 1).astype(int)
    jobs = [(items[bounds[c]:bounds[c + 1]], lay.k) for c in range(chunks) if bounds[c + 1] > bounds[c]]

    def put(res):
        for s, q, sb, b, xb in res:
            lay.band_view(pools["Q"], s)[: q.shape[0]] = q
            lay.band_view(pools["Sbar"], s)[: sb.shape[0]] = sb
            lay.rhs_view(pools["B"], s)[: b.shape[0]] = b
            lay.rhs_view(pools["Xbar"], s)[: xb.shape[0]] = xb
    if workers > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            for res in pool.imap_unordered(_fill_worker, jobs):
                put(res)
    else:
        for j in jobs:
            put(_fill_worker(j))
    return pools


# ---------------------------------------------------------------------------
# Graph GMRF (Sec. 2 graph precisions; the spatial workload of Sec. 5.3 has a
# graph of 11284 nodes whose precision reaches bandwidth 117 after
# reordering).  Synthetic stand-in: a random geometric graph in a rectangle of
# unit area (aspect ratio `aspect`), precision kappa^2 I + graph Laplacian
# (SPD), nodes reordered by reverse Cuthill-McKee so that the precision is
# banded.  At 11284 nodes, mean degree 6 and aspect 2 the band is l = 140 with
# scipy 1.18 (other scipy versions break the ordering's ties differently: 162
# was seen).
# ---------------------------------------------------------------------------

def gmrf_graph(N: int, mean_degree: float = 6.0, kappa2: float = 0.1, aspect: float = 2.0,
               seed: int = BASE_SEED):
    """Returns (Q, l, perm, edges): Q in lower band storage (l+1, N) in the
    reordered numbering, perm[new] = old node index, edges (E, 2) in the old
    numbering."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    from scipy.spatial import cKDTree
    rng = rng_for(seed)
    pts = rng.uniform(0.0, 1.0, (N, 2))
    pts[:, 0] *= aspect
    pts[:, 1] /= aspect
    r = math.sqrt(mean_degree / (math.pi * N))
    pairs = np.array(sorted(cKDTree(pts).query_pairs(r)), dtype=np.int64).reshape(-1, 2)
    A = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(N, N))
    A = (A + A.T).tocsr()
    perm = np.asarray(reverse_cuthill_mckee(A, symmetric_mode=True), dtype=np.int64)
    inv = np.empty(N, dtype=np.int64)
    inv[perm] = np.arange(N)
    pi, pj = inv[pairs[:, 0]], inv[pairs[:, 1]]
    lo, hi = np.minimum(pi, pj), np.maximum(pi, pj)
    l = int((hi - lo).max()) if len(pairs) else 0
    deg = np.bincount(np.concatenate([pairs[:, 0], pairs[:, 1]]), minlength=N).astype(np.float64)
    Q = np.zeros((l + 1, N))
    Q[0] = kappa2 + deg[perm]
    Q[hi - lo, lo] = -1.0
    return zero_corners(Q), l, perm, pairs
