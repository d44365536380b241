"""The premise of the wide-band segment acceptance (host-side simulation).

A speculative segment starts from a zero state some rows before its first
output row.  The banded Cholesky of the block sweeps keeps pending Schur sums
of l + 1 columns and adds one rank-1 update per row; this test runs that
recurrence in FP32 (numpy, in the same order as the kernels but with a
separate multiply and add where they fuse) once from row 0 and once cold from
a later row.  At l = 16 the cold run becomes bit-identical to the full run
after a few blocks of l rows, which is what the bitwise segment check of the
register-window sweeps relies on.  At l = 64 it never does, yet the
difference stays at the level of single rounding errors: the reason the
block sweeps accept a segment start within a tolerance of the state's scale
instead of bit for bit.
"""
import numpy as np

from paper_1902_10078_gb300 import workloads as W


def _cholesky_rows(Q, j0, nrows):
    """Columns j0 .. j0 + nrows - 1 of L, pending-Schur-sum order, FP32, zero start."""
    l = Q.shape[0] - 1
    lw = l + 1
    pend = np.zeros((lw, lw), dtype=np.float32)      # slot c mod (l+1): pending sums of column c
    out = np.zeros((nrows, lw), dtype=np.float32)
    for q in range(nrows):
        j = j0 + q
        sj = j % lw
        a = Q[:, j] - pend[sj]
        a[l] = Q[l, j]
        r = np.float32(1) / np.sqrt(a[0])
        col = a * r
        pend[sj] = 0
        for y in range(1, lw):                       # column j + y gets L[j+y+f, j] L[j+y, j]
            pend[(j + y) % lw, :lw - y] += col[y:] * col[y]
        out[q] = col
    return out


def _cold_vs_full(l, blocks, start_blocks):
    n = blocks * l
    Q = W.spd_band(W.rng_for(5), n, l).astype(np.float32)
    full = _cholesky_rows(Q, 0, n)
    j0 = start_blocks * l
    cold = _cholesky_rows(Q, j0, n - j0)
    diff = np.abs(cold - full[j0:]).max(axis=1)
    return diff, np.abs(full).max()


def test_narrow_band_cold_start_becomes_bit_identical():
    diff, _ = _cold_vs_full(16, 90, 10)
    differing = np.nonzero(diff)[0]
    assert differing.size and differing.max() < 16 * 16      # equal bit for bit within 16 l rows
    assert not diff[16 * 16:].any()


def test_wide_band_cold_start_stays_at_rounding_noise():
    l = 64
    diff, scale = _cold_vs_full(l, 90, 10)
    late = diff[-10 * l:]
    assert late.any()                                        # never bit-identical ...
    assert late.max() <= 2.0 ** -20 * scale                  # ... but far inside 2^-16 of the scale
    assert diff[8 * l:].max() <= 2.0 ** -20 * scale          # once converged, for good
