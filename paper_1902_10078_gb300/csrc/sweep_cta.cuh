// Block-cooperative sweeps for wide bands: one thread block per chain, the
// computed window of the recurrence in shared memory, every O(l^2) step of a
// row spread over the block's threads, the inputs staged in shared memory one
// tile of rows ahead of use.
//
// The recurrences and formulas are those of the register-window sweeps
// (sweep_impl.cuh) with a runtime bandwidth l:
//   forward : CHOL (Alg. 1, column order with pending Schur sums), SOLVE
//             (y = L^{-1} b), ALG4 (reverse mode of the row-ordered
//             Takahashi recursion, one adjoint per unordered pair)
//   backward: TAKA (Alg. 3, row order), SOLVE (x = L^{-T} y), ALG2 (Alg. 2
//             in column-reverse order, with the solve-adjoint outer products
//             and the log-det term added to column j of L-bar first)
//
// Windows.  A band window W of a pair quantity (pending Schur sums, pair
// adjoints, the Sigma block, pending L-bar) holds the entries (r, c), r >= c,
// of l + 1 consecutive columns c: entry (r, c) sits at W[slot(c) rs + (r - c)]
// with slot(c) = c mod (l+1) and rs = l + 1 rounded up to even (an odd stride
// keeps a warp that walks across slots clear of bank conflicts); moving the
// window by one column retires one slot and reuses it for the column entering
// on the other side (zeroed first) -- nothing is copied.  RHS windows are
// (l+1)-slot rings.
//
// Input streams.  Every input (a band read column by column, or a block of
// right-hand sides) goes through a ring of columns in shared memory, filled by
// element-wise cp.async copies one tile of kCtaTile rows ahead of use, so that
// a row does not wait on L2 or DRAM.  A stream spans the columns it needs
// around the current one ("ahead" in the sweep direction, "behind" against
// it): the Sigma block of Alg. 4 spans l columns of S ahead, the L entries of
// Alg. 2 l columns of L ahead, the X rows of the solve-adjoint outer products
// l rows behind.  Where the rings do not fit next to the window (FP64 at the
// widest bands) the wide spans, then all streams, are read from global memory
// (L2) instead: cta_tier picks the level per launch.
//
// Per row: three block barriers (load / finish the row's scalars / window
// update), one more per tile for the copies.  Row-by-row reductions (a
// matrix-vector product with a window) give each output a group of lanes of
// one warp (cta_rows_reduce).
//
// Segments.  A long instance is cut into segments run by separate blocks; a
// segment other than the first in sweep order starts `warm` rows early from a
// zero state (cold start) and saves the state it reached at its first output
// row, and every segment saves its state after its last row.  A verify pass
// then compares each boundary and reruns from the exact state the segments
// whose start was not close enough (cta_states_close).
#pragma once

#include "sweep_impl.cuh"

namespace bnd {

constexpr int kCtaThreads = 512;
constexpr int kCtaWarps = kCtaThreads / kWarp;
constexpr int kCtaMaxK = 16;                     // right-hand sides one block sweep carries
static_assert(kCtaMaxK <= kCtaWarps, "one warp per right-hand side in the solve reductions");
constexpr int kCtaTile = 8;                      // rows per prefetched tile of the input streams
constexpr size_t kCtaSmemLimit = 232448;         // 227 KB of shared memory per block

__host__ __device__ inline int cta_even(int x) { return (x + 1) & ~1; }
// Right-hand sides the block sweeps of a plan with k columns carry at once
// (the RHS windows and streams are sized for them).
__host__ __device__ inline int cta_rhs(int k) { return k < kCtaMaxK ? k : kCtaMaxK; }
// Ring of an input stream of `rows` rows spanning `span` columns besides the current one.
__host__ __device__ inline int64_t cta_ring_elems(int rows, int span) {
    return (int64_t)(span + 2 * kCtaTile) * cta_even(rows);
}
// Staging level of a launch: 2 = every stream in a ring, 1 = the wide spans
// (Sigma block, L window, X rows) read from global memory, 0 = every stream
// read from global memory.
enum : int { kTierDirect = 0, kTierNarrow = 1, kTierAll = 2 };

// Shared-memory elements of a block sweep (direction fwd, flags fl) for
// bandwidth l, km = cta_rhs(k) right-hand sides and staging level tier.
__host__ __device__ inline int64_t cta_smem_elems(bool fwd, int fl, int l, int km, int tier) {
    const int lw = l + 1, rs = cta_even(lw);
    int64_t e = (int64_t)lw * rs;                                  // computed window
    e += (int64_t)km * lw;                                         // RHS window
    e += 8 * (int64_t)lw + 2 * kCtaWarps + 4 * kCtaMaxK + 16;      // row vectors, partial sums, scalars
    if (tier >= kTierNarrow) {
        e += cta_ring_elems(lw, 0) + cta_ring_elems(km, 0);        // Q or L column, right-hand sides
        if (fwd ? (fl & F_ALG4) != 0 : (fl & B_ALG2) != 0) e += cta_ring_elems(lw, 0);   // Sbar / Lbar
    }
    if (tier >= kTierAll) {
        if (fwd && (fl & F_ALG4)) e += cta_ring_elems(lw, l);                          // S ahead
        if (!fwd && (fl & B_ALG2)) e += cta_ring_elems(lw, l) + cta_ring_elems(km, l); // L ahead, X behind
    }
    return e;
}
template <typename T>
__host__ __device__ inline bool cta_fits(bool fwd, int fl, int l, int km, int tier) {
    // 1 KB is left for the verify kernel's static shared memory
    return sizeof(T) * (size_t)cta_smem_elems(fwd, fl, l, km, tier) <= kCtaSmemLimit - 1024;
}
// Highest staging level that fits, or -1 when even the direct form does not.
template <typename T>
__host__ __device__ inline int cta_tier(bool fwd, int fl, int l, int km) {
    for (int t = kTierAll; t >= kTierDirect; --t)
        if (cta_fits<T>(fwd, fl, l, km, t)) return t;
    return -1;
}
// The block sweeps serve bandwidth l with km right-hand sides in dtype T when
// every sweep kind fits, at least in the direct form.
template <typename T>
__host__ __device__ inline bool cta_serves(int l, int km) {
    return cta_tier<T>(true, F_CHOL | F_SOLVE, l, km) >= 0 && cta_tier<T>(true, F_ALG4 | F_SOLVE, l, km) >= 0 &&
           cta_tier<T>(false, B_TAKA | B_SOLVE, l, km) >= 0 &&
           cta_tier<T>(false, B_ALG2 | B_SOLVE | B_OUTER, l, km) >= 0;
}
// Words of a block sweep's state snapshot: the band window and the RHS ring,
// rotated so that the slot of the current column comes first.
__host__ __device__ inline int64_t cta_state_words(int l, int km) {
    const int64_t lw = l + 1;
    return lw * cta_even(l + 1) + (int64_t)km * lw;
}

template <typename T>
__device__ __forceinline__ T cta_block_sum(T v, T *red) {
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = T(0);
    for (int w = 0; w < kCtaWarps; ++w) s += red[w];
    return s;
}

// out(t, sum_{q = 1..nq} f(t, q, .)) for t = 1..nt, with G lanes of one warp
// per t (G the largest power of two up to 32 with nt G <= kCtaThreads): each
// lane folds a strided share of q into its accumulator, the G partial sums
// meet in log2 G shuffles.  Every thread of the block must call it.
template <typename T, class F, class Out>
__device__ __forceinline__ void cta_rows_reduce(int nt, int nq, F f, Out out) {
    int G = kWarp;
    while (G > 1 && nt * G > kCtaThreads) G >>= 1;
    const int per_pass = kCtaThreads / G;
    const int g = (int)threadIdx.x % G;
    for (int t0 = 1; t0 <= nt; t0 += per_pass) {
        const int t = t0 + (int)threadIdx.x / G;
        T acc = T(0);
        if (t <= nt)
            for (int q = 1 + g; q <= nq; q += G) acc = f(t, q, acc);
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (g == 0 && t <= nt) out(t, acc);
    }
}

__device__ __forceinline__ int wrap_slot(int s, int lw) { return s >= lw ? s - lw : (s < 0 ? s + lw : s); }

// Save (or load) the state of a block sweep whose current column has slot sj:
// word x < (l+1) rs is entry f of the window column rel slots after sj
// (x = rel rs + f), then RHS ring row r < km, rel slots after sj.  Whole block.
template <typename T>
__device__ void cta_state_io(T *W, T *U, int l, int km, int sj, T *snap, bool save) {
    const int lw = l + 1, rs = cta_even(lw), nw = lw * rs;
    __syncthreads();
    for (int x = threadIdx.x; x < nw + km * lw; x += kCtaThreads) {
        T *live;
        if (x < nw) {
            const int rel = x / rs, f = x - rel * rs;
            live = W + wrap_slot(sj + rel, lw) * rs + f;
        } else {
            const int y = x - nw, r = y / lw, rel = y - r * lw;
            live = U + r * lw + wrap_slot(sj + rel, lw);
        }
        if (save) snap[x] = *live;
        else *live = snap[x];
    }
    __syncthreads();
}

// Acceptance of a speculative segment start.  Once a cold start has forgotten
// its zero state mathematically, the two runs differ only by rounding, but
// above l of about 50 they never become equal bit for bit: a one-ulp
// difference in one window entry reaches l others through the row's O(l^2)
// update, and enough of those survive rounding to keep the difference alive
// for good, at about one ulp of the state's largest entry -- the rounding
// noise either run carries anyway.  (At l <= 32 the difference dies out within
// a few blocks of l rows, as it does for the register-window sweeps, which
// compare bit for bit.)  So a boundary passes when the two snapshots agree
// word for word within StateTol times the largest magnitude of their part of
// the state (the band window as a whole; each RHS row on its own); a start
// that has not converged is off by orders of magnitude more.  Bitwise-equal
// words always agree (NaN included); any other NaN fails.
template <typename T> struct StateTol;
template <> struct StateTol<float> { static constexpr float value = 1.52587890625e-05f; };        // 2^-16
template <> struct StateTol<double> { static constexpr double value = 5.684341886080802e-14; };   // 2^-44

template <typename T>
__device__ __forceinline__ void state_word_cmp(T a, T b, T &dmax, T &amax, bool &bad) {
    const bool same = sizeof(T) == 4 ? __float_as_uint((float)a) == __float_as_uint((float)b)
                                     : __double_as_longlong((double)a) == __double_as_longlong((double)b);
    if (same) {
        if (a == a) amax = fmax(amax, fabs(a));
        return;
    }
    const T d = fabs(a - b);
    if (!(d == d)) bad = true;
    else dmax = fmax(dmax, d);
    amax = fmax(amax, fmax(fabs(a), fabs(b)));
}

// Whole block: true when snapshots x and y (cta_state_io layout, bandwidth l,
// km RHS rows) are close in the sense above.
template <typename T>
__device__ bool cta_states_close(const T *x, const T *y, int l, int km) {
    __shared__ T buf[2 * kCtaWarps];
    const int lw = l + 1, nw = lw * cta_even(lw);
    const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
    const T tol = StateTol<T>::value;
    bool ok = true;
    T dm = T(0), am = T(0);
    bool bad = false;
    for (int w = tid; w < nw; w += kCtaThreads) state_word_cmp(x[w], y[w], dm, am, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    if (lane == 0) { buf[warp] = dm; buf[kCtaWarps + warp] = am; }
    for (int r = warp; r < km; r += kCtaWarps) {             // RHS row r: warp r
        T rd = T(0), ra = T(0);
        bool rb = false;
        for (int i = lane; i < lw; i += kWarp) state_word_cmp(x[nw + r * lw + i], y[nw + r * lw + i], rd, ra, rb);
        rb = __any_sync(0xffffffffu, rb);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rd = fmax(rd, __shfl_xor_sync(0xffffffffu, rd, o));
            ra = fmax(ra, __shfl_xor_sync(0xffffffffu, ra, o));
        }
        if (rb || !(rd <= tol * ra)) ok = false;
    }
    if (bad) ok = false;
    __syncthreads();
    T wd = T(0), wa = T(0);
    for (int w = 0; w < kCtaWarps; ++w) {
        wd = fmax(wd, buf[w]);
        wa = fmax(wa, buf[kCtaWarps + w]);
    }
    if (!(wd <= tol * wa)) ok = false;
    return __syncthreads_and(ok) != 0;        // its barrier also keeps buf until every thread has read it
}

// First row of a block sweep over chain c (forward: the rows run upward from
// it; backward: downward): a cold start of a segment that is not the first in
// sweep order begins `warm` rows outside the segment.
__device__ __forceinline__ int64_t cta_first_row(const ChainCtx &c, bool fwd, int mode) {
    if (fwd) return (mode == RUN_COLD && !c.first) ? imax64(c.a - c.warm, 0) : c.a;
    return (mode == RUN_COLD && !c.last) ? imin64(c.b - 1 + c.warm, c.n - 1) : c.b - 1;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid) {
    const int nb = valid ? (int)sizeof(T) : 0;       // src-size 0: zero fill, nothing is read
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(nb) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(nb) : "memory");
}
__device__ __forceinline__ void cta_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cta_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One input stream of a block sweep.  Sweep position q (0 at the chain's
// first row) is column j0 + dir q; element e of the column o positions ahead
// of the current one (o < 0: behind) is at(e, o).  Columns outside [0, n), and
// band elements (e, c) with c + e >= n, read as zero.  Staged: a ring of
// span + 2 kCtaTile columns in shared memory, position q in slot q mod nslot,
// filled by issue_first / issue_next.  Direct (no ring): read from global
// memory at the use.
template <typename T>
struct CtaStream {
    const T *g;          // element (e, column c) at g[e * stride + c * cs]
    int64_t stride, cs, n, jfirst, jc;
    int rows, dir;
    bool band;
    int ahead, behind;
    T *ring;             // nullptr: direct
    int rs, nslot, cur;

    // Returns the shared memory after the ring (unchanged when direct or absent).
    __device__ T *setup(const T *g_, int64_t stride_, int64_t cs_, int rows_, int rows_cap, bool band_, int ahead_,
                        int behind_, bool staged, int64_t j0, int dir_, int64_t n_, T *mem) {
        g = g_; stride = stride_; cs = cs_; rows = rows_; band = band_; ahead = ahead_; behind = behind_;
        jfirst = jc = j0; dir = dir_; n = n_;
        rs = cta_even(rows_cap);
        nslot = ahead + behind + 2 * kCtaTile;
        cur = 0;
        ring = (staged && g) ? mem : nullptr;
        return ring ? mem + (int64_t)nslot * rs : mem;
    }
    __device__ __forceinline__ bool inside(int64_t c, int e) const { return c >= 0 && c < n && (!band || c + e < n); }
    // copies of positions [q0, q1] (at most nslot of them)
    __device__ void issue(int64_t q0, int64_t q1) {
        if (!ring || rows <= 0) return;
        const int cnt = (int)(q1 - q0 + 1) * rows;
        int s0 = (int)(q0 % nslot);
        if (s0 < 0) s0 += nslot;
        for (int x = threadIdx.x; x < cnt; x += kCtaThreads) {
            const int dq = x / rows, e = x - dq * rows;
            const int64_t c = jfirst + (int64_t)dir * (q0 + dq);
            const bool ok = inside(c, e);
            int sl = s0 + dq;
            if (sl >= nslot) sl -= nslot;
            cp_async_elem(ring + sl * rs + e, ok ? g + e * stride + c * cs : g, ok);
        }
    }
    // the positions the first tile needs (its rows' whole span); a later tile starting at q0
    // adds the ones that enter `ahead` positions in front of it
    __device__ void issue_first() { issue(-(int64_t)behind, (int64_t)kCtaTile - 1 + ahead); }
    __device__ void issue_next(int64_t q0) { issue(q0 + ahead, q0 + kCtaTile - 1 + ahead); }
    __device__ __forceinline__ T at(int e, int o) const {
        if (ring) return ring[wrap_slot(cur + o, nslot) * rs + e];
        const int64_t c = jc + (int64_t)dir * o;
        return (g && inside(c, e)) ? g[e * stride + c * cs] : T(0);
    }
    // The column o positions ahead: element e at p[e * step] (no zero fill: the caller stays
    // inside the band and the matrix).
    __device__ __forceinline__ const T *col(int o, int64_t &step) const {
        if (ring) {
            step = 1;
            return ring + wrap_slot(cur + o, nslot) * rs;
        }
        step = stride;
        return g + (jc + (int64_t)dir * o) * cs;
    }
    __device__ __forceinline__ void advance() {
        jc += dir;
        if (ring) cur = wrap_slot(cur + 1, nslot);
    }
};

// Tile loop of a block sweep: positions [0, npos) in tiles of kCtaTile; the
// copies of tile t + 1 are issued before tile t runs and waited for after it.
// issue(q0): every stream's copies for the tile starting at q0 (q0 = 0: the
// first tile's whole span); row(q) runs one row; advance() moves every stream.
template <class Issue, class Row, class Advance>
__device__ __forceinline__ void cta_tiles(int64_t npos, Issue issue, Row row, Advance advance) {
    issue((int64_t)0);
    cta_commit();
    cta_wait_all();
    __syncthreads();
    for (int64_t q0 = 0; q0 < npos; q0 += kCtaTile) {
        issue(q0 + kCtaTile);
        cta_commit();
        const int64_t q1 = imin64(q0 + kCtaTile, npos);
        for (int64_t q = q0; q < q1; ++q) {
            row(q);
            advance();
        }
        cta_wait_all();
        __syncthreads();
    }
}

// ===========================================================================
// Forward: CHOL [+ SOLVE], SOLVE, ALG4 [+ SOLVE]; one block per chain.
// ===========================================================================
template <typename T, int FL>
__device__ void run_fwd_cta(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, T *sm, int mode,
                            const T *exact, int tier) {
    constexpr bool CHOL = (FL & F_CHOL) != 0, ALG4 = (FL & F_ALG4) != 0;
    const bool SOLVE = (FL & F_SOLVE) != 0 && P.k > 0;
    const int kk = SOLVE ? A.kk : 0;
    const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
    const int l = c.l, lw = l + 1, rs = cta_even(lw);
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    const int km = cta_rhs(P.k);
    T *W = sm;                                   // band window: pending Schur sums or pair adjoints
    T *U = W + (int64_t)lw * rs;                 // RHS ring (pending solve sums), km x lw
    T *lc = U + (int64_t)km * lw;                // column j of L (CHOL) or of the input L
    T *av = lc + lw;                             // CHOL: a_d; ALG4: b
    T *sr = av + lw;                             // ALG4: Sigma[i, i+t]
    T *uv = sr + lw;                             // ALG4: U[t]
    T *bu = uv + lw;                             // ALG4: bU[t]
    T *red = bu + 3 * lw;                        // block partial sums
    T *yv = red + 2 * kCtaWarps;                 // SOLVE: y_r of the row
    T *mem = yv + 4 * kCtaMaxK + 16;
    const int64_t j0 = cta_first_row(c, true, mode);
    const bool narrow = tier >= kTierNarrow, wide = tier >= kTierAll;
    CtaStream<T> sQ, sB, sSb, sS;
    mem = sQ.setup(CHOL ? A.Q + c.band : A.Lin + c.band, ld, cs, lw, lw, true, 0, 0, narrow, j0, 1, n, mem);
    mem = sB.setup(SOLVE ? A.Bin + c.rhs + (int64_t)A.rhs0 * c.ldr : nullptr, c.ldr, cs, kk, km, false, 0, 0, narrow,
                   j0, 1, n, mem);
    mem = sSb.setup(ALG4 ? A.Sbar + c.band : nullptr, ld, cs, lw, lw, true, 0, 0, narrow, j0, 1, n, mem);
    mem = sS.setup(ALG4 ? A.S + c.band : nullptr, ld, cs, lw, lw, true, l, 0, wide, j0, 1, n, mem);
    for (int64_t x = tid; x < (int64_t)(mem - sm); x += kCtaThreads) sm[x] = T(0);
    __syncthreads();
    T *Lo = CHOL ? A.L + c.band : nullptr;
    T *Lbo = ALG4 ? A.Lbar + c.band : nullptr;
    T *Xo = SOLVE ? A.Xout + c.rhs : nullptr;
    int32_t info = 0;
    int sj = (int)(j0 % lw);                     // slot of column j: j mod (l + 1)
    if (mode == RUN_EXACT && exact) cta_state_io(W, U, l, km, sj, const_cast<T *>(exact), false);
    auto row = [&](int64_t q) {
        const int64_t j = j0 + q;
        const bool out = j >= c.a;                // warm-up rows only carry the state
        if (j == c.a && !c.first) cta_state_io(W, U, l, km, sj, snap_ptr<T>(P, c.gseg, 0), true);
        const int dmax = (int)imin64(l, n - 1 - j);
        // ---- phase A: the row's inputs, the retired window column
        for (int d = tid; d <= l; d += kCtaThreads) {
            const T in = sQ.at(d, 0);
            if (CHOL) av[d] = (d < l) ? in - W[sj * rs + d] : in;
            else lc[d] = in;
            if (ALG4) {
                sr[d] = sS.at(d, 0);
                av[d] = W[sj * rs + d] + sSb.at(d, 0);
            }
            W[sj * rs + d] = T(0);                // retire column j; the slot serves column j + l + 1
        }
        if (SOLVE && tid < kk) {
            yv[tid] = sB.at(tid, 0) - U[tid * lw + sj];
            U[tid * lw + sj] = T(0);
        }
        __syncthreads();
        // ---- phase B: pivot / reciprocal, column of L, the row's scalars
        T rinv;
        if (CHOL) {
            const T piv = av[0];
            rinv = Num<T>::rsq(piv);
            if (out && tid == 0 && !(piv > T(0)) && info == 0) info = (int32_t)(j + 1);
            for (int d = tid; d <= l; d += kCtaThreads) {
                const T v = (d == 0) ? piv * rinv : av[d] * rinv;
                lc[d] = d <= dmax ? v : T(0);
                if (out) Lo[(int64_t)d * ld + j * cs] = d <= dmax ? v : T(0);
            }
        } else {
            rinv = Num<T>::rcp(lc[0]);
        }
        if (SOLVE && tid < kk) {
            // y_r needs only the pivot; the column of L is read after the barrier below
            const T y = yv[tid] * rinv;
            yv[tid] = y;
            if (out) Xo[(int64_t)(A.rhs0 + tid) * c.ldr + j * cs] = y;
        }
        if (ALG4) {
            const T b0 = av[0];
            for (int t = 1 + tid; t <= l; t += kCtaThreads) {
                const T u = lc[t] * rinv;
                uv[t] = u;
                bu[t] = -b0 * sr[t];
                av[t] = fma(-b0, u, av[t]);
            }
        }
        __syncthreads();
        // ---- phase C: window update
        if (CHOL) {
            // S(j+x, j+y) += L[j+x, j] L[j+y, j], 1 <= y <= x <= l: warp w takes the window columns
            // j+y, y = w+1, w+1+kCtaWarps, ..., its lanes the entries f = x - y of a column
            for (int y = 1 + warp; y <= l; y += kCtaWarps) {
                const T ly = lc[y];
                T *col = W + wrap_slot(sj + y, lw) * rs;
                for (int f = lane; f <= l - y; f += kWarp) col[f] = fma(lc[y + f], ly, col[f]);
            }
        }
        if (SOLVE) {
            // pending solve sums of columns j+1..j+l: warp r takes RHS r
            for (int r = warp; r < kk; r += kCtaWarps)
                for (int d = 1 + lane; d <= l; d += kWarp) {
                    const int ix = r * lw + wrap_slot(sj + d, lw);
                    U[ix] = fma(lc[d], yv[r], U[ix]);
                }
        }
        if (ALG4) {
            const int64_t i = j;
            // bU[t] -= sum_q b[q] Sigma(i+t, i+q); Sigma(i+b, i+a), a <= b, is entry b - a of
            // column i + a of S, a positions ahead in the S stream
            T part = T(0);
            cta_rows_reduce<T>(
                l, l,
                [&](int t, int qq, T acc) { return fma(av[qq], t < qq ? sS.at(qq - t, t) : sS.at(t - qq, qq), acc); },
                [&](int t, T acc) {
                    const T v = bu[t] - acc;
                    if (out && t <= dmax) {
                        T *p = &Lbo[(int64_t)t * ld + i * cs];
                        const T o = v * rinv;
                        *p = A.acc ? (*p + o) : o;
                    }
                    part = fma(v, lc[t], part);
                });
            // pair adjoints: pend(i+x, i+y) -= b[x] U[y] (+ b[y] U[x] for x != y), 1 <= y <= x <= l,
            // columns y over the warps and entries f = x - y over the lanes as above
            for (int y = 1 + warp; y <= l; y += kCtaWarps) {
                const T ay = av[y], uy = uv[y];
                T *col = W + wrap_slot(sj + y, lw) * rs;
                for (int f = lane; f <= l - y; f += kWarp) {
                    T v = col[f];
                    v = fma(-av[y + f], uy, v);
                    if (f) v = fma(-ay, uv[y + f], v);
                    col[f] = v;
                }
            }
            // diagonal of L-bar: -2 b0 / L_ii^3 - (sum_t bU[t] L[i+t, i]) / L_ii^2
            const T s = cta_block_sum(part, red);
            if (out && tid == 0) {
                const T r2 = rinv * rinv;
                const T o = T(-2) * av[0] * r2 * rinv - s * r2;
                T *p = &Lbo[i * cs];
                *p = A.acc ? (*p + o) : o;
                for (int t = dmax + 1; t <= l; ++t) Lbo[(int64_t)t * ld + i * cs] = T(0);   // corners
            }
        }
        __syncthreads();
    };
    auto issue = [&](int64_t q0) {
        CtaStream<T> *st[4] = {&sQ, &sB, &sSb, &sS};
        for (CtaStream<T> *x : st) {
            if (q0 == 0) x->issue_first();
            else x->issue_next(q0);
        }
    };
    auto advance = [&] {
        sj = wrap_slot(sj + 1, lw);
        sQ.advance(); sB.advance(); sSb.advance(); sS.advance();
    };
    cta_tiles(c.b - j0, issue, row, advance);
    if (!c.last) cta_state_io(W, U, l, km, sj, snap_ptr<T>(P, c.gseg, 1), true);
    if (CHOL) {
        // log det Q = 2 sum_j log L_jj over the segment's rows, summed by the whole block from
        // the diagonal it wrote (a logarithm per row on one thread would sit on every row's
        // critical path: FP64 is slow on this part)
        double part = 0.0;
        for (int64_t j = c.a + tid; j < c.b; j += kCtaThreads) part += log((double)Lo[j * cs]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        double *dred = reinterpret_cast<double *>(sm);
        __syncthreads();
        if (lane == 0) dred[warp] = part;
        __syncthreads();
        if (tid == 0) {
            double ldacc = 0.0;
            for (int w = 0; w < kCtaWarps; ++w) ldacc += dred[w];
            ldacc *= 2.0;
            if (c.first && c.last) {
                if (A.logdet) A.logdet[c.inst] = info ? (double)NAN : ldacc;
                A.info[c.inst] = info;
            } else {
                P.seg_logdet[c.gseg] = ldacc;
                P.seg_info[c.gseg] = info;
            }
        }
        __syncthreads();
    }
}

// ===========================================================================
// Backward: TAKA [+ SOLVE], SOLVE, ALG2 [+ SOLVE + OUTER]; one block per chain.
// ===========================================================================
template <typename T, int FL>
__device__ void run_bwd_cta(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, T *sm, int mode,
                            const T *exact, int tier) {
    constexpr bool TAKA = (FL & B_TAKA) != 0, ALG2 = (FL & B_ALG2) != 0;
    const bool SOLVE = (FL & B_SOLVE) != 0 && P.k > 0;
    const bool OUTER = (FL & B_OUTER) != 0 && SOLVE && ALG2;
    const int kk = SOLVE ? A.kk : 0;
    const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
    const int l = c.l, lw = l + 1, rs = cta_even(lw);
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    const int km = cta_rhs(P.k);
    T *W = sm;                                   // TAKA: Sigma window; ALG2: pending L-bar
    T *U = W + (int64_t)lw * rs;                 // SOLVE: ring of x (the sweep's output rows), km x lw
    T *lc = U + (int64_t)km * lw;                // column j of L
    T *rw = lc + lw;                             // TAKA: Sigma[i, i+q]; ALG2: L-bar / Q-bar of column j
    T *red = rw + 6 * lw;                        // block partial sums
    T *sc = red + 2 * kCtaWarps;                 // per-RHS scalars: x_j, y, ybar
    T *mem = sc + 4 * kCtaMaxK + 16;
    const int64_t j0 = cta_first_row(c, false, mode);
    const bool narrow = tier >= kTierNarrow, wide = tier >= kTierAll;
    const T *Lg = A.Lin + c.band;
    CtaStream<T> sL, sB, sLb, sLw, sX;
    mem = sL.setup(Lg, ld, cs, lw, lw, true, 0, 0, narrow, j0, -1, n, mem);
    mem = sB.setup(SOLVE ? A.Bin + c.rhs + (int64_t)A.rhs0 * c.ldr : nullptr, c.ldr, cs, kk, km, false, 0, 0, narrow,
                   j0, -1, n, mem);
    mem = sLb.setup(ALG2 ? A.Lbar_in + c.band : nullptr, ld, cs, lw, lw, true, 0, 0, narrow, j0, -1, n, mem);
    mem = sLw.setup(ALG2 ? Lg : nullptr, ld, cs, lw, lw, true, l, 0, wide, j0, -1, n, mem);
    mem = sX.setup(OUTER ? A.Xin + c.rhs + (int64_t)A.rhs0 * c.ldr : nullptr, c.ldr, cs, kk, km, false, 0, l, wide,
                   j0, -1, n, mem);
    for (int64_t x = tid; x < (int64_t)(mem - sm); x += kCtaThreads) sm[x] = T(0);
    __syncthreads();
    T *So = TAKA ? A.Sout + c.band : nullptr;
    T *Qo = ALG2 ? A.Qbar + c.band : nullptr;
    T *Xo = SOLVE ? A.Xout + c.rhs : nullptr;
    const T two_ldbar = (ALG2 && A.ldbar) ? T(2.0 * A.ldbar[c.inst]) : T(0);
    int sj = (int)(j0 % lw);                     // slot of column j: j mod (l + 1)
    if (mode == RUN_EXACT && exact) cta_state_io(W, U, l, km, sj, const_cast<T *>(exact), false);
    auto row = [&](int64_t q) {
        const int64_t j = j0 - q;
        const bool out = j < c.b;                 // warm-up rows only carry the state
        if (j == c.b - 1 && !c.last) cta_state_io(W, U, l, km, sj, snap_ptr<T>(P, c.gseg, 0), true);
        const int dmax = (int)imin64(l, n - 1 - j);
        // ---- phase A: column j of L, pending L-bar of column j, its retirement
        for (int d = tid; d <= l; d += kCtaThreads) lc[d] = sL.at(d, 0);
        if (ALG2) {
            for (int d = tid; d <= l; d += kCtaThreads) {
                const T v = sLb.at(d, 0);
                rw[d] = d >= 1 ? v + W[sj * rs + d] : v;        // pending L-bar of (j+d, j)
                W[sj * rs + d] = T(0);                          // retire column j
            }
        }
        __syncthreads();
        const T rinv = Num<T>::rcp(lc[0]);
        if (SOLVE && warp < kk) {
            // warp r: x_j = (b_j - sum_d L[j+d, j] x_{j+d}) / L_jj of RHS r, and (OUTER) y_r = (L^T X)[j]
            const int r = warp;
            T acc = T(0);
            for (int d = 1 + lane; d <= dmax; d += kWarp) acc = fma(lc[d], U[r * lw + wrap_slot(sj + d, lw)], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const T bj = sB.at(r, 0);
                const T xj = (bj - acc) * rinv;
                sc[r] = xj;
                sc[2 * kCtaMaxK + r] = bj;              // ybar of the OUTER term (Bin = Ybar)
                if (out) Xo[(int64_t)(A.rhs0 + r) * c.ldr + j * cs] = xj;
            }
            if (OUTER) {
                T y = T(0);
                for (int d = lane; d <= dmax; d += kWarp) y = fma(lc[d], sX.at(r, -d), y);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
                if (lane == 0) sc[kCtaMaxK + r] = y;
            }
        }
        if (TAKA) {
            // Sigma[i, i+q] = -sum_t U[t] Sigma(i+t, i+q), U[t] = L[i+t, i] / L_ii
            cta_rows_reduce<T>(
                l, l,
                [&](int qq, int t, T acc) {
                    const int a = t < qq ? t : qq, b = t < qq ? qq : t;
                    return fma(lc[t], W[wrap_slot(sj + a, lw) * rs + (b - a)], acc);
                },
                [&](int qq, T acc) { rw[qq] = qq <= dmax ? -acc * rinv : T(0); });
        }
        __syncthreads();
        if (TAKA) {
            const int64_t i = j;
            T part = T(0);
            for (int t = 1 + tid; t <= l; t += kCtaThreads) part = fma(lc[t], rw[t], part);
            const T s = cta_block_sum(part, red);
            const T diag = rinv * rinv - s * rinv;
            // outputs, then the new window column i: Sigma(i+q, i) for q = 0..l-1
            for (int qq = tid; qq <= l; qq += kCtaThreads) {
                const T v = qq == 0 ? diag : rw[qq];
                if (out) So[(int64_t)qq * ld + i * cs] = qq <= dmax ? v : T(0);
                if (qq < l) W[sj * rs + qq] = qq <= dmax ? v : T(0);
            }
        }
        if (SOLVE && tid < kk) U[tid * lw + sj] = sc[tid];      // x_j enters the ring
        if (ALG2) {
            // column j of L-bar: outer terms, log-det term, then Alg. 2 (off-diagonals first)
            if (OUTER) {
                // rw[d] -= sum_r X[j+d, r] ybar_r + x_{j+d, r} y_r (x_j itself is still in sc), lane
                // groups over d
                cta_rows_reduce<T>(
                    l + 1, kk,
                    [&](int t, int q, T acc) {
                        const int d = t - 1, r = q - 1;
                        const T bb = d == 0 ? sc[r] : U[r * lw + wrap_slot(sj + d, lw)];
                        acc = fma(sX.at(r, -d), sc[2 * kCtaMaxK + r], acc);
                        return fma(bb, sc[kCtaMaxK + r], acc);
                    },
                    [&](int t, T acc) { rw[t - 1] -= acc; });
                __syncthreads();
            }
            T part = T(0);
            for (int d = tid; d <= l; d += kCtaThreads) {
                T v = rw[d];
                if (d == 0) {
                    v = fma(two_ldbar, rinv, v);
                    rw[0] = v;
                } else {
                    const T qb = d <= dmax ? v * rinv : T(0);
                    rw[d] = qb;
                    part = fma(-qb, lc[d], part);
                }
            }
            const T s = cta_block_sum(part, red);        // (its barrier also publishes rw)
            const T qb0 = T(0.5) * (rw[0] + s) * rinv;
            for (int d = tid; out && d <= l; d += kCtaThreads) {
                const T v = d == 0 ? qb0 : rw[d];
                T *p = &Qo[(int64_t)d * ld + j * cs];
                *p = d <= dmax ? (A.acc ? (*p + v) : v) : T(0);
            }
            // pending L-bar of the window columns m = j - e, e = 1..nm: L[j+d, m] gets -Qb[d] L[j, m]
            // (d >= 1, d + e <= l); L[j, m] gets -2 Qb[0] L[j, m] - sum_d Qb[d] L[j+d, m]
            // (G lanes of a warp per column, as in cta_rows_reduce, with the column's pointers and
            // L[j, m] held across the lane's terms)
            const int nm = (int)imin64((int64_t)l, j);
            int G = kWarp;
            while (G > 1 && nm * G > kCtaThreads) G >>= 1;
            const int per_pass = kCtaThreads / G, g = tid % G;
            for (int e0 = 1; e0 <= nm; e0 += per_pass) {
                const int e = e0 + tid / G;
                T acc = T(0), ljm = T(0);
                T *wc = W;
                if (e <= nm) {
                    int64_t st;
                    const T *lcol = sLw.col(e, st);               // column m = j - e of L
                    wc = W + wrap_slot(sj - e, lw) * rs;           // its pending L-bar
                    ljm = lcol[e * st];                            // L[j, m]
                    const int dl = dmax < l - e ? dmax : l - e;    // L[j+d, m] inside the band
                    const T *pl = lcol + (int64_t)(1 + g + e) * st; // L[j+d, m], d = 1 + g, 1 + g + G, ...
                    const int64_t pstep = (int64_t)G * st;
                    for (int d = 1 + g; d <= dl; d += G, pl += pstep) {
                        const T qb = rw[d];
                        wc[d + e] = fma(-qb, ljm, wc[d + e]);
                        acc = fma(qb, *pl, acc);
                    }
                }
                for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (g == 0 && e <= nm) wc[e] = wc[e] - T(2) * qb0 * ljm - acc;
            }
        }
        __syncthreads();
        // column j + l leaves the TAKA window and the x ring (row j - 1 reads columns j ..
        // j + l - 1) and its slot is the next row's: cleared, so that a saved state holds
        // live columns only
        const int sx = wrap_slot(sj + l, lw);
        for (int r = tid; SOLVE && r < kk; r += kCtaThreads) U[r * lw + sx] = T(0);
        if (TAKA)
            for (int f = tid; f < rs; f += kCtaThreads) W[sx * rs + f] = T(0);
    };
    auto issue = [&](int64_t q0) {
        CtaStream<T> *st[5] = {&sL, &sB, &sLb, &sLw, &sX};
        for (CtaStream<T> *x : st) {
            if (q0 == 0) x->issue_first();
            else x->issue_next(q0);
        }
    };
    auto advance = [&] {
        sj = wrap_slot(sj - 1, lw);
        sL.advance(); sB.advance(); sLb.advance(); sLw.advance(); sX.advance();
    };
    cta_tiles(j0 - c.a + 1, issue, row, advance);
    if (!c.first) cta_state_io(W, U, l, km, sj, snap_ptr<T>(P, c.gseg, 1), true);
}

}  // namespace bnd
