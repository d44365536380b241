// Block-cooperative sweeps for wide bands: one thread block per chain, the
// computed window of the recurrence in shared memory, every O(l^2) step of a
// row spread over the block's threads.
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
// of l + 1 consecutive columns c: entry (r, c) sits at W[slot(c) (l+1) +
// (r - c)] with slot(c) = c mod (l+1), so moving the window by one column
// retires one slot and reuses it for the column entering on the other side
// (zeroed first) -- nothing is copied.  RHS windows are (l+1)-slot rings.
// Input-derived windows (the Sigma block of Alg. 4 from S, the L entries of
// Alg. 2) are read from the inputs directly: the few columns they span stay
// in L2.
//
// Per row: three block barriers (load / finish the row's scalars / window
// update).  The O(l^2) work of a row (rank-1 window update, or a matrix-vector
// product with a window and a rank-1 update) is spread over the block.
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
constexpr size_t kCtaSmemLimit = 232448;         // 227 KB of shared memory per block

// Shared-memory elements of a block sweep for bandwidth l (one band window,
// two RHS windows, row vectors, partial sums).
__host__ __device__ inline int64_t cta_smem_elems(int l) {
    const int64_t lw = l + 1;
    return lw * lw + 2 * (int64_t)kCtaMaxK * lw + 6 * lw + 2 * kCtaWarps + 4 * kCtaMaxK + 8;
}
// The block sweeps serve bandwidth l in dtype T when its windows fit (1 KB is
// left for the verify kernel's static shared memory).
template <typename T>
__host__ __device__ inline bool cta_fits(int l) {
    return sizeof(T) * (size_t)cta_smem_elems(l) <= kCtaSmemLimit - 1024;
}
// Words of a block sweep's state snapshot: the band window and the RHS ring,
// rotated so that the slot of the current column comes first.
__host__ __device__ inline int64_t cta_state_words(int l) {
    const int64_t lw = l + 1;
    return lw * lw + (int64_t)kCtaMaxK * lw;
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

// The pairs (x, y), 1 <= y <= x <= l, of a triangle folded into a rectangle of
// ceil(l/2) rows of l + 1 entries: rectangle row i holds triangle row i
// (entries 0..i) followed by triangle row l-1-i, so the rectangle has no holes
// (odd l: the last rectangle row is half padding).  Thread t visits entries
// t, t + kCtaThreads, ... without divisions inside the loop.
struct FoldIter {
    int l, lw, i, b, di, db, np, p;
    __device__ FoldIter(int l_, int tid) : l(l_), lw(l_ + 1) {
        np = ((l + 1) / 2) * lw;
        p = tid;
        i = tid / lw;
        b = tid - i * lw;
        di = kCtaThreads / lw;
        db = kCtaThreads - di * lw;
    }
    __device__ __forceinline__ bool valid() const { return p < np; }
    __device__ __forceinline__ bool pair(int &x, int &y) const {
        int xr, yr;
        bool ok;
        if (b <= i) { xr = i; yr = b; ok = xr < l; }
        else { xr = l - 1 - i; yr = b - i - 1; ok = xr > i; }   // odd l: the middle row appears once
        x = xr + 1;
        y = yr + 1;
        return ok;
    }
    __device__ __forceinline__ void next() {
        p += kCtaThreads;
        i += di;
        b += db;
        if (b >= lw) { b -= lw; ++i; }
    }
};

__device__ __forceinline__ int wrap_slot(int s, int lw) { return s >= lw ? s - lw : (s < 0 ? s + lw : s); }

// Save (or load) the state of a block sweep whose current column has slot sj:
// word x < (l+1)^2 is entry f of the window column rel slots after sj
// (x = rel (l+1) + f), then RHS ring row r, rel slots after sj.  Whole block.
template <typename T>
__device__ void cta_state_io(T *W, T *U, int l, int sj, T *snap, bool save) {
    const int lw = l + 1, nw = lw * lw;
    __syncthreads();
    for (int x = threadIdx.x; x < nw + kCtaMaxK * lw; x += kCtaThreads) {
        T *live;
        if (x < nw) {
            const int rel = x / lw, f = x - rel * lw;
            live = W + wrap_slot(sj + rel, lw) * lw + f;
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

// Whole block: true when snapshots x and y (cta_state_io layout, bandwidth l)
// are close in the sense above.
template <typename T>
__device__ bool cta_states_close(const T *x, const T *y, int l) {
    __shared__ T buf[2 * kCtaWarps];
    const int lw = l + 1, nw = lw * lw;
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
    for (int r = warp; r < kCtaMaxK; r += kCtaWarps) {       // RHS row r: warp r
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

// ===========================================================================
// Forward: CHOL [+ SOLVE], SOLVE, ALG4 [+ SOLVE]; one block per chain.
// ===========================================================================
template <typename T, int FL>
__device__ void run_fwd_cta(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, T *sm, int mode,
                            const T *exact) {
    constexpr bool CHOL = (FL & F_CHOL) != 0, ALG4 = (FL & F_ALG4) != 0;
    const bool SOLVE = (FL & F_SOLVE) != 0 && P.k > 0;
    const int kk = SOLVE ? A.kk : 0;
    const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
    const int l = c.l, lw = l + 1;
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    T *W = sm;                                   // band window: pending Schur sums or pair adjoints
    T *U = W + (int64_t)lw * lw;                 // RHS rings, kCtaMaxK x lw
    T *lc = U + 2 * (int64_t)kCtaMaxK * lw;      // column j of L (CHOL) or of the input L
    T *av = lc + lw;                             // CHOL: a_d; ALG4: b
    T *sr = av + lw;                             // ALG4: Sigma[i, i+t]
    T *uv = sr + lw;                             // ALG4: U[t]
    T *bu = uv + lw;                             // ALG4: bU[t]
    T *red = bu + 2 * lw;                        // block partial sums (2 sets)
    T *yv = red + 2 * kCtaWarps;                 // SOLVE: y_r of the row
    for (int64_t x = tid; x < cta_smem_elems(l); x += kCtaThreads) sm[x] = T(0);
    __syncthreads();
    const T *Qi = CHOL ? A.Q + c.band : nullptr;
    const T *Li = CHOL ? nullptr : A.Lin + c.band;
    T *Lo = CHOL ? A.L + c.band : nullptr;
    const T *Si = ALG4 ? A.S + c.band : nullptr;
    const T *Sbi = ALG4 ? A.Sbar + c.band : nullptr;
    T *Lbo = ALG4 ? A.Lbar + c.band : nullptr;
    const T *Bi = SOLVE ? A.Bin + c.rhs : nullptr;
    T *Xo = SOLVE ? A.Xout + c.rhs : nullptr;
    int32_t info = 0;
    const int64_t j0 = cta_first_row(c, true, mode);
    int sj = (int)(j0 % lw);                     // slot of column j: j mod (l + 1)
    if (mode == RUN_EXACT && exact) cta_state_io(W, U, l, sj, const_cast<T *>(exact), false);
    for (int64_t j = j0; j < c.b; ++j, sj = wrap_slot(sj + 1, lw)) {
        const bool out = j >= c.a;                // warm-up rows only carry the state
        if (j == c.a && !c.first) cta_state_io(W, U, l, sj, snap_ptr<T>(P, c.gseg, 0), true);
        const int dmax = (int)imin64(l, n - 1 - j);
        // ---- phase A: the row's inputs, the retired window column
        for (int d = tid; d <= l; d += kCtaThreads) {
            const bool in = d <= dmax;
            if (CHOL) {
                const T q = in ? Qi[(int64_t)d * ld + j * cs] : T(0);
                av[d] = (d < l) ? q - W[sj * lw + d] : q;
            } else {
                lc[d] = in ? Li[(int64_t)d * ld + j * cs] : T(0);
            }
            if (ALG4) {
                sr[d] = in ? Si[(int64_t)d * ld + j * cs] : T(0);
                av[d] = W[sj * lw + d] + (in ? Sbi[(int64_t)d * ld + j * cs] : T(0));
            }
            W[sj * lw + d] = T(0);                // retire column j; the slot serves column j + l + 1
        }
        if (SOLVE && tid < kk) {
            const int64_t co = (int64_t)(A.rhs0 + tid) * c.ldr;
            yv[tid] = Bi[co + j * cs] - U[tid * lw + sj];
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
        if (SOLVE) {
            __syncthreads();                      // lc complete (CHOL) before the RHS rows use it
            if (tid < kk) {
                const T y = yv[tid] * rinv;
                yv[tid] = y;
                if (out) Xo[(int64_t)(A.rhs0 + tid) * c.ldr + j * cs] = y;
            }
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
            // S(j+x, j+y) += L[j+x, j] L[j+y, j], 1 <= y <= x <= l
            for (FoldIter it(l, tid); it.valid(); it.next()) {
                int x, y;
                if (!it.pair(x, y)) continue;
                const int ix = wrap_slot(sj + y, lw) * lw + (x - y);
                W[ix] = fma(lc[x], lc[y], W[ix]);
            }
        }
        if (SOLVE) {
            for (int e = tid; e < kk * l; e += kCtaThreads) {
                const int r = e / l, d = e - r * l + 1;
                const int ix = r * lw + wrap_slot(sj + d, lw);
                U[ix] = fma(lc[d], yv[r], U[ix]);
            }
        }
        if (ALG4) {
            const int64_t i = j;
            // bU[t] -= sum_q b[q] Sigma(i+t, i+q): one warp per t, lanes over q
            T part = T(0);
            for (int t = 1 + warp; t <= l; t += kCtaWarps) {
                T acc = T(0);
                for (int q = 1 + lane; q <= l; q += kWarp) {
                    const int a = t < q ? t : q, b = t < q ? q : t;
                    const T sig = (i + b < n) ? Si[(int64_t)(b - a) * ld + (i + a) * cs] : T(0);
                    acc = fma(av[q], sig, acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                const T v = bu[t] - acc;
                if (lane == 0) {
                    if (out && t <= dmax) {
                        T *p = &Lbo[(int64_t)t * ld + i * cs];
                        const T o = v * rinv;
                        *p = A.acc ? (*p + o) : o;
                    }
                    part = fma(v, lc[t], part);
                }
            }
            // pair adjoints: pend(i+t, i+q) -= b[q] U[t] (+ b[t] U[q] for t != q)
            for (FoldIter it(l, tid); it.valid(); it.next()) {
                int x, y;
                if (!it.pair(x, y)) continue;
                const int ix = wrap_slot(sj + y, lw) * lw + (x - y);
                T v = W[ix];
                v = fma(-av[x], uv[y], v);
                if (x != y) v = fma(-av[y], uv[x], v);
                W[ix] = v;
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
    }
    if (!c.last) cta_state_io(W, U, l, sj, snap_ptr<T>(P, c.gseg, 1), true);
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
                            const T *exact) {
    constexpr bool TAKA = (FL & B_TAKA) != 0, ALG2 = (FL & B_ALG2) != 0;
    const bool SOLVE = (FL & B_SOLVE) != 0 && P.k > 0;
    const bool OUTER = (FL & B_OUTER) != 0 && SOLVE && ALG2;
    const int kk = SOLVE ? A.kk : 0;
    const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
    const int l = c.l, lw = l + 1;
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    T *W = sm;                                   // TAKA: Sigma window; ALG2: pending L-bar
    T *U = W + (int64_t)lw * lw;                 // SOLVE: ring of x (the sweep's output rows)
    T *xv = U + (int64_t)kCtaMaxK * lw;          // OUTER: X[j+d], d = 0..l, of every RHS (kk x lw)
    T *lc = xv + (int64_t)kCtaMaxK * lw;         // column j of L
    T *rw = lc + lw;                             // TAKA: Sigma[i, i+q]; ALG2: L-bar / Q-bar of column j
    T *red = rw + 5 * lw;                        // block partial sums (2 sets)
    T *sc = red + 2 * kCtaWarps;                 // per-RHS scalars: x_j, y, ybar, x0
    for (int64_t x = tid; x < cta_smem_elems(l); x += kCtaThreads) sm[x] = T(0);
    __syncthreads();
    const T *Li = A.Lin + c.band;
    T *So = TAKA ? A.Sout + c.band : nullptr;
    const T *Lbi = ALG2 ? A.Lbar_in + c.band : nullptr;
    T *Qo = ALG2 ? A.Qbar + c.band : nullptr;
    const T *Bi = SOLVE ? A.Bin + c.rhs : nullptr;
    T *Xo = SOLVE ? A.Xout + c.rhs : nullptr;
    const T *Xi = OUTER ? A.Xin + c.rhs : nullptr;
    const T two_ldbar = (ALG2 && A.ldbar) ? T(2.0 * A.ldbar[c.inst]) : T(0);
#define LIN(r_, m_) Li[(int64_t)((r_) - (m_)) * ld + (m_) * cs]
    const int64_t j0 = cta_first_row(c, false, mode);
    int sj = (int)(j0 % lw);                     // slot of column j: j mod (l + 1)
    if (mode == RUN_EXACT && exact) cta_state_io(W, U, l, sj, const_cast<T *>(exact), false);
    for (int64_t j = j0; j >= c.a; --j, sj = wrap_slot(sj - 1, lw)) {
        const bool out = j < c.b;                 // warm-up rows only carry the state
        if (j == c.b - 1 && !c.last) cta_state_io(W, U, l, sj, snap_ptr<T>(P, c.gseg, 0), true);
        const int dmax = (int)imin64(l, n - 1 - j);
        // ---- phase A: column j of L; SOLVE reductions x_j = (b_j - sum_d L[j+d,j] x_{j+d}) / L_jj
        for (int d = tid; d <= l; d += kCtaThreads) lc[d] = d <= dmax ? Li[(int64_t)d * ld + j * cs] : T(0);
        if (ALG2) {
            for (int d = tid; d <= l; d += kCtaThreads) {
                const T v = d <= dmax ? Lbi[(int64_t)d * ld + j * cs] : T(0);
                rw[d] = d >= 1 ? v + W[sj * lw + d] : v;        // pending L-bar of (j+d, j)
                W[sj * lw + d] = T(0);                          // retire column j
            }
        }
        if (OUTER) {
            for (int e = tid; e < kk * lw; e += kCtaThreads) {
                const int r = e / lw, d = e - r * lw;
                xv[r * lw + d] = d <= dmax ? Xi[(int64_t)(A.rhs0 + r) * c.ldr + (j + d) * cs] : T(0);
            }
        }
        __syncthreads();
        const T rinv = Num<T>::rcp(lc[0]);
        if (SOLVE && warp < kk) {
            // warp r: x_j of RHS r, and (OUTER) y_r = (L^T X)[j]
            const int r = warp;
            const int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
            T acc = T(0);
            for (int d = 1 + lane; d <= dmax; d += kWarp) acc = fma(lc[d], U[r * lw + wrap_slot(sj + d, lw)], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const T bj = Bi[co + j * cs];
                const T xj = (bj - acc) * rinv;
                sc[r] = xj;
                sc[2 * kCtaMaxK + r] = bj;              // ybar of the OUTER term (Bin = Ybar)
                if (out) Xo[co + j * cs] = xj;
            }
            if (OUTER) {
                T y = T(0);
                for (int d = lane; d <= dmax; d += kWarp) y = fma(lc[d], xv[r * lw + d], y);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
                if (lane == 0) sc[kCtaMaxK + r] = y;
            }
        }
        if (TAKA) {
            // Sigma[i, i+q] = -sum_t U[t] Sigma(i+t, i+q), U[t] = L[i+t, i] / L_ii: one warp per q
            const int64_t i = j;
            for (int q = 1 + warp; q <= l; q += kCtaWarps) {
                T acc = T(0);
                for (int t = 1 + lane; t <= l; t += kWarp) {
                    const int a = t < q ? t : q, b = t < q ? q : t;
                    acc = fma(lc[t], W[wrap_slot(sj + a, lw) * lw + (b - a)], acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) rw[q] = q <= dmax ? -acc * rinv : T(0);
            }
        }
        __syncthreads();
        if (TAKA) {
            const int64_t i = j;
            T part = T(0);
            for (int t = 1 + tid; t <= l; t += kCtaThreads) part = fma(lc[t], rw[t], part);
            const T s = cta_block_sum(part, red);
            const T diag = rinv * rinv - s * rinv;
            // outputs, then the new window column i: Sigma(i+q, i) for q = 0..l-1
            for (int q = tid; q <= l; q += kCtaThreads) {
                const T v = q == 0 ? diag : rw[q];
                if (out) So[(int64_t)q * ld + i * cs] = q <= dmax ? v : T(0);
                if (q < l) W[sj * lw + q] = q <= dmax ? v : T(0);
            }
        }
        if (SOLVE && tid < kk) U[tid * lw + sj] = sc[tid];      // x_j enters the ring
        if (ALG2) {
            // column j of L-bar: outer terms, log-det term, then Alg. 2 (off-diagonals first)
            T part = T(0);
            for (int d = tid; d <= l; d += kCtaThreads) {
                T v = rw[d];
                if (OUTER) {
                    for (int r = 0; r < kk; ++r) {
                        const T ybar = sc[2 * kCtaMaxK + r], y = sc[kCtaMaxK + r];
                        const T bb = d == 0 ? sc[r] : U[r * lw + wrap_slot(sj + d, lw)];
                        v = fma(-xv[r * lw + d], ybar, v);
                        v = fma(-bb, y, v);
                    }
                }
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
            // pending L-bar of the window columns m in [j - l, j): L[j+d, m] gets -Qb[d] L[j, m]
            // (d >= 1, j + d - m <= l); L[j, m] gets -2 Qb[0] L[j, m] - sum_d Qb[d] L[j+d, m]
            const int nm = (int)imin64((int64_t)l, j);      // window columns m = j-1 .. j-nm
            for (int e0 = warp; e0 < nm; e0 += kCtaWarps) {
                const int e = nm - e0;                    // m = j - e, e = 1..nm
                const int64_t m = j - e;
                const int dlim = (int)imin64((int64_t)dmax, (int64_t)(l - e));
                const int sm_ = wrap_slot(sj - e, lw) * lw;
                const T ljm = LIN(j, m);
                T acc = T(0);
                for (int d = 1 + lane; d <= dlim; d += kWarp) {
                    const T qb = rw[d];
                    acc = fma(qb, LIN(j + d, m), acc);
                    W[sm_ + d + e] = fma(-qb, ljm, W[sm_ + d + e]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) W[sm_ + e] = W[sm_ + e] - T(2) * qb0 * ljm - acc;
            }
        }
        __syncthreads();
        // column j + l leaves the TAKA window and the x ring (row j - 1 reads columns j ..
        // j + l - 1) and its slot is the next row's: cleared, so that a saved state holds
        // live columns only
        const int sx = wrap_slot(sj + l, lw);
        for (int r = tid; SOLVE && r < kk; r += kCtaThreads) U[r * lw + sx] = T(0);
        if (TAKA)
            for (int f = tid; f < lw; f += kCtaThreads) W[sx * lw + f] = T(0);
    }
    if (!c.first) cta_state_io(W, U, l, sj, snap_ptr<T>(P, c.gseg, 1), true);
#undef LIN
}

}  // namespace bnd
