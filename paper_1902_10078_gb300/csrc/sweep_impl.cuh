// Sequential-in-n band sweeps of the banded operators (register-window and
// generic forms).  Included by the per-dtype translation units.
//
// Every sweep walks the columns of one chain (a row segment of one instance)
// in one direction and carries a small window of state in registers:
//
//   forward sweeps (j ascending)
//     CHOL  : Cholesky, Alg. 1, in column (left-looking, pending-sum) order:
//             a_d = Q[j+d, j] - sum_{m<j} L[j+d, m] L[j, m]; L_jj = sqrt(a_0);
//             L[j+d, j] = a_d / L_jj.  Same entries and formulas as Alg. 1;
//             only the order in which entries are produced differs.
//     SOLVE : y = L^{-1} b in column (axpy) order.
//     ALG4  : reverse mode of the subset inverse (Alg. 4), taken as the exact
//             reverse of the row-ordered Takahashi recursion below; the pair
//             adjoints of the symmetric S are one value per unordered pair
//             (i, j), seeded with the gradient of the stored entry.
//   backward sweeps (j descending)
//     TAKA  : subset inverse, Alg. 3, in row order: for i descending,
//             Sym[i, i+q] = -sum_t U[i, i+t] Sym[i+t, i+q] (q = l..1), then
//             Sym[i, i] = 1/L_ii^2 - sum_t U[i, i+t] Sym[i, i+t],
//             U[i, m] = L[m, i] / L_ii.  Same recursion as Alg. 3.
//     SOLVE : x = L^{-T} y (dot order).
//     ALG2  : reverse mode of the Cholesky (Alg. 2) in column-reverse order,
//             with the Table-1 solve adjoint outer products and the log-det
//             term added to Lbar of each column before it is consumed.
//
// Long instances are split into segments.  A segment whose start is not the
// instance's boundary starts `warm` columns early from a cold (zero) state;
// the state entering its first output column is saved ("start snapshot"),
// and the state after its last output column likewise ("end snapshot").  A
// verify pass compares neighbours bit for bit and reruns mismatching
// segments from the exact end snapshot of their predecessor.
#pragma once

#include <climits>
#include <utility>

#include "common.cuh"
#include "sweep_io.cuh"

namespace bnd {

// ---------------------------------------------------------------------------
// Flags
// ---------------------------------------------------------------------------
enum : int { F_CHOL = 1, F_SOLVE = 2, F_ALG4 = 4 };
enum : int { B_TAKA = 1, B_SOLVE = 2, B_ALG2 = 4, B_OUTER = 8 };

template <typename T>
struct SweepArgs {
    const T *Q;          // CHOL input
    T *L;                // CHOL output
    const T *Lin;        // L input of every other sweep
    const T *S;          // ALG4 input
    const T *Sbar;       // ALG4 input
    T *Sout;             // TAKA output
    T *Lbar;             // ALG4 output (accumulated when acc)
    const T *Lbar_in;    // ALG2 input
    T *Qbar;             // ALG2 output (accumulated when acc)
    T *scratch;          // generic path band scratch 1 (zeroed before the launch)
    T *scratch2;         // generic path band scratch 2
    const T *Bin;        // SOLVE input (B or Y)
    T *Xout;             // SOLVE output
    const T *Xin;        // ALG2+OUTER: forward output X (Y = L^T X)
    const T *Ybar;       // ALG2+OUTER: Ybar (= Bin of the fused backward)
    int32_t rhs0;        // first RHS column handled by this launch
    int32_t kk;          // RHS columns handled by this launch (<= the kernel's K)
    int32_t acc;         // accumulate into Lbar / Qbar
    const double *ldbar; // ALG2: per-instance log-det cotangent (nullable)
    double *logdet;      // CHOL: per-instance log det (final)
    int32_t *info;       // CHOL: per-instance info (final)
    int32_t kind;        // SweepKind of this launch (snapshots, counters)
};

template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float rcp(float x) { return 1.0f / x; }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};
// FP64 reciprocal and reciprocal square root of the per-row critical path.
// FP64 arithmetic on this part is slow (about 64 cycles per dependent FMA), so
// instead of the IEEE division and the library rsqrt these take the FP32
// hardware estimate (relative error below 2^-22) and refine it with two
// Newton-Raphson steps, each of which about squares the relative error
// (2^-44, then below the FP64 rounding unit): accurate to about one ulp, not
// correctly rounded, and without branches inside the FP32 exponent range
// (outside it, and for zero, negative or non-finite arguments, the IEEE
// operation is used).
//   1/x:       r <- r + r (1 - x r)
//   1/sqrt(x): r <- r + (r / 2) (1 - x r^2)
__device__ __forceinline__ double rcp_newton(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-36 && ax < 1e36)) return 1.0 / x;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)x));
    double r = (double)rf;
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ double rsqrt_newton(double x) {
    if (!(x > 1e-36 && x < 1e36)) return rsqrt(x);
    float rf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)x));
    double r = (double)rf;
    double e = fma(-x * r, r, 1.0);
    r = fma(0.5 * r, e, r);
    e = fma(-x * r, r, 1.0);
    return fma(0.5 * r, e, r);
}
template <> struct Num<double> {
    static __device__ __forceinline__ double rsq(double x) { return rsqrt_newton(x); }
    static __device__ __forceinline__ double rcp(double x) { return rcp_newton(x); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

// Index of the unordered pair (a, b), 0 <= a, b < L, in a packed triangle.
__host__ __device__ constexpr int tri(int a, int b, int L) {
    return (a <= b) ? (a * L - (a * (a - 1)) / 2 + (b - a)) : (b * L - (b * (b - 1)) / 2 + (a - b));
}
template <int L> struct Tri { static constexpr int N = L * (L + 1) / 2; };

// Per-chain context: instance view plus the segment's rows.
struct ChainCtx {
    int64_t n, band, ld, rhs, ldr;
    int64_t cs;          // column stride
    int64_t a, b;        // output rows [a, b)
    int64_t gseg;        // global segment id
    int64_t warm;        // warm-up rows of a speculative start
    int32_t inst;        // instance index
    int32_t l;
    bool first, last;    // first / last segment of the instance
};

template <typename T>
__device__ __forceinline__ T *snap_ptr(const PlanDev &P, int64_t gseg, int which) {
    return reinterpret_cast<T *>(P.snap) + (gseg * 2 + which) * P.snap_words;
}

// Bitwise equality of two state snapshots.
template <typename T>
__device__ inline bool snap_equal(const T *x, const T *y, int64_t words) {
    bool eq = true;
    for (int64_t w = 0; w < words; ++w) {
        if (sizeof(T) == 4) eq &= (__float_as_uint((float)x[w]) == __float_as_uint((float)y[w]));
        else eq &= (__double_as_longlong((double)x[w]) == __double_as_longlong((double)y[w]));
    }
    return eq;
}

// Warp-wide minimum / maximum (every lane of the warp must call).
__device__ __forceinline__ int64_t warp_min64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ int64_t warp_max64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Bounds guard of a step: boundary tiles check, interior tiles compile the check away.
template <bool CHECK>
__device__ __forceinline__ bool inb(int64_t x, int64_t n) { return !CHECK || x < n; }

// Sum of log pivots: log det Q = sum_j log(piv_j) with piv_j = L_jj^2.  FP64
// instances sum log() in double; FP32 instances use logf with a compensated
// (Kahan) float sum, converted to double once per chain, which keeps FP64
// arithmetic (slow on this part) off the per-row path.
template <typename T> struct LogSum;
// FP64: the running product of the pivots kept as m 2^e with m in [0.5, 1) (one
// multiplication and a few integer operations per row), and one logarithm at
// the end: a logarithm per row costs some 40 FP64 operations on this part's
// slow FP64 pipe.  Each row rounds the product once, so the relative error of
// the product after n rows is below n 2^-53 (an absolute error below n 2^-53
// in the log-det).  Pivots whose product leaves the normal range (or that are
// not positive: the factorization has failed then) go to a plain sum of
// logarithms instead.
template <> struct LogSum<double> {
    double m = 1.0, slow = 0.0;
    long long e = 0;
    __device__ __forceinline__ void add(double piv) {
        const double p = m * piv;
        if (p >= 2.2250738585072014e-308 && p <= 1.7976931348623157e308) {
            const long long b = __double_as_longlong(p);
            e += ((b >> 52) & 0x7ff) - 1022;
            m = __longlong_as_double((b & ~(0x7ffLL << 52)) | (1022LL << 52));
        } else {
            slow += log(piv);
        }
    }
    __device__ __forceinline__ double value() const { return log(m) + (double)e * 0.6931471805599453 + slow; }
};
template <> struct LogSum<float> {
    float s = 0.0f, comp = 0.0f;
    __device__ __forceinline__ void add(float piv) {
        const float y = logf(piv) - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)comp; }
};

// Start modes of a chain run.
enum : int { RUN_COLD = 0, RUN_EXACT = 1 };

// Interior tiles of bandwidths up to this value unroll their rows (the step
// body is instantiated once per row of the tile); wider bands keep one copy of
// the body, whose size otherwise overflows the instruction cache.
#ifndef BND_INTERIOR_UNROLL_MAX_L
#define BND_INTERIOR_UNROLL_MAX_L 4
#endif

// ===========================================================================
// Register-window forward sweep: CHOL [+ SOLVE], SOLVE, ALG4 [+ SOLVE]
// Input streams:  [0, L]      Q (CHOL) or L, diagonal d, column j
//                 RHS block   B column r, row j                      (SOLVE)
//                 [SA, SA+L)  S diagonal d at column j+1+L-d         (ALG4: new block entries)
//                 SL          S diagonal L at column j               (ALG4)
//                 [SB, SB+L]  Sbar diagonal d at column j            (ALG4)
// Output streams: [0, L] L (CHOL) or Lbar (ALG4); then the RHS block (SOLVE)
// ===========================================================================
template <typename T, int L, int K, int FL>
struct FwdReg {
    static constexpr int NT = Tri<L>::N;
    static constexpr bool CHOL = (FL & F_CHOL) != 0;
    static constexpr bool SOLVE = (FL & F_SOLVE) != 0 && K > 0;
    static constexpr bool ALG4 = (FL & F_ALG4) != 0;
    static constexpr int KK = SOLVE ? K : 1;
    static constexpr int I_RHS = L + 1;
    static constexpr int I_SA = I_RHS + (SOLVE ? KK : 0);
    static constexpr int I_SL = I_SA + L;
    static constexpr int I_SB = I_SL + 1;
    static constexpr int NIN = I_SA + (ALG4 ? 2 * L + 2 : 0);
    static constexpr bool BAND_OUT = CHOL || ALG4;
    static constexpr int O_RHS = BAND_OUT ? L + 1 : 0;
    static constexpr int NOUT = O_RHS + (SOLVE ? KK : 0);
    __host__ __device__ static constexpr StreamSpec in_spec(int s) {
        if (s <= L) return StreamSpec{CHOL ? POOL_Q : POOL_LIN, s, 0};
        if (SOLVE && s < I_SA) return StreamSpec{POOL_BIN, s - I_RHS, 0};
        if (s < I_SL) return StreamSpec{POOL_S, s - I_SA, 1 + L - (s - I_SA)};
        if (s == I_SL) return StreamSpec{POOL_S, L, 0};
        return StreamSpec{POOL_SBAR, s - I_SB, 0};
    }
    __host__ __device__ static constexpr StreamSpec out_spec(int o) {
        if (BAND_OUT && o <= L) return StreamSpec{CHOL ? POOL_LOUT : POOL_LBAR, o, 0};
        return StreamSpec{POOL_XOUT, o - O_RHS, 0};
    }

    // computed state
    T pw[NT];           // CHOL: pending Schur sums, pair (c-j, r-j) in [0, L-1]
    T pend[NT];         // ALG4: pending pair adjoints, pair (t, q) relative to i, in [0, L-1]
    T u[KK][L];         // SOLVE: pending sums for rows j..j+L-1
    // input-derived state
    T sblk[NT];         // ALG4: Sigma block of rows/cols i+1..i+L, pair (t-1, q-1)
    T srow[L];          // ALG4: Sigma[i, i+d], d < L, carried from the previous block

    static constexpr int snap_words() { return (CHOL ? NT : 0) + (ALG4 ? NT : 0) + (SOLVE ? K * L : 0); }

    __device__ void save(T *dst) const {
        int o = 0;
        if (CHOL) { _Pragma("unroll") for (int x = 0; x < NT; ++x) dst[o++] = pw[x]; }
        if (ALG4) { _Pragma("unroll") for (int x = 0; x < NT; ++x) dst[o++] = pend[x]; }
        if (SOLVE) { _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) dst[o++] = u[r][d]; }
    }
    __device__ void load_state(const T *src) {
        int o = 0;
        if (CHOL) { _Pragma("unroll") for (int x = 0; x < NT; ++x) pw[x] = src[o++]; }
        if (ALG4) { _Pragma("unroll") for (int x = 0; x < NT; ++x) pend[x] = src[o++]; }
        if (SOLVE) { _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) u[r][d] = src[o++]; }
    }
    __device__ void zero() {
        _Pragma("unroll") for (int x = 0; x < NT; ++x) { pw[x] = T(0); pend[x] = T(0); sblk[x] = T(0); }
        _Pragma("unroll") for (int d = 0; d < L; ++d) srow[d] = T(0);
        _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) u[r][d] = T(0);
    }

    // Preload the ALG4 Sigma block and row for iteration i0 (direct loads, once per chain).
    __device__ void preload(const SweepArgs<T> &A, const ChainCtx &c, int64_t i0) {
        if (!ALG4) return;
        const T *S = A.S + c.band;
        _Pragma("unroll") for (int t = 1; t <= L; ++t)
            _Pragma("unroll") for (int q = t; q <= L; ++q) {
                int64_t col = i0 + t, row = i0 + q;
                sblk[tri(t - 1, q - 1, L)] = (row < c.n) ? S[(int64_t)(q - t) * c.ld + col * c.cs] : T(0);
            }
        _Pragma("unroll") for (int d = 0; d < L; ++d) srow[d] = (i0 + d < c.n) ? S[(int64_t)d * c.ld + i0 * c.cs] : T(0);
    }

    // One column / row step.  `out` selects whether outputs are written.
    template <bool CHECK, class IO>
    __device__ __forceinline__ void step(IO &io, const SweepArgs<T> &A, const ChainCtx &c, int64_t j, int tp, bool out,
                                         LogSum<T> &ld, int32_t &info) {
        const int64_t n = c.n;
        T Lc[L + 1];
        T rinv;
        if (CHOL) {
            T a[L + 1];
            _Pragma("unroll") for (int d = 0; d <= L; ++d) {
                T q = inb<CHECK>(j + d, n) ? io.in(d, j, tp) : T(0);
                a[d] = (d < L) ? (q - pw[tri(0, d, L)]) : q;
            }
            T piv = a[0];
            if (!(piv > T(0)) && out && info == 0) info = (int32_t)(j + 1);
            rinv = Num<T>::rsq(piv);
            Lc[0] = piv * rinv;
            _Pragma("unroll") for (int d = 1; d <= L; ++d) Lc[d] = a[d] * rinv;
            if (out) {
                _Pragma("unroll") for (int d = 0; d <= L; ++d) io.template out<CHECK>(d, j, tp, inb<CHECK>(j + d, n) ? Lc[d] : T(0));
                ld.add(piv);
            }
            // pending sums for the window of column j+1: pair (a', b') <- (a'+1, b'+1) + Lc[1+a'] Lc[1+b']
            T npw[NT];
            _Pragma("unroll") for (int x = 0; x < L; ++x)
                _Pragma("unroll") for (int y = x; y < L; ++y) {
                    T old = (y + 1 <= L - 1) ? pw[tri(x + 1, y + 1, L)] : T(0);
                    npw[tri(x, y, L)] = fma(Lc[1 + x], Lc[1 + y], old);
                }
            _Pragma("unroll") for (int x = 0; x < NT; ++x) pw[x] = npw[x];
        } else {
            _Pragma("unroll") for (int d = 0; d <= L; ++d) Lc[d] = inb<CHECK>(j + d, n) ? io.in(d, j, tp) : T(0);
            rinv = Num<T>::rcp(Lc[0]);
        }
        if (ALG4) {
            const int64_t i = j;
            T U[L + 1], sr[L + 1], b[L + 1], bU[L + 1];
            _Pragma("unroll") for (int t = 0; t <= L; ++t) {
                const bool in = inb<CHECK>(i + t, n);
                U[t] = Lc[t] * rinv;
                sr[t] = (t < L) ? srow[t] : (in ? io.in(I_SL, j, tp) : T(0));
                T sb = in ? io.in(I_SB + t, j, tp) : T(0);
                b[t] = (t < L ? pend[tri(0, t, L)] : T(0)) + sb;
                bU[t] = T(0);
            }
            // reverse of Sym[i,i] = rinv^2 - sum_t U[t] Sym[i, i+t]
            T bvi2 = b[0];
            _Pragma("unroll") for (int t = 1; t <= L; ++t) {
                bU[t] = -b[0] * sr[t];
                b[t] = fma(-b[0], U[t], b[t]);
            }
            // reverse of Sym[i, i+q] = -sum_t U[t] Sigma[i+t, i+q], q = 1..L
            T npend[NT];
            _Pragma("unroll") for (int x = 0; x < NT; ++x) npend[x] = T(0);
            _Pragma("unroll") for (int t = 1; t < L; ++t)
                _Pragma("unroll") for (int q = t; q < L; ++q) npend[tri(t - 1, q - 1, L)] = pend[tri(t, q, L)];
            _Pragma("unroll") for (int q = 1; q <= L; ++q) {
                _Pragma("unroll") for (int t = 1; t <= L; ++t) {
                    bU[t] = fma(-b[q], sblk[tri(t - 1, q - 1, L)], bU[t]);
                    npend[tri(t - 1, q - 1, L)] = fma(-b[q], U[t], npend[tri(t - 1, q - 1, L)]);
                }
            }
            _Pragma("unroll") for (int x = 0; x < NT; ++x) pend[x] = npend[x];
            if (out) {
                // bL = transpose(bU) / vec ; bvec = -2 bvi2 / vec^3 - sum_t bU[t] L[i+t, i] / vec^2
                T s = T(0);
                _Pragma("unroll") for (int t = 1; t <= L; ++t) s = fma(bU[t], Lc[t], s);
                T r2 = rinv * rinv;
                io.template out<CHECK>(0, j, tp, T(-2) * bvi2 * r2 * rinv - s * r2);
                _Pragma("unroll") for (int t = 1; t <= L; ++t) io.template out<CHECK>(t, j, tp, inb<CHECK>(i + t, n) ? bU[t] * rinv : T(0));
            }
            // the next row comes from the block; then shift the block to rows/cols i+2..i+L+1
            _Pragma("unroll") for (int d = 0; d < L; ++d) srow[d] = sblk[tri(0, d, L)];
            T nblk[NT];
            _Pragma("unroll") for (int t = 1; t < L; ++t)
                _Pragma("unroll") for (int q = t; q < L; ++q) nblk[tri(t - 1, q - 1, L)] = sblk[tri(t, q, L)];
            _Pragma("unroll") for (int t = 1; t <= L; ++t) {
                // new entry Sigma[i+1+t, i+1+L]: diagonal L-t at column i+1+t (stream I_SA + L - t)
                nblk[tri(t - 1, L - 1, L)] = inb<CHECK>(i + 1 + L, n) ? io.in(I_SA + L - t, j, tp) : T(0);
            }
            _Pragma("unroll") for (int x = 0; x < NT; ++x) sblk[x] = nblk[x];
        }
        if (SOLVE) {
            _Pragma("unroll") for (int r = 0; r < KK; ++r) {
                const bool on = r < A.kk;
                T y = ((on ? io.in(I_RHS + r, j, tp) : T(0)) - u[r][0]) * rinv;
                if (out) io.template out<CHECK>(O_RHS + r, j, tp, y);
                _Pragma("unroll") for (int d = 0; d < L; ++d) {
                    T old = (d + 1 < L) ? u[r][d + 1] : T(0);
                    u[r][d] = fma(Lc[1 + d], y, old);
                }
            }
        }
    }
};

// ===========================================================================
// Register-window backward sweep: TAKA [+ SOLVE], SOLVE, ALG2 [+ SOLVE + OUTER]
// Input streams:  [0, L]     L diagonal d at column j;  with ALG2: diagonal 0 at
//                            column j and diagonal e at column j-1-e (window)
//                 RHS block  Bin column r, row j                     (SOLVE)
//                 [LB, LB+L] Lbar_in diagonal d at column j          (ALG2)
//                 X block    Xin column r, row j                     (OUTER)
// Output streams: [0, L] S (TAKA) or Qbar (ALG2); then the RHS block (SOLVE)
// ===========================================================================
template <typename T, int L, int K, int FL>
struct BwdReg {
    static constexpr int NT = Tri<L>::N;
    static constexpr bool TAKA = (FL & B_TAKA) != 0;
    static constexpr bool SOLVE = (FL & B_SOLVE) != 0 && K > 0;
    static constexpr bool ALG2 = (FL & B_ALG2) != 0;
    static constexpr bool OUTER = (FL & B_OUTER) != 0 && SOLVE && ALG2;
    static constexpr int KK = (SOLVE ? K : 1);
    static constexpr int I_RHS = L + 1;
    static constexpr int I_LB = I_RHS + (SOLVE ? KK : 0);
    static constexpr int I_X = I_LB + (ALG2 ? L + 1 : 0);
    static constexpr int NIN = I_X + (OUTER ? KK : 0);
    static constexpr bool BAND_OUT = TAKA || ALG2;
    static constexpr int O_RHS = BAND_OUT ? L + 1 : 0;
    static constexpr int NOUT = O_RHS + (SOLVE ? KK : 0);
    __host__ __device__ static constexpr StreamSpec in_spec(int s) {
        if (s <= L) return StreamSpec{POOL_LIN, s, (ALG2 && s > 0) ? -(1 + s) : 0};
        if (SOLVE && s < I_LB) return StreamSpec{POOL_BIN, s - I_RHS, 0};
        if (ALG2 && s < I_X) return StreamSpec{POOL_LBARIN, s - I_LB, 0};
        return StreamSpec{POOL_XIN, s - I_X, 0};
    }
    __host__ __device__ static constexpr StreamSpec out_spec(int o) {
        if (BAND_OUT && o <= L) return StreamSpec{TAKA ? POOL_SOUT : POOL_QBAR, o, 0};
        return StreamSpec{POOL_XOUT, o - O_RHS, 0};
    }

    // computed state
    T sblk[NT];         // TAKA: Sigma block rows/cols i+1..i+L, pair (t-1, q-1)
    T pend[NT];         // ALG2: pending Lbar of entries (j+1+f, j-e), e in [0,L-1], f in [0, L-1-e]
    T xw[KK][L];        // SOLVE: x_{j+1..j+L}
    // input-derived state
    T lwin[NT];         // ALG2: L[j+f, j-e], e in [1,L], f in [0, L-e]  -> pair (e-1, e-1+f)
    T lcol[L + 1];      // ALG2: L[j+d, j], d >= 1, carried from the previous window
    T xin[KK][L];       // OUTER: forward X_{j+1..j+L}
    T two_ldbar;        // ALG2: 2 * log-det cotangent of the instance

    static constexpr int snap_words() { return (TAKA ? NT : 0) + (ALG2 ? NT : 0) + (SOLVE ? K * L : 0); }

    __device__ void save(T *dst) const {
        int o = 0;
        if (TAKA) { _Pragma("unroll") for (int x = 0; x < NT; ++x) dst[o++] = sblk[x]; }
        if (ALG2) { _Pragma("unroll") for (int x = 0; x < NT; ++x) dst[o++] = pend[x]; }
        if (SOLVE) { _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) dst[o++] = xw[r][d]; }
    }
    __device__ void load_state(const T *src) {
        int o = 0;
        if (TAKA) { _Pragma("unroll") for (int x = 0; x < NT; ++x) sblk[x] = src[o++]; }
        if (ALG2) { _Pragma("unroll") for (int x = 0; x < NT; ++x) pend[x] = src[o++]; }
        if (SOLVE) { _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) xw[r][d] = src[o++]; }
    }
    __device__ void zero() {
        _Pragma("unroll") for (int x = 0; x < NT; ++x) { sblk[x] = T(0); pend[x] = T(0); lwin[x] = T(0); }
        _Pragma("unroll") for (int d = 0; d <= L; ++d) lcol[d] = T(0);
        _Pragma("unroll") for (int r = 0; r < KK; ++r) _Pragma("unroll") for (int d = 0; d < L; ++d) { xw[r][d] = T(0); xin[r][d] = T(0); }
    }

    // Preload input-derived windows for the first iteration j0 (direct loads, once per chain).
    __device__ void preload(const SweepArgs<T> &A, const ChainCtx &c, int64_t j0) {
        two_ldbar = A.ldbar ? T(2.0 * A.ldbar[c.inst]) : T(0);
        if (ALG2) {
            const T *Li = A.Lin + c.band;
            _Pragma("unroll") for (int e = 1; e <= L; ++e)
                _Pragma("unroll") for (int f = 0; f <= L - e; ++f) {
                    int64_t col = j0 - e, row = j0 + f;
                    lwin[tri(e - 1, e - 1 + f, L)] = (col >= 0 && row < c.n) ? Li[(int64_t)(e + f) * c.ld + col * c.cs] : T(0);
                }
            _Pragma("unroll") for (int d = 1; d <= L; ++d) lcol[d] = (j0 + d < c.n) ? Li[(int64_t)d * c.ld + j0 * c.cs] : T(0);
        }
        if (OUTER) {
            const T *Xi = A.Xin + c.rhs;
            _Pragma("unroll") for (int r = 0; r < KK; ++r) {
                const bool on = r < A.kk;
                int64_t co = (int64_t)(A.rhs0 + (on ? r : 0)) * c.ldr;
                _Pragma("unroll") for (int d = 0; d < L; ++d) xin[r][d] = (on && j0 + 1 + d < c.n) ? Xi[co + (j0 + 1 + d) * c.cs] : T(0);
            }
        }
    }

    template <bool CHECK, class IO>
    __device__ __forceinline__ void step(IO &io, const SweepArgs<T> &A, const ChainCtx &c, int64_t j, int tp, bool out) {
        const int64_t n = c.n;
        T Lc[L + 1];
        if (ALG2) {
            Lc[0] = io.in(0, j, tp);
            _Pragma("unroll") for (int d = 1; d <= L; ++d) Lc[d] = lcol[d];
        } else {
            _Pragma("unroll") for (int d = 0; d <= L; ++d) Lc[d] = inb<CHECK>(j + d, n) ? io.in(d, j, tp) : T(0);
        }
        const T rinv = Num<T>::rcp(Lc[0]);
        T xj[KK];
        if (SOLVE) {
            _Pragma("unroll") for (int r = 0; r < KK; ++r) {
                const bool on = r < A.kk;
                T s = on ? io.in(I_RHS + r, j, tp) : T(0);
                _Pragma("unroll") for (int d = L; d >= 1; --d) s = fma(-Lc[d], xw[r][d - 1], s);
                xj[r] = s * rinv;
            }
        }
        if (TAKA) {
            const int64_t i = j;
            T U[L + 1], row[L + 1];
            _Pragma("unroll") for (int t = 1; t <= L; ++t) U[t] = Lc[t] * rinv;
            // Sym[i, i+q] = -sum_t U[t] Sigma[i+t, i+q], q = L..1 (freshest block term last)
            _Pragma("unroll") for (int q = L; q >= 1; --q) {
                T s = T(0);
                _Pragma("unroll") for (int t = L; t >= 1; --t) s = fma(U[t], sblk[tri(t - 1, q - 1, L)], s);
                row[q] = -s;
            }
            {
                T s = T(0);
                _Pragma("unroll") for (int t = L; t >= 1; --t) s = fma(U[t], row[t], s);
                row[0] = rinv * rinv - s;
            }
            if (out) { _Pragma("unroll") for (int q = 0; q <= L; ++q) io.template out<CHECK>(q, j, tp, inb<CHECK>(i + q, n) ? row[q] : T(0)); }
            // shift: new block rows/cols i..i+L-1 : (0, q) <- row[q]; (t, q) <- old (t-1, q-1)
            T nblk[NT];
            _Pragma("unroll") for (int q = 0; q < L; ++q) nblk[tri(0, q, L)] = inb<CHECK>(i + q, n) ? row[q] : T(0);
            _Pragma("unroll") for (int t = 1; t < L; ++t)
                _Pragma("unroll") for (int q = t; q < L; ++q) nblk[tri(t, q, L)] = sblk[tri(t - 1, q - 1, L)];
            _Pragma("unroll") for (int x = 0; x < NT; ++x) sblk[x] = nblk[x];
        }
        if (ALG2) {
            T Lb[L + 1];
            _Pragma("unroll") for (int d = 0; d <= L; ++d) {
                T v = inb<CHECK>(j + d, n) ? io.in(I_LB + d, j, tp) : T(0);
                Lb[d] = (d >= 1) ? (v + pend[tri(0, d - 1, L)]) : v;
            }
            if (OUTER) {
                // Lbar -= band(X Ybar^T) + band(Bbar Y^T) with Y = L^T X, Bbar = L^{-T} Ybar
                _Pragma("unroll") for (int r = 0; r < KK; ++r) {
                    const bool on = r < A.kk;
                    T x0 = on ? io.in(I_X + r, j, tp) : T(0);
                    T ybar = on ? io.in(I_RHS + r, j, tp) : T(0);
                    T y = Lc[0] * x0;
                    _Pragma("unroll") for (int d = 1; d <= L; ++d) y = fma(Lc[d], xin[r][d - 1], y);
                    Lb[0] = fma(-x0, ybar, Lb[0]);
                    Lb[0] = fma(-xj[r], y, Lb[0]);
                    _Pragma("unroll") for (int d = 1; d <= L; ++d) {
                        Lb[d] = fma(-xin[r][d - 1], ybar, Lb[d]);
                        Lb[d] = fma(-xw[r][d - 1], y, Lb[d]);
                    }
                    _Pragma("unroll") for (int d = L - 1; d >= 1; --d) xin[r][d] = xin[r][d - 1];
                    xin[r][0] = x0;
                }
            }
            Lb[0] = fma(two_ldbar, rinv, Lb[0]);
            // Alg. 2 for column j: off-diagonals first, then the diagonal
            T Qb[L + 1];
            _Pragma("unroll") for (int d = 1; d <= L; ++d) {
                Qb[d] = Lb[d] * rinv;
                Lb[0] = fma(-Qb[d], Lc[d], Lb[0]);
            }
            Qb[0] = T(0.5) * Lb[0] * rinv;
            if (out) { _Pragma("unroll") for (int d = 0; d <= L; ++d) io.template out<CHECK>(d, j, tp, inb<CHECK>(j + d, n) ? Qb[d] : T(0)); }
            // new pending for iteration j-1 (entries (j+f', j-1-e')): carry old (e, f), e >= 1 -> (e-1, f+1)
            T np[NT];
            _Pragma("unroll") for (int e2 = 0; e2 < L; ++e2)
                _Pragma("unroll") for (int f2 = 0; f2 <= L - 1 - e2; ++f2) {
                    T old = (f2 >= 1 && e2 + 1 <= L - 1) ? pend[tri(e2 + 1, e2 + 1 + (f2 - 1), L)] : T(0);
                    np[tri(e2, e2 + f2, L)] = old;
                }
            // contributions of column j: L[j+d, m] gets -Qb[d] L[j, m], L[j, m] gets -Qb[d] L[j+d, m]
            // (d = 0: -2 Qb[0] L[j, m]) for m in [j+d-L, j-1].  m = j-1-e2, L[j+f, m] = lwin(e=e2+1, f).
            _Pragma("unroll") for (int e2 = 0; e2 < L; ++e2) {
                const int e = e2 + 1;
                T ljm = lwin[tri(e - 1, e - 1, L)];
                np[tri(e2, e2, L)] = fma(T(-2) * Qb[0], ljm, np[tri(e2, e2, L)]);
                _Pragma("unroll") for (int d = 1; d <= L - e; ++d) {
                    T ljdm = lwin[tri(e - 1, e - 1 + d, L)];
                    np[tri(e2, e2 + d, L)] = fma(-Qb[d], ljm, np[tri(e2, e2 + d, L)]);
                    np[tri(e2, e2, L)] = fma(-Qb[d], ljdm, np[tri(e2, e2, L)]);
                }
            }
            _Pragma("unroll") for (int x = 0; x < NT; ++x) pend[x] = np[x];
            // column j-1 of L (below the diagonal) is window column e = 1; then shift the window:
            // (e, f) -> (e-1, f+1) for e >= 2, new f = 0 entries L[j-1, j-1-e] (stream e)
            _Pragma("unroll") for (int d = 1; d <= L; ++d) lcol[d] = lwin[tri(0, d - 1, L)];
            T nw[NT];
            _Pragma("unroll") for (int e = 1; e <= L; ++e)
                _Pragma("unroll") for (int f = 0; f <= L - e; ++f) {
                    T v;
                    if (f >= 1) v = lwin[tri(e, e + f - 1, L)];
                    else v = io.in(e, j, tp);      // L[j-1, j-1-e] (zero when the column is < 0)
                    nw[tri(e - 1, e - 1 + f, L)] = v;
                }
            _Pragma("unroll") for (int x = 0; x < NT; ++x) lwin[x] = nw[x];
        }
        if (SOLVE) {
            if (out) { _Pragma("unroll") for (int r = 0; r < KK; ++r) io.template out<CHECK>(O_RHS + r, j, tp, xj[r]); }
            _Pragma("unroll") for (int r = 0; r < KK; ++r) {
                _Pragma("unroll") for (int d = L - 1; d >= 1; --d) xw[r][d] = xw[r][d - 1];
                xw[r][0] = xj[r];
            }
        }
    }
};


// ===========================================================================
// Chain drivers (register windows, any IO)
// ===========================================================================
template <typename T>
__device__ __forceinline__ ChainPtrs<T> chain_ptrs(const SweepArgs<T> &A, const ChainCtx &c) {
    ChainPtrs<T> P;
    P.in[POOL_Q] = A.Q ? A.Q + c.band : nullptr;
    P.in[POOL_LIN] = A.Lin ? A.Lin + c.band : nullptr;
    P.in[POOL_S] = A.S ? A.S + c.band : nullptr;
    P.in[POOL_SBAR] = A.Sbar ? A.Sbar + c.band : nullptr;
    P.in[POOL_LBARIN] = A.Lbar_in ? A.Lbar_in + c.band : nullptr;
    P.in[POOL_BIN] = A.Bin ? A.Bin + c.rhs : nullptr;
    P.in[POOL_XIN] = A.Xin ? A.Xin + c.rhs : nullptr;
    P.out[POOL_LOUT - POOL_LOUT] = A.L ? A.L + c.band : nullptr;
    P.out[POOL_LBAR - POOL_LOUT] = A.Lbar ? A.Lbar + c.band : nullptr;
    P.out[POOL_SOUT - POOL_LOUT] = A.Sout ? A.Sout + c.band : nullptr;
    P.out[POOL_QBAR - POOL_LOUT] = A.Qbar ? A.Qbar + c.band : nullptr;
    P.out[POOL_XOUT - POOL_LOUT] = A.Xout ? A.Xout + c.rhs : nullptr;
    P.ld = c.ld; P.ldr = c.ldr; P.cs = c.cs; P.n = c.n; P.rhs0 = A.rhs0; P.acc = A.acc; P.kk = A.kk;
    return P;
}

template <typename T, int L, int K, int FL, class IO>
__device__ void run_fwd_reg(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, int mode,
                            const T *exact_state, IO &io) {
    using SW = FwdReg<T, L, K, FL>;
    constexpr int TW = IO::TW;
    SW s;
    s.zero();
    int64_t j0 = c.a;
    if (mode == RUN_COLD && !c.first) j0 = imax64(c.a - c.warm, 0);
    if (mode == RUN_EXACT && exact_state) s.load_state(exact_state);
    if (c.inst >= 0) s.preload(A, c, j0);
    const int64_t jend = c.b - 1;
    const int64_t m0 = floordiv(j0, TW), m1 = floordiv(jend, TW);
    int64_t w0 = m0, w1 = m1;
    if constexpr (IO::kWarpUniform) {
        // cooperative copies: the warp walks the union of its lanes' tiles
        w0 = warp_min64(c.inst >= 0 ? m0 : INT64_MAX);
        w1 = warp_max64(c.inst >= 0 ? m1 : INT64_MIN);
    }
    io.begin_tiles(w0, c.a, c.b);
    LogSum<T> ld;
    int32_t info = 0;
    for (int64_t m = w0; m <= w1; ++m) {
        io.tile_begin(m);
        const int64_t jt = m * TW;
        if (jt == c.a && !c.first) s.save(snap_ptr<T>(P, c.gseg, 0));
        const bool has_out = jt >= c.a;
        // interior tile: every column of the tile and every streamed column (offsets <= L + 1) is inside the matrix
        const bool interior = jt >= j0 && jt + TW - 1 <= jend && jt + TW + 2 * L + 1 < c.n;
        if (interior) {
            if constexpr (L <= BND_INTERIOR_UNROLL_MAX_L) {
#pragma unroll
                for (int u = 0; u < TW; ++u) s.template step<false>(io, A, c, jt + u, u, has_out, ld, info);
            } else {
#pragma unroll 1
                for (int u = 0; u < TW; ++u) s.template step<false>(io, A, c, jt + u, u, has_out, ld, info);
            }
        } else {
            for (int u = 0; u < TW; ++u) {
                const int64_t j = jt + u;
                if (j < j0 || j > jend) continue;
                s.template step<true>(io, A, c, j, u, has_out, ld, info);
            }
        }
        io.tile_end(m, has_out);
    }
    io.finish();
    if (c.inst < 0) return;
    if (!c.last) s.save(snap_ptr<T>(P, c.gseg, 1));
    const double ldacc = ld.value();
    if (FL & F_CHOL) {
        if (c.first && c.last) {
            if (A.logdet) A.logdet[c.inst] = info ? (double)NAN : ldacc;
            A.info[c.inst] = info;
        } else {
            P.seg_logdet[c.gseg] = ldacc;
            P.seg_info[c.gseg] = info;
        }
    }
}

template <typename T, int L, int K, int FL, class IO>
__device__ void run_bwd_reg(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, int mode,
                            const T *exact_state, IO &io) {
    using SW = BwdReg<T, L, K, FL>;
    constexpr int TW = IO::TW;
    SW s;
    s.zero();
    int64_t j0 = c.b - 1;
    if (mode == RUN_COLD && !c.last) j0 = imin64(c.b - 1 + c.warm, c.n - 1);
    if (mode == RUN_EXACT && exact_state) s.load_state(exact_state);
    if (c.inst >= 0) s.preload(A, c, j0);
    const int64_t m0 = floordiv(j0, TW), m1 = floordiv(c.a, TW);
    int64_t w0 = m0, w1 = m1;
    if constexpr (IO::kWarpUniform) {
        w0 = warp_max64(c.inst >= 0 ? m0 : INT64_MIN);
        w1 = warp_min64(c.inst >= 0 ? m1 : INT64_MAX);
    }
    io.begin_tiles(w0, c.a, c.b);
    for (int64_t m = w0; m >= w1; --m) {
        io.tile_begin(m);
        const int64_t jt = m * TW;
        if (jt + TW - 1 == c.b - 1 && !c.last) s.save(snap_ptr<T>(P, c.gseg, 0));
        const bool has_out = jt < c.b;
        // interior tile: all its columns inside [a, j0], rows below n, window columns >= 0
        const bool interior = jt >= c.a && jt + TW - 1 <= j0 && jt + TW + L < c.n && jt - 1 - L >= 0;
        if (interior) {
            if constexpr (L <= BND_INTERIOR_UNROLL_MAX_L) {
#pragma unroll
                for (int u = TW - 1; u >= 0; --u) s.template step<false>(io, A, c, jt + u, u, has_out);
            } else {
#pragma unroll 1
                for (int u = TW - 1; u >= 0; --u) s.template step<false>(io, A, c, jt + u, u, has_out);
            }
        } else {
            for (int u = TW - 1; u >= 0; --u) {
                const int64_t j = jt + u;
                if (j < c.a || j > j0) continue;
                s.template step<true>(io, A, c, j, u, has_out);
            }
        }
        io.tile_end(m, has_out);
    }
    io.finish();
    if (c.inst >= 0 && !c.first) s.save(snap_ptr<T>(P, c.gseg, 1));
}

// ===========================================================================
// Generic forms for any bandwidth: one chain per instance, the windows live in
// the outputs themselves and in two band-shaped scratch pools (zeroed before
// the launch).  Same formulas as the register forms.
// ===========================================================================
template <typename T, int FL>
__device__ void run_fwd_generic(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c) {
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    const int l = c.l;
    constexpr bool CHOL = (FL & F_CHOL) != 0, ALG4 = (FL & F_ALG4) != 0;
    const bool SOLVE = (FL & F_SOLVE) != 0 && P.k > 0;
    const int K = SOLVE ? A.kk : 0;
    double ldacc = 0.0;
    int32_t info = 0;
    T *Lw = CHOL ? A.L + c.band : nullptr;
    const T *Lr = CHOL ? (const T *)(A.L + c.band) : A.Lin + c.band;
#define LL(i_, j_) Lr[(int64_t)((i_) - (j_)) * ld + (j_) * cs]
    for (int64_t j = 0; j < n; ++j) {
        const int dmax = (int)imin64(l, n - 1 - j);
        T rinv;
        if (CHOL) {
            const T *Q = A.Q + c.band;
            T s = T(0);
            for (int64_t m = imax64(j - l, 0); m < j; ++m) s = fma(LL(j, m), LL(j, m), s);
            T piv = Q[j * cs] - s;
            if (!(piv > T(0)) && info == 0) info = (int32_t)(j + 1);
            T ljj = Num<T>::sqrt_(piv);
            rinv = T(1) / ljj;
            ldacc += log((double)piv);
            for (int d = 1; d <= dmax; ++d) {
                T t = T(0);
                for (int64_t m = imax64(j + d - l, 0); m < j; ++m) t = fma(LL(j + d, m), LL(j, m), t);
                Lw[(int64_t)d * ld + (j) * cs] = (Q[(int64_t)d * ld + (j) * cs] - t) * rinv;
            }
            Lw[j * cs] = ljj;
            for (int d = dmax + 1; d <= l; ++d) Lw[(int64_t)d * ld + (j) * cs] = T(0);
        } else {
            rinv = T(1) / Lr[j * cs];
        }
        if (SOLVE) {
            const T *Bi = A.Bin + c.rhs;
            T *Xo = A.Xout + c.rhs;
            for (int r = 0; r < K; ++r) {
                int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                T s = Bi[co + (j) * cs];
                for (int64_t m = imax64(j - l, 0); m < j; ++m) s = fma(-LL(j, m), Xo[co + (m) * cs], s);
                Xo[co + (j) * cs] = s * rinv;
            }
        }
        if (ALG4) {
            // scratch : pair adjoint of the pair (i, i+q) at [q][i]
            // scratch2: bU[i, i+t] at [t][i]
            const T *S = A.S + c.band;
            const T *Sb = A.Sbar + c.band;
            T *Pp = A.scratch + c.band;
            T *bU = A.scratch2 + c.band;
            T *Lb = A.Lbar + c.band;
            const int64_t i = j;
#define SYM(a_, b_) (((a_) >= (b_)) ? S[(int64_t)((a_) - (b_)) * ld + (b_) * cs] : S[(int64_t)((b_) - (a_)) * ld + (a_) * cs])
#define PAIR(a_, b_) (((a_) >= (b_)) ? Pp[(int64_t)((a_) - (b_)) * ld + (b_) * cs] : Pp[(int64_t)((b_) - (a_)) * ld + (a_) * cs])
            for (int q = 0; q <= dmax; ++q) Pp[(int64_t)q * ld + (i) * cs] += Sb[(int64_t)q * ld + (i) * cs];
            const T b0 = Pp[i * cs];
            for (int t = 1; t <= dmax; ++t) {
                T Ut = LL(i + t, i) * rinv;
                bU[(int64_t)t * ld + (i) * cs] = -b0 * SYM(i, i + t);
                Pp[(int64_t)t * ld + (i) * cs] = fma(-b0, Ut, Pp[(int64_t)t * ld + (i) * cs]);
            }
            for (int q = 1; q <= dmax; ++q) {
                const T bq = Pp[(int64_t)q * ld + (i) * cs];
                for (int t = 1; t <= dmax; ++t) {
                    T Ut = LL(i + t, i) * rinv;
                    bU[(int64_t)t * ld + (i) * cs] = fma(-bq, SYM(i + t, i + q), bU[(int64_t)t * ld + (i) * cs]);
                    T &pr = PAIR(i + t, i + q);
                    pr = fma(-bq, Ut, pr);
                }
            }
            T s = T(0);
            for (int t = 1; t <= dmax; ++t) s = fma(bU[(int64_t)t * ld + (i) * cs], LL(i + t, i), s);
            const T r2 = rinv * rinv;
            const T bvec = T(-2) * b0 * r2 * rinv - s * r2;
            for (int t = 0; t <= l; ++t) {
                T v = (t == 0) ? bvec : (t <= dmax ? bU[(int64_t)t * ld + (i) * cs] * rinv : T(0));
                T *p = &Lb[(int64_t)t * ld + (i) * cs];
                *p = (t <= dmax) ? (A.acc ? (*p + v) : v) : T(0);                  // corners: 0
            }
#undef SYM
#undef PAIR
        }
    }
#undef LL
    if (CHOL) {
        if (A.logdet) A.logdet[c.inst] = info ? (double)NAN : ldacc;
        A.info[c.inst] = info;
    }
}

template <typename T, int FL>
__device__ void run_bwd_generic(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c) {
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    const int l = c.l;
    constexpr bool TAKA = (FL & B_TAKA) != 0, ALG2 = (FL & B_ALG2) != 0;
    const bool SOLVE = (FL & B_SOLVE) != 0 && P.k > 0;
    const bool OUTER = (FL & B_OUTER) != 0 && SOLVE && ALG2;
    const int K = SOLVE ? A.kk : 0;
    const T *Lr = A.Lin + c.band;
#define LL(i_, j_) Lr[(int64_t)((i_) - (j_)) * ld + (j_) * cs]
    for (int64_t j = n - 1; j >= 0; --j) {
        const int dmax = (int)imin64(l, n - 1 - j);
        const T rinv = T(1) / Lr[j * cs];
        if (SOLVE) {
            const T *Bi = A.Bin + c.rhs;
            T *Xo = A.Xout + c.rhs;
            for (int r = 0; r < K; ++r) {
                int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                T s = Bi[co + (j) * cs];
                for (int d = dmax; d >= 1; --d) s = fma(-LL(j + d, j), Xo[co + (j + d) * cs], s);
                Xo[co + (j) * cs] = s * rinv;
            }
        }
        if (TAKA) {
            T *So = A.Sout + c.band;
            const int64_t i = j;
#define SIG(a_, b_) (((a_) >= (b_)) ? So[(int64_t)((a_) - (b_)) * ld + (b_) * cs] : So[(int64_t)((b_) - (a_)) * ld + (a_) * cs])
            for (int q = dmax; q >= 1; --q) {
                T s = T(0);
                for (int t = dmax; t >= 1; --t) s = fma(LL(i + t, i) * rinv, SIG(i + t, i + q), s);
                So[(int64_t)q * ld + (i) * cs] = -s;
            }
            T s = T(0);
            for (int t = dmax; t >= 1; --t) s = fma(LL(i + t, i) * rinv, So[(int64_t)t * ld + (i) * cs], s);
            So[i * cs] = rinv * rinv - s;
            for (int q = dmax + 1; q <= l; ++q) So[(int64_t)q * ld + (i) * cs] = T(0);
#undef SIG
        }
        if (ALG2) {
            // scratch : pending Lbar of entry (r, m) at [r-m][m]
            // scratch2: Lbar (then Qbar) of column j
            T *Pp = A.scratch + c.band;
            T *W = A.scratch2 + c.band;
            const T *Lbi = A.Lbar_in + c.band;
            T *Qo = A.Qbar + c.band;
            for (int d = 0; d <= dmax; ++d) W[(int64_t)d * ld + (j) * cs] = Lbi[(int64_t)d * ld + (j) * cs] + (d >= 1 ? Pp[(int64_t)d * ld + (j) * cs] : T(0));
            if (OUTER) {
                const T *Yb = A.Ybar + c.rhs;
                const T *Xi = A.Xin + c.rhs;
                const T *Bb = A.Xout + c.rhs;
                for (int r = 0; r < K; ++r) {
                    int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                    T y = T(0);
                    for (int d = 0; d <= dmax; ++d) y = fma(LL(j + d, j), Xi[co + (j + d) * cs], y);
                    const T ybar = Yb[co + (j) * cs];
                    for (int d = 0; d <= dmax; ++d) {
                        T v = W[(int64_t)d * ld + (j) * cs];
                        v = fma(-Xi[co + (j + d) * cs], ybar, v);
                        v = fma(-Bb[co + (j + d) * cs], y, v);
                        W[(int64_t)d * ld + (j) * cs] = v;
                    }
                }
            }
            if (A.ldbar) W[j * cs] = W[j * cs] + T(2.0 * A.ldbar[c.inst]) * rinv;
            T lb0 = W[j * cs];
            for (int d = 1; d <= dmax; ++d) {
                T qb = W[(int64_t)d * ld + (j) * cs] * rinv;
                W[(int64_t)d * ld + (j) * cs] = qb;
                lb0 = fma(-qb, LL(j + d, j), lb0);
            }
            W[j * cs] = T(0.5) * lb0 * rinv;
            for (int d = 0; d <= l; ++d) {
                T *p = &Qo[(int64_t)d * ld + (j) * cs];
                *p = (d <= dmax) ? (A.acc ? (*p + W[(int64_t)d * ld + (j) * cs]) : W[(int64_t)d * ld + (j) * cs]) : T(0);
            }
            for (int d = 0; d <= dmax; ++d) {
                const T qb = W[(int64_t)d * ld + (j) * cs];
                for (int64_t m = imax64(j + d - l, 0); m < j; ++m) {
                    if (d == 0) {
                        Pp[(int64_t)(j - m) * ld + (m) * cs] = fma(T(-2) * qb, LL(j, m), Pp[(int64_t)(j - m) * ld + (m) * cs]);
                    } else {
                        Pp[(int64_t)(j + d - m) * ld + (m) * cs] = fma(-qb, LL(j, m), Pp[(int64_t)(j + d - m) * ld + (m) * cs]);
                        Pp[(int64_t)(j - m) * ld + (m) * cs] = fma(-qb, LL(j + d, m), Pp[(int64_t)(j - m) * ld + (m) * cs]);
                    }
                }
            }
        }
    }
#undef LL
}

}  // namespace bnd
