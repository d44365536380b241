// Warp-cooperative sweeps for wide bands (bandwidths above the register-window
// limit): one warp per instance.  The windows live in memory exactly as in the
// generic forms (the outputs themselves and two band-shaped scratch pools,
// zeroed before the launch), with the same formulas; every inner loop over
// the diagonals or the window columns of a row is split across the 32 lanes,
// sums over a lane-split index are reduced with shuffles, and a warp barrier
// closes each phase whose results other lanes read.  Additions the generic
// forms make in one sequence are here summed per lane, then across lanes:
// the rounding differs, the values do not.
//
// Ownership that keeps the lanes' writes disjoint:
//   Alg. 1 column j      lane d writes L[j+d, j]
//   Alg. 4 row i         lane t owns bU[i, i+t] and the pair adjoints
//                        (i+t, i+q) with q >= t (both orders of the pair)
//   Alg. 2 column j      lane d owns Lbar[j+d, j]; lane m owns every pending
//                        entry of column m (rows j .. j+l)
//   Alg. 3 row i         lane q writes Sigma[i, i+q]
#pragma once

#include "sweep_impl.cuh"

namespace bnd {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int FL>
__device__ void run_fwd_wide(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, int lane) {
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
#define AT(p_, d_, j_) p_[(int64_t)(d_) * ld + (j_) * cs]
    for (int64_t j = 0; j < n; ++j) {
        const int dmax = (int)imin64(l, n - 1 - j);
        const int64_t m0 = imax64(j - l, 0);
        T rinv;
        if (CHOL) {
            const T *Q = A.Q + c.band;
            T s = T(0);
            for (int64_t m = m0 + lane; m < j; m += kWarp) s = fma(LL(j, m), LL(j, m), s);
            s = warp_sum(s);
            const T piv = Q[j * cs] - s;
            if (!(piv > T(0)) && info == 0) info = (int32_t)(j + 1);
            const T ljj = Num<T>::sqrt_(piv);
            rinv = T(1) / ljj;
            if (lane == 0) ldacc += log((double)piv);
            for (int d = 1 + lane; d <= dmax; d += kWarp) {
                T t = T(0);
                for (int64_t m = imax64(j + d - l, 0); m < j; ++m) t = fma(LL(j + d, m), LL(j, m), t);
                AT(Lw, d, j) = (AT(Q, d, j) - t) * rinv;
            }
            if (lane == 0) Lw[j * cs] = ljj;
            for (int d = dmax + 1 + lane; d <= l; d += kWarp) AT(Lw, d, j) = T(0);
            __syncwarp();
        } else {
            rinv = T(1) / Lr[j * cs];
        }
        if (SOLVE) {
            const T *Bi = A.Bin + c.rhs;
            T *Xo = A.Xout + c.rhs;
            for (int r = 0; r < K; ++r) {
                const int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                T s = T(0);
                for (int64_t m = m0 + lane; m < j; m += kWarp) s = fma(LL(j, m), Xo[co + m * cs], s);
                s = warp_sum(s);
                if (lane == 0) Xo[co + j * cs] = (Bi[co + j * cs] - s) * rinv;
            }
            __syncwarp();
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
            for (int q = lane; q <= dmax; q += kWarp) AT(Pp, q, i) += AT(Sb, q, i);
            __syncwarp();
            const T b0 = Pp[i * cs];
            for (int t = 1 + lane; t <= dmax; t += kWarp) {
                const T Ut = LL(i + t, i) * rinv;
                AT(bU, t, i) = -b0 * SYM(i, i + t);
                AT(Pp, t, i) = fma(-b0, Ut, AT(Pp, t, i));
            }
            __syncwarp();
            T s = T(0);
            for (int t = 1 + lane; t <= dmax; t += kWarp) {
                const T Ut = LL(i + t, i) * rinv;
                const T bt = AT(Pp, t, i);
                T acc = AT(bU, t, i);
                for (int q = 1; q <= dmax; ++q) acc = fma(-AT(Pp, q, i), SYM(i + t, i + q), acc);
                AT(bU, t, i) = acc;
                for (int q = t; q <= dmax; ++q) {
                    T &pr = PAIR(i + t, i + q);
                    pr = fma(-AT(Pp, q, i), Ut, pr);
                    if (q != t) pr = fma(-bt, LL(i + q, i) * rinv, pr);
                }
                s = fma(acc, LL(i + t, i), s);
            }
            s = warp_sum(s);
            __syncwarp();                      // bU[i, i+t] was written by the lane that owns t
            const T r2 = rinv * rinv;
            const T bvec = T(-2) * b0 * r2 * rinv - s * r2;
            for (int t = lane; t <= l; t += kWarp) {
                const T v = (t == 0) ? bvec : (t <= dmax ? AT(bU, t, i) * rinv : T(0));
                T *p = &AT(Lb, t, i);
                *p = (t <= dmax) ? (A.acc ? (*p + v) : v) : T(0);                  // corners: 0
            }
            __syncwarp();
#undef SYM
#undef PAIR
        }
    }
#undef AT
#undef LL
    if (CHOL && lane == 0) {
        if (A.logdet) A.logdet[c.inst] = info ? (double)NAN : ldacc;
        A.info[c.inst] = info;
    }
}

template <typename T, int FL>
__device__ void run_bwd_wide(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, int lane) {
    const int64_t n = c.n, ld = c.ld, cs = c.cs;
    const int l = c.l;
    constexpr bool TAKA = (FL & B_TAKA) != 0, ALG2 = (FL & B_ALG2) != 0;
    const bool SOLVE = (FL & B_SOLVE) != 0 && P.k > 0;
    const bool OUTER = (FL & B_OUTER) != 0 && SOLVE && ALG2;
    const int K = SOLVE ? A.kk : 0;
    const T *Lr = A.Lin + c.band;
#define LL(i_, j_) Lr[(int64_t)((i_) - (j_)) * ld + (j_) * cs]
#define AT(p_, d_, j_) p_[(int64_t)(d_) * ld + (j_) * cs]
    for (int64_t j = n - 1; j >= 0; --j) {
        const int dmax = (int)imin64(l, n - 1 - j);
        const T rinv = T(1) / Lr[j * cs];
        if (SOLVE) {
            const T *Bi = A.Bin + c.rhs;
            T *Xo = A.Xout + c.rhs;
            for (int r = 0; r < K; ++r) {
                const int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                T s = T(0);
                for (int d = 1 + lane; d <= dmax; d += kWarp) s = fma(LL(j + d, j), Xo[co + (j + d) * cs], s);
                s = warp_sum(s);
                if (lane == 0) Xo[co + j * cs] = (Bi[co + j * cs] - s) * rinv;
            }
            __syncwarp();
        }
        if (TAKA) {
            T *So = A.Sout + c.band;
            const int64_t i = j;
#define SIG(a_, b_) (((a_) >= (b_)) ? So[(int64_t)((a_) - (b_)) * ld + (b_) * cs] : So[(int64_t)((b_) - (a_)) * ld + (a_) * cs])
            for (int q = 1 + lane; q <= dmax; q += kWarp) {
                T s = T(0);
                for (int t = dmax; t >= 1; --t) s = fma(LL(i + t, i) * rinv, SIG(i + t, i + q), s);
                AT(So, q, i) = -s;
            }
            __syncwarp();
            T s = T(0);
            for (int t = 1 + lane; t <= dmax; t += kWarp) s = fma(LL(i + t, i) * rinv, AT(So, t, i), s);
            s = warp_sum(s);
            if (lane == 0) So[i * cs] = rinv * rinv - s;
            for (int q = dmax + 1 + lane; q <= l; q += kWarp) AT(So, q, i) = T(0);
            __syncwarp();
#undef SIG
        }
        if (ALG2) {
            // scratch : pending Lbar of entry (r, m) at [r-m][m]
            // scratch2: Lbar (then Qbar) of column j
            T *Pp = A.scratch + c.band;
            T *W = A.scratch2 + c.band;
            const T *Lbi = A.Lbar_in + c.band;
            T *Qo = A.Qbar + c.band;
            for (int d = lane; d <= dmax; d += kWarp)
                AT(W, d, j) = AT(Lbi, d, j) + (d >= 1 ? AT(Pp, d, j) : T(0));
            if (OUTER) {
                const T *Yb = A.Ybar + c.rhs;
                const T *Xi = A.Xin + c.rhs;
                const T *Bb = A.Xout + c.rhs;
                for (int r = 0; r < K; ++r) {
                    const int64_t co = (int64_t)(A.rhs0 + r) * c.ldr;
                    T y = T(0);
                    for (int d = lane; d <= dmax; d += kWarp) y = fma(LL(j + d, j), Xi[co + (j + d) * cs], y);
                    y = warp_sum(y);
                    const T ybar = Yb[co + j * cs];
                    for (int d = lane; d <= dmax; d += kWarp) {
                        T v = AT(W, d, j);
                        v = fma(-Xi[co + (j + d) * cs], ybar, v);
                        v = fma(-Bb[co + (j + d) * cs], y, v);
                        AT(W, d, j) = v;
                    }
                }
            }
            // Alg. 2 for column j: off-diagonals first, then the diagonal
            T part = T(0);
            for (int d = lane; d <= dmax; d += kWarp) {         // same owner of W[d, j] as above
                if (d == 0) continue;
                const T qb = AT(W, d, j) * rinv;
                AT(W, d, j) = qb;
                part = fma(-qb, LL(j + d, j), part);
            }
            part = warp_sum(part);
            if (lane == 0) {
                T w0 = W[j * cs];
                if (A.ldbar) w0 = w0 + T(2.0 * A.ldbar[c.inst]) * rinv;
                W[j * cs] = T(0.5) * (w0 + part) * rinv;
            }
            __syncwarp();
            for (int d = lane; d <= l; d += kWarp) {
                T *p = &AT(Qo, d, j);
                *p = (d <= dmax) ? (A.acc ? (*p + AT(W, d, j)) : AT(W, d, j)) : T(0);
            }
            // pending entries of the window columns m in [j - l, j): lane m owns column m
            for (int64_t m = imax64(j - l, 0) + lane; m < j; m += kWarp) {
                const T ljm = LL(j, m);
                T pjm = AT(Pp, j - m, m);
                pjm = fma(T(-2) * W[j * cs], ljm, pjm);
                for (int d = 1; d <= dmax && j + d - m <= l; ++d) {
                    const T qb = AT(W, d, j);
                    AT(Pp, j + d - m, m) = fma(-qb, ljm, AT(Pp, j + d - m, m));
                    pjm = fma(-qb, LL(j + d, m), pjm);
                }
                AT(Pp, j - m, m) = pjm;
            }
            __syncwarp();
        }
    }
#undef AT
#undef LL
}

}  // namespace bnd
