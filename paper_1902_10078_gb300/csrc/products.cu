// Products P and O (Sec. 4.1): band x band projected onto a target band,
// band x vectors, and the band-projected outer product.  Every output column
// is independent, so these are one-thread-per-column kernels over a flat list
// of tiles (binary searched): 256 columns of an instance in rows plans, 8
// columns of a 32-lane group in panel plans (coalesced across the lanes).
#include "common.cuh"
#include "products.cuh"

namespace bnd {

// Element (i, j) of op(M) for a general band (lo, up) stored with
// M[i, j] = M'[up + i - j][j]; zero outside the band or the matrix.
template <typename T>
__device__ __forceinline__ T band_get(const T *M, int64_t ld, int64_t cs, int lo, int up, bool trans, int64_t n,
                                      int64_t i, int64_t j) {
    if (trans) { int64_t t = i; i = j; j = t; }
    if (i < 0 || j < 0 || i >= n || j >= n) return T(0);
    const int64_t dd = i - j;
    if (dd > lo || -dd > up) return T(0);
    return M[(int64_t)(up + dd) * ld + j * cs];
}

__device__ __forceinline__ int find_tile_owner(const int64_t *prefix, int count, int64_t tile) {
    int lo = 0, hi = count;               // prefix[lo] <= tile < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

// Instance and column of this thread: rows plans give each block 256 columns
// of one instance; panel plans give it 8 columns of the 32 lanes of one
// group (thread t: lane t % 32, column t / 32), so each warp reads and writes
// 32 adjacent elements.  False if the thread has no element.
__device__ __forceinline__ bool locate(const PlanDev &P, int &inst, int64_t &j) {
    const int64_t tile = blockIdx.x;
    if (tile >= P.ntiles) return false;
    if (P.ngroups > 0) {
        const int g = find_tile_owner(P.tile_prefix, P.ngroups, tile);
        inst = P.group_first[g] + (int)(threadIdx.x % kWarp);
        if (inst >= P.group_first[g + 1]) return false;
        j = (tile - P.tile_prefix[g]) * 8 + threadIdx.x / kWarp;
    } else {
        inst = find_tile_owner(P.tile_prefix, P.count, tile);
        j = (tile - P.tile_prefix[inst]) * 256 + threadIdx.x;
    }
    return j < P.inst[inst].n;
}

template <typename T>
__global__ void __launch_bounds__(256) product_kernel(PlanDev P, ProdArgs<T> A) {
    int inst;
    int64_t j;
    if (!locate(P, inst, j)) return;
    const InstDev I = P.inst[inst];
    const int64_t n = I.n, ld = I.ld, cs = I.cs;
    const T *Am = A.A + I.band;
    const T *Bm = A.B + I.band;
    T *Cm = A.C + I.band;
    const int alo = A.alo < 0 ? I.l : A.alo, blo = A.blo < 0 ? I.l : A.blo, clo = A.clo < 0 ? I.l : A.clo;
    const int alo_op = A.transA ? A.aup : alo, aup_op = A.transA ? alo : A.aup;
    const int blo_op = A.transB ? A.bup : blo, bup_op = A.transB ? blo : A.bup;
    for (int r = 0; r < clo + A.cup + 1; ++r) {
        const int64_t i = j + (r - A.cup);
        T s = T(0);
        if (i >= 0 && i < n) {
            const int64_t t0 = imax64(imax64(i - alo_op, j - bup_op), 0);
            const int64_t t1 = imin64(imin64(i + aup_op, j + blo_op), n - 1);
            for (int64_t t = t0; t <= t1; ++t)
                s = fma(band_get(Am, ld, cs, alo, A.aup, A.transA != 0, n, i, t),
                        band_get(Bm, ld, cs, blo, A.bup, A.transB != 0, n, t, j), s);
            s *= A.alpha;
        }
        T *p = &Cm[(int64_t)r * ld + j * cs];
        *p = (A.acc && i >= 0 && i < n) ? (*p + s) : s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) outer_kernel(PlanDev P, OuterArgs<T> A) {
    int inst;
    int64_t j;
    if (!locate(P, inst, j)) return;
    const InstDev I = P.inst[inst];
    const int64_t n = I.n, ld = I.ld, cs = I.cs;
    const T *M = A.M + I.rhs;
    const T *V = A.V + I.rhs;
    T *Cm = A.C + I.band;
    const int clo = A.clo < 0 ? I.l : A.clo;
    for (int r = 0; r < clo + A.cup + 1; ++r) {
        const int64_t i = j + (r - A.cup);
        T s = T(0);
        if (i >= 0 && i < n) {
            for (int c = 0; c < A.k; ++c) s = fma(M[(int64_t)c * I.ldr + i * cs], V[(int64_t)c * I.ldr + j * cs], s);
            s *= A.alpha;
        }
        T *p = &Cm[(int64_t)r * ld + j * cs];
        *p = (A.acc && i >= 0 && i < n) ? (*p + s) : s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) matvec_kernel(PlanDev P, MatvecArgs<T> A) {
    int inst;
    int64_t i;
    if (!locate(P, inst, i)) return;
    const InstDev I = P.inst[inst];
    const int64_t n = I.n;
    const T *Am = A.A + I.band;
    const T *V = A.V + I.rhs;
    T *Po = A.P + I.rhs;
    const int alo = A.alo < 0 ? I.l : A.alo;
    const int alo_op = A.transA ? A.aup : alo, aup_op = A.transA ? alo : A.aup;
    const int64_t t0 = imax64(i - alo_op, 0), t1 = imin64(i + aup_op, n - 1);
    for (int c = 0; c < A.k; ++c) {
        T s = T(0);
        for (int64_t t = t0; t <= t1; ++t)
            s = fma(band_get(Am, I.ld, I.cs, alo, A.aup, A.transA != 0, n, i, t), V[(int64_t)c * I.ldr + t * I.cs], s);
        s *= A.alpha;
        T *p = &Po[(int64_t)c * I.ldr + i * I.cs];
        *p = A.acc ? (*p + s) : s;
    }
}

// Alg. 5, one thread per output column c: O = band_{olo,oup}(L^{-1} R) is the
// lower triangular solve restricted to the rows c - oup .. c + olo of column
// c (rows above c - rup are exactly 0 since oup >= rup); the transposed form
// O = band(L^{-T} R) solves upward from row c + olo (rows below c + rlo are
// exactly 0 since olo >= rlo).  Each entry uses only entries of its own
// column, which is why the columns are independent -- the same dependency
// Alg. 5 follows diagonal by diagonal.  The thread reads back its own writes.
template <typename T>
__global__ void __launch_bounds__(256) solve_band_kernel(PlanDev P, SolveBandArgs<T> A) {
    int inst;
    int64_t c;
    if (!locate(P, inst, c)) return;
    const InstDev I = P.inst[inst];
    const int64_t n = I.n, ld = I.ld, cs = I.cs;
    const int l = I.l;
    const T *Lm = A.L + I.band;
    const T *R = A.R + I.band;
    T *O = A.O + I.band;
#define LAT(r_, m_) Lm[(int64_t)((r_) - (m_)) * ld + (m_) * cs]
#define OAT(r_) O[(int64_t)(A.oup + (r_) - c) * ld + c * cs]
    const int64_t r0 = imax64(c - A.oup, 0), r1 = imin64(c + A.olo, n - 1);
    if (!A.trans) {
        for (int64_t r = r0; r <= r1; ++r) {
            const int64_t k = r - c;
            T s = (k <= A.rlo && -k <= A.rup) ? R[(int64_t)(A.rup + k) * ld + c * cs] : T(0);
            for (int64_t m = imax64(r - l, r0); m < r; ++m) s = fma(-LAT(r, m), OAT(m), s);
            OAT(r) = s / LAT(r, r);
        }
    } else {
        for (int64_t r = r1; r >= r0; --r) {
            const int64_t k = r - c;
            T s = (k <= A.rlo && -k <= A.rup) ? R[(int64_t)(A.rup + k) * ld + c * cs] : T(0);
            for (int64_t m = imin64(r + l, r1); m > r; --m) s = fma(-LAT(m, r), OAT(m), s);
            OAT(r) = s / LAT(r, r);
        }
    }
    // band entries outside the matrix: 0
    for (int64_t k = -A.oup; k <= A.olo; ++k)
        if (c + k < 0 || c + k >= n) O[(int64_t)(A.oup + k) * ld + c * cs] = T(0);
#undef LAT
#undef OAT
}

// dst (+)= src restricted to dst's band (entries of dst outside src's band or
// outside the matrix: 0, or unchanged when accumulating).
template <typename T>
__global__ void __launch_bounds__(256) band_copy_kernel(PlanDev P, BandCopyArgs<T> A) {
    int inst;
    int64_t c;
    if (!locate(P, inst, c)) return;
    const InstDev I = P.inst[inst];
    for (int k = -A.dup; k <= A.dlo; ++k) {
        const bool in = c + k >= 0 && c + k < I.n && k <= A.slo && -k <= A.sup;
        const T v = in ? A.src[I.band + (int64_t)(A.sup + k) * I.ld + c * I.cs] : T(0);
        T *p = &A.dst[I.band + (int64_t)(A.dup + k) * I.ld + c * I.cs];
        const bool inside = c + k >= 0 && c + k < I.n;
        *p = A.acc ? (inside ? *p + v : T(0)) : v;
    }
}

// dst += src over the lower band of every instance (corners written as 0).
template <typename T>
__global__ void __launch_bounds__(256) band_add_kernel(PlanDev P, const T *src, T *dst) {
    int inst;
    int64_t j;
    if (!locate(P, inst, j)) return;
    const InstDev I = P.inst[inst];
    for (int d = 0; d <= I.l; ++d) {
        const int64_t o = I.band + (int64_t)d * I.ld + j * I.cs;
        dst[o] = (j + d < I.n) ? dst[o] + src[o] : T(0);
    }
}

template <typename T>
cudaError_t launch_band_add(const bnd_plan *p, const T *src, T *dst, cudaStream_t s) {
    if (p->ntiles == 0) return cudaSuccess;
    band_add_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, src, dst);
    return cudaGetLastError();
}
template cudaError_t launch_band_add<float>(const bnd_plan *, const float *, float *, cudaStream_t);
template cudaError_t launch_band_add<double>(const bnd_plan *, const double *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_product(const bnd_plan *p, const ProdArgs<T> &A, cudaStream_t s) {
    if (p->ntiles == 0) return cudaSuccess;
    product_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, A);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_outer(const bnd_plan *p, const OuterArgs<T> &A, cudaStream_t s) {
    if (p->ntiles == 0 || A.k == 0) return cudaSuccess;
    outer_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, A);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_matvec(const bnd_plan *p, const MatvecArgs<T> &A, cudaStream_t s) {
    if (p->ntiles == 0 || A.k == 0) return cudaSuccess;
    matvec_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_band(const bnd_plan *p, const SolveBandArgs<T> &A, cudaStream_t s) {
    if (p->ntiles == 0) return cudaSuccess;
    solve_band_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, A);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_band_copy(const bnd_plan *p, const BandCopyArgs<T> &A, cudaStream_t s) {
    if (p->ntiles == 0) return cudaSuccess;
    band_copy_kernel<T><<<(unsigned)p->ntiles, 256, 0, s>>>(p->dev, A);
    return cudaGetLastError();
}
template cudaError_t launch_solve_band<float>(const bnd_plan *, const SolveBandArgs<float> &, cudaStream_t);
template cudaError_t launch_solve_band<double>(const bnd_plan *, const SolveBandArgs<double> &, cudaStream_t);
template cudaError_t launch_band_copy<float>(const bnd_plan *, const BandCopyArgs<float> &, cudaStream_t);
template cudaError_t launch_band_copy<double>(const bnd_plan *, const BandCopyArgs<double> &, cudaStream_t);

template cudaError_t launch_product<float>(const bnd_plan *, const ProdArgs<float> &, cudaStream_t);
template cudaError_t launch_product<double>(const bnd_plan *, const ProdArgs<double> &, cudaStream_t);
template cudaError_t launch_outer<float>(const bnd_plan *, const OuterArgs<float> &, cudaStream_t);
template cudaError_t launch_outer<double>(const bnd_plan *, const OuterArgs<double> &, cudaStream_t);
template cudaError_t launch_matvec<float>(const bnd_plan *, const MatvecArgs<float> &, cudaStream_t);
template cudaError_t launch_matvec<double>(const bnd_plan *, const MatvecArgs<double> &, cudaStream_t);

}  // namespace bnd
