// Products P and O (Sec. 4.1): band x band projected onto a target band,
// band x vectors, and the band-projected outer product.  Every output column
// is independent, so these are one-thread-per-column kernels over a flat list
// of 256-column tiles (tile prefix per instance, binary searched).
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

__device__ __forceinline__ int find_instance(const int64_t *prefix, int count, int64_t tile) {
    int lo = 0, hi = count;               // prefix[lo] <= tile < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) product_kernel(PlanDev P, ProdArgs<T> A) {
    const int64_t tile = blockIdx.x;
    if (tile >= P.ntiles) return;
    const int inst = find_instance(P.tile_prefix, P.count, tile);
    const InstDev I = P.inst[inst];
    const int64_t j = (tile - P.tile_prefix[inst]) * 256 + threadIdx.x;
    if (j >= I.n) return;
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
    const int64_t tile = blockIdx.x;
    if (tile >= P.ntiles) return;
    const int inst = find_instance(P.tile_prefix, P.count, tile);
    const InstDev I = P.inst[inst];
    const int64_t j = (tile - P.tile_prefix[inst]) * 256 + threadIdx.x;
    if (j >= I.n) return;
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
    const int64_t tile = blockIdx.x;
    if (tile >= P.ntiles) return;
    const int inst = find_instance(P.tile_prefix, P.count, tile);
    const InstDev I = P.inst[inst];
    const int64_t i = (tile - P.tile_prefix[inst]) * 256 + threadIdx.x;
    if (i >= I.n) return;
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

// dst += src over the lower band of every instance (corners written as 0).
template <typename T>
__global__ void __launch_bounds__(256) band_add_kernel(PlanDev P, const T *src, T *dst) {
    const int64_t tile = blockIdx.x;
    if (tile >= P.ntiles) return;
    const int inst = find_instance(P.tile_prefix, P.count, tile);
    const InstDev I = P.inst[inst];
    const int64_t j = (tile - P.tile_prefix[inst]) * 256 + threadIdx.x;
    if (j >= I.n) return;
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

template cudaError_t launch_product<float>(const bnd_plan *, const ProdArgs<float> &, cudaStream_t);
template cudaError_t launch_product<double>(const bnd_plan *, const ProdArgs<double> &, cudaStream_t);
template cudaError_t launch_outer<float>(const bnd_plan *, const OuterArgs<float> &, cudaStream_t);
template cudaError_t launch_outer<double>(const bnd_plan *, const OuterArgs<double> &, cudaStream_t);
template cudaError_t launch_matvec<float>(const bnd_plan *, const MatvecArgs<float> &, cudaStream_t);
template cudaError_t launch_matvec<double>(const bnd_plan *, const MatvecArgs<double> &, cudaStream_t);

}  // namespace bnd
