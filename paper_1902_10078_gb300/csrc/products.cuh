// Launcher declarations of the product kernels and the sweeps.
#pragma once

#include "common.cuh"

namespace bnd {

template <typename T>
struct ProdArgs {
    const T *A; const T *B; T *C;
    int alo, aup, blo, bup, clo, cup;
    int transA, transB;
    int acc;
    T alpha;
};

template <typename T>
struct OuterArgs {
    const T *M; const T *V; T *C;      // M, V: RHS pools; C: band pool
    int clo, cup;
    int k;
    int acc;
    T alpha;
};

template <typename T>
struct MatvecArgs {
    const T *A; const T *V; T *P;      // A: band pool; V, P: RHS pools
    int alo, aup, transA;
    int k;
    int acc;
    T alpha;
};

template <typename T>
struct SolveBandArgs {
    const T *L; const T *R; T *O;      // L: lower band l (per instance); R, O: general bands
    int rlo, rup, olo, oup;
    int trans;
};

template <typename T>
struct BandCopyArgs {                  // dst (dlo, dup) (+)= src (slo, sup) on dst's band
    const T *src; T *dst;
    int slo, sup, dlo, dup;
    int acc;
};

template <typename T> cudaError_t launch_product(const bnd_plan *p, const ProdArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_solve_band(const bnd_plan *p, const SolveBandArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_band_copy(const bnd_plan *p, const BandCopyArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_outer(const bnd_plan *p, const OuterArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_matvec(const bnd_plan *p, const MatvecArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_band_add(const bnd_plan *p, const T *src, T *dst, cudaStream_t s);

template <typename T> struct SweepArgs;
template <typename T> cudaError_t launch_fwd(const bnd_plan *p, int fl, int K, const SweepArgs<T> &A, cudaStream_t s);
template <typename T> cudaError_t launch_bwd(const bnd_plan *p, int fl, int K, const SweepArgs<T> &A, cudaStream_t s);

}  // namespace bnd
