// Staged per-bandwidth sweep kernels (row plans: StagedIO; panel plans:
// PanelIO) and their launcher.  Each sweep_staged_l<L>.cu instantiates the
// launcher for one bandwidth, both dtypes and every sweep of the dispatch.
#pragma once

#include "sweep_launch.cuh"

namespace bnd {

// ---------------------------------------------------------------------------
// Staged kernel for one bandwidth L: block b runs warp tasks
// [task0 + WPB b, task0 + WPB (b+1)) of the bandwidth's task range (ordered
// longest first); each lane runs one chain.  Row plans stage every lane's own
// rows (StagedIO); panel plans stage the group's interleaved columns with the
// whole warp (PanelIO), so idle lanes stay in the loop.
// ---------------------------------------------------------------------------
template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
struct StagedIOOf {
    using SW = typename SweepOf<T, L, K, FL, FWD>::type;
    using type = typename std::conditional<PANEL, PanelIO<T, SW, RingDepth<L>::R, FWD ? 1 : -1>,
                                           StagedIO<T, SW, RingDepth<L>::R, FWD ? 1 : -1>>::type;
};

template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
__global__ void __launch_bounds__(kWarp * kStagedWarpsPerBlock)
staged_kernel(PlanDev P, SweepArgs<T> A, int32_t task0, int32_t ntasks) {
    using IO = typename StagedIOOf<T, L, K, FL, FWD, PANEL>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int t = blockIdx.x * kStagedWarpsPerBlock + warp;
    if (t >= ntasks) return;
    const Task task = P.tasks[task0 + t];
    const Chain ch = P.chains[(int64_t)task.chain0 + lane];
    T *wsm = reinterpret_cast<T *>(smem_raw) + (size_t)warp * IO::kWarpElems;
    if constexpr (PANEL) {
        const ChainCtx c = ch.inst >= 0 ? make_ctx(P, ch.inst, ch.seg) : idle_ctx();
        const ChainPtrs<T> ptrs = chain_ptrs(A, c);
        IO io(ptrs, A, task, wsm, lane);
        run_reg<T, L, K, FL, FWD>(P, A, c, RUN_COLD, nullptr, io);
    } else {
        if (ch.inst < 0) return;
        const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
        const ChainPtrs<T> ptrs = chain_ptrs(A, c);
        IO io(ptrs, wsm, lane);
        run_reg<T, L, K, FL, FWD>(P, A, c, RUN_COLD, nullptr, io);
    }
}

template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
constexpr size_t staged_smem_bytes() {
    return sizeof(T) * (size_t)StagedIOOf<T, L, K, FL, FWD, PANEL>::type::kWarpElems * kStagedWarpsPerBlock;
}

template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
static cudaError_t launch_staged_lp(const bnd_plan *p, const SweepArgs<T> &A, cudaStream_t s) {
    const int32_t t0 = p->class_task0[L], nt = p->class_task0[L + 1] - t0;
    if (nt <= 0) return cudaSuccess;
    constexpr size_t smem = staged_smem_bytes<T, L, K, FL, FWD, PANEL>();
    static PerDeviceSlots attr;       // the attribute is set once on every device the kernel runs on
    const int ok = per_device(attr, [] {
        return cudaFuncSetAttribute(staged_kernel<T, L, K, FL, FWD, PANEL>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess ? 1 : -1;
    });
    if (ok <= 0) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((nt + kStagedWarpsPerBlock - 1) / kStagedWarpsPerBlock);
    staged_kernel<T, L, K, FL, FWD, PANEL><<<blocks, kWarp * kStagedWarpsPerBlock, smem, s>>>(p->dev, A, t0, nt);
    return cudaGetLastError();
}

template <typename T, int L, int K, int FL, bool FWD>
cudaError_t launch_staged_l(const bnd_plan *p, const SweepArgs<T> &A, cudaStream_t s) {
    return p->layout == kLayoutPanels ? launch_staged_lp<T, L, K, FL, FWD, true>(p, A, s)
                                      : launch_staged_lp<T, L, K, FL, FWD, false>(p, A, s);
}

}  // namespace bnd

// The (K, flags, direction) combinations dispatch_fwd / dispatch_bwd launch.
#define BND_STAGED_ONE(T, L, K, FL, FWD) \
    template cudaError_t launch_staged_l<T, L, K, FL, FWD>(const bnd_plan *, const SweepArgs<T> &, cudaStream_t);
#define BND_STAGED_DTYPE(T, L)                                                                                    \
    BND_STAGED_ONE(T, L, 0, F_CHOL, true) BND_STAGED_ONE(T, L, 0, F_ALG4, true)                                   \
    BND_STAGED_ONE(T, L, 1, F_CHOL | F_SOLVE, true) BND_STAGED_ONE(T, L, 4, F_CHOL | F_SOLVE, true)               \
    BND_STAGED_ONE(T, L, 1, F_SOLVE, true) BND_STAGED_ONE(T, L, 4, F_SOLVE, true)                                 \
    BND_STAGED_ONE(T, L, 1, F_ALG4 | F_SOLVE, true) BND_STAGED_ONE(T, L, 4, F_ALG4 | F_SOLVE, true)               \
    BND_STAGED_ONE(T, L, 0, B_TAKA, false) BND_STAGED_ONE(T, L, 0, B_ALG2, false)                                 \
    BND_STAGED_ONE(T, L, 1, B_TAKA | B_SOLVE, false) BND_STAGED_ONE(T, L, 4, B_TAKA | B_SOLVE, false)             \
    BND_STAGED_ONE(T, L, 1, B_SOLVE, false) BND_STAGED_ONE(T, L, 4, B_SOLVE, false)                               \
    BND_STAGED_ONE(T, L, 1, B_ALG2 | B_SOLVE | B_OUTER, false)                                                    \
    BND_STAGED_ONE(T, L, 4, B_ALG2 | B_SOLVE | B_OUTER, false)
#define BND_STAGED_INSTANCES(L) \
    namespace bnd {             \
    BND_STAGED_DTYPE(float, L)  \
    BND_STAGED_DTYPE(double, L) \
    }
