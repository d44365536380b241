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
// Panel tiles by whole-block bulk copies completing on shared-memory barriers
// instead of per-lane 16-byte cp.async pieces (a build option: measured slower
// on the uneven batch, see the design notes).
#ifndef BND_PANEL_BULK
#define BND_PANEL_BULK 0
#endif
template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
struct StagedIOOf {
    using SW = typename SweepOf<T, L, K, FL, FWD>::type;
    using type = typename std::conditional<PANEL, PanelIO<T, SW, RingDepth<L>::R, FWD ? 1 : -1, BND_PANEL_BULK != 0>,
                                           StagedIO<T, SW, RingDepth<L>::R, FWD ? 1 : -1>>::type;
};

// Minimum resident blocks per SM asked of the register allocator (unset: none).
#ifdef BND_STAGED_MINB
#define BND_STAGED_BOUNDS __launch_bounds__(kWarp * kStagedWarpsPerBlock, BND_STAGED_MINB)
#else
#define BND_STAGED_BOUNDS __launch_bounds__(kWarp * kStagedWarpsPerBlock)
#endif

template <typename T, int L, int K, int FL, bool FWD, bool PANEL>
__global__ void BND_STAGED_BOUNDS
staged_kernel(PlanDev P, SweepArgs<T> A, int32_t task0, int32_t ntasks, int32_t rerun) {
    using IO = typename StagedIOOf<T, L, K, FL, FWD, PANEL>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int t = blockIdx.x * kStagedWarpsPerBlock + warp;
    if (t >= ntasks) return;
    int32_t task = task0 + t;
    bool mine = true;                  // this lane runs its chain
    if (rerun) {
        // rerun pass: warp t takes the t-th queued task of this bandwidth; only its flagged
        // lanes rerun, from the exact state their predecessor segment left; the flags are
        // cleared for the next sweep
        if (t >= (int)P.rerun_cnt[L]) return;
        task = P.rerun_list[task0 + t];
        const int64_t ci = (int64_t)task * kWarp + lane;
        mine = P.chain_flag[ci] != 0;
        if (mine) P.chain_flag[ci] = 0;
        if (lane == 0) P.task_flag[task] = 0u;
    }
    const Task tk = P.tasks[task];
    const Chain ch = P.chains[(int64_t)tk.chain0 + lane];
    const int mode = rerun ? RUN_EXACT : RUN_COLD;
    T *wsm = reinterpret_cast<T *>(smem_raw) + (size_t)warp * IO::kWarpElems;
    if constexpr (PANEL) {
        const bool run = ch.inst >= 0 && mine;
        const ChainCtx c = run ? make_ctx(P, ch.inst, ch.seg) : idle_ctx();
        const T *exact = (run && rerun) ? exact_start<T, FWD>(P, c) : nullptr;
        const ChainPtrs<T> ptrs = chain_ptrs(A, c);
        IO io(ptrs, A, tk, wsm, lane, P.counters + kTimeoutCounter);
        run_reg<T, L, K, FL, FWD>(P, A, c, mode, exact, io);
    } else {
        if (ch.inst < 0 || !mine) return;
        const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
        const T *exact = rerun ? exact_start<T, FWD>(P, c) : nullptr;
        const ChainPtrs<T> ptrs = chain_ptrs(A, c);
        IO io(ptrs, wsm, lane);
        run_reg<T, L, K, FL, FWD>(P, A, c, mode, exact, io);
    }
}

// Mark pass of the staged reruns: one thread per chain of the bandwidth's
// tasks compares the state its segment started from (speculative warm-up)
// bit for bit with the exact state the neighbouring segment left at that
// boundary, and on a mismatch flags the chain and queues its task once.
template <typename T, int L, int K, int FL, bool FWD>
__global__ void __launch_bounds__(256) mark_kernel(PlanDev P, int32_t task0, int32_t ntasks, int32_t kind) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ntasks * kWarp) return;
    const int64_t ci = (int64_t)task0 * kWarp + i;
    const Chain ch = P.chains[ci];
    if (ch.inst < 0) return;
    const InstDev I = P.inst[ch.inst];
    if (I.nseg <= 1) return;
    constexpr int words = SweepOf<T, L, K, FL, FWD>::type::snap_words();
    const int64_t g = I.seg0 + ch.seg;
    bool eq;
    if (FWD) {
        if (ch.seg == 0) return;
        eq = snap_equal(snap_ptr<T>(P, g - 1, 1), (const T *)snap_ptr<T>(P, g, 0), words);
    } else {
        if (ch.seg == I.nseg - 1) return;
        eq = snap_equal(snap_ptr<T>(P, g + 1, 1), (const T *)snap_ptr<T>(P, g, 0), words);
    }
    if (eq) return;
    P.chain_flag[ci] = 1;
    const int32_t task = (int32_t)(ci / kWarp);
    if (atomicExch(&P.task_flag[task], 1u) == 0u) {
        const uint32_t k = atomicAdd(&P.rerun_cnt[L], 1u);
        P.rerun_list[task0 + k] = task;
    }
    atomicAdd(P.counters + kNumSweepKinds + kind, 1u);
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
    staged_kernel<T, L, K, FL, FWD, PANEL><<<blocks, kWarp * kStagedWarpsPerBlock, smem, s>>>(p->dev, A, t0, nt, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || p->nsegs <= p->count || p->no_staged_rerun) return e;
    // staged reruns of the segments whose speculative start was wrong (same stream: after the sweep)
    e = cudaMemsetAsync(p->dev.rerun_cnt + L, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t nch = (int64_t)nt * kWarp;
    mark_kernel<T, L, K, FL, FWD><<<(unsigned)((nch + 255) / 256), 256, 0, s>>>(p->dev, t0, nt, A.kind);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    staged_kernel<T, L, K, FL, FWD, PANEL><<<blocks, kWarp * kStagedWarpsPerBlock, smem, s>>>(p->dev, A, t0, nt, 1);
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
