// Persistent sweep kernels, the segment verify/fixup kernel and their host
// launchers.  Included (once) by each per-dtype, per-direction translation unit.
#pragma once

#include "sweep_impl.cuh"

namespace bnd {

// ---------------------------------------------------------------------------
// Dispatch of one chain run on its (warp-uniform) bandwidth.
// ---------------------------------------------------------------------------
template <typename T, int K, int FL, bool FWD>
__device__ __forceinline__ void run_chain(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c,
                                          int mode, const T *exact) {
#define BND_CASE(LV)                                                         \
    case LV:                                                                 \
        if constexpr (FWD) run_fwd_reg<T, LV, K, FL>(P, A, c, mode, exact); \
        else run_bwd_reg<T, LV, K, FL>(P, A, c, mode, exact);               \
        break;
    switch (c.l) {
        BND_CASE(1)
        BND_CASE(2)
        BND_CASE(3)
        BND_CASE(4)
        BND_CASE(5)
        BND_CASE(6)
        BND_CASE(7)
        BND_CASE(8)
        default:
            if constexpr (FWD) run_fwd_generic<T, FL>(P, A, c);
            else run_bwd_generic<T, FL>(P, A, c);
    }
#undef BND_CASE
}

// Number of state words compared at a segment boundary.
template <typename T, int K, int FL, bool FWD>
__device__ __forceinline__ int state_words(int l) {
#define BND_SW(LV) \
    case LV: return FWD ? FwdReg<T, LV, K, FL>::snap_words() : BwdReg<T, LV, K, FL>::snap_words();
    switch (l) {
        BND_SW(1) BND_SW(2) BND_SW(3) BND_SW(4) BND_SW(5) BND_SW(6) BND_SW(7) BND_SW(8)
        default: return 0;
    }
#undef BND_SW
}

__device__ __forceinline__ ChainCtx make_ctx(const PlanDev &P, int32_t inst, int32_t seg) {
    const InstDev I = P.inst[inst];
    ChainCtx c;
    c.n = I.n; c.band = I.band; c.ld = I.ld; c.rhs = I.rhs; c.ldr = I.ldr; c.l = I.l;
    c.inst = inst;
    c.gseg = I.seg0 + seg;
    c.a = (int64_t)seg * I.seg_len;
    c.b = imin64(c.a + I.seg_len, I.n);
    c.first = (seg == 0);
    c.last = (seg == I.nseg - 1);
    return c;
}

// ---------------------------------------------------------------------------
// Persistent sweep kernel: each warp takes 32-chain tasks from a queue
// ordered longest first; each lane runs one chain.
// ---------------------------------------------------------------------------
template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(128) sweep_kernel(PlanDev P, SweepArgs<T> A) {
    const int lane = threadIdx.x & (kWarp - 1);
    unsigned int *head = P.counters + A.kind;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(head, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= P.ntasks) break;
        const Task task = P.tasks[t];
        const Chain ch = P.chains[(int64_t)task.chain0 + lane];
        if (ch.inst >= 0) {
            const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
            run_chain<T, K, FL, FWD>(P, A, c, RUN_COLD, nullptr);
        }
    }
}

// ---------------------------------------------------------------------------
// Verify / fixup: one thread per segmented instance walks its segment
// boundaries in sweep order.  A segment whose cold-started state differs
// (bitwise) from its predecessor's exact end state is rerun from that exact
// state, which rewrites its outputs and its own end state.  Forward sweeps
// that compute the Cholesky then reduce the per-segment log-det and info.
// ---------------------------------------------------------------------------
template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(64) verify_kernel(PlanDev P, SweepArgs<T> A) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= P.count) return;
    const InstDev I = P.inst[inst];
    if (I.nseg <= 1) return;
    const int words = state_words<T, K, FL, FWD>(I.l);
    unsigned int fixes = 0;
    if (FWD) {
        for (int p = 1; p < I.nseg; ++p) {
            const int64_t g = I.seg0 + p;
            const T *prev_end = snap_ptr<T>(P, g - 1, 1);
            if (!snap_equal(prev_end, (const T *)snap_ptr<T>(P, g, 0), words)) {
                run_chain<T, K, FL, FWD>(P, A, make_ctx(P, inst, p), RUN_EXACT, prev_end);
                ++fixes;
            }
        }
    } else {
        for (int p = I.nseg - 2; p >= 0; --p) {
            const int64_t g = I.seg0 + p;
            const T *next_end = snap_ptr<T>(P, g + 1, 1);
            if (!snap_equal(next_end, (const T *)snap_ptr<T>(P, g, 0), words)) {
                run_chain<T, K, FL, FWD>(P, A, make_ctx(P, inst, p), RUN_EXACT, next_end);
                ++fixes;
            }
        }
    }
    if constexpr (FWD && (FL & F_CHOL)) {
        double ld = 0.0;
        int32_t info = 0;
        for (int p = 0; p < I.nseg; ++p) {
            ld += P.seg_logdet[I.seg0 + p];
            if (info == 0) info = P.seg_info[I.seg0 + p];
        }
        if (A.logdet) A.logdet[inst] = info ? (double)NAN : ld;
        A.info[inst] = info;
    }
    if (fixes) atomicAdd(P.counters + kNumSweepKinds + A.kind, fixes);
}

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
template <typename T, int K, int FL, bool FWD>
static cudaError_t launch_sweep_t(const bnd_plan *p, const SweepArgs<T> &A, cudaStream_t s) {
    static int blocks_per_sm = -1;
    static int num_sms = 0;
    if (blocks_per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<T, K, FL, FWD>, 128, 0);
        blocks_per_sm = b > 0 ? b : 1;
    }
    int bps = p->blocks_per_sm > 0 ? p->blocks_per_sm : blocks_per_sm;
    int64_t blocks = (int64_t)num_sms * bps;
    const int64_t need = (p->ntasks + 3) / 4;          // 4 warps per block
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaMemsetAsync(p->dev.counters + A.kind, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    sweep_kernel<T, K, FL, FWD><<<(unsigned)blocks, 128, 0, s>>>(p->dev, A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p->nsegs > p->count) {
        verify_kernel<T, K, FL, FWD><<<(p->count + 63) / 64, 64, 0, s>>>(p->dev, A);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace bnd

namespace bnd {

// (flags, K) -> kernel instantiation.  K = 0 for sweeps without right-hand
// sides, 1 for a single column, 4 for up to four columns (runtime kk <= 4).
template <typename T>
cudaError_t dispatch_fwd(const bnd_plan *p, int fl, int K, const SweepArgs<T> &A, cudaStream_t s) {
    switch (fl) {
        case F_CHOL: return launch_sweep_t<T, 0, F_CHOL, true>(p, A, s);
        case F_ALG4: return launch_sweep_t<T, 0, F_ALG4, true>(p, A, s);
        case F_CHOL | F_SOLVE:
            return K == 1 ? launch_sweep_t<T, 1, F_CHOL | F_SOLVE, true>(p, A, s)
                          : launch_sweep_t<T, 4, F_CHOL | F_SOLVE, true>(p, A, s);
        case F_SOLVE:
            return K == 1 ? launch_sweep_t<T, 1, F_SOLVE, true>(p, A, s)
                          : launch_sweep_t<T, 4, F_SOLVE, true>(p, A, s);
        case F_ALG4 | F_SOLVE:
            return K == 1 ? launch_sweep_t<T, 1, F_ALG4 | F_SOLVE, true>(p, A, s)
                          : launch_sweep_t<T, 4, F_ALG4 | F_SOLVE, true>(p, A, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t dispatch_bwd(const bnd_plan *p, int fl, int K, const SweepArgs<T> &A, cudaStream_t s) {
    switch (fl) {
        case B_TAKA: return launch_sweep_t<T, 0, B_TAKA, false>(p, A, s);
        case B_ALG2: return launch_sweep_t<T, 0, B_ALG2, false>(p, A, s);
        case B_TAKA | B_SOLVE:
            return K == 1 ? launch_sweep_t<T, 1, B_TAKA | B_SOLVE, false>(p, A, s)
                          : launch_sweep_t<T, 4, B_TAKA | B_SOLVE, false>(p, A, s);
        case B_SOLVE:
            return K == 1 ? launch_sweep_t<T, 1, B_SOLVE, false>(p, A, s)
                          : launch_sweep_t<T, 4, B_SOLVE, false>(p, A, s);
        case B_ALG2 | B_SOLVE | B_OUTER:
            return K == 1 ? launch_sweep_t<T, 1, B_ALG2 | B_SOLVE | B_OUTER, false>(p, A, s)
                          : launch_sweep_t<T, 4, B_ALG2 | B_SOLVE | B_OUTER, false>(p, A, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bnd
