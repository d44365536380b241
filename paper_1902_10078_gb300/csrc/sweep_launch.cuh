// Sweep kernels (staged per-bandwidth for row and panel plans, one warp per
// instance for wide bands, persistent direct), the segment verify/fixup
// kernel and their host launcher.  Included (once) by each per-dtype,
// per-direction translation unit.
#pragma once

#include <mutex>
#include <type_traits>

#include "sweep_cta.cuh"
#include "sweep_impl.cuh"
#include "sweep_wide.cuh"

namespace bnd {

#ifndef BND_STAGED_WPB
#define BND_STAGED_WPB 2
#endif
#ifndef BND_RING_SMALL_L
#define BND_RING_SMALL_L 4
#endif
#ifndef BND_RING_LARGE_L
#define BND_RING_LARGE_L 2
#endif
constexpr int kStagedWarpsPerBlock = BND_STAGED_WPB;

// One-time per-device values (kernel occupancy, function attributes set on a
// device).  Each caller keeps one slot table per kernel; the first launch on a
// device fills that device's slot under the table's mutex, so two host
// threads or two devices never see a half-written or foreign value.  A
// failed computation (value <= 0) is not cached.
constexpr int kMaxDevices = 64;
struct PerDeviceSlots {
    std::mutex mu;
    int value[kMaxDevices] = {};
};
template <class F>
inline int per_device(PerDeviceSlots &t, F compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute();
    std::lock_guard<std::mutex> lock(t.mu);
    if (t.value[dev] <= 0) t.value[dev] = compute();
    return t.value[dev];
}

// Ring depth (tiles per stream) of the staged kernels: short iterations
// (small l) want a deeper prefetch to cover the memory latency, long ones
// (large l, more streams) a shallower one to fit shared memory.
template <int L>
struct RingDepth { static constexpr int R = L <= 4 ? BND_RING_SMALL_L : BND_RING_LARGE_L; };

template <typename T, int L, int K, int FL, bool FWD>
struct SweepOf {
    using type = typename std::conditional<FWD, FwdReg<T, L, K, FL>, BwdReg<T, L, K, FL>>::type;
};

template <typename T, int L, int K, int FL, bool FWD, class IO>
__device__ __forceinline__ void run_reg(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c, int mode,
                                        const T *exact, IO &io) {
    if constexpr (FWD) run_fwd_reg<T, L, K, FL>(P, A, c, mode, exact, io);
    else run_bwd_reg<T, L, K, FL>(P, A, c, mode, exact, io);
}

// One chain with direct global I/O, dispatched on its bandwidth.
template <typename T, int K, int FL, bool FWD>
__device__ __forceinline__ void run_chain_direct(const PlanDev &P, const SweepArgs<T> &A, const ChainCtx &c,
                                                 int mode, const T *exact) {
    const ChainPtrs<T> ptrs = chain_ptrs(A, c);
#define BND_CASE(LV)                                                                    \
    case LV: {                                                                          \
        DirectIO<T, typename SweepOf<T, LV, K, FL, FWD>::type> io(ptrs);               \
        run_reg<T, LV, K, FL, FWD>(P, A, c, mode, exact, io);                          \
        break;                                                                          \
    }
    switch (c.l) {
        BND_CASE(1) BND_CASE(2) BND_CASE(3) BND_CASE(4) BND_CASE(5) BND_CASE(6) BND_CASE(7) BND_CASE(8)
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
    case LV: return SweepOf<T, LV, K, FL, FWD>::type::snap_words();
    switch (l) {
        BND_SW(1) BND_SW(2) BND_SW(3) BND_SW(4) BND_SW(5) BND_SW(6) BND_SW(7) BND_SW(8)
        default: return 0;
    }
#undef BND_SW
}

__device__ __forceinline__ ChainCtx make_ctx(const PlanDev &P, int32_t inst, int32_t seg) {
    const InstDev I = P.inst[inst];
    ChainCtx c;
    c.n = I.n; c.band = I.band; c.ld = I.ld; c.rhs = I.rhs; c.ldr = I.ldr; c.cs = I.cs; c.l = I.l;
    c.inst = inst;
    c.warm = I.warm;
    c.gseg = I.seg0 + seg;
    c.a = (int64_t)seg * I.seg_len;
    c.b = imin64(c.a + I.seg_len, I.n);
    c.first = (seg == 0);
    c.last = (seg == I.nseg - 1);
    return c;
}

// Context of an idle lane of a panel task: no rows, nothing written.
__device__ __forceinline__ ChainCtx idle_ctx() {
    ChainCtx c;
    c.n = 0; c.band = 0; c.ld = 0; c.rhs = 0; c.ldr = 0; c.cs = kPanelLanes; c.l = 0;
    c.inst = -1; c.warm = 0; c.gseg = 0; c.a = 0; c.b = 0;
    c.first = true; c.last = true;
    return c;
}

// Exact start state of a rerun segment: the end snapshot of the segment before
// it in sweep order (forward sweeps: the one above; backward: the one below).
template <typename T, bool FWD>
__device__ __forceinline__ const T *exact_start(const PlanDev &P, const ChainCtx &c) {
    return snap_ptr<T>(P, FWD ? c.gseg - 1 : c.gseg + 1, 1);
}

// Staged per-bandwidth launcher: defined in sweep_staged.cuh and explicitly
// instantiated per bandwidth in its own translation unit (sweep_staged_l*.cu),
// so the large staged kernels compile in parallel.
template <typename T, int L, int K, int FL, bool FWD>
cudaError_t launch_staged_l(const bnd_plan *p, const SweepArgs<T> &A, cudaStream_t s);

// ---------------------------------------------------------------------------
// Wide-band kernel: one warp per chain of the generic bandwidth class (l = 0
// or l above the register-window limit; such chains are whole instances).
// ---------------------------------------------------------------------------
constexpr int kWideWarpsPerBlock = 4;

template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(kWarp * kWideWarpsPerBlock)
wide_kernel(PlanDev P, SweepArgs<T> A, int64_t chain0, int64_t nchains) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x % kWarp;
    if (w >= nchains) return;
    const Chain ch = P.chains[chain0 + w];
    if (ch.inst < 0) return;
    const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
    if constexpr (FWD) run_fwd_wide<T, FL>(P, A, c, lane);
    else run_bwd_wide<T, FL>(P, A, c, lane);
}

// Block-per-chain kernel of the generic bandwidth class: the computed window
// in shared memory (sweep_cta.cuh).  Used when the window of the widest
// instance fits the per-block shared memory.

template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(kCtaThreads) cta_kernel(PlanDev P, SweepArgs<T> A, int64_t chain0, int64_t nchains,
                                                          int tier) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t w = blockIdx.x;
    if (w >= nchains) return;
    const Chain ch = P.chains[chain0 + w];
    if (ch.inst < 0) return;
    const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
    T *sm = reinterpret_cast<T *>(smem_raw);
    if constexpr (FWD) run_fwd_cta<T, FL>(P, A, c, sm, RUN_COLD, nullptr, tier);
    else run_bwd_cta<T, FL>(P, A, c, sm, RUN_COLD, nullptr, tier);
}

// Segment boundaries of the block sweeps, compared in parallel: block w takes
// chain chain0 + w (instance i, segment b >= 1) and flags boundary b of i
// (between segments b-1 and b) in chain_flag when the state the later segment
// in sweep order started from speculatively is not close to the end state
// its neighbour left.
template <typename T, bool FWD>
__global__ void __launch_bounds__(kCtaThreads) cta_compare_kernel(PlanDev P, int64_t chain0, int64_t nchains) {
    const int64_t w = blockIdx.x;
    if (w >= nchains) return;
    const Chain ch = P.chains[chain0 + w];
    if (ch.inst < 0 || ch.seg == 0) return;
    const InstDev I = P.inst[ch.inst];
    const int64_t g = I.seg0 + ch.seg;
    const T *x = FWD ? snap_ptr<T>(P, g - 1, 1) : snap_ptr<T>(P, g, 1);
    const T *y = FWD ? snap_ptr<T>(P, g, 0) : snap_ptr<T>(P, g - 1, 0);
    const bool ok = cta_states_close(x, y, I.l, cta_rhs(P.k));
    if (threadIdx.x == 0) P.chain_flag[chain0 + w] = ok ? 0 : 1;
}

// Fixup of the segmented block-sweep instances: one block per instance.  From
// the first flagged boundary in sweep order the block reruns, one after the
// other, every segment whose start state is still not close to the end state
// its (possibly rerun) neighbour left, from that exact state; the flags are
// cleared for the next launch.  The segments' log-det / info are reduced by
// verify_kernel after.
template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(kCtaThreads) cta_verify_kernel(PlanDev P, SweepArgs<T> A, int tier) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const InstDev I = P.inst[blockIdx.x];
    if ((I.l >= 1 && I.l <= kRegMaxL) || I.nseg <= 1) return;
    __shared__ int first_s;
    auto boundary_ok = [&](int b) {           // whole block; b joins segments b-1 and b
        const int64_t g = I.seg0 + b;
        const T *x = FWD ? snap_ptr<T>(P, g - 1, 1) : snap_ptr<T>(P, g, 1);
        const T *y = FWD ? snap_ptr<T>(P, g, 0) : snap_ptr<T>(P, g - 1, 0);
        return cta_states_close(x, y, I.l, cta_rhs(P.k));
    };
    if (threadIdx.x == 0) first_s = FWD ? I.nseg : 0;
    __syncthreads();
    for (int b = 1 + (int)threadIdx.x; b < I.nseg; b += kCtaThreads) {
        uint8_t *f = P.chain_flag + P.seg_chain[I.seg0 + b];
        if (*f) {
            if (FWD) atomicMin(&first_s, b);
            else atomicMax(&first_s, b);
            *f = 0;
        }
    }
    __syncthreads();
    const int first = first_s;
    T *sm = reinterpret_cast<T *>(smem_raw);
    unsigned int fixes = 0;
    if (FWD) {
        for (int b = first; b < I.nseg; ++b) {
            if (b > first && boundary_ok(b)) continue;
            __syncthreads();
            run_fwd_cta<T, FL>(P, A, make_ctx(P, blockIdx.x, b), sm, RUN_EXACT, snap_ptr<T>(P, I.seg0 + b - 1, 1),
                               tier);
            __syncthreads();
            ++fixes;
        }
    } else {
        for (int b = first; b >= 1; --b) {
            if (b < first && boundary_ok(b)) continue;
            __syncthreads();
            run_bwd_cta<T, FL>(P, A, make_ctx(P, blockIdx.x, b - 1), sm, RUN_EXACT, snap_ptr<T>(P, I.seg0 + b, 1),
                               tier);
            __syncthreads();
            ++fixes;
        }
    }
    if (threadIdx.x == 0 && fixes) atomicAdd(P.counters + kNumSweepKinds + A.kind, fixes);
}

template <typename T, int K, int FL, bool FWD>
static cudaError_t launch_wide(const bnd_plan *p, const SweepArgs<T> &A, int32_t t0, int32_t nt, cudaStream_t s) {
    if (nt <= 0) return cudaSuccess;
    // block kernels at the highest staging level whose rings fit next to the window
    const int tier = cta_tier<T>(FWD, FL, p->max_l, cta_rhs(p->k));
    if (p->wide_cta && tier >= 0) {
        const size_t cta_bytes = sizeof(T) * (size_t)cta_smem_elems(FWD, FL, p->max_l, cta_rhs(p->k), tier);
        static PerDeviceSlots attr;
        const int ok = per_device(attr, [] {
            return cudaFuncSetAttribute(cta_kernel<T, K, FL, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kCtaSmemLimit) == cudaSuccess ? 1 : -1;
        });
        if (ok <= 0) return cudaErrorInvalidValue;
        const int64_t nch = (int64_t)nt * kWarp;
        cta_kernel<T, K, FL, FWD><<<(unsigned)nch, kCtaThreads, cta_bytes, s>>>(p->dev, A, (int64_t)t0 * kWarp, nch,
                                                                                tier);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || !p->wide_segmented) return e;
        static PerDeviceSlots vattr;
        const int vok = per_device(vattr, [] {
            // the verify kernel has a few hundred bytes of static shared memory besides the window
            return cudaFuncSetAttribute(cta_verify_kernel<T, K, FL, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kCtaSmemLimit - 1024) == cudaSuccess ? 1 : -1;
        });
        if (vok <= 0) return cudaErrorInvalidValue;
        cta_compare_kernel<T, FWD><<<(unsigned)nch, kCtaThreads, 0, s>>>(p->dev, (int64_t)t0 * kWarp, nch);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cta_verify_kernel<T, K, FL, FWD><<<(unsigned)p->count, kCtaThreads, cta_bytes, s>>>(p->dev, A, tier);
        return cudaGetLastError();
    }
    // windows too large for shared memory: one warp per chain, windows in global memory
    const int64_t nch = (int64_t)nt * kWarp;
    const int64_t blocks = (nch + kWideWarpsPerBlock - 1) / kWideWarpsPerBlock;
    wide_kernel<T, K, FL, FWD><<<(unsigned)blocks, kWarp * kWideWarpsPerBlock, 0, s>>>(p->dev, A, (int64_t)t0 * kWarp,
                                                                                       nch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent direct kernel: warps take 32-chain tasks of [task0, task0+ntasks)
// from a queue; each lane runs one chain with direct global I/O.  Used for
// bandwidths above the register-window limit and for unaligned layouts.
// ---------------------------------------------------------------------------
template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(128) sweep_kernel(PlanDev P, SweepArgs<T> A, int32_t task0, int32_t ntasks) {
    const int lane = threadIdx.x & (kWarp - 1);
    unsigned int *head = P.counters + A.kind;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(head, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntasks) break;
        const Task task = P.tasks[task0 + t];
        const Chain ch = P.chains[(int64_t)task.chain0 + lane];
        if (ch.inst >= 0) {
            const ChainCtx c = make_ctx(P, ch.inst, ch.seg);
            run_chain_direct<T, K, FL, FWD>(P, A, c, RUN_COLD, nullptr);
        }
    }
}

// ---------------------------------------------------------------------------
// Verify / fixup: one warp per segmented instance.  The lanes compare the
// segment boundaries in parallel; from the first boundary (in sweep order)
// whose cold-started state differs bitwise from its predecessor's exact end
// state, lane 0 reruns segments from the exact state, one after the other,
// as long as the rerun changes the next boundary.  Forward Cholesky sweeps
// then reduce the per-segment log-det (a fixed tree over the lanes) and info.
// ---------------------------------------------------------------------------
constexpr int kVerifyWarps = 4;

template <typename T, int K, int FL, bool FWD>
__global__ void __launch_bounds__(kWarp * kVerifyWarps) verify_kernel(PlanDev P, SweepArgs<T> A) {
    const int inst = blockIdx.x * kVerifyWarps + threadIdx.x / kWarp;
    const int lane = threadIdx.x % kWarp;
    if (inst >= P.count) return;
    const InstDev I = P.inst[inst];
    if (I.nseg <= 1) return;
    const int words = state_words<T, K, FL, FWD>(I.l);
    // boundary b (1 <= b < nseg) joins segments b-1 and b; in sweep order the
    // forward sweeps meet them ascending, the backward sweeps descending
    auto boundary_ok = [&](int b) {
        const int64_t g = I.seg0 + b;
        return FWD ? snap_equal(snap_ptr<T>(P, g - 1, 1), (const T *)snap_ptr<T>(P, g, 0), words)
                   : snap_equal(snap_ptr<T>(P, g, 1), (const T *)snap_ptr<T>(P, g - 1, 0), words);
    };
    int first = FWD ? I.nseg : 0;          // first failing boundary in sweep order (none: past the end)
    for (int b = 1 + lane; b < I.nseg; b += kWarp)
        if (!boundary_ok(b)) first = FWD ? min(first, b) : max(first, b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int v = __shfl_xor_sync(0xffffffffu, first, o);
        first = FWD ? min(first, v) : max(first, v);
    }
    unsigned int fixes = 0;
    if (lane == 0) {
        // from the first failure on, walk the boundaries in sweep order: a rerun rewrites the
        // segment's end state, which the next boundary then compares against
        if (FWD) {
            for (int b = first; b < I.nseg; ++b) {
                if (b > first && boundary_ok(b)) continue;
                run_chain_direct<T, K, FL, FWD>(P, A, make_ctx(P, inst, b), RUN_EXACT,
                                                snap_ptr<T>(P, I.seg0 + b - 1, 1));
                ++fixes;
            }
        } else {
            for (int b = first; b >= 1; --b) {
                if (b < first && boundary_ok(b)) continue;
                run_chain_direct<T, K, FL, FWD>(P, A, make_ctx(P, inst, b - 1), RUN_EXACT,
                                                snap_ptr<T>(P, I.seg0 + b, 1));
                ++fixes;
            }
        }
    }
    __syncwarp();
    if constexpr (FWD && (FL & F_CHOL)) {
        double ld = 0.0;
        int bad = I.nseg;                  // first segment with a failed pivot
        for (int p = lane; p < I.nseg; p += kWarp) {
            ld += P.seg_logdet[I.seg0 + p];
            if (P.seg_info[I.seg0 + p] != 0) bad = min(bad, p);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ld += __shfl_xor_sync(0xffffffffu, ld, o);
            bad = min(bad, __shfl_xor_sync(0xffffffffu, bad, o));
        }
        if (lane == 0) {
            const int32_t info = bad < I.nseg ? P.seg_info[I.seg0 + bad] : 0;
            if (A.logdet) A.logdet[inst] = info ? (double)NAN : ld;
            A.info[inst] = info;
        }
    }
    if (lane == 0 && fixes) atomicAdd(P.counters + kNumSweepKinds + A.kind, fixes);
}

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
inline bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

template <typename T>
inline bool args_aligned16(const SweepArgs<T> &A) {
    return aligned16(A.Q) && aligned16(A.L) && aligned16(A.Lin) && aligned16(A.S) && aligned16(A.Sbar) &&
           aligned16(A.Sout) && aligned16(A.Lbar) && aligned16(A.Lbar_in) && aligned16(A.Qbar) &&
           aligned16(A.Bin) && aligned16(A.Xout) && aligned16(A.Xin) && aligned16(A.Ybar);
}

template <typename T, int K, int FL, bool FWD>
static cudaError_t launch_direct(const bnd_plan *p, const SweepArgs<T> &A, int32_t t0, int32_t nt, cudaStream_t s) {
    if (nt <= 0) return cudaSuccess;
    static PerDeviceSlots occ, sms;
    const int blocks_per_sm = per_device(occ, [] {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<T, K, FL, FWD>, 128, 0);
        return b > 0 ? b : 1;
    });
    const int num_sms = per_device(sms, [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v;
    });
    const int bps = p->blocks_per_sm > 0 ? p->blocks_per_sm : blocks_per_sm;
    int64_t blocks = (int64_t)num_sms * bps;
    const int64_t need = (nt + 3) / 4;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaMemsetAsync(p->dev.counters + A.kind, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    sweep_kernel<T, K, FL, FWD><<<(unsigned)blocks, 128, 0, s>>>(p->dev, A, t0, nt);
    return cudaGetLastError();
}

template <typename T, int K, int FL, bool FWD>
static cudaError_t launch_sweep_t(const bnd_plan *p, const SweepArgs<T> &A, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const bool staged = p->layout != kLayoutStrided && p->staged_ok && args_aligned16(A) && !p->force_direct;
    if (!staged) {
        // the block kernels need no alignment beyond the element size: they keep the generic
        // class (segmented or not) whenever their windows fit
        const int32_t nwide = p->class_task0[1] - p->class_task0[0];
        if (p->wide_cta && nwide > 0) {
            e = launch_wide<T, K, FL, FWD>(p, A, p->class_task0[0], nwide, s);
            if (e == cudaSuccess) e = launch_direct<T, K, FL, FWD>(p, A, p->class_task0[1], p->ntasks - p->class_task0[1], s);
        } else {
            e = launch_direct<T, K, FL, FWD>(p, A, 0, p->ntasks, s);
        }
    } else {
        // fork: one side stream per bandwidth class, each waiting on the main stream
        e = cudaEventRecord(p->ev_fork, s);
        for (int c = 0; c <= kRegMaxL && e == cudaSuccess; ++c) {
            if (p->class_task0[c + 1] - p->class_task0[c] <= 0) continue;
            cudaStream_t side = p->side[c];
            e = cudaStreamWaitEvent(side, p->ev_fork, 0);
            if (e != cudaSuccess) break;
            switch (c) {
                case 0: e = launch_wide<T, K, FL, FWD>(p, A, p->class_task0[0], p->class_task0[1] - p->class_task0[0], side); break;
                case 1: e = launch_staged_l<T, 1, K, FL, FWD>(p, A, side); break;
                case 2: e = launch_staged_l<T, 2, K, FL, FWD>(p, A, side); break;
                case 3: e = launch_staged_l<T, 3, K, FL, FWD>(p, A, side); break;
                case 4: e = launch_staged_l<T, 4, K, FL, FWD>(p, A, side); break;
                case 5: e = launch_staged_l<T, 5, K, FL, FWD>(p, A, side); break;
                case 6: e = launch_staged_l<T, 6, K, FL, FWD>(p, A, side); break;
                case 7: e = launch_staged_l<T, 7, K, FL, FWD>(p, A, side); break;
                case 8: e = launch_staged_l<T, 8, K, FL, FWD>(p, A, side); break;
            }
            if (e == cudaSuccess) e = cudaEventRecord(p->ev_join[c], side);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join[c], 0);
        }
    }
    if (e != cudaSuccess) return e;
    if (p->nsegs > p->count) {
        verify_kernel<T, K, FL, FWD><<<(p->count + kVerifyWarps - 1) / kVerifyWarps, kWarp * kVerifyWarps, 0, s>>>(
            p->dev, A);
        e = cudaGetLastError();
    }
    return e;
}

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
