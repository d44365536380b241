// Stream I/O of the register-window sweeps.
//
// A sweep reads a fixed set of input streams and writes a fixed set of
// output streams.  A stream is one row of a pool (a diagonal d of a band
// operand, B'[d][*], or one right-hand-side column) read at column j + off at
// iteration j; consecutive columns are cs elements apart (1 for row plans,
// 32 for panel plans).  Three implementations:
//
//  DirectIO : plain global loads / stores by the calling thread (used by the
//             verify/fixup pass, which runs one chain per thread, and by the
//             direct kernels of unaligned or general-stride batches).
//  PanelIO  : panel plans; the warp's lanes are the 32 lanes of one instance
//             group, so the warp stages each tile of a stream as one
//             contiguous block (defined below).
//  StagedIO : row plans; per-lane shared-memory rings.  Each lane prefetches its own
//             chain's streams R tiles ahead with 16-byte cp.async copies
//             (one 16-byte tile = TW columns), waits with per-iteration commit
//             groups, and collects outputs in a tile buffer written back with
//             one 16-byte vector store per stream when a tile is complete, or
//             with scalar stores at ragged edges and in accumulate mode.
//             (Per-lane TMA bulk stores were tried: with 32 different
//             addresses per warp they are issued lane by lane, which cost
//             more than the stores themselves.)  Lanes only touch their own
//             slices, so no cross-lane synchronisation is needed.
#pragma once

#include "common.cuh"

namespace bnd {

// Source / destination pools of a stream.
enum : int { POOL_Q = 0, POOL_LIN, POOL_S, POOL_SBAR, POOL_LBARIN, POOL_BIN, POOL_XIN,   // inputs
             POOL_LOUT = 16, POOL_LBAR, POOL_SOUT, POOL_QBAR, POOL_XOUT };             // outputs

struct StreamSpec {
    int pool;      // POOL_*
    int row;       // diagonal d (band pools) or RHS column offset r (RHS pools)
    int off;       // column offset relative to the iteration column
};

__host__ __device__ constexpr bool is_rhs_pool(int p) { return p == POOL_BIN || p == POOL_XIN || p == POOL_XOUT; }

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Optional L2 prefetch size of the streaming copies (128 or 256 bytes per
// request).  Off by default: with thousands of streams in flight the extra
// lines crowd L2 and measured no faster.
#ifndef BND_L2_PREFETCH
#define BND_L2_PREFETCH 0
#endif
#if BND_L2_PREFETCH == 256
#define BND_L2_HINT ".L2::256B"
#elif BND_L2_PREFETCH == 128
#define BND_L2_HINT ".L2::128B"
#else
#define BND_L2_HINT ""
#endif
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;   // src-size 0: zero fill, nothing is read
    asm volatile("cp.async.cg.shared.global" BND_L2_HINT " [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Shared-memory barriers and bulk copies (the bulk-copy panel I/O, a build
// option): one thread arms a barrier with the bytes it expects and issues
// whole-block copies from global memory that complete on it; readers wait for
// the barrier's phase with a bounded number of polls.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// 16-byte aligned source and destination, size a multiple of 16 bytes; completes on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// Polls of a barrier wait before it gives up (counted in the plan's timeout counter).
constexpr uint32_t kBulkSpinLimit = 1u << 24;

template <typename T> struct SweepArgs;

// ---------------------------------------------------------------------------
// Pool pointers of one chain (instance offsets applied).
// ---------------------------------------------------------------------------
template <typename T>
struct ChainPtrs {
    const T *in[7];
    T *out[5];
    int64_t ld, ldr, n, rhs0;
    int64_t cs;     // column stride (1: contiguous rows; 32: panel lanes)
    int acc;
    int kk;         // active RHS columns of this launch

    __device__ bool active(const StreamSpec &s) const { return !is_rhs_pool(s.pool) || s.row < kk; }

    __device__ const T *in_row(const StreamSpec &s) const {
        const int64_t stride = is_rhs_pool(s.pool) ? ldr : ld;
        const int64_t row = is_rhs_pool(s.pool) ? (rhs0 + s.row) : s.row;
        return in[s.pool] + row * stride;
    }
    __device__ T *out_row(const StreamSpec &s) const {
        const int64_t stride = is_rhs_pool(s.pool) ? ldr : ld;
        const int64_t row = is_rhs_pool(s.pool) ? (rhs0 + s.row) : s.row;
        return out[s.pool - POOL_LOUT] + row * stride;
    }
};

// ---------------------------------------------------------------------------
// DirectIO
// ---------------------------------------------------------------------------
template <typename T, class SW>
struct DirectIO {
    const ChainPtrs<T> &P;
    __device__ DirectIO(const ChainPtrs<T> &p) : P(p) {}
    static constexpr int TW = 1;
    static constexpr bool kWarpUniform = false;
    __device__ void begin_tiles(int64_t, int64_t, int64_t) {}
    __device__ __forceinline__ void tile_begin(int64_t) {}
    __device__ __forceinline__ void tile_end(int64_t, bool) {}
    __device__ __forceinline__ T in(int S, int64_t j, int) const {
        const StreamSpec s = SW::in_spec(S);
        const int64_t c = j + s.off;
        if (c < 0 || c >= P.n || !P.active(s)) return T(0);
        return P.in_row(s)[c * P.cs];
    }
    template <bool CHECK>
    __device__ __forceinline__ void out(int O, int64_t j, int, T v) {
        const StreamSpec s = SW::out_spec(O);
        if (!P.active(s)) return;
        T *p = P.out_row(s) + j * P.cs;
        const bool corner = !is_rhs_pool(s.pool) && (j + s.row >= P.n);
        *p = corner ? T(0) : (P.acc ? (*p + v) : v);
    }
    __device__ void finish() {}
};

// ---------------------------------------------------------------------------
// StagedIO
//
// Ring layout (per warp): stream S owns depth(S) slots of 32 lanes x TW
// columns; element (S, slot q, lane, u) sits at base(S) + (q 32 + lane) TW + u.
// Slots are keyed by the ROW tile (iteration tile) they serve, modulo the
// stream's depth.  An aligned stream (offset a multiple of TW) needs one data
// tile per row tile.  A lagged stream (any other offset) needs two aligned data
// tiles per row tile, m + fo and m + fo + 1 (fo = floor(off / TW)); the row
// tile m "owns" the one that is new in the sweep direction and borrows the
// other from the previous row tile, so lagged streams keep R + 1 slots and
// every copy is one aligned 16-byte chunk.
// ---------------------------------------------------------------------------
template <typename T, class SW, int R, int DIR>
struct StagedIO {
    static constexpr int NIN = SW::NIN;
    static constexpr int NOUT = SW::NOUT;
    static constexpr int TW = 16 / (int)sizeof(T);     // columns per tile (one 16-byte chunk)
    static constexpr int RL = R + 1;                    // slots of a lagged stream
    static constexpr bool kWarpUniform = false;

    __host__ __device__ static constexpr int off_of(int S) { return SW::in_spec(S).off; }
    __host__ __device__ static constexpr bool lagged(int S) { return (off_of(S) % TW) != 0; }
    __host__ __device__ static constexpr int depth(int S) { return lagged(S) ? RL : R; }
    __host__ __device__ static constexpr int fo_of(int S) {      // floor(off / TW)
        return off_of(S) >= 0 ? off_of(S) / TW : -((-off_of(S) + TW - 1) / TW);
    }
    __host__ __device__ static constexpr int rem_of(int S) { return off_of(S) - fo_of(S) * TW; }
    __host__ __device__ static constexpr int base(int S) {
        int b = 0;
        for (int x = 0; x < S; ++x) b += depth(x) * kWarp * TW;
        return b;
    }
    static constexpr int kRingElems = base(NIN);
    static constexpr int kOutElems = (NOUT > 0 ? NOUT : 1) * kWarp * TW;
    static constexpr int kWarpElems = kRingElems + kOutElems;

    const ChainPtrs<T> &P;
    T *ring;        // this lane's ring (lane offset applied)
    T *outb;        // this lane's out tile: element (o, u) at outb[o 32 TW + u]
    int64_t a, b;   // output columns [a, b)
    // slots (mod R, mod R + 1) of the current row tile and of the next row tile to issue
    int cR, cL, iR, iL;
    const T *curR, *curLo, *curHi;   // current aligned slot; lagged low / high data tiles

    __device__ StagedIO(const ChainPtrs<T> &p, T *warp_smem, int lane)
        : P(p), ring(warp_smem + lane * TW), outb(warp_smem + kRingElems + lane * TW) {}

    __device__ static __forceinline__ int wrap_add(int x, int d, int mod) {
        x += d;
        return x >= mod ? x - mod : (x < 0 ? x + mod : x);
    }

    // Copy into slot q the data tile that stream S needs for row tile m (for a
    // lagged stream: the tile row tile m owns).  Columns outside [0, n) are
    // zero filled, not read; a chunk that starts inside [0, n) is copied whole
    // (the tail past n lies in the row padding, ld >= n rounded up to TW, and
    // the sweeps mask those columns).
    __device__ __forceinline__ void issue(int S, int64_t m, int q) {
        const StreamSpec s = SW::in_spec(S);
        const int64_t c0 = lagged(S) ? (m + fo_of(S) + (DIR > 0 ? 1 : 0)) * TW : m * TW + s.off;
        T *dst = ring + base(S) + q * kWarp * TW;
        const bool valid = P.active(s) && c0 >= 0 && c0 < P.n;
        cp_async16(dst, valid ? P.in_row(s) + c0 : P.in[s.pool], valid);
    }
    __device__ __forceinline__ void issue_all(int64_t m, int qR, int qL) {
#pragma unroll
        for (int S = 0; S < NIN; ++S) issue(S, m, lagged(S) ? qL : qR);
    }

    // Chain start: row tiles m0, m0 + DIR, ..., m0 + DIR (R-2) are issued (one
    // commit group each); the first group also holds the lagged streams' tiles
    // owned by row tile m0 - DIR.
    __device__ void begin_tiles(int64_t m0, int64_t a_, int64_t b_) {
        a = a_;
        b = b_;
        cR = (int)(((m0 % R) + R) % R);
        cL = (int)(((m0 % RL) + RL) % RL);
        const int pL = wrap_add(cL, -DIR, RL);
#pragma unroll
        for (int S = 0; S < NIN; ++S)
            if (lagged(S)) issue(S, m0 - DIR, pL);
        iR = cR;
        iL = cL;
        for (int t = 0; t < R - 1; ++t) {
            issue_all(m0 + DIR * t, iR, iL);
            cp_async_commit();
            iR = wrap_add(iR, DIR, R);
            iL = wrap_add(iL, DIR, RL);
        }
    }

    // Row tile m (= m0 + DIR t for the t-th call): issue row tile m + DIR (R-1),
    // then wait until row tile m has landed.
    __device__ __forceinline__ void tile_begin(int64_t m) {
        issue_all(m + DIR * (R - 1), iR, iL);
        cp_async_commit();
        iR = wrap_add(iR, DIR, R);
        iL = wrap_add(iL, DIR, RL);
        cp_async_wait<R - 1>();
        curR = ring + cR * kWarp * TW;
        const T *own = ring + cL * kWarp * TW;
        const T *prev = ring + wrap_add(cL, -DIR, RL) * kWarp * TW;
        curLo = DIR > 0 ? prev : own;
        curHi = DIR > 0 ? own : prev;
        cR = wrap_add(cR, DIR, R);
        cL = wrap_add(cL, DIR, RL);
    }

    // Value of stream S at iteration j, position u = j mod TW inside the current tile.
    __device__ __forceinline__ T in(int S, int64_t, int u) const {
        if (lagged(S)) {
            const int p = u + rem_of(S);
            return p < TW ? curLo[base(S) + p] : curHi[base(S) + p - TW];
        }
        return curR[base(S) + u];
    }

    template <bool CHECK>
    __device__ __forceinline__ void out(int O, int64_t, int u, T v) { outb[O * kWarp * TW + u] = v; }

    // Write the out tile of tile m (columns [m TW, m TW + TW) intersected with [a, b) and [0, n)):
    // a full tile goes out as one 16-byte vector store per stream, a ragged one element-wise.
    __device__ void tile_end(int64_t m, bool has_out) {
        if (!has_out) return;
        const int64_t g0 = m * TW;
        const bool full = !P.acc && g0 >= a && g0 + TW <= b && g0 + TW <= P.n;
#pragma unroll
        for (int O = 0; O < NOUT; ++O) {
            const StreamSpec s = SW::out_spec(O);
            if (!P.active(s)) continue;
            T *dst = P.out_row(s) + g0;
            const T *src = outb + O * kWarp * TW;
            if (full) {
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
            } else {
                for (int u = 0; u < TW; ++u) {
                    const int64_t c = g0 + u;
                    if (c < a || c >= b || c >= P.n) continue;
                    const bool corner = !is_rhs_pool(s.pool) && (c + s.row >= P.n);
                    dst[u] = corner ? T(0) : (P.acc ? (dst[u] + src[u]) : src[u]);
                }
            }
        }
    }

    __device__ void finish() { cp_async_wait<0>(); }
};

// ---------------------------------------------------------------------------
// PanelIO (panel plans: 32 instances interleaved per column, cs = 32)
//
// The warp's lanes are lanes 0..31 of one instance group at the same segment,
// so column c of a stream row is 32 adjacent elements and TW consecutive
// columns are one contiguous block of TW * 32 elements.  Inputs go through a
// per-warp ring [stream][slot][u][lane]: the warp copies each block with
// 16-byte cp.async, every lane a 16-byte piece, whatever the stream's column
// offset (a row shift of whole 32-element columns), and each lane reads its
// own column u with a bank-conflict-free shared load.  Outputs need no
// staging: every lane stores its element of column j, and the warp's stores
// of one column form one contiguous run.  The loop over tiles is uniform over
// the warp (the copies are cooperative); lanes outside their own rows skip
// the steps.
// ---------------------------------------------------------------------------
template <typename T, class SW, int R, int DIR, bool BULK = false>
struct PanelIO {
    static constexpr int NIN = SW::NIN;
    static constexpr int NOUT = SW::NOUT;
    static constexpr int TW = 4;                                     // columns per tile
    static constexpr int kTileElems = TW * kWarp;
    static constexpr int kPieces = kTileElems * (int)sizeof(T) / (16 * kWarp);   // 16-byte pieces per lane
    static constexpr int kPieceElems = 16 / (int)sizeof(T);
    static constexpr int kRingElems = NIN * R * kTileElems;
    // BULK: one shared-memory barrier per ring slot after the ring
    static constexpr int kBarElems = BULK ? (R * 8 + (int)sizeof(T) - 1) / (int)sizeof(T) : 0;
    static constexpr int kWarpElems = kRingElems + kBarElems;
    static constexpr bool kWarpUniform = true;
    static_assert(kPieces >= 1, "a tile must give every lane at least one 16-byte piece");

    // column offsets of the input streams (a tile of every stream is inside
    // [0, gn) when m TW + kMinOff >= 0 and m TW + TW + kMaxOff <= gn)
    __host__ __device__ static constexpr int min_off() {
        int v = 0;
        for (int S = 0; S < NIN; ++S) v = SW::in_spec(S).off < v ? SW::in_spec(S).off : v;
        return v;
    }
    __host__ __device__ static constexpr int max_off() {
        int v = 0;
        for (int S = 0; S < NIN; ++S) v = SW::in_spec(S).off > v ? SW::in_spec(S).off : v;
        return v;
    }

    // Offsets inside a group's region fit in 32 bits (the plan checks
    // (l + 1) ld and k ldr against 2^31), so every address below is a 64-bit
    // pool base plus a 32-bit element offset.
    const T *gin[7];                // per input pool: base of lane 0's row 0 (RHS: of column rhs0)
    T *gout[5];                     // per output pool: base of this lane's row 0 (RHS: column rhs0)
    int32_t gld, gldr;              // row strides of the group (elements)
    int64_t gn;                     // rows present in the group
    int32_t kk;                     // active RHS columns of the launch
    int32_t acc;
    int64_t n;                      // this lane's order (corner test of the checked stores)
    T *ring;                        // the warp's ring
    int lane;
    int cR, iR;                     // ring slots of the current row tile and of the next one to issue
    const T *cur;                   // this lane's column in the current slot
    uint64_t *bars;                 // BULK: barrier of each slot
    uint32_t par;                   // BULK: parity of the next phase to wait for, bit q for slot q
    uint32_t *err;                  // BULK: count of waits that gave up
    bool bulk_ok;                   // BULK: every input stream active (whole blocks can be copied)

    __device__ PanelIO(const ChainPtrs<T> &p, const SweepArgs<T> &A, const Task &g, T *warp_smem, int lane_,
                       uint32_t *err_ = nullptr)
        : ring(warp_smem), lane(lane_), bars(reinterpret_cast<uint64_t *>(warp_smem + kRingElems)), par(0),
          err(err_) {
        gld = (int32_t)g.gld;
        gldr = (int32_t)g.gldr;
        gn = g.gn;
        kk = p.kk;
        acc = p.acc;
        n = p.n;
        const int64_t r0 = (int64_t)p.rhs0 * g.gldr;
        gin[POOL_Q] = A.Q + g.gband;
        gin[POOL_LIN] = A.Lin + g.gband;
        gin[POOL_S] = A.S + g.gband;
        gin[POOL_SBAR] = A.Sbar + g.gband;
        gin[POOL_LBARIN] = A.Lbar_in + g.gband;
        gin[POOL_BIN] = A.Bin + g.grhs + r0;
        gin[POOL_XIN] = A.Xin + g.grhs + r0;
        gout[POOL_LOUT - POOL_LOUT] = A.L + g.gband + lane;
        gout[POOL_LBAR - POOL_LOUT] = A.Lbar + g.gband + lane;
        gout[POOL_SOUT - POOL_LOUT] = A.Sout + g.gband + lane;
        gout[POOL_QBAR - POOL_LOUT] = A.Qbar + g.gband + lane;
        gout[POOL_XOUT - POOL_LOUT] = A.Xout + g.grhs + r0 + lane;
        bulk_ok = true;
#pragma unroll
        for (int S = 0; S < NIN; ++S) bulk_ok = bulk_ok && active(SW::in_spec(S));
    }

    __device__ static __forceinline__ int wrap_add(int x, int d) {
        x += d;
        return x >= R ? x - R : (x < 0 ? x + R : x);
    }
    __device__ __forceinline__ int32_t row_off(const StreamSpec &s) const {
        return s.row * (is_rhs_pool(s.pool) ? gldr : gld);
    }
    __device__ __forceinline__ bool active(const StreamSpec &s) const { return !is_rhs_pool(s.pool) || s.row < kk; }

    // Copy into slot q the block of stream S for row tile m: columns
    // m TW + off .. + TW - 1 of all 32 lanes.  Columns outside [0, gn) are
    // zero filled, not read (ALL: the caller knows every column is inside).
    template <bool ALL>
    __device__ __forceinline__ void issue(int S, int64_t m, int q) {
        const StreamSpec s = SW::in_spec(S);
        const int64_t c0 = m * TW + s.off;
        const bool act = active(s);
        const T *base = gin[s.pool];
        T *dst = ring + (S * R + q) * kTileElems;
#pragma unroll
        for (int t = 0; t < kPieces; ++t) {
            const int e = (lane + kWarp * t) * kPieceElems;        // element offset inside the block
            bool valid = act;
            if (!ALL) {
                const int64_t c = c0 + e / kWarp;
                valid = valid && c >= 0 && c < gn;
            }
            // an invalid piece reads nothing (source size 0): the address is only a placeholder
            const int32_t o = valid ? row_off(s) + (int32_t)c0 * kWarp + e : 0;
            cp_async16(dst + e, base + o, valid);
        }
    }
    template <bool ALL>
    __device__ __forceinline__ void issue_all(int64_t m, int q) {
#pragma unroll
        for (int S = 0; S < NIN; ++S) issue<ALL>(S, m, q);
    }
    __device__ __forceinline__ void issue_tile(int64_t m, int q) {
        const bool inside = m * TW + min_off() >= 0 && m * TW + TW + max_off() <= gn;
        if constexpr (BULK) {
            if (inside && bulk_ok) {
                // one thread arms the slot's barrier and copies every stream's block whole
                if (lane == 0) {
                    fence_proxy_async_smem();        // the lanes' earlier reads of the slot come first
                    mbar_arrive_expect_tx(bars + q, (uint32_t)(NIN * kTileElems * sizeof(T)));
#pragma unroll
                    for (int S = 0; S < NIN; ++S) {
                        const StreamSpec s = SW::in_spec(S);
                        const int64_t c0 = m * TW + s.off;
                        bulk_g2s(ring + (S * R + q) * kTileElems, gin[s.pool] + row_off(s) + (int32_t)c0 * kWarp,
                                 (uint32_t)(kTileElems * sizeof(T)), bars + q);
                    }
                }
                return;
            }
            // edge tiles (zero fill) and partially active launches: the pieces, and a plain
            // arrival so that the slot's barrier phase completes
            if (inside) issue_all<true>(m, q);
            else issue_all<false>(m, q);
            if (lane == 0) mbar_arrive(bars + q);
            return;
        }
        if (inside) issue_all<true>(m, q);
        else issue_all<false>(m, q);
    }
    // BULK: wait for the next phase of slot q (bounded; a wait that gives up is counted)
    __device__ __forceinline__ void wait_slot(int q) {
        const uint32_t ph = (par >> q) & 1u;
        uint32_t spins = 0;
        while (!mbar_test_wait(bars + q, ph)) {
            if (++spins >= kBulkSpinLimit) {
                if (lane == 0 && err) atomicAdd(err, 1u);
                break;
            }
        }
        par ^= 1u << q;
    }

    __device__ void begin_tiles(int64_t m0, int64_t, int64_t) {
        cR = (int)(((m0 % R) + R) % R);
        iR = cR;
        if constexpr (BULK) {
            if (lane == 0) {
                for (int q = 0; q < R; ++q) mbar_init(bars + q, 1);
                mbar_init_fence();
            }
            __syncwarp();
        }
        for (int t = 0; t < R - 1; ++t) {
            issue_tile(m0 + DIR * t, iR);
            cp_async_commit();
            iR = wrap_add(iR, DIR);
        }
    }

    __device__ __forceinline__ void tile_begin(int64_t m) {
        __syncwarp();                      // every lane is done with the slot about to be refilled
        issue_tile(m + DIR * (R - 1), iR);
        cp_async_commit();
        iR = wrap_add(iR, DIR);
        cp_async_wait<R - 1>();
        if constexpr (BULK) wait_slot(cR);   // the whole-block copies of tile m have landed
        __syncwarp();                      // the other lanes' pieces of tile m have landed
        cur = ring + cR * kTileElems + lane;
        cR = wrap_add(cR, DIR);
    }

    __device__ __forceinline__ T in(int S, int64_t, int u) const { return cur[S * R * kTileElems + u * kWarp]; }

    // Every lane stores its own element; the warp's stores of one column are
    // one contiguous run of 32 elements.  Interior tiles (CHECK false) of a
    // launch that does not accumulate store plainly: the sweep guarantees the
    // element is inside the matrix there.  (Staging the tile in shared memory
    // for 16-byte block stores measured slower: the extra shared memory cost
    // more resident warps than the wider stores gained.)
    template <bool CHECK>
    __device__ __forceinline__ void out(int O, int64_t j, int, T v) {
        const StreamSpec s = SW::out_spec(O);
        if (!active(s)) return;
        T *p = gout[s.pool - POOL_LOUT] + (row_off(s) + (int32_t)j * kWarp);
        if (!CHECK && !acc) {
            *p = v;
            return;
        }
        const bool corner = !is_rhs_pool(s.pool) && (j + s.row >= n);
        *p = corner ? T(0) : (acc ? (*p + v) : v);
    }

    __device__ __forceinline__ void tile_end(int64_t, bool) {}
    __device__ void finish() {
        cp_async_wait<0>();
        if constexpr (BULK) {
            // the R - 1 tiles issued ahead of the last one are still owed to their barriers:
            // wait for them, so that no copy is left in flight into this block's shared memory
            int q = cR;
            for (int t = 0; t < R - 1; ++t) {
                wait_slot(q);
                q = wrap_add(q, DIR);
            }
            __syncwarp();
        }
    }
};

}  // namespace bnd
