// Stream I/O of the register-window sweeps.
//
// A sweep reads a fixed set of input streams and writes a fixed set of
// output streams.  A stream is one contiguous row of a pool (a diagonal d of
// a band operand, B'[d][*], or one right-hand-side column) read at column
// j + off at iteration j.  Two implementations:
//
//  DirectIO : plain global loads / stores by the calling thread (used by the
//             verify/fixup pass, which runs one chain per thread).
//  StagedIO : per-lane shared-memory rings.  Each lane prefetches its own
//             chain's streams D columns ahead with 16-byte cp.async copies
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
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;   // src-size 0: zero fill, nothing is read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(n) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src, bool valid) {
    const int n = valid ? BYTES : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Pool pointers of one chain (instance offsets applied).
// ---------------------------------------------------------------------------
template <typename T>
struct ChainPtrs {
    const T *in[7];
    T *out[5];
    int64_t ld, ldr, n, rhs0;
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
    __device__ void begin_tiles(int64_t, int64_t, int64_t) {}
    __device__ __forceinline__ void tile_begin(int64_t) {}
    __device__ __forceinline__ void tile_end(int64_t, bool) {}
    __device__ __forceinline__ T in(int S, int64_t j, int) const {
        const StreamSpec s = SW::in_spec(S);
        const int64_t c = j + s.off;
        if (c < 0 || c >= P.n || !P.active(s)) return T(0);
        return P.in_row(s)[c];
    }
    __device__ __forceinline__ void out(int O, int64_t j, int, T v) {
        const StreamSpec s = SW::out_spec(O);
        if (!P.active(s)) return;
        T *p = P.out_row(s) + j;
        const bool corner = !is_rhs_pool(s.pool) && (j + s.row >= P.n);
        *p = corner ? T(0) : (P.acc ? (*p + v) : v);
    }
    __device__ void finish() {}
};

// ---------------------------------------------------------------------------
// StagedIO
// ---------------------------------------------------------------------------
template <typename T, class SW, int R>
struct StagedIO {
    static constexpr int NIN = SW::NIN;
    static constexpr int NOUT = SW::NOUT;
    static constexpr int TW = 16 / (int)sizeof(T);     // columns per tile (one 16-byte chunk)
    static constexpr int kRingElems = NIN * R * kWarp * TW;
    static constexpr int kOutElems = (NOUT > 0 ? NOUT : 1) * kWarp * TW;
    static constexpr int kWarpElems = kRingElems + kOutElems;

    const ChainPtrs<T> &P;
    T *ring;        // this lane's ring: element (s, slot, u) at ring[((s R + slot) 32) TW + u]
    T *outb;        // this lane's out tile: element (o, u) at outb[o 32 TW + u]
    int dir;        // +1 forward, -1 backward
    int64_t a, b;   // output columns [a, b)
    int slot;       // ring slot of the current tile
    T *cur;         // ring + slot offset of the current tile

    __device__ StagedIO(const ChainPtrs<T> &p, T *warp_smem, int lane, int dir_)
        : P(p), ring(warp_smem + lane * TW), outb(warp_smem + kRingElems + lane * TW), dir(dir_) {}

    // Copy the tile of stream S that holds the values of iterations [m TW, m TW + TW) into slot q:
    // columns m TW + off .. +TW-1.  Streams whose offset is a multiple of TW move as one 16-byte
    // chunk; the others element by element.  Columns outside [0, n) are zero filled, not read.
    __device__ __forceinline__ void issue(int S, int64_t m, int q) {
        const StreamSpec s = SW::in_spec(S);
        T *dst = ring + (S * R + q) * kWarp * TW;
        const int64_t c0 = m * TW + s.off;
        const T *row = P.in_row(s);
        const bool act = P.active(s);
        if ((s.off % TW) == 0) {
            const bool valid = act && c0 >= 0 && c0 < P.n;
            cp_async16(dst, valid ? row + c0 : P.in[s.pool], valid);
        } else {
#pragma unroll
            for (int u = 0; u < TW; ++u) {
                const int64_t c = c0 + u;
                const bool valid = act && c >= 0 && c < P.n;
                cp_async_small<sizeof(T)>(dst + u, valid ? row + c : P.in[s.pool], valid);
            }
        }
    }

    __device__ __forceinline__ int slot_of(int64_t m) const { return (int)(((m % R) + R) % R); }

    // Chain start: tiles m0, m0 + dir, ..., m0 + dir (R-2) are issued (one commit group each).
    __device__ void begin_tiles(int64_t m0, int64_t a_, int64_t b_) {
        a = a_;
        b = b_;
        for (int t = 0; t < R - 1; ++t) {
            const int64_t m = m0 + dir * t;
#pragma unroll
            for (int S = 0; S < NIN; ++S) issue(S, m, slot_of(m));
            cp_async_commit();
        }
    }

    // Tile m: issue tile m + dir (R-1), then wait until tile m has landed.
    __device__ __forceinline__ void tile_begin(int64_t m) {
        const int64_t mn = m + dir * (R - 1);
        const int qn = slot_of(mn);
#pragma unroll
        for (int S = 0; S < NIN; ++S) issue(S, mn, qn);
        cp_async_commit();
        cp_async_wait<R - 1>();
        slot = slot_of(m);
        cur = ring + slot * kWarp * TW;
    }

    // Value of stream S at iteration j, position u = j mod TW inside the current tile.
    __device__ __forceinline__ T in(int S, int64_t, int u) const { return cur[S * R * kWarp * TW + u]; }

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

}  // namespace bnd
