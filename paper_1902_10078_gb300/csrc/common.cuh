// Shared definitions of the banded-operator CUDA library (device and host).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/banded.h"

namespace bnd {

constexpr int kWarp = 32;
constexpr int kRegMaxL = 8;        // bandwidths 1..kRegMaxL run the register-window kernels
constexpr int kMaxK = 4;           // right-hand sides per register-window sweep

// One chain: the rows [a, b) of one instance, run by one lane.  The lane
// starts its recurrence `warm` rows before a (forward sweeps) or after b
// (backward sweeps) from a cold state; only rows in [a, b) are written.
struct Chain {
    int32_t inst;      // instance index, -1 for an idle padding lane
    int32_t seg;       // segment index within the instance (0 = first row block)
    int64_t a, b;      // output rows [a, b)
};

// Per-instance data uploaded to the workspace.
struct InstDev {
    int64_t n, band, ld, rhs, ldr;
    int64_t cs;        // column stride of the band and RHS block (1: contiguous rows)
    int32_t l;
    int32_t nseg;      // number of row segments
    int64_t seg0;      // global id of the instance's first segment (ids are consecutive)
    int64_t seg_len;   // rows per segment (the last one may be shorter)
    int64_t warm;      // warm-up rows of a speculative segment start
};

// A warp task: 32 consecutive entries of the chain table (all the same l).
// In a panel plan, chain p of a task is lane p of one instance group, all at
// the same segment, and the task carries the group's panel geometry.
struct Task {
    int32_t chain0;    // first chain index
    int32_t l;         // bandwidth shared by the task's chains
    int64_t gband;     // panel plans: band offset of lane 0 of the group
    int64_t grhs;      // panel plans: RHS offset of lane 0 of the group
    int64_t gld, gldr; // panel plans: row strides of the group
    int64_t gn;        // panel plans: rows present in the group (its largest n)
};

// Arrangements of a batch in its pools.
enum : int32_t { kLayoutRows = 0, kLayoutPanels = 1, kLayoutStrided = 2 };
constexpr int kPanelLanes = 32;    // column stride of a panel group

// Sweep kinds (for state snapshots and fixup counters).
enum SweepKind : int32_t { kSweepChol = 0, kSweepTaka = 1, kSweepTakaBar = 2, kSweepCholBar = 3,
                           kSweepFSolve = 4, kSweepBSolve = 5, kNumSweepKinds = 6 };
// Plan counters: task queue heads [0, kinds), fixup counts [kinds, 2 kinds),
// then the count of bounded device waits that gave up (must stay 0).
constexpr int kTimeoutCounter = 2 * kNumSweepKinds;
constexpr int kNumCounters = 2 * kNumSweepKinds + 1;

// Device view of a bound plan.
struct PlanDev {
    const InstDev *inst;
    const Chain *chains;
    const Task *tasks;
    const int64_t *tile_prefix;  // products: prefix of 256-column tiles per instance (rows plans) or of
                                 // 8-column tiles per panel group (panel plans: 32 lanes x 8 columns)
    int64_t ntiles;
    const int32_t *group_first;  // panel plans: first instance of each group (ngroups + 1 entries)
    int32_t ngroups;             // 0 for rows / strided plans
    int32_t ntasks;
    int32_t count;
    int64_t nchains;
    int32_t k;
    int32_t warm;
    // workspace areas
    int64_t nsegs;
    uint32_t *counters;      // [kNumCounters]: task queue heads, fixup counters, wait timeouts
    void *snap;              // per segment: 2 snapshots (start, end) of snap_words elements
    int64_t snap_words;
    double *seg_logdet;      // per segment partial log-det
    int32_t *seg_info;       // per segment first failing row + 1 (0 = none)
    void *rhs_tmp;           // RHS-shaped scratch pool
    void *rhs_tmp2;          // second RHS-shaped scratch pool
    void *band_tmp;          // band-shaped scratch pool (fused backward intermediate)
    void *band_tmp2;         // band-shaped scratch pools of the generic (wide band) path
    void *band_tmp3;
    // staged reruns of segments whose speculative start state was wrong
    const int32_t *seg_chain;  // per global segment: index of the chain that runs it
    uint32_t *rerun_cnt;       // per bandwidth class: tasks queued for a rerun
    int32_t *rerun_list;       // task ids, class c's queue at [class_task0[c], class_task0[c+1])
    uint32_t *task_flag;       // per task: queued (1) or not (0)
    uint8_t *chain_flag;       // per chain: rerun this lane (1) or not (0)
};

__host__ __device__ inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// Size in elements of the per-chain state snapshot for bandwidth l and k RHS.
__host__ __device__ inline int64_t snap_words_for(int l, int k) {
    // the largest sweep state: Schur window l(l+1)/2 + pending RHS l*k (+1 guard)
    int64_t t = (int64_t)l * (l + 1) / 2;
    return 2 * t + 2 * (int64_t)l * k + 8;
}

}  // namespace bnd

// Host-side plan (defined in plan.cpp, used by abi.cu).
struct bnd_plan {
    bnd_dtype dtype;
    int32_t count;
    int32_t k;
    int32_t warm;
    int64_t seg_len;
    int32_t blocks_per_sm;
    int32_t max_l;
    int64_t nchains;
    int64_t nsegs;
    int32_t ntasks;
    int64_t snap_words;
    int64_t band_pool_elems;   // extent of a band pool implied by the instances
    int64_t rhs_pool_elems;    // extent of an RHS pool implied by the instances
    // host tables
    bnd::InstDev *inst;
    bnd::Chain *chains;
    bnd::Task *tasks;
    int64_t *tile_prefix;
    int64_t ntiles;
    int32_t *group_first;      // panel plans: groups (ngroups + 1 entries)
    int32_t ngroups;
    int32_t has_generic;       // some instance runs the generic (any-bandwidth) path
    int32_t wide_cta;          // the block kernels serve the generic class (its windows fit)
    int32_t wide_segmented;    // some generic-class instance is cut into segments
    // tasks are grouped by bandwidth class: class 0 = generic (l = 0 or l > kRegMaxL),
    // class c = bandwidth c; class c owns tasks [class_task0[c], class_task0[c+1])
    int32_t class_task0[bnd::kRegMaxL + 2];
    int32_t layout;            // kLayoutRows, kLayoutPanels or kLayoutStrided
    int32_t staged_ok;         // every offset / stride allows 16-byte tiles
    int32_t warm_per_l, warm_base;   // tuning: warm-up rows = warm_per_l * l + warm_base (if > 0)
    int32_t force_direct;      // tuning: never use the staged kernels
    int32_t seg_by_warm;       // tuning: segment length proportional to the warm-up
    int32_t no_staged_rerun;   // tuning: leave every mismatching segment to the serial verify pass
    cudaStream_t side[bnd::kRegMaxL + 1];
    cudaEvent_t ev_fork;
    cudaEvent_t ev_join[bnd::kRegMaxL + 1];
    int32_t streams_ready;
    // workspace layout (byte offsets)
    size_t off_inst, off_chains, off_tasks, off_tiles, off_counters, off_snap, off_logdet, off_info,
        off_rhs_tmp, off_rhs_tmp2, off_band_tmp, off_band_tmp2, off_band_tmp3, off_seg_chain, off_rerun_cnt, off_groups,
        off_rerun_list, off_task_flag, off_chain_flag, ws_bytes;
    int32_t *seg_chain;        // host table uploaded at bind
    // bound workspace
    void *ws;
    bnd::PlanDev dev;
    int bound;
};
