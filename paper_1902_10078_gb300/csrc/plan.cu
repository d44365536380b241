// Host-side plan: validation, recognition of the batch's arrangement (rows,
// 32-lane panels, general strides), segmentation of long instances into
// chains, grouping of chains into warp tasks (equal-bandwidth chains for
// rows; one (group, segment) per task for panels), longest-first task order,
// and the device workspace layout.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "sweep_cta.cuh"

using namespace bnd;

namespace {

// Default segment length (rows).  Row plans: long segments, because the
// per-lane streams make DRAM, not latency, the limit and more chains only add
// warm-up rows.  Panel plans: short segments, because their sweeps are bound
// by the latency of the per-row recurrence and need many resident chains.
constexpr int64_t kDefaultSegLenRows = 2048;
constexpr int64_t kDefaultSegLenPanels = 384;
// A batch too small to give the GPU about this many chains at the default
// length (a single long chain, a few instances) is cut into shorter segments,
// down to kMinSegLen rows: its sweeps are bound by the per-row latency, and the
// time of a sweep is that of one chain, segment plus warm-up rows.
constexpr int64_t kTargetChains = 16384;
constexpr int64_t kMinSegLen = 32;
// Wide bands (one thread block per segment): the time of a sweep is that of
// its longest segment, so the wide instances are cut into about one segment
// per SM of a GB300 (152) in all, each at least one warm-up long.
constexpr int64_t kWideTargetSegs = 152;

// Default warm-up of a speculative segment start.  The cold-started state
// forgets its start at a rate per block of l rows, so the warm-up grows with
// l.  Measured on the uneven batch (FP32, 384-row panel segments, staged
// reruns on): 16 l + 32 rows converged everywhere and was the fastest;
// 12 l + 32 left 7 of 162k segments to rerun, 8 l + 32 left 1671 (each rerun
// pass costs more than the warm-up rows it saves).  FP64 needs roughly twice
// the distance to reach its smaller rounding unit.
int64_t default_warm(bnd_dtype dt, int l) {
    const int64_t w = dt == BND_F32 ? 16 * (int64_t)l + 32 : 48 * (int64_t)l + 64;
    return (w + 3) / 4 * 4;
}
// Wide bands accept a segment start within the rounding noise of the state
// (not bit for bit), which a cold start reaches in fewer rows.  Measured on the
// wide-band workload (n = 2e5, l = 64 and 128, 16 right-hand sides): no rerun
// from 8 l + 32 rows (FP32) and 16 l + 64 (FP64) on, and every shorter
// warm-up of the sweep ran faster (FP32 l = 64: 31.4 ms per fused step at
// 8 l + 32 vs 39.7 at 16 l + 32; FP64 l = 128: 332 ms at 16 l + 64 vs 977 at
// 48 l + 64).
int64_t default_warm_wide(bnd_dtype dt, int l) {
    const int64_t w = dt == BND_F32 ? 8 * (int64_t)l + 32 : 16 * (int64_t)l + 64;
    return (w + 3) / 4 * 4;
}
constexpr int32_t kMaxBand = 1024;
constexpr int32_t kMaxRhs = 64;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace {

int64_t col_stride(const bnd_inst &I) { return I.cs <= 1 ? 1 : (int64_t)I.cs; }

// Panel groups: a group is a run of at most 32 consecutive descriptors with
// column stride 32 whose band (and RHS) offsets increase by one and which
// share l, ld and ldr; lane p is the p-th descriptor of the run.  Fills
// `groups` with the first descriptor of every group (plus `count` at the
// end) and returns false if some descriptor cannot belong to a panel.
// *aligned tells whether every group base allows 16-byte copies.
bool detect_panels(int32_t count, const bnd_inst *inst, int32_t k, int64_t tw, std::vector<int32_t> &groups,
                   bool *aligned) {
    *aligned = true;
    groups.clear();
    for (int32_t i = 0; i < count; ++i) {
        const bnd_inst &I = inst[i];
        if (I.cs != kPanelLanes || I.ld % kPanelLanes || (k > 0 && I.ldr % kPanelLanes)) return false;
        // the panel kernels address a group's region with 32-bit element offsets
        if ((int64_t)(I.l + 1) * I.ld > INT32_MAX || (int64_t)k * I.ldr > INT32_MAX) return false;
        bool cont = false;
        if (!groups.empty()) {
            const int32_t g0 = groups.back();
            const bnd_inst &H = inst[g0];
            const int64_t p = i - g0;
            cont = p < kPanelLanes && I.l == H.l && I.ld == H.ld && I.band == H.band + p &&
                   (k == 0 || (I.ldr == H.ldr && I.rhs == H.rhs + p));
        }
        if (!cont) {
            groups.push_back(i);
            if (I.band % tw || (k > 0 && I.rhs % tw)) *aligned = false;
        }
    }
    groups.push_back(count);
    return true;
}

// Segment count and length for `n` rows (nearest count of seg_len-row
// segments, length a multiple of 4 rows); one segment when not split.
void segmentation(int64_t n, int64_t seg_len, int64_t warm, bool reg, int64_t *nseg_out, int64_t *len_out) {
    int64_t nseg = 1;
    if (reg && seg_len > 0 && n > seg_len + warm) {
        nseg = (n + seg_len / 2) / seg_len;
        if (nseg < 1) nseg = 1;
    }
    int64_t len = (n + nseg - 1) / nseg;
    len = (len + 3) / 4 * 4;
    *nseg_out = (n + len - 1) / len;
    *len_out = len;
}

}  // namespace

extern "C" bnd_status bnd_plan_create(bnd_plan **out, bnd_dtype dtype, int32_t count, const bnd_inst *inst,
                                      int32_t k, const bnd_tuning *tuning) {
    if (!out) return BND_EINVAL;
    *out = nullptr;
    if (dtype != BND_F32 && dtype != BND_F64) return BND_EINVAL;
    if (count < 0 || (count > 0 && !inst)) return BND_EINVAL;
    if (k < 0 || k > kMaxRhs) return BND_EINVAL;
    bool all_rows = true;
    for (int32_t i = 0; i < count; ++i) {
        const bnd_inst &I = inst[i];
        if (I.cs < 0) return BND_EINVAL;
        const int64_t cs = col_stride(I);
        if (I.n < 1 || I.l < 0 || I.l > kMaxBand || I.band < 0) return BND_EINVAL;
        if (I.n > INT64_MAX / cs || I.ld < I.n * cs) return BND_EINVAL;
        if (k > 0 && (I.ldr < I.n * cs || I.rhs < 0)) return BND_EINVAL;
        if (cs != 1) all_rows = false;
    }
    bnd_plan *p = new (std::nothrow) bnd_plan();
    if (!p) return BND_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->dtype = dtype;
    p->count = count;
    p->k = k;
    const size_t esz = dtype == BND_F32 ? 4 : 8;
    p->warm = 0;                                      // 0: per-bandwidth default
    p->seg_len = 0;
    const int64_t user_seg_len = tuning ? tuning->seg_len : 0;
    if (tuning) {
        if (tuning->seg_len != 0) p->seg_len = tuning->seg_len;
        if (tuning->warmup > 0) p->warm = tuning->warmup;
        if (tuning->blocks_per_sm > 0) p->blocks_per_sm = tuning->blocks_per_sm;
        p->force_direct = (tuning->flags & 1) != 0;
        p->seg_by_warm = (tuning->flags & 2) != 0;
        p->no_staged_rerun = (tuning->flags & 4) != 0;
        if (tuning->warm_per_l > 0) {
            p->warm_per_l = tuning->warm_per_l;
            p->warm_base = tuning->warm_base > 0 ? tuning->warm_base : 0;
        }
    }
    const int64_t tw = 16 / (int64_t)esz;                 // elements per 16-byte tile
    p->staged_ok = 1;
    std::vector<int32_t> groups;          // panel plans: first descriptor of each group, then count
    std::vector<int32_t> group_of((size_t)count, 0);
    if (all_rows) {
        p->layout = kLayoutRows;
    } else {
        bool aligned = true;
        p->layout = detect_panels(count, inst, k, tw, groups, &aligned) ? kLayoutPanels : kLayoutStrided;
        if (p->layout == kLayoutStrided || !aligned) p->staged_ok = 0;
        if (p->layout == kLayoutPanels)
            for (size_t g = 0; g + 1 < groups.size(); ++g)
                for (int32_t i = groups[g]; i < groups[g + 1]; ++i) group_of[(size_t)i] = (int32_t)g;
    }
    const bool panels = p->layout == kLayoutPanels;
    if (p->seg_len == 0) {
        p->seg_len = panels ? kDefaultSegLenPanels : kDefaultSegLenRows;
        // rows that run as lanes: every instance (rows), or 32 lanes of each group's longest n (panels)
        int64_t lane_rows = 0;
        if (panels) {
            for (size_t g = 0; g + 1 < groups.size(); ++g) {
                int64_t gn = 0;
                for (int32_t i = groups[g]; i < groups[g + 1]; ++i) gn = std::max(gn, inst[i].n);
                lane_rows += gn * kPanelLanes;
            }
        } else {
            for (int32_t i = 0; i < count; ++i) lane_rows += inst[i].n;
        }
        if (lane_rows / p->seg_len < kTargetChains)
            p->seg_len = std::max<int64_t>(kMinSegLen, (lane_rows / kTargetChains + 3) / 4 * 4);
    }

    // wide-band instances (l = 0 or above the register-window limit) run on the block kernels
    // when the widest one's windows fit; those with l > 0 are then segmented too
    int32_t max_wide_l = -1;
    int64_t wide_rows = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (inst[i].l >= 1 && inst[i].l <= kRegMaxL) continue;
        max_wide_l = std::max(max_wide_l, inst[i].l);
        if (inst[i].l > 0) wide_rows += inst[i].n;
    }
    p->wide_cta = max_wide_l >= 0 && (dtype == BND_F32 ? cta_serves<float>(max_wide_l, cta_rhs(k))
                                                       : cta_serves<double>(max_wide_l, cta_rhs(k)));

    std::vector<InstDev> idev((size_t)count);
    int64_t nsegs = 0;
    int32_t max_l = 0;
    bool has_generic = false;
    int64_t band_extent = 0, rhs_extent = 0;
    for (int32_t i = 0; i < count; ++i) {
        const bnd_inst &I = inst[i];
        InstDev &D = idev[(size_t)i];
        D.n = I.n; D.band = I.band; D.ld = I.ld; D.rhs = I.rhs; D.ldr = I.ldr; D.l = I.l;
        D.cs = col_stride(I);
        const bool reg = I.l >= 1 && I.l <= kRegMaxL;
        if (!reg) has_generic = true;
        if (p->warm > 0) D.warm = ((int64_t)p->warm + 3) / 4 * 4;
        else if (p->warm_per_l > 0) D.warm = ((int64_t)p->warm_per_l * I.l + p->warm_base + 3) / 4 * 4;
        else D.warm = (!reg && p->wide_cta) ? default_warm_wide(dtype, I.l) : default_warm(dtype, I.l);
        // segment length: the same for every bandwidth, or (flag) scaled with the warm-up so
        // that every bandwidth pays the same fraction of extra rows (seg_len at 128 warm-up rows)
        int64_t seg_len = p->seg_len;
        if (seg_len > 0 && p->seg_by_warm) seg_len = std::max<int64_t>(64, seg_len * D.warm / 128);
        int64_t nseg = 1, len = I.n;
        if (!reg) {
            if (p->wide_cta && I.l > 0 && p->seg_len > 0) {
                const int64_t wl = user_seg_len > 0 ? user_seg_len
                                                    : std::max<int64_t>(D.warm, (wide_rows + kWideTargetSegs - 1) /
                                                                                    kWideTargetSegs);
                segmentation(I.n, wl, D.warm, true, &nseg, &len);
            }
            if (!panels && (I.band % tw || I.ld % tw || (k > 0 && (I.rhs % tw || I.ldr % tw)))) p->staged_ok = 0;
        } else if (panels) {
            // one segment length for the whole group, set by its longest member
            const int32_t g = group_of[(size_t)i], g0 = groups[(size_t)g], g1 = groups[(size_t)g + 1];
            int64_t gn = 0;
            for (int32_t q = g0; q < g1; ++q) gn = std::max(gn, inst[q].n);
            int64_t gseg = 1;
            segmentation(gn, seg_len, D.warm, reg, &gseg, &len);
            nseg = (I.n + len - 1) / len;
        } else {
            segmentation(I.n, seg_len, D.warm, reg, &nseg, &len);
            if (I.band % tw || I.ld % tw || (k > 0 && (I.rhs % tw || I.ldr % tw))) p->staged_ok = 0;
        }
        D.nseg = (int32_t)nseg;
        D.seg_len = len;
        D.seg0 = nsegs;
        nsegs += nseg;
        max_l = std::max(max_l, I.l);
        band_extent = std::max(band_extent, I.band + (int64_t)(I.l + 1) * I.ld);
        if (k > 0) rhs_extent = std::max(rhs_extent, I.rhs + (int64_t)k * I.ldr);
    }
    p->nsegs = nsegs;
    p->max_l = max_l;
    p->band_pool_elems = band_extent;
    p->rhs_pool_elems = rhs_extent;
    p->snap_words = snap_words_for(std::min(max_l, kRegMaxL), std::max(k, kMaxK));
    for (int32_t i = 0; i < count; ++i) {
        const InstDev &D = idev[(size_t)i];
        if (D.nseg > 1 && !(D.l >= 1 && D.l <= kRegMaxL)) {
            p->wide_segmented = 1;
            p->snap_words = std::max<int64_t>(p->snap_words, cta_state_words(D.l, cta_rhs(k)));
        }
    }

    struct TaskTmp { std::vector<Chain> c; int32_t l; int32_t cls; double cost; Task geo; };
    auto class_of = [](int l) { return (l >= 1 && l <= kRegMaxL) ? l : 0; };
    auto chain_rows = [&](const Chain &c) {
        return c.b - c.a + (c.seg > 0 ? idev[(size_t)c.inst].warm : 0);
    };
    auto pad_chain = []() { Chain pad; pad.inst = -1; pad.seg = 0; pad.a = pad.b = 0; return pad; };
    std::vector<TaskTmp> tt;
    auto group_tasks_by_l = [&](std::vector<Chain> &ch) {
        // chains of equal l, longest first, 32 to a task
        std::stable_sort(ch.begin(), ch.end(), [&](const Chain &x, const Chain &y) {
            const int lx = idev[(size_t)x.inst].l, ly = idev[(size_t)y.inst].l;
            if (lx != ly) return lx < ly;
            return (x.b - x.a) > (y.b - y.a);
        });
        for (size_t s = 0; s < ch.size();) {
            const int32_t l = idev[(size_t)ch[s].inst].l;
            TaskTmp t;
            t.l = l;
            t.cls = class_of(l);
            t.cost = 0;
            std::memset(&t.geo, 0, sizeof(t.geo));
            while (s < ch.size() && (int)t.c.size() < kWarp && idev[(size_t)ch[s].inst].l == l) {
                t.cost = std::max(t.cost, (double)chain_rows(ch[s]) * (double)(l + 2) * (double)(l + 2));
                t.c.push_back(ch[s]);
                ++s;
            }
            while ((int)t.c.size() < kWarp) t.c.push_back(pad_chain());
            tt.push_back(std::move(t));
        }
    };
    std::vector<Chain> loose;      // chains not bound to a panel lane
    for (int32_t i = 0; i < count; ++i) {
        const InstDev &D = idev[(size_t)i];
        if (panels && class_of(D.l) != 0) continue;
        for (int32_t s = 0; s < D.nseg; ++s) {
            Chain c;
            c.inst = i; c.seg = s;
            c.a = (int64_t)s * D.seg_len;
            c.b = std::min(c.a + D.seg_len, D.n);
            loose.push_back(c);
        }
    }
    group_tasks_by_l(loose);
    if (panels) {
        // one task per (group, segment): chain p is lane p of the group at that segment
        for (size_t g = 0; g + 1 < groups.size(); ++g) {
            const int32_t g0 = groups[g], g1 = groups[g + 1];
            const InstDev &H = idev[(size_t)g0];
            if (class_of(H.l) == 0) continue;
            int32_t gseg = 0;
            int64_t gn = 0;
            for (int32_t q = g0; q < g1; ++q) {
                gseg = std::max(gseg, idev[(size_t)q].nseg);
                gn = std::max(gn, idev[(size_t)q].n);
            }
            for (int32_t s = 0; s < gseg; ++s) {
                TaskTmp t;
                t.l = H.l;
                t.cls = class_of(H.l);
                t.cost = 0;
                t.geo.chain0 = 0; t.geo.l = H.l;
                t.geo.gband = H.band; t.geo.grhs = H.rhs; t.geo.gld = H.ld; t.geo.gldr = H.ldr; t.geo.gn = gn;
                for (int32_t p2 = 0; p2 < kWarp; ++p2) {
                    const int32_t q = g0 + p2;
                    if (q < g1 && s < idev[(size_t)q].nseg) {
                        const InstDev &D = idev[(size_t)q];
                        Chain c;
                        c.inst = q; c.seg = s;
                        c.a = (int64_t)s * D.seg_len;
                        c.b = std::min(c.a + D.seg_len, D.n);
                        t.cost = std::max(t.cost, (double)chain_rows(c) * (double)(H.l + 2) * (double)(H.l + 2));
                        t.c.push_back(c);
                    } else {
                        t.c.push_back(pad_chain());
                    }
                }
                tt.push_back(std::move(t));
            }
        }
    }
    std::stable_sort(tt.begin(), tt.end(), [](const TaskTmp &x, const TaskTmp &y) {
        if (x.cls != y.cls) return x.cls < y.cls;
        return x.cost > y.cost;
    });
    for (int c = 0; c <= kRegMaxL + 1; ++c) p->class_task0[c] = 0;
    {
        int32_t t = 0;
        for (int c = 0; c <= kRegMaxL; ++c) {
            p->class_task0[c] = t;
            while (t < (int32_t)tt.size() && tt[(size_t)t].cls == c) ++t;
        }
        p->class_task0[kRegMaxL + 1] = t;
    }
    p->ntasks = (int32_t)tt.size();
    p->nchains = (int64_t)tt.size() * kWarp;
    p->inst = (InstDev *)std::malloc(sizeof(InstDev) * std::max<size_t>(1, (size_t)count));
    p->chains = (Chain *)std::malloc(sizeof(Chain) * std::max<size_t>(1, (size_t)p->nchains));
    p->tasks = (Task *)std::malloc(sizeof(Task) * std::max<size_t>(1, tt.size()));
    if (!p->inst || !p->chains || !p->tasks) { bnd_plan_destroy(p); return BND_EINVAL; }
    if (count) std::memcpy(p->inst, idev.data(), sizeof(InstDev) * (size_t)count);
    for (size_t t = 0; t < tt.size(); ++t) {
        p->tasks[t] = tt[t].geo;
        p->tasks[t].chain0 = (int32_t)(t * kWarp);
        p->tasks[t].l = tt[t].l;
        for (int c = 0; c < kWarp; ++c) p->chains[t * kWarp + c] = tt[t].c[(size_t)c];
    }
    // chain running each global segment (staged reruns address segments through it)
    p->seg_chain = (int32_t *)std::malloc(sizeof(int32_t) * std::max<size_t>(1, (size_t)nsegs));
    if (!p->seg_chain) { bnd_plan_destroy(p); return BND_EINVAL; }
    for (int64_t g = 0; g < nsegs; ++g) p->seg_chain[g] = -1;
    for (int64_t c = 0; c < p->nchains; ++c) {
        const Chain &ch = p->chains[c];
        if (ch.inst >= 0) p->seg_chain[idev[(size_t)ch.inst].seg0 + ch.seg] = (int32_t)c;
    }
    // product tiles: 256 columns of one instance (rows plans), or 8 columns of the 32 lanes of
    // a panel group (panel plans: a warp reads one column of the group, 32 adjacent elements)
    if (panels) {
        p->ngroups = (int32_t)groups.size() - 1;
        p->group_first = (int32_t *)std::malloc(sizeof(int32_t) * groups.size());
        p->tile_prefix = (int64_t *)std::malloc(sizeof(int64_t) * groups.size());
        if (!p->group_first || !p->tile_prefix) { bnd_plan_destroy(p); return BND_EINVAL; }
        p->tile_prefix[0] = 0;
        for (int32_t g = 0; g <= p->ngroups; ++g) p->group_first[g] = groups[(size_t)g];
        for (int32_t g = 0; g < p->ngroups; ++g) {
            int64_t gn = 0;
            for (int32_t i = groups[(size_t)g]; i < groups[(size_t)g + 1]; ++i) gn = std::max(gn, inst[i].n);
            p->tile_prefix[g + 1] = p->tile_prefix[g] + (gn + 7) / 8;
        }
        p->ntiles = p->tile_prefix[p->ngroups];
    } else {
        p->ngroups = 0;
        p->tile_prefix = (int64_t *)std::malloc(sizeof(int64_t) * ((size_t)count + 1));
        if (!p->tile_prefix) { bnd_plan_destroy(p); return BND_EINVAL; }
        p->tile_prefix[0] = 0;
        for (int32_t i = 0; i < count; ++i) p->tile_prefix[i + 1] = p->tile_prefix[i] + (idev[(size_t)i].n + 255) / 256;
        p->ntiles = p->tile_prefix[count];
    }
    p->has_generic = has_generic ? 1 : 0;

    // workspace layout
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    p->off_inst = take(sizeof(InstDev) * (size_t)count);
    p->off_chains = take(sizeof(Chain) * (size_t)p->nchains);
    p->off_tasks = take(sizeof(Task) * (size_t)p->ntasks);
    p->off_tiles = take(sizeof(int64_t) * ((size_t)std::max(count, p->ngroups) + 1));
    p->off_groups = take(sizeof(int32_t) * ((size_t)p->ngroups + 1));
    p->off_counters = take(sizeof(unsigned int) * kNumCounters);
    p->off_snap = take(esz * (size_t)nsegs * 2 * (size_t)p->snap_words);
    p->off_logdet = take(sizeof(double) * (size_t)nsegs);
    p->off_info = take(sizeof(int32_t) * (size_t)nsegs);
    p->off_rhs_tmp = take(esz * (size_t)rhs_extent);
    p->off_rhs_tmp2 = take(esz * (size_t)rhs_extent);
    p->off_band_tmp = take(esz * (size_t)band_extent);
    p->off_band_tmp2 = take(has_generic ? esz * (size_t)band_extent : 0);
    p->off_band_tmp3 = take(has_generic ? esz * (size_t)band_extent : 0);
    p->off_seg_chain = take(sizeof(int32_t) * (size_t)nsegs);
    p->off_rerun_cnt = take(sizeof(uint32_t) * (kRegMaxL + 1));
    p->off_rerun_list = take(sizeof(int32_t) * (size_t)p->ntasks);
    p->off_task_flag = take(sizeof(uint32_t) * (size_t)p->ntasks);
    p->off_chain_flag = take((size_t)p->nchains);
    p->ws_bytes = o;
    *out = p;
    return BND_OK;
}

extern "C" size_t bnd_plan_workspace_bytes(const bnd_plan *p) { return p ? p->ws_bytes : 0; }

extern "C" int64_t bnd_plan_chains(const bnd_plan *p) { return p ? p->nsegs : 0; }

extern "C" int64_t bnd_plan_tasks(const bnd_plan *p) { return p ? p->ntasks : 0; }

extern "C" int32_t bnd_plan_layout(const bnd_plan *p) { return p ? p->layout : -1; }

extern "C" bnd_status bnd_plan_bind(bnd_plan *p, void *ws, size_t ws_bytes, void *stream) {
    if (!p || (!ws && p->ws_bytes) || ws_bytes < p->ws_bytes) return BND_EINVAL;
    if (((uintptr_t)ws & 255) != 0) return BND_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = (char *)ws;
    p->ws = ws;
    PlanDev &d = p->dev;
    d.inst = (const InstDev *)(base + p->off_inst);
    d.chains = (const Chain *)(base + p->off_chains);
    d.tasks = (const Task *)(base + p->off_tasks);
    d.tile_prefix = (const int64_t *)(base + p->off_tiles);
    d.ntasks = p->ntasks;
    d.count = p->count;
    d.nchains = p->nchains;
    d.nsegs = p->nsegs;
    d.ntiles = p->ntiles;
    d.ngroups = p->ngroups;
    d.group_first = (const int32_t *)(base + p->off_groups);
    d.k = p->k;
    d.warm = p->warm;
    d.counters = (unsigned int *)(base + p->off_counters);
    d.snap = base + p->off_snap;
    d.snap_words = p->snap_words;
    d.seg_logdet = (double *)(base + p->off_logdet);
    d.seg_info = (int32_t *)(base + p->off_info);
    d.rhs_tmp = base + p->off_rhs_tmp;
    d.rhs_tmp2 = base + p->off_rhs_tmp2;
    d.band_tmp = base + p->off_band_tmp;
    d.band_tmp2 = base + p->off_band_tmp2;
    d.band_tmp3 = base + p->off_band_tmp3;
    d.seg_chain = (const int32_t *)(base + p->off_seg_chain);
    d.rerun_cnt = (uint32_t *)(base + p->off_rerun_cnt);
    d.rerun_list = (int32_t *)(base + p->off_rerun_list);
    d.task_flag = (uint32_t *)(base + p->off_task_flag);
    d.chain_flag = (uint8_t *)(base + p->off_chain_flag);
    cudaError_t e = cudaSuccess;
    if (!p->streams_ready) {
        for (int c = 0; c <= kRegMaxL && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&p->side[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[c], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return BND_ECUDA;
        p->streams_ready = 1;
    }
    if (p->count) e = cudaMemcpyAsync(base + p->off_inst, p->inst, sizeof(InstDev) * (size_t)p->count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && p->nchains) e = cudaMemcpyAsync(base + p->off_chains, p->chains, sizeof(Chain) * (size_t)p->nchains, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && p->ntasks) e = cudaMemcpyAsync(base + p->off_tasks, p->tasks, sizeof(Task) * (size_t)p->ntasks, cudaMemcpyHostToDevice, s);
    const size_t ntab = (size_t)(p->ngroups > 0 ? p->ngroups : p->count) + 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + p->off_tiles, p->tile_prefix, sizeof(int64_t) * ntab, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && p->ngroups > 0)
        e = cudaMemcpyAsync(base + p->off_groups, p->group_first, sizeof(int32_t) * ((size_t)p->ngroups + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + p->off_counters, 0, sizeof(unsigned int) * kNumCounters, s);
    if (e == cudaSuccess && p->nsegs)
        e = cudaMemcpyAsync(base + p->off_seg_chain, p->seg_chain, sizeof(int32_t) * (size_t)p->nsegs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + p->off_rerun_cnt, 0, sizeof(uint32_t) * (kRegMaxL + 1), s);
    if (e == cudaSuccess && p->ntasks) e = cudaMemsetAsync(base + p->off_task_flag, 0, sizeof(uint32_t) * (size_t)p->ntasks, s);
    if (e == cudaSuccess && p->nchains) e = cudaMemsetAsync(base + p->off_chain_flag, 0, (size_t)p->nchains, s);
    // pageable sources: make sure the copies have consumed the host tables before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return BND_ECUDA;
    p->bound = 1;
    return BND_OK;
}

extern "C" void bnd_plan_destroy(bnd_plan *p) {
    if (!p) return;
    if (p->streams_ready) {
        for (int c = 0; c <= kRegMaxL; ++c) {
            cudaStreamDestroy(p->side[c]);
            cudaEventDestroy(p->ev_join[c]);
        }
        cudaEventDestroy(p->ev_fork);
    }
    std::free(p->inst);
    std::free(p->chains);
    std::free(p->tasks);
    std::free(p->tile_prefix);
    std::free(p->group_first);
    std::free(p->seg_chain);
    delete p;
}

extern "C" bnd_status bnd_plan_fixups(const bnd_plan *p, int32_t kind, int64_t *out, void *stream) {
    if (!p || !p->bound || !out || kind < 0 || kind > kNumSweepKinds) return BND_EINVAL;
    unsigned int v = 0;
    const int slot = kind == kNumSweepKinds ? kTimeoutCounter : kNumSweepKinds + kind;
    cudaError_t e = cudaMemcpyAsync(&v, p->dev.counters + slot, sizeof(v), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return BND_ECUDA;
    *out = v;
    return BND_OK;
}
