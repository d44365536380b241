"""Benchmark: band entries/s of the fused forward + backward step of the
banded operators (Cholesky, solves, log-det, subset inverse and their
adjoints) on the uneven batch, batched vs plain, with its HBM roofline.

Workload ("uneven batch", 4096 instances): n log-uniform in [1000, 65536],
l uniform in {1, 2, 3, 5, 7}, k = 4 right-hand sides, FP32, seeded synthetic
SPD bands Q = band(L0 L0^T) + 1e-3 I with N(0,1) right-hand sides and
cotangents (Xbar, Sbar) and ldbar = 1/2.  One step = banded_gmm_forward +
banded_gmm_backward over the whole batch.  Inputs (~4.3 GB) are larger than
L2, so no flush is needed between steps.

Output: one JSON line (rank 0).  `value` is device-timed (inputs resident in
HBM, CUDA graph replay); `e2e` adds the pinned host->device copy of the
step's inputs and the device->host read of the step's result (log-dets and
info) through the same public API.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1902_10078_gb300 import workloads as W  # noqa: E402

METRIC = "band entries/s fwd+bwd (chol/solve/subinv), batched vs plain; % of HBM roofline"
UNIT = "entries/s"
LAYOUT_NOTE = {
    "panels": "lower-band storage (l+1) x n per instance, 32 instances of equal l interleaved per column "
              "(column stride 32); instances ordered by (l, n)",
    "rows": "lower-band storage (l+1) x n per instance, each diagonal contiguous (column stride 1)",
}
WORKLOAD = "uneven batch: 4096 instances, n log-uniform [1000, 65536], l in {1,2,3,5,7}, k=4 RHS, FP32"


# --------------------------------------------------------------------------- inputs

def batch_layout(count, k, ls, panels, rank=0, world=1, strong=False):
    """The uneven batch of `rank`: its pool layout, every slot's seed and the
    original index of every slot.

    Weak scaling (default): every rank draws its own batch of `count`
    instances; instance i (original order) has the i-th drawn shape and seed
    BASE_SEED + rank * count + i.  Strong scaling: one batch of `count`
    instances (rank 0's draw) is split over the ranks by shard.partition
    (longest-processing-time on n (l+1)^2), each rank keeping its share with
    the shapes and seeds the instances have in the whole batch.  A panel
    layout reorders the rank's instances (panel_order) and carries each one's
    seed along, so slot p holds original instance order[p] whatever the
    arrangement."""
    from paper_1902_10078_gb300 import batch as BT
    from paper_1902_10078_gb300 import binding as B
    from paper_1902_10078_gb300 import shard
    if strong:
        ns, lss = W.batched_shapes(count, seed=W.BASE_SEED, ls=ls)
        mine = shard.partition([int(x) for x in ns], [int(x) for x in lss], world)[rank]
        seed0 = W.BASE_SEED
    else:
        ns, lss = W.batched_shapes(count, seed=W.BASE_SEED + rank * 7919, ls=ls)
        mine = list(range(count))
        seed0 = W.BASE_SEED + rank * count
    sub_ns, sub_ls = [int(ns[i]) for i in mine], [int(lss[i]) for i in mine]
    local = BT.panel_order(sub_ns, sub_ls) if panels else list(range(len(mine)))
    order = [int(mine[q]) for q in local]
    lay = BT.Layout([int(ns[i]) for i in order], [int(lss[i]) for i in order], k, B.BND_F32, panels=panels)
    seeds = [seed0 + i for i in order]
    return lay, seeds, order


def cpu_sample(count, size):
    """Original indices of the bounded sample the oracle runs (the same instances
    in the CPU baseline, the reference arm and the parity check of the GPU run)."""
    rng = np.random.Generator(np.random.PCG64(11))
    return np.sort(rng.choice(count, size=min(size, count), replace=False))


# --------------------------------------------------------------------------- clocks

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- our arm

def algorithmic_bytes(lay, w=4):
    """Two-call (forward | backward) algorithmic bytes per step.

    forward : Q read, L write, S write (band); B read, X write (RHS)
    backward: L read, S read, Sbar read, Qbar write (band); X read, Xbar read, Bbar write (RHS)
    -> per instance w * n * (7 (l+1) + 5 k); fused floor w * n * (4 (l+1) + 4 k).
    """
    fwd = bwd = floor = 0
    for n, l in zip(lay.ns, lay.ls):
        fwd += w * n * (3 * (l + 1) + 2 * lay.k)
        bwd += w * n * (4 * (l + 1) + 3 * lay.k)
        floor += w * n * (4 * (l + 1) + 4 * lay.k)
    return fwd, bwd, floor


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gmm_backward_traffic.json")


# Sources of the kernels the uneven batch runs (register-window sweeps, staged
# I/O, reruns, verify, plan and entry points); the wide-band block kernels,
# the one-warp fallback, the products and the allocation-free solve are not
# among them.
HOT_SOURCES = ("common.cuh", "sweep_impl.cuh", "sweep_io.cuh", "sweep_staged.cuh", "sweep_launch.cuh", "plan.cu",
               "abi.cu", "sweep_fwd_float.cu", "sweep_bwd_float.cu") + tuple(f"sweep_staged_l{i}.cu" for i in range(1, 9))


def _code_only(text):
    """C/C++ source without its comments and blank-line differences (a comment
    edit does not change a kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def source_hash():
    """Hash of the code of the uneven batch's kernels and the C header: a
    stored DRAM traffic figure is only reported while the kernels it was
    measured on are unchanged."""
    import hashlib
    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_1902_10078_gb300", "csrc", f) for f in sorted(HOT_SOURCES)]
    files.append(os.path.join(ROOT, "include", "banded.h"))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(call, entries):
    """DRAM bytes per launch of `call` from the committed ncu summary, scaled from
    the captured case to `entries` band entries; None if absent or stale."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("call") != call or t.get("source_hash") != source_hash():
        return None
    return t["dram_bytes_per_call"] * entries / t["band_entries"]


def summarize_ncu(args):
    """Sum dram__bytes_{read,write} of every kernel in an ncu --csv capture of one
    banded_gmm_backward call (bench.py --profile-once) and store it with the
    source hash and the captured case's band entries."""
    import csv
    rows = list(csv.reader(open(args.summarize_ncu)))
    h = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    idx = {k: j for j, k in enumerate(rows[h])}
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total, launches, per = 0.0, set(), {}
    for r in rows[h + 1:]:
        if len(r) < len(rows[h]) or not r[idx["Metric Name"]].startswith("dram__bytes_"):
            continue
        v = float(r[idx["Metric Value"]].replace(",", "")) * unit[r[idx["Metric Unit"]]]
        total += v
        launches.add(r[idx["ID"]])
        name = r[idx["Kernel Name"]].split("(")[0]
        per[name] = per.get(name, 0.0) + v
    out = {"call": "banded_gmm_backward", "source_hash": source_hash(), "dram_bytes_per_call": total,
           "band_entries": args.summarize_entries, "launches": len(launches), "capture": args.summarize_cmd,
           "per_kernel_bytes": per}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("dram_bytes_per_call", "band_entries", "launches")}))


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings (every rank gets the result):
    the slowest rank sets the job's time."""
    import torch
    if world <= 1:
        return [float(v) for v in values]
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def sum_over_ranks(value, world, device):
    """Sum of a per-rank count over the ranks (every rank gets the result)."""
    import torch
    if world <= 1:
        return float(value)
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_ours(args, rank, world, device_index):
    import torch
    import torch.distributed as dist

    from paper_1902_10078_gb300 import batch as BT
    from paper_1902_10078_gb300 import binding as B

    count = args.count
    panels = args.layout == "panels"
    strong = args.scaling == "strong"
    lay, seeds, order = batch_layout(count, args.k, tuple(int(x) for x in args.ls.split(",")), panels, rank,
                                     world, strong)
    count = lay.count                      # this rank's instances
    host = W.fill_pools(lay, seeds, args.workers)
    torch.cuda.set_device(device_index)
    from paper_1902_10078_gb300 import build as bld
    bld.build()
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    L, S, Qb = lay.band_pool(), lay.band_pool(), lay.band_pool()
    X, Bb = lay.rhs_pool(), lay.rhs_pool()
    logdet = torch.empty(count, dtype=torch.float64, device="cuda")
    info = torch.empty(count, dtype=torch.int32, device="cuda")
    ldbar = torch.full((count,), 0.5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    tuning = dict(seg_len=args.seg_len, warmup=args.warm, flags=args.flags, warm_per_l=args.warm_per_l,
                  warm_base=args.warm_base)
    autotuned = None
    if args.autotune:
        def make_step(pl):
            def one():
                B.banded_gmm_forward(pl.handle, dev["Q"], dev["B"], L, X, S, logdet, info)
                B.banded_gmm_backward(pl.handle, L, X, S, dev["Xbar"], dev["Sbar"], ldbar, Qb, Bb)
            return one
        best, timings = BT.autotune(lay, make_step, use_cache=False)
        tuning.update(best)
        autotuned = {"chosen": best, "ms_per_candidate": timings}
    plan = BT.Plan(lay, tuning)
    expect = B.LAYOUT_PANELS if panels else B.LAYOUT_ROWS
    assert B.bnd_plan_layout(plan.handle) == expect, "the plan did not take the intended arrangement"

    def fwd():
        B.banded_gmm_forward(plan.handle, dev["Q"], dev["B"], L, X, S, logdet, info)

    def bwd():
        B.banded_gmm_backward(plan.handle, L, X, S, dev["Xbar"], dev["Sbar"], ldbar, Qb, Bb)

    def step():
        fwd()
        bwd()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0, "non-SPD instance in the benchmark batch"
    if args.profile_once:
        # one forward and one backward call inside NVTX ranges, for an ncu capture
        torch.cuda.nvtx.range_push("gmm_forward")
        fwd()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_push("gmm_backward")
        bwd()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        entries = int(sum(n * (l + 1) for n, l in zip(lay.ns, lay.ls)))
        print(json.dumps({"profile_once": True, "band_entries": entries}), flush=True)
        return None
    fixups = sum(B.bnd_plan_fixups(plan.handle, kk) for kk in range(6))
    assert B.bnd_plan_fixups(plan.handle, 6) == 0, "a bounded device wait gave up"

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()

    clocks = Clocks(device_index)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps

    # per-call durations (eager, events on the launching stream) for the roofline
    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    ms_fwd = timed(fwd, max(2, args.steps // 2))
    ms_bwd = timed(bwd, max(2, args.steps // 2))

    # end to end through the public API, every step moving all of its inputs in from pinned host
    # memory and all of its results (forward X, S, log-dets and info; backward Qbar and Bbar) back to
    # pinned host memory, pipelined over two buffer sets: step i's inputs cross on one copy stream
    # while step i-1 computes, and its results cross on a second copy stream while step i+1 computes
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
    in_keys = ("Q", "B", "Xbar", "Sbar")
    sets = [dict(dev=dev, out=dict(L=L, X=X, S=S, Qbar=Qb, Bbar=Bb, logdet=logdet, info=info))]
    sets.append(dict(dev={k: torch.empty_like(v) for k, v in dev.items()},
                     out={k: torch.empty_like(v) for k, v in sets[0]["out"].items()}))
    out_keys = ("X", "S", "Qbar", "Bbar", "logdet", "info")
    back = [{k: torch.empty(st["out"][k].shape, dtype=st["out"][k].dtype).pin_memory() for k in out_keys}
            for st in sets]
    ncs = max(1, args.copy_streams)                     # copy streams per direction
    s_in = [torch.cuda.Stream() for _ in range(ncs)]
    s_out = [torch.cuda.Stream() for _ in range(ncs)]
    s_comp = torch.cuda.Stream()
    ev_in = [[torch.cuda.Event() for _ in range(ncs)] for _ in sets]
    ev_comp = [torch.cuda.Event() for _ in sets]
    ev_out = [[torch.cuda.Event() for _ in range(ncs)] for _ in sets]

    def pieces(dst, src):
        """Contiguous pieces of a copy, one per copy stream."""
        d, s_ = dst.view(-1), src.view(-1)
        step_ = (d.numel() + ncs - 1) // ncs
        return [(d[o:o + step_], s_[o:o + step_]) for o in range(0, d.numel(), step_)]

    def e2e_steps(count):
        for i in range(count):
            b = i % 2
            st = sets[b]
            for c, sc in enumerate(s_in):
                sc.wait_event(ev_comp[b])               # the step that last read these inputs is done
                with torch.cuda.stream(sc):
                    for k in in_keys:
                        for p_i, (dd, ss) in enumerate(pieces(st["dev"][k], pinned[k])):
                            if p_i == c:
                                dd.copy_(ss, non_blocking=True)
                    ev_in[b][c].record(sc)
            for c in range(ncs):
                s_comp.wait_event(ev_in[b][c])
                s_comp.wait_event(ev_out[b][c])         # this set's previous results are out
            with torch.cuda.stream(s_comp):
                d, o = st["dev"], st["out"]
                B.banded_gmm_forward(plan.handle, d["Q"], d["B"], o["L"], o["X"], o["S"], o["logdet"], o["info"])
                B.banded_gmm_backward(plan.handle, o["L"], o["X"], o["S"], d["Xbar"], d["Sbar"], ldbar, o["Qbar"],
                                      o["Bbar"])
                ev_comp[b].record(s_comp)
            for c, sc in enumerate(s_out):
                sc.wait_event(ev_comp[b])
                with torch.cuda.stream(sc):
                    for k in out_keys:
                        for p_i, (dd, ss) in enumerate(pieces(back[b][k], st["out"][k])):
                            if p_i == c:
                                dd.copy_(ss, non_blocking=True)
                    ev_out[b][c].record(sc)

    e2e_steps(2)
    torch.cuda.synchronize()
    e_reps = max(4, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s_in[0])
    for sc in s_in[1:] + [s_comp] + s_out:
        sc.wait_event(a)                                # nothing of the timed steps starts before a
    e2e_steps(e_reps)
    for evs in ev_out:                                  # b after every result copy
        for ev in evs:
            s_comp.wait_event(ev)
    b.record(s_comp)
    torch.cuda.synchronize()
    ms_e2e = a.elapsed_time(b) / e_reps
    h2d = sum(pinned[k].numel() * pinned[k].element_size() for k in in_keys)
    d2h = sum(v.numel() * v.element_size() for v in back[0].values())

    # outputs of the instances the oracle samples (parity check of this very run)
    sample_out = None
    if rank == 0 and not args.no_cpu_baseline:
        slot_of = {int(o): p for p, o in enumerate(order)}
        sample_out = {}
        for i in cpu_sample(args.count, args.cpu_sample):
            if int(i) not in slot_of:      # strong scaling: held by another rank
                continue
            p = slot_of[int(i)]
            sample_out[int(i)] = dict(
                L=lay.band_view(L, p).cpu().numpy(), S=lay.band_view(S, p).cpu().numpy(),
                Qbar=lay.band_view(Qb, p).cpu().numpy(), X=lay.rhs_view(X, p).cpu().numpy(),
                Bbar=lay.rhs_view(Bb, p).cpu().numpy(), logdet=float(logdet[p]), info=int(info[p]))

    entries = int(sum(n * (l + 1) for n, l in zip(lay.ns, lay.ls)))
    ms, ms_e2e, ms_fwd, ms_bwd = max_over_ranks([ms, ms_e2e, ms_fwd, ms_bwd], world, "cuda")
    entries_all = sum_over_ranks(entries, world, "cuda")

    plain = None
    if args.plain and rank == 0:
        plain = run_plain(args, lay, host, torch, B, BT)

    # kernels per step: 4 sweeps x (one kernel per bandwidth class present + the verify pass when segmented)
    classes = len(set(int(l) if 1 <= int(l) <= 8 else 0 for l in lay.ls))
    # (a segmented plan adds, per bandwidth class, the mark kernel and the staged rerun pass, and
    # one verify kernel per sweep: the launch list of profiles/ shows 64 kernels per step here)
    segmented = plan.chains > count
    reruns = segmented and not (int(tuning.get("flags") or 0) & 4)
    launches_per_step = 4 * (classes * (3 if reruns else 1) + (1 if segmented else 0))
    fwd_b, bwd_b, floor_b = algorithmic_bytes(lay)
    return dict(lay=lay, plan=plan, ms=ms, ms_e2e=ms_e2e, ms_fwd=ms_fwd, ms_bwd=ms_bwd, entries=entries,
                entries_all=entries_all,
                autotuned=autotuned,
                fwd_bytes=fwd_b, bwd_bytes=bwd_b, floor_bytes=floor_b, clocks=clk, h2d=h2d, d2h=d2h,
                fixups=fixups, plain=plain, launches=launches_per_step * args.steps, sample_out=sample_out)


def run_plain(args, lay, host, torch, B, BT):
    """The same kernels, one instance per launch, on one stream, no graph: time
    a fixed sample of instances and scale to the whole batch by band entries."""
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.sort(rng.choice(lay.count, size=min(args.plain_sample, lay.count), replace=False))
    t_total = 0.0
    ent = 0
    for i in idx:
        sub = BT.Layout([lay.ns[i]], [lay.ls[i]], lay.k, lay.dtype)
        plan = BT.Plan(sub, dict(seg_len=args.seg_len, warmup=args.warm))

        def cut_band(key):
            return torch.from_numpy(sub.pack_band([lay.band_view(host[key], i)])).cuda()

        def cut_rhs(key):
            return torch.from_numpy(sub.pack_rhs([lay.rhs_view(host[key], i)])).cuda()
        Q, Sb, Bm, Xb = cut_band("Q"), cut_band("Sbar"), cut_rhs("B"), cut_rhs("Xbar")
        L, S, Qb = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        X, Bb = torch.empty_like(Bm), torch.empty_like(Bm)
        ld = torch.empty(1, dtype=torch.float64, device="cuda")
        inf = torch.empty(1, dtype=torch.int32, device="cuda")
        ldb = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")

        def one():
            B.banded_gmm_forward(plan.handle, Q, Bm, L, X, S, ld, inf)
            B.banded_gmm_backward(plan.handle, L, X, S, Xb, Sb, ldb, Qb, Bb)
        one()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        one()
        b.record()
        torch.cuda.synchronize()
        t_total += a.elapsed_time(b)
        ent += lay.ns[i] * (lay.ls[i] + 1)
        plan.close()
    total_entries = sum(n * (l + 1) for n, l in zip(lay.ns, lay.ls))
    ms_full = t_total * total_entries / ent
    return {"value": total_entries / (ms_full * 1e-3), "unit": UNIT, "ms_per_step_scaled": ms_full,
            "sample_instances": int(len(idx)), "note": "one instance per launch, same kernels, one stream, "
            "no graph; timed on a fixed sample and scaled to the batch by band entries"}


# --------------------------------------------------------------------------- oracle arm

# FP32 parity tolerances against the FP64 oracle (normwise per array per instance):
# forward arrays and log-det 1e-4, gradients 1e-3.
PARITY_TOL = {"L": 1e-4, "S": 1e-4, "X": 1e-4, "logdet": 1e-4, "Qbar": 1e-3, "Bbar": 1e-3}


def cpu_baseline(args, sample_count=None, gpu_out=None):
    """The FP64 C oracle on a bounded sample of the batch's own instances
    (same shapes and seeds as the GPU run's rank 0, FP32-rounded inputs).
    With `gpu_out` (sampled GPU outputs by original index) it also returns the
    worst normwise error of every output against the oracle."""
    import oracle as O
    count = args.count
    ls = tuple(int(x) for x in args.ls.split(","))
    ns, lss = W.batched_shapes(count, seed=W.BASE_SEED, ls=ls)
    idx = cpu_sample(count, sample_count or args.cpu_sample)
    insts = [W.make_instance(int(ns[i]), int(lss[i]), args.k, W.BASE_SEED + int(i)) for i in idx]
    for ins in insts:                      # the CPU sees the same FP32-rounded inputs
        for key in ("Q", "B", "Xbar", "Sbar"):
            setattr(ins, key, getattr(ins, key).astype(np.float32).astype(np.float64))
    O.lib()
    t = time.perf_counter()
    res, threads = O.batch_step(insts)
    dt = time.perf_counter() - t
    ent = sum(i.n * (i.l + 1) for i in insts)
    cb = {"value": ent / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
          "sample": f"{len(insts)} of {count} instances ({ent} band entries), FP64 C oracle, "
                    f"OpenMP over instances, {dt:.2f} s"}
    parity = None
    if gpu_out is not None:
        worst = {k: 0.0 for k in PARITY_TOL}
        bad = 0
        for i, r in zip(idx, res):
            if int(i) not in gpu_out:       # strong scaling: held by another rank
                continue
            g = gpu_out[int(i)]
            bad += int(g["info"] != 0 or r["info"] != 0)
            for key in ("L", "S", "Qbar"):
                worst[key] = max(worst[key], _normwise(g[key][: r[key].shape[0]], r[key]))
            for key in ("X", "Bbar"):
                worst[key] = max(worst[key], _normwise(g[key], r[key]))
            worst["logdet"] = max(worst["logdet"], abs(g["logdet"] - r["logdet"]) / max(1.0, abs(r["logdet"])))
        parity = {"instances": sum(int(int(i) in gpu_out) for i in idx), "max_normwise_err": worst, "tol": PARITY_TOL, "non_spd": bad,
                  "pass": bad == 0 and all(worst[k] <= PARITY_TOL[k] for k in worst)}
    return cb, dt, parity


def _normwise(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b), initial=0.0))


# --------------------------------------------------------------------------- the other configurations

PEAKS_FILE = os.path.join(ROOT, "profiles", "peaks_gb300.json")


def compute_peaks():
    """FP32 / FP64 FMA throughput measured by microbench/peaks.cu (committed summary)."""
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def run_config(args):
    """Supplementary measurements of the other workload configurations (one
    JSON line each; the headline line is the uneven batch).  Every number is
    timed with CUDA events on the launching stream after warm-up calls."""
    import torch

    from paper_1902_10078_gb300 import batch as BT
    from paper_1902_10078_gb300 import binding as B
    from paper_1902_10078_gb300 import build as bld
    from paper_1902_10078_gb300 import losses as LS
    torch.cuda.set_device(0)
    bld.build()
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def gmm_setup(shapes, k, dt, tuning=None, panels=False):
        insts = [W.make_instance(n, l, k, W.BASE_SEED + i) for i, (n, l) in enumerate(shapes)]
        lay = BT.Layout([s[0] for s in shapes], [s[1] for s in shapes], k, dt, panels=panels)
        plan = BT.Plan(lay, tuning)
        dev = {key: torch.from_numpy(pool).cuda() for key, pool in (
            ("Q", lay.pack_band([i.Q for i in insts])), ("Sbar", lay.pack_band([i.Sbar for i in insts])),
            ("B", lay.pack_rhs([i.B for i in insts])), ("Xbar", lay.pack_rhs([i.Xbar for i in insts])))}
        L, S, Qb = lay.band_pool(), lay.band_pool(), lay.band_pool()
        X, Bb = lay.rhs_pool(), lay.rhs_pool()
        ld = torch.empty(lay.count, dtype=torch.float64, device="cuda")
        info = torch.empty(lay.count, dtype=torch.int32, device="cuda")
        ldb = torch.full((lay.count,), 0.5, dtype=torch.float64, device="cuda")

        def step():
            B.banded_gmm_forward(plan.handle, dev["Q"], dev["B"], L, X, S, ld, info)
            B.banded_gmm_backward(plan.handle, L, X, S, dev["Xbar"], dev["Sbar"], ldb, Qb, Bb)
        return lay, plan, step, info

    lines = []
    dts = {"f64": B.BND_F64, "f32": B.BND_F32}
    peaks = compute_peaks()
    if args.config == 0:
        import oracle as O
        tuning = {key: v for key, v in (("seg_len", args.seg_len), ("warm_per_l", args.warm_per_l),
                                         ("warm_base", args.warm_base)) if v}
        for name, dt in dts.items():
            lay, plan, step, info = gmm_setup([(1000, 2)], 1, dt, tuning or None)
            ms = timed(step, 200)
            fix = sum(B.bnd_plan_fixups(plan.handle, kk) for kk in range(6))
            ins = W.make_instance(1000, 2, 1, W.BASE_SEED)
            O.lib()
            reps, t0 = 200, time.perf_counter()
            for _ in range(reps):
                O.batch_step([ins])
            cpu_us = 1e6 * (time.perf_counter() - t0) / reps
            lines.append({"config": f"plain single instance n=1000, l=2, 1 RHS, {name}: fused Cholesky + solve + "
                          "log-det + subset inverse, forward and backward", "us_per_step": 1e3 * ms,
                          "segments": plan.chains, "segment_fixups_last_step": fix, "tuning": tuning,
                          "oracle_us_per_step_1core": cpu_us,
                          "bound": "the per-row dependent chain of each segment (FP64: ~650-cycle sqrt and "
                                   "division, 64-cycle FMA on this part)"})
    elif args.config == 1:
        from oracle import losses as OL
        n, l = 100_000, 3
        Q, b, Wt = W.long_chain_config(n, l)
        t0 = time.perf_counter()
        OL.chain_loss(Q, b, Wt)
        cpu_ms = 1e3 * (time.perf_counter() - t0)
        for name, dt in dts.items():
            lay = BT.Layout([n], [l], 1, dt)
            plan = BT.Plan(lay)
            Qd = torch.tensor(lay.pack_band([Q]), device="cuda", requires_grad=True)
            bd = torch.tensor(lay.pack_rhs([b[None]]), device="cuda")
            Wd = torch.tensor(lay.pack_band([Wt]), device="cuda")
            wsym = LS.symmetric_weights(lay)

            def step():
                Qd.grad = None
                loss, _ = LS.chain_loss(plan, Qd, bd, Wd, wsym)
                loss.backward()
            ms = timed(step, 20)
            lines.append({"config": f"long chain n={n}, l={l}, loss forward + backward through autograd, {name}",
                          "ms_per_step": ms, "ns_per_row": 1e6 * ms / n, "segments": plan.chains,
                          "oracle_ms_per_step_1core": cpu_ms})
    elif args.config == 3:
        # fused forward + backward with all 16 right-hand sides in each sweep (wide-band block kernels)
        for l in args.wide_ls:
            for name in args.wide_dtypes:
                dt = dts[name]
                n, k = args.wide_n, 16
                tuning = {key: v for key, v in (("seg_len", args.seg_len), ("warm_per_l", args.warm_per_l),
                                                 ("warm_base", args.warm_base)) if v}
                lay, plan, step, info = gmm_setup([(n, l)], k, dt, tuning or None)
                step()
                torch.cuda.synchronize()
                ms = timed(step, 10)
                fixups = [B.bnd_plan_fixups(plan.handle, kk) for kk in range(6)]
                flops = 9.0 * n * l * l
                pk = peaks.get("fp64_fma_tflops" if name == "f64" else "fp32_fma_tflops")
                gf = flops / (ms * 1e-3) / 1e9
                lines.append({"config": f"wide band n={n}, l={l}, k={k}, {name}: Cholesky, Q^-1 B, subset inverse "
                              "and their adjoints (fused forward + backward)", "ms_per_step": ms,
                              "segments": plan.chains, "segment_fixups_last_step_by_sweep_kind": fixups,
                              "tuning": tuning, "gflops_per_s": gf, "flops_per_step": flops,
                              "info": int(info[0].item()),
                              "roofline": {"bound": "fp64" if name == "f64" else "fp32", "achieved_tflops": gf / 1e3,
                                           "peak_tflops": pk, "frac": (gf / 1e3) / pk if pk else None,
                                           "peak_source": "measured (microbench/peaks.cu)"},
                              "path": "one thread block per segment, computed window in shared memory, "
                                      "O(l^2) row work spread over 512 threads; segment starts accepted "
                                      "within the state's rounding noise"})
    elif args.config == 4:
        count, n = 256, 50_000
        procs = W.matern_batch(count, n)
        for name, dt in dts.items():
            lay = BT.Layout([2 * n] * count, [3] * count, 1, dt, panels=True)
            plan = BT.Plan(lay)
            Lq = torch.tensor(lay.pack_band([p.Lq for p in procs]), device="cuda", requires_grad=True)
            m = torch.tensor(lay.pack_rhs([p.m[None] for p in procs]), device="cuda", requires_grad=True)
            ells = torch.tensor([p.lengthscale for p in procs], dtype=torch.float64, device="cuda",
                                requires_grad=True)
            prior = LS.MaternPrior(lay, [p.t for p in procs], 1.0)
            wsym, dmask = LS.symmetric_weights(lay), LS.diagonal_mask(lay)

            def step():
                Lq.grad = m.grad = ells.grad = None
                kl = LS.matern_kl(plan, prior, ells, Lq, m, wsym, dmask)
                kl.backward()

            def prior_only():
                e = ells.detach().requires_grad_(True)
                Mp = prior.band(e)
                Mp.sum().backward()
            ms = timed(step, 5)
            ms_prior = timed(prior_only, 5)
            lines.append({"config": f"Matern-3/2 KL, {count} processes x {2 * n} states, l=3, forward + backward "
                          f"in L_q, m and the lengthscales, {name}", "ms_per_step": ms,
                          "ms_prior_construction_fwd_bwd": ms_prior,
                          "band_entries_per_s": count * 2 * n * 4 / (ms * 1e-3),
                          "note": "includes the FP64 torch construction of the prior factor M (flat over all "
                                  "processes) and its backward, timed alone in ms_prior_construction_fwd_bwd"})
    elif args.config == 5:
        # graph GMRF of the spatial workload's size: 11284 nodes, reverse Cuthill-McKee band
        Qg, l, _, _ = W.gmrf_graph(11284)
        n = Qg.shape[1]
        ins = W.make_instance(n, l, 1, W.BASE_SEED)
        ins.Q = Qg
        variants = [(name, None) for name in args.wide_dtypes] + [(name, -1) for name in args.wide_dtypes]
        for name, seg in variants:
            dt = dts[name]
            tuning = {key: v for key, v in (("seg_len", args.seg_len if seg is None else seg),
                                             ("warm_per_l", args.warm_per_l), ("warm_base", args.warm_base)) if v}
            lay = BT.Layout([n], [l], 1, dt)
            plan = BT.Plan(lay, tuning or None)
            dev = {key: torch.from_numpy(pool).cuda() for key, pool in (
                ("Q", lay.pack_band([ins.Q])), ("Sbar", lay.pack_band([ins.Sbar])),
                ("B", lay.pack_rhs([ins.B])), ("Xbar", lay.pack_rhs([ins.Xbar])))}
            L, S, Qb = lay.band_pool(), lay.band_pool(), lay.band_pool()
            X, Bb = lay.rhs_pool(), lay.rhs_pool()
            ld = torch.empty(1, dtype=torch.float64, device="cuda")
            info = torch.empty(1, dtype=torch.int32, device="cuda")
            ldb = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")

            def step():
                B.banded_gmm_forward(plan.handle, dev["Q"], dev["B"], L, X, S, ld, info)
                B.banded_gmm_backward(plan.handle, L, X, S, dev["Xbar"], dev["Sbar"], ldb, Qb, Bb)
            ms = timed(step, 5)
            fixups = [B.bnd_plan_fixups(plan.handle, kk) for kk in range(6)]
            flops = 9.0 * n * l * l
            pk = peaks.get("fp64_fma_tflops" if name == "f64" else "fp32_fma_tflops")
            gf = flops / (ms * 1e-3) / 1e9
            lines.append({"config": f"graph GMRF, {n} nodes (random geometric graph, kappa^2 I + Laplacian), "
                          f"reverse Cuthill-McKee band l={l}, 1 RHS, {name}: fused forward + backward",
                          "ms_per_step": ms, "segments": plan.chains,
                          "segment_fixups_last_step_by_sweep_kind": fixups, "tuning": tuning,
                          "gflops_per_s": gf, "info": int(info[0].item()),
                          "roofline": {"bound": "fp64" if name == "f64" else "fp32", "achieved_tflops": gf / 1e3,
                                       "peak_tflops": pk, "frac": (gf / 1e3) / pk if pk else None}})
    for line in lines:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: a batch of --count instances per GPU; strong: one batch split over the GPUs")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--copy-streams", type=int, default=1, help="end-to-end: copy streams per direction")
    ap.add_argument("--seg-len", type=int, default=0, help="rows per segment (0: the library default)")
    ap.add_argument("--warm", type=int, default=0, help="warm-up rows (0: per-bandwidth default)")
    ap.add_argument("--flags", type=int, default=0, help="plan tuning flags (see bnd_tuning)")
    ap.add_argument("--warm-per-l", type=int, default=0, help="warm-up rows per unit of bandwidth (0: default)")
    ap.add_argument("--warm-base", type=int, default=0, help="warm-up rows added to warm_per_l * l")
    ap.add_argument("--ls", default="1,2,3,5,7", help="bandwidths drawn uniformly (profiling cases)")
    ap.add_argument("--layout", default="panels", choices=["panels", "rows"],
                    help="pool arrangement: 32-instance panels (cs = 32) or one contiguous row per diagonal")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--plain", type=int, default=1)
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--cpu-sample", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="choose the segment length by timing candidates on this batch first")
    ap.add_argument("--config", type=int, default=None, choices=[0, 1, 3, 4, 5],
                    help="time another workload configuration instead of the uneven batch")
    ap.add_argument("--wide-ls", type=int, nargs="+", default=[64, 128], help="bandwidths of --config 3")
    ap.add_argument("--wide-dtypes", nargs="+", default=["f32", "f64"], help="dtypes of --config 3")
    ap.add_argument("--wide-n", type=int, default=200_000, help="rows of --config 3 (smaller: profiling cases)")
    ap.add_argument("--profile-once", action="store_true",
                    help="run one forward and one backward call in NVTX ranges (for ncu) and exit")
    ap.add_argument("--summarize-ncu", default=None, help="ncu --csv file of one backward call -> profiles/")
    ap.add_argument("--summarize-entries", type=int, default=0, help="band entries of the captured case")
    ap.add_argument("--summarize-cmd", default="", help="the capture command, recorded with the summary")
    args = ap.parse_args()
    if args.summarize_ncu:
        summarize_ncu(args)
        return
    if args.config is not None:
        run_config(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        for _ in range(max(args.warmup, 0)):
            cpu_baseline(args, sample_count=max(8, args.cpu_sample // 8))
        cb = None
        for _ in range(args.steps):
            cb, dt, _ = cpu_baseline(args, sample_count=max(8, args.cpu_sample // 8))
            steps.append(dt)
        line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(steps), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "step": "bounded sample of the batch per step"},
                "impl": "reference", "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample", "value")},
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    r = run_ours(args, rank, world, local)
    if rank != 0 or r is None:
        return
    peaks, peak_kind = measured_peaks()
    lay = r["lay"]
    entries_all = r["entries_all"]
    scaling = args.scaling
    value = entries_all / (r["ms"] * 1e-3)
    # dominant fused call and its algorithmic bytes per launch
    if r["ms_bwd"] >= r["ms_fwd"]:
        dom, dom_ms, dom_bytes = "banded_gmm_backward", r["ms_bwd"], r["bwd_bytes"]
    else:
        dom, dom_ms, dom_bytes = "banded_gmm_forward", r["ms_fwd"], r["fwd_bytes"]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    step_gbs = (r["fwd_bytes"] + r["bwd_bytes"]) / (r["ms"] * 1e-3) / 1e9
    cb = parity = None
    if not args.no_cpu_baseline:
        cb, _, parity = cpu_baseline(args, gpu_out=r["sample_out"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": scaling,
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "layout": LAYOUT_NOTE[args.layout],
                   "instances_per_gpu": lay.count, "band_entries_per_gpu": r["entries"],
                   "rows_per_gpu": int(sum(lay.ns)), "k": lay.k, "seg_len": args.seg_len or ("library default: 384" if args.layout == "panels" else "library default: 2048"), "warmup_rows": args.warm or (f"{args.warm_per_l} l + {args.warm_base}" if args.warm_per_l else "library default"),
                   "chains": r["plan"].chains, "warp_tasks": r["plan"].tasks, "graph": True,
                   "l2": "inputs (~%.1f GB) exceed L2; no flush" % (r["h2d"] / 1e9),
                   "parallelism": (f"one batch of {args.count} instances split by shard.partition (strong), "
                                   f"dp{world}" if scaling == "strong" else
                                   f"a batch of {args.count} instances per GPU (weak), dp{world}"),
                   "segment_fixups": r["fixups"]},
        "e2e": {"value": entries_all / (r["ms_e2e"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"], "ms_per_step": r["ms_e2e"],
                "note": "public API calls; every step copies all its inputs in from pinned host memory and all "
                        "its results out to pinned host memory; steps pipelined over two buffer sets (inputs "
                        "of step i+1 and results of step i-1 cross while step i computes)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": stored_traffic(dom, r["entries"]),
                     "traffic_note": "DRAM read+write bytes per call from the committed ncu summary "
                                     "(profiles/gmm_backward_traffic.json), scaled by band entries; "
                                     "null when the CUDA sources changed since the capture",
                     "peak_source": f"{peak_kind} hbm_gbs", "ms_per_launch": dom_ms,
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "step_gbs": step_gbs, "step_frac": step_gbs / peaks["hbm_gbs"],
                     "fused_floor_frac": r["floor_bytes"] / (r["ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "ms_forward": r["ms_fwd"], "ms_backward": r["ms_bwd"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "cpu_baseline": cb,
        "parity": parity,
    }
    if r["autotuned"] is not None:
        line["config"]["autotuned"] = r["autotuned"]
    if r["plain"] is not None:
        line["plain"] = r["plain"]
        line["batched_vs_plain"] = value / r["plain"]["value"]
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
