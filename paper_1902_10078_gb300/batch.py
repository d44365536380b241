"""Pooled HBM layout of a batch of banded instances, and plan ownership.

A batch of ``count`` instances (order n_i, bandwidth l_i, k right-hand sides)
lives in two kinds of pools, in one of two arrangements:

* rows (``panels=False``): instance i occupies ``rows_i * ld_i`` elements of a
  band pool from ``band_i``; row d (a diagonal, Sec. 4.3 storage) is
  contiguous; ``ld_i = round_up(n_i, align)`` and every offset is a multiple
  of ``align`` elements.  RHS pools: ``k * ldr_i`` elements from ``rhs_i``,
  column r contiguous.
* panels (``panels=True``): consecutive instances of equal bandwidth form
  groups of up to 32; lane p of a group stores element (d, j) at
  ``band_g + p + d * ld_g + 32 j`` (column stride 32), so column j of the
  group's 32 instances is 32 adjacent elements.  ``ld_g = 32 * N_g`` with
  ``N_g`` the group's largest n rounded up to 4.  Order the instances with
  ``panel_order`` so that groups are full and their n are close.

``rows`` is ``l_i + 1 + extra_rows`` (``extra_rows`` > 0 leaves room for
product operands with a wider band).  Host-side packing helpers move numpy
arrays in and out of pools; they are plumbing, not arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

TORCH_DT = {B.BND_F32: torch.float32, B.BND_F64: torch.float64}
NP_DT = {B.BND_F32: np.float32, B.BND_F64: np.float64}
PANEL_LANES = 32


def _round_up(x, a):
    return (x + a - 1) // a * a


def panel_order(ns, ls):
    """Instance order that fills panel groups: by bandwidth, then longest first."""
    return sorted(range(len(ns)), key=lambda i: (int(ls[i]), -int(ns[i]), i))


class Layout:
    def __init__(self, ns, ls, k: int, dtype: int = B.BND_F32, extra_rows: int = 0, align: int = 32,
                 panels: bool = False):
        self.ns = [int(n) for n in ns]
        self.ls = [int(l) for l in ls]
        self.count = len(self.ns)
        self.k = int(k)
        self.dtype = dtype
        self.extra_rows = int(extra_rows)
        self.align = int(align)
        self.panels = bool(panels)
        self.rows = [l + 1 + self.extra_rows for l in self.ls]
        self.cs = PANEL_LANES if self.panels else 1
        kk = max(self.k, 1)
        self.band_off, self.rhs_off, self.ld = [], [], []
        self.group, self.lane, self.groups = [], [], []     # panels: group id / lane of each instance
        ob = orr = 0
        if not self.panels:
            for i in range(self.count):
                ld = _round_up(self.ns[i], align)
                self.ld.append(ld)
                self.band_off.append(ob)
                self.rhs_off.append(orr)
                ob += self.rows[i] * ld
                orr += kk * ld
        else:
            i = 0
            while i < self.count:
                j = i
                while j < self.count and j - i < PANEL_LANES and self.ls[j] == self.ls[i]:
                    j += 1
                ng = _round_up(max(self.ns[i:j]), 4)
                ld = PANEL_LANES * ng
                g = len(self.groups)
                self.groups.append((i, j, ob, orr, ng))
                for q in range(i, j):
                    self.ld.append(ld)
                    self.band_off.append(ob + (q - i))
                    self.rhs_off.append(orr + (q - i))
                    self.group.append(g)
                    self.lane.append(q - i)
                ob = _round_up(ob + self.rows[i] * ld, align)
                orr = _round_up(orr + kk * ld, align)
                i = j
        self.band_elems = max(ob, 1)
        self.rhs_elems = max(orr, 1)

    @property
    def torch_dtype(self):
        return TORCH_DT[self.dtype]

    @property
    def np_dtype(self):
        return NP_DT[self.dtype]

    def insts(self):
        return [dict(n=self.ns[i], l=self.ls[i], band=self.band_off[i], ld=self.ld[i],
                     rhs=self.rhs_off[i], ldr=self.ld[i], cs=self.cs) for i in range(self.count)]

    # --- views of one instance inside a flat pool (numpy array or tensor) ---
    def band_view(self, pool, i):
        """(rows_i, n_i) strided view of instance i's band region."""
        n, rows, ld = self.ns[i], self.rows[i], self.ld[i]
        if not self.panels:
            o = self.band_off[i]
            return pool[o:o + rows * ld].reshape(rows, ld)[:, :n]
        _, _, ob, _, ng = self.groups[self.group[i]]
        return pool[ob:ob + rows * ld].reshape(rows, ng, PANEL_LANES)[:, :n, self.lane[i]]

    def rhs_view(self, pool, i):
        """(k, n_i) strided view of instance i's RHS block."""
        n, ld, kk = self.ns[i], self.ld[i], max(self.k, 1)
        if not self.panels:
            o = self.rhs_off[i]
            return pool[o:o + kk * ld].reshape(kk, ld)[:, :n]
        _, _, _, orr, ng = self.groups[self.group[i]]
        return pool[orr:orr + kk * ld].reshape(kk, ng, PANEL_LANES)[:, :n, self.lane[i]]

    # --- pools -------------------------------------------------------------
    def band_pool(self, device="cuda", fill=0.0):
        return torch.full((self.band_elems,), fill, dtype=self.torch_dtype, device=device)

    def rhs_pool(self, device="cuda", fill=0.0):
        return torch.full((self.rhs_elems,), fill, dtype=self.torch_dtype, device=device)

    def pack_band(self, arrays, fill=0.0) -> np.ndarray:
        """arrays[i]: (r_i, n_i) with r_i <= rows_i -> flat host pool."""
        pool = np.full(self.band_elems, fill, dtype=self.np_dtype)
        for i, a in enumerate(arrays):
            a = np.asarray(a)
            self.band_view(pool, i)[: a.shape[0]] = a
        return pool

    def unpack_band(self, pool, rows=None):
        pool = pool.detach().cpu().numpy() if isinstance(pool, torch.Tensor) else pool
        out = []
        for i in range(self.count):
            r = self.ls[i] + 1 if rows is None else rows
            out.append(np.array(self.band_view(pool, i)[:r], dtype=np.float64))
        return out

    def pack_rhs(self, arrays, fill=0.0) -> np.ndarray:
        pool = np.full(self.rhs_elems, fill, dtype=self.np_dtype)
        for i, a in enumerate(arrays):
            a = np.asarray(a)
            a = a[None] if a.ndim == 1 else a
            self.rhs_view(pool, i)[: a.shape[0]] = a
        return pool

    def unpack_rhs(self, pool):
        pool = pool.detach().cpu().numpy() if isinstance(pool, torch.Tensor) else pool
        return [np.array(self.rhs_view(pool, i)[: self.k], dtype=np.float64) for i in range(self.count)]

    def to_device(self, host: np.ndarray, device="cuda"):
        return torch.from_numpy(host).to(device)


class Plan:
    """Owns a C-ABI plan and the device workspace bound to it."""

    def __init__(self, layout: Layout, tuning=None, device="cuda", stream=None):
        self.layout = layout
        self.handle = B.bnd_plan_create(layout.dtype, layout.insts(), layout.k, tuning)
        self.ws_bytes = B.bnd_plan_workspace_bytes(self.handle)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        B.bnd_plan_bind(self.handle, self.ws, self.ws_bytes, stream)
        self.chains = B.bnd_plan_chains(self.handle)
        self.tasks = B.bnd_plan_tasks(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.bnd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Autotuning of the schedule
# ---------------------------------------------------------------------------

def workload_signature(layout) -> str:
    """Key of a batch for the tuning cache: dtype, arrangement, k and a coarse
    histogram of (bandwidth, log2 n) over the instances."""
    import collections
    import math
    hist = collections.Counter((l, int(math.log2(max(n, 1)))) for n, l in zip(layout.ns, layout.ls))
    parts = [f"dt{layout.dtype}", "panels" if layout.panels else "rows", f"k{layout.k}"]
    parts += [f"l{l}n{b}x{c}" for (l, b), c in sorted(hist.items())]
    return ";".join(parts)


def _cache_path():
    import os
    return os.environ.get("BND_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_1902_10078_gb300", "autotune.json"))


def _cuda_timer(fn, reps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


# Default candidates: the library defaults, segment length x warm-up slope (rows
# per unit of bandwidth, plus 32), the direct kernels at the library defaults,
# and no segmentation at all (for inputs whose cold starts converge too slowly:
# every segment would be rerun after the parallel pass).
DEFAULT_CANDIDATES = tuple(
    [dict()]
    + [dict(seg_len=s, warm_per_l=w, warm_base=32) for s in (256, 384, 512, 768) for w in (12, 16, 24)]
    + [dict(flags=1), dict(seg_len=-1)])


def _candidate_key(c):
    return ",".join(f"{k}={c[k]}" for k in sorted(c)) or "library defaults"


def autotune(layout, make_step, candidates=DEFAULT_CANDIDATES, reps=3, warmup=2, use_cache=True,
             plan_factory=None, timer=None):
    """Choose the schedule of a batch by timing one step per candidate.

    A candidate is a tuning dict (segment length, warm-up slope, flags: staged
    or direct kernels) or a bare segment length.  `make_step(plan)` returns a
    callable that runs one step of the caller's workload on `plan`.  Each
    candidate gets its own plan; the fastest tuning is returned (with the
    timings by candidate) and stored in a JSON cache keyed by
    `workload_signature` (path: $BND_AUTOTUNE_CACHE, default
    ~/.cache/paper_1902_10078_gb300/autotune.json), which later calls consult
    first.  `plan_factory` and `timer` replace Plan construction and
    CUDA-event timing (tests)."""
    import json
    import os
    key = workload_signature(layout)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key]["tuning"]), cache[key].get("timings", {})
    plan_factory = plan_factory or (lambda tuning: Plan(layout, tuning))
    timer = timer or _cuda_timer
    timings, by_key = {}, {}
    for cand in candidates:
        tuning = dict(seg_len=int(cand)) if not isinstance(cand, dict) else dict(cand)
        k = _candidate_key(tuning)
        plan = plan_factory(tuning)
        try:
            timings[k] = float(timer(make_step(plan), reps, warmup))
            by_key[k] = tuning
        finally:
            close = getattr(plan, "close", None)
            if close:
                close()
    best = min(timings, key=timings.get)
    if use_cache:
        cache[key] = {"tuning": by_key[best], "timings": timings}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(by_key[best]), timings
