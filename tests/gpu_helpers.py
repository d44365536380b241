"""Shared helpers of the GPU parity tests (inputs, packing, comparisons)."""
import numpy as np
import torch

from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300 import workloads as W

# Tolerances (normwise: max |gpu - oracle| / max |oracle| per array per instance).
# FP64: the method is exact; both sides round differently -> 1e-10.
# FP32: forward arrays and log-det 1e-4, gradients 1e-3 (inputs are rounded to
# FP32 first and the oracle is fed the same rounded values).
TOL = {
    B.BND_F64: dict(fwd=1e-10, logdet=1e-10, grad=1e-10),
    B.BND_F32: dict(fwd=1e-4, logdet=1e-4, grad=1e-3),
}

MIXED = [(1, 1), (2, 2), (3, 1), (5, 3), (17, 2), (100, 7), (1000, 5), (2500, 3), (4100, 8), (777, 1),
         (64, 4), (300, 6), (9, 7), (2049, 2)]

# Panel batches: runs of equal l form groups of up to 32 lanes.  A full group
# plus a partial one (l = 2, 35 instances), lanes of very different n inside
# a group (n = 1 next to n = 4100), single-lane groups, and bandwidths of the
# generic path (l = 0, 12).  Ordered by (l, -n) as panel_order does.
PANEL_MIX = sorted([(1, 1), (2, 1), (3, 1), (300, 1), (1000, 1), (4100, 1)]
                   + [(5 + 97 * i, 2) for i in range(35)]
                   + [(2500, 3), (2400, 3), (17, 3), (1000, 5), (999, 5), (64, 5), (9, 7), (100, 7), (300, 7),
                      (4100, 8), (2049, 8), (50, 12), (300, 12), (7, 0)],
                   key=lambda s: (s[1], -s[0]))
ARRANGEMENTS = ["rows", "panels"]


def shapes_for(arr):
    return MIXED if arr == "rows" else PANEL_MIX


def rounded(a, dtype):
    return np.asarray(a, dtype=BT.NP_DT[dtype]).astype(np.float64)


def make_instances(shapes, k, seed=1000, dtype=B.BND_F32):
    insts = [W.make_instance(n, l, k, seed + i) for i, (n, l) in enumerate(shapes)]
    for ins in insts:
        ins.Q = rounded(ins.Q, dtype)
        ins.B = rounded(ins.B, dtype)
        ins.Xbar = rounded(ins.Xbar, dtype)
        ins.Sbar = rounded(ins.Sbar, dtype)
    return insts


def setup(shapes, k, dtype, tuning=None, extra_rows=0, seed=1000, arr="rows"):
    """Instances, layout and bound plan; `arr` picks the pool arrangement and
    the plan must recognise it (rows, or 32-lane panels)."""
    insts = make_instances(shapes, k, seed, dtype)
    panels = arr == "panels"
    lay = BT.Layout([s[0] for s in shapes], [s[1] for s in shapes], k, dtype, extra_rows=extra_rows, panels=panels)
    plan = BT.Plan(lay, tuning)
    want = B.LAYOUT_PANELS if panels else B.LAYOUT_ROWS
    assert B.bnd_plan_layout(plan.handle) == want, "plan arrangement"
    return insts, lay, plan


def dev(lay, host):
    return lay.to_device(host)


def relerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 0.0
    num = np.max(np.abs(a - b)) if b.size else 0.0
    return float(num / den) if den > 0 else float(num)


def assert_close(name, got, ref, tol):
    e = relerr(got, ref)
    assert e <= tol, f"{name}: normwise error {e:.3e} > {tol:.1e}"
    return e


def sync():
    torch.cuda.synchronize()
