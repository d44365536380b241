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


def setup(shapes, k, dtype, tuning=None, extra_rows=0, seed=1000):
    insts = make_instances(shapes, k, seed, dtype)
    lay = BT.Layout([s[0] for s in shapes], [s[1] for s in shapes], k, dtype, extra_rows=extra_rows)
    plan = BT.Plan(lay, tuning)
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
