"""GPU parity at the benchmarked uneven batch itself.

The whole 4096-instance batch (n log-uniform in [1000, 65536], l in
{1, 2, 3, 5, 7}, k = 4, FP32) in the 32-lane panel arrangement, planned with
the library defaults (384-row segments, 16 l + 32 warm-up rows: the launch
configuration bench.py times), runs one fused forward + backward step.
Every instance must factor (info = 0); a sample of instances -- the longest
one of every bandwidth plus a seeded random draw -- is compared element by
element with the FP64 oracle on the same FP32-rounded inputs.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import TOL, assert_close
from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()
    O.lib()


def test_uneven_batch_default_plan_matches_oracle():
    count, k = 4096, 4
    ns, ls = W.batched_shapes(count)
    order = BT.panel_order(ns, ls)
    lay = BT.Layout([int(ns[i]) for i in order], [int(ls[i]) for i in order], k, B.BND_F32, panels=True)
    seeds = [W.BASE_SEED + int(i) for i in order]
    host = W.fill_pools(lay, seeds, workers=8)
    plan = BT.Plan(lay)                                   # library defaults
    assert B.bnd_plan_layout(plan.handle) == B.LAYOUT_PANELS
    assert plan.chains > 4 * count                        # long instances really are segmented
    dev = {key: torch.from_numpy(v).cuda() for key, v in host.items()}
    L, S, Qb = lay.band_pool(), lay.band_pool(), lay.band_pool()
    X, Bb = lay.rhs_pool(), lay.rhs_pool()
    logdet = torch.empty(count, dtype=torch.float64, device="cuda")
    info = torch.empty(count, dtype=torch.int32, device="cuda")
    ldbar = torch.full((count,), 0.5, dtype=torch.float64, device="cuda")
    B.banded_gmm_forward(plan.handle, dev["Q"], dev["B"], L, X, S, logdet, info)
    B.banded_gmm_backward(plan.handle, L, X, S, dev["Xbar"], dev["Sbar"], ldbar, Qb, Bb)
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0

    # sample: the longest instance of every bandwidth, and 24 random slots
    slots = set()
    for l in sorted(set(lay.ls)):
        cand = [p for p in range(count) if lay.ls[p] == l]
        slots.add(max(cand, key=lambda p: lay.ns[p]))
    rng = W.rng_for(2024)
    slots.update(int(p) for p in rng.choice(count, size=24, replace=False))
    slots = sorted(slots)
    assert max(lay.ns[p] for p in slots) >= 60000
    insts = []
    for p in slots:
        ins = W.make_instance(lay.ns[p], lay.ls[p], k, seeds[p])
        for key in ("Q", "B", "Xbar", "Sbar"):
            setattr(ins, key, getattr(ins, key).astype(np.float32).astype(np.float64))
        insts.append(ins)
    res, _ = O.batch_step(insts)
    tol = TOL[B.BND_F32]
    for p, r in zip(slots, res):
        def band(pool):
            return lay.band_view(pool, p)[: lay.ls[p] + 1].cpu().numpy().astype(np.float64)

        def rhs(pool):
            return lay.rhs_view(pool, p).cpu().numpy().astype(np.float64)
        tag = f"slot {p} (n={lay.ns[p]}, l={lay.ls[p]})"
        assert_close(f"{tag} L", band(L), r["L"], tol["fwd"])
        assert_close(f"{tag} S", band(S), r["S"], tol["fwd"])
        assert_close(f"{tag} X", rhs(X), r["X"], tol["fwd"])
        assert_close(f"{tag} Qbar", band(Qb), r["Qbar"], tol["grad"])
        assert_close(f"{tag} Bbar", rhs(Bb), r["Bbar"], tol["grad"])
        assert abs(float(logdet[p]) - r["logdet"]) <= tol["logdet"] * max(1.0, abs(r["logdet"])), tag
