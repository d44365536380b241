"""GPU parity at the wide-band workload itself.

One instance of n = 200000 rows with 16 right-hand sides at l = 64 and 128
(FP32) and l = 64 (FP64), planned with the library defaults: the block
kernels cut it into about 152 segments whose starts are accepted within the
rounding noise of the state (the launch configuration `bench.py --config 3`
times).  One fused forward + backward step is compared element by element
(normwise per output) with the FP64 oracle on the same rounded inputs; no
segment may need a rerun.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import TOL, assert_close, make_instances
from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()
    O.lib()


@pytest.mark.parametrize("l,dtype", [(64, B.BND_F32), (128, B.BND_F32), (64, B.BND_F64)])
def test_wide_band_workload_matches_oracle(l, dtype):
    n, k = 200_000, 16
    ins = make_instances([(n, l)], k, seed=W.BASE_SEED, dtype=dtype)[0]
    lay = BT.Layout([n], [l], k, dtype)
    plan = BT.Plan(lay)                                   # library defaults
    assert plan.chains > 64                               # cut into segments over the SMs
    dev = lambda a: torch.from_numpy(a).cuda()            # noqa: E731
    Q, Bm = dev(lay.pack_band([ins.Q])), dev(lay.pack_rhs([ins.B]))
    L, S, X = lay.band_pool(), lay.band_pool(), lay.rhs_pool()
    logdet = torch.empty(1, dtype=torch.float64, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    B.banded_gmm_forward(plan.handle, Q, Bm, L, X, S, logdet, info)
    fwd_fix = [B.bnd_plan_fixups(plan.handle, kk) for kk in range(6)]
    Xb, Sb = dev(lay.pack_rhs([ins.Xbar])), dev(lay.pack_band([ins.Sbar]))
    ldb = torch.full((1,), float(ins.ldbar), dtype=torch.float64, device="cuda")
    Qb, Bb = lay.band_pool(), lay.rhs_pool()
    B.banded_gmm_backward(plan.handle, L, X, S, Xb, Sb, ldb, Qb, Bb)
    bwd_fix = [B.bnd_plan_fixups(plan.handle, kk) for kk in range(6)]
    torch.cuda.synchronize()
    assert int(info[0]) == 0
    assert sum(fwd_fix) == 0 and sum(bwd_fix) == 0, (fwd_fix, bwd_fix)
    r = O.batch_step([ins])[0][0]
    tol = TOL[dtype]
    assert_close("L", lay.unpack_band(L)[0], r["L"], tol["fwd"])
    assert_close("S", lay.unpack_band(S)[0], r["S"], tol["fwd"])
    assert_close("X", lay.unpack_rhs(X)[0], r["X"], tol["fwd"])
    assert_close("Qbar", lay.unpack_band(Qb)[0], r["Qbar"], tol["grad"])
    assert_close("Bbar", lay.unpack_rhs(Bb)[0], r["Bbar"], tol["grad"])
    assert abs(float(logdet[0]) - r["logdet"]) <= tol["logdet"] * max(1.0, abs(r["logdet"]))
