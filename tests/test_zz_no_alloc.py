"""The allocation-free precision solve against the planned one.

banded_solve_precision_noalloc serves callers that cannot allocate device
memory (not even a workspace): it keeps its one intermediate vector in a fixed
array inside the library.  Here it is called twice in a row through the C ABI
(the second call reuses the array the first one left behind) and each result
is compared with banded_solve (mode 2, planned path) within the tolerances of
the other parity tests.  The file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import TOL, assert_close, dev, rounded, setup, sync
from paper_1902_10078_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
@pytest.mark.parametrize("n,l", [(5000, 3), (777, 8), (300, 12)])
def test_noalloc_matches_planned_solve_twice(dtype, n, l):
    insts, lay, plan = setup([(n, l)], 1, dtype, dict(seg_len=-1))
    Ls = [rounded(O.cholesky(insts[0].Q)[0], dtype)]
    L = dev(lay, lay.pack_band(Ls))
    rng = np.random.Generator(np.random.PCG64(4242))
    for call in range(2):
        bvec = rounded(rng.normal(size=(1, n)), dtype)
        bp = dev(lay, lay.pack_rhs([bvec]))
        ref = lay.rhs_pool(fill=0.0)
        B.banded_solve(plan.handle, L, bp, ref, 2)
        x = torch.full((n,), 7.0, dtype=lay.torch_dtype, device="cuda")
        B.banded_solve_precision_noalloc(dtype, n, l, L, lay.ld[0], bp, x)
        sync()
        got = x.cpu().numpy().astype(np.float64)
        want = lay.unpack_rhs(ref)[0][0]
        assert_close(f"call {call}", got, want, TOL[dtype]["fwd"])
        assert_close(f"call {call} vs oracle", got, O.solve_precision(Ls[0], bvec[0]), TOL[dtype]["fwd"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BandedError) as e:
        B.banded_solve_precision_noalloc(B.BND_F64, (1 << 21) + 1, 2, x, (1 << 21) + 1, x[:4], x[4:])
    assert e.value.status == 1
