"""GPU: segmentation, edge cases and failure reporting.

* Splitting instances into speculative segments must not change any output:
  after the verify/fixup pass every band and RHS output of the register-window
  bandwidths (l <= 8) is bitwise equal to the unsplit run (only the log-det,
  summed per segment, may differ in its last bits).  Wide bands accept a
  segment start within the rounding noise of the state: their outputs agree
  with the unsplit run to a few ulps of each output's largest entry.  A
  one-row warm-up forces the fixup path (then bitwise equal for all widths).
* Degenerate shapes (n = 1, n <= l, l = 0 and bandwidths above the
  register-window limit) agree with the oracle.
* Undefined corners of the inputs are never read (NaN there changes nothing)
  and are written as 0.
* A non-SPD instance reports info = first failing row + 1 while the other
  instances are unaffected.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import ARRANGEMENTS, TOL, assert_close, dev, setup, sync
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300.workloads import zero_corners

pytestmark = pytest.mark.gpu

LONG = [(6000, 1), (5000, 3), (7001, 7), (4500, 2), (3333, 5), (300, 4), (4096, 8)]
# panels: several lanes per group, lanes that end segments early or are idle in later ones
LONG_PANELS = sorted([(6000, 1), (5900, 1), (100, 1), (5000, 3), (4999, 3), (7001, 7), (6000, 7), (3333, 5),
                      (4096, 8), (4500, 2), (4000, 2), (300, 4), (1, 4)], key=lambda s: (s[1], -s[0]))


def long_for(arr):
    return LONG if arr == "rows" else LONG_PANELS


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()


def run_gmm(lay, plan, insts, pad=0.0, out_fill=0.0):
    """Fused forward + backward; `pad` fills the input pools outside the
    instances, `out_fill` pre-fills the output pools."""
    Q = dev(lay, lay.pack_band([i.Q for i in insts], fill=pad))
    Bp = dev(lay, lay.pack_rhs([i.B for i in insts], fill=pad))
    L, S, X = lay.band_pool(fill=out_fill), lay.band_pool(fill=out_fill), lay.rhs_pool(fill=out_fill)
    logdet = torch.empty(lay.count, dtype=torch.float64, device="cuda")
    info = torch.empty(lay.count, dtype=torch.int32, device="cuda")
    B.banded_gmm_forward(plan.handle, Q, Bp, L, X, S, logdet, info)
    Xb = dev(lay, lay.pack_rhs([i.Xbar for i in insts], fill=pad))
    Sb = dev(lay, lay.pack_band([i.Sbar for i in insts], fill=pad))
    ldb = torch.full((lay.count,), 0.5, dtype=torch.float64, device="cuda")
    Qb, Bb = lay.band_pool(fill=out_fill), lay.rhs_pool(fill=out_fill)
    B.banded_gmm_backward(plan.handle, L, X, S, Xb, Sb, ldb, Qb, Bb)
    sync()
    return dict(L=L, S=S, X=X, Qb=Qb, Bb=Bb, logdet=logdet.cpu().numpy(), info=info.cpu().numpy())


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F32, B.BND_F64])
@pytest.mark.parametrize("warm", [0, 1])
@pytest.mark.parametrize("flags", [0, 1])
def test_segmented_is_bitwise_equal_to_whole(dtype, warm, flags, arr):
    # staged (flags 0) and direct (flags 1) kernels run the same arithmetic: bitwise equal to each other too
    shapes = long_for(arr)
    insts, lay, whole = setup(shapes, 4, dtype, dict(seg_len=-1, flags=1), arr=arr)
    ref = run_gmm(lay, whole, insts)
    _, _, seg = setup(shapes, 4, dtype, dict(seg_len=512, warmup=warm, flags=flags), arr=arr)
    assert seg.chains > lay.count
    got = run_gmm(lay, seg, insts)
    for key in ("L", "S", "X", "Qb", "Bb"):
        assert torch.equal(got[key], ref[key]), f"{key} differs between segmented and whole runs"
    assert np.all(got["info"] == 0)
    # the log-det is summed per segment: FP32 sums (compensated) may differ in the last bits
    assert np.allclose(got["logdet"], ref["logdet"], rtol=1e-12 if dtype == B.BND_F64 else 2e-6, atol=0)
    if warm == 1:
        # a one-row warm-up cannot converge: the verify pass must have rerun segments
        assert sum(B.bnd_plan_fixups(seg.handle, kind) for kind in range(4)) > 0


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_degenerate_shapes(dtype, arr):
    shapes = [(1, 1), (1, 7), (2, 5), (3, 3), (4, 0), (40, 0), (50, 12), (23, 9), (200, 16), (8, 30)]
    insts, lay, plan = setup(shapes, 2, dtype, dict(seg_len=-1), arr=arr)
    got = run_gmm(lay, plan, insts)
    res, _ = O.batch_step(insts)
    tol = TOL[dtype]
    Lg, Sg, Qg = lay.unpack_band(got["L"]), lay.unpack_band(got["S"]), lay.unpack_band(got["Qb"])
    Xg, Bg = lay.unpack_rhs(got["X"]), lay.unpack_rhs(got["Bb"])
    for c, r in enumerate(res):
        assert got["info"][c] == 0
        assert_close("L", Lg[c], r["L"], tol["fwd"])
        assert_close("S", Sg[c], r["S"], tol["fwd"])
        assert_close("X", Xg[c], r["X"], tol["fwd"])
        assert_close("Qbar", Qg[c], r["Qbar"], tol["grad"])
        assert_close("Bbar", Bg[c], r["Bbar"], tol["grad"])
        assert abs(got["logdet"][c] - r["logdet"]) <= tol["logdet"] * max(1, abs(r["logdet"]))


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F32, B.BND_F64])
def test_corners_never_read_and_written_zero(dtype, arr):
    shapes = [(50, 3), (9, 3), (700, 5), (3000, 2), (2999, 2)]
    insts, lay, plan = setup(shapes, 1, dtype, dict(seg_len=256, warmup=64), arr=arr)
    for ins in insts:
        zero_corners(ins.Q, fill=np.nan)
        zero_corners(ins.Sbar, fill=np.nan)
    got = run_gmm(lay, plan, insts)
    for ins in insts:                         # the oracle sees zeros in the corners
        zero_corners(ins.Q)
        zero_corners(ins.Sbar)
    res, _ = O.batch_step(insts)
    for key, ref_key in (("L", "L"), ("S", "S"), ("Qb", "Qbar")):
        arrs = lay.unpack_band(got[key])
        for c, r in enumerate(res):
            a = arrs[c]
            assert np.all(np.isfinite(a)), key
            for d in range(1, a.shape[0]):
                assert np.all(a[d, a.shape[1] - d:] == 0.0), f"{key} corner not zero"
            assert_close(key, a, r[ref_key], TOL[dtype]["grad"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
@pytest.mark.parametrize("tune", [dict(seg_len=-1), dict(seg_len=128, warmup=32)])
def test_not_spd_reports_info(dtype, tune, arr):
    shapes = [(600, 3), (800, 3), (500, 3)]
    insts, lay, plan = setup(shapes, 1, dtype, tune, arr=arr)
    insts[1].Q[0, 437] = -50.0          # instance 1 fails at row 437 at the latest
    Lo, inf = O.cholesky(insts[1].Q)
    assert inf > 0
    Q = dev(lay, lay.pack_band([i.Q for i in insts]))
    L = lay.band_pool()
    logdet = torch.empty(lay.count, dtype=torch.float64, device="cuda")
    info = torch.empty(lay.count, dtype=torch.int32, device="cuda")
    B.banded_cholesky(plan.handle, Q, L, logdet, info)
    sync()
    info = info.cpu().numpy()
    assert info[0] == 0 and info[2] == 0
    assert info[1] == inf
    assert np.isnan(float(logdet[1]))
    Lg = lay.unpack_band(L)
    good = inf - 1
    assert_close("rows before the failure", Lg[1][:, : max(good - 3, 1)], Lo[:, : max(good - 3, 1)],
                 TOL[dtype]["fwd"])
    for c in (0, 2):
        assert_close("unaffected instance", Lg[c], O.cholesky(insts[c].Q)[0], TOL[dtype]["fwd"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F32, B.BND_F64])
@pytest.mark.parametrize("tune", [dict(seg_len=-1), dict(seg_len=256, warmup=64)])
def test_padding_never_read_nor_written(dtype, arr, tune):
    """Pool elements outside every instance (row padding, absent or shorter
    panel lanes) hold NaN on input and a sentinel on output: the results
    match the oracle and the sentinel survives everywhere outside."""
    shapes = [(3000, 2), (2999, 2), (17, 2), (1, 2), (700, 5), (650, 5), (9, 3)]
    insts, lay, plan = setup(shapes, 3, dtype, tune, arr=arr)
    sentinel = 7.25
    got = run_gmm(lay, plan, insts, pad=np.nan, out_fill=sentinel)
    res, _ = O.batch_step(insts)
    inside_b = np.zeros(lay.band_elems, bool)
    inside_r = np.zeros(lay.rhs_elems, bool)
    for i in range(lay.count):
        lay.band_view(inside_b, i)[: lay.ls[i] + 1] = True
        lay.rhs_view(inside_r, i)[: lay.k] = True
    for key, inside in (("L", inside_b), ("S", inside_b), ("Qb", inside_b), ("X", inside_r), ("Bb", inside_r)):
        a = got[key].cpu().numpy()
        assert np.all(a[~inside] == sentinel), f"{key}: a write landed outside the instances"
    tol = TOL[dtype]
    for key, ref_key, unpack, t in (("L", "L", lay.unpack_band, "fwd"), ("S", "S", lay.unpack_band, "fwd"),
                                    ("Qb", "Qbar", lay.unpack_band, "grad"), ("X", "X", lay.unpack_rhs, "fwd"),
                                    ("Bb", "Bbar", lay.unpack_rhs, "grad")):
        arrs = unpack(got[key])
        for c, r in enumerate(res):
            assert np.all(np.isfinite(arrs[c])), key
            assert_close(key, arrs[c], r[ref_key], tol[t])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_wide_bands_warp_kernel(dtype, arr):
    """Bandwidths above the register-window limit, whole instances on the
    block kernels (one thread block per instance, windows in shared memory):
    the fused step agrees with the oracle at l = 40, 64, 128."""
    shapes = [(3000, 64), (1500, 128), (700, 40), (130, 128)]
    insts, lay, plan = setup(shapes, 4, dtype, dict(seg_len=-1), arr=arr)
    got = run_gmm(lay, plan, insts)
    res, _ = O.batch_step(insts)
    tol = TOL[dtype]
    Lg, Sg, Qg = lay.unpack_band(got["L"]), lay.unpack_band(got["S"]), lay.unpack_band(got["Qb"])
    Xg, Bg = lay.unpack_rhs(got["X"]), lay.unpack_rhs(got["Bb"])
    for c, r in enumerate(res):
        assert got["info"][c] == 0
        assert_close("L", Lg[c], r["L"], tol["fwd"])
        assert_close("S", Sg[c], r["S"], tol["fwd"])
        assert_close("X", Xg[c], r["X"], tol["fwd"])
        assert_close("Qbar", Qg[c], r["Qbar"], tol["grad"])
        assert_close("Bbar", Bg[c], r["Bbar"], tol["grad"])
        assert abs(got["logdet"][c] - r["logdet"]) <= tol["logdet"] * max(1, abs(r["logdet"]))


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", [B.BND_F32, B.BND_F64])
@pytest.mark.parametrize("warm", [0, 1])
def test_wide_bands_segmented(dtype, warm, arr):
    """Wide bands cut into segments on the block kernels.  With the default
    warm-up the segment starts are accepted within the rounding noise of the
    state (above l of about 50 a cold start never meets the exact state bit for
    bit): few reruns, and every output within a few ulps of its largest entry
    of the whole-instance run.  A one-row warm-up makes the verify pass rerun
    the segments from the exact state: then bitwise equal."""
    shapes = [(3000, 40), (2600, 64), (1900, 12), (700, 9), (2400, 100)]
    shapes = sorted(shapes, key=lambda s: (s[1], -s[0])) if arr == "panels" else shapes
    insts, lay, whole = setup(shapes, 4, dtype, dict(seg_len=-1), arr=arr)
    tuning = dict(seg_len=500) if warm == 0 else dict(seg_len=500, warmup=1)
    _, _, seg = setup(shapes, 4, dtype, tuning, arr=arr)
    boundaries = seg.chains - whole.chains
    assert boundaries > 0
    a = run_gmm(lay, whole, insts)
    b = run_gmm(lay, seg, insts)
    fixups = sum(B.bnd_plan_fixups(seg.handle, kk) for kk in range(6))
    if warm:
        assert fixups > 0                      # the one-row warm-up really forced reruns
        for key in ("L", "S", "X", "Qb", "Bb"):
            assert torch.equal(a[key], b[key]), key
    else:
        # the gmm step runs four sweeps, each with `boundaries` boundaries
        assert fixups <= max(1, boundaries // 2), (fixups, boundaries)
        rel = 2.0 ** -13 if dtype == B.BND_F32 else 2.0 ** -40
        for key, unpack in (("L", lay.unpack_band), ("S", lay.unpack_band), ("X", lay.unpack_rhs),
                            ("Qb", lay.unpack_band), ("Bb", lay.unpack_rhs)):
            for c, (u, v) in enumerate(zip(unpack(a[key]), unpack(b[key]))):
                scale = np.abs(u).max()
                assert np.abs(u - v).max() <= rel * scale, (key, c, np.abs(u - v).max() / scale)
    assert np.array_equal(a["info"], b["info"])
    assert np.allclose(a["logdet"], b["logdet"], rtol=1e-12 if dtype == B.BND_F64 else 1e-6)
    res, _ = O.batch_step(insts)
    tol = TOL[dtype]
    Lg, Qg = lay.unpack_band(b["L"]), lay.unpack_band(b["Qb"])
    for c, r in enumerate(res):
        assert_close("L", Lg[c], r["L"], tol["fwd"])
        assert_close("Qbar", Qg[c], r["Qbar"], tol["grad"])


@pytest.mark.parametrize("k", [1, 3])
def test_wide_band_fp64_few_rhs_on_the_block_kernel(k):
    """The block kernels size their RHS windows for the plan's k: FP64 at l = 160
    fits one block with up to a few right-hand sides (with 16 it would not).
    The fused step agrees with the oracle, whole and segmented."""
    shapes = [(1500, 160)]
    tol = TOL[B.BND_F64]
    for tuning in (dict(seg_len=-1), dict(seg_len=400, warmup=16)):
        insts, lay, plan = setup(shapes, k, B.BND_F64, tuning)
        got = run_gmm(lay, plan, insts)
        res, _ = O.batch_step(insts)
        r = res[0]
        assert got["info"][0] == 0
        assert_close("L", lay.unpack_band(got["L"])[0], r["L"], tol["fwd"])
        assert_close("S", lay.unpack_band(got["S"])[0], r["S"], tol["fwd"])
        assert_close("X", lay.unpack_rhs(got["X"])[0], r["X"], tol["fwd"])
        assert_close("Qbar", lay.unpack_band(got["Qb"])[0], r["Qbar"], tol["grad"])
        assert_close("Bbar", lay.unpack_rhs(got["Bb"])[0], r["Bbar"], tol["grad"])
        assert abs(got["logdet"][0] - r["logdet"]) <= tol["logdet"] * max(1, abs(r["logdet"]))


def run_separate(lay, plan, insts):
    """Forward + backward through the separate operators (any number of RHS):
    C, (L L^T)^{-1} B, I; then the solve, subset-inverse and Cholesky adjoints
    accumulated into one L-bar (Table 1, Alg. 4, Alg. 2 with the log-det term)."""
    Q = dev(lay, lay.pack_band([i.Q for i in insts]))
    Bp = dev(lay, lay.pack_rhs([i.B for i in insts]))
    Xb = dev(lay, lay.pack_rhs([i.Xbar for i in insts]))
    Sb = dev(lay, lay.pack_band([i.Sbar for i in insts]))
    L, S, Lb, Qb = (lay.band_pool() for _ in range(4))
    X, Bb = lay.rhs_pool(), lay.rhs_pool()
    logdet = torch.empty(lay.count, dtype=torch.float64, device="cuda")
    info = torch.empty(lay.count, dtype=torch.int32, device="cuda")
    ldb = torch.full((lay.count,), 0.5, dtype=torch.float64, device="cuda")
    B.banded_cholesky(plan.handle, Q, L, logdet, info)
    B.banded_solve(plan.handle, L, Bp, X, 2)
    B.banded_subset_inverse(plan.handle, L, S)
    B.banded_solve_vjp(plan.handle, L, X, Xb, 2, Bb, Lb, 0)
    B.banded_subset_inverse_vjp(plan.handle, L, S, Sb, Lb, 1)
    B.banded_cholesky_vjp(plan.handle, L, Lb, ldb, Qb, 0)
    sync()
    return dict(L=L, S=S, X=X, Qb=Qb, Bb=Bb, logdet=logdet.cpu().numpy(), info=info.cpu().numpy())


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_wide_bands_sixteen_rhs(dtype):
    """The wide-band workload's shape at a few thousand rows: l = 64 and 128 with
    16 right-hand sides (four RHS blocks per solve), against the oracle."""
    shapes = [(2500, 64), (2000, 128)]
    insts, lay, plan = setup(shapes, 16, dtype, dict(seg_len=-1))
    got = run_separate(lay, plan, insts)
    res, _ = O.batch_step(insts)
    tol = TOL[dtype]
    Lg, Sg, Qg = lay.unpack_band(got["L"]), lay.unpack_band(got["S"]), lay.unpack_band(got["Qb"])
    Xg, Bg = lay.unpack_rhs(got["X"]), lay.unpack_rhs(got["Bb"])
    for c, r in enumerate(res):
        assert got["info"][c] == 0
        assert_close("L", Lg[c], r["L"], tol["fwd"])
        assert_close("S", Sg[c], r["S"], tol["fwd"])
        assert_close("X", Xg[c], r["X"], tol["fwd"])
        assert_close("Qbar", Qg[c], r["Qbar"], tol["grad"])
        assert_close("Bbar", Bg[c], r["Bbar"], tol["grad"])
        assert abs(got["logdet"][c] - r["logdet"]) <= tol["logdet"] * max(1, abs(r["logdet"]))


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_graph_gmrf_reordered(dtype):
    """A random-geometric-graph GMRF (kappa^2 I + Laplacian, 2000 nodes) reordered
    by reverse Cuthill-McKee to bandwidth 85: the fused step on the wide-band
    kernels against the oracle."""
    from paper_1902_10078_gb300 import workloads as W
    from gpu_helpers import rounded
    from paper_1902_10078_gb300 import batch as BT
    Qg, l, _, _ = W.gmrf_graph(2000)
    n = Qg.shape[1]
    ins = W.make_instance(n, l, 4, 2024)
    ins.Q = rounded(Qg, dtype)
    for key in ("B", "Xbar", "Sbar"):
        setattr(ins, key, rounded(getattr(ins, key), dtype))
    lay = BT.Layout([n], [l], 4, dtype)
    plan = BT.Plan(lay)
    got = run_gmm(lay, plan, [ins])
    r = O.batch_step([ins])[0][0]
    tol = TOL[dtype]
    assert got["info"][0] == 0
    assert_close("L", lay.unpack_band(got["L"])[0], r["L"], tol["fwd"])
    assert_close("S", lay.unpack_band(got["S"])[0], r["S"], tol["fwd"])
    assert_close("X", lay.unpack_rhs(got["X"])[0], r["X"], tol["fwd"])
    assert_close("Qbar", lay.unpack_band(got["Qb"])[0], r["Qbar"], tol["grad"])
    assert_close("Bbar", lay.unpack_rhs(got["Bb"])[0], r["Bbar"], tol["grad"])
    assert abs(got["logdet"][0] - r["logdet"]) <= tol["logdet"] * max(1, abs(r["logdet"]))
