"""GPU parity: every operator of the C ABI against the FP64 oracle.

Inputs are seeded synthetic SPD bands (workloads.py), rounded to the tested
dtype before both sides see them.  Batches mix bandwidths 0..12, ragged n
(1, 2, 3, 5, 17, ... 4100) and run both as whole chains and split into
segments (speculative starts + verify/fixup), so several tiles, segment
boundaries and ragged tails are covered.  Every operator runs on both pool
arrangements: contiguous rows (cs = 1) and 32-lane panels (cs = 32), the
latter with full, partial and single-lane groups.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import ARRANGEMENTS, TOL, assert_close, dev, rounded, setup, shapes_for, sync
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300.workloads import zero_corners

pytestmark = pytest.mark.gpu

DTYPES = [B.BND_F64, B.BND_F32]
TUNINGS = {"whole": dict(seg_len=-1), "seg": dict(seg_len=256, warmup=64),
           "direct": dict(seg_len=256, warmup=64, flags=1)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def oracle_L(insts, dtype):
    return [rounded(O.cholesky(i.Q)[0], dtype) for i in insts]


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
def test_cholesky_and_logdet(dtype, tune, arr):
    insts, lay, plan = setup(shapes_for(arr), 1, dtype, TUNINGS[tune], arr=arr)
    Q = dev(lay, lay.pack_band([i.Q for i in insts]))
    L = lay.band_pool(fill=7.0)
    logdet = torch.empty(lay.count, dtype=torch.float64, device="cuda")
    info = torch.full((lay.count,), -1, dtype=torch.int32, device="cuda")
    B.banded_cholesky(plan.handle, Q, L, logdet, info)
    sync()
    Lg = lay.unpack_band(L)
    tol = TOL[dtype]
    for c, ins in enumerate(insts):
        Lo, inf = O.cholesky(ins.Q)
        assert inf == 0 and int(info[c]) == 0
        assert_close(f"L[{c}]", Lg[c], Lo, tol["fwd"])
        ld = O.logdet(Lo)
        assert abs(float(logdet[c]) - ld) <= tol["logdet"] * max(1.0, abs(ld))


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_solve(dtype, tune, mode, k, arr):
    insts, lay, plan = setup(shapes_for(arr), k, dtype, TUNINGS[tune], arr=arr)
    Ls = oracle_L(insts, dtype)
    L = dev(lay, lay.pack_band(Ls))
    Bp = dev(lay, lay.pack_rhs([i.B for i in insts]))
    X = lay.rhs_pool(fill=3.0)
    B.banded_solve(plan.handle, L, Bp, X, mode)
    sync()
    Xg = lay.unpack_rhs(X)
    for c, ins in enumerate(insts):
        ref = O.solve_precision(Ls[c], ins.B) if mode == 2 else O.solve(Ls[c], ins.B, mode)
        assert_close(f"X[{c}]", Xg[c], ref, TOL[dtype]["fwd"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
def test_subset_inverse(dtype, tune, arr):
    insts, lay, plan = setup(shapes_for(arr), 1, dtype, TUNINGS[tune], arr=arr)
    Ls = oracle_L(insts, dtype)
    L = dev(lay, lay.pack_band(Ls))
    S = lay.band_pool(fill=5.0)
    B.banded_subset_inverse(plan.handle, L, S)
    sync()
    Sg = lay.unpack_band(S)
    for c in range(lay.count):
        assert_close(f"S[{c}]", Sg[c], O.subset_inverse(Ls[c]), TOL[dtype]["fwd"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
@pytest.mark.parametrize("acc", [0, 1])
def test_cholesky_vjp(dtype, tune, acc, arr):
    insts, lay, plan = setup(shapes_for(arr), 1, dtype, TUNINGS[tune], arr=arr)
    Ls = oracle_L(insts, dtype)
    rng = np.random.Generator(np.random.PCG64(5))
    Lbars = [zero_corners(rounded(rng.normal(size=L.shape), dtype)) for L in Ls]
    ldbar = rng.normal(size=lay.count)
    prior = [rounded(rng.normal(size=L.shape), dtype) for L in Ls]
    L = dev(lay, lay.pack_band(Ls))
    Lb = dev(lay, lay.pack_band(Lbars))
    ldb = torch.tensor(ldbar, dtype=torch.float64, device="cuda")
    Qb = dev(lay, lay.pack_band(prior)) if acc else lay.band_pool(fill=9.0)
    B.banded_cholesky_vjp(plan.handle, L, Lb, ldb, Qb, acc)
    sync()
    Qg = lay.unpack_band(Qb)
    for c in range(lay.count):
        Lbar = Lbars[c].copy()
        Lbar[0] += 2.0 * ldbar[c] / Ls[c][0]
        ref = O.cholesky_vjp(Ls[c], Lbar)
        if acc:
            ref = ref + zero_corners(prior[c].copy())
        assert_close(f"Qbar[{c}]", Qg[c], ref, TOL[dtype]["grad"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
@pytest.mark.parametrize("acc", [0, 1])
def test_subset_inverse_vjp(dtype, tune, acc, arr):
    insts, lay, plan = setup(shapes_for(arr), 1, dtype, TUNINGS[tune], arr=arr)
    Ls = oracle_L(insts, dtype)
    Ss = [rounded(O.subset_inverse(L), dtype) for L in Ls]
    rng = np.random.Generator(np.random.PCG64(6))
    prior = [rounded(rng.normal(size=L.shape), dtype) for L in Ls]
    L = dev(lay, lay.pack_band(Ls))
    S = dev(lay, lay.pack_band(Ss))
    Sb = dev(lay, lay.pack_band([i.Sbar for i in insts]))
    Lb = dev(lay, lay.pack_band(prior)) if acc else lay.band_pool(fill=4.0)
    B.banded_subset_inverse_vjp(plan.handle, L, S, Sb, Lb, acc)
    sync()
    Lg = lay.unpack_band(Lb)
    for c, ins in enumerate(insts):
        ref = O.subset_inverse_vjp(Ls[c], Ss[c], ins.Sbar)
        if acc:
            ref = ref + zero_corners(prior[c].copy())
        assert_close(f"Lbar[{c}]", Lg[c], ref, TOL[dtype]["grad"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 4])
def test_solve_vjp(dtype, mode, k, arr):
    insts, lay, plan = setup(shapes_for(arr), k, dtype, TUNINGS["seg"], arr=arr)
    Ls = oracle_L(insts, dtype)
    refs_X, refs_Bb, refs_Lb = [], [], []
    for c, ins in enumerate(insts):
        if mode == 2:
            Y = O.solve(Ls[c], ins.B, 0)
            X = rounded(O.solve(Ls[c], Y, 1), dtype)
            Ybar, Lb1 = O.solve_vjp(Ls[c], 1, X, ins.Xbar)
            Y = O.band_matvec(Ls[c], Ls[c].shape[0] - 1, 0, 1, X)      # Y = L^T X, as the library forms it
            Bbar, Lb2 = O.solve_vjp(Ls[c], 0, Y, Ybar)
            Lbar = Lb1 + Lb2
        else:
            X = rounded(O.solve(Ls[c], ins.B, mode), dtype)
            Bbar, Lbar = O.solve_vjp(Ls[c], mode, X, ins.Xbar)
        refs_X.append(X)
        refs_Bb.append(Bbar)
        refs_Lb.append(Lbar)
    L = dev(lay, lay.pack_band(Ls))
    X = dev(lay, lay.pack_rhs(refs_X))
    Xb = dev(lay, lay.pack_rhs([i.Xbar for i in insts]))
    Bb = lay.rhs_pool(fill=2.0)
    Lb = lay.band_pool(fill=2.0)
    B.banded_solve_vjp(plan.handle, L, X, Xb, mode, Bb, Lb, 0)
    sync()
    Bg, Lg = lay.unpack_rhs(Bb), lay.unpack_band(Lb)
    for c in range(lay.count):
        assert_close(f"Bbar[{c}]", Bg[c], refs_Bb[c], TOL[dtype]["grad"])
        assert_close(f"Lbar[{c}]", Lg[c], refs_Lb[c], TOL[dtype]["grad"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tune", list(TUNINGS))
@pytest.mark.parametrize("k", [1, 2, 4])
def test_fused_gmm_step(dtype, tune, k, arr):
    insts, lay, plan = setup(shapes_for(arr), k, dtype, TUNINGS[tune], arr=arr)
    res, _ = O.batch_step(insts)
    Q = dev(lay, lay.pack_band([i.Q for i in insts]))
    Bp = dev(lay, lay.pack_rhs([i.B for i in insts]))
    L, S = lay.band_pool(fill=1.0), lay.band_pool(fill=1.0)
    X = lay.rhs_pool(fill=1.0)
    logdet = torch.empty(lay.count, dtype=torch.float64, device="cuda")
    info = torch.empty(lay.count, dtype=torch.int32, device="cuda")
    B.banded_gmm_forward(plan.handle, Q, Bp, L, X, S, logdet, info)
    Xb = dev(lay, lay.pack_rhs([i.Xbar for i in insts]))
    Sb = dev(lay, lay.pack_band([i.Sbar for i in insts]))
    ldb = torch.full((lay.count,), 0.5, dtype=torch.float64, device="cuda")
    Qb, Bb = lay.band_pool(fill=1.0), lay.rhs_pool(fill=1.0)
    B.banded_gmm_backward(plan.handle, L, X, S, Xb, Sb, ldb, Qb, Bb)
    sync()
    tol = TOL[dtype]
    Lg, Sg, Qg = lay.unpack_band(L), lay.unpack_band(S), lay.unpack_band(Qb)
    Xg, Bg = lay.unpack_rhs(X), lay.unpack_rhs(Bb)
    for c, r in enumerate(res):
        assert int(info[c]) == 0
        assert_close(f"L[{c}]", Lg[c], r["L"], tol["fwd"])
        assert_close(f"X[{c}]", Xg[c], r["X"], tol["fwd"])
        assert_close(f"S[{c}]", Sg[c], r["S"], tol["fwd"])
        assert abs(float(logdet[c]) - r["logdet"]) <= tol["logdet"] * max(1.0, abs(r["logdet"]))
        assert_close(f"Qbar[{c}]", Qg[c], r["Qbar"], tol["grad"])
        assert_close(f"Bbar[{c}]", Bg[c], r["Bbar"], tol["grad"])


PROD = [((2, 0), 0, (2, 0), 1, (2, 2)), ((2, 0), 0, (2, 0), 1, (2, 0)), ((3, 0), 1, (3, 0), 0, (3, 0)),
        ((1, 2), 0, (2, 1), 0, (3, 3)), ((1, 2), 1, (0, 3), 1, (1, 1)), ((3, 1), 0, (2, 2), 1, (6, 2))]


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", range(len(PROD)))
def test_products(dtype, case, arr):
    from test_oracle_pins import rand_general
    (alo, aup), ta, (blo, bup), tb, (clo, cup) = PROD[case]
    shapes = [(n, 8) for n in (1, 2, 7, 300, 1500)]        # 9 rows per instance: room for every operand
    insts, lay, plan = setup(shapes, 2, dtype, TUNINGS["whole"], arr=arr)
    As = [rounded(rand_general(n, alo, aup, 10 + i), dtype) for i, (n, _) in enumerate(shapes)]
    Bs = [rounded(rand_general(n, blo, bup, 20 + i), dtype) for i, (n, _) in enumerate(shapes)]
    Cbs = [rounded(rand_general(n, clo, cup, 30 + i), dtype) for i, (n, _) in enumerate(shapes)]
    A, Bm, Cb = dev(lay, lay.pack_band(As)), dev(lay, lay.pack_band(Bs)), dev(lay, lay.pack_band(Cbs))
    Cm = lay.band_pool(fill=3.0)
    B.banded_product(plan.handle, A, alo, aup, ta, Bm, blo, bup, tb, Cm, clo, cup, 0)
    Ab, Bb = lay.band_pool(fill=3.0), lay.band_pool(fill=3.0)
    B.banded_product_vjp(plan.handle, A, alo, aup, ta, Bm, blo, bup, tb, Cb, clo, cup, Ab, Bb, 0)
    sync()
    Cg = lay.unpack_band(Cm, rows=clo + cup + 1)
    Abg, Bbg = lay.unpack_band(Ab, rows=alo + aup + 1), lay.unpack_band(Bb, rows=blo + bup + 1)
    for c in range(lay.count):
        assert_close("C", Cg[c], O.product(As[c], alo, aup, ta, Bs[c], blo, bup, tb, clo, cup), TOL[dtype]["fwd"])
        ra, rb = O.product_vjp(As[c], alo, aup, ta, Bs[c], blo, bup, tb, Cbs[c], clo, cup)
        assert_close("Abar", Abg[c], ra, TOL[dtype]["grad"])
        assert_close("Bbar", Bbg[c], rb, TOL[dtype]["grad"])


@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_outer_and_matvec(dtype, arr):
    from test_oracle_pins import rand_general
    shapes = [(n, 8) for n in (1, 3, 50, 999)]
    insts, lay, plan = setup(shapes, 3, dtype, TUNINGS["whole"], arr=arr)
    rng = np.random.Generator(np.random.PCG64(3))
    Ms = [rounded(rng.normal(size=(3, n)), dtype) for n, _ in shapes]
    Vs = [rounded(rng.normal(size=(3, n)), dtype) for n, _ in shapes]
    As = [rounded(rand_general(n, 2, 3, 40 + i), dtype) for i, (n, _) in enumerate(shapes)]
    M, V, A = dev(lay, lay.pack_rhs(Ms)), dev(lay, lay.pack_rhs(Vs)), dev(lay, lay.pack_band(As))
    Cm = lay.band_pool(fill=3.0)
    B.banded_outer(plan.handle, M, V, Cm, 4, 2, 0)
    P0, P1 = lay.rhs_pool(fill=3.0), lay.rhs_pool(fill=3.0)
    B.banded_matvec(plan.handle, A, 2, 3, 0, V, P0, 0)
    B.banded_matvec(plan.handle, A, 2, 3, 1, V, P1, 0)
    sync()
    Cg = lay.unpack_band(Cm, rows=7)
    P0g, P1g = lay.unpack_rhs(P0), lay.unpack_rhs(P1)
    for c in range(lay.count):
        assert_close("outer", Cg[c], O.outer(Ms[c], Vs[c], 4, 2), TOL[dtype]["fwd"])
        assert_close("matvec", P0g[c], O.band_matvec(As[c], 2, 3, 0, Vs[c]), TOL[dtype]["fwd"])
        assert_close("matvecT", P1g[c], O.band_matvec(As[c], 2, 3, 1, Vs[c]), TOL[dtype]["fwd"])


# --------------------------------------------------------------------------- Alg. 5 (banded RHS)

@pytest.mark.parametrize("arr", ARRANGEMENTS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("trans", [0, 1])
def test_solve_band_and_vjp(dtype, trans, arr):
    """banded_solve_band (Alg. 5) and its Table 1 adjoint against the oracle:
    mixed bandwidths of L, a (2, 3) banded right-hand side, ragged n."""
    from test_oracle_pins import rand_general
    rlo, rup = 2, 3
    olo, oup = (4, 3) if trans == 0 else (2, 5)
    shapes = [(1, 2), (4, 3), (17, 5), (300, 1), (1000, 2), (1501, 3)]
    rows = max(rlo + rup + 1, olo + oup + 1)
    ins_l = max(l for _, l in shapes)
    insts, lay, plan = setup(sorted(shapes, key=lambda s: (s[1], -s[0])), 1, dtype, TUNINGS["whole"],
                             extra_rows=rows, arr=arr)
    Ls = [rounded(O.cholesky(i.Q)[0], dtype) for i in insts]
    Rs = [rounded(rand_general(i.n, rlo, rup, 70 + c), dtype) for c, i in enumerate(insts)]
    Obs = [rounded(rand_general(i.n, olo, oup, 80 + c), dtype) for c, i in enumerate(insts)]
    L, R, Ob = dev(lay, lay.pack_band(Ls)), dev(lay, lay.pack_band(Rs)), dev(lay, lay.pack_band(Obs))
    Om, G = lay.band_pool(fill=3.0), lay.band_pool(fill=3.0)
    Rb, Lb = lay.band_pool(fill=3.0), lay.band_pool(fill=0.0)
    B.banded_solve_band(plan.handle, L, R, rlo, rup, Om, olo, oup, trans)
    B.banded_solve_band_vjp(plan.handle, L, Om, olo, oup, Ob, trans, rlo, rup, G, Rb, Lb, 0)
    sync()
    Og = lay.unpack_band(Om, rows=olo + oup + 1)
    Rbg = lay.unpack_band(Rb, rows=rlo + rup + 1)
    Lbg = lay.unpack_band(Lb)
    assert ins_l + 1 + rows >= rows
    for c, i in enumerate(insts):
        ref = O.solve_band(Ls[c], Rs[c], rlo, rup, trans, olo, oup)
        assert_close("O", Og[c], ref, TOL[dtype]["fwd"])
        rrb, rlb = O.solve_band_vjp(Ls[c], trans, ref, olo, oup, Obs[c], rlo, rup)
        assert_close("Rbar", Rbg[c], rrb, TOL[dtype]["grad"])
        assert_close("Lbar", Lbg[c], rlb, TOL[dtype]["grad"])


def test_solve_band_rejects_inexact_bands():
    shapes = [(10, 2)]
    insts, lay, plan = setup(shapes, 1, B.BND_F64, TUNINGS["whole"], extra_rows=8)
    x = lay.band_pool()
    y, z = lay.band_pool(), lay.band_pool()
    with pytest.raises(B.BandedError):
        B.banded_solve_band(plan.handle, x, y, 1, 3, z, 2, 2, 0)      # oup < rup
    with pytest.raises(B.BandedError):
        B.banded_solve_band(plan.handle, x, y, 3, 1, z, 2, 2, 1)      # olo < rlo
