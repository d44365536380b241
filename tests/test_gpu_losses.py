"""GPU: the workload losses composed from the CUDA operators, forward and
reverse mode through the torch.autograd.Function adjoints.

* Long chain (n = 100000, l = 3, one RHS): loss = -1/2 b^T Q^{-1} b +
  1/2 log det Q + 1/2 tr(band(Q^{-1}) W).  Value and stored-entry gradient
  against the FP64 oracle composition; in FP64 the autograd gradient also
  matches central finite differences of the GPU loss on 50 random stored
  entries.
* Matern-3/2 state-space KL: sum over processes of KL(N(m, (Lq Lq^T)^{-1}) ||
  N(0, Q_p^{-1})) with Q_p = M^T M built from (t, lengthscale), on the
  workload's own Exp(1) gaps.  Value against the oracle; gradients in the
  lengthscales, Lq and m element by element against the oracle's composed
  KL adjoint, on a small batch and on a slice of the full-size batch (256
  processes, N = 100000 states each).
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import losses as OL
from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300 import losses as LS
from paper_1902_10078_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()
    O.lib()


def rounded(a, dtype):
    return np.asarray(a, dtype=BT.NP_DT[dtype]).astype(np.float64)


# --------------------------------------------------------------------------- long chain

@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_long_chain_loss_and_gradient(dtype):
    n, l = 100_000, 3
    Q, b, Wt = W.long_chain_config(n, l)
    Q, b, Wt = rounded(Q, dtype), rounded(b, dtype), rounded(Wt, dtype)
    lay = BT.Layout([n], [l], 1, dtype)
    plan = BT.Plan(lay)
    Qd = torch.tensor(lay.pack_band([Q]), device="cuda", requires_grad=True)
    bd = torch.tensor(lay.pack_rhs([b[None]]), device="cuda")
    Wd = torch.tensor(lay.pack_band([Wt]), device="cuda")
    wsym = LS.symmetric_weights(lay)
    loss, info = LS.chain_loss(plan, Qd, bd, Wd, wsym)
    loss.backward()
    assert int(info.abs().sum()) == 0
    ref_loss, ref_Qbar = OL.chain_loss(Q, b, Wt)
    tol_v, tol_g = (1e-10, 1e-10) if dtype == B.BND_F64 else (1e-4, 1e-3)
    assert abs(float(loss.detach()) - ref_loss) <= tol_v * max(1.0, abs(ref_loss))
    g = lay.unpack_band(Qd.grad)[0]
    err = np.max(np.abs(g - ref_Qbar)) / np.max(np.abs(ref_Qbar))
    assert err <= tol_g, err
    if dtype != B.BND_F64:
        return
    rng = W.rng_for(4242)
    view = lay.band_view(Qd.data, 0)
    with torch.no_grad():
        for _ in range(50):
            d, j = int(rng.integers(0, l + 1)), int(rng.integers(0, n - l))
            h = 1e-5 * max(1.0, abs(Q[d, j]))
            old = float(view[d, j])
            view[d, j] = old + h
            lp = float(LS.chain_loss(plan, Qd, bd, Wd, wsym)[0])
            view[d, j] = old - h
            lm = float(LS.chain_loss(plan, Qd, bd, Wd, wsym)[0])
            view[d, j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[d, j]) <= 1e-5 * max(1.0, abs(fd)), (d, j, fd, g[d, j])


# --------------------------------------------------------------------------- Matern KL

def matern_setup(count, n, dtype, panels=True, seed=W.BASE_SEED, min_gap=0.0):
    procs = W.matern_batch(count, n, seed)
    for p in procs:                       # optional floor on the gaps (gradient checks by differences)
        p.t = p.t + min_gap * np.arange(p.t.shape[0])
    N = 2 * n
    lay = BT.Layout([N] * count, [3] * count, 1, dtype, panels=panels)
    plan = BT.Plan(lay)
    Lq = torch.tensor(lay.pack_band([rounded(p.Lq, dtype) for p in procs]), device="cuda", requires_grad=True)
    m = torch.tensor(lay.pack_rhs([rounded(p.m, dtype)[None] for p in procs]), device="cuda", requires_grad=True)
    ells = torch.tensor([p.lengthscale for p in procs], dtype=torch.float64, device="cuda", requires_grad=True)
    ctx = dict(prior=LS.MaternPrior(lay, [p.t for p in procs], 1.0), wsym=LS.symmetric_weights(lay),
               dmask=LS.diagonal_mask(lay))
    return procs, lay, plan, Lq, m, ells, ctx


def gpu_kl(plan, ctx, ells, Lq, m):
    return LS.matern_kl(plan, ctx["prior"], ells, Lq, m, ctx["wsym"], ctx["dmask"])


def oracle_kl(procs, dtype, ells=None, Lqs=None, ms=None):
    tot = 0.0
    for i, p in enumerate(procs):
        ell = p.lengthscale if ells is None else ells[i]
        Lq = rounded(p.Lq, dtype) if Lqs is None else Lqs[i]
        m = rounded(p.m, dtype) if ms is None else ms[i]
        tot += OL.matern_kl(p.t, ell, p.variance, Lq, m)
    return tot


def check_kl_gradients(procs, dtype, lay, Lq, m, ells, idx, tol):
    """GPU gradients of the processes in `idx` against the oracle's composed KL
    adjoint (normwise per array per process; the lengthscale gradient relative
    to max(1, |ref|))."""
    gL = lay.unpack_band(Lq.grad)
    gm = lay.unpack_rhs(m.grad)
    ge = ells.grad.detach().cpu().numpy()
    worst = dict(Lq=0.0, m=0.0, ell=0.0)
    for i in idx:
        p = procs[i]
        _, rL, rm, re = OL.matern_kl_grad(p.t, p.lengthscale, p.variance, rounded(p.Lq, dtype),
                                          rounded(p.m, dtype))
        worst["Lq"] = max(worst["Lq"], relerr(gL[i], rL))
        worst["m"] = max(worst["m"], relerr(gm[i][0], rm))
        worst["ell"] = max(worst["ell"], abs(float(ge[i]) - re) / max(1.0, abs(re)))
    for key, v in worst.items():
        assert v <= tol, f"{key} gradient: error {v:.3e} > {tol:.1e}"
    return worst


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_matern_kl_value_and_gradients(dtype):
    # the workload's own gaps (Exp(1), no floor): Q_p reaches ~1e15 at the smallest ones
    count, n = 6, 1500
    procs, lay, plan, Lq, m, ells, ctx = matern_setup(count, n, dtype)
    assert B.bnd_plan_layout(plan.handle) == B.LAYOUT_PANELS
    kl = gpu_kl(plan, ctx, ells, Lq, m)
    kl.backward()
    ref = oracle_kl(procs, dtype)
    tol_v, tol_g = (1e-10, 1e-10) if dtype == B.BND_F64 else (1e-4, 1e-3)
    assert abs(float(kl.detach()) - ref) <= tol_v * max(1.0, abs(ref)), (float(kl.detach()), ref)
    check_kl_gradients(procs, dtype, lay, Lq, m, ells, range(count), tol_g)


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_matern_kl_full_size(dtype):
    count, n = 256, 50_000
    procs, lay, plan, Lq, m, ells, ctx = matern_setup(count, n, dtype)
    kl = gpu_kl(plan, ctx, ells, Lq, m)
    kl.backward()
    ref = oracle_kl(procs, dtype)
    tol, tol_g = (1e-10, 1e-10) if dtype == B.BND_F64 else (1e-4, 1e-3)
    assert abs(float(kl.detach()) - ref) <= tol * max(1.0, abs(ref)), (float(kl.detach()), ref)
    # gradients of a slice of the batch (first, middle, last panel groups) against the oracle adjoint
    check_kl_gradients(procs, dtype, lay, Lq, m, ells, [0, 31, 32, 128, 255], tol_g)


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_recomputed_factor_gives_identical_gradients(dtype):
    """The loss with the Cholesky factor recomputed in the backward (nothing but Q,
    X and S kept between the passes) gives bitwise the same value and gradient
    as the loss that keeps L, on a segmented mixed batch."""
    shapes = [(20000, 3), (5000, 1), (777, 7), (12000, 5)]
    lay = BT.Layout([s[0] for s in shapes], [s[1] for s in shapes], 1, dtype, panels=True)
    plan = BT.Plan(lay)
    rng = W.rng_for(606)
    Qs = [rounded(W.spd_band(W.rng_for(607 + i), n, l), dtype) for i, (n, l) in enumerate(shapes)]
    bs = [rounded(rng.normal(size=(1, n)), dtype) for n, _ in shapes]
    Ws = [rounded(W.symmetric_band_weights(rng, n, l), dtype) for n, l in shapes]
    wsym = LS.symmetric_weights(lay)
    grads, vals = [], []
    for rec in (False, True):
        Qd = torch.tensor(lay.pack_band(Qs), device="cuda", requires_grad=True)
        bd = torch.tensor(lay.pack_rhs(bs), device="cuda")
        Wd = torch.tensor(lay.pack_band(Ws), device="cuda")
        loss, info = LS.chain_loss(plan, Qd, bd, Wd, wsym, recompute_L=rec)
        loss.backward()
        assert int(info.abs().sum()) == 0
        vals.append(float(loss.detach()))
        grads.append(Qd.grad.detach().clone())
    assert vals[0] == vals[1]
    assert torch.equal(grads[0], grads[1])
