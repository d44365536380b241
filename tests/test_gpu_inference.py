"""GPU: the inference compositions of Sec. 3 on the CUDA operators.

* Marginal likelihood of a GMRF with partial Gaussian observations (Sec. 3.1).
* Whitened log joint for HMC, F = L_Q^{-T} v (Sec. 3.2).
* Matern-3/2 GP regression in state-space form through natural parameters
  (App. C).
Values per instance against the oracle compositions (which are pinned against
dense Gaussian formulas); gradients (autograd through the CUDA adjoints)
against central differences of the oracle values.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import losses as OL
from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B
from paper_1902_10078_gb300 import inference as INF
from paper_1902_10078_gb300 import losses as LS
from paper_1902_10078_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(3000, 3), (1500, 2), (700, 5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_1902_10078_gb300.build as bld
    bld.build()
    O.lib()


def rounded(a, dtype):
    return np.asarray(a, dtype=BT.NP_DT[dtype]).astype(np.float64)


def gmrf_case(dtype, arr, seed=300):
    rng = W.rng_for(seed)
    Qs, obs, ys = [], [], []
    for i, (n, l) in enumerate(SHAPES):
        Qs.append(rounded(W.spd_band(W.rng_for(seed + 1 + i), n, l), dtype))
        o = np.sort(rng.choice(n, size=n // 3, replace=False))
        obs.append(o)
        ys.append(rounded(rng.normal(size=o.shape[0]), dtype))
    shapes = SHAPES
    lay = BT.Layout([s[0] for s in shapes], [s[1] for s in shapes], 1, dtype, panels=(arr == "panels"))
    plan = BT.Plan(lay)
    return lay, plan, Qs, obs, ys


@pytest.mark.parametrize("arr", ["rows", "panels"])
@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_marginal_likelihood(dtype, arr):
    lay, plan, Qs, obs, ys = gmrf_case(dtype, arr)
    diag_idx, rhs_idx, inst = INF.observation_index(lay, obs)
    Q = torch.tensor(lay.pack_band(Qs), device="cuda", requires_grad=True)
    y = torch.tensor(np.concatenate(ys), dtype=torch.float64, device="cuda")
    tau2 = torch.tensor([0.3, 0.5, 0.2], dtype=torch.float64, device="cuda", requires_grad=True)
    ll = INF.marginal_likelihood(plan, Q, diag_idx, rhs_idx, inst, y, tau2)
    ll.sum().backward()
    tol = 1e-10 if dtype == B.BND_F64 else 1e-4
    for i in range(len(Qs)):
        ref = OL.marginal_likelihood(Qs[i], obs[i], ys[i], float(tau2.detach()[i]))
        got = float(ll.detach()[i])
        assert abs(got - ref) <= tol * max(1.0, abs(ref)), (i, got, ref)
    if dtype != B.BND_F64:
        return
    gQ = lay.unpack_band(Q.grad)
    for i in range(len(Qs)):
        t0 = float(tau2.detach()[i])
        h = 1e-6 * t0
        fd = (OL.marginal_likelihood(Qs[i], obs[i], ys[i], t0 + h)
              - OL.marginal_likelihood(Qs[i], obs[i], ys[i], t0 - h)) / (2 * h)
        assert abs(float(tau2.grad[i]) - fd) <= 1e-6 * max(1.0, abs(fd)), (i, float(tau2.grad[i]), fd)
        rng = W.rng_for(900 + i)
        for _ in range(4):
            d, j = int(rng.integers(0, SHAPES[i][1] + 1)), int(rng.integers(0, SHAPES[i][0] - SHAPES[i][1]))
            hq = 1e-6
            Qp, Qm = Qs[i].copy(), Qs[i].copy()
            Qp[d, j] += hq
            Qm[d, j] -= hq
            fd = (OL.marginal_likelihood(Qp, obs[i], ys[i], t0) - OL.marginal_likelihood(Qm, obs[i], ys[i], t0)) / (2 * hq)
            assert abs(gQ[i][d, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, d, j, gQ[i][d, j], fd)


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_whitened_log_joint(dtype):
    lay, plan, Qs, obs, ys = gmrf_case(dtype, "rows", seed=400)
    _, rhs_idx, inst = INF.observation_index(lay, obs)
    rng = W.rng_for(401)
    vs = [rounded(rng.normal(size=n), dtype) for n, _ in SHAPES]
    Q = torch.tensor(lay.pack_band(Qs), device="cuda", requires_grad=True)
    v = torch.tensor(lay.pack_rhs([x[None] for x in vs]), device="cuda", requires_grad=True)
    y = torch.tensor(np.concatenate(ys), dtype=torch.float64, device="cuda")
    tau2 = torch.tensor([0.4, 0.4, 0.4], dtype=torch.float64, device="cuda")
    lj = INF.whitened_log_joint(plan, Q, v, rhs_idx, inst, y, tau2)
    lj.sum().backward()
    tol = 1e-10 if dtype == B.BND_F64 else 1e-4
    for i in range(len(Qs)):
        ref = OL.whitened_log_joint(Qs[i], vs[i], obs[i], ys[i], 0.4)
        assert abs(float(lj[i]) - ref) <= tol * max(1.0, abs(ref)), (i, float(lj[i]), ref)
    if dtype != B.BND_F64:
        return
    gv = lay.unpack_rhs(v.grad)
    gQ = lay.unpack_band(Q.grad)
    for i in range(len(Qs)):
        rng = W.rng_for(910 + i)
        for _ in range(4):
            j = int(rng.integers(0, SHAPES[i][0]))
            vp, vm = vs[i].copy(), vs[i].copy()
            vp[j] += 1e-6
            vm[j] -= 1e-6
            fd = (OL.whitened_log_joint(Qs[i], vp, obs[i], ys[i], 0.4)
                  - OL.whitened_log_joint(Qs[i], vm, obs[i], ys[i], 0.4)) / 2e-6
            assert abs(gv[i][0, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, j, gv[i][0, j], fd)
            d, j = int(rng.integers(0, SHAPES[i][1] + 1)), int(rng.integers(0, SHAPES[i][0] - SHAPES[i][1]))
            Qp, Qm = Qs[i].copy(), Qs[i].copy()
            Qp[d, j] += 1e-6
            Qm[d, j] -= 1e-6
            fd = (OL.whitened_log_joint(Qp, vs[i], obs[i], ys[i], 0.4)
                  - OL.whitened_log_joint(Qm, vs[i], obs[i], ys[i], 0.4)) / 2e-6
            assert abs(gQ[i][d, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, d, j, gQ[i][d, j], fd)


@pytest.mark.parametrize("dtype", [B.BND_F64, B.BND_F32])
def test_ssm_gpr(dtype):
    # gaps of at least 0.05: at the Exp(1) workload's smallest gaps the posterior
    # precision Q_p + H^T H / tau2 has a condition number near 1e15, and the FP64
    # Cholesky log-determinants of two correct implementations then agree only to
    # ~1e-8 (the KL test avoids this by taking log det Q_p from the factor M; the
    # posterior precision has no such factor)
    count, n = 4, 2000
    procs = W.matern_batch(count, n, seed=500)
    for p in procs:
        p.t = p.t + 0.05 * np.arange(p.t.shape[0])
    rng = W.rng_for(501)
    ys = [rng.normal(size=n) for _ in range(count)]
    lay = BT.Layout([2 * n] * count, [3] * count, 1, dtype, panels=True)
    plan = BT.Plan(lay)
    prior = LS.MaternPrior(lay, [p.t for p in procs], 1.0)
    obs = [2 * np.arange(n) for _ in range(count)]
    diag_idx, rhs_idx, inst = INF.observation_index(lay, obs)
    ells = torch.tensor([p.lengthscale for p in procs], dtype=torch.float64, device="cuda", requires_grad=True)
    tau2 = torch.tensor([0.1, 0.2, 0.3, 0.05], dtype=torch.float64, device="cuda", requires_grad=True)
    y = torch.tensor(np.concatenate(ys), dtype=torch.float64, device="cuda")
    lp = INF.ssm_gpr_log_marginal(plan, prior, ells, y, tau2, diag_idx, rhs_idx, inst)
    lp.sum().backward()
    tol_v, tol_g = (1e-10, 1e-6) if dtype == B.BND_F64 else (1e-4, 1e-3)
    for i, p in enumerate(procs):
        t2 = float(tau2.detach()[i])
        ref = OL.ssm_gpr_log_marginal(p.t, p.lengthscale, 1.0, ys[i], t2)
        assert abs(float(lp[i]) - ref) <= tol_v * max(1.0, abs(ref)), (i, float(lp[i]), ref)
        h = 1e-6 * p.lengthscale
        fd = (OL.ssm_gpr_log_marginal(p.t, p.lengthscale + h, 1.0, ys[i], t2)
              - OL.ssm_gpr_log_marginal(p.t, p.lengthscale - h, 1.0, ys[i], t2)) / (2 * h)
        assert abs(float(ells.grad[i]) - fd) <= tol_g * max(1.0, abs(fd)), (i, float(ells.grad[i]), fd)
        h = 1e-6 * t2
        fd = (OL.ssm_gpr_log_marginal(p.t, p.lengthscale, 1.0, ys[i], t2 + h)
              - OL.ssm_gpr_log_marginal(p.t, p.lengthscale, 1.0, ys[i], t2 - h)) / (2 * h)
        assert abs(float(tau2.grad[i]) - fd) <= tol_g * max(1.0, abs(fd)), (i, float(tau2.grad[i]), fd)
