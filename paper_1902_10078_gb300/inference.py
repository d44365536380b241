"""Inference compositions of Sec. 3 over the banded operators: the marginal
likelihood of a GMRF with partial Gaussian observations, the whitened log
joint that HMC samples, and state-space GP regression through natural
parameters.  Every Cholesky, solve and product runs in the CUDA kernels (with
their adjoints under autograd); torch only adds scalars to the band's
diagonal and forms sums of squares (in FP64).

Observations of a batch are given as flat index tensors into the layout's
pools: `diag_idx` (the band-pool element of each observed node's diagonal
entry), `rhs_idx` (the RHS-pool element of that node), and `inst` (the
instance of each observation), so that one call serves the whole batch.
"""
from __future__ import annotations

import math

import torch

from . import autograd as AG


def observation_index(layout, obs, device="cuda"):
    """Flat pool indices of the observed nodes: obs[i] lists the observed node
    indices of instance i.  Returns (diag_idx, rhs_idx, inst) int64 tensors."""
    flat_b = torch.arange(layout.band_elems, dtype=torch.int64)
    flat_r = torch.arange(layout.rhs_elems, dtype=torch.int64)
    d, r, w = [], [], []
    for i, o in enumerate(obs):
        o = torch.as_tensor(o, dtype=torch.int64)
        d.append(layout.band_view(flat_b, i)[0, o])
        r.append(layout.rhs_view(flat_r, i)[0, o])
        w.append(torch.full((o.shape[0],), i, dtype=torch.int64))
    return torch.cat(d).to(device), torch.cat(r).to(device), torch.cat(w).to(device)


def _scatter_rhs(layout, rhs_idx, values, like):
    out = torch.zeros(layout.rhs_elems, dtype=like.dtype, device=like.device)
    return out.index_put((rhs_idx,), values.to(like.dtype))


def marginal_likelihood(plan, Q, diag_idx, rhs_idx, inst, y, tau2, logdet_prior=None):
    """Per-instance log p(y | theta) of f ~ N(0, Q^{-1}) observed with noise tau2
    (Sec. 3.1, marginal-likelihood equation):

      -n/2 log 2 pi - log|L| + log|L_Q| - n/2 log tau2 - y^T y / (2 tau2)
      + |L^{-1} E^T y|^2 / (2 tau2^2),    L L^T = Q + E^T E / tau2,  L_Q L_Q^T = Q,

    E^T E being diagonal, the posterior precision keeps Q's band.  Q: band pool;
    y: (nobs,) observations in the order of the index tensors; tau2: (count,)
    FP64.  `logdet_prior` (count,) replaces log|Q| (2 log|L_Q|) when the prior
    precision comes factored.  Differentiable in Q, y and tau2."""
    lay = plan.layout
    tau2_obs = tau2[inst]
    Qpost = Q.index_add(0, diag_idx, (1.0 / tau2_obs).to(Q.dtype))
    L, ld_post, _ = AG.cholesky(plan, Qpost)
    if logdet_prior is None:
        _, logdet_prior, _ = AG.cholesky(plan, Q)
    Ey = _scatter_rhs(lay, rhs_idx, y, Q)
    R = AG.solve(plan, L, Ey, 0)
    count = lay.count
    nobs = torch.zeros(count, dtype=torch.float64, device=Q.device).index_add(
        0, inst, torch.ones_like(tau2_obs))
    yy = torch.zeros(count, dtype=torch.float64, device=Q.device).index_add(0, inst, y.to(torch.float64) ** 2)
    rr = _per_instance_sq(lay, R, Q.device)
    return (-0.5 * nobs * math.log(2 * math.pi) - 0.5 * ld_post + 0.5 * logdet_prior - 0.5 * nobs * torch.log(tau2)
            - yy / (2 * tau2) + rr / (2 * tau2 * tau2))


def _per_instance_sq(layout, P, device):
    """sum over each instance's RHS entries of P^2 (FP64), as a (count,) tensor."""
    owner = _rhs_owner(layout, device)
    v = P.to(torch.float64) ** 2
    return torch.zeros(layout.count, dtype=torch.float64, device=device).index_add(0, owner[0], v[owner[1]])


def _rhs_owner(layout, device):
    """(instance, pool index) of every RHS element of the layout's first column
    (cached on the layout)."""
    cache = layout.__dict__.setdefault("_rhs_owner_cache", {})
    if str(device) not in cache:
        flat = torch.arange(layout.rhs_elems, dtype=torch.int64)
        idx = [layout.rhs_view(flat, i)[0] for i in range(layout.count)]
        own = [torch.full((x.shape[0],), i, dtype=torch.int64) for i, x in enumerate(idx)]
        cache[str(device)] = (torch.cat(own).to(device), torch.cat(idx).to(device))
    return cache[str(device)]


def whitened_log_joint(plan, Q, v, rhs_idx, inst, y, tau2):
    """Per-instance log p(v) + sum_i log N(y_i; F_i, tau2) with F = L_Q^{-T} v
    (Sec. 3.2 and the HMC log-likelihood pseudocode; log p(theta) is the
    caller's).  v: RHS pool (k = 1) of white noise; y: (nobs,) observations
    at the RHS-pool positions rhs_idx.  Differentiable in Q and v."""
    lay = plan.layout
    L, _, _ = AG.cholesky(plan, Q)
    F = AG.solve(plan, L, v, 1)
    Nn = torch.tensor([float(n) for n in lay.ns], dtype=torch.float64, device=Q.device)
    vv = _per_instance_sq(lay, v, Q.device)
    r = y.to(torch.float64) - F[rhs_idx].to(torch.float64)
    tau2_obs = tau2[inst]
    lik = torch.zeros(lay.count, dtype=torch.float64, device=Q.device).index_add(
        0, inst, -0.5 * torch.log(2 * math.pi * tau2_obs) - r * r / (2 * tau2_obs))
    return -0.5 * Nn * math.log(2 * math.pi) - 0.5 * vv + lik


def ssm_gpr_log_marginal(plan, prior, ells, y, tau2, diag_idx, rhs_idx, inst):
    """Per-process log p(y) of Matern-3/2 GP regression in state-space form (App.
    C, GP regression with banded matrices): prior precision Q_p = M^T M from
    `prior` (a losses.MaternPrior, differentiable in the lengthscales), every
    f state observed (the index tensors select the f entries) with noise tau2;
    the marginal likelihood with log|Q_p| = 2 sum log|M_ii| from the factor."""
    from .losses import diagonal_mask
    M = prior.band(ells)
    Qp = AG.product(plan, M, (3, 0), 1, M, (3, 0), 0, (3, 0))
    dmask = diagonal_mask(plan.layout, M.device)
    one = torch.ones((), dtype=M.dtype, device=M.device)
    logm = torch.log(torch.where(dmask, M, one).abs().to(torch.float64))
    owner = _band_diag_owner(plan.layout, M.device)
    logdet_prior = 2.0 * torch.zeros(plan.layout.count, dtype=torch.float64, device=M.device).index_add(
        0, owner[0], logm[owner[1]])
    return marginal_likelihood(plan, Qp, diag_idx, rhs_idx, inst, y, tau2, logdet_prior=logdet_prior)


def _band_diag_owner(layout, device):
    """(instance, pool index) of every diagonal band entry (cached on the layout)."""
    cache = layout.__dict__.setdefault("_diag_owner_cache", {})
    if str(device) not in cache:
        flat = torch.arange(layout.band_elems, dtype=torch.int64)
        idx = [layout.band_view(flat, i)[0] for i in range(layout.count)]
        own = [torch.full((x.shape[0],), i, dtype=torch.int64) for i, x in enumerate(idx)]
        cache[str(device)] = (torch.cat(own).to(device), torch.cat(idx).to(device))
    return cache[str(device)]
