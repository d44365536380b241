"""Losses of the precision-parameterised Gaussian models, composed from the
banded operators (Sec. 3).  The operators and their adjoints run in the CUDA
kernels; torch only forms elementwise products and reductions of their
outputs (accumulated in FP64).

Trace over lower-band storage: for symmetric A, B stored by their lower band,
tr(A B) = sum_j A_jj B_jj + 2 sum_{d>=1} sum_j A[d, j] B[d, j], because each
stored off-diagonal entry stands for two entries of the full matrix.
"""
from __future__ import annotations

import torch

from . import autograd as AG


def symmetric_weights(layout, device="cuda"):
    """Band pool with 1 on the diagonal row, 2 on the off-diagonal rows, 0 at corners/padding."""
    w = torch.zeros(layout.band_elems, dtype=torch.float64)
    for i in range(layout.count):
        n, l = layout.ns[i], layout.ls[i]
        v = layout.band_view(w, i)
        v[0, :n] = 1.0
        for d in range(1, min(l, n - 1) + 1):
            v[d, : n - d] = 2.0
    return w.to(device=device)


def chain_loss(plan, Q, b, W, wsym):
    """-1/2 b^T Q^{-1} b + 1/2 log det Q + 1/2 tr(band(Q^{-1}) W), summed over instances.

    Q, W: band pools (W symmetric with the bandwidth of Q); b: RHS pool (k = 1);
    wsym: symmetric_weights(layout).  Differentiable in Q (and b) through the
    fused GMM step kernels."""
    X, S, logdet, _L, info = AG.gmm_step(plan, Q, b)
    quad = (b.to(torch.float64) * X.to(torch.float64)).sum()
    trace = (wsym * S.to(torch.float64) * W.to(torch.float64)).sum()
    return -0.5 * quad + 0.5 * logdet.sum() + 0.5 * trace, info
