"""Pooled HBM layout of a batch of banded instances, and plan ownership.

A batch of ``count`` instances (order n_i, bandwidth l_i, k right-hand sides)
lives in two kinds of pools:

* band pools: instance i occupies ``rows * ld_i`` elements starting at
  ``band_i``; row d (a diagonal, Sec. 4.3 storage) is contiguous;
  ``ld_i = round_up(n_i, align)`` and every offset is a multiple of ``align``
  elements, so each diagonal starts on a 128-byte boundary.
* RHS pools: instance i occupies ``k * ldr_i`` elements from ``rhs_i``,
  column r contiguous.

``rows`` is ``l_i + 1 + extra_rows`` (``extra_rows`` > 0 leaves room for
product operands with a wider band).  Host-side packing helpers move numpy
arrays in and out of pools; they are plumbing, not arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

TORCH_DT = {B.BND_F32: torch.float32, B.BND_F64: torch.float64}
NP_DT = {B.BND_F32: np.float32, B.BND_F64: np.float64}


def _round_up(x, a):
    return (x + a - 1) // a * a


class Layout:
    def __init__(self, ns, ls, k: int, dtype: int = B.BND_F32, extra_rows: int = 0, align: int = 32):
        self.ns = [int(n) for n in ns]
        self.ls = [int(l) for l in ls]
        self.count = len(self.ns)
        self.k = int(k)
        self.dtype = dtype
        self.extra_rows = int(extra_rows)
        self.align = int(align)
        self.ld = [_round_up(n, align) for n in self.ns]
        self.rows = [l + 1 + self.extra_rows for l in self.ls]
        self.band_off = []
        o = 0
        for i in range(self.count):
            self.band_off.append(o)
            o += self.rows[i] * self.ld[i]
        self.band_elems = max(o, 1)
        self.rhs_off = []
        o = 0
        for i in range(self.count):
            self.rhs_off.append(o)
            o += max(self.k, 1) * self.ld[i]
        self.rhs_elems = max(o, 1)

    @property
    def torch_dtype(self):
        return TORCH_DT[self.dtype]

    @property
    def np_dtype(self):
        return NP_DT[self.dtype]

    def insts(self):
        return [dict(n=self.ns[i], l=self.ls[i], band=self.band_off[i], ld=self.ld[i],
                     rhs=self.rhs_off[i], ldr=self.ld[i]) for i in range(self.count)]

    # --- pools -------------------------------------------------------------
    def band_pool(self, device="cuda", fill=0.0):
        return torch.full((self.band_elems,), fill, dtype=self.torch_dtype, device=device)

    def rhs_pool(self, device="cuda", fill=0.0):
        return torch.full((self.rhs_elems,), fill, dtype=self.torch_dtype, device=device)

    def pack_band(self, arrays, fill=0.0) -> np.ndarray:
        """arrays[i]: (r_i, n_i) with r_i <= rows_i -> flat host pool."""
        pool = np.full(self.band_elems, fill, dtype=self.np_dtype)
        for i, a in enumerate(arrays):
            a = np.asarray(a)
            r, n, ld, o = a.shape[0], self.ns[i], self.ld[i], self.band_off[i]
            view = pool[o:o + self.rows[i] * ld].reshape(self.rows[i], ld)
            view[:r, :n] = a
        return pool

    def unpack_band(self, pool, rows=None):
        pool = pool.detach().cpu().numpy() if isinstance(pool, torch.Tensor) else pool
        out = []
        for i in range(self.count):
            r = self.ls[i] + 1 if rows is None else rows
            ld, o = self.ld[i], self.band_off[i]
            out.append(pool[o:o + self.rows[i] * ld].reshape(self.rows[i], ld)[:r, : self.ns[i]].astype(np.float64))
        return out

    def pack_rhs(self, arrays, fill=0.0) -> np.ndarray:
        pool = np.full(self.rhs_elems, fill, dtype=self.np_dtype)
        for i, a in enumerate(arrays):
            a = np.asarray(a)
            a = a[None] if a.ndim == 1 else a
            ld, o = self.ld[i], self.rhs_off[i]
            view = pool[o:o + self.k * ld].reshape(self.k, ld)
            view[: a.shape[0], : self.ns[i]] = a
        return pool

    def unpack_rhs(self, pool):
        pool = pool.detach().cpu().numpy() if isinstance(pool, torch.Tensor) else pool
        out = []
        for i in range(self.count):
            ld, o = self.ld[i], self.rhs_off[i]
            out.append(pool[o:o + self.k * ld].reshape(self.k, ld)[:, : self.ns[i]].astype(np.float64))
        return out

    def to_device(self, host: np.ndarray, device="cuda"):
        return torch.from_numpy(host).to(device)


class Plan:
    """Owns a C-ABI plan and the device workspace bound to it."""

    def __init__(self, layout: Layout, tuning=None, device="cuda", stream=None):
        self.layout = layout
        self.handle = B.bnd_plan_create(layout.dtype, layout.insts(), layout.k, tuning)
        self.ws_bytes = B.bnd_plan_workspace_bytes(self.handle)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        B.bnd_plan_bind(self.handle, self.ws, self.ws_bytes, stream)
        self.chains = B.bnd_plan_chains(self.handle)
        self.tasks = B.bnd_plan_tasks(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.bnd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
