"""ctypes binding of the C ABI declared in include/banded.h.

Argument marshalling only: every function here has the name of the C entry
point it calls, converts tensors to device pointers and the current torch
stream to a cudaStream_t, and raises ``BandedError`` on a non-zero status.
No arithmetic of the operators happens in Python.  The shared library is
built in-tree by ``paper_1902_10078_gb300.build``; if it is missing the first
call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_libbanded.so")

BND_F32, BND_F64 = 0, 1
LAYOUT_ROWS, LAYOUT_PANELS, LAYOUT_STRIDED = 0, 1, 2
STATUS = {0: "BND_OK", 1: "BND_EINVAL", 2: "BND_ENOTSPD", 3: "BND_ECUDA", 4: "BND_ETIMEOUT", 5: "BND_EALIGN"}

# Every symbol include/banded.h declares (checked by the ABI tests).
EXPORTS = [
    "bnd_plan_create", "bnd_plan_workspace_bytes", "bnd_plan_bind", "bnd_plan_destroy",
    "bnd_plan_chains", "bnd_plan_tasks", "bnd_plan_layout", "bnd_plan_fixups",
    "banded_cholesky", "banded_cholesky_vjp", "banded_solve", "banded_solve_vjp",
    "banded_subset_inverse", "banded_subset_inverse_vjp",
    "banded_gmm_forward", "banded_gmm_backward",
    "banded_product", "banded_outer", "banded_matvec", "banded_product_vjp",
    "banded_solve_band", "banded_solve_band_vjp",
    "banded_solve_precision_noalloc",
    "bnd_version",
]


class BandedError(RuntimeError):
    def __init__(self, name, status):
        super().__init__(f"{name} failed: {STATUS.get(status, status)}")
        self.status = status


class bnd_inst(C.Structure):
    _fields_ = [("n", C.c_int64), ("band", C.c_int64), ("ld", C.c_int64), ("rhs", C.c_int64),
                ("ldr", C.c_int64), ("l", C.c_int32), ("cs", C.c_int32)]


class bnd_tuning(C.Structure):
    _fields_ = [("seg_len", C.c_int64), ("warmup", C.c_int32), ("blocks_per_sm", C.c_int32), ("flags", C.c_int32),
                ("warm_per_l", C.c_int32), ("warm_base", C.c_int32)]


_lib = None
_vp = C.c_void_p
_i32 = C.c_int32


def lib():
    """Load the in-tree CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    sig = {
        "bnd_plan_create": (_i32, [C.POINTER(_vp), _i32, _i32, C.POINTER(bnd_inst), _i32, C.POINTER(bnd_tuning)]),
        "bnd_plan_workspace_bytes": (C.c_size_t, [_vp]),
        "bnd_plan_bind": (_i32, [_vp, _vp, C.c_size_t, _vp]),
        "bnd_plan_destroy": (None, [_vp]),
        "bnd_plan_chains": (C.c_int64, [_vp]),
        "bnd_plan_tasks": (C.c_int64, [_vp]),
        "bnd_plan_layout": (_i32, [_vp]),
        "bnd_plan_fixups": (_i32, [_vp, _i32, C.POINTER(C.c_int64), _vp]),
        "banded_cholesky": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
        "banded_cholesky_vjp": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp]),
        "banded_solve": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
        "banded_solve_vjp": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp]),
        "banded_subset_inverse": (_i32, [_vp, _vp, _vp, _vp]),
        "banded_subset_inverse_vjp": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp]),
        "banded_gmm_forward": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "banded_solve_band": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _i32, _i32, _i32, _vp]),
        "banded_solve_band_vjp": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _i32,
                                         _vp]),
        "banded_gmm_backward": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "banded_product": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _i32, _i32, _i32, _vp, _i32, _i32, _i32, _vp]),
        "banded_outer": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _vp]),
        "banded_matvec": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp]),
        "banded_product_vjp": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _i32, _i32, _i32, _vp, _i32, _i32,
                                      _vp, _vp, _i32, _vp]),
        "banded_solve_precision_noalloc": (_i32, [_i32, C.c_int64, _i32, _vp, C.c_int64, _vp, _vp, _vp]),
        "bnd_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _p(x):
    """Device pointer of a tensor (or an int / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return x.data_ptr()


def _s(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(name, st):
    if st != 0:
        raise BandedError(name, st)


# --------------------------------------------------------------------------- plans

def bnd_plan_create(dtype: int, insts, k: int, tuning=None):
    arr = (bnd_inst * max(1, len(insts)))()
    for i, d in enumerate(insts):
        arr[i] = bnd_inst(int(d["n"]), int(d["band"]), int(d["ld"]), int(d.get("rhs", 0)), int(d.get("ldr", d["n"])),
                          int(d["l"]), int(d.get("cs", 1)))
    tp = None
    if tuning is not None:
        tp = C.pointer(bnd_tuning(int(tuning.get("seg_len", 0)), int(tuning.get("warmup", 0)),
                                  int(tuning.get("blocks_per_sm", 0)), int(tuning.get("flags", 0)),
                                  int(tuning.get("warm_per_l", 0)), int(tuning.get("warm_base", 0))))
    h = _vp()
    _check("bnd_plan_create", lib().bnd_plan_create(C.byref(h), dtype, len(insts), arr, int(k), tp))
    return h.value


def bnd_plan_workspace_bytes(plan) -> int:
    return int(lib().bnd_plan_workspace_bytes(plan))


def bnd_plan_bind(plan, ws, nbytes: int, stream=None):
    _check("bnd_plan_bind", lib().bnd_plan_bind(plan, _p(ws), int(nbytes), _s(stream)))


def bnd_plan_destroy(plan):
    if plan:
        lib().bnd_plan_destroy(plan)


def bnd_plan_chains(plan) -> int:
    return int(lib().bnd_plan_chains(plan))


def bnd_plan_tasks(plan) -> int:
    return int(lib().bnd_plan_tasks(plan))


def bnd_plan_layout(plan) -> int:
    """0: rows (cs = 1), 1: panels (cs = 32 groups), 2: general strides."""
    return int(lib().bnd_plan_layout(plan))


def bnd_plan_fixups(plan, kind: int, stream=None) -> int:
    v = C.c_int64(0)
    _check("bnd_plan_fixups", lib().bnd_plan_fixups(plan, int(kind), C.byref(v), _s(stream)))
    return int(v.value)


def bnd_version() -> str:
    return lib().bnd_version().decode()


# --------------------------------------------------------------------------- operators

def banded_cholesky(plan, Q, L, logdet, info, stream=None):
    _check("banded_cholesky", lib().banded_cholesky(plan, _p(Q), _p(L), _p(logdet), _p(info), _s(stream)))


def banded_cholesky_vjp(plan, L, Lbar, ldbar, Qbar, accumulate=0, stream=None):
    _check("banded_cholesky_vjp",
           lib().banded_cholesky_vjp(plan, _p(L), _p(Lbar), _p(ldbar), _p(Qbar), int(accumulate), _s(stream)))


def banded_solve(plan, L, B, X, mode: int, stream=None):
    _check("banded_solve", lib().banded_solve(plan, _p(L), _p(B), _p(X), int(mode), _s(stream)))


def banded_solve_vjp(plan, L, X, Xbar, mode: int, Bbar, Lbar, accumulate=0, stream=None):
    _check("banded_solve_vjp", lib().banded_solve_vjp(plan, _p(L), _p(X), _p(Xbar), int(mode), _p(Bbar), _p(Lbar),
                                                      int(accumulate), _s(stream)))


def banded_subset_inverse(plan, L, S, stream=None):
    _check("banded_subset_inverse", lib().banded_subset_inverse(plan, _p(L), _p(S), _s(stream)))


def banded_subset_inverse_vjp(plan, L, S, Sbar, Lbar, accumulate=0, stream=None):
    _check("banded_subset_inverse_vjp",
           lib().banded_subset_inverse_vjp(plan, _p(L), _p(S), _p(Sbar), _p(Lbar), int(accumulate), _s(stream)))


def banded_gmm_forward(plan, Q, B, L, X, S, logdet, info, stream=None):
    _check("banded_gmm_forward", lib().banded_gmm_forward(plan, _p(Q), _p(B), _p(L), _p(X), _p(S), _p(logdet),
                                                          _p(info), _s(stream)))


def banded_gmm_backward(plan, L, X, S, Xbar, Sbar, ldbar, Qbar, Bbar, stream=None):
    _check("banded_gmm_backward", lib().banded_gmm_backward(plan, _p(L), _p(X), _p(S), _p(Xbar), _p(Sbar),
                                                            _p(ldbar), _p(Qbar), _p(Bbar), _s(stream)))


def banded_product(plan, A, alo, aup, transA, B, blo, bup, transB, Cm, clo, cup, accumulate=0, stream=None):
    _check("banded_product", lib().banded_product(plan, _p(A), alo, aup, int(transA), _p(B), blo, bup, int(transB),
                                                  _p(Cm), clo, cup, int(accumulate), _s(stream)))


def banded_outer(plan, M, V, Cm, clo, cup, accumulate=0, stream=None):
    _check("banded_outer", lib().banded_outer(plan, _p(M), _p(V), _p(Cm), clo, cup, int(accumulate), _s(stream)))


def banded_matvec(plan, A, alo, aup, transA, V, P, accumulate=0, stream=None):
    _check("banded_matvec", lib().banded_matvec(plan, _p(A), alo, aup, int(transA), _p(V), _p(P), int(accumulate),
                                                _s(stream)))


def banded_product_vjp(plan, A, alo, aup, transA, B, blo, bup, transB, Cbar, clo, cup, Abar, Bbar, accumulate=0,
                       stream=None):
    _check("banded_product_vjp",
           lib().banded_product_vjp(plan, _p(A), alo, aup, int(transA), _p(B), blo, bup, int(transB), _p(Cbar), clo,
                                    cup, _p(Abar), _p(Bbar), int(accumulate), _s(stream)))


def banded_solve_precision_noalloc(dtype: int, n: int, l: int, L, ld: int, b, x, stream=None):
    """x = (L L^T)^{-1} b for one instance without any allocation (fixed library scratch)."""
    _check("banded_solve_precision_noalloc",
           lib().banded_solve_precision_noalloc(int(dtype), int(n), int(l), _p(L), int(ld), _p(b), _p(x), _s(stream)))


def banded_solve_band(plan, L, R, rlo: int, rup: int, O, olo: int, oup: int, trans: int, stream=None):
    """Alg. 5: O = band_{olo,oup}(op(L)^{-1} R)."""
    _check("banded_solve_band", lib().banded_solve_band(plan, _p(L), _p(R), int(rlo), int(rup), _p(O), int(olo),
                                                        int(oup), int(trans), _s(stream)))


def banded_solve_band_vjp(plan, L, O, olo: int, oup: int, Obar, trans: int, rlo: int, rup: int, G, Rbar, Lbar,
                          accumulate: int = 0, stream=None):
    """Table 1 (solve matrix-matrix) adjoint of banded_solve_band."""
    _check("banded_solve_band_vjp", lib().banded_solve_band_vjp(plan, _p(L), _p(O), int(olo), int(oup), _p(Obar),
                                                                int(trans), int(rlo), int(rup), _p(G), _p(Rbar),
                                                                _p(Lbar), int(accumulate), _s(stream)))
