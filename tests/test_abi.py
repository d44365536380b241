"""C ABI: the library loads, exports every declared symbol, and the host-side
plan logic (validation, segmentation, task grouping) behaves as documented.
Runs without a GPU: nothing here enqueues device work."""
import os
import re

import pytest

from paper_1902_10078_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "banded.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("banded_", "bnd_"))))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        import paper_1902_10078_gb300.build as bld
        bld.build()
    return B.lib()


def test_header_declares_the_bound_functions():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert B.bnd_version().startswith("banded-gb300")


def _insts(ns, ls, k=1, align=32):
    out, o, r = [], 0, 0
    for n, l in zip(ns, ls):
        ld = (n + align - 1) // align * align
        out.append(dict(n=n, l=l, band=o, ld=ld, rhs=r, ldr=ld))
        o += (l + 1) * ld
        r += k * ld
    return out


@pytest.mark.parametrize("bad", [dict(n=0), dict(l=-1), dict(l=2000), dict(ld=3)])
def test_plan_rejects_bad_descriptors(lib, bad):
    d = _insts([10], [2])[0]
    d.update(bad)
    with pytest.raises(B.BandedError) as e:
        B.bnd_plan_create(B.BND_F32, [d], 1)
    assert e.value.status == 1


def test_plan_rejects_bad_k(lib):
    with pytest.raises(B.BandedError):
        B.bnd_plan_create(B.BND_F32, _insts([10], [2]), 65)


def test_plan_segments_long_instances(lib):
    # n = 10000 with 1024-row segments -> round(10000/1024) = 10 segments; short ones stay whole
    ins = _insts([10000, 500, 3000], [3, 3, 7])
    p = B.bnd_plan_create(B.BND_F32, ins, 1, dict(seg_len=1024, warmup=64))
    try:
        assert B.bnd_plan_chains(p) == 10 + 1 + 3
        # tasks group equal bandwidths 32 chains at a time: l=3 -> 11 chains, l=7 -> 3 chains
        assert B.bnd_plan_tasks(p) == 2
        assert B.bnd_plan_workspace_bytes(p) > 0
    finally:
        B.bnd_plan_destroy(p)


def test_plan_never_splits_when_asked(lib):
    p = B.bnd_plan_create(B.BND_F64, _insts([100000], [2]), 1, dict(seg_len=-1))
    try:
        assert B.bnd_plan_chains(p) == 1
    finally:
        B.bnd_plan_destroy(p)


def test_plan_keeps_wide_bands_whole(lib):
    # bandwidths above the register-window limit run one chain per instance
    p = B.bnd_plan_create(B.BND_F64, _insts([50000, 50000], [12, 3]), 1, dict(seg_len=1024))
    try:
        assert B.bnd_plan_chains(p) == 1 + 49
    finally:
        B.bnd_plan_destroy(p)


def test_many_tasks_for_many_instances(lib):
    ns = [1000 + 7 * i for i in range(100)]
    ls = [1 + (i % 5) for i in range(100)]
    p = B.bnd_plan_create(B.BND_F32, _insts(ns, ls, k=4), 4, dict(seg_len=-1))
    try:
        assert B.bnd_plan_chains(p) == 100
        assert B.bnd_plan_tasks(p) == 5          # 20 instances per bandwidth -> one task each
    finally:
        B.bnd_plan_destroy(p)
