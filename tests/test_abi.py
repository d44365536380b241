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


def test_plan_segments_wide_bands_on_the_block_kernels(lib):
    # bandwidths above the register-window limit run on the block kernels, which take
    # segments too (here the asked 1024 rows); without a length, about one segment per
    # SM (152) over all wide instances, each at least one warm-up long (8 l + 32 rows in
    # FP32, 16 l + 64 in FP64 for wide bands); seg_len = -1 keeps them whole
    p = B.bnd_plan_create(B.BND_F64, _insts([50000, 50000], [12, 3]), 1, dict(seg_len=1024))
    try:
        assert B.bnd_plan_chains(p) == 49 + 49
    finally:
        B.bnd_plan_destroy(p)
    p = B.bnd_plan_create(B.BND_F64, _insts([200000], [128]), 1)
    try:
        assert B.bnd_plan_chains(p) == round(200000 / (16 * 128 + 64))
    finally:
        B.bnd_plan_destroy(p)
    p = B.bnd_plan_create(B.BND_F32, _insts([200000], [64]), 1)
    try:
        assert B.bnd_plan_chains(p) == 152
    finally:
        B.bnd_plan_destroy(p)
    p = B.bnd_plan_create(B.BND_F64, _insts([50000], [12]), 1, dict(seg_len=-1))
    try:
        assert B.bnd_plan_chains(p) == 1
    finally:
        B.bnd_plan_destroy(p)
    # the RHS windows are sized for min(k, 16) columns: FP64 at l = 162 fits a block with one
    # right-hand side (so it is segmented), not with 16 (one warp per instance, whole)
    p = B.bnd_plan_create(B.BND_F64, _insts([200000], [162], k=1), 1)
    try:
        assert B.bnd_plan_chains(p) > 1
    finally:
        B.bnd_plan_destroy(p)
    p = B.bnd_plan_create(B.BND_F64, _insts([200000], [162], k=16), 16)
    try:
        assert B.bnd_plan_chains(p) == 1
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


def _panel_insts(ns, ls, k=1):
    from paper_1902_10078_gb300 import batch as BT
    return BT.Layout(ns, ls, k, B.BND_F32, panels=True).insts()


def test_plan_recognises_rows_and_panels(lib):
    p = B.bnd_plan_create(B.BND_F32, _insts([100, 200], [2, 3]), 1)
    try:
        assert B.bnd_plan_layout(p) == B.LAYOUT_ROWS
    finally:
        B.bnd_plan_destroy(p)
    p = B.bnd_plan_create(B.BND_F32, _panel_insts([100, 200, 50], [2, 2, 3]), 1)
    try:
        assert B.bnd_plan_layout(p) == B.LAYOUT_PANELS
    finally:
        B.bnd_plan_destroy(p)


def test_panel_tasks_follow_groups(lib):
    # 40 instances of l = 3 -> groups of 32 and 8 lanes; the group's longest n (5000) sets the
    # segment length (1024 -> round(5000 / 1024) = 5 segments of 1000 rows); one task per
    # (group, segment), lanes past their own end idle
    ns = sorted([5000 - 10 * i for i in range(40)], reverse=True)
    ins = _panel_insts(ns, [3] * 40)
    p = B.bnd_plan_create(B.BND_F32, ins, 1, dict(seg_len=1024, warmup=64))
    try:
        assert B.bnd_plan_layout(p) == B.LAYOUT_PANELS
        assert B.bnd_plan_tasks(p) == 5 + 5
        assert B.bnd_plan_chains(p) == sum((n + 999) // 1000 for n in ns)
    finally:
        B.bnd_plan_destroy(p)


def test_panel_groups_break_on_bandwidth_and_offsets(lib):
    ins = _panel_insts([100] * 5 + [90] * 3, [2] * 5 + [4] * 3)
    p = B.bnd_plan_create(B.BND_F32, ins, 1, dict(seg_len=-1))
    try:
        assert B.bnd_plan_layout(p) == B.LAYOUT_PANELS
        assert B.bnd_plan_tasks(p) == 2          # one task per group
    finally:
        B.bnd_plan_destroy(p)
    # a column stride other than 1 or 32 (or ld not a multiple of 32) is a general strided batch
    odd = [dict(n=10, l=2, band=0, ld=40, rhs=0, ldr=40, cs=4)]
    p = B.bnd_plan_create(B.BND_F32, odd, 1)
    try:
        assert B.bnd_plan_layout(p) == B.LAYOUT_STRIDED
    finally:
        B.bnd_plan_destroy(p)


@pytest.mark.parametrize("bad", [dict(cs=-1), dict(cs=32, ld=32 * 9), dict(cs=2, ld=19)])
def test_plan_rejects_bad_strides(lib, bad):
    d = dict(n=10, l=2, band=0, ld=400, rhs=0, ldr=400)
    d.update(bad)
    with pytest.raises(B.BandedError) as e:
        B.bnd_plan_create(B.BND_F32, [d], 1)
    assert e.value.status == 1


# The allocation-free solve validates its pointers on the host before any CUDA
# call: every case below is rejected there (fake addresses are never used).
_BASE = 1 << 40


@pytest.mark.parametrize("x_off,b_off,why", [
    (0, 0, "x is b"),
    (8 * 10, 8 * 50, "x overlaps the tail of b"),
    (8 * 90, 8 * 50, "x overlaps the head of b"),
    (8 * 300, 8 * 1000, "x overlaps L"),
])
def test_noalloc_rejects_overlapping_output(lib, x_off, b_off, why):
    n, l, ld = 100, 2, 128
    L = _BASE
    b = _BASE + (1 << 20) + b_off if why != "x overlaps L" else _BASE + (1 << 20)
    x = (_BASE + (1 << 20) + x_off) if why != "x overlaps L" else _BASE + x_off
    with pytest.raises(B.BandedError) as e:
        B.banded_solve_precision_noalloc(B.BND_F64, n, l, L, ld, b, x, stream=0)
    assert e.value.status == 1, why


def test_noalloc_rejects_misaligned_and_bad_sizes(lib):
    with pytest.raises(B.BandedError) as e:
        B.banded_solve_precision_noalloc(B.BND_F64, 10, 2, _BASE + 4, 16, _BASE + 4096, _BASE + 8192, stream=0)
    assert e.value.status == 5
    for n, l, ld in ((0, 1, 8), (10, -1, 16), (10, 2, 9)):
        with pytest.raises(B.BandedError) as e:
            B.banded_solve_precision_noalloc(B.BND_F64, n, l, _BASE, ld, _BASE + 4096, _BASE + 8192, stream=0)
        assert e.value.status == 1


def test_small_batches_get_short_segments(lib):
    # one long chain cannot fill the GPU at the 2048-row default: the default length
    # drops so that about 16k chains run, but never below 32 rows
    p = B.bnd_plan_create(B.BND_F32, _insts([100000], [3]), 1)
    try:
        assert B.bnd_plan_chains(p) == round(100000 / 32)
    finally:
        B.bnd_plan_destroy(p)
    # a batch with enough rows keeps the 2048-row default
    ns = [60000] * 600
    p = B.bnd_plan_create(B.BND_F32, _insts(ns, [2] * 600), 1)
    try:
        assert B.bnd_plan_chains(p) == 600 * round(60000 / 2048)
    finally:
        B.bnd_plan_destroy(p)
