"""Host-side pieces of bench.py: the algorithmic byte counts (the two-call
floor of the uneven batch), the stored-traffic staleness rule and the ncu
summary writer."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1902_10078_gb300 import batch as BT  # noqa: E402
from paper_1902_10078_gb300 import binding as B  # noqa: E402


def test_algorithmic_bytes_match_the_two_call_floor():
    lay = BT.Layout([1000, 2000], [2, 7], 4, B.BND_F32)
    fwd, bwd, floor = bench.algorithmic_bytes(lay)
    w = 4
    assert fwd + bwd == sum(w * n * (7 * (l + 1) + 5 * 4) for n, l in zip(lay.ns, lay.ls))
    assert fwd == sum(w * n * (3 * (l + 1) + 2 * 4) for n, l in zip(lay.ns, lay.ls))
    assert floor == sum(w * n * (4 * (l + 1) + 4 * 4) for n, l in zip(lay.ns, lay.ls))


def test_stored_traffic_requires_matching_sources(tmp_path, monkeypatch):
    f = tmp_path / "t.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.stored_traffic("banded_gmm_backward", 10) is None          # absent
    f.write_text(json.dumps({"call": "banded_gmm_backward", "source_hash": bench.source_hash(),
                             "dram_bytes_per_call": 200.0, "band_entries": 5}))
    assert bench.stored_traffic("banded_gmm_backward", 10) == 400.0         # scaled by band entries
    assert bench.stored_traffic("banded_gmm_forward", 10) is None           # another call
    f.write_text(json.dumps({"call": "banded_gmm_backward", "source_hash": "0" * 16,
                             "dram_bytes_per_call": 200.0, "band_entries": 5}))
    assert bench.stored_traffic("banded_gmm_backward", 10) is None          # stale sources


def test_summarize_ncu_sums_dram_bytes(tmp_path, monkeypatch):
    out = tmp_path / "t.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(out))
    csv = tmp_path / "c.csv"
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"'
    rows = ['"0","void k1(int)","dram__bytes_read.sum","Mbyte","1.5"',
            '"0","void k1(int)","dram__bytes_write.sum","Kbyte","500"',
            '"0","void k1(int)","gpu__time_duration.sum","usecond","10"',
            '"1","void k2(int)","dram__bytes_read.sum","byte","1,000"']
    csv.write_text("==PROF== note\n" + hdr + "\n" + "\n".join(rows) + "\n")

    class A:
        summarize_ncu = str(csv)
        summarize_entries = 123
        summarize_cmd = "cmd"
    bench.summarize_ncu(A)
    t = json.loads(out.read_text())
    assert t["dram_bytes_per_call"] == 1.5e6 + 5e5 + 1000
    assert t["launches"] == 2 and t["band_entries"] == 123 and t["source_hash"] == bench.source_hash()


def test_strong_scaling_layouts_cover_the_batch_once():
    """bench.py --scaling strong: the ranks' layouts hold every instance of the one
    batch exactly once, each with the shape and seed it has in the whole batch."""
    import bench
    from paper_1902_10078_gb300 import workloads as W
    count = 200
    ns, ls = W.batched_shapes(count, seed=W.BASE_SEED, ls=(1, 2, 3, 5, 7))
    seen = []
    for rank in range(2):
        lay, seeds, order = bench.batch_layout(count, 4, (1, 2, 3, 5, 7), True, rank, 2, True)
        for p, i in enumerate(order):
            assert (lay.ns[p], lay.ls[p]) == (int(ns[i]), int(ls[i]))
            assert seeds[p] == W.BASE_SEED + i
        seen += order
    assert sorted(seen) == list(range(count))


def test_source_hash_ignores_comments_only():
    """The stored traffic stays valid across comment edits of the hot sources,
    not across code edits."""
    code = "int f(int x) {\n    return x + 1;  // one more\n}\n/* block\n comment */\n"
    assert bench._code_only(code) == bench._code_only(code.replace("one more", "the successor"))
    assert bench._code_only(code) == bench._code_only("int f(int x) {\n\n    return x + 1;\n}\n")
    assert bench._code_only(code) != bench._code_only(code.replace("x + 1", "x + 2"))
