"""Schedule autotuner: candidate selection, signature and cache (host logic;
plans and timings are replaced by fakes, so no GPU is needed)."""
import json

from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B


class FakePlan:
    def __init__(self, tuning):
        self.tuning = tuning
        self.closed = False

    def close(self):
        self.closed = True


def test_autotune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("BND_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    lay = BT.Layout([5000, 6000, 300], [3, 3, 7], 4, B.BND_F32, panels=True)
    made = []

    def factory(tuning):
        p = FakePlan(tuning)
        made.append(p)
        return p

    cost = {256: 3.0, 384: 1.5, 512: 2.0}
    tuning, timings = BT.autotune(lay, lambda plan: plan.tuning["seg_len"], candidates=(256, 384, 512),
                                  plan_factory=factory, timer=lambda seg, reps, warmup: cost[seg])
    assert tuning == {"seg_len": 384}
    assert timings == {"seg_len=256": 3.0, "seg_len=384": 1.5, "seg_len=512": 2.0}
    assert all(p.closed for p in made) and len(made) == 3
    stored = json.load(open(tmp_path / "tune.json"))
    assert stored[BT.workload_signature(lay)]["tuning"] == {"seg_len": 384}
    # a second call is answered from the cache without building plans
    tuning2, _ = BT.autotune(lay, lambda plan: None, plan_factory=lambda t: 1 / 0, timer=None)
    assert tuning2 == {"seg_len": 384}


def test_autotune_searches_segments_warmups_and_kernels(tmp_path, monkeypatch):
    """The default candidates cover the library defaults, segment length x
    warm-up slope, the direct kernels and no segmentation; the fastest dict is
    returned whole."""
    monkeypatch.setenv("BND_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    lay = BT.Layout([5000, 6000, 300], [3, 3, 7], 4, B.BND_F32, panels=True)

    def cost(tuning):
        if not tuning or tuning.get("flags") or tuning["seg_len"] < 0:
            return 9.0
        return abs(tuning["seg_len"] - 512) / 100 + abs(tuning["warm_per_l"] - 16)

    tuning, timings = BT.autotune(lay, lambda plan: plan.tuning, plan_factory=FakePlan,
                                  timer=lambda t, reps, warmup: cost(t))
    assert tuning == {"seg_len": 512, "warm_per_l": 16, "warm_base": 32}
    assert len(timings) == len(BT.DEFAULT_CANDIDATES) == 15


def test_signature_separates_workloads():
    a = BT.Layout([5000, 6000], [3, 3], 4, B.BND_F32, panels=True)
    b = BT.Layout([5000, 6000], [3, 3], 4, B.BND_F32, panels=False)
    c = BT.Layout([5000, 6000], [3, 5], 4, B.BND_F32, panels=True)
    d = BT.Layout([5001, 6001], [3, 3], 4, B.BND_F32, panels=True)
    assert len({BT.workload_signature(x) for x in (a, b, c)}) == 3
    assert BT.workload_signature(a) == BT.workload_signature(d)     # same coarse histogram
