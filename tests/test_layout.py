"""Host-side pool layouts (batch.Layout): offsets, strides and views of the
rows and panel arrangements, and pack/unpack round trips."""
import numpy as np
import pytest

from paper_1902_10078_gb300 import batch as BT
from paper_1902_10078_gb300 import binding as B


def test_rows_layout_offsets_and_round_trip():
    ns, ls = [5, 40, 33], [2, 1, 3]
    lay = BT.Layout(ns, ls, 2, B.BND_F64)
    assert lay.cs == 1 and lay.ld == [32, 64, 64]
    assert lay.band_off == [0, 3 * 32, 3 * 32 + 2 * 64]
    rng = np.random.default_rng(0)
    arrs = [rng.normal(size=(l + 1, n)) for n, l in zip(ns, ls)]
    rhs = [rng.normal(size=(2, n)) for n in ns]
    pool, rpool = lay.pack_band(arrs, fill=np.nan), lay.pack_rhs(rhs, fill=np.nan)
    for a, b in zip(arrs, lay.unpack_band(pool)):
        assert np.array_equal(a, b)
    for a, b in zip(rhs, lay.unpack_rhs(rpool)):
        assert np.array_equal(a, b)
    # element (d, j) of instance i sits at band + d ld + j
    i, d, j = 2, 3, 7
    assert pool[lay.band_off[i] + d * lay.ld[i] + j] == arrs[i][d, j]


def test_panel_layout_groups_lanes_and_views():
    ns = [100, 90, 80, 7] + [50] * 33
    ls = [2, 2, 2, 2] + [4] * 33
    lay = BT.Layout(ns, ls, 1, B.BND_F32, panels=True)
    # runs of equal l, at most 32 lanes: l=2 (4 lanes), l=4 (32 + 1 lanes)
    assert [(g[0], g[1]) for g in lay.groups] == [(0, 4), (4, 36), (36, 37)]
    assert lay.cs == 32 and all(ld % 32 == 0 for ld in lay.ld)
    for g, (i0, i1, ob, orr, ng) in enumerate(lay.groups):
        assert ng == (max(ns[i0:i1]) + 3) // 4 * 4
        for p, i in enumerate(range(i0, i1)):
            assert lay.band_off[i] == ob + p and lay.rhs_off[i] == orr + p and lay.lane[i] == p
            assert lay.ld[i] == 32 * ng
        assert ob % 32 == 0
    rng = np.random.default_rng(1)
    arrs = [rng.normal(size=(l + 1, n)).astype(np.float32) for n, l in zip(ns, ls)]
    pool = lay.pack_band(arrs, fill=np.nan)
    back = lay.unpack_band(pool)
    for a, b in zip(arrs, back):
        assert np.array_equal(a.astype(np.float64), b)
    # column j of a group's lanes is contiguous: element (d, j) of lane p at band_g + d ld + 32 j + p
    i, d, j = 2, 1, 11
    assert pool[lay.band_off[i] + d * lay.ld[i] + 32 * j] == arrs[i][d, j]
    # everything outside the instances kept the fill
    inside = np.zeros(lay.band_elems, bool)
    for k in range(lay.count):
        lay.band_view(inside, k)[: ls[k] + 1] = True
    assert np.all(np.isnan(pool[~inside]))
    assert lay.band_elems >= max(ob + (ls[i0] + 1) * 32 * ng for i0, _, ob, _, ng in lay.groups)


def test_panel_order_fills_groups():
    ns, ls = [10, 500, 20, 400, 30], [3, 1, 3, 1, 2]
    order = BT.panel_order(ns, ls)
    assert [ls[i] for i in order] == [1, 1, 2, 3, 3]
    assert [ns[i] for i in order] == [500, 400, 30, 20, 10]


@pytest.mark.parametrize("panels", [False, True])
def test_layout_insts_describe_the_pools(panels):
    lay = BT.Layout([64, 3], [1, 1], 2, B.BND_F32, panels=panels)
    for d in lay.insts():
        assert d["cs"] == (32 if panels else 1)
        assert d["ld"] >= d["n"] * d["cs"] and d["ldr"] >= d["n"] * d["cs"]


def test_gmrf_graph_is_banded_spd_laplacian():
    """The synthetic graph GMRF: after the reverse Cuthill-McKee reordering every
    edge lies inside the returned band, the diagonal is kappa^2 + degree, and the
    precision is SPD (dense eigenvalues at small N)."""
    import numpy as np
    from paper_1902_10078_gb300 import workloads as W
    N = 300
    Q, l, perm, edges = W.gmrf_graph(N, seed=5)
    assert Q.shape == (l + 1, N)
    assert sorted(perm.tolist()) == list(range(N))
    inv = np.empty(N, dtype=int)
    inv[perm] = np.arange(N)
    D = W.dense_from_lower_band(Q, True)
    for a, b in edges:
        i, j = inv[a], inv[b]
        assert abs(i - j) <= l and D[i, j] == -1.0
    assert np.count_nonzero(np.tril(D, -1)) == len(edges)
    assert np.allclose(np.diag(D) - 0.1, -(D - np.diag(np.diag(D))).sum(axis=1))
    assert np.linalg.eigvalsh(D).min() > 0.0
    assert l < N // 4                          # the reordering made it narrow
