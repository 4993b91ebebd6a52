"""Cosine engine with the XY-separation interval-competition shift (Sec.
3.2.1 (2)) against the oracle's statement of it: the synthesised shift, the
exact overlap there, the decision and the gate, field by field, on same-seed
and random pairs of the small and 512² configurations, with and without gates,
plus clips of more than 32 polygons (the lanes' second round)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    return pcl.Context(0)


def _pairs(wl, rng, k):
    lab = wl.label
    idx = np.arange(wl.n)
    same = [(i, j) for s in np.unique(lab[lab >= 0]) for i in idx[lab == s] for j in idx[lab == s] if i != j]
    same = np.array(same, dtype=np.int64).reshape(-1, 2)
    if len(same) > k:
        same = same[rng.choice(len(same), k, replace=False)]
    rnd = rng.integers(0, wl.n, size=(k, 2))
    return np.concatenate([same, rnd, [[0, 0], [3, 3]]])


def _check(ctx, torch_cuda, wl, pairs, gates, **kw):
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_engine=pcl.ENGINE_XYSEP,
                   flags=0 if gates else pcl.P_NO_GATES, **kw)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    tp = torch_cuda.from_numpy(np.ascontiguousarray(pairs.astype(np.int32))).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE_XYSEP, use_gates=gates, **kw)
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    np.testing.assert_array_equal((g["flags"] & oracle.F_ALIGNED) > 0, al)
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f][al], o[f][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(g["sim"][al].astype(np.float64) - o["sim"][al]).max(initial=0) <= 1e-5
    return g, o


@pytest.mark.parametrize("gates", [True, False])
def test_xysep_small_config(ctx, torch_cuda, gates):
    wl = synth.preset("small", seed=1)
    pairs = _pairs(wl, np.random.default_rng(5), 2000)
    g, o = _check(ctx, torch_cuda, wl, pairs, gates, cos_num=80)
    assert ((o["flags"] & oracle.F_ALIGNED) > 0).sum() > 100


def test_xysep_512_and_many_polygons(ctx, torch_cuda):
    wl = synth.generate(7, n_clips=80, n_seeds=8, n_copies=60, window_dbu=2048, margin_dbu=128,
                        min_rects=20, max_rects=70, min_side=16, max_side=80, grid=8, spacing=12)
    assert np.diff(wl.rect_off.astype(np.int64)).max() > 32
    pairs = _pairs(wl, np.random.default_rng(6), 300)
    _check(ctx, torch_cuda, wl, pairs, False)


def test_xysep_translates_land_on_exact_shift(ctx, torch_cuda):
    base = [[100, 120, 160, 180], [220, 300, 300, 330], [330, 90, 380, 250]]
    clips = [base] + [[[r[0] + tx, r[1] + ty, r[2] + tx, r[3] + ty] for r in base]
                      for tx, ty in [(8, -12), (-32, 32), (6, -6), (5, -7), (100, 0)]]
    wl = synth.from_lists(clips, 512, 4, 32)
    pairs = np.array([[0, k] for k in range(1, len(clips))], dtype=np.int64)
    g, _ = _check(ctx, torch_cuda, wl, pairs, False)
    assert list(zip(g["dx_dbu"], g["dy_dbu"])) == [(-8, 12), (32, -32), (-8, 8), (-4, 8), (-32, 0)]
