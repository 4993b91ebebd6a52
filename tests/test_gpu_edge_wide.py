"""Edge mode on clips with many polygons: the edge screen's warp-cooperative
correspondence holds up to 32 or 64 large-side polygons in registers and
falls back to a chunked scan beyond; the one-pair-per-warp Min-Max falls back
to the per-thread procedure beyond 64.  Clips of 28-89 polygons, plus regular
arrays of exactly 31, 32, 33, 63, 64, 65 and 70 squares with translated and
jittered copies, exercise every path.  Candidate sets and gate counts are
compared exactly with the oracle, records field by field (Sec. 2.2.2,
Sec. 3.2.2 Eq. 6)."""
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


def _squares(k, dx=0, dy=0, jitter=None, W=1024, side=20, pitch=36, x0=80, y0=80):
    """k squares on a 20-column grid, moved by (dx, dy); jitter[i] moves square
    i's right edge (a size change the Min-Max tolerance must absorb or not)"""
    out = []
    for i in range(k):
        x, y = x0 + (i % 20) * pitch + dx, y0 + (i // 20) * pitch + dy
        e = 0 if jitter is None else int(jitter[i])
        out.append([x, y, min(x + side + e, W), min(y + side, W)])
    return out


@pytest.fixture(scope="module")
def wide_wl():
    base = synth.generate(5, n_clips=240, n_seeds=24, n_copies=180, window_dbu=1024, margin_dbu=64,
                          min_rects=30, max_rects=100, min_side=16, max_side=60, grid=8, spacing=12)
    rng = np.random.default_rng(7)
    extra = []
    for k in (31, 32, 33, 63, 64, 65, 70):
        extra.append(_squares(k))
        extra.append(_squares(k, dx=5, dy=-3))                                   # pure translate
        extra.append(_squares(k, dx=-2, dy=4, jitter=rng.integers(-3, 4, k)))    # within tolerance or not
        extra.append(_squares(k - 1, dx=1))                                       # one polygon fewer
    clips = [base.clip(i).tolist() for i in range(base.n)] + extra
    return synth.from_lists(clips, base.window_dbu, base.pitch_dbu, base.marker_dbu)


def _gpu_set(ctx, wl, P):
    import paper_2512_13133_gb300 as pcl
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    return cs


def test_wide_workload_spans_the_paths(wide_wl):
    c = np.diff(wide_wl.rect_off.astype(np.int64))
    assert (c <= 32).sum() > 0 and ((c > 32) & (c <= 64)).sum() > 10 and (c > 64).sum() > 10


def test_edge_candidates_many_polygons_exact(ctx, wide_wl):
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(wide_wl.window_dbu, wide_wl.pitch_dbu, wide_wl.marker_dbu)
    cs = _gpu_set(ctx, wide_wl, P)
    gp, gcounts = pcl.candidates(ctx, P, pcl.MODE_EDGE, cs)
    op, ocounts = oracle.ClipSet(wide_wl).candidates(oracle.MODE_EDGE)
    got = set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist()))
    assert got == set(map(tuple, op.astype(np.int64).tolist()))
    assert len(got) > 50  # correspondences were really checked
    np.testing.assert_array_equal(gcounts[:6], ocounts[:6].astype(np.int64))


@pytest.mark.parametrize("gates", [True, False])
def test_edge_records_many_polygons(ctx, torch_cuda, wide_wl, gates):
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(wide_wl.window_dbu, wide_wl.pitch_dbu, wide_wl.marker_dbu,
                   flags=0 if gates else pcl.P_NO_GATES)
    cs = _gpu_set(ctx, wide_wl, P)
    orc = oracle.ClipSet(wide_wl)
    op, _ = orc.candidates(oracle.MODE_EDGE)
    n = wide_wl.n
    rng = np.random.default_rng(3)
    tail = np.arange(n - 28, n)  # the square arrays: every pair among them
    sq = np.array([(i, j) for i in tail for j in tail if i != j])
    pairs = np.concatenate([op.astype(np.int64), op[:, ::-1].astype(np.int64), sq,
                            rng.integers(0, n, size=(600, 2))])
    tp = torch_cuda.from_numpy(np.ascontiguousarray(pairs.astype(np.int32))).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, tp))
    o = orc.match(pairs, oracle.MODE_EDGE, use_gates=gates)
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    np.testing.assert_array_equal((g["flags"] & oracle.F_ALIGNED) > 0, al)
    assert al.sum() > 100 and o["pass_"].sum() > 10
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f][al], o[f][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    np.testing.assert_array_equal((g["flags"] & oracle.F_EDGE_VERIFY_FAIL) > 0,
                                  (o["flags"] & oracle.F_EDGE_VERIFY_FAIL) > 0)
