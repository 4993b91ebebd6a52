"""Self-join candidates at clip counts around the tile sizes of the screens
(the edge screen takes 32 row clips and 256 column clips per block; the band
join walks bands of the area order): 2, 3, 31, 33, 257 and 300 clips, with
empty clips and identical copies mixed in.  Candidate sets and gate counts
must equal the oracle's exhaustive screen exactly, in both modes."""
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


def _workload(n):
    base = synth.preset("small", seed=3, n_clips=max(n, 4), n_seeds=max(1, n // 6), n_copies=int(0.6 * max(n, 4)))
    clips = [base.clip(i).tolist() for i in range(n)]
    # empty clips and exact duplicates at tile edges
    for k in (0, n // 2, n - 1):
        if 0 <= k < n and k % 3 == 0:
            clips[k] = []
    if n > 32:
        clips[32] = list(clips[31])
    return synth.from_lists(clips, base.window_dbu, base.pitch_dbu, base.marker_dbu)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 257, 300])
@pytest.mark.parametrize("mode", [1, 2])
def test_candidates_at_tile_edges(ctx, n, mode):
    import paper_2512_13133_gb300 as pcl
    wl = _workload(n)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    gp, gcounts = pcl.candidates(ctx, P, mode, cs)
    op, ocounts = oracle.ClipSet(wl).candidates(mode, cos_num=80)
    got = set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist()))
    assert got == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gcounts[:6], ocounts[:6].astype(np.int64))
    assert gcounts[:6].sum() == n * (n - 1) // 2


@pytest.mark.parametrize("tol", [4, 6])
def test_candidates_and_records_across_edge_gate_bounds(ctx, torch_cuda, tol):
    """Clips whose passing edge pairs sit exactly on E2's bound (bbox sizes
    2*tol apart, residual tol) or have unequal polygon counts with far wider
    bboxes (synth.gate_bounds_set, built for tol = 4): candidate sets, gate
    counts and the records of every pair equal the oracle's in both modes,
    and the passing pairs are among the candidates."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.gate_bounds_set(41, tol_dbu=4)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, edge_tol_dbu=tol)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    orc = oracle.ClipSet(wl)
    n = wl.n
    allp = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.int64)
    for mode in (1, 2):
        gp, gcounts = pcl.candidates(ctx, P, mode, cs)
        op, ocounts = orc.candidates(mode, edge_tol_dbu=tol)
        got = set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist()))
        assert got == set(map(tuple, op.astype(np.int64).tolist()))
        np.testing.assert_array_equal(gcounts[:6], ocounts[:6].astype(np.int64))
        tp = torch_cuda.from_numpy(allp.astype(np.int32)).cuda()
        g = pcl.records_to_numpy(pcl.match(ctx, P, mode, cs, cs, tp))
        o = orc.match(allp, mode, edge_tol_dbu=tol)
        np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
        np.testing.assert_array_equal(g["pass_"], o["pass_"])
        al = (o["flags"] & oracle.F_ALIGNED) > 0
        for f in ("dx_dbu", "dy_dbu"):
            np.testing.assert_array_equal(g[f][al], o[f][al])
        np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
        assert int(o["pass_"].sum()) >= 48
        passing = {(int(a), int(b)) for a, b in allp[o["pass_"] > 0]}
        assert passing <= got


@pytest.mark.parametrize("n", [33, 300, 1000])
@pytest.mark.parametrize("mode", [1, 2])
def test_topological_prescreen_candidates_match_oracle(ctx, torch_cuda, n, mode):
    """the lossy topological pre-screen (PCL_P_TOPO_HASH): candidate sets and
    gate counts (T0 included) equal the oracle's screen with the same rule"""
    import paper_2512_13133_gb300 as pcl
    wl = _workload(n)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80, edge_tol_dbu=8, flags=pcl.P_TOPO_HASH)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    gp, gc = pcl.candidates(ctx, P, mode, cs)
    op, oc = oracle.ClipSet(wl).candidates(mode, cos_num=80, edge_tol_dbu=8, topo=True)
    got = set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist()))
    assert got == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gc[:7], oc[:7].astype(np.int64))
    assert gc[:7].sum() == n * (n - 1) // 2
