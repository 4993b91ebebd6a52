"""Degrees, surprisal weights and first-step scores of the pass graph on the
GPU (Sec. 3.3.1, Eqs. 7-9) against the oracle's plain loops, exact, and the
coarse-to-fine loop with a low-resolution coarse stage (Sec. 3.1 stages 2-4:
relaxed decisions at half the resolution, strict ones at full resolution)
against the same sequence run on the oracle."""
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


@pytest.mark.parametrize("n,m,seed", [(1, 0, 0), (10, 14, 1), (1000, 5000, 2), (200_000, 3_000_000, 3)])
def test_surprisal_matches_oracle_on_random_graphs(ctx, torch_cuda, n, m, seed):
    import paper_2512_13133_gb300 as pcl
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, size=(m, 2))
    e = e[e[:, 0] != e[:, 1]]
    te = torch_cuda.from_numpy(e.astype(np.int32).reshape(-1, 2)).cuda()
    deg, w, sc = pcl.pcl_surprisal(ctx, te, n)
    if n <= 1000:
        odeg, ow, osc = oracle.surprisal_scores(n, e)
    else:  # the oracle's loops restated with numpy scatter-adds for size
        odeg = np.zeros(n, np.int64)
        np.add.at(odeg, e[:, 0], 1)
        np.add.at(odeg, e[:, 1], 1)
        ow = (np.int64(1) << 32) // (1 + odeg)
        osc = ow.copy()
        np.add.at(osc, e[:, 0], ow[e[:, 1]])
        np.add.at(osc, e[:, 1], ow[e[:, 0]])
        k = rng.choice(n, 200, replace=False)
        d2, w2, s2 = oracle.surprisal_scores(n, e)
        assert (d2[k] == odeg[k]).all() and (s2[k] == osc[k]).all()
    np.testing.assert_array_equal(deg.cpu().numpy().astype(np.int64), odeg)
    np.testing.assert_array_equal(w.cpu().numpy(), ow)
    np.testing.assert_array_equal(sc.cpu().numpy(), osc)


def test_surprisal_of_a_pass_graph_and_device_count(ctx, torch_cuda, small_wl):
    """the pass graph of the 1,000-clip set at T = 0.80, its length read on
    the device (d_n) from a buffer with room to spare"""
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(small_wl.window_dbu, small_wl.pitch_dbu, small_wl.marker_dbu, cos_num=80)
    cs = pcl.alloc_clipset(P, small_wl.rect_off, small_wl.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    gp, _ = pcl.candidates(ctx, P, pcl.MODE_COSINE, cs)
    rec = pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, gp)
    out = torch_cuda.zeros((gp.shape[0] + 100, 2), dtype=torch_cuda.int32, device="cuda")
    cnt = torch_cuda.zeros(1, dtype=torch_cuda.int64, device="cuda")
    pcl.pcl_compact_pass(ctx, rec, out, cnt)
    m = int(cnt.item())
    assert m > 100
    deg, w, sc = pcl.pcl_surprisal(ctx, out, small_wl.n, d_n=cnt)
    e = out[:m].cpu().numpy().astype(np.int64)
    odeg, ow, osc = oracle.surprisal_scores(small_wl.n, e)
    np.testing.assert_array_equal(deg.cpu().numpy().astype(np.int64), odeg)
    np.testing.assert_array_equal(sc.cpu().numpy(), osc)


@pytest.mark.parametrize("mode", [1, 2])
def test_low_resolution_coarse_stage_matches_oracle(ctx, torch_cuda, small_wl, mode):
    """coarse stage at pitch 8 dbu (64^2 px, S = 4) with relaxed thresholds
    (cosine 0.78, edge tol + 2), strict decisions at pitch 4 (128^2 px,
    cosine 0.80 / edge tol 6): the same sequence on the oracle gives the same
    clusters"""
    import paper_2512_13133_gb300 as pcl
    from paper_2512_13133_gb300 import loop
    P = pcl.params(small_wl.window_dbu, small_wl.pitch_dbu, small_wl.marker_dbu, cos_num=80, edge_tol_dbu=6)
    cs = pcl.alloc_clipset(P, small_wl.rect_off, small_wl.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    rep, ncl, rounds, info = loop.coarse_to_fine(ctx, P, cs, small_wl.rect_off, small_wl.rects, mode=mode)
    # the oracle: the same workload at both pitches
    coarse = synth.Workload(small_wl.name, small_wl.window_dbu, 8, small_wl.marker_dbu, small_wl.rect_off,
                            small_wl.rects, small_wl.label)
    oc, of = oracle.ClipSet(coarse), oracle.ClipSet(small_wl)
    kw_c = dict(cos_num=78, edge_tol_dbu=8)
    op, _ = oc.candidates(mode, **kw_c)
    assert int(len(op)) == info["coarse_pairs"]
    r_c = oc.match(op, mode, **kw_c)
    r_f = of.match(op, mode, cos_num=80, edge_tol_dbu=6)
    if mode == 2:
        def ok(r, tol):
            good = ((r["flags"] & oracle.F_ALIGNED) > 0) & ((r["flags"] & oracle.F_EDGE_VERIFY_FAIL) == 0)
            return good & (r["score"] <= tol)
        relaxed, strict = ok(r_c, 8), ok(r_f, 6)
    else:
        relaxed, strict = r_c["pass_"] > 0, r_f["pass_"] > 0
    assert int(relaxed.sum()) == info["relaxed"] and int(strict.sum()) == info["strict"]
    rep2, ncl2, _ = oracle.cluster_loop(small_wl.n, op, strict, relaxed)
    assert ncl == ncl2
    assert rep.tolist() == rep2.tolist()
    assert ncl < small_wl.n - (50 if mode == 1 else 20)  # clusters form
