"""Cluster parity of the coarse-to-fine loop (Sec. 3.1 stages 2-4, Sec. 3.3)
fed by the GPU's candidates and records, against the oracle's records and its
eager set cover, in both constraint modes.

Cosine mode runs on the 1,000-clip set at T = 0.80 (strict) and 0.78
(relaxed): at the configured T = 0.95 almost no copy of this generator passes,
so no cluster would form.  Edge mode runs on the full 100,000-clip scale set:
every GPU candidate's record is compared with the oracle's field by field, and
the cluster assignment with the oracle's loop.  The oracle's eager set cover
recomputes every score at every step (quadratic in the clip count), so the
oracle loop runs on each connected component of the relaxed graph on its own:
the loop never relates clips of different components (a strict pass implies a
relaxed one, so every edge the loop reads lies inside a component), and
relabelling a component's clips in increasing order keeps every index tie
rule.
"""
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


def _oracle_loop_by_component(n, pairs, strict, relaxed):
    """oracle.cluster_loop run on each connected component of the relaxed
    graph; returns (rep_of, n_clusters)"""
    parent = np.arange(n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in pairs[relaxed]:
        ra, rb = find(int(a)), find(int(b))
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    root = np.array([find(i) for i in range(n)])
    rep_of = np.arange(n)
    n_clusters = 0
    order = np.argsort(root, kind="stable")
    rs = root[order]
    starts = np.flatnonzero(np.r_[True, rs[1:] != rs[:-1]])
    ends = np.r_[starts[1:], n]
    inside = root[pairs[:, 0]] == root[pairs[:, 1]]
    pr_root = root[pairs[:, 0]]
    by_root = {}
    for k in np.flatnonzero(inside):
        by_root.setdefault(int(pr_root[k]), []).append(k)
    for s, e in zip(starts, ends):
        nodes = np.sort(order[s:e])
        if len(nodes) == 1:
            n_clusters += 1
            continue
        sel = np.array(by_root.get(int(rs[s]), []), dtype=np.int64)
        loc = np.searchsorted(nodes, pairs[sel])
        r, k, _ = oracle.cluster_loop(len(nodes), loc, strict[sel], relaxed[sel])
        rep_of[nodes] = nodes[r]
        n_clusters += k
    return rep_of, n_clusters


def test_cosine_cluster_loop_matches_oracle(ctx, torch_cuda, small_wl, small_set):
    import paper_2512_13133_gb300 as pcl
    n = small_wl.n
    P_relax = pcl.params(small_wl.window_dbu, small_wl.pitch_dbu, small_wl.marker_dbu, cos_num=78)
    P_strict = pcl.params(small_wl.window_dbu, small_wl.pitch_dbu, small_wl.marker_dbu, cos_num=80)
    cs = pcl.alloc_clipset(P_relax, small_wl.rect_off, small_wl.rects)
    pcl.pcl_rasterize(ctx, P_relax, cs)
    gp, _ = pcl.candidates(ctx, P_relax, pcl.MODE_COSINE, cs)
    g_relax = pcl.records_to_numpy(pcl.match(ctx, P_relax, pcl.MODE_COSINE, cs, cs, gp))
    g_strict = pcl.records_to_numpy(pcl.match(ctx, P_strict, pcl.MODE_COSINE, cs, cs, gp))
    pairs = np.stack([g_relax["a"], g_relax["b"]], 1).astype(np.int64)
    rep, ncl, rounds = pcl.pcl_cluster_loop(pairs, g_strict["pass_"], g_relax["pass_"], n)

    op, _ = small_set.candidates(oracle.MODE_COSINE, cos_num=78)
    assert set(map(tuple, op.astype(np.int64).tolist())) == set(map(tuple, pairs.tolist()))
    o_relax = small_set.match(op, oracle.MODE_COSINE, cos_num=78)
    o_strict = small_set.match(op, oracle.MODE_COSINE, cos_num=80)
    rep2, ncl2, _ = oracle.cluster_loop(n, op, o_strict["pass_"] > 0, o_relax["pass_"] > 0)
    assert int(o_strict["pass_"].sum()) >= 100  # clusters do form at these thresholds
    assert ncl == ncl2
    assert rep.tolist() == rep2.tolist()
    assert ncl < n - 100


@pytest.mark.parametrize("tol,tol_relax", [(4, 6), (8, 10)])
def test_scale_edge_records_and_clusters_match_oracle(ctx, torch_cuda, tol, tol_relax):
    """100,000 clips of 256^2 px: every edge candidate's record (at the
    relaxed tolerance) equals the oracle's, and the loop's clusters equal the
    oracle loop's (strict tol, relaxed tol + 2 dbu)"""
    import paper_2512_13133_gb300 as pcl
    wl = synth.preset("scale", seed=1)
    n = wl.n
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, edge_tol_dbu=tol_relax)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    gp, gc = pcl.candidates(ctx, P, pcl.MODE_EDGE, cs, cap=1 << 24)
    assert int(gc[:6].sum()) == n * (n - 1) // 2
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, gp))
    pairs = np.stack([g["a"], g["b"]], 1).astype(np.int64)
    orc = oracle.ClipSet(wl, raster=False)
    o = orc.match(pairs, oracle.MODE_EDGE, edge_tol_dbu=tol_relax)
    for f in ("dx_dbu", "dy_dbu", "pass_"):
        np.testing.assert_array_equal(g[f].astype(np.int64), o[f].astype(np.int64), err_msg=f)
    np.testing.assert_array_equal(g["score"].astype(np.int64), o["score"])
    np.testing.assert_array_equal(g["flags"] & 0x38F, o["flags"] & 0x38F)

    def decisions(r, flag_aligned, flag_verify):
        ok = ((r["flags"] & flag_aligned) > 0) & ((r["flags"] & flag_verify) == 0)
        sc = r["score"].astype(np.int64)
        return ok & (sc <= tol), ok & (sc <= tol_relax)

    s_g, r_g = decisions(g, pcl.F_ALIGNED, pcl.F_EDGE_VERIFY_FAIL)
    rep, ncl, _ = pcl.pcl_cluster_loop(pairs, s_g, r_g, n)
    s_o, r_o = decisions(o, oracle.F_ALIGNED, oracle.F_EDGE_VERIFY_FAIL)
    rep2, ncl2 = _oracle_loop_by_component(n, pairs, s_o, r_o)
    assert ncl == ncl2
    np.testing.assert_array_equal(rep, rep2)
    if tol == 8:
        assert ncl < n - 1000  # copies cluster at the loose tolerance
