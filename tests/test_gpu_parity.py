"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bars: bit-exact rasters, signatures, candidate sets, gate counts, shifts,
overlaps and decisions; |sim_gpu - sim_oracle| <= 1e-5 (FP32 cosine); identical
cluster counts.  Workloads are seeded synthetic clip sets (``synth``).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIM_TOL = 1e-5


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


def _gpu_set(ctx, wl, P, with_spec=True):
    import paper_2512_13133_gb300 as pcl
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=with_spec)
    pcl.pcl_rasterize(ctx, P, cs)
    return cs


def _P(wl, **kw):
    import paper_2512_13133_gb300 as pcl
    return pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, **kw)


def _edge_case_workload(W=512, M=32):
    clips = [
        [],                                              # empty
        [],                                              # empty
        [[0, 0, W, W]],                                  # full window
        [[0, 0, 40, 40]],                                # corner, border edges
        [[W - 30, W - 50, W, W]],                        # far corner
        [[100, 100, 101, 101]],                          # sub-pixel rect (no centre inside)
        [[98, 98, 103, 103]],                            # covers exactly one centre
        [[-20, 50, 60, 90], [200, -10, 260, W + 30]],    # coordinates outside the window
        [[10, 10, 200, 200], [100, 100, 300, 300]],      # overlapping rectangles (union)
        [[10, 10, 200, 200], [100, 100, 300, 300]],      # duplicate of the previous clip
    ]
    return synth.from_lists(clips, W, 4, M)


@pytest.mark.parametrize("W,M", [(256, 16), (512, 32), (1024, 64), (2048, 128)])
def test_raster_and_signatures_bit_exact(ctx, W, M):
    import paper_2512_13133_gb300 as pcl
    base = synth.generate(3, n_clips=60, n_seeds=10, n_copies=30, window_dbu=W, margin_dbu=M,
                          min_rects=1, max_rects=30)
    ec = _edge_case_workload(W, M)
    wl = synth.from_lists([base.clip(i).tolist() for i in range(base.n)] +
                          [ec.clip(i).tolist() for i in range(ec.n)], W, 4, M)
    P = _P(wl)
    cs = _gpu_set(ctx, wl, P)
    imgs = pcl.unpack_bits(cs)
    sig = pcl.signatures(cs)
    orc = oracle.ClipSet(wl)
    for c in range(wl.n):
        np.testing.assert_array_equal(imgs[c], orc.image(c), err_msg=f"clip {c}")
        so = orc.signature(c)
        assert sig["pop"][c] == orc.pop(c)
        np.testing.assert_array_equal(sig["rows"][c], so["rows"])
        np.testing.assert_array_equal(sig["cols"][c], so["cols"])
        np.testing.assert_array_equal(sig["blk"][c], so["blk"])
        np.testing.assert_array_equal(sig["dil"][c], so["dil"])


@pytest.mark.parametrize("W,M", [(256, 16), (1024, 64), (2048, 128)])
def test_edge_screen_signatures(ctx, W, M):
    """The edge screen's per-clip structures against their definitions: the
    64 x 64 occupancy grid (cell side W/64; a rectangle of positive area marks
    the cells floor(x0 / c) .. floor((x1 - 1) / c) on both axes, clamped), the
    rectangles' ascending-area order (ties by index) and the bounding box of
    the edges not on the window border."""
    base = synth.generate(5, n_clips=60, n_seeds=10, n_copies=30, window_dbu=W, margin_dbu=M,
                          min_rects=1, max_rects=40)
    ec = _edge_case_workload(W, M)
    wl = synth.from_lists([base.clip(i).tolist() for i in range(base.n)] +
                          [ec.clip(i).tolist() for i in range(ec.n)], W, 4, M)
    cs = _gpu_set(ctx, wl, _P(wl))
    n, nr = wl.n, int(wl.rect_off[-1])
    occ = cs.occ[:n * 512].cpu().numpy().view(np.uint64).reshape(n, 64)
    ro = cs.rorder[:2 * nr].cpu().numpy().view(np.uint16)
    es = cs.esig[:n * 32].cpu().numpy().view(np.int32).reshape(n, 8)
    csz = W // 64

    def cell(v):
        return min(max(v // csz, 0), 63)

    for c in range(n):
        r = wl.clip(c).astype(np.int64)
        grid = np.zeros(64, np.uint64)
        for x0, y0, x1, y1 in r.tolist():
            if x1 <= x0 or y1 <= y0:
                continue
            m = 0
            for cx in range(cell(x0), cell(x1 - 1) + 1):
                m |= 1 << cx
            for cy in range(cell(y0), cell(y1 - 1) + 1):
                grid[cy] |= np.uint64(m)
        np.testing.assert_array_equal(occ[c], grid, err_msg=f"grid of clip {c}")
        o0 = int(wl.rect_off[c])
        area = (r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1])
        np.testing.assert_array_equal(ro[o0:o0 + len(r)], np.argsort(area, kind="stable"), err_msg=f"order {c}")
        xs = [x0 for x0 in r[:, 0].tolist() if x0 != 0] + [x1 for x1 in r[:, 2].tolist() if x1 != W]
        ys = [y0 for y0 in r[:, 1].tolist() if y0 != 0] + [y1 for y1 in r[:, 3].tolist() if y1 != W]
        border = int(len(xs) + len(ys) < 4 * len(r))
        exp = [len(r), int(bool(xs)), min(xs) if xs else 0, max(xs) if xs else 0,
               int(bool(ys)), min(ys) if ys else 0, max(ys) if ys else 0, border]
        np.testing.assert_array_equal(es[c], exp, err_msg=f"edge signature of clip {c}")


def _pairs_set(t):
    a = t.cpu().numpy().astype(np.int64)
    return set(map(tuple, a.tolist()))


@pytest.mark.parametrize("mode", [1, 2])
def test_candidates_small_config_exact(ctx, small_wl, small_set, mode):
    import paper_2512_13133_gb300 as pcl
    P = _P(small_wl)
    cs = _gpu_set(ctx, small_wl, P)
    gp, gcounts = pcl.candidates(ctx, P, mode, cs)
    op, ocounts = small_set.candidates(mode)
    assert _pairs_set(gp) == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gcounts[:6], ocounts[:6].astype(np.int64))


def _compare_records(g, o, cosine=True):
    assert len(g) == len(o)
    np.testing.assert_array_equal(g["a"], o["a"])
    np.testing.assert_array_equal(g["b"], o["b"])
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    np.testing.assert_array_equal((g["flags"] & oracle.F_ALIGNED) > 0, al)
    np.testing.assert_array_equal(g["dx_dbu"][al], o["dx_dbu"][al])
    np.testing.assert_array_equal(g["dy_dbu"][al], o["dy_dbu"][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(g["sim"][al].astype(np.float64) - o["sim"][al]).max(initial=0) <= SIM_TOL
    if not cosine:
        np.testing.assert_array_equal((g["flags"] & oracle.F_EDGE_VERIFY_FAIL) > 0,
                                      (o["flags"] & oracle.F_EDGE_VERIFY_FAIL) > 0)


def _hard_pairs(wl, rng, k):
    """same-seed pairs (the ones with large overlaps) plus random pairs"""
    lab = wl.label
    idx = np.arange(wl.n)
    same = [(i, j) for s in np.unique(lab[lab >= 0]) for i in idx[lab == s] for j in idx[lab == s] if i < j]
    same = np.array(same, dtype=np.int64).reshape(-1, 2)
    if len(same) > k:
        same = same[rng.choice(len(same), k, replace=False)]
    rnd = rng.integers(0, wl.n, size=(k, 2))
    return np.concatenate([same, rnd[rnd[:, 0] != rnd[:, 1]]])


@pytest.mark.parametrize("gates", [True, False])
def test_cosine_match_small_config(ctx, torch_cuda, small_wl, small_set, gates):
    import paper_2512_13133_gb300 as pcl
    rng = np.random.default_rng(1)
    flags = 0 if gates else pcl.P_NO_GATES
    P = _P(small_wl, flags=flags)
    cs = _gpu_set(ctx, small_wl, P)
    pairs = _hard_pairs(small_wl, rng, 1500)
    if gates:
        op, _ = small_set.candidates(oracle.MODE_COSINE)
        pairs = np.concatenate([pairs, op.astype(np.int64)])
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    o = small_set.match(pairs, oracle.MODE_COSINE, use_gates=gates)
    _compare_records(g, o)
    assert ((g["flags"] & pcl.F_FFT_GUARD) > 0).mean() < 0.01


@pytest.mark.parametrize("gates", [True, False])
def test_edge_match_small_config(ctx, torch_cuda, small_wl, small_set, gates):
    import paper_2512_13133_gb300 as pcl
    rng = np.random.default_rng(2)
    P = _P(small_wl, flags=0 if gates else pcl.P_NO_GATES)
    cs = _gpu_set(ctx, small_wl, P, with_spec=False)
    pairs = _hard_pairs(small_wl, rng, 3000)
    op, _ = small_set.candidates(oracle.MODE_EDGE)
    pairs = np.concatenate([pairs, op.astype(np.int64), pairs[:, ::-1]])
    tp = torch_cuda.from_numpy(np.ascontiguousarray(pairs.astype(np.int32))).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, tp))
    o = small_set.match(pairs, oracle.MODE_EDGE, use_gates=gates)
    _compare_records(g, o, cosine=False)


def test_cosine_translates_and_edge_cases(ctx, torch_cuda):
    import paper_2512_13133_gb300 as pcl
    from tests.test_oracle_pins import _translate_workload
    wl = _translate_workload(5, k=20)
    ec = _edge_case_workload()
    wl = synth.from_lists([wl.clip(i).tolist() for i in range(wl.n)] +
                          [ec.clip(i).tolist() for i in range(ec.n)], 512, 4, 32)
    n = wl.n
    pairs = np.array([(i, j) for i in range(n) for j in range(n) if i != j], dtype=np.int64)
    orc = oracle.ClipSet(wl)
    for flags in (0, pcl.P_NO_GATES):
        P = _P(wl, flags=flags)
        cs = _gpu_set(ctx, wl, P)
        tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
        g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
        o = orc.match(pairs, oracle.MODE_COSINE, use_gates=flags == 0)
        _compare_records(g, o)
        assert g["pass_"].sum() >= 40
        ge = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, tp))
        oe = orc.match(pairs, oracle.MODE_EDGE, use_gates=flags == 0)
        _compare_records(ge, oe, cosine=False)


def test_pcm_peak_matches_oracle_where_unambiguous(ctx, torch_cuda, small_wl, small_set):
    import paper_2512_13133_gb300 as pcl
    rng = np.random.default_rng(3)
    P = _P(small_wl, flags=pcl.P_NO_GATES)
    cs = _gpu_set(ctx, small_wl, P)
    pairs = _hard_pairs(small_wl, rng, 150)[:200]
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    checked = 0
    S = small_set.S
    for r, (a, b) in zip(g, pairs):
        w = small_set.pcm_window(int(a), int(b))
        top = np.sort(w.ravel())[::-1]
        if top[0] - top[1] <= 1e-3 * abs(top[0]):
            continue  # parity unpinned: near tie
        dx, dy = oracle.window_peak(w, S)
        assert (r["pcm_dx_dbu"], r["pcm_dy_dbu"]) == (dx * 4, dy * 4)
        checked += 1
    assert checked > 100


def test_cluster_count_matches_oracle(ctx, torch_cuda, small_wl, small_set):
    import paper_2512_13133_gb300 as pcl
    # relaxed edge tolerance for the coarse stage, strict 4 dbu
    P = _P(small_wl, edge_tol_dbu=6)
    cs = _gpu_set(ctx, small_wl, P, with_spec=False)
    gp, _ = pcl.candidates(ctx, P, pcl.MODE_EDGE, cs)
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, gp))
    pairs = np.stack([g["a"], g["b"]], 1).astype(np.int64)
    ver = ((g["flags"] & pcl.F_ALIGNED) > 0) & ((g["flags"] & pcl.F_EDGE_VERIFY_FAIL) == 0)
    rep, ncl, _ = pcl.pcl_cluster_loop(pairs, ver & (g["score"] <= 4), ver & (g["score"] <= 6), small_wl.n)
    op, _ = small_set.candidates(oracle.MODE_EDGE, edge_tol_dbu=6)
    o = small_set.match(op, oracle.MODE_EDGE, edge_tol_dbu=6)
    over = ((o["flags"] & oracle.F_ALIGNED) > 0) & ((o["flags"] & oracle.F_EDGE_VERIFY_FAIL) == 0)
    rep2, ncl2, _ = oracle.cluster_loop(small_wl.n, op, over & (o["score"] <= 4), over & (o["score"] <= 6))
    assert ncl == ncl2
    assert rep.tolist() == rep2.tolist()


def test_full_size_sampled_parity(ctx, torch_cuda):
    """scale configuration (100k clips, 256^2): candidates of the full GPU run
    restricted to a 1500-clip sample equal the oracle's on that sample; a
    sample of matched pairs agrees record by record."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.preset("scale", seed=1)
    P = _P(wl)
    cs = _gpu_set(ctx, wl, P)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(wl.n, 1500, replace=False))
    inv = -np.ones(wl.n, np.int64)
    inv[sample] = np.arange(len(sample))
    sub = wl.subset(sample)
    orc = oracle.ClipSet(sub)
    for mode in (pcl.MODE_COSINE, pcl.MODE_EDGE):
        gp, gc = pcl.candidates(ctx, P, mode, cs, cap=1 << 24)
        assert int(gc[:6].sum()) == wl.n * (wl.n - 1) // 2
        a = gp.cpu().numpy().astype(np.int64)
        keep = (inv[a[:, 0]] >= 0) & (inv[a[:, 1]] >= 0)
        mine = {(int(inv[x]), int(inv[y])) for x, y in a[keep]}
        op, _ = orc.candidates(mode)
        assert mine == set(map(tuple, op.astype(np.int64).tolist()))
        # record parity on up to 2000 GPU candidates plus random pairs
        pick = a[rng.choice(len(a), min(2000, len(a)), replace=False)] if len(a) else a
        rnd = rng.integers(0, wl.n, size=(500, 2))
        pick = np.concatenate([pick, rnd[rnd[:, 0] != rnd[:, 1]]])
        tp = torch_cuda.from_numpy(pick.astype(np.int32)).cuda()
        g = pcl.records_to_numpy(pcl.match(ctx, P, mode, cs, cs, tp))
        full = oracle.ClipSet(wl.subset(np.unique(pick)))
        loc = -np.ones(wl.n, np.int64)
        u = np.unique(pick)
        loc[u] = np.arange(len(u))
        o = full.match(loc[pick], mode)
        o["a"], o["b"] = pick[:, 0], pick[:, 1]
        _compare_records(g, o, cosine=(mode == pcl.MODE_COSINE))


def test_unsupported_and_invalid(ctx, torch_cuda):
    import paper_2512_13133_gb300 as pcl
    # 512² with a marker of 40 px: beyond S <= N/16 for the cosine engines
    wl = synth.from_lists([[[0, 0, 100, 100]], [[10, 10, 90, 90]]], 2048, 4, 160)
    P = _P(wl)
    cs = _gpu_set(ctx, wl, P)
    tp = torch_cuda.tensor([[0, 1]], dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(pcl.PclError) as e:
        pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp)
    assert e.value.status == pcl.PCL_ERR_UNSUPPORTED
    # edge mode covers N = 512
    r = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_EDGE, cs, cs, tp))
    assert r["flags"][0] & pcl.F_ALIGNED


@pytest.mark.parametrize("gates", [True, False])
def test_cosine_512_exact_scan_matches_oracle(ctx, torch_cuda, gates):
    """512² rasters (S = 32): gates, then the exact window scan; records equal
    the oracle's (shift, overlap, decision; |sim diff| <= 1e-5)."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.generate(12, n_clips=60, n_seeds=8, n_copies=40, window_dbu=2048, margin_dbu=128,
                        min_rects=5, max_rects=40)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80 if gates else 95,
                   flags=0 if gates else pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    rng = np.random.default_rng(4)
    lab = wl.label
    same = np.array([(i, j) for i in range(wl.n) for j in range(wl.n) if i != j and lab[i] >= 0 and lab[i] == lab[j]])
    k = 40 if gates else 12
    pairs = np.concatenate([same[rng.choice(len(same), min(k, len(same)), replace=False)],
                            rng.integers(0, wl.n, size=(k // 2, 2)), [[3, 3], [0, 5]]]).astype(np.int64)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE, use_gates=gates, cos_num=80 if gates else 95)
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    assert al.sum() > 0
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f][al], o[f][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(g["sim"][al].astype(np.float64) - o["sim"][al]).max() <= 1e-5


@pytest.mark.parametrize("M", [4, 52, 100])
def test_cosine_512_exact_scan_other_markers(ctx, torch_cuda, M):
    """512² exact window scan at markers whose shift range S = M / p is not a
    multiple of 8 (1, 13, 25 px): the dx chunks start at multiples of 8 and the
    shifts outside the window are dropped; records equal the oracle's."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.generate(21, n_clips=40, n_seeds=6, n_copies=28, window_dbu=2048, margin_dbu=128,
                        min_rects=5, max_rects=40)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, M, cos_num=80, flags=pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    rng = np.random.default_rng(M)
    lab = wl.label
    same = np.array([(i, j) for i in range(wl.n) for j in range(wl.n) if i != j and lab[i] >= 0 and lab[i] == lab[j]])
    pairs = np.concatenate([same[rng.choice(len(same), min(10, len(same)), replace=False)],
                            rng.integers(0, wl.n, size=(4, 2)), [[3, 3]]]).astype(np.int64)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    o = oracle.ClipSet(wl, marker_dbu=M).match(pairs, oracle.MODE_COSINE, use_gates=False, cos_num=80)
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    assert al.sum() >= 10
    assert np.abs(o["dx_dbu"][al]).max() <= M and np.abs(o["dy_dbu"][al]).max() <= M
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f][al], o[f][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(g["sim"][al].astype(np.float64) - o["sim"][al]).max() <= 1e-5


def test_exact_scan_prunes_by_profile_bounds(ctx, torch_cuda):
    """The 512² scan counts only the groups of shifts whose profile bound
    reaches an overlap already found: a clip against itself needs a few
    groups, a clip against an empty clip (bounds 0 = the best overlap) every
    group; the counters add up per aligned pair and the records stay the
    oracle's."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.generate(12, n_clips=30, n_seeds=6, n_copies=20, window_dbu=2048, margin_dbu=128,
                        min_rects=5, max_rects=40)
    clips = [wl.clip(i).tolist() for i in range(wl.n)] + [[]]
    wl = synth.from_lists(clips, 2048, 4, 128)
    empty = wl.n - 1
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80, flags=pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    S = wl.marker_dbu // wl.pitch_dbu
    groups = (2 * S + 1) * (S // 8 + (S + 7) // 8 + 1)

    def run(pairs):
        pcl.pcl_stats_get(ctx, reset=True)
        tp = torch_cuda.tensor(pairs, dtype=torch_cuda.int32, device="cuda")
        g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
        return g, pcl.pcl_stats_get(ctx, reset=True)

    same = [[i, i] for i in range(6)]
    g, (ev, tot) = run(same)
    assert tot == len(same) * groups
    assert 0 < ev <= 0.25 * tot
    assert (g["dx_dbu"] == 0).all() and (g["dy_dbu"] == 0).all() and (g["pass_"] == 1).all()
    g, (ev, tot) = run([[0, empty], [empty, 1]])
    assert ev == tot == 2 * groups
    pairs = np.array([[0, 1], [2, 7], [3, 11], [empty, 4]], dtype=np.int64)
    g, (ev, tot) = run(pairs.tolist())
    assert 0 < ev <= tot == len(pairs) * groups
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE, use_gates=False, cos_num=80)
    for f in ("dx_dbu", "dy_dbu", "pass_"):
        np.testing.assert_array_equal(g[f], o[f])
    np.testing.assert_array_equal(g["score"].astype(np.int64), o["score"])
