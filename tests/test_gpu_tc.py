"""Tensor-core direct correlation (a8) against the oracle and the FFT engine:
exact shifts, overlaps and decisions, |sim diff| <= 1e-5, for the three
(N, S) geometries the engine covers -- (64, 4), (128, 8), (256, 16) -- with
FP16, BF16 and E4M3 operands, member batches from one pair to a full item, and the
error for a geometry it does not cover."""
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


def _workload(kind):
    if kind == "n64":
        return synth.generate(5, n_clips=300, n_seeds=30, n_copies=200, window_dbu=256, margin_dbu=16,
                              min_rects=3, max_rects=12)
    if kind == "n128":
        return synth.preset("small", seed=6, n_clips=400, n_seeds=40, n_copies=260)
    return synth.preset("scale", seed=7, n_clips=500, n_seeds=50, n_copies=330)


def _pairs(wl, rng, k):
    lab = wl.label
    same = [(i, j) for i in range(wl.n) for j in range(wl.n) if i != j and lab[i] >= 0 and lab[i] == lab[j]]
    same = np.array(same, dtype=np.int64).reshape(-1, 2)
    if len(same) > k:
        same = same[rng.choice(len(same), k, replace=False)]
    rnd = rng.integers(0, wl.n, size=(k // 4, 2))
    p = np.concatenate([same, rnd[rnd[:, 0] != rnd[:, 1]]])
    return p[np.lexsort((p[:, 1], p[:, 0]))]


@pytest.mark.parametrize("kind", ["n64", "n128", "n256"])
@pytest.mark.parametrize("gates", [False, True])
@pytest.mark.parametrize("engine", ["f16", "bf16", "e4m3"])
def test_tc_engine_matches_oracle_and_fft(torch_cuda, kind, gates, engine):
    import paper_2512_13133_gb300 as pcl
    wl = _workload(kind)
    rng = np.random.default_rng(11)
    pairs = _pairs(wl, rng, 1200)
    flags = 0 if gates else pcl.P_NO_GATES
    num = 80 if gates else 95  # with gates, a looser threshold lets pairs through to the engine
    ctx = pcl.Context(0)
    eng = {"f16": pcl.ENGINE_TC_DIRECT, "bf16": pcl.ENGINE_TC_DIRECT_BF16, "e4m3": pcl.ENGINE_TC_DIRECT_FP8}[engine]
    Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=num, cos_engine=eng, flags=flags)
    Pf = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=num, flags=flags)
    cs = pcl.alloc_clipset(Pf, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, Pf, cs)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    gt = pcl.records_to_numpy(pcl.match(ctx, Pt, pcl.MODE_COSINE, cs, cs, tp))
    assert pcl.pcl_device_error(ctx) == 0
    gf = pcl.records_to_numpy(pcl.match(ctx, Pf, pcl.MODE_COSINE, cs, cs, tp))
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE, use_gates=gates, cos_num=num)
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    assert al.sum() > 0
    np.testing.assert_array_equal(gt["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(gt["pass_"], o["pass_"])
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(gt[f][al], o[f][al])
    np.testing.assert_array_equal(gt["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(gt["sim"][al].astype(np.float64) - o["sim"][al]).max() <= 1e-5
    for f in ("dx_dbu", "dy_dbu", "score", "pass_"):
        np.testing.assert_array_equal(gt[f], gf[f])
    ctx.close()


def _dense_pairs(wl, rng, reps, per_rep):
    """reps representatives, each listed with per_rep distinct members (b != a)."""
    out = []
    for a in rng.choice(wl.n, reps, replace=False):
        bs = rng.choice(np.delete(np.arange(wl.n), a), per_rep, replace=False)
        out += [(int(a), int(b)) for b in sorted(bs)]
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("engine", ["f16", "bf16", "e4m3"])
def test_tc_full_items_and_split_segments(torch_cuda, engine):
    """Representatives with 1, 31, 32, 33 and 70 members: full items of 32
    members, a segment split over three items, and ragged last items."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.preset("scale", seed=8, n_clips=300, n_seeds=30, n_copies=200)
    rng = np.random.default_rng(5)
    pairs = np.concatenate([_dense_pairs(wl, rng, 1, k) for k in (1, 31, 32, 33, 70)])
    eng = {"f16": pcl.ENGINE_TC_DIRECT, "bf16": pcl.ENGINE_TC_DIRECT_BF16, "e4m3": pcl.ENGINE_TC_DIRECT_FP8}[engine]
    ctx = pcl.Context(0)
    Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_engine=eng, flags=pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(Pt, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, Pt, cs)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    gt = pcl.records_to_numpy(pcl.match(ctx, Pt, pcl.MODE_COSINE, cs, cs, tp))
    assert pcl.pcl_device_error(ctx) == 0
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE, use_gates=False)
    for f in ("dx_dbu", "dy_dbu", "pass_"):
        np.testing.assert_array_equal(gt[f], o[f])
    np.testing.assert_array_equal(gt["score"].astype(np.int64), o["score"])
    ctx.close()


def test_tc_rejects_uncovered_geometry(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    wl = synth.preset("scale", seed=9, n_clips=20, n_seeds=4, n_copies=10)
    ctx = pcl.Context(0)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, 80, cos_engine=pcl.ENGINE_TC_DIRECT)  # N = 256, S = 20 > N/16
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    tp = torch_cuda.from_numpy(np.array([[0, 1]], dtype=np.int32)).cuda()
    with pytest.raises(pcl.PclError) as ei:
        pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp)
    assert ei.value.status == pcl.PCL_ERR_UNSUPPORTED
    ctx.close()


def test_tc_wait_limit_times_out_and_context_recovers(torch_cuda):
    """A wait limit far below the engine's hand-over times (1 ns) makes the
    tensor-core launch give up: pcl_device_error reports PCL_ERR_TIMEOUT and
    clears the word.  No GPU fault: the kernel drains its tensor-core work and
    returns.  With the default limit restored, the same context gives the
    oracle's records again."""
    import paper_2512_13133_gb300 as pcl
    wl = _workload("n256")
    rng = np.random.default_rng(12)
    pairs = _pairs(wl, rng, 800)
    ctx = pcl.Context(0)
    Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_engine=pcl.ENGINE_TC_DIRECT,
                    flags=pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(Pt, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, Pt, cs)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    assert pcl.pcl_device_error(ctx) == 0
    pcl.pcl_set_wait_limit(ctx, 1)
    pcl.match(ctx, Pt, pcl.MODE_COSINE, cs, cs, tp)
    with pytest.raises(pcl.PclError) as e:
        pcl.pcl_device_error(ctx)
    assert e.value.status == pcl.PCL_ERR_TIMEOUT
    assert pcl.pcl_device_error(ctx) == 0  # reported once, then cleared
    pcl.pcl_set_wait_limit(ctx, 0)
    g = pcl.records_to_numpy(pcl.match(ctx, Pt, pcl.MODE_COSINE, cs, cs, tp))
    assert pcl.pcl_device_error(ctx) == 0
    o = oracle.ClipSet(wl).match(pairs, oracle.MODE_COSINE, use_gates=False)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f], o[f])
    np.testing.assert_array_equal(g["score"].astype(np.int64), o["score"])
    ctx.close()


@pytest.mark.parametrize("N,S", [(64, 2), (128, 5), (256, 7), (256, 11), (256, 0)])
@pytest.mark.parametrize("engine", ["f16", "e4m3"])
def test_tc_engine_smaller_markers(torch_cuda, N, S, engine):
    """Markers below N/16: the kernel of the size correlates its full window
    and the argmax keeps the shifts |dx|, |dy| <= S; shift, overlap and
    decision equal the oracle's at that marker (and the FFT engine's)."""
    import paper_2512_13133_gb300 as pcl
    kind = {64: "n64", 128: "n128", 256: "n256"}[N]
    wl = _workload(kind)
    M = S * wl.pitch_dbu
    rng = np.random.default_rng(N + S)
    pairs = _pairs(wl, rng, 400)
    eng = {"f16": pcl.ENGINE_TC_DIRECT, "e4m3": pcl.ENGINE_TC_DIRECT_FP8}[engine]
    ctx = pcl.Context(0)
    Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, M, cos_engine=eng, flags=pcl.P_NO_GATES)
    Pf = pcl.params(wl.window_dbu, wl.pitch_dbu, M, flags=pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(Pf, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, Pf, cs)
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    gt = pcl.records_to_numpy(pcl.match(ctx, Pt, pcl.MODE_COSINE, cs, cs, tp))
    assert pcl.pcl_device_error(ctx) == 0
    o = oracle.ClipSet(wl, marker_dbu=M).match(pairs, oracle.MODE_COSINE, use_gates=False)
    assert np.abs(gt["dx_dbu"]).max() <= M and np.abs(gt["dy_dbu"]).max() <= M
    for f in ("dx_dbu", "dy_dbu", "pass_"):
        np.testing.assert_array_equal(gt[f], o[f])
    np.testing.assert_array_equal(gt["score"].astype(np.int64), o["score"])
    assert np.abs(gt["sim"].astype(np.float64) - o["sim"]).max() <= 1e-5
    if S > 0:
        gf = pcl.records_to_numpy(pcl.match(ctx, Pf, pcl.MODE_COSINE, cs, cs, tp))
        for f in ("dx_dbu", "dy_dbu", "score", "pass_"):
            np.testing.assert_array_equal(gt[f], gf[f])
    ctx.close()
