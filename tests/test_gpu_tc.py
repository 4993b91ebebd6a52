"""Tensor-core direct correlation (a8) against the oracle and the FFT engine:
exact shifts, overlaps and decisions, |sim diff| <= 1e-5, on raster sizes that
need one, three and nine 128-shift tiles."""
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
def test_tc_engine_matches_oracle_and_fft(torch_cuda, kind, gates):
    import paper_2512_13133_gb300 as pcl
    wl = _workload(kind)
    rng = np.random.default_rng(11)
    pairs = _pairs(wl, rng, 1200)
    flags = 0 if gates else pcl.P_NO_GATES
    num = 80 if gates else 95  # with gates, a looser threshold lets pairs through to the engine
    ctx = pcl.Context(0)
    Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=num, cos_engine=pcl.ENGINE_TC_DIRECT,
                    flags=flags)
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
