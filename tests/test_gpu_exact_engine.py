"""The exact-scan cosine engine (PCL_ENGINE_EXACT_SCAN) at 128² and 256²
against the oracle and against the FFT engine, through the C ABI.

The engine counts c(s) by popcount over the groups of shifts whose projection-
profile bound reaches an overlap already counted, so its shift, overlap and
decision must be the oracle's exact argmax (tie order (-c, |dx|+|dy|, dy, dx))
and its similarity within 1e-5.
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


def _pairs(wl, k, seed):
    rng = np.random.default_rng(seed)
    lab = wl.label
    same = np.array([(i, j) for i in range(wl.n) for j in range(wl.n) if i != j and lab[i] >= 0 and lab[i] == lab[j]])
    return np.concatenate([same[rng.choice(len(same), min(k, len(same)), replace=False)],
                           rng.integers(0, wl.n, size=(k // 2, 2)), [[3, 3], [0, 5]]]).astype(np.int64)


@pytest.mark.parametrize("W,M", [(512, 32), (1024, 64), (1024, 28)])
@pytest.mark.parametrize("gates", [True, False])
def test_exact_scan_engine_matches_oracle(ctx, torch_cuda, W, M, gates):
    """128² (S = 8) and 256² (S = 16, and S = 7: chunks of dx not aligned to
    the window), with and without the lossless gates; empty clips included."""
    import paper_2512_13133_gb300 as pcl
    base = synth.generate(7, n_clips=60, n_seeds=8, n_copies=40, window_dbu=W, margin_dbu=M,
                          min_rects=5, max_rects=40)
    wl = synth.from_lists([base.clip(i).tolist() for i in range(base.n)] + [[], []], W, 4, M)
    wl.label[:base.n] = base.label
    cn = 80 if gates else 95
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, M, cos_num=cn, cos_engine=pcl.ENGINE_EXACT_SCAN,
                   flags=0 if gates else pcl.P_NO_GATES)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    pairs = np.concatenate([_pairs(wl, 40, W + M), [[wl.n - 1, wl.n - 2], [wl.n - 1, 2], [4, wl.n - 2]]])
    tp = torch_cuda.from_numpy(pairs.astype(np.int32)).cuda()
    g = pcl.records_to_numpy(pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp))
    o = oracle.ClipSet(wl, marker_dbu=M).match(pairs, oracle.MODE_COSINE, use_gates=gates, cos_num=cn)
    al = (o["flags"] & oracle.F_ALIGNED) > 0
    assert al.sum() >= 10
    np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15)
    np.testing.assert_array_equal(g["pass_"], o["pass_"])
    for f in ("dx_dbu", "dy_dbu"):
        np.testing.assert_array_equal(g[f][al], o[f][al])
    np.testing.assert_array_equal(g["score"][al].astype(np.int64), o["score"][al])
    assert np.abs(g["sim"][al].astype(np.float64) - o["sim"][al]).max() <= SIM_TOL


def test_exact_scan_engine_equals_fft_engine(ctx, torch_cuda, small_wl):
    """On the small configuration (128², S = 8) every same-seed pair gets the
    FFT engine's shift, overlap and decision from the exact scan, which needs
    no spectra and counts part of the window (pcl_stats_get)."""
    import paper_2512_13133_gb300 as pcl
    wl = small_wl
    lab = wl.label
    pairs = np.array([(i, j) for i in range(wl.n) for j in range(i + 1, wl.n) if lab[i] >= 0 and lab[i] == lab[j]],
                     dtype=np.int32)
    tp = torch_cuda.from_numpy(np.ascontiguousarray(pairs)).cuda()
    Pf = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, flags=pcl.P_NO_GATES)
    csf = pcl.alloc_clipset(Pf, wl.rect_off, wl.rects, with_spec=True)
    pcl.pcl_rasterize(ctx, Pf, csf)
    f = pcl.records_to_numpy(pcl.match(ctx, Pf, pcl.MODE_COSINE, csf, csf, tp))
    Pe = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_engine=pcl.ENGINE_EXACT_SCAN,
                    flags=pcl.P_NO_GATES)
    cse = pcl.alloc_clipset(Pe, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, Pe, cse)
    pcl.pcl_stats_get(ctx, reset=True)
    e = pcl.records_to_numpy(pcl.match(ctx, Pe, pcl.MODE_COSINE, cse, cse, tp))
    ev, tot = pcl.pcl_stats_get(ctx, reset=True)
    S = wl.marker_dbu // wl.pitch_dbu
    assert tot == len(pairs) * (2 * S + 1) * (S // 8 + (S + 7) // 8 + 1)
    assert 0 < ev < tot
    for fld in ("dx_dbu", "dy_dbu", "score", "pass_"):
        np.testing.assert_array_equal(e[fld], f[fld], err_msg=fld)
    assert np.abs(e["sim"].astype(np.float64) - f["sim"].astype(np.float64)).max() <= SIM_TOL
    assert ((e["flags"] & pcl.F_ALIGNED) > 0).all()


def test_exact_scan_engine_limits(ctx, torch_cuda):
    """64² and S > N/16 are outside the engine; the PCM-peak rule too."""
    import paper_2512_13133_gb300 as pcl
    wl = synth.from_lists([[[0, 0, 100, 100]], [[10, 10, 90, 90]]], 256, 4, 16)
    tp = torch_cuda.tensor([[0, 1]], dtype=torch_cuda.int32, device="cuda")
    for W, M, rule in ((256, 16, pcl.SHIFT_EXACT_ARGMAX), (512, 64, pcl.SHIFT_EXACT_ARGMAX),
                       (512, 32, pcl.SHIFT_PCM_PEAK)):
        w = synth.from_lists([wl.clip(0).tolist(), wl.clip(1).tolist()], W, 4, M)
        P = pcl.params(W, 4, M, cos_engine=pcl.ENGINE_EXACT_SCAN, shift_rule=rule)
        cs = pcl.alloc_clipset(P, w.rect_off, w.rects, with_spec=False)
        pcl.pcl_rasterize(ctx, P, cs)
        with pytest.raises(pcl.PclError) as err:
            pcl.match(ctx, P, pcl.MODE_COSINE, cs, cs, tp)
        assert err.value.status == pcl.PCL_ERR_UNSUPPORTED
