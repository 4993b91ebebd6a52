"""One persistent launch over a mixed batch (a9): four raster sizes, cosine
and edge pairs interleaved in one list, Zipf-length candidate lists.  The
records equal those of the per-class entry points and the oracle's, 512²
cosine items (exact window scan) included."""
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
def batch(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    wls, pairs, modes = synth.batched(3, clips_per_class=240)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(pairs), min(len(pairs), 60000), replace=False))
    pairs, modes = pairs[pick], modes[pick]
    order = np.lexsort((pairs[:, 1], pairs[:, 0], modes))  # cosine first, then by class and a
    pairs, modes = pairs[order], modes[order]
    ctx = pcl.Context(0)
    Ps, sets = [], []
    for wl in wls:
        P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
        # the 512² class holds no spectra: its cosine items take the exact window scan
        cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=wl.raster_n <= 256)
        pcl.pcl_rasterize(ctx, P, cs)
        Ps.append(P)
        sets.append(cs)
    work = np.zeros(len(pairs), dtype=pcl.WORK_DTYPE)
    work["cls"], work["a"], work["b"], work["mode"] = pairs[:, 0], pairs[:, 1], pairs[:, 2], modes
    n_cos = int((modes == 1).sum())
    tw = torch_cuda.from_numpy(work.view(np.uint8).reshape(-1, 12)).cuda()
    return dict(pcl=pcl, wls=wls, pairs=pairs, modes=modes, ctx=ctx, Ps=Ps, sets=sets, tw=tw, n_cos=n_cos)


def _run_mixed(b, radix, torch, items=0):
    pcl = b["pcl"]
    out = torch.empty((b["tw"].shape[0], 40), dtype=torch.uint8, device="cuda")
    pcl.pcl_match_mixed(b["ctx"], b["Ps"], b["sets"], b["tw"], b["n_cos"], out, pcl.Tuning(radix, 0, items))
    return pcl.records_to_numpy(out)


EXACT = ["a", "b", "dx_dbu", "dy_dbu", "score", "pass_", "mode"]


@pytest.mark.parametrize("radix,items", [(2, 0), (4, 0), (2, 8), (4, 32), (2, 64), (2, 1)])
def test_mixed_equals_per_class_entry_points(batch, torch_cuda, radix, items):
    """every tuning (register DFT radix, cosine items per warp per round)
    gives the per-class entry points' records"""
    pcl = batch["pcl"]
    g = _run_mixed(batch, radix, torch_cuda, items)
    pairs, modes = batch["pairs"], batch["modes"]
    for k, wl in enumerate(batch["wls"]):
        for mode in (1, 2):
            sel = np.flatnonzero((pairs[:, 0] == k) & (modes == mode))
            if len(sel) == 0:
                continue
            tp = torch_cuda.from_numpy(pairs[sel, 1:].astype(np.int32)).cuda()
            r = pcl.records_to_numpy(pcl.match(batch["ctx"], batch["Ps"][k], mode, batch["sets"][k],
                                               batch["sets"][k], tp))
            for f in EXACT:
                np.testing.assert_array_equal(g[f][sel], r[f], err_msg=f"class {k} mode {mode} field {f}")
            np.testing.assert_array_equal(g["flags"][sel] & 0x39F, r["flags"] & 0x39F)
            assert np.abs(g["sim"][sel] - r["sim"]).max(initial=0) <= 1e-6


def test_mixed_matches_oracle_sample(batch, torch_cuda):
    g = _run_mixed(batch, 4, torch_cuda)
    pairs, modes = batch["pairs"], batch["modes"]
    rng = np.random.default_rng(1)
    for k, wl in enumerate(batch["wls"]):
        orc = oracle.ClipSet(wl)
        for mode in (1, 2):
            sel = np.flatnonzero((pairs[:, 0] == k) & (modes == mode))
            # every aligned pair plus a random sample of the rest
            al = sel[(g["flags"][sel] & (1 << 9)) > 0]
            sel = np.unique(np.concatenate([al[:400], rng.choice(sel, min(400, len(sel)), replace=False)]))
            o = orc.match(pairs[sel, 1:], mode)
            for f in ["dx_dbu", "dy_dbu", "pass_"]:
                m = (o["flags"] & oracle.F_ALIGNED) > 0 if f != "pass_" else np.ones(len(sel), bool)
                np.testing.assert_array_equal(g[f][sel][m], o[f][m], err_msg=f"class {k} mode {mode} {f}")
            np.testing.assert_array_equal(g["flags"][sel] & 15, o["flags"] & 15)
            m = (o["flags"] & oracle.F_ALIGNED) > 0
            np.testing.assert_array_equal(g["score"][sel][m].astype(np.int64), o["score"][m])


def test_mixed_without_gates_and_pcm_rule(torch_cuda):
    """Gates off: every non-empty item reaches its alignment engine (edge
    items the whole-warp Min-Max, cosine items the FFT body or, at 512², the
    exact window scan) and the records still equal the per-class entry
    points'.  With shift_rule = PCM_PEAK the 512² class has no engine: its
    cosine items are reported unsupported, the other classes are unaffected."""
    import paper_2512_13133_gb300 as pcl
    wls, pairs, modes = synth.batched(5, clips_per_class=48)
    rng = np.random.default_rng(2)
    pick = np.sort(rng.choice(len(pairs), min(len(pairs), 1500), replace=False))
    pairs, modes = pairs[pick], modes[pick]
    order = np.lexsort((pairs[:, 1], pairs[:, 0], modes))
    pairs, modes = pairs[order], modes[order]
    ctx = pcl.Context(0)
    work = np.zeros(len(pairs), dtype=pcl.WORK_DTYPE)
    work["cls"], work["a"], work["b"], work["mode"] = pairs[:, 0], pairs[:, 1], pairs[:, 2], modes
    n_cos = int((modes == 1).sum())
    tw = torch_cuda.from_numpy(work.view(np.uint8).reshape(-1, 12)).cuda()
    for flags, rule in ((pcl.P_NO_GATES, pcl.SHIFT_EXACT_ARGMAX), (0, pcl.SHIFT_PCM_PEAK)):
        Ps, sets = [], []
        for wl in wls:
            P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, flags=flags, shift_rule=rule)
            cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=wl.raster_n <= 256)
            pcl.pcl_rasterize(ctx, P, cs)
            Ps.append(P)
            sets.append(cs)
        out = torch_cuda.empty((len(pairs), 40), dtype=torch_cuda.uint8, device="cuda")
        pcl.pcl_match_mixed(ctx, Ps, sets, tw, n_cos, out, pcl.Tuning(2, 0))
        g = pcl.records_to_numpy(out)
        for k, wl in enumerate(wls):
            for mode in (1, 2):
                sel = np.flatnonzero((pairs[:, 0] == k) & (modes == mode))
                if len(sel) == 0:
                    continue
                if mode == 1 and wl.raster_n == 512 and rule == pcl.SHIFT_PCM_PEAK:
                    assert np.all((g["flags"][sel] & 15) == pcl.GATE_UNSUPPORTED)
                    continue
                tp = torch_cuda.from_numpy(pairs[sel, 1:].astype(np.int32)).cuda()
                r = pcl.records_to_numpy(pcl.match(ctx, Ps[k], mode, sets[k], sets[k], tp))
                for f in EXACT:
                    np.testing.assert_array_equal(g[f][sel], r[f], err_msg=f"class {k} mode {mode} field {f}")
                np.testing.assert_array_equal(g["flags"][sel] & 0x39F, r["flags"] & 0x39F)
        if flags:
            assert ((g["flags"] & pcl.F_ALIGNED) > 0).sum() > len(pairs) // 2


def test_mixed_full_size_sampled_parity(torch_cuda):
    """Batched form at full size in the launch configuration the benchmark
    times (autotuned radix and CTAs per SM): 1,000,000 clips (250,000 per
    size class, 64² to 512²), ~3.6e8 Zipf-listed items of both modes in one
    persistent launch.  Per class and mode, up to 300 aligned items and 300
    random ones equal the oracle's records (gate, shift, overlap, decision)."""
    import paper_2512_13133_gb300 as pcl
    from paper_2512_13133_gb300 import autotune
    wls, pairs, modes = synth.batched(1, clips_per_class=250_000)
    # cosine first; within a mode the generator's (class, a) order is kept
    order = np.concatenate([np.flatnonzero(modes == 1), np.flatnonzero(modes == 2)])
    pairs, modes = pairs[order], modes[order]
    assert len(pairs) > 3e8
    ctx = pcl.Context(0)
    Ps, sets = [], []
    for wl in wls:
        P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
        Ps.append(P)
        sets.append(pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=wl.raster_n <= 256))
    work = np.zeros(len(pairs), dtype=pcl.WORK_DTYPE)
    work["cls"], work["a"], work["b"], work["mode"] = pairs[:, 0], pairs[:, 1], pairs[:, 2], modes
    n_cos = int((modes == 1).sum())
    tw = torch_cuda.from_numpy(work.view(np.uint8).reshape(-1, 12)).cuda()
    del work
    out = torch_cuda.empty((len(pairs), 40), dtype=torch_cuda.uint8, device="cuda")

    def raster_all():
        for P, cs in zip(Ps, sets):
            pcl.pcl_rasterize(ctx, P, cs)

    raster_all()
    tune, _ = autotune.tune_mixed(ctx, Ps, sets, tw, n_cos, out, reset=raster_all)
    raster_all()
    pcl.pcl_match_mixed(ctx, Ps, sets, tw, n_cos, out, tune)
    torch_cuda.cuda.synchronize()
    rng = np.random.default_rng(2)
    checked = aligned = 0
    for k, wl in enumerate(wls):
        for mode in (1, 2):
            sel = np.flatnonzero((pairs[:, 0] == k) & (modes == mode))
            if not len(sel):
                continue
            probe = sel[rng.choice(len(sel), min(len(sel), 20000), replace=False)]
            gp = pcl.records_to_numpy(out[torch_cuda.from_numpy(probe).cuda()])
            al = probe[(gp["flags"] & (1 << 9)) > 0][:300]
            pick = np.unique(np.concatenate([al, rng.choice(sel, min(300, len(sel)), replace=False)]))
            g = pcl.records_to_numpy(out[torch_cuda.from_numpy(pick).cuda()])
            ids = np.unique(pairs[pick, 1:].ravel())
            loc = np.searchsorted(ids, pairs[pick, 1:])
            o = oracle.ClipSet(wl.subset(ids)).match(loc, mode)
            np.testing.assert_array_equal(g["flags"] & 15, o["flags"] & 15, err_msg=f"class {k} mode {mode}")
            np.testing.assert_array_equal(g["pass_"], o["pass_"], err_msg=f"class {k} mode {mode}")
            m = (o["flags"] & oracle.F_ALIGNED) > 0
            for f in ("dx_dbu", "dy_dbu"):
                np.testing.assert_array_equal(g[f][m], o[f][m], err_msg=f"class {k} mode {mode} {f}")
            np.testing.assert_array_equal(g["score"][m].astype(np.int64), o["score"][m])
            assert np.abs(g["sim"][m].astype(np.float64) - o["sim"][m]).max(initial=0) <= 1e-5
            checked += len(pick)
            aligned += int(m.sum())
    assert checked > 3000 and aligned > 1000


def test_mixed_graph_replay_equals_eager(batch, torch_cuda):
    """The mixed launch captured once in a CUDA graph and replayed three
    times: each replay rewrites every record (the output is refilled with a
    different byte pattern before each) and equals the eager launch field by
    field, so the work cursor and counters the launch resets are reset inside
    the captured work; a sample of the replayed records equals the oracle's."""
    torch = torch_cuda
    pcl = batch["pcl"]
    tune = pcl.Tuning(4, 0)
    eager = _run_mixed(batch, 4, torch)
    out = torch.empty((batch["tw"].shape[0], 40), dtype=torch.uint8, device="cuda")

    def step():
        pcl.pcl_match_mixed(batch["ctx"], batch["Ps"], batch["sets"], batch["tw"], batch["n_cos"], out, tune)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # warm-up outside the capture (grows the context workspace)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step()
    fields = [f for f in pcl.REC_DTYPE.names if f != "reserved"]
    for k in range(3):
        out.fill_(0x5A + 0x31 * k)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        g = pcl.records_to_numpy(out)
        for f in fields:
            np.testing.assert_array_equal(g[f], eager[f], err_msg=f"replay {k} field {f}")
    pairs, modes = batch["pairs"], batch["modes"]
    rng = np.random.default_rng(9)
    for k, wl in enumerate(batch["wls"]):
        for mode in (1, 2):
            sel = np.flatnonzero((pairs[:, 0] == k) & (modes == mode))
            if not len(sel):
                continue
            al = sel[(g["flags"][sel] & (1 << 9)) > 0][:100]
            sel = np.unique(np.concatenate([al, rng.choice(sel, min(100, len(sel)), replace=False)]))
            o = oracle.ClipSet(wl).match(pairs[sel, 1:], mode)
            np.testing.assert_array_equal(g["flags"][sel] & 15, o["flags"] & 15)
            np.testing.assert_array_equal(g["pass_"][sel], o["pass_"])
            m = (o["flags"] & oracle.F_ALIGNED) > 0
            for f in ("dx_dbu", "dy_dbu"):
                np.testing.assert_array_equal(g[f][sel][m], o[f][m])
            np.testing.assert_array_equal(g["score"][sel][m].astype(np.int64), o["score"][m])
