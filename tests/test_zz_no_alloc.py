"""The allocation-free cosine candidate entry point against pcl_candidates.

pcl_candidates_cosine_noalloc exists for callers that cannot let the library
call cudaMalloc (device memory owned by another allocator with a fixed
budget, or a service loop that must not synchronise the device to allocate).
It must return exactly what the regular entry point returns -- the candidate
pairs and the gate counts are integers, so the comparison is exact -- and
keep doing so on consecutive calls, since its scratch array persists between
calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pairs(t):
    return set(map(tuple, t.cpu().numpy().astype(np.int64).tolist()))


def _workload(preset, clips):
    if preset == "big512":
        # 512^2 px clips (W = 2048 dbu, S = 32 = N/16), the largest raster the
        # cosine gates take: the area histogram alone is then 2 MiB of scratch
        return synth.generate(5, n_clips=clips, n_seeds=clips // 20, n_copies=int(0.7 * clips), window_dbu=2048,
                              margin_dbu=128, min_rects=5, max_rects=40)
    base = synth.PRESETS[preset]
    f = clips / base["n_clips"]
    return synth.preset(preset, seed=5, n_clips=clips, n_seeds=max(1, int(base["n_seeds"] * f)),
                        n_copies=int(base["n_copies"] * f))


@pytest.mark.parametrize("preset,clips", [("small", 1000), ("scale", 20000), ("big512", 3000)])
def test_noalloc_matches_regular_entry_point_twice(torch_cuda, preset, clips):
    import paper_2512_13133_gb300 as pcl
    torch = torch_cuda
    wl = _workload(preset, clips)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
    ctx = pcl.Context(0)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    ref_pairs, ref_gates = pcl.candidates(ctx, P, pcl.MODE_COSINE, cs, cap=1 << 22)
    cap = max(int(ref_pairs.shape[0]), 1)
    for _ in range(2):
        out = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        gates = torch.zeros(16, dtype=torch.int64, device="cuda")
        pcl.pcl_candidates_cosine_noalloc(ctx, P, cs, out, cnt, gates)
        m = int(cnt.item())
        assert m == ref_pairs.shape[0]
        assert _pairs(out[:m]) == _pairs(ref_pairs)
        np.testing.assert_array_equal(gates.cpu().numpy(), ref_gates)
    ctx.close()


def test_noalloc_rejects_sizes_above_its_scratch(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    torch = torch_cuda
    wl = synth.preset("small", seed=2, n_clips=50, n_seeds=5, n_copies=20)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
    ctx = pcl.Context(0)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    out = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    # the size check happens before any kernel touches the buffers
    with pytest.raises(pcl.PclError) as e:
        pcl.pcl_candidates_cosine_noalloc(ctx, P, cs, out, cnt, None, n_clips=5_000_000)
    assert e.value.status == pcl.PCL_ERR_INVALID
    assert "8 MiB" in str(e.value)
    ctx.close()


def test_noalloc_first_call_on_a_fresh_context_allocates_nothing(torch_cuda):
    """The point of the entry point: a call takes no device memory.  A fresh
    context calls it before the regular entry point has ever grown that
    context's workspace; the device's free memory (cudaMemGetInfo) is the
    same before and after the call, and the result equals the regular entry
    point's computed afterwards on the same context.  The very first call in
    a process may make the CUDA driver load the library's device code (and
    with it the fixed scratch array), so one call on another context comes
    first."""
    import paper_2512_13133_gb300 as pcl
    torch = torch_cuda
    wl = _workload("scale", 5000)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
    warm = pcl.Context(0)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(warm, P, cs)
    cap = 1 << 16
    out = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    gates = torch.zeros(16, dtype=torch.int64, device="cuda")
    pcl.pcl_candidates_cosine_noalloc(warm, P, cs, out, cnt, gates)
    torch.cuda.synchronize()
    warm.close()
    ctx = pcl.Context(0)
    cnt.zero_()
    gates.zero_()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pcl.pcl_candidates_cosine_noalloc(ctx, P, cs, out, cnt, gates)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    m = int(cnt.item())
    assert m <= cap
    got, got_gates = _pairs(out[:m]), gates.cpu().numpy().copy()
    ref_pairs, ref_gates = pcl.candidates(ctx, P, pcl.MODE_COSINE, cs, cap=cap)
    assert got == _pairs(ref_pairs)
    np.testing.assert_array_equal(got_gates, ref_gates)
    ctx.close()


def test_noalloc_limit_for_512_px_clips(torch_cuda):
    """At 512^2 px the scratch holds 8 (N^2 + 2) + 8 n + 192 bytes for at most
    786,406 clips; one clip more is refused before any kernel runs."""
    import paper_2512_13133_gb300 as pcl
    torch = torch_cuda
    wl = _workload("big512", 40)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
    N = wl.raster_n
    n_max = ((8 << 20) - 8 * (N * N + 2) - 192) // 8
    assert n_max == 786_406
    ctx = pcl.Context(0)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    out = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pcl.PclError) as e:
        pcl.pcl_candidates_cosine_noalloc(ctx, P, cs, out, cnt, None, n_clips=n_max + 1)
    assert e.value.status == pcl.PCL_ERR_INVALID
    assert "8 MiB" in str(e.value) and str(n_max + 1) in str(e.value)
    ctx.close()
