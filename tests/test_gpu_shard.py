"""Several GPUs sharing one problem, checked on one GPU through the C ABI:
the shards of pcl_candidates_shard partition the self-join exactly as
shard.pair_shard states (disjoint, union = pcl_candidates, gate counts summing
to its counts), and a server over a range view of the library returns the
whole-library server's pass pairs of that range."""
import time

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


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    return pcl.Context(0)


def _pairset(t):
    a = t.cpu().numpy().astype(np.int64) if hasattr(t, "cpu") else np.asarray(t, np.int64)
    return set(map(tuple, a.reshape(-1, 2).tolist()))


@pytest.mark.parametrize("n", [2, 33, 300, 1000])
def test_candidate_shards_partition_the_self_join(ctx, torch_cuda, n):
    import paper_2512_13133_gb300 as pcl
    from paper_2512_13133_gb300 import shard
    wl = synth.preset("small", seed=5, n_clips=n, n_seeds=max(1, n // 10), n_copies=int(0.6 * n))
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80, edge_tol_dbu=12)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    for mode in (pcl.MODE_COSINE, pcl.MODE_EDGE):
        full, gfull = pcl.candidates(ctx, P, mode, cs)
        full = _pairset(full)
        assert int(gfull[:6].sum()) == n * (n - 1) // 2
        for S in (2, 3, 5):
            seen, gsum = set(), np.zeros(16, np.int64)
            for s in range(S):
                part, g = pcl.candidates(ctx, P, mode, cs, shard=s, n_shards=S)
                arr = part.cpu().numpy().astype(np.int64)
                if len(arr):
                    assert (shard.pair_shard(arr, n, mode, S) == s).all()
                mine = _pairset(arr)
                assert len(mine) == len(arr) and not (mine & seen)
                seen |= mine
                gsum += g
            assert seen == full, (mode, S)
            np.testing.assert_array_equal(gsum, gfull)
    with pytest.raises(pcl.PclError):
        pcl.candidates(ctx, P, pcl.MODE_EDGE, cs, shard=3, n_shards=3)


def _wait(srv, rid, timeout=60.0):
    t0 = time.time()
    while True:
        for c in srv.poll():
            if c["id"] == rid:
                return c
        assert time.time() - t0 < timeout
        time.sleep(0.001)


@pytest.mark.parametrize("mode", ["cosine", "edge"])
def test_server_over_a_library_range(ctx, torch_cuda, mode):
    import paper_2512_13133_gb300 as pcl
    from paper_2512_13133_gb300 import shard
    lib = synth.preset("small", seed=6, n_clips=900, n_seeds=90, n_copies=540)
    cosine = mode == "cosine"
    P = pcl.params(lib.window_dbu, lib.pitch_dbu, lib.marker_dbu, cos_num=80, edge_tol_dbu=12)
    m = pcl.MODE_COSINE if cosine else pcl.MODE_EDGE
    cs = pcl.alloc_clipset(P, lib.rect_off, lib.rects)
    pcl.pcl_rasterize(ctx, P, cs)
    qsrc = lib.subset(np.arange(0, lib.n, 5))
    kw = dict(max_inflight=2, max_query_clips=256, cand_per_query=1024, mem_budget=1 << 29, mode=m)
    whole = pcl.Server(ctx, P, cs, **kw)
    assert whole.submit(qsrc.rect_off, qsrc.rects, 1)
    ref = _pairset(_wait(whole, 1)["pass_pairs"])
    whole.close()
    assert len(ref) >= qsrc.n
    merged = set()
    for lo, hi in shard.library_ranges(lib.n, 3):
        view = cs.view(P, lo, hi)
        srv = pcl.Server(ctx, P, view, **kw)
        assert srv.submit(qsrc.rect_off, qsrc.rects, 2)
        got = _wait(srv, 2)
        assert got["status"] == 0
        part = {(a, b + lo) for a, b in _pairset(got["pass_pairs"])}
        assert part == {p for p in ref if lo <= p[1] < hi}
        merged |= part
        srv.close()
    assert merged == ref
