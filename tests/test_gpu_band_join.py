"""The cosine band join at 256² and 512² rasters (at 256² each lane of a warp
sums the first chunk of the G3 density bound for its own band member, member
block words staged in shared memory by 16-byte copies), against the oracle's
exhaustive screen: candidate sets and gate counts exact, at two thresholds
(T = 0.80 gives bands of hundreds of members, so full and partial groups of 32
members and many G3 survivors).  A clip set whose block array is not 16-byte
aligned takes the warp-per-member path and must give the same result."""
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


def _workload(n, window_dbu):
    base = synth.generate(21, n_clips=n, n_seeds=max(1, n // 8), n_copies=n // 2, window_dbu=window_dbu,
                          margin_dbu=window_dbu // 16, min_rects=4, max_rects=30)
    clips = [base.clip(i).tolist() for i in range(n)]
    for k in (0, n // 3):
        clips[k] = []
    clips[n - 1] = list(clips[n - 2])
    return synth.from_lists(clips, base.window_dbu, base.pitch_dbu, base.marker_dbu)


def _misaligned_blk(torch, cs):
    """The same clip set with its block array moved to an address 4 bytes past
    a 16-byte boundary (same contents)."""
    import dataclasses
    nbytes = cs.blk.numel()
    raw = torch.empty(nbytes + 32, dtype=torch.uint8, device=cs.blk.device)
    off = (-raw.data_ptr()) % 16 + 4
    view = raw[off:off + nbytes]
    view.copy_(cs.blk)
    assert view.data_ptr() % 16 == 4
    return dataclasses.replace(cs, blk=view)


@pytest.mark.parametrize("window_dbu,n", [(1024, 420), (2048, 260)])
@pytest.mark.parametrize("cos_num", [80, 95])
def test_band_join_matches_oracle(ctx, torch_cuda, window_dbu, n, cos_num):
    import paper_2512_13133_gb300 as pcl
    wl = _workload(n, window_dbu)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=cos_num)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    assert cs.blk.data_ptr() % 16 == 0
    op, ocounts = oracle.ClipSet(wl).candidates(pcl.MODE_COSINE, cos_num=cos_num)
    want = set(map(tuple, op.astype(np.int64).tolist()))
    # the G3 bound decides a good share of the band pairs and keeps some
    assert ocounts[pcl.GATE_G3_DENSITY] > 1000
    for c in (cs, _misaligned_blk(torch_cuda, cs)):
        gp, gcounts = pcl.candidates(ctx, P, pcl.MODE_COSINE, c)
        got = set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist()))
        assert got == want
        np.testing.assert_array_equal(gcounts[:6], ocounts[:6].astype(np.int64))
        assert gcounts[:6].sum() == n * (n - 1) // 2


@pytest.mark.parametrize("window_dbu", [1024, 2048])
@pytest.mark.parametrize("n_shards", [1, 3])
def test_band_join_shards(ctx, torch_cuda, window_dbu, n_shards):
    """Shards of the band join (members b > a of representatives a = s + k S,
    compacted to the low lanes before the lane-per-member chunk at 256²) add
    up to the self-join, with the oracle's gate counts."""
    import paper_2512_13133_gb300 as pcl
    wl = _workload(200, window_dbu)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    op, ocounts = oracle.ClipSet(wl).candidates(pcl.MODE_COSINE, cos_num=80)
    torch = torch_cuda
    got, counts = set(), np.zeros(16, np.int64)
    for s in range(n_shards):
        out = torch.empty((200 * 200, 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        gates = torch.zeros(16, dtype=torch.int64, device="cuda")
        pcl.pcl_candidates_shard(ctx, P, pcl.MODE_COSINE, cs, s, n_shards, out, cnt, gates)
        k = int(cnt.item())
        part = set(map(tuple, out[:k].cpu().numpy().astype(np.int64).tolist()))
        assert not (part & got)
        got |= part
        counts += gates.cpu().numpy()
    assert got == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(counts[:6], ocounts[:6].astype(np.int64))


@pytest.mark.parametrize("window_dbu,na,nb", [(1024, 60, 1500), (2048, 40, 400)])
def test_cross_join_matches_oracle(ctx, torch_cuda, window_dbu, na, nb):
    """Query x library candidates (the cross join of the serving loop, also
    lane-per-member in its first chunk) at 256² and 512², with the library's
    block array aligned and not: the oracle's exhaustive two-set screen."""
    import paper_2512_13133_gb300 as pcl
    wl = _workload(na + nb, window_dbu)
    wa, wb = wl.subset(np.arange(0, na)), wl.subset(np.arange(na, na + nb))
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=80)
    ca = pcl.alloc_clipset(P, wa.rect_off, wa.rects, with_spec=False)
    cb = pcl.alloc_clipset(P, wb.rect_off, wb.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, ca)
    pcl.pcl_rasterize(ctx, P, cb)
    op, oc = oracle.ClipSet(synth.concat(wa, wb)).candidates_ab(na, pcl.MODE_COSINE, cos_num=80)
    assert oc[pcl.GATE_G3_DENSITY] > 1000
    want = set(map(tuple, op.astype(np.int64).tolist()))
    for lib in (cb, _misaligned_blk(torch_cuda, cb)):
        gp, gc = pcl.candidates(ctx, P, pcl.MODE_COSINE, ca, b=lib)
        assert set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist())) == want
        np.testing.assert_array_equal(gc[:6], oc[:6].astype(np.int64))
