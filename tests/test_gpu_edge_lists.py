"""The edge screen's correspondence list: pairs all of whose smaller-clip
polygons meet occupied cells go to a list whose correspondence a second
kernel checks; past the list's end (2^24 entries at most, one per 256 pairs
screened, at least 65,536) the screen checks them itself.  A set of nine in
ten exact copies of one pattern sends most pairs there, far more than the
list holds, so both paths run.  Candidates and gate counts must equal the
oracle's exhaustive screen, for the self-join and for two sets."""
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


def _one_pattern(n):
    """n clips: nine in ten exact copies of one pattern (every pair of copies
    passes all grid tests), the rest copies with edges jittered and other
    patterns"""
    base = synth.generate(31, n_clips=n, n_seeds=max(1, n // 50), n_copies=n // 2, window_dbu=1024,
                          margin_dbu=64, min_rects=6, max_rects=20, edge_jitter=3)
    one = base.clip(1).tolist()
    clips = [list(one) if k % 10 else base.clip(k).tolist() for k in range(n)]
    return synth.from_lists(clips, base.window_dbu, base.pitch_dbu, base.marker_dbu)


@pytest.mark.parametrize("n", [700, 1500])
def test_edge_lists_overflow_self_join(ctx, n):
    import paper_2512_13133_gb300 as pcl
    wl = _one_pattern(n)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=95, edge_tol_dbu=4)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    op, oc = oracle.ClipSet(wl).candidates(pcl.MODE_EDGE, cos_num=95, edge_tol_dbu=4)
    # most pairs pass every grid test: far more than the list's 65,536 entries
    assert len(op) > max(0.7 * (n * (n - 1) // 2), 2 * 65536)
    gp, gc = pcl.candidates(ctx, P, pcl.MODE_EDGE, cs)
    assert set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist())) == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gc[:7], oc[:7].astype(np.int64))


def test_edge_lists_overflow_two_sets(ctx):
    import paper_2512_13133_gb300 as pcl
    wl = _one_pattern(900)
    wa, wb = wl.subset(np.arange(0, 300)), wl.subset(np.arange(300, 900))
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, cos_num=95, edge_tol_dbu=4)
    ca = pcl.alloc_clipset(P, wa.rect_off, wa.rects, with_spec=False)
    cb = pcl.alloc_clipset(P, wb.rect_off, wb.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, ca)
    pcl.pcl_rasterize(ctx, P, cb)
    op, oc = oracle.ClipSet(synth.concat(wa, wb)).candidates_ab(300, pcl.MODE_EDGE, cos_num=95, edge_tol_dbu=4)
    assert len(op) > max(0.7 * 300 * 600, 2 * 65536)
    gp, gc = pcl.candidates(ctx, P, pcl.MODE_EDGE, ca, b=cb)
    assert set(map(tuple, gp.cpu().numpy().astype(np.int64).tolist())) == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gc[:7], oc[:7].astype(np.int64))
