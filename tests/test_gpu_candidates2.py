"""Two-set candidate generation (pcl_candidates with a member set b): every
pair of clip i of a and clip j of b goes through the gates of its mode (Sec.
3.1 stage 1; Sec. 2.3 makes every pair of patterns a candidate).  Candidate
sets and gate counts equal the oracle's exhaustive two-set screen exactly, at
sizes around the tiles of the screens (32 clips of a x 256 clips of b in edge
mode, library chunks of 1,024 area-order positions in cosine mode) with
empty clips in both sets, and on a 256^2 px sample of the scale workload."""
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


def _with_empties(wl, every):
    clips = [wl.clip(i).tolist() for i in range(wl.n)]
    for k in range(0, len(clips), every):
        clips[k] = []
    return synth.from_lists(clips, wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)


def _check(ctx, wa, wb, mode, cos_num=80):
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(wa.window_dbu, wa.pitch_dbu, wa.marker_dbu, cos_num=cos_num)
    ca = pcl.alloc_clipset(P, wa.rect_off, wa.rects, with_spec=False)
    cb = pcl.alloc_clipset(P, wb.rect_off, wb.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, ca)
    pcl.pcl_rasterize(ctx, P, cb)
    gp, gc = pcl.candidates(ctx, P, mode, ca, b=cb)
    op, oc = oracle.ClipSet(synth.concat(wa, wb)).candidates_ab(wa.n, mode, cos_num=cos_num)
    got = gp.cpu().numpy().astype(np.int64)
    assert len(got) == len(op)
    assert set(map(tuple, got.tolist())) == set(map(tuple, op.astype(np.int64).tolist()))
    np.testing.assert_array_equal(gc[:6], oc[:6].astype(np.int64))
    assert int(gc[:6].sum()) == wa.n * wb.n
    return len(op)


@pytest.mark.parametrize("na,nb", [(1, 1), (2, 3), (33, 300), (300, 257), (31, 1100)])
@pytest.mark.parametrize("mode", [1, 2])
def test_two_set_candidates_match_oracle(ctx, mode, na, nb):
    base = synth.preset("small", seed=7, n_clips=1600, n_seeds=160, n_copies=960)
    wa = _with_empties(base.subset(np.arange(0, na)), 13)
    wb = _with_empties(base.subset(np.arange(na, na + nb)), 17)
    _check(ctx, wa, wb, mode)


def test_two_set_candidates_on_scale_sample(ctx, torch_cuda):
    # 400 query clips against 12,000 library clips of the scale recipe (256^2
    # px, S = 16), at the configured T = 0.95 and a relaxed T = 0.80
    wl = synth.preset("scale", seed=3, n_clips=12_400, n_seeds=620, n_copies=8_680)
    rng = np.random.default_rng(3)
    q = np.sort(rng.choice(wl.n, 400, replace=False))
    lib = np.setdiff1d(np.arange(wl.n), q)
    wa, wb = wl.subset(q), wl.subset(lib)
    kept = 0
    for mode in (1, 2):
        for cos_num in (95, 80):
            kept += _check(ctx, wa, wb, mode, cos_num=cos_num)
    assert kept > 0


def test_two_set_candidates_empty_sets(ctx, torch_cuda):
    import paper_2512_13133_gb300 as pcl
    base = synth.preset("small", seed=7)
    wa = base.subset(np.arange(0, 40))
    wz = synth.from_lists([], base.window_dbu, base.pitch_dbu, base.marker_dbu)
    P = pcl.params(base.window_dbu, base.pitch_dbu, base.marker_dbu)
    ca = pcl.alloc_clipset(P, wa.rect_off, wa.rects, with_spec=False)
    cz = pcl.alloc_clipset(P, wz.rect_off, wz.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, ca)
    for mode in (1, 2):
        for x, y in ((ca, cz), (cz, ca)):
            gp, gc = pcl.candidates(ctx, P, mode, x, b=y)
            assert gp.shape[0] == 0 and int(gc.sum()) == 0
