"""Cosine with re-extraction of the member's window (Sec. 2.1, Eq. 2 at every
shift; clips carry the layout over [-M, W + M)^2): GPU records against the
oracle's -- best shift, overlap c(s*), pixel count n_B(s*) of the moved
window, decision exact, |sim diff| <= 1e-5 -- on clips whose geometry crosses
the window border, for 64^2 to 512^2 px, with empty clips, translates that
need the halo to reach sim 1, and a pair count limited on the device."""
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


def _gpu(ctx, wl):
    import paper_2512_13133_gb300 as pcl
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P, cs)
    hb, nb = pcl.alloc_halo(P, cs)
    pcl.pcl_rasterize_halo(ctx, P, cs, hb, nb)
    return P, cs, hb, nb


def _match(ctx, torch, P, cs, hb, nb, pairs, d_n=None):
    import paper_2512_13133_gb300 as pcl
    tp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    out = torch.zeros((len(pairs), 40), dtype=torch.uint8, device="cuda")
    pcl.pcl_match_halo(ctx, P, cs, cs, hb, nb, tp, out, d_n=d_n)
    return pcl.records_to_numpy(out)


def _compare(g, o):
    for f in ("dx_dbu", "dy_dbu", "pass_"):
        np.testing.assert_array_equal(g[f].astype(np.int64), o[f].astype(np.int64), err_msg=f)
    np.testing.assert_array_equal(g["score"].astype(np.int64), o["score"])
    np.testing.assert_array_equal(g["reserved"].astype(np.int64), o["pad"].astype(np.int64))
    np.testing.assert_array_equal(g["flags"] & 0x30F, o["flags"] & 0x30F)
    assert np.abs(g["sim"].astype(np.float64) - o["sim"]).max(initial=0) <= 1e-5


def _pairs(wl, rng, k):
    lab = wl.label
    same = np.array([(i, j) for i in range(wl.n) for j in range(wl.n)
                     if i != j and lab[i] >= 0 and lab[i] == lab[j]], dtype=np.int64).reshape(-1, 2)
    if len(same) > k:
        same = same[rng.choice(len(same), k, replace=False)]
    rnd = rng.integers(0, wl.n, size=(k // 3, 2))
    return np.concatenate([same, rnd, [[0, 0], [1, 1]]]).astype(np.int64)


@pytest.mark.parametrize("N,k", [(64, 240), (128, 240), (256, 90), (512, 12)])
def test_halo_records_match_oracle(ctx, torch_cuda, N, k):
    W = 4 * N
    wl = synth.generate(30 + N, n_clips=120, n_seeds=12, n_copies=80, window_dbu=W, margin_dbu=W // 16,
                        min_rects=5, max_rects=40, halo_dbu=W // 16)
    # two empty clips at the end
    clips = [wl.clip(i).tolist() for i in range(wl.n)] + [[], []]
    wl = synth.Workload(wl.name, W, 4, W // 16, *_offsets(clips), np.r_[wl.label, -1, -1].astype(np.int32))
    P, cs, hb, nb = _gpu(ctx, wl)
    rng = np.random.default_rng(N)
    pairs = np.concatenate([_pairs(wl, rng, k), [[wl.n - 1, wl.n - 2], [wl.n - 1, 3], [3, wl.n - 1]]])
    g = _match(ctx, torch_cuda, P, cs, hb, nb, pairs)
    o = oracle.ClipSet(wl, halo=True).match(pairs, oracle.MODE_COSINE_HALO)
    _compare(g, o)
    assert int(o["pass_"].sum()) >= 3


def _offsets(clips):
    off = np.zeros(len(clips) + 1, dtype=np.uint32)
    off[1:] = np.cumsum([len(c) for c in clips])
    rects = np.array([r for c in clips for r in c], dtype=np.int32).reshape(-1, 4)
    return off, rects


def test_halo_translates_across_the_border(ctx, torch_cuda):
    """geometry crossing the window border, the member a translate of the
    representative's layout: re-extraction at s = -t/p gives sim 1"""
    W, M = 512, 32
    a = [[-20, 40, 60, 100], [200, -24, 260, 30], [300, 300, 530, 340], [100, 480, 180, 540], [240, 200, 300, 260]]
    clips = [a]
    shifts = [(12, -20), (-32, 8), (28, 28), (-4, 32), (0, 0)]
    for tx, ty in shifts:
        b = [[r[0] + tx, r[1] + ty, r[2] + tx, r[3] + ty] for r in a]
        clips.append([[max(r[0], -M), max(r[1], -M), min(r[2], W + M), min(r[3], W + M)] for r in b])
    wl = synth.from_lists(clips, W, 4, M)
    P, cs, hb, nb = _gpu(ctx, wl)
    pairs = np.array([(0, k) for k in range(1, len(clips))] + [(k, 0) for k in range(1, len(clips))])
    g = _match(ctx, torch_cuda, P, cs, hb, nb, pairs)
    o = oracle.ClipSet(wl, halo=True).match(pairs, oracle.MODE_COSINE_HALO)
    _compare(g, o)
    for k, (tx, ty) in enumerate(shifts):
        assert (g["dx_dbu"][k], g["dy_dbu"][k]) == (-tx, -ty)
        assert g["sim"][k] == 1.0 and g["pass_"][k] == 1


def test_halo_pair_count_on_the_device(ctx, torch_cuda):
    wl = synth.generate(77, n_clips=60, n_seeds=6, n_copies=40, window_dbu=512, margin_dbu=32, min_rects=3,
                        max_rects=12, halo_dbu=32)
    P, cs, hb, nb = _gpu(ctx, wl)
    pairs = np.random.default_rng(1).integers(0, wl.n, size=(50, 2))
    d_n = torch_cuda.tensor([31], dtype=torch_cuda.int64, device="cuda")
    g = _match(ctx, torch_cuda, P, cs, hb, nb, pairs, d_n=d_n)
    o = oracle.ClipSet(wl, halo=True).match(pairs[:31], oracle.MODE_COSINE_HALO)
    _compare(g[:31], o)
    assert (g[31:]["flags"] == 0).all() and (g[31:]["a"] == 0).all()  # not written


def test_halo_bounds_skip_groups_of_shifts(ctx, torch_cuda):
    """The pair kernel skips the groups of shifts whose similarity bound is
    below the best found: on same-seed pairs part of the window is counted,
    with an empty representative every group is (no bound applies), and the
    records stay the oracle's."""
    import paper_2512_13133_gb300 as pcl
    W = 1024
    wl = synth.generate(41, n_clips=80, n_seeds=8, n_copies=56, window_dbu=W, margin_dbu=64,
                        min_rects=5, max_rects=40, halo_dbu=64)
    clips = [wl.clip(i).tolist() for i in range(wl.n)] + [[]]
    wl = synth.Workload(wl.name, W, 4, 64, *_offsets(clips), np.r_[wl.label, -1].astype(np.int32))
    P, cs, hb, nb = _gpu(ctx, wl)
    S = 16
    groups = (2 * S + 1) * ((2 * S) // 8 + 1)
    lab = wl.label
    same = np.array([(i, j) for i in range(wl.n) for j in range(wl.n)
                     if i != j and lab[i] >= 0 and lab[i] == lab[j]], dtype=np.int64)[:60]
    pcl.pcl_stats_get(ctx, reset=True, kernel="halo")
    g = _match(ctx, torch_cuda, P, cs, hb, nb, same)
    ev, tot = pcl.pcl_stats_get(ctx, reset=True, kernel="halo")
    assert tot == len(same) * groups and 0 < ev < 0.6 * tot
    o = oracle.ClipSet(wl, halo=True).match(same, oracle.MODE_COSINE_HALO)
    _compare(g, o)
    empty = wl.n - 1
    g = _match(ctx, torch_cuda, P, cs, hb, nb, np.array([[empty, 3], [empty, 7]]))
    ev, tot = pcl.pcl_stats_get(ctx, reset=True, kernel="halo")
    assert ev == tot == 2 * groups
