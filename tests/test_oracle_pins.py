"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests retypes the oracle's formula: each compares it with a
worked example of the paper, a closed form, an invariant, a brute force over
a tiny case, or a library routine.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden_raster():
    rects, rows, in_img = [], [], False
    with open(os.path.join(GOLDEN, "raster_8x8.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line == "image":
                in_img = True
            elif in_img:
                rows.append([int(c) for c in line])
            else:
                rects.append([int(v) for v in line.split()[1:]])
    return rects, np.array(rows, dtype=np.uint8)


def test_raster_golden_8x8():
    rects, expect = _read_golden_raster()
    img = oracle.rasterize(32, 4, rects)
    assert img.shape == (8, 8)
    np.testing.assert_array_equal(img, expect)


def _centres_in(lo, hi, p, N):
    # closed form: number of i in [0, N) with lo <= p*i + p/2 < hi
    first = -((-(2 * lo - p)) // (2 * p))          # ceil((2lo - p) / 2p)
    last = -((-(2 * hi - p)) // (2 * p))           # ceil((2hi - p) / 2p)
    return max(0, min(last, N) - max(first, 0))


@pytest.mark.parametrize("p", [4, 3, 8])
def test_raster_single_rect_closed_form(p):
    rng = np.random.default_rng(7 + p)
    W = 64 * p
    N = W // p
    for _ in range(200):
        x0, x1 = sorted(rng.integers(0, W + 1, size=2))
        y0, y1 = sorted(rng.integers(0, W + 1, size=2))
        if x0 == x1 or y0 == y1:
            continue
        img = oracle.rasterize(W, p, [[x0, y0, x1, y1]])
        assert int(img.sum()) == _centres_in(x0, x1, p, N) * _centres_in(y0, y1, p, N)


def test_raster_union_of_overlaps():
    # overlapping rectangles union (0/1 image), never sum
    img = oracle.rasterize(64, 4, [[0, 0, 40, 40], [20, 20, 64, 64]])
    assert img.max() == 1
    a = oracle.rasterize(64, 4, [[0, 0, 40, 40]])
    b = oracle.rasterize(64, 4, [[20, 20, 64, 64]])
    np.testing.assert_array_equal(img, np.maximum(a, b))


@pytest.mark.parametrize("N", [64, 128, 96])
def test_corr_words_equals_pixel_loop(N):
    rng = np.random.default_rng(N)
    for t in range(6):
        A = (rng.random((N, N)) < 0.3).astype(np.uint8)
        B = (rng.random((N, N)) < 0.4).astype(np.uint8)
        for dx, dy in [(0, 0), (1, 0), (0, -1), (-7, 5), (13, -9), (63, 2), (-64, 1), (65, -3)]:
            assert oracle.corr_words(A, B, dx, dy) == oracle.corr_pixel(A, B, dx, dy)


def test_corr_matches_numpy_correlation():
    # c(s) = sum_x A(x) B(x - s): compare with an explicit numpy shift + sum
    rng = np.random.default_rng(3)
    N = 64
    A = (rng.random((N, N)) < 0.5).astype(np.uint8)
    B = (rng.random((N, N)) < 0.5).astype(np.uint8)
    for dx, dy in [(3, -2), (-5, 4), (0, 7)]:
        Bs = np.zeros_like(B)
        # Bs(x) = B(x - s): move B by +s
        ys, xs = np.nonzero(B)
        ys2, xs2 = ys + dy, xs + dx
        ok = (ys2 >= 0) & (ys2 < N) & (xs2 >= 0) & (xs2 < N)
        Bs[ys2[ok], xs2[ok]] = 1
        assert oracle.corr_pixel(A, B, dx, dy) == int((A.astype(int) * Bs).sum())


def test_self_similarity_is_one_at_zero(small_set):
    for c in range(0, 60, 7):
        r = small_set.pair(c, c)
        assert r["dx_dbu"] == 0 and r["dy_dbu"] == 0
        assert r["score"] == small_set.pop(c)
        assert abs(r["sim"] - 1.0) < 1e-15
        assert r["pass_"] == 1


def test_swap_symmetry_cosine(small_set):
    rng = np.random.default_rng(11)
    S = small_set.S
    for _ in range(80):
        a, b = (int(v) for v in rng.integers(0, small_set.n, size=2))
        if a == b:
            continue
        r1 = small_set.pair(a, b, use_gates=False)
        r2 = small_set.pair(b, a, use_gates=False)
        assert r1["score"] == r2["score"]
        assert abs(r1["sim"] - r2["sim"]) < 1e-12
        assert r1["pass_"] == r2["pass_"]
        if (r1["dx_dbu"], r1["dy_dbu"]) != (-r2["dx_dbu"], -r2["dy_dbu"]):
            # tied maximum: the negated shift must still be a maximiser
            cw = small_set.corr_window(b, a)
            dx, dy = -r1["dx_dbu"] // small_set.p, -r1["dy_dbu"] // small_set.p
            assert cw[dy + S, dx + S] == r2["score"]


def _translate(rects, tx, ty):
    return [[r[0] + tx, r[1] + ty, r[2] + tx, r[3] + ty] for r in rects]


def test_pure_translate_gives_negated_shift_and_sim_one():
    base = [[100, 120, 160, 180], [220, 300, 300, 330], [330, 90, 380, 250]]
    for tx, ty in [(8, -12), (-32, 32), (4, 0), (0, -28)]:
        wl = synth.from_lists([base, _translate(base, tx, ty)], 512, 4, 32)
        cs = oracle.ClipSet(wl)
        r = cs.pair(0, 1, use_gates=False)
        assert (r["dx_dbu"], r["dy_dbu"]) == (-tx, -ty)
        assert abs(r["sim"] - 1.0) < 1e-15 and r["pass_"] == 1


def test_translation_invariance_of_pair():
    rng = np.random.default_rng(5)
    a = [[100, 100, 180, 150], [250, 260, 300, 400], [120, 300, 200, 340]]
    b = [[106, 96, 190, 150], [250, 268, 296, 400], [128, 304, 200, 344]]
    wl = synth.from_lists([a, b], 512, 4, 32)
    ref = oracle.ClipSet(wl).pair(0, 1, use_gates=False)
    for _ in range(4):
        tx, ty = (int(4 * v) for v in rng.integers(-20, 21, size=2))
        wl2 = synth.from_lists([_translate(a, tx, ty), _translate(b, tx, ty)], 512, 4, 32)
        r = oracle.ClipSet(wl2).pair(0, 1, use_gates=False)
        assert r["score"] == ref["score"] and abs(r["sim"] - ref["sim"]) < 1e-15
        assert (r["dx_dbu"], r["dy_dbu"]) == (ref["dx_dbu"], ref["dy_dbu"])


def test_tie_order_of_shifts():
    # A: one pixel at x index 5; B: pixels at x indices 4 and 6 (same row).
    # c(s) = B(5 - dx): maxima at dx = +1 and dx = -1 (both |s| = 1, dy = 0);
    # the tie order (-c, |dx|+|dy|, dy, dx) picks dx = -1.
    a = [[20, 20, 24, 24]]
    b = [[16, 20, 20, 24], [24, 20, 28, 24]]
    wl = synth.from_lists([a, b], 64, 4, 8)
    r = oracle.ClipSet(wl).pair(0, 1, use_gates=False)
    assert (r["dx_dbu"], r["dy_dbu"], r["score"]) == (-4, 0, 1)


def test_tie_order_dy_then_length():
    # vertical tie: B has pixels above and below A's pixel -> dy = -1 wins
    a = [[20, 20, 24, 24]]
    b = [[20, 16, 24, 20], [20, 24, 24, 28]]
    r = oracle.ClipSet(synth.from_lists([a, b], 64, 4, 8)).pair(0, 1, use_gates=False)
    assert (r["dx_dbu"], r["dy_dbu"]) == (0, -4)
    # |dx|+|dy| before dy: candidates (dx, dy) = (0, 1) and (-1, -1) -> (0, 1)
    b = [[20, 16, 24, 20], [24, 24, 28, 28]]
    r = oracle.ClipSet(synth.from_lists([a, b], 64, 4, 8)).pair(0, 1, use_gates=False)
    assert (r["dx_dbu"], r["dy_dbu"]) == (0, 4)


def _translate_workload(seed, k=24):
    """k random interior clips and, for each, a pure translate and a
    one-pixel-edge variant: pairs that pass and need a non-zero shift."""
    rng = np.random.default_rng(seed)
    clips = []
    for _ in range(k):
        rects = []
        while len(rects) < int(rng.integers(2, 6)):
            x0, y0 = (int(40 + 10 * v) for v in rng.integers(0, 38, size=2))
            w, h = (int(10 * v) for v in rng.integers(3, 9, size=2))
            r = [x0, y0, x0 + w, y0 + h]
            if all(r[2] + 20 <= q[0] or q[2] + 20 <= r[0] or r[3] + 20 <= q[1] or q[3] + 20 <= r[1]
                   for q in rects):
                rects.append(r)
        tx, ty = (int(4 * v) for v in rng.integers(-8, 9, size=2))
        var = [list(r) for r in rects]
        var[0][2] += 4
        clips += [rects, _translate(rects, tx, ty), _translate(var, -ty, tx)]
    return synth.from_lists(clips, 512, 4, 32)


def test_gates_keep_shifted_passing_pairs():
    cs = oracle.ClipSet(_translate_workload(31))
    n = cs.n
    allp = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.uint32)
    brute = cs.match(allp, oracle.MODE_COSINE, use_gates=False)
    passing = {(int(r["a"]), int(r["b"])) for r in brute if r["pass_"]}
    assert len(passing) >= 2 * 24
    kept, _ = cs.candidates(oracle.MODE_COSINE)
    assert passing <= set(map(tuple, kept.tolist()))
    for r in brute:
        b = cs.gate_bounds(int(r["a"]), int(r["b"]))
        assert (b >= r["score"]).all()


def test_pcm_delta_on_cyclic_shift():
    # Eqs. 3-5: g = f moved by (x0, y0) -> r = delta at the shift.  With the
    # member B = A moved by t, the surface built from C = F_A conj(F_B)
    # peaks at -t (the shift that re-aligns B).
    rng = np.random.default_rng(2)
    L = 48
    A = (rng.random((L, L)) < 0.4).astype(np.uint8)
    for tx, ty in [(5, -3), (-11, 7), (0, 0)]:
        B = np.roll(np.roll(A, ty, axis=0), tx, axis=1)
        r = oracle.pcm_surface(A, B, L)
        iy, ix = np.unravel_index(np.argmax(r), r.shape)
        assert (iy, ix) == ((-ty) % L, (-tx) % L)
        assert abs(r[iy, ix] - 1.0) < 1e-9
        r2 = r.copy()
        r2[iy, ix] = 0
        assert np.abs(r2).max() < 1e-9


def test_pcm_peak_on_padded_translate_matches_exact_argmax():
    base = [[100, 120, 160, 180], [220, 300, 300, 330], [330, 90, 380, 250]]
    wl = synth.from_lists([base, _translate(base, 12, -20)], 512, 4, 32)
    cs = oracle.ClipSet(wl)
    w = cs.pcm_window(0, 1)
    dx, dy = oracle.window_peak(w, cs.S)
    assert (dx * 4, dy * 4) == (-12, 20)


def test_decision_integer_rule_vs_float64():
    rng = np.random.default_rng(9)
    T = Fraction(95, 100)
    n_checked = 0
    for _ in range(20000):
        pa, pb = (int(v) for v in rng.integers(1, 65536, size=2))
        c = int(rng.integers(0, min(pa, pb) + 1))
        sim = c / np.sqrt(float(pa) * float(pb))
        if abs(sim - 0.95) < 1e-9:
            continue
        assert oracle.cos_exceeds(c, pa, pb, 95, 100) == (sim > float(T))
        n_checked += 1
    assert n_checked > 19000
    # exact tie: sim = 0.95 exactly is not "> T" (strict, Eq. 2)
    assert not oracle.cos_exceeds(95, 100, 100, 95, 100)
    assert oracle.cos_exceeds(96, 100, 100, 95, 100)
    assert not oracle.cos_exceeds(0, 0, 0, 95, 100)


def _golden_minmax():
    vals = {}
    with open(os.path.join(GOLDEN, "minmax_worked_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    return vals


def test_minmax_worked_example():
    g = _golden_minmax()
    d = [g["d_min"], 5, 7, g["d_max"]]
    T, E = oracle.minmax_closed(d, 64)
    assert (T, E) == (g["T_opt"], g["E_min"])
    e, lo, hi = oracle.minmax_scan(d, 64)
    assert e == g["E_min"] and lo == hi == g["T_opt"]


def test_minmax_closed_form_equals_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(500):
        n = int(rng.integers(1, 12))
        M = int(rng.integers(0, 40))
        d = rng.integers(-60, 61, size=n).astype(np.int32)
        T, E = oracle.minmax_closed(d, M)
        e, lo, hi = oracle.minmax_scan(d, M)
        assert E == e
        assert lo <= T <= hi
        assert T == -oracle.minmax_closed(-d, M)[0]   # odd symmetry of trunc


def test_minmax_linf_separable_2d():
    # L_inf separability (Sec. 3.2.2): the 2-D optimum of max_i ||d_i - T||_inf
    # equals the larger of the two 1-D optima.
    rng = np.random.default_rng(8)
    for _ in range(60):
        n = int(rng.integers(1, 6))
        dx = rng.integers(-15, 16, size=n)
        dy = rng.integers(-15, 16, size=n)
        M = 16
        best = min(max(max(abs(dx - tx)), max(abs(dy - ty)))
                   for tx in range(-M, M + 1) for ty in range(-M, M + 1))
        _, ex = oracle.minmax_closed(dx, M)
        _, ey = oracle.minmax_closed(dy, M)
        assert best == max(ex, ey)


def _edge_pair(a_rects, b_rects, tol, W=512, M=32):
    wl = synth.from_lists([a_rects, b_rects], W, 4, M)
    return oracle.ClipSet(wl).pair(0, 1, mode=oracle.MODE_EDGE, edge_tol_dbu=tol)


def test_edge_worked_example_pair():
    # member edges displaced so that d = e_A - e_B is 2 (left) and 10 (right):
    # interval [2, 10] -> T = 6, E = 4 (Sec. 3.2.2); passes at tol 4 only.
    a = [[100, 100, 200, 180]]
    b = [[98, 100, 190, 180]]
    r = _edge_pair(a, b, 4)
    assert (r["dx_dbu"], r["dy_dbu"], r["score"], r["pass_"]) == (6, 0, 4, 1)
    assert _edge_pair(a, b, 3)["pass_"] == 0


def test_edge_exactly_one_overlap_rule():
    # Sec. 2.2.2 condition 1: a polygon of the smaller pattern overlapping two
    # polygons of the other fails; overlapping exactly one passes.
    a = [[100, 100, 300, 140]]
    b_two = [[100, 100, 190, 140], [210, 100, 300, 140]]
    r = _edge_pair(a, b_two, 4)
    assert r["pass_"] == 0 and (r["flags"] & 15) == oracle.GATE_E1_MATCH
    b_one = [[102, 100, 300, 141], [400, 400, 450, 450]]
    r = _edge_pair(a, b_one, 4)
    assert r["pass_"] == 1


def test_edge_swap_symmetry(small_set):
    rng = np.random.default_rng(12)
    hits = 0
    for _ in range(400):
        a, b = (int(v) for v in rng.integers(0, small_set.n, size=2))
        if a == b:
            continue
        r1 = small_set.pair(a, b, mode=oracle.MODE_EDGE)
        r2 = small_set.pair(b, a, mode=oracle.MODE_EDGE)
        assert r1["pass_"] == r2["pass_"]
        assert (r1["flags"] & 15) == (r2["flags"] & 15)
        if r1["flags"] & oracle.F_ALIGNED:
            hits += 1
            assert (r1["dx_dbu"], r1["dy_dbu"]) == (-r2["dx_dbu"], -r2["dy_dbu"])
            assert r1["score"] == r2["score"]
    assert hits > 0


def test_edge_empty_cases():
    assert _edge_pair([], [], 4)["pass_"] == 1
    r = _edge_pair([], [[10, 10, 50, 50]], 4)
    assert r["pass_"] == 0 and (r["flags"] & 15) == oracle.GATE_E1_MATCH


def test_cosine_empty_cases():
    wl = synth.from_lists([[], [], [[10, 10, 50, 50]]], 512, 4, 32)
    cs = oracle.ClipSet(wl)
    r = cs.pair(0, 1)
    assert r["pass_"] == 1 and r["sim"] == 1.0 and r["flags"] & oracle.F_EMPTY
    r = cs.pair(0, 2)
    assert r["pass_"] == 0
    r = cs.pair(0, 2, use_gates=False)
    assert r["pass_"] == 0 and r["sim"] == 0.0


def _bbox(rects):
    r = np.asarray(rects)
    return int(r[:, 2].max() - r[:, 0].min()), int(r[:, 3].max() - r[:, 1].min())


def test_gates_are_lossless_across_edge_bounds():
    # Sec. 3.1 stage 1: a gate may only reject pairs that fail.  The set has
    # passing pairs in both modes, among them edge pairs whose bbox sizes
    # differ by exactly 2*tol (E2's bound) and passing pairs of unequal
    # polygon counts whose bbox widths differ far more (E2 not applicable).
    tol = 4
    wl = synth.gate_bounds_set(41, tol_dbu=tol)
    cs = oracle.ClipSet(wl)
    n = cs.n
    allp = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.uint32)
    passing = {}
    for mode in (oracle.MODE_COSINE, oracle.MODE_EDGE):
        kept, counts = cs.candidates(mode, edge_tol_dbu=tol)
        assert int(counts.sum()) == len(allp)
        brute = cs.match(allp, mode, use_gates=False, edge_tol_dbu=tol)
        passing[mode] = {(int(r["a"]), int(r["b"])) for r in brute if r["pass_"]}
        assert passing[mode] <= set(map(tuple, kept.tolist()))
    assert len(passing[oracle.MODE_COSINE]) >= 3 * 16
    assert len(passing[oracle.MODE_EDGE]) >= 5 * 16
    at_bound = unequal = 0
    for a, b in passing[oracle.MODE_EDGE]:
        ra, rb = wl.clip(a), wl.clip(b)
        (wa, ha), (wb, hb) = _bbox(ra), _bbox(rb)
        if len(ra) == len(rb) and max(abs(wa - wb), abs(ha - hb)) == 2 * tol:
            at_bound += 1
        if len(ra) != len(rb) and abs(wa - wb) > 2 * tol:
            unequal += 1
    assert at_bound >= 16 and unequal >= 16


def _all_pairs(n):
    iu = np.triu_indices(n, 1)
    return np.stack(iu, 1).astype(np.uint32)


@pytest.mark.slow
@pytest.mark.parametrize("cos_num,tol", [(95, 4), (80, 8)])
def test_gates_are_lossless_on_every_small_config_pair(small_set, cos_num, tol):
    # brute force over all 499,500 pairs of the 1,000-clip set: at the
    # configured thresholds (T = 0.95, tol = 4) and at relaxed ones where many
    # copies pass (T = 0.80, tol = 8: jitter of +/-8 dbu per edge then puts
    # bbox differences on both sides of E2's 2*tol = 16)
    allp = _all_pairs(small_set.n)
    for mode in (oracle.MODE_COSINE, oracle.MODE_EDGE):
        kept, counts = small_set.candidates(mode, cos_num=cos_num, edge_tol_dbu=tol)
        assert int(counts.sum()) == len(allp)
        brute = small_set.match(allp, mode, use_gates=False, cos_num=cos_num, edge_tol_dbu=tol)
        passing = {(int(r["a"]), int(r["b"])) for r in brute if r["pass_"]}
        if cos_num == 80:
            assert len(passing) >= 200
        assert passing <= set(map(tuple, kept.tolist()))


def test_gate_bounds_dominate_every_shift(small_set):
    # the profile and density bounds hold for every shift of the window, not
    # only the best one; G1's sqrt(min/max) bounds the similarity itself
    rng = np.random.default_rng(21)
    for _ in range(40):
        a, b = (int(v) for v in rng.integers(0, small_set.n, size=2))
        cw = small_set.corr_window(a, b)
        sa, sb = small_set.signature(a), small_set.signature(b)
        S = small_set.S
        N = small_set.N
        # independent restatement of the row-profile bound per dy
        for dy in range(-S, S + 1):
            ub = sum(min(sa["rows"][j], sb["rows"][j - dy]) for j in range(N) if 0 <= j - dy < N)
            assert cw[dy + S].max() <= ub
        for dx in range(-S, S + 1):
            ub = sum(min(sa["cols"][i], sb["cols"][i - dx]) for i in range(N) if 0 <= i - dx < N)
            assert cw[:, dx + S].max() <= ub
        pa, pb = small_set.pop(a), small_set.pop(b)
        assert cw.max() <= min(pa, pb)


def test_signature_consistency(small_set):
    for c in range(0, 50, 5):
        img = small_set.image(c)
        sg = small_set.signature(c)
        np.testing.assert_array_equal(sg["rows"], img.sum(axis=1))
        np.testing.assert_array_equal(sg["cols"], img.sum(axis=0))
        nb = img.shape[0] // 16
        np.testing.assert_array_equal(sg["blk"], img.reshape(nb, 16, nb, 16).sum(axis=(1, 3)))


# ---------------------------------------------------------------- set cover

def test_surprisal_scores_by_hand():
    # Graph: 0-{1,2,3}; {1,2,3} x {7,8,9}; 4-{5,6}.  Eqs. 7-9 in 2^32 fixed
    # point: f = 1 + deg; S = floor(2^32 / f).
    edges = [(0, 1), (0, 2), (0, 3), (4, 5), (4, 6)]
    edges += [(u, v) for u in (1, 2, 3) for v in (7, 8, 9)]
    unc = np.ones(10, bool)
    assert oracle.score_of(10, edges, unc, 4) == 1431655765 + 2 * 2147483648
    assert oracle.score_of(10, edges, unc, 1) == 858993459 + 4 * 1073741824
    order, rep = oracle.setcover_eager(10, edges)
    # surprisal prefers the rare pair {5, 6} (a count-based greedy would take 1)
    assert order == [4, 1, 2, 3]
    assert rep.tolist() == [1, 1, 2, 3, 4, 4, 4, 1, 1, 1]


def test_first_step_scores_by_hand():
    # the graph of test_surprisal_scores_by_hand, every node uncovered:
    # degrees 3,4,4,4,2,1,1,3,3,3; node 5: S_5 + S_4 = 2^31 + floor(2^32/3)
    edges = [(0, 1), (0, 2), (0, 3), (4, 5), (4, 6)]
    edges += [(u, v) for u in (1, 2, 3) for v in (7, 8, 9)]
    deg, w, sc = oracle.surprisal_scores(10, edges)
    assert deg.tolist() == [3, 4, 4, 4, 2, 1, 1, 3, 3, 3]
    assert w[0] == 1 << 30 and w[1] == 858993459 and w[5] == 1 << 31
    assert sc[5] == (1 << 31) + 1431655765
    assert sc[4] == 1431655765 + 2 * (1 << 31)
    unc = np.ones(10, bool)
    for j in range(10):
        assert sc[j] == oracle.score_of(10, edges, unc, j)


def test_setcover_path_graph():
    order, rep = oracle.setcover_eager(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    assert order == [1, 3]
    assert rep.tolist() == [1, 1, 1, 3, 3]


def test_cluster_loop_by_hand():
    """The loop's reading worked by hand on three small graphs (S = 2^32/f,
    f = 1 + degree in the relaxed graph of the round; ties to the lower index)."""
    # Path 0-1-2-3, all relaxed, 1-2 not strict.  S = 1/2, 1/3, 1/3, 1/2 (x 2^32):
    # gains 0.83, 1.17, 1.17, 0.83 -> rep 1 covers {0, 1, 2}; then 3 alone (gain
    # 1/2) -> rep 3.  Member 0 passes strict with 1; 2 fails with 1 and, as an
    # orphan, tries reps 1, 3 in order: strict with 3 -> 2 joins 3.  One round.
    rep, ncl, rounds = oracle.cluster_loop(4, [(0, 1), (1, 2), (2, 3)], np.array([True, False, True]),
                                           np.array([True, True, True]))
    assert (rep.tolist(), ncl, rounds) == ([1, 1, 3, 3], 2, 1)
    # Path 0-1-2, 1-2 not strict, 2 has no strict partner: rep 1 covers all,
    # 2 is an orphan no rep accepts, so it is re-injected and becomes its own
    # representative in round 2.
    rep, ncl, rounds = oracle.cluster_loop(3, [(0, 1), (1, 2)], np.array([True, False]), np.array([True, True]))
    assert (rep.tolist(), ncl, rounds) == ([1, 1, 2], 2, 2)
    # 0-1 and 2-3 strict, 1-2 relaxed only, 4 isolated: S = 1/2, 1/3, 1/3, 1/2, 1;
    # rep 1 first (1.17), then the isolated 4 (gain 1, rarer than 3's 1/2), then 3;
    # the orphan 2 joins 3 (reps tried in index order 1, 3, 4).
    rep, ncl, rounds = oracle.cluster_loop(5, [(0, 1), (2, 3), (1, 2)], np.array([True, True, False]),
                                           np.array([True, True, True]))
    assert (rep.tolist(), ncl, rounds) == ([1, 1, 3, 3, 4], 3, 1)


def test_cluster_loop_invariants(small_set):
    pairs, _ = small_set.candidates(oracle.MODE_EDGE, edge_tol_dbu=6)
    rec = small_set.match(pairs, oracle.MODE_EDGE, edge_tol_dbu=6)
    verified = (rec["flags"] & oracle.F_ALIGNED) > 0
    verified &= (rec["flags"] & oracle.F_EDGE_VERIFY_FAIL) == 0
    strict = verified & (rec["score"] <= 4)
    relaxed = verified & (rec["score"] <= 6)
    rep_of, ncl, rounds = oracle.cluster_loop(small_set.n, pairs, strict, relaxed)
    assert (rep_of >= 0).all()
    reps = set(np.unique(rep_of).tolist())
    assert len(reps) == ncl
    assert all(rep_of[r] == r for r in reps)
    ok = {(int(a), int(b)) for (a, b), s in zip(pairs.tolist(), strict) if s}
    for k, r in enumerate(rep_of.tolist()):
        if k != r:
            assert (min(k, r), max(k, r)) in ok
    assert rounds >= 1


# ---- XY-separation interval competition (Sec. 3.2.1 (2)) --------------------

def _xysep(a_rects, b_rects, W=512, M=32, **kw):
    wl = synth.from_lists([a_rects, b_rects], W, 4, M)
    cs = oracle.ClipSet(wl)
    return cs, cs.pair(0, 1, mode=oracle.MODE_COSINE_XYSEP, use_gates=False, **kw)


def test_xysep_worked_example_narrowest_interval_wins():
    # Worked by hand from the four steps.  Pre-alignment: A's non-border edge
    # bbox is x 100..332, y 100..400, B's x 108..344, y 100..404, so s0 =
    # (trunc(-20/2), trunc(-4/2)) = (-10, -2); at s0 each polygon of A meets
    # exactly its counterpart.  Displacements d = e_A - e_B:
    #   pair 1: x {100-108, 200-220} = {-8, -20} (Q 12), y {0, 0}   (Q 0)
    #   pair 2: x {300-312, 332-344} = {-12, -12} (Q 0), y {-4, -4} (Q 0)
    # x: pair 2 wins (Q 0 < 12), T_x = -12 -> -3 px (pair 1 would give -14 ->
    # -4 px); y: tie at Q 0, the first polygon (pair 1) wins, T_y = 0 (pair 2
    # would give -1 px).  Reported shift (-12, 0) dbu.
    a = [[100, 100, 200, 148], [300, 300, 332, 400]]
    b = [[108, 100, 220, 148], [312, 304, 344, 404]]
    cs, r = _xysep(a, b)
    assert (r["dx_dbu"], r["dy_dbu"]) == (-12, 0)
    A, B = cs.image(0), cs.image(1)
    assert r["score"] == oracle.corr_pixel(A, B, -3, 0)
    # the exact argmax is at least as good and here strictly better (it also
    # aligns pair 2 in y), so the interval shift loses overlap on this pair
    e = cs.pair(0, 1, use_gates=False)
    assert e["score"] >= r["score"]


def test_xysep_pure_translate_matches_exact_argmax():
    base = [[100, 120, 160, 180], [220, 300, 300, 330], [330, 90, 380, 250]]
    for tx, ty in [(8, -12), (-32, 32), (4, 0), (0, -28)]:
        cs, r = _xysep(base, _translate(base, tx, ty))
        assert (r["dx_dbu"], r["dy_dbu"]) == (-tx, -ty)
        assert r["score"] == cs.pop(0) and abs(r["sim"] - 1.0) < 1e-15 and r["pass_"] == 1


def test_xysep_swap_negates_shift_without_ties():
    # distinct qualities on both axes, so no tie rule is involved
    a = [[100, 100, 200, 148], [300, 300, 332, 400]]
    b = [[108, 102, 212, 148], [312, 304, 344, 404]]
    _, r1 = _xysep(a, b)
    _, r2 = _xysep(b, a)
    assert (r2["dx_dbu"], r2["dy_dbu"]) == (-r1["dx_dbu"], -r1["dy_dbu"])
    assert r1["score"] == r2["score"]


def test_xysep_shift_clamped_to_marker():
    # a translate of 100 dbu lies outside M = 32: the pre-alignment clamps, the
    # interval midpoint clamps, and the raster shift stays at -S
    base = [[100, 120, 160, 180], [220, 300, 300, 330]]
    _, r = _xysep(base, _translate(base, 100, 0))
    assert r["dx_dbu"] == -32


def test_xysep_never_beats_exact(small_wl):
    cs = oracle.ClipSet(small_wl)
    rng = np.random.default_rng(9)
    lab = small_wl.label
    idx = np.flatnonzero(lab >= 0)
    pairs = []
    for s in np.unique(lab[idx])[:40]:
        m = idx[lab[idx] == s]
        pairs += [(i, j) for i in m for j in m if i != j]
    pairs = np.array(pairs + [tuple(x) for x in rng.integers(0, small_wl.n, size=(300, 2))], dtype=np.int64)
    x = cs.match(pairs, oracle.MODE_COSINE_XYSEP, use_gates=False)
    e = cs.match(pairs, oracle.MODE_COSINE, use_gates=False)
    assert np.all(x["score"] <= e["score"])
    assert np.all(x["pass_"] <= e["pass_"])
    # where the interval shift lands on the exact optimum, the records agree
    hit = x["score"] == e["score"]
    assert hit.any()
    np.testing.assert_array_equal(x["pass_"][hit], e["pass_"][hit])


def test_xysep_dbu_shift_rounds_half_away_from_zero():
    # a translate by a non-multiple of the 4-dbu pitch: T = -t exactly, then
    # the raster shift T / 4 is rounded half away from zero:
    #   t = (6, -6):  T = (-6, 6)  -> (-1.5, 1.5)  -> (-2, 2) px = (-8, 8) dbu
    #   t = (5, -7):  T = (-5, 7)  -> (-1.25, 1.75) -> (-1, 2) px = (-4, 8) dbu
    base = [[100, 120, 160, 180], [220, 300, 300, 330], [330, 90, 380, 250]]
    for (tx, ty), want in [((6, -6), (-8, 8)), ((5, -7), (-4, 8))]:
        _, r = _xysep(base, _translate(base, tx, ty))
        assert (r["dx_dbu"], r["dy_dbu"]) == want


@pytest.mark.parametrize("mode", [oracle.MODE_COSINE, oracle.MODE_EDGE])
def test_two_set_screen_is_the_union_self_join_across_the_sets(small_wl, mode):
    # Sec. 2.3: every pair of patterns is a candidate before the screening;
    # the A x B screen must keep exactly the cross pairs the self-join of the
    # union keeps, with A's clips first
    a = small_wl.subset(np.arange(0, 150))
    b = small_wl.subset(np.arange(150, 420))
    cs = oracle.ClipSet(synth.concat(a, b))
    p, c = cs.candidates_ab(a.n, mode, cos_num=80)
    assert int(c.sum()) == a.n * b.n
    q, _ = cs.candidates(mode, cos_num=80)
    q = q.astype(np.int64)
    sel = (q[:, 0] < a.n) & (q[:, 1] >= a.n)
    assert set(map(tuple, p.astype(np.int64).tolist())) == set(map(tuple, (q[sel] - [0, a.n]).tolist()))


# ---------------------------------------------------------------- re-extraction (Sec. 2.1)

def test_halo_without_border_content_equals_window_cosine():
    # every rectangle at least M from the window border: the moved window
    # never meets halo content, n_B(s) = |B| at every shift, and the
    # re-extraction reading reduces to the fixed-window cosine of Eq. 2
    wl = synth.gate_bounds_set(43)
    cs = oracle.ClipSet(wl, halo=True)
    n = cs.n
    pairs = np.array([(i, j) for i in range(n) for j in range(n) if i != j], dtype=np.int64)[::7]
    h = cs.match(pairs, oracle.MODE_COSINE_HALO)
    w = cs.match(pairs, oracle.MODE_COSINE, use_gates=False)
    for f in ("dx_dbu", "dy_dbu", "score", "pass_"):
        np.testing.assert_array_equal(h[f], w[f])
    np.testing.assert_allclose(h["sim"], w["sim"], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(h["pad"], cs.pops()[pairs[:, 1]])
    assert h["pass_"].sum() >= 10


def test_halo_translate_across_the_border_gives_sim_one():
    # the layout around a clip moved by t: re-extracting the member's window
    # at s = -t/p recovers the representative's window exactly (sim 1), even
    # where geometry crosses the window border; the fixed-window reading does
    # not (content that left the window is lost)
    W, M = 512, 32
    a = [[-20, 40, 60, 100], [200, -24, 260, 30], [300, 300, 530, 340], [100, 480, 180, 540], [240, 200, 300, 260]]
    clips = [a]
    for tx, ty in [(12, -20), (-32, 8), (28, 28), (-4, 32)]:
        b = [[r[0] + tx, r[1] + ty, r[2] + tx, r[3] + ty] for r in a]
        b = [[max(r[0], -M), max(r[1], -M), min(r[2], W + M), min(r[3], W + M)] for r in b]
        clips.append(b)
    cs = oracle.ClipSet(synth.from_lists(clips, W, 4, M), halo=True)
    for k, (tx, ty) in enumerate([(12, -20), (-32, 8), (28, 28), (-4, 32)], start=1):
        r = cs.pair(0, k, oracle.MODE_COSINE_HALO)
        assert (r["dx_dbu"], r["dy_dbu"]) == (-tx, -ty)
        assert r["sim"] == 1.0 and r["pass_"] == 1
        assert r["score"] == cs.pop(0) == r["pad"]
        assert cs.pair(0, k, use_gates=False)["sim"] < 1.0


def test_halo_windows_equal_numpy_slices_and_exact_argmax():
    from fractions import Fraction
    wl = synth.generate(9, n_clips=24, n_seeds=4, n_copies=14, window_dbu=256, margin_dbu=16, min_rects=3,
                        max_rects=12, halo_dbu=16)
    cs = oracle.ClipSet(wl, halo=True)
    S, N, p, M = cs.S, cs.N, cs.p, cs.M
    rng = np.random.default_rng(4)
    for _ in range(40):
        a, b = (int(v) for v in rng.integers(0, wl.n, size=2))
        A = oracle.rasterize(wl.window_dbu, p, wl.clip(a))
        Hb = oracle.rasterize(wl.window_dbu + 2 * M, p, wl.clip(b) + M)
        c, nb = cs.halo_window(a, b)
        best = None
        pa = int(A.sum())
        for dy in range(-S, S + 1):
            for dx in range(-S, S + 1):
                win = Hb[S - dy:S - dy + N, S - dx:S - dx + N].astype(np.int64)
                assert c[dy + S, dx + S] == int((win * A).sum())
                assert nb[dy + S, dx + S] == int(win.sum())
                cc, nn = int(c[dy + S, dx + S]), int(nb[dy + S, dx + S])
                sim2 = Fraction(1) if pa == 0 and nn == 0 else (Fraction(0) if pa == 0 or nn == 0
                                                                 else Fraction(cc * cc, pa * nn))
                key = (-sim2, abs(dx) + abs(dy), dy, dx)
                if best is None or key < best[0]:
                    best = (key, dx, dy, cc, nn, sim2)
        r = cs.pair(a, b, oracle.MODE_COSINE_HALO)
        assert (r["dx_dbu"], r["dy_dbu"]) == (best[1] * p, best[2] * p)
        assert r["score"] == best[3] and r["pad"] == best[4]
        assert r["pass_"] == int(best[3] > 0 and best[5] > Fraction(95 * 95, 100 * 100)
                                 or (pa == 0 and best[4] == 0))


@pytest.mark.parametrize("mode", [oracle.MODE_COSINE, oracle.MODE_EDGE])
def test_topological_prescreen_keeps_the_same_class_pairs_of_the_lossless_screen(small_wl, mode):
    # the lossy pre-screen keeps exactly the lossless candidates whose clips
    # have the same polygon count (saturated at 63), and counts every pair of
    # different counts as its rejection (sum over classes of the pair counts)
    sub = small_wl.subset(np.arange(400))
    cs = oracle.ClipSet(sub)
    cnt = np.minimum(np.diff(sub.rect_off.astype(np.int64)), 63)
    full, fc = cs.candidates(mode, cos_num=80, edge_tol_dbu=8)
    topo, tc = cs.candidates(mode, cos_num=80, edge_tol_dbu=8, topo=True)
    keep = {(int(a), int(b)) for a, b in full.astype(np.int64) if cnt[a] == cnt[b]}
    assert set(map(tuple, topo.astype(np.int64).tolist())) == keep
    n = sub.n
    same = sum(int(k) * (int(k) - 1) // 2 for k in np.bincount(cnt))
    assert int(tc[oracle.GATE_T0_TOPO]) == n * (n - 1) // 2 - same
    assert int(tc.sum()) == n * (n - 1) // 2
    assert 0 < len(keep) < len(full)
