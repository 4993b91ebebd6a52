"""CPU ORACLE -- test infrastructure, not product code.

A plain, slow, obviously-correct CPU statement of the method, written from the
paper (arXiv 2512.13133).  It backs the parity tests, the package smoke check
and the benchmark's CPU-baseline leg; nothing else may import it, and the
product path never calls it.  It shares no code with the CUDA library: only
the seeded rectangle generator (``synth``) serves both.

Pieces and the passages they follow:

* rasterisation, correlation, cosine decision, gates, brute-force shift scan,
  edge Min-Max procedure: ``pcl_oracle.c`` (Sec. 2.2.1 Eq. 2, Sec. 2.2.2,
  Sec. 3.2.1 Eqs. 3-5, Sec. 3.2.2 Eq. 6, Sec. 3.1 stage 1);
* cosine with re-extraction of the member's window at each shift (Sec. 2.1,
  Eq. 2; halo rasters over [-M, W + M)^2): ``pcl_oracle.c``;
* phase-correlation surface: numpy FFT in float64 (Sec. 3.2.1 Eqs. 3-5) --
  a library FFT used as one step, with no blocking or pruning;
* surprisal set cover, eager greedy (Sec. 3.3, Eqs. 7-9) and the
  coarse-to-fine loop (Sec. 3.1 stages 2-4): plain Python below.

Parity notes: the set-cover / loop cluster count beyond its invariants is
"parity unpinned" (no external value to compare with).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "pcl_oracle.c")

MODE_COSINE = 1
MODE_EDGE = 2
MODE_COSINE_XYSEP = 3  # cosine mode, shift by XY-separation interval competition (Sec. 3.2.1 (2))
MODE_COSINE_HALO = 4   # cosine mode, the member's window re-extracted at each shift (Sec. 2.1)

GATE_NONE = 0
GATE_G1_AREA = 1
GATE_G2_PROFILE = 2
GATE_G3_DENSITY = 3
GATE_E1_MATCH = 4
GATE_E2_BBOX = 5
GATE_T0_TOPO = 6  # lossy topological pre-screen (candidate screens only)

F_NEAR_BAND = 1 << 4
F_EDGE_VERIFY_FAIL = 1 << 7
F_EMPTY = 1 << 8
F_ALIGNED = 1 << 9

REC_DTYPE = np.dtype([
    ("a", "<u4"), ("b", "<u4"), ("dx_dbu", "<i4"), ("dy_dbu", "<i4"), ("sim", "<f8"),
    ("score", "<i8"), ("flags", "<u4"), ("pass_", "<i4"), ("mode", "<i4"), ("pad", "<i4")])
assert REC_DTYPE.itemsize == 48


class _Params(ctypes.Structure):
    _fields_ = [("pitch_dbu", ctypes.c_int32), ("window_dbu", ctypes.c_int32),
                ("marker_dbu", ctypes.c_int32), ("cos_num", ctypes.c_uint32),
                ("cos_den", ctypes.c_uint32), ("edge_tol_dbu", ctypes.c_int32),
                ("use_gates", ctypes.c_int32), ("use_topo", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, pthreads)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.orc_set_create.restype = P
    lib.orc_set_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
    lib.orc_set_add_halo.argtypes = [P]
    lib.orc_halo_window.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_halo_pair.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_set_create_ex.restype = P
    lib.orc_set_create_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int]
    lib.orc_set_free.argtypes = [P]
    lib.orc_set_N.argtypes = [P]
    lib.orc_set_pop.restype = ctypes.c_int64
    lib.orc_set_pop.argtypes = [P, ctypes.c_int]
    lib.orc_set_image.argtypes = [P, ctypes.c_int, P]
    lib.orc_set_sig.argtypes = [P, ctypes.c_int, P, P, P, P]
    lib.orc_rasterize.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P]
    lib.orc_corr_pixel.restype = ctypes.c_int64
    lib.orc_corr_pixel.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_corr_words_img.restype = ctypes.c_int64
    lib.orc_corr_words_img.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_corr_window.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
    lib.orc_cosine_pair.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_edge_pair.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_xysep_pair.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_minmax_scan.restype = ctypes.c_int
    lib.orc_minmax_scan.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_minmax_closed.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.orc_cos_exceeds.restype = ctypes.c_int
    lib.orc_cos_exceeds.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                    ctypes.c_uint32]
    lib.orc_gate_bounds.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
    lib.orc_match.argtypes = [P, P, ctypes.c_int, P, ctypes.c_size_t, P, ctypes.c_int]
    lib.orc_candidates.restype = ctypes.c_int64
    lib.orc_candidates.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_int]
    lib.orc_candidates_ab.restype = ctypes.c_int64
    lib.orc_candidates_ab.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_int]
    _lib = lib
    return lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def params(window_dbu: int, pitch_dbu: int = 4, marker_dbu: int = 32, cos_num: int = 95,
           cos_den: int = 100, edge_tol_dbu: int = 4, use_gates: bool = True, topo: bool = False) -> _Params:
    return _Params(pitch_dbu, window_dbu, marker_dbu, cos_num, cos_den, edge_tol_dbu,
                   int(bool(use_gates)), int(bool(topo)))


def rasterize(window_dbu: int, pitch_dbu: int, rects) -> np.ndarray:
    """0/1 image [N, N] indexed [y, x] (Sec. 2.2.1 step 1, pixel-centre reading)."""
    lib = _load()
    r = np.ascontiguousarray(np.asarray(rects, dtype=np.int32).reshape(-1, 4))
    N = window_dbu // pitch_dbu
    img = np.zeros((N, N), dtype=np.uint8)
    lib.orc_rasterize(window_dbu, pitch_dbu, r.ctypes.data, r.shape[0], img.ctypes.data)
    return img


def corr_pixel(A: np.ndarray, B: np.ndarray, dx: int, dy: int) -> int:
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    return int(lib.orc_corr_pixel(A.ctypes.data, B.ctypes.data, A.shape[0], dx, dy))


def corr_words(A: np.ndarray, B: np.ndarray, dx: int, dy: int) -> int:
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    return int(lib.orc_corr_words_img(A.ctypes.data, B.ctypes.data, A.shape[0], dx, dy))


def cos_exceeds(c: int, pa: int, pb: int, num: int, den: int) -> bool:
    """Eq. 2 threshold test with strict '>' in exact integers."""
    return bool(_load().orc_cos_exceeds(c, pa, pb, num, den))


def minmax_scan(d, M: int):
    lib = _load()
    d = np.ascontiguousarray(d, dtype=np.int32)
    lo, hi = ctypes.c_int(), ctypes.c_int()
    e = lib.orc_minmax_scan(d.ctypes.data, d.shape[0], M, ctypes.byref(lo), ctypes.byref(hi))
    return e, lo.value, hi.value


def minmax_closed(d, M: int):
    lib = _load()
    d = np.ascontiguousarray(d, dtype=np.int32)
    T, E = ctypes.c_int(), ctypes.c_int()
    lib.orc_minmax_closed(d.ctypes.data, d.shape[0], M, ctypes.byref(T), ctypes.byref(E))
    return T.value, E.value


def fft_size(N: int) -> int:
    """FFT side L = 9N/8 (a 2^a * 3^2 size with L >= N + N/8, so every shift
    |s| <= N/8 of the zero-padded linear correlation is alias-free)."""
    return 9 * N // 8


class ClipSet:
    """Rasters and gate signatures of a workload, held by the C oracle.

    raster=False keeps the rectangles only (no images, no signatures): such a
    set serves edge mode alone, whose procedure reads rectangles, and is
    cheap to build for large workloads.  halo=True also rasterises each
    clip over [-M, W + M)^2 (its halo raster, side N + 2S) for the
    re-extraction mode MODE_COSINE_HALO."""

    def __init__(self, wl, marker_dbu: int | None = None, raster: bool = True, halo: bool = False):
        self._lib = _load()
        self.W = int(wl.window_dbu)
        self.p = int(wl.pitch_dbu)
        self.M = int(wl.marker_dbu if marker_dbu is None else marker_dbu)
        self.N = self.W // self.p
        self.S = self.M // self.p
        self.n = wl.n
        self.rect_off = np.ascontiguousarray(wl.rect_off, dtype=np.uint32)
        self.rects = np.ascontiguousarray(wl.rects, dtype=np.int32)
        self.raster = bool(raster)
        h = self._lib.orc_set_create_ex(self.W, self.p, self.M, self.rect_off.ctypes.data,
                                        self.rects.ctypes.data, self.n, int(self.raster))
        if not h:
            raise ValueError("oracle rejected the clip-set parameters")
        self._h = ctypes.c_void_p(h)
        self.halo = bool(halo) and self.raster
        if self.halo:
            self._lib.orc_set_add_halo(self._h)

    def _need_halo(self):
        if not self.halo:
            raise ValueError("oracle clip set built without halo rasters")

    def halo_window(self, a: int, b: int):
        """(c(s), n_B(s)) of the re-extraction reading for every shift,
        indexed [dy + S, dx + S]"""
        self._need_halo()
        K = 2 * self.S + 1
        c = np.zeros((K, K), dtype=np.int64)
        nb = np.zeros((K, K), dtype=np.int64)
        self._lib.orc_halo_window(self._h, a, b, c.ctypes.data, nb.ctypes.data)
        return c, nb

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.orc_set_free(h)
            self._h = None

    def params(self, **kw) -> _Params:
        kw.setdefault("marker_dbu", self.M)
        return params(self.W, self.p, **kw)

    def _need_raster(self):
        if not self.raster:
            raise ValueError("geometry-only oracle clip set: edge mode only")

    def image(self, c: int) -> np.ndarray:
        self._need_raster()
        img = np.zeros((self.N, self.N), dtype=np.uint8)
        self._lib.orc_set_image(self._h, c, img.ctypes.data)
        return img

    def pop(self, c: int) -> int:
        self._need_raster()
        return int(self._lib.orc_set_pop(self._h, c))

    def pops(self) -> np.ndarray:
        return np.array([self.pop(i) for i in range(self.n)], dtype=np.int64)

    def signature(self, c: int):
        self._need_raster()
        nb = (self.N + 15) // 16
        rows = np.zeros(self.N, np.int32)
        cols = np.zeros(self.N, np.int32)
        blk = np.zeros(nb * nb, np.int32)
        dil = np.zeros(nb * nb, np.int32)
        self._lib.orc_set_sig(self._h, c, rows.ctypes.data, cols.ctypes.data, blk.ctypes.data,
                              dil.ctypes.data)
        return dict(rows=rows, cols=cols, blk=blk.reshape(nb, nb), dil=dil.reshape(nb, nb))

    def gate_bounds(self, a: int, b: int) -> np.ndarray:
        """upper bounds of c(s) over the window: [G1 area, G2 profile, G3 density]"""
        self._need_raster()
        out = np.zeros(3, dtype=np.int64)
        self._lib.orc_gate_bounds(self._h, a, b, out.ctypes.data)
        return out

    def corr_window(self, a: int, b: int) -> np.ndarray:
        """exact c(s) for |dx|,|dy| <= S, indexed [dy + S, dx + S]"""
        self._need_raster()
        K = 2 * self.S + 1
        out = np.zeros((K, K), dtype=np.int64)
        self._lib.orc_corr_window(self._h, a, b, out.ctypes.data)
        return out

    def pair(self, a: int, b: int, mode: int = MODE_COSINE, **kw) -> np.void:
        if mode != MODE_EDGE:
            self._need_raster()
        rec = np.zeros(1, dtype=REC_DTYPE)
        p = self.params(**kw)
        if mode == MODE_COSINE_HALO:
            self._need_halo()
        fn = {MODE_COSINE: self._lib.orc_cosine_pair, MODE_EDGE: self._lib.orc_edge_pair,
              MODE_COSINE_XYSEP: self._lib.orc_xysep_pair, MODE_COSINE_HALO: self._lib.orc_halo_pair}[mode]
        fn(self._h, a, b, ctypes.byref(p), rec.ctypes.data)
        return rec[0]

    def match(self, pairs, mode: int = MODE_COSINE, threads: int | None = None, **kw) -> np.ndarray:
        """one record per (a, b) pair, in order (brute-force shift scan)."""
        if mode != MODE_EDGE:
            self._need_raster()
        if mode == MODE_COSINE_HALO:
            self._need_halo()
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.uint32).reshape(-1, 2))
        out = np.zeros(pr.shape[0], dtype=REC_DTYPE)
        p = self.params(**kw)
        self._lib.orc_match(self._h, ctypes.byref(p), mode, pr.ctypes.data, pr.shape[0],
                            out.ctypes.data, threads or default_threads())
        return out

    def candidates(self, mode: int = MODE_COSINE, threads: int | None = None, **kw):
        """exhaustive self-join gate screen; returns (pairs[m, 2], gate_counts[16])"""
        if mode != MODE_EDGE:
            self._need_raster()
        p = self.params(**kw)
        counts = np.zeros(16, dtype=np.uint64)
        m = self._lib.orc_candidates(self._h, ctypes.byref(p), mode, None, 0, counts.ctypes.data,
                                     threads or default_threads())
        pairs = np.zeros((max(int(m), 1), 2), dtype=np.uint32)
        self._lib.orc_candidates(self._h, ctypes.byref(p), mode, pairs.ctypes.data, m,
                                 counts.ctypes.data, threads or default_threads())
        return pairs[:m], counts

    def candidates_ab(self, n_a: int, mode: int = MODE_COSINE, threads: int | None = None, **kw):
        """exhaustive two-set gate screen of a set holding the clips of A
        (0 .. n_a - 1) then those of B: every pair (i, n_a + j); returns
        (pairs[m, 2] as (i, j) with j relative to B, gate_counts[16])"""
        if mode != MODE_EDGE:
            self._need_raster()
        p = self.params(**kw)
        counts = np.zeros(16, dtype=np.uint64)
        m = self._lib.orc_candidates_ab(self._h, ctypes.byref(p), mode, n_a, None, 0, counts.ctypes.data,
                                        threads or default_threads())
        pairs = np.zeros((max(int(m), 1), 2), dtype=np.uint32)
        self._lib.orc_candidates_ab(self._h, ctypes.byref(p), mode, n_a, pairs.ctypes.data, m,
                                    counts.ctypes.data, threads or default_threads())
        return pairs[:m], counts

    # -- phase correlation (Sec. 3.2.1, Eqs. 3-5) ---------------------------
    def pcm_window(self, a: int, b: int, L: int | None = None, eps: float = 1e-6) -> np.ndarray:
        """r(s) = IFFT(R)(s), R = C / |C| with C = F_A conj(F_B), on an L x L
        zero-padded grid; bins with |C| <= eps * |A||B| (= eps * max |C|) are
        set to 0 (guard reading; the paper is silent on zero bins).  Indexed
        [dy + S, dx + S]; the peak is the shift applied to B."""
        return pcm_window(self.image(a), self.image(b), self.S, L or fft_size(self.N), eps)


def pcm_surface(A: np.ndarray, B: np.ndarray, L: int, eps: float = 1e-6) -> np.ndarray:
    """Full L x L phase-correlation surface r = IFFT(C/|C|), C = F_A conj(F_B)
    (Eqs. 4-5 with f = A the reference and g = B the member; with the member
    moved by t the peak sits at -t, i.e. at the shift that re-aligns it)."""
    fa = np.fft.fft2(A.astype(np.float64), s=(L, L))
    fb = np.fft.fft2(B.astype(np.float64), s=(L, L))
    C = fa * np.conj(fb)
    mag = np.abs(C)
    thr = eps * float(A.sum()) * float(B.sum())
    R = np.where(mag > thr, C / np.where(mag > 0, mag, 1.0), 0.0)
    return np.fft.ifft2(R).real


def pcm_window(A: np.ndarray, B: np.ndarray, S: int, L: int, eps: float = 1e-6) -> np.ndarray:
    assert A.shape[0] + S <= L
    r = pcm_surface(A, B, L, eps)
    idx = np.arange(-S, S + 1) % L
    return r[np.ix_(idx, idx)]


def window_peak(surface: np.ndarray, S: int):
    """argmax over the window with the tie order (-value, |dx|+|dy|, dy, dx)."""
    K = 2 * S + 1
    best = None
    for iy in range(K):
        for ix in range(K):
            dy, dx = iy - S, ix - S
            key = (-surface[iy, ix], abs(dx) + abs(dy), dy, dx)
            if best is None or key < best[0]:
                best = (key, dx, dy)
    return best[1], best[2]


# ---------------------------------------------------------------- set cover

def surprisal_weights(n: int, edges: np.ndarray) -> np.ndarray:
    """S_i = floor(2^32 / f_i), f_i = 1 + |neighbours(i)| (Eqs. 7-8).  Reading:
    the reciprocal is held in 32-bit fixed point so that score sums are exact
    integers."""
    deg = np.zeros(n, dtype=np.int64)
    if len(edges):
        e = np.asarray(edges, dtype=np.int64)
        np.add.at(deg, e[:, 0], 1)
        np.add.at(deg, e[:, 1], 1)
    return (np.int64(1) << 32) // (1 + deg)


def setcover_eager(n: int, edges) -> tuple[list[int], np.ndarray]:
    """Surprisal greedy set cover of Sec. 3.3 evaluated eagerly (every score
    recomputed at every step -- the "standard greedy" of Table 2).

    Universe: all n clips; the set of candidate j is {j} U N(j).  Reading:
    only uncovered clips are candidate representatives (a representative must
    belong to its own cluster), so S_j of Eq. 9 is always counted.  Ties:
    higher score, then lower index.  Each clip joins the earliest-selected
    representative that covers it.  Returns (selection order, rep_of)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    nbrs = [[] for _ in range(n)]
    for i, j in e:
        nbrs[int(i)].append(int(j))
        nbrs[int(j)].append(int(i))
    w = surprisal_weights(n, e)
    unc = np.ones(n, dtype=bool)
    rep_of = np.full(n, -1, dtype=np.int64)
    order: list[int] = []
    while unc.any():
        best, best_j = -1, -1
        for j in range(n):
            if not unc[j]:
                continue
            sc = int(w[j]) + sum(int(w[k]) for k in nbrs[j] if unc[k])
            if sc > best:
                best, best_j = sc, j
        j = best_j
        order.append(j)
        for k in [j] + nbrs[j]:
            if unc[k]:
                unc[k] = False
                rep_of[k] = j
    return order, rep_of


def surprisal_scores(n: int, edges):
    """Degrees, surprisal weights and first-step scores of Sec. 3.3.1 with
    every node uncovered: deg(i) = number of edges at i, S_i =
    floor(2^32 / (1 + deg(i))) (Eqs. 7-8), Score_j = S_j + sum of S_k over
    the neighbours k of j (Eq. 9).  Plain loops over the edge list (each
    listed edge counts once per endpoint).  Returns (deg, S, Score) as int64
    arrays."""
    deg = np.zeros(n, dtype=np.int64)
    for a, b in np.asarray(edges, dtype=np.int64).reshape(-1, 2).tolist():
        deg[a] += 1
        deg[b] += 1
    w = np.array([(1 << 32) // (1 + int(d)) for d in deg], dtype=np.int64)
    score = w.copy()
    for a, b in np.asarray(edges, dtype=np.int64).reshape(-1, 2).tolist():
        score[a] += w[b]
        score[b] += w[a]
    return deg, w, score


def score_of(n: int, edges, uncovered: np.ndarray, j: int) -> int:
    """Score_j of Eq. 9 for a given uncovered set (j assumed uncovered)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = surprisal_weights(n, e)
    nb = set(e[e[:, 0] == j, 1].tolist()) | set(e[e[:, 1] == j, 0].tolist())
    return int(w[j]) + sum(int(w[k]) for k in nb if uncovered[k])


def cluster_loop(n: int, cand_pairs, strict: np.ndarray, relaxed: np.ndarray, max_rounds: int = 1000):
    """Coarse-to-fine closed loop of Sec. 3.1 (stages 2-4).

    Reading (the paper fixes neither the relaxation nor the re-injection):
    round r works on the remaining set R.  The graph holds the candidate pairs
    inside R whose relaxed decision passes; the set cover picks
    representatives and tentative members; a member is accepted iff its
    strict decision against its representative passes.  Rejected members
    (orphans) try the representatives finalised so far in index order under
    the strict decision; the rest form the next R.  Every round finalises at
    least one representative, so the loop ends.

    cand_pairs[m, 2] with strict[m] / relaxed[m] booleans.  Returns
    (rep_of, n_clusters, rounds)."""
    pairs = np.asarray(cand_pairs, dtype=np.int64).reshape(-1, 2)
    key = {}
    for (a, b), s in zip(pairs.tolist(), np.asarray(strict, bool).tolist()):
        key[(min(a, b), max(a, b))] = s

    def strict_ok(a, b):
        return key.get((min(a, b), max(a, b)), False)

    rep_of = np.full(n, -1, dtype=np.int64)
    reps: list[int] = []
    remaining = np.arange(n)
    relaxed = np.asarray(relaxed, bool)
    rounds = 0
    while len(remaining) and rounds < max_rounds:
        rounds += 1
        inR = np.zeros(n, bool)
        inR[remaining] = True
        sel = relaxed & inR[pairs[:, 0]] & inR[pairs[:, 1]] if len(pairs) else np.zeros(0, bool)
        sub = pairs[sel]
        loc = -np.ones(n, dtype=np.int64)
        loc[remaining] = np.arange(len(remaining))
        order, rep_local = setcover_eager(len(remaining), loc[sub] if len(sub) else sub)
        orphans = []
        for j in order:
            g = int(remaining[j])
            reps.append(g)
            rep_of[g] = g
        for k_loc, r_loc in enumerate(rep_local.tolist()):
            k, r = int(remaining[k_loc]), int(remaining[r_loc])
            if k == r:
                continue
            if strict_ok(r, k):
                rep_of[k] = r
            else:
                orphans.append(k)
        nxt = []
        rs = sorted(reps)
        for k in sorted(orphans):
            for r in rs:
                if strict_ok(r, k):
                    rep_of[k] = r
                    break
            else:
                nxt.append(k)
        remaining = np.array(nxt, dtype=np.int64)
    return rep_of, len(reps), rounds
