"""Seeded synthetic Manhattan clip workloads, shared by the oracle and the CUDA path.

This module holds no similarity arithmetic: it only asks ``pcl_synth.c`` to
place rectangles and returns them as numpy arrays.  Workload presets follow the
clip counts, window sizes, rectangle counts and perturbations of the
benchmark configurations (the contest data of the paper, Sec. 4, is not
available, so these synthetic sets stand in for it):

* ``small``  - 1,000 clips, W = 512 dbu (128^2 px at 4 dbu/px), 3-12 rects,
  100 seeds, 600 perturbed copies (edges +/-8 dbu, clip +/-32 dbu), marker
  half-width 32 dbu.
* ``scale``  - 100,000 clips, W = 1024 dbu (256^2 px), 5-40 rects, 5,000 seeds,
  70,000 perturbed copies (edges +/-8 dbu, clip +/-64 dbu), marker half-width
  64 dbu.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libpclsynth.so")
_SRC = os.path.join(_HERE, "pcl_synth.c")


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_clips", ctypes.c_uint32),
        ("n_seeds", ctypes.c_uint32),
        ("n_copies", ctypes.c_uint32),
        ("window_dbu", ctypes.c_int32),
        ("margin_dbu", ctypes.c_int32),
        ("min_rects", ctypes.c_int32),
        ("max_rects", ctypes.c_int32),
        ("min_side", ctypes.c_int32),
        ("max_side", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("spacing", ctypes.c_int32),
        ("edge_jitter", ctypes.c_int32),
        ("shift_max", ctypes.c_int32),
        ("halo_dbu", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the generator with gcc (host code only, portable C)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.pcl_synth_generate.restype = ctypes.c_int64
        lib.pcl_synth_generate.argtypes = [
            ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Workload:
    """Clips as rectangle lists plus the parameters they were drawn for."""
    name: str
    window_dbu: int
    pitch_dbu: int
    marker_dbu: int
    rect_off: np.ndarray          # uint32 [n+1]
    rects: np.ndarray             # int32 [R, 4] x0, y0, x1, y1
    label: np.ndarray             # int32 [n] seed index or -1
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.rect_off.shape[0] - 1)

    @property
    def raster_n(self) -> int:
        return self.window_dbu // self.pitch_dbu

    def clip(self, i: int) -> np.ndarray:
        return self.rects[self.rect_off[i]:self.rect_off[i + 1]]

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.clip(int(i)) for i in idx]
        counts = np.array([p.shape[0] for p in parts], dtype=np.int64)
        off = np.zeros(len(parts) + 1, dtype=np.uint32)
        off[1:] = np.cumsum(counts)
        rects = np.concatenate(parts, axis=0) if parts else np.zeros((0, 4), np.int32)
        return Workload(self.name + "[sub]", self.window_dbu, self.pitch_dbu, self.marker_dbu,
                        off, np.ascontiguousarray(rects, dtype=np.int32), self.label[idx].copy(),
                        dict(self.meta))


PRESETS = {
    "small": dict(n_clips=1000, n_seeds=100, n_copies=600, window_dbu=512, margin_dbu=32,
                  min_rects=3, max_rects=12, min_side=20, max_side=120, grid=10, spacing=20,
                  edge_jitter=8, shift_max=32, pitch_dbu=4),
    "scale": dict(n_clips=100_000, n_seeds=5_000, n_copies=70_000, window_dbu=1024, margin_dbu=64,
                  min_rects=5, max_rects=40, min_side=20, max_side=120, grid=10, spacing=20,
                  edge_jitter=8, shift_max=64, pitch_dbu=4),
}


def generate(seed: int = 1, *, n_clips: int, n_seeds: int, n_copies: int, window_dbu: int,
             margin_dbu: int, min_rects: int, max_rects: int, min_side: int = 20,
             max_side: int = 120, grid: int = 10, spacing: int = 20, edge_jitter: int = 8,
             shift_max: int | None = None, pitch_dbu: int = 4, name: str = "custom", halo_dbu: int = 0) -> Workload:
    """halo_dbu > 0 keeps each clip's rectangles over [-halo, W + halo)^2
    (the layout around the window) instead of cutting them to the window."""
    lib = _load()
    cfg = _Cfg(seed, n_clips, n_seeds, n_copies, window_dbu, margin_dbu, min_rects, max_rects,
               min_side, max_side, grid, spacing, edge_jitter,
               margin_dbu if shift_max is None else shift_max, halo_dbu)
    cap = int(n_clips) * int(max(max_rects, 1))
    off = np.zeros(n_clips + 1, dtype=np.uint32)
    rects = np.zeros((cap, 4), dtype=np.int32)
    label = np.zeros(n_clips, dtype=np.int32)
    total = lib.pcl_synth_generate(ctypes.byref(cfg), off.ctypes.data, rects.ctypes.data, cap,
                                   label.ctypes.data)
    if total < 0:
        raise ValueError("pcl_synth_generate rejected the configuration")
    return Workload(name, window_dbu, pitch_dbu, margin_dbu, off, rects[:total].copy(), label,
                    dict(seed=seed, n_seeds=n_seeds, n_copies=n_copies, min_rects=min_rects,
                         max_rects=max_rects, halo_dbu=halo_dbu))


def preset(name: str, seed: int = 1, **over) -> Workload:
    kw = dict(PRESETS[name])
    kw.update(over)
    return generate(seed, name=name, **kw)


def from_lists(clips, window_dbu: int, pitch_dbu: int = 4, marker_dbu: int = 0,
               name: str = "lists") -> Workload:
    """Workload from explicit rectangle lists (hand-written test cases)."""
    counts = [len(c) for c in clips]
    off = np.zeros(len(clips) + 1, dtype=np.uint32)
    off[1:] = np.cumsum(counts)
    flat = [r for c in clips for r in c]
    rects = np.array(flat, dtype=np.int32).reshape(-1, 4)
    return Workload(name, window_dbu, pitch_dbu, marker_dbu, off, rects,
                    np.full(len(clips), -1, np.int32))


def concat(first: Workload, second: Workload, name: str = "concat") -> Workload:
    """The clips of `first` followed by those of `second` (same window, pitch
    and marker); clip k of `second` becomes clip first.n + k."""
    off = np.concatenate([first.rect_off[:-1], second.rect_off + first.rect_off[-1]]).astype(np.uint32)
    rects = np.ascontiguousarray(np.concatenate([first.rects, second.rects]), dtype=np.int32)
    return Workload(name, first.window_dbu, first.pitch_dbu, first.marker_dbu, off, rects,
                    np.concatenate([first.label, second.label]), dict(first.meta))


def gate_bounds_set(seed: int, k: int = 16, tol_dbu: int = 4) -> Workload:
    """Clips placed so that both constraint modes pass across the edge gates'
    bounds (W = 512 dbu, 4 dbu/px, marker half-width 32 dbu).  Per random
    interior clip A (5-8 rectangles of sides 40-60 dbu, one in each chosen
    cell of a 3 x 3 grid of 88-dbu cells, so >= 20 dbu apart), four clips:
      A;
      A moved by a pixel multiple (at most 24 dbu per axis);
      A moved by a pixel multiple (at most 16 dbu) with every rectangle
        shrunk by tol_dbu on each side (bbox width and height tol_dbu * 2
        below A's);
      A plus two 20 x 20 dbu rectangles placed symmetrically left and right
        of A's bbox, 40-76 dbu beyond it (two polygons more, bbox centre
        unchanged, bbox width far larger)."""
    rng = np.random.default_rng(seed)
    clips = []

    def moved(rs, tx, ty):
        return [[r[0] + tx, r[1] + ty, r[2] + tx, r[3] + ty] for r in rs]

    for _ in range(k):
        rects = []
        for c in rng.permutation(9)[: int(rng.integers(5, 9))]:
            ox, oy = (int(4 * v) for v in rng.integers(0, 3, size=2))
            x0, y0 = 140 + 88 * int(c % 3) + ox, 140 + 88 * int(c // 3) + oy
            w, h = (int(4 * v) for v in rng.integers(10, 16, size=2))
            rects.append([x0, y0, x0 + w, y0 + h])
        tx, ty = (int(4 * v) for v in rng.integers(-6, 7, size=2))
        t = tol_dbu
        shrunk = [[r[0] + t, r[1] + t, r[2] - t, r[3] - t] for r in rects]
        qx, qy = (int(4 * v) for v in rng.integers(-4, 5, size=2))
        lx = min(r[0] for r in rects)
        ux = max(r[2] for r in rects)
        ly = min(r[1] for r in rects)
        e = int(4 * rng.integers(15, 25))
        extra = [[lx - e, ly, lx - e + 20, ly + 20], [ux + e - 20, ly, ux + e, ly + 20]]
        clips += [rects, moved(rects, tx, ty), moved(shrunk, qx, qy), rects + extra]
    return from_lists(clips, 512, 4, 32, name="gate_bounds")


def batched(seed: int = 1, clips_per_class: int = 1000, sizes=(64, 128, 256, 512), pitch_dbu: int = 4,
            zipf_s: float = 1.1, max_list: int = 5000, same_seed_frac: float = 0.5, min_rects: int = 5,
            max_rects: int = 40):
    """Mixed-size batch: one clip set per raster size (W = N * pitch, marker
    half-width W/16, 70 % perturbed copies), and per clip a candidate list of
    Zipf(zipf_s) length truncated to [1, max_list]; a partner is drawn from the
    clip's seed group with probability same_seed_frac (when it has one), else
    uniformly from its size class.  Each pair gets a mode, cosine or edge,
    with probability 1/2.  Returns (workloads, pairs[m, 3] = (class, a, b),
    modes[m])."""
    rng = np.random.default_rng(seed)
    wls = []
    for k, N in enumerate(sizes):
        W = N * pitch_dbu
        M = W // 16
        n_seeds = max(1, clips_per_class // 20)
        wls.append(generate(seed * 101 + k, n_clips=clips_per_class, n_seeds=n_seeds,
                            n_copies=int(0.7 * clips_per_class), window_dbu=W, margin_dbu=M,
                            min_rects=min_rects, max_rects=max_rects, pitch_dbu=pitch_dbu, name=f"batched{N}"))
    # truncated Zipf: P(k) proportional to k^-s on [1, max_list] (inverse CDF)
    ks = np.arange(1, max_list + 1, dtype=np.float64)
    cdf = np.cumsum(ks ** -zipf_s)
    cdf /= cdf[-1]
    out = []
    for k, wl in enumerate(wls):
        n = wl.n
        lab = wl.label.astype(np.int64)
        lens = 1 + np.searchsorted(cdf, rng.random(n), side="right")
        lens = np.minimum(lens, max_list)
        a = np.repeat(np.arange(n), lens)
        b = rng.integers(0, n, size=a.shape[0])
        # same-seed partners: members of each seed group, grouped by label
        order = np.argsort(lab, kind="stable")
        ls = lab[order]
        first = np.searchsorted(ls, lab, side="left")
        size = np.searchsorted(ls, lab, side="right") - first
        same = (rng.random(a.shape[0]) < same_seed_frac) & (lab[a] >= 0) & (size[a] > 1)
        pick = first[a[same]] + (rng.random(int(same.sum())) * size[a[same]]).astype(np.int64)
        b[same] = order[pick]
        keep = a != b
        out.append(np.stack([np.full(int(keep.sum()), k), a[keep], b[keep]], 1))
    pairs = np.concatenate(out).astype(np.int64)
    modes = np.where(rng.random(len(pairs)) < 0.5, 1, 2).astype(np.int64)
    return wls, pairs, modes
