"""Python binding of libpcl (include/pcl.h): argument marshalling only.

Every step of the similarity path runs in the CUDA kernels of ``libpcl.so``;
this module loads that library (and fails loudly when it is missing), passes
plain pointers and sizes across the C ABI, and uses PyTorch for device memory
and streams.  Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))

PCL_OK = 0
PCL_ERR_INVALID = 1
PCL_ERR_OOM = 2
PCL_ERR_CUDA = 3
PCL_ERR_TIMEOUT = 4
PCL_ERR_BUSY = 5
PCL_ERR_UNSUPPORTED = 6

MODE_COSINE = 1
MODE_EDGE = 2
ENGINE_FFT_PCM = 0
ENGINE_TC_DIRECT = 1
ENGINE_TC_DIRECT_FP8 = 2
ENGINE_XYSEP = 3  # shift by XY-separation interval competition (Sec. 3.2.1 (2))
ENGINE_TC_DIRECT_BF16 = 4
ENGINE_EXACT_SCAN = 5  # bound-pruned exact window scan (N = 128, 256, 512; no spectra)
SHIFT_EXACT_ARGMAX = 0
SHIFT_PCM_PEAK = 1
P_NO_GATES = 1
P_NO_PCM = 2
P_TOPO_HASH = 4  # self-join candidates: lossy topological pre-screen first

GATE_NONE = 0
GATE_G1_AREA = 1
GATE_G2_PROFILE = 2
GATE_G3_DENSITY = 3
GATE_E1_MATCH = 4
GATE_E2_BBOX = 5
GATE_T0_TOPO = 6
GATE_UNSUPPORTED = 14
GATE_BAD_INDEX = 15
F_NEAR_BAND = 1 << 4
F_FFT_GUARD = 1 << 5
F_PCM_AGREES = 1 << 6
F_EDGE_VERIFY_FAIL = 1 << 7
F_EMPTY = 1 << 8
F_ALIGNED = 1 << 9

REC_DTYPE = np.dtype([
    ("a", "<u4"), ("b", "<u4"), ("dx_dbu", "<i4"), ("dy_dbu", "<i4"), ("sim", "<f4"),
    ("score", "<u4"), ("pcm_dx_dbu", "<i4"), ("pcm_dy_dbu", "<i4"), ("flags", "<u2"),
    ("pass_", "u1"), ("mode", "u1"), ("reserved", "<u4")])
assert REC_DTYPE.itemsize == 40


class PclError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pcl status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("pitch_dbu", ctypes.c_int32), ("window_dbu", ctypes.c_int32),
                ("marker_dbu", ctypes.c_int32), ("cos_num", ctypes.c_uint32),
                ("cos_den", ctypes.c_uint32), ("edge_tol_dbu", ctypes.c_int32),
                ("cos_engine", ctypes.c_uint32), ("shift_rule", ctypes.c_uint32),
                ("near_band", ctypes.c_float), ("flags", ctypes.c_uint32)]


def params(window_dbu: int, pitch_dbu: int = 4, marker_dbu: int = 32, cos_num: int = 95,
           cos_den: int = 100, edge_tol_dbu: int = 4, cos_engine: int = ENGINE_FFT_PCM,
           shift_rule: int = SHIFT_EXACT_ARGMAX, near_band: float = 1e-4, flags: int = 0) -> Params:
    return Params(pitch_dbu, window_dbu, marker_dbu, cos_num, cos_den, edge_tol_dbu, cos_engine,
                  shift_rule, near_band, flags)


class _Clipset(ctypes.Structure):
    _fields_ = [("n_clips", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("rect_off", ctypes.c_void_p), ("rects", ctypes.c_void_p),
                ("bits", ctypes.c_void_p), ("pop", ctypes.c_void_p), ("prof", ctypes.c_void_p),
                ("blk", ctypes.c_void_p), ("esig", ctypes.c_void_p), ("occ", ctypes.c_void_p),
                ("rorder", ctypes.c_void_p), ("spec", ctypes.c_void_p), ("spec_state", ctypes.c_void_p)]


class _Sizes(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_uint64), ("pop", ctypes.c_uint64), ("prof", ctypes.c_uint64),
                ("blk", ctypes.c_uint64), ("esig", ctypes.c_uint64), ("occ", ctypes.c_uint64),
                ("rorder", ctypes.c_uint64), ("spec", ctypes.c_uint64),
                ("spec_state", ctypes.c_uint64), ("N", ctypes.c_int32), ("S", ctypes.c_int32),
                ("L", ctypes.c_int32), ("Ls", ctypes.c_int32)]


class _Pair(ctypes.Structure):
    _fields_ = [("a", ctypes.c_uint32), ("b", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("fft_radix", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("items_per_warp", ctypes.c_uint32)]


WORK_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("cls", "<u2"), ("mode", "<u2")])
assert WORK_DTYPE.itemsize == 12


class _ServerCfg(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("max_query_clips", ctypes.c_uint32),
                ("max_query_rects", ctypes.c_uint64), ("cand_per_query", ctypes.c_uint32),
                ("pass_copy", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class _Completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_queries", ctypes.c_uint32),
                ("n_candidates", ctypes.c_uint64), ("n_pass", ctypes.c_uint64), ("pass_", ctypes.c_void_p),
                ("t_submit_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64), ("size_class", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("n_records", ctypes.c_uint64), ("records", ctypes.c_void_p)]


_lib = None
_VP = ctypes.c_void_p
_U64 = ctypes.c_uint64


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpcl.so; raises if it cannot be built or loaded (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libpcl not built at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    st = ctypes.c_int
    sig = {
        "pcl_create": ([ctypes.POINTER(_VP), ctypes.c_int], st),
        "pcl_destroy": ([_VP], None),
        "pcl_last_error": ([_VP], ctypes.c_char_p),
        "pcl_status_string": ([st], ctypes.c_char_p),
        "pcl_params_validate": ([ctypes.POINTER(Params)], st),
        "pcl_clipset_sizes_get": ([ctypes.POINTER(Params), ctypes.c_uint32, _U64, ctypes.POINTER(_Sizes)], st),
        "pcl_rasterize": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), _VP], st),
        "pcl_spectra": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), _VP, ctypes.c_uint32, _VP], st),
        "pcl_candidates": ([_VP, ctypes.POINTER(Params), ctypes.c_uint32, ctypes.POINTER(_Clipset),
                            ctypes.POINTER(_Clipset), _VP, _U64, _VP, _VP, _VP], st),
        "pcl_candidates_shard": ([_VP, ctypes.POINTER(Params), ctypes.c_uint32, ctypes.POINTER(_Clipset),
                                  ctypes.c_uint32, ctypes.c_uint32, _VP, _U64, _VP, _VP, _VP], st),
        "pcl_candidates_cosine_noalloc": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), _VP, _U64,
                                           _VP, _VP, _VP], st),
        "pcl_match_pairs": ([_VP, ctypes.POINTER(Params), ctypes.c_uint32, ctypes.POINTER(_Clipset),
                             ctypes.POINTER(_Clipset), _VP, _U64, _VP, _VP, _VP], st),
        "pcl_device_error": ([_VP, ctypes.POINTER(ctypes.c_int)], st),
        "pcl_set_wait_limit": ([_VP, _U64], st),
        "pcl_stats_get": ([_VP, _VP, ctypes.c_int], st),
        "pcl_surprisal": ([_VP, _VP, _U64, _VP, ctypes.c_uint32, _VP, _VP, _VP, _VP], st),
        "pcl_halo_sizes_get": ([ctypes.POINTER(Params), ctypes.c_uint32, ctypes.POINTER(_U64),
                                ctypes.POINTER(_U64)], st),
        "pcl_rasterize_halo": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), _VP, _VP, _VP], st),
        "pcl_match_halo": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), ctypes.POINTER(_Clipset), _VP,
                            _VP, _VP, _U64, _VP, _VP, _VP], st),
        "pcl_compact_pass": ([_VP, _VP, _U64, _VP, _VP, _U64, _VP, _VP], st),
        "pcl_match_mixed": ([_VP, _VP, _VP, ctypes.c_uint32, _VP, _U64, _U64, _VP, ctypes.POINTER(Tuning), _VP], st),
        "pcl_server_create": ([_VP, ctypes.POINTER(Params), ctypes.POINTER(_Clipset), ctypes.POINTER(_ServerCfg),
                               ctypes.POINTER(_VP)], st),
        "pcl_server_create_classes": ([_VP, _VP, _VP, ctypes.c_uint32, ctypes.POINTER(_ServerCfg),
                                       ctypes.POINTER(_VP)], st),
        "pcl_server_submit": ([_VP, _VP, _VP, ctypes.c_uint32, _U64], st),
        "pcl_server_submit_class": ([_VP, ctypes.c_uint32, _VP, _VP, ctypes.c_uint32, _U64], st),
        "pcl_server_poll": ([_VP, ctypes.POINTER(_Completion), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)], st),
        "pcl_server_release": ([_VP, _U64], st),
        "pcl_server_stats": ([_VP, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_U64)], st),
        "pcl_server_destroy": ([_VP], None),
        "pcl_setcover": ([_VP, _U64, ctypes.c_uint32, _VP, _VP, ctypes.POINTER(ctypes.c_uint32)], st),
        "pcl_cluster_loop": ([_VP, _VP, _VP, _U64, ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_uint32),
                              ctypes.POINTER(ctypes.c_uint32)], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    """Entry points declared in include/pcl.h (for the ABI load test)."""
    import re
    with open(os.path.join(_build.INCLUDE, "pcl.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:const char \*|pcl_status |void )(pcl_\w+)\(", txt, re.M)))


# ---------------------------------------------------------------- plumbing

def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Context:
    """Owns a pcl_ctx (device binding, error string, grow-only workspace)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = _VP()
        s = self.lib.pcl_create(ctypes.byref(h), device)
        if s != PCL_OK:
            raise PclError(s, "pcl_create failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.pcl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, s: int, what: str):
        if s != PCL_OK:
            msg = self.lib.pcl_last_error(self.h).decode() if self.h else ""
            raise PclError(s, f"{what}: {msg}")


@dataclass
class ClipSet:
    """Device buffers of a clip set (PyTorch-allocated) and its C view."""
    n: int
    N: int
    S: int
    L: int
    Ls: int
    rect_off: object
    rects: object
    bits: object
    pop: object
    prof: object
    blk: object
    esig: object
    occ: object
    rorder: object
    spec: object
    spec_state: object

    def view(self, P: Params, c0: int, c1: int) -> "ClipSet":
        """Clips [c0, c1) as a clip set of their own, sharing this set's
        device memory (no copy): per-clip arrays start at clip c0, the
        rectangle offsets keep indexing this set's rectangle array.  Clip k of
        the view is clip c0 + k here."""
        if not 0 <= c0 <= c1 <= self.n:
            raise ValueError("clip range out of bounds")
        one, two = clipset_sizes(P, 1), clipset_sizes(P, 2)

        def part(t, field):
            if t is None:
                return None
            per = int(getattr(two, field)) - int(getattr(one, field))
            return t[c0 * per:c1 * per]

        return ClipSet(c1 - c0, self.N, self.S, self.L, self.Ls, self.rect_off[c0:c1 + 1], self.rects,
                       part(self.bits, "bits"), part(self.pop, "pop"), part(self.prof, "prof"),
                       part(self.blk, "blk"), part(self.esig, "esig"), part(self.occ, "occ"), self.rorder,
                       part(self.spec, "spec"), part(self.spec_state, "spec_state"))

    def cstruct(self) -> _Clipset:
        return _Clipset(self.n, 0, _ptr(self.rect_off), _ptr(self.rects), _ptr(self.bits), _ptr(self.pop),
                        _ptr(self.prof), _ptr(self.blk), _ptr(self.esig), _ptr(self.occ), _ptr(self.rorder),
                        _ptr(self.spec), _ptr(self.spec_state))


def clipset_sizes(P: Params, n: int, n_rects: int = 0) -> _Sizes:
    lib = load()
    sz = _Sizes()
    s = lib.pcl_clipset_sizes_get(ctypes.byref(P), n, n_rects, ctypes.byref(sz))
    if s != PCL_OK:
        raise PclError(s, "pcl_clipset_sizes_get: invalid parameters")
    return sz


def alloc_clipset(P: Params, rect_off, rects, device="cuda", with_spec: bool = True) -> ClipSet:
    """Allocate the device buffers of a clip set; rect_off/rects are copied to
    the device if given as host arrays (numpy) or used as-is (torch CUDA)."""
    torch = _torch()
    if isinstance(rect_off, np.ndarray):
        rect_off = torch.from_numpy(np.ascontiguousarray(rect_off, dtype=np.uint32).view(np.int32)).to(device)
    if isinstance(rects, np.ndarray):
        r = np.ascontiguousarray(rects, dtype=np.int32).reshape(-1)
        if r.size == 0:
            r = np.zeros(4, np.int32)
        rects = torch.from_numpy(r).to(device)
    n = int(rect_off.numel()) - 1
    sz = clipset_sizes(P, n, int(rects.numel()) // 4)

    def buf(nbytes):
        return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)

    spec = buf(sz.spec) if with_spec else None
    state = torch.zeros(max(int(sz.spec_state), 16), dtype=torch.uint8, device=device) if with_spec else None
    return ClipSet(n, sz.N, sz.S, sz.L, sz.Ls, rect_off, rects, buf(sz.bits), buf(sz.pop), buf(sz.prof),
                   buf(sz.blk), buf(sz.esig), buf(sz.occ), buf(sz.rorder), spec, state)


# ---------------------------------------------------------------- entry points

def pcl_rasterize(ctx: Context, P: Params, cs: ClipSet, stream=None) -> None:
    c = cs.cstruct()
    ctx.check(ctx.lib.pcl_rasterize(ctx.h, ctypes.byref(P), ctypes.byref(c), _stream_ptr(stream)),
              "pcl_rasterize")


def pcl_spectra(ctx: Context, P: Params, cs: ClipSet, clip_list=None, stream=None) -> None:
    c = cs.cstruct()
    n_list = 0 if clip_list is None else int(clip_list.numel())
    ctx.check(ctx.lib.pcl_spectra(ctx.h, ctypes.byref(P), ctypes.byref(c), _ptr(clip_list), n_list,
                                  _stream_ptr(stream)), "pcl_spectra")


def pcl_candidates(ctx: Context, P: Params, mode: int, cs: ClipSet, out_pairs, d_count, d_gates=None,
                   stream=None, b: ClipSet | None = None) -> None:
    """out_pairs: int32 CUDA tensor [cap, 2]; d_count: int64 CUDA tensor [1];
    d_gates: int64 CUDA tensor [16] (accumulated) or None; b: second clip set
    (pairs of cs x b) or None (self-join of cs)."""
    c = cs.cstruct()
    cb = b.cstruct() if b is not None else None
    cap = 0 if out_pairs is None else int(out_pairs.shape[0])
    ctx.check(ctx.lib.pcl_candidates(ctx.h, ctypes.byref(P), mode, ctypes.byref(c),
                                     ctypes.byref(cb) if cb is not None else None, _ptr(out_pairs), cap,
                                     _ptr(d_count), _ptr(d_gates), _stream_ptr(stream)), "pcl_candidates")


def pcl_candidates_shard(ctx: Context, P: Params, mode: int, cs: ClipSet, shard: int, n_shards: int, out_pairs,
                         d_count, d_gates=None, stream=None) -> None:
    """pcl_candidates_shard: the pairs of shard `shard` of `n_shards` only."""
    c = cs.cstruct()
    cap = 0 if out_pairs is None else int(out_pairs.shape[0])
    ctx.check(ctx.lib.pcl_candidates_shard(ctx.h, ctypes.byref(P), mode, ctypes.byref(c), shard, n_shards,
                                           _ptr(out_pairs), cap, _ptr(d_count), _ptr(d_gates),
                                           _stream_ptr(stream)), "pcl_candidates_shard")


def pcl_candidates_cosine_noalloc(ctx: Context, P: Params, cs: ClipSet, out_pairs, d_count, d_gates=None,
                                  stream=None, n_clips: int | None = None) -> None:
    """Cosine candidates without device allocation (fixed library scratch);
    arguments as pcl_candidates.  n_clips overrides the clip count passed
    across the ABI (used to exercise the size limit)."""
    c = cs.cstruct()
    if n_clips is not None:
        c.n_clips = n_clips
    cap = 0 if out_pairs is None else int(out_pairs.shape[0])
    ctx.check(ctx.lib.pcl_candidates_cosine_noalloc(ctx.h, ctypes.byref(P), ctypes.byref(c), _ptr(out_pairs), cap,
                                                    _ptr(d_count), _ptr(d_gates), _stream_ptr(stream)),
              "pcl_candidates_cosine_noalloc")


def pcl_match_pairs(ctx: Context, P: Params, mode: int, a: ClipSet, b: ClipSet, pairs, out_rec,
                    d_n=None, stream=None) -> None:
    """pairs: int32 CUDA tensor [n, 2]; out_rec: uint8 CUDA tensor [n, 40];
    d_n: optional int64 CUDA tensor [1] limiting the count on the device."""
    ca, cb = a.cstruct(), b.cstruct()
    n = int(pairs.shape[0])
    ctx.check(ctx.lib.pcl_match_pairs(ctx.h, ctypes.byref(P), mode, ctypes.byref(ca), ctypes.byref(cb),
                                      _ptr(pairs), n, _ptr(d_n), _ptr(out_rec), _stream_ptr(stream)),
              "pcl_match_pairs")


def pcl_match_mixed(ctx: Context, params_list, sets, work, n_cosine: int, out_rec, tune: Tuning | None = None,
                    stream=None) -> None:
    """params_list/sets: per size class; work: uint8 CUDA tensor [n, 12] of
    pcl_work (cosine items first); out_rec: uint8 CUDA tensor [n, 40]."""
    k = len(sets)
    P_arr = (Params * k)(*params_list)
    S_arr = (_Clipset * k)(*[c.cstruct() for c in sets])
    n = int(work.shape[0])
    ctx.check(ctx.lib.pcl_match_mixed(ctx.h, ctypes.cast(P_arr, _VP), ctypes.cast(S_arr, _VP), k, _ptr(work),
                                      n_cosine, n, _ptr(out_rec), ctypes.byref(tune) if tune else None,
                                      _stream_ptr(stream)), "pcl_match_mixed")


def pcl_device_error(ctx: Context) -> int:
    """Synchronise and return the device error word (0: none); raises
    PclError(PCL_ERR_TIMEOUT) when a bounded device wait ran out."""
    f = ctypes.c_int()
    ctx.check(ctx.lib.pcl_device_error(ctx.h, ctypes.byref(f)), "pcl_device_error")
    return int(f.value)


def pcl_surprisal(ctx: Context, edges, n_nodes: int, d_n=None, stream=None):
    """Degrees (int32), surprisal weights and first-step scores (int64) of
    the graph of an int32 CUDA pair tensor [m, 2] on n_nodes nodes, as CUDA
    tensors (Sec. 3.3.1, Eqs. 7-9)."""
    torch = _torch()
    dev = edges.device
    deg = torch.empty(max(n_nodes, 1), dtype=torch.int32, device=dev)
    w = torch.empty(max(n_nodes, 1), dtype=torch.int64, device=dev)
    sc = torch.empty(max(n_nodes, 1), dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.pcl_surprisal(ctx.h, _ptr(edges), int(edges.shape[0]), _ptr(d_n), n_nodes, _ptr(deg), _ptr(w),
                                    _ptr(sc), _stream_ptr(stream)), "pcl_surprisal")
    return deg[:n_nodes], w[:n_nodes], sc[:n_nodes]


def alloc_halo(P: Params, cs: ClipSet):
    """device buffers (halo rasters, moved-window pixel counts) for the
    clips of cs under P"""
    torch = _torch()
    hb, nb = _U64(), _U64()
    s = load().pcl_halo_sizes_get(ctypes.byref(P), cs.n, ctypes.byref(hb), ctypes.byref(nb))
    if s != PCL_OK:
        raise PclError(s, "pcl_halo_sizes_get")
    dev = cs.bits.device
    return (torch.empty(max(int(hb.value), 16), dtype=torch.uint8, device=dev),
            torch.empty(max(int(nb.value), 16), dtype=torch.uint8, device=dev))


def pcl_rasterize_halo(ctx: Context, P: Params, cs: ClipSet, hbits, norms, stream=None) -> None:
    c = cs.cstruct()
    ctx.check(ctx.lib.pcl_rasterize_halo(ctx.h, ctypes.byref(P), ctypes.byref(c), _ptr(hbits), _ptr(norms),
                                         _stream_ptr(stream)), "pcl_rasterize_halo")


def pcl_match_halo(ctx: Context, P: Params, a: ClipSet, b: ClipSet, hbits_b, norms_b, pairs, out_rec, d_n=None,
                   stream=None) -> None:
    """records of the re-extraction reading for an int32 CUDA pair tensor
    [n, 2] into a uint8 CUDA tensor [n, 40]"""
    ca, cb = a.cstruct(), b.cstruct()
    ctx.check(ctx.lib.pcl_match_halo(ctx.h, ctypes.byref(P), ctypes.byref(ca), ctypes.byref(cb), _ptr(hbits_b),
                                     _ptr(norms_b), _ptr(pairs), int(pairs.shape[0]), _ptr(d_n), _ptr(out_rec),
                                     _stream_ptr(stream)), "pcl_match_halo")


def pcl_set_wait_limit(ctx: Context, ns: int) -> None:
    """Limit of each bounded device-side wait (ns; 0 = one second)."""
    ctx.check(ctx.lib.pcl_set_wait_limit(ctx.h, int(ns)), "pcl_set_wait_limit")


def pcl_stats_get(ctx: Context, reset: bool = False, kernel: str = "exact") -> tuple:
    """(groups of shifts counted, groups in the windows) of the exact window
    scan (kernel="exact") or of the re-extraction pair kernel ("halo") since
    the context was created or last reset; synchronous."""
    out = (ctypes.c_uint64 * 4)()
    ctx.check(ctx.lib.pcl_stats_get(ctx.h, ctypes.cast(out, _VP), 1 if reset else 0), "pcl_stats_get")
    k = {"exact": 0, "halo": 2}[kernel]
    return int(out[k]), int(out[k + 1])


def pcl_compact_pass(ctx: Context, rec, out_pairs, d_count, d_n=None, stream=None) -> None:
    n = int(rec.shape[0])
    cap = int(out_pairs.shape[0])
    ctx.check(ctx.lib.pcl_compact_pass(ctx.h, _ptr(rec), n, _ptr(d_n), _ptr(out_pairs), cap, _ptr(d_count),
                                       _stream_ptr(stream)), "pcl_compact_pass")


def pcl_setcover(edges: np.ndarray, n_nodes: int):
    """Host lazy greedy (Sec. 3.3).  Returns (order, rep_of) as numpy arrays."""
    lib = load()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
    rep = np.zeros(max(n_nodes, 1), dtype=np.uint32)
    order = np.zeros(max(n_nodes, 1), dtype=np.uint32)
    k = ctypes.c_uint32()
    s = lib.pcl_setcover(e.ctypes.data if e.size else None, e.shape[0], n_nodes, rep.ctypes.data,
                         order.ctypes.data, ctypes.byref(k))
    if s != PCL_OK:
        raise PclError(s, "pcl_setcover")
    return order[:k.value].astype(np.int64), rep[:n_nodes].astype(np.int64)


def pcl_cluster_loop(pairs: np.ndarray, strict: np.ndarray, relaxed: np.ndarray, n_nodes: int):
    """Host coarse-to-fine loop (Sec. 3.1).  Returns (rep_of, n_clusters, rounds)."""
    lib = load()
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.uint32).reshape(-1, 2))
    s8 = np.ascontiguousarray(np.asarray(strict, dtype=np.uint8))
    r8 = np.ascontiguousarray(np.asarray(relaxed, dtype=np.uint8))
    rep = np.zeros(max(n_nodes, 1), dtype=np.uint32)
    ncl, nr = ctypes.c_uint32(), ctypes.c_uint32()
    s = lib.pcl_cluster_loop(p.ctypes.data if p.size else None, s8.ctypes.data if s8.size else None,
                             r8.ctypes.data if r8.size else None, p.shape[0], n_nodes, rep.ctypes.data,
                             ctypes.byref(ncl), ctypes.byref(nr))
    if s != PCL_OK:
        raise PclError(s, "pcl_cluster_loop")
    return rep[:n_nodes].astype(np.int64), int(ncl.value), int(nr.value)


# ---------------------------------------------------------------- helpers

def records_to_numpy(rec) -> np.ndarray:
    """uint8 [n, 40] tensor (any device) -> structured numpy records"""
    a = rec.detach().to("cpu").contiguous().numpy()
    return a.reshape(-1).view(REC_DTYPE)


def unpack_bits(cs: ClipSet) -> np.ndarray:
    """raster bits -> uint8 images [n, N, N] indexed [clip, y, x] (for tests)"""
    w = cs.bits[: cs.n * cs.N * (cs.N // 64) * 8].cpu().numpy().view(np.uint64)
    w = w.reshape(cs.n, cs.N, cs.N // 64)
    b = np.unpackbits(w.view(np.uint8).reshape(cs.n, cs.N, -1), axis=2, bitorder="little")
    return b.reshape(cs.n, cs.N, cs.N)


def blk_positions(nb: int) -> np.ndarray:
    """[nb, nb] storage positions of the 16x16 blocks (by, bx) in a clip set's
    blk buffer (the layout documented at pcl_clipset in pcl.h)"""
    by, bx = np.meshgrid(np.arange(nb), np.arange(nb), indexing="ij")
    q = nb // 4
    return ((by % 4) * 4 + bx % 4) * q * q + (by // 4) * q + bx // 4


def signatures(cs: ClipSet):
    """pop, profiles, block counts, edge signatures as numpy (for tests)"""
    n, N = cs.n, cs.N
    nb = N // 16
    pop = cs.pop[: 4 * n].cpu().numpy().view(np.uint32)
    prof = cs.prof[: 4 * n * N].cpu().numpy().view(np.uint16).reshape(n, 2, N)
    stored = cs.blk[: 4 * n * nb * nb].cpu().numpy().view(np.uint16).reshape(n, 2, nb * nb)
    blk = stored[:, :, blk_positions(nb)]  # back to row-major (by, bx)
    esig = cs.esig[: 32 * n].cpu().numpy().view(np.int32).reshape(n, 8)
    return dict(pop=pop, rows=prof[:, 0], cols=prof[:, 1], blk=blk[:, 0], dil=blk[:, 1], esig=esig)


def candidates(ctx: Context, P: Params, mode: int, cs: ClipSet, cap: int = 1 << 20, stream=None,
               shard: int = 0, n_shards: int = 1, b: ClipSet | None = None):
    """Self-join candidate pairs of `mode` (re-runs once with the exact capacity
    if `cap` was too small), those of one shard of the pair space, or with
    `b` the pairs of cs x b.  Returns (pairs int32 [m, 2] CUDA, gate counts
    numpy int64 [16])."""
    torch = _torch()
    dev = cs.bits.device
    for _ in range(2):
        out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        gates = torch.zeros(16, dtype=torch.int64, device=dev)
        if n_shards == 1:
            pcl_candidates(ctx, P, mode, cs, out, cnt, gates, stream, b=b)
        else:
            pcl_candidates_shard(ctx, P, mode, cs, shard, n_shards, out, cnt, gates, stream)
        m = int(cnt.item())
        if m <= cap:
            return out[:m], gates.cpu().numpy()
        cap = m
    raise PclError(PCL_ERR_BUSY, "candidate capacity")


def match(ctx: Context, P: Params, mode: int, a: ClipSet, b: ClipSet, pairs, stream=None):
    """Records (uint8 CUDA tensor [n, 40]) for an int32 CUDA pair tensor [n, 2]."""
    torch = _torch()
    out = torch.empty((int(pairs.shape[0]), 40), dtype=torch.uint8, device=pairs.device)
    pcl_match_pairs(ctx, P, mode, a, b, pairs.contiguous(), out, None, stream)
    return out


class Server:
    """pcl_server_*: resident libraries (one per size class) and continuously
    batched query requests.  `P` and `library` are one parameter block and
    one clip set, or equal-length lists of them (size class c = P[c],
    library[c])."""

    def __init__(self, ctx: Context, P, library, max_inflight: int = 8,
                 max_query_clips: int = 4096, max_query_rects: int = 4096 * 48, cand_per_query: int = 256,
                 pass_copy: int = 1 << 16, mem_budget: int = 8 << 30, mode: int = MODE_COSINE):
        self.ctx = ctx
        self.lib = ctx.lib
        Ps = list(P) if isinstance(P, (list, tuple)) else [P]
        libs = list(library) if isinstance(library, (list, tuple)) else [library]
        if len(Ps) != len(libs):
            raise ValueError("one parameter block per library")
        self.library = libs  # keeps the library buffers alive
        self._P = (Params * len(Ps))(*Ps)
        self._cl = (_Clipset * len(libs))(*[c.cstruct() for c in libs])
        cfg = _ServerCfg(max_inflight, max_query_clips, max_query_rects, cand_per_query, pass_copy, mem_budget,
                         mode, 0)
        h = _VP()
        ctx.check(self.lib.pcl_server_create_classes(ctx.h, ctypes.cast(self._P, _VP), ctypes.cast(self._cl, _VP),
                                                     len(libs), ctypes.byref(cfg), ctypes.byref(h)),
                  "pcl_server_create")
        self.h = h
        self._keep = {}

    def submit(self, rect_off: np.ndarray, rects: np.ndarray, request_id: int, cls: int = 0) -> bool:
        """True if admitted, False if busy (no slot or memory); raises on errors."""
        off = np.ascontiguousarray(rect_off, dtype=np.uint32)
        r = np.ascontiguousarray(rects, dtype=np.int32).reshape(-1)
        st = self.lib.pcl_server_submit_class(self.h, cls, off.ctypes.data, r.ctypes.data if r.size else None,
                                              off.shape[0] - 1, request_id)
        if st == PCL_ERR_BUSY:
            return False
        self.ctx.check(st, "pcl_server_submit")
        return True

    def poll(self, cap: int = 64) -> list[dict]:
        """Finished requests; their pass lists and records are copied out and
        the slots released."""
        arr = (_Completion * cap)()
        n = ctypes.c_uint32()
        self.ctx.check(self.lib.pcl_server_poll(self.h, arr, cap, ctypes.byref(n)), "pcl_server_poll")
        out = []
        for c in arr[: n.value]:
            k = int(c.n_pass)
            if k:
                buf = (ctypes.c_uint32 * (2 * k)).from_address(c.pass_)
                pairs = np.frombuffer(buf, dtype=np.uint32).reshape(k, 2).copy()
            else:
                pairs = np.zeros((0, 2), np.uint32)
            nr = int(c.n_records)
            if nr and c.records:
                rbuf = (ctypes.c_uint8 * (40 * nr)).from_address(c.records)
                recs = np.frombuffer(rbuf, dtype=np.uint8).copy().view(REC_DTYPE)
            else:
                recs = np.zeros(0, dtype=REC_DTYPE)
            out.append(dict(id=int(c.request_id), status=int(c.status), n_queries=int(c.n_queries),
                            n_candidates=int(c.n_candidates), pass_pairs=pairs, records=recs,
                            size_class=int(c.size_class), t_submit_ns=int(c.t_submit_ns),
                            t_done_ns=int(c.t_done_ns)))
            self.ctx.check(self.lib.pcl_server_release(self.h, c.request_id), "pcl_server_release")
        return out

    def stats(self):
        k = ctypes.c_uint32()
        f = _U64()
        self.ctx.check(self.lib.pcl_server_stats(self.h, ctypes.byref(k), ctypes.byref(f)), "pcl_server_stats")
        return int(k.value), int(f.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.pcl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
