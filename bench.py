#!/usr/bin/env python3
"""Benchmark: aligned pair-similarities per second of the pairwise
optimal-alignment similarity path on one GB300 (or N of them: a clip set per
rank, or with --scaling strong one clip set whose self-join the ranks split).

A step is one pass of the whole path over one clip set resident in HBM:
rasterisation + signatures, the cosine candidate screen (area band join with
G3/G2 bounds), the edge candidate screen (E2 bbox + E1 correspondence over all
pairs), FFT phase-correlation cosine matching of the cosine candidates
(including the forward FFTs of the clips they reference) and Min-Max matching
of the edge candidates, and the compaction of the pass lists.

  value  = pairs that reached an alignment engine per second (cosine FFT-PCM
           + edge Min-Max), summed over ranks / max step time over ranks
  e2e    = the same through the public API from pinned host rectangles
           (host->device copy of the clip set and device->host read of the
           pass lists inside the timed region)

Workload: the synthetic "scale" clip set (100,000 clips of 1024 x 1024 dbu,
256^2 px at 4 dbu/px, 5-40 rectangles, 70% perturbed copies of 5,000 seeds,
marker +/-64 dbu, cosine 0.95, edge tolerance 4 dbu).  Inputs exceed L2 and
L2 is also flushed between timed steps.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "aligned pair-similarities/sec at oracle-exact decisions"
UNIT = "pairs/s"
COS_NUM, COS_DEN, TOL = 95, 100, 4
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="scale", choices=["scale", "small"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="clips in the oracle sample (0: auto)")
    ap.add_argument("--clips", type=int, default=0,
                    help="override the clip count (seeds and copies scale with it; profiling runs)")
    ap.add_argument("--no-fft-engine", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: each rank its own clip set (weak), or one clip set whose self-join the ranks "
                         "split with pcl_candidates_shard (strong)")
    ap.add_argument("--library-clips", type=int, default=2_000_000,
                    help="clips of the large serving library (tensor-core cosine and edge; 0: skip)")
    ap.add_argument("--class-library-clips", type=int, default=100_000,
                    help="clips of each 64^2, 128^2 and 512^2 px library of the size-class serving measurement")
    ap.add_argument("--topo-clips", type=int, default=1_000_000,
                    help="clips of the topological pre-screen recall measurement (0: skip)")
    ap.add_argument("--no-next", action="store_true", help="skip re-extraction, GPU surprisal and the coarse loop")
    ap.add_argument("--only", default="", choices=["", "edge", "band", "fft", "tc", "exact", "halo", "scan"],
                    help="time one stage alone with only its buffers (single-kernel profiling runs)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--precision-sample", type=int, default=100_000,
                    help="same-seed pairs checked against the FP64 oracle per engine (0: skip)")
    ap.add_argument("--batch-clips", type=int, default=25000, help="clips per size class of the mixed batch")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


# DRAM bytes (read + write) per launch of the kernels on the default scale
# workload, from single-pass ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum) of `bench.py --only edge|band` at 100,000 clips
# and of `bench.py --only fft --clips 10000` (the FFT figure is per pair:
# every pair reads its member's spectrum, so a launch's traffic grows with
# its pairs).  A
# figure counts only while the kernel's sources hash as they did when it was
# taken; otherwise the bench reports null.
TRAFFIC = {
    "cand_edge": {"sources": {"paper_2512_13133_gb300/csrc/edge.cu":
                              "7349ebd251d836e7fc04690f8b35fdd30c83e684cafe58233c1fb6738c3a06b4",
                              "paper_2512_13133_gb300/csrc/edge_dev.cuh":
                              "91b43fe9f14b6cc097d8b42b10055358e7d3ba02c7518a45ff01bacbb54247c7"},
                  # the screen (1.63 GB + 201.62 MB) and its list's check (257.92 + 16.15 MB)
                  "bytes": 1.63e9 + 201.62e6 + 257.92e6 + 16.15e6},
    "cand_cos": {"sources": {"paper_2512_13133_gb300/csrc/gates.cu":
                             "5935883332fb8b84d06ddb62a40a0e119ddaeb97da669f62ebc438834c34e99b",
                             "paper_2512_13133_gb300/csrc/gates.cuh":
                             "7383112e07955c850196dd11d6cdf0d93e2e08c1eab2c834c73868a92928f7d0"},
                 "bytes": 185.34e6 + 4.26e6},
    "fft_pair": {"sources": {"paper_2512_13133_gb300/csrc/fft.cu":
                             "177f4ab710f11721ca4eafa1eb5504eab2340ddff890639dd517e226bbcea14a",
                             "paper_2512_13133_gb300/csrc/fft_dev.cuh":
                             "4d9f3af534542246324fde57ec52870a89fd65b7e26992bfb3de8f32547de133"},
                 "bytes_per_pair": (21.04e9 + 6.18e6) / 56470},
}


def captured_traffic(stage: str, default_workload: bool, pairs: int = 0):
    """per-launch DRAM bytes of a stage's kernel if the capture still applies"""
    import hashlib
    t = TRAFFIC.get(stage)
    if not t or not default_workload:
        return None
    for rel, digest in t["sources"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return t["bytes_per_pair"] * pairs if "bytes_per_pair" in t else t["bytes"]


def alu_peak_tops(sm_mhz: float) -> float:
    # 152 SMs x 128 INT32/FP32 lanes per SM per clock
    return 152 * 128 * sm_mhz * 1e6 / 1e12


def popc_peak_t(sm_mhz: float) -> float:
    # 152 SMs x 16 population counts per SM per clock (a quarter of the
    # 64-lane integer pipe)
    return 152 * 16 * sm_mhz * 1e6 / 1e12


def popc_bound(pairs: int, ms: float, K: int, N: int, done: float = 1.0) -> dict:
    """Popcount view of a window scan: by definition (2S+1)^2 N N/32 popcounts
    of 32-bit words per pair, times the fraction of the window the scan
    counted (done; the 512^2 scan skips groups of shifts by their profile
    bounds); the carry-save sums issue 11 popcounts per 16 words, so this is
    an effective rate of the popcount pipe."""
    per = K * K * N * N / 32
    ach = pairs * per * done / (ms / 1e3) / 1e12
    return {"achieved": ach, "peak": popc_peak_t(2070.0), "unit": "T popc/s", "frac": ach / popc_peak_t(2070.0),
            "work": f"{per:.3g} 32-bit popcounts per pair by definition x {done:.4f} of the window counted",
            "peak_source": "derived: 152 SMs x 16 popcounts x 2.07 GHz"}


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def plain_e1_tests_per_pair(wl, n_sample: int = 20000, seed: int = 0) -> float:
    """Mean number of rectangle-overlap tests the plain E1 procedure (Sec.
    2.2.2 condition 1 as written: every polygon of the smaller clip, in input
    order, against every polygon of the other clip at the pre-alignment, until
    one has a partner count other than 1) spends per random pair of the
    workload.  Used as the algorithmic work of the edge screen."""
    rng = np.random.default_rng(seed)
    W, M = wl.window_dbu, wl.marker_dbu
    off, R = wl.rect_off.astype(np.int64), wl.rects.astype(np.int64)

    def bbox(r, lo, hi):
        v = np.concatenate([r[:, lo][r[:, lo] != 0], r[:, hi][r[:, hi] != W]])
        return (int(v.min()) + int(v.max())) if v.size else None

    tot = 0
    for _ in range(n_sample):
        a, b = (int(v) for v in rng.integers(0, wl.n, 2))
        ra, rb = R[off[a]:off[a + 1]], R[off[b]:off[b + 1]]
        if len(ra) == 0 or len(rb) == 0:
            continue
        s = []
        for lo, hi in ((0, 2), (1, 3)):
            ca, cb = bbox(ra, lo, hi), bbox(rb, lo, hi)
            s.append(0 if ca is None or cb is None else max(-M, min(M, int((ca - cb) / 2))))
        small_a = len(ra) <= len(rb)
        rs, rl = (ra, rb + [s[0], s[1], s[0], s[1]]) if small_a else (rb + [s[0], s[1], s[0], s[1]], ra)
        for p in rs:
            hit = (p[0] < rl[:, 2]) & (rl[:, 0] < p[2]) & (p[1] < rl[:, 3]) & (rl[:, 1] < p[3])
            tot += len(rl)
            if hit.sum() != 1:
                break
    return tot / n_sample


def serving_requests(wl, n_req: int, seed: int = 7, max_clips: int = 4096):
    """Query batches for the serving measurement: batch sizes log-uniform on
    [1, max_clips]; each query clip is a library clip moved by U{-8..8} dbu
    per axis and cut to the window (a new clip with matches in the library)."""
    rng = np.random.default_rng(seed)
    W = wl.window_dbu
    off, R = wl.rect_off.astype(np.int64), wl.rects.astype(np.int64)
    reqs = []
    for _ in range(n_req):
        k = int(np.exp(rng.uniform(0.0, np.log(max_clips))))
        idx = rng.integers(0, wl.n, size=max(k, 1))
        parts, counts = [], []
        for i in idx:
            r = R[off[i]:off[i + 1]].copy()
            t = rng.integers(-8, 9, size=2)
            r[:, [0, 2]] += t[0]
            r[:, [1, 3]] += t[1]
            np.clip(r, 0, W, out=r)
            r = r[(r[:, 0] < r[:, 2]) & (r[:, 1] < r[:, 3])]
            parts.append(r)
            counts.append(len(r))
        ro = np.zeros(len(parts) + 1, np.uint32)
        ro[1:] = np.cumsum(counts)
        reqs.append((ro, np.concatenate(parts).astype(np.int32) if parts else np.zeros((0, 4), np.int32)))
    return reqs


def run_serving(pcl, ctx, P, cs, wl, seconds: float = 2.0, mode: int = 1, cand_per_query: int = 0):
    """Continuous batching against the resident library: a closed-loop burst
    gives the saturation rate, then Poisson arrivals at 50 % and 90 % of it
    give p50/p99 latency (arrival to device completion).  mode: cosine (the
    engine P names behind the area band join: FFT or tensor-core direct
    correlation) or edge (every query x library pair through the edge gates
    and Min-Max).  P, cs and wl may be lists (one resident library per raster
    size class): each request then draws its class uniformly."""
    Ps = list(P) if isinstance(P, (list, tuple)) else [P]
    css = list(cs) if isinstance(cs, (list, tuple)) else [cs]
    wls = list(wl) if isinstance(wl, (list, tuple)) else [wl]
    if not cand_per_query:
        cand_per_query = 64 if mode == pcl.MODE_COSINE else 1024
    srv = pcl.Server(ctx, Ps, css, max_inflight=8, max_query_clips=4096, max_query_rects=4096 * 48,
                     cand_per_query=cand_per_query, mem_budget=24 << 30, mode=mode)
    per_class = [serving_requests(w, 256 // len(wls) or 1, seed=7 + c) for c, w in enumerate(wls)]
    crng = np.random.default_rng(17)
    reqs = [(c, *per_class[c][k % len(per_class[c])])
            for k, c in enumerate(crng.integers(0, len(wls), size=256).tolist())]

    def drive(arrivals):
        """arrivals: monotonic ns per request (None: closed loop)"""
        t0 = time.monotonic_ns()
        queue, done, nxt = [], {}, 0
        arr = {}
        lat, pairs, clips, bad = [], 0, 0, 0
        lat_cls, work_cls = {}, {}
        n_total = len(arrivals) if arrivals is not None else None
        deadline = t0 + int(seconds * 1e9)
        rid = 0
        while True:
            now = time.monotonic_ns()
            if arrivals is None:
                if now < deadline and len(queue) < 8:
                    queue.append((rid, now))
                    rid += 1
            else:
                while nxt < n_total and t0 + arrivals[nxt] <= now:
                    queue.append((nxt, t0 + arrivals[nxt]))
                    nxt += 1
            while queue:
                r, ta = queue[0]
                cl, ro, rr = reqs[r % len(reqs)]
                if not srv.submit(ro, rr, r, cls=cl):
                    break
                arr[r] = ta
                queue.pop(0)
            for c in srv.poll():
                lat.append((c["t_done_ns"] - arr[c["id"]]) / 1e6)
                lat_cls.setdefault(c["size_class"], []).append(lat[-1])
                wk = work_cls.setdefault(c["size_class"], [0, 0])
                wk[0] += c["n_candidates"]
                wk[1] += c["n_queries"]
                pairs += c["n_candidates"]
                clips += c["n_queries"]
                bad += c["status"] != 0  # candidate capacity exceeded (or a device wait ran out)
                done[c["id"]] = c
            if arrivals is None:
                if now >= deadline and not queue and len(done) == rid:
                    break
            elif nxt >= n_total and not queue and len(done) == n_total:
                break
            time.sleep(0.0002)
        wall = (time.monotonic_ns() - t0) / 1e9
        out = dict(requests=len(done), not_ok=bad, wall_s=wall, pairs_per_s=pairs / wall, query_clips_per_s=clips / wall,
                   p50_ms=float(np.percentile(lat, 50)) if lat else None,
                   p99_ms=float(np.percentile(lat, 99)) if lat else None)
        if len(wls) > 1:
            out["per_class"] = {f"{wls[k].raster_n}px": {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                                                         "p99_ms": float(np.percentile(v, 99)),
                                                         "candidates_per_query_clip":
                                                             work_cls[k][0] / max(work_cls[k][1], 1)}
                                for k, v in sorted(lat_cls.items())}
        return out

    drive(None)  # warm-up
    sat = drive(None)
    rps_sat = sat["requests"] / sat["wall_s"]
    rng = np.random.default_rng(3)
    eng = {pcl.ENGINE_FFT_PCM: "fft", pcl.ENGINE_TC_DIRECT: "tc_f16", pcl.ENGINE_TC_DIRECT_BF16: "tc_bf16",
           pcl.ENGINE_TC_DIRECT_FP8: "tc_e4m3"}
    out = {"mode": "cosine" if mode == pcl.MODE_COSINE else "edge",
           "library_clips": wls[0].n if len(wls) == 1 else {f"{w.raster_n}px": w.n for w in wls},
           "engine": (eng.get(Ps[0].cos_engine, "?") if len(wls) == 1 else
                      {f"{w.raster_n}px": ("exact scan" if w.raster_n == 512 else eng.get(p_.cos_engine, "?"))
                       for w, p_ in zip(wls, Ps)}) if mode == pcl.MODE_COSINE else "min-max",
           "batch_clips": "log-uniform 1..4096", "saturation": sat, "poisson": []}
    for frac in (0.5, 0.9):
        lam = frac * rps_sat
        n = max(8, int(lam * seconds))
        gaps = rng.exponential(1.0 / lam, size=n)
        arrivals = (np.cumsum(gaps) * 1e9).astype(np.int64)
        r = drive(arrivals)
        r["lambda_rps"] = lam
        r["load"] = frac
        out["poisson"].append(r)
    srv.close()
    return out


def _precision_worker(job):
    """Oracle records (exact argmax, FP64 similarity) of one shard of the
    precision sample: the shard's clips only, one host thread."""
    sub, local, cos_num, cos_den = job
    import oracle
    o = oracle.ClipSet(sub).match(local, oracle.MODE_COSINE, threads=1, use_gates=False,
                                  cos_num=cos_num, cos_den=cos_den)
    return {f: o[f].copy() for f in ("dx_dbu", "dy_dbu", "score", "sim", "pass_")}


def precision_report(wl, fp, recs_by_engine, sample: int, near_bit: int, seed: int = 5):
    """Per-result error against the FP64 oracle on a seeded sample of the
    same-seed list fp (whole seed groups, so each oracle shard rasterises
    only its own clips): shift, overlap and decision mismatches and the
    distribution of |sim - sim_fp64| for every engine's records of fp."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    rng = np.random.default_rng(seed)
    grp = wl.label[fp[:, 0]].astype(np.int64)
    labels = rng.permutation(np.unique(grp))
    cnt = np.bincount(grp, minlength=int(grp.max()) + 1)
    k = int(np.searchsorted(np.cumsum(cnt[labels]), sample)) + 1
    chosen = np.isin(grp, labels[:k])
    rows = np.flatnonzero(chosen)
    if len(rows) > sample:
        rows = np.sort(rng.choice(rows, sample, replace=False))
    workers = max(1, min(16, os.cpu_count() or 1))
    shards = np.array_split(np.sort(np.unique(grp[rows])), workers)
    jobs, parts = [], []
    for sh in shards:
        r = rows[np.isin(grp[rows], sh)]
        if not len(r):
            continue
        ids = np.unique(fp[r].ravel())
        loc = np.searchsorted(ids, fp[r])
        jobs.append((wl.subset(ids), loc.astype(np.int64), COS_NUM, COS_DEN))
        parts.append(r)
    t0 = time.time()
    # spawned workers (no fork after CUDA initialisation); a worker that dies
    # raises instead of leaving the map waiting
    with ProcessPoolExecutor(len(jobs), mp_context=mp.get_context("spawn")) as pool:
        outs = list(pool.map(_precision_worker, jobs))
    o = {f: np.concatenate([x[f] for x in outs]) for f in outs[0]}
    r = np.concatenate(parts)
    rep = {"sample_pairs": int(len(r)), "clips": int(sum(j[0].n for j in jobs)), "oracle_s": time.time() - t0,
           "oracle_threads": len(jobs)}
    for name, g in recs_by_engine.items():
        g = g[r]
        err = np.abs(g["sim"].astype(np.float64) - o["sim"])
        rep[name] = {"shift_mismatch": int(((g["dx_dbu"] != o["dx_dbu"]) | (g["dy_dbu"] != o["dy_dbu"])).sum()),
                     "overlap_mismatch": int((g["score"].astype(np.int64) != o["score"]).sum()),
                     "decision_mismatch": int((g["pass_"] != o["pass_"]).sum()),
                     "sim_abs_err_max": float(err.max()), "sim_abs_err_mean": float(err.mean()),
                     "sim_abs_err_p99": float(np.percentile(err, 99)),
                     "near_band": int(((g["flags"] & near_bit) > 0).sum())}
    return rep


def run_batched(pcl, ctx, dev, clips_per_class: int, steps: int, seed: int = 1):
    """Mixed batch: four raster sizes (64^2..512^2), truncated-Zipf candidate
    lists, cosine and edge pairs 50/50, all in one persistent launch per step
    (plus the rasterisation of each class and the spectra of referenced
    clips).  Times eager launches and the same step replayed from a captured
    CUDA graph; the launch parameters come from the autotuner."""
    import torch

    import synth
    from paper_2512_13133_gb300 import autotune
    wls, pairs, modes = synth.batched(seed, clips_per_class=clips_per_class)
    # cosine first; within a mode the generator's (class, a) order is kept (a
    # stable partition: linear time at the configured 3.6e8 items)
    order = np.concatenate([np.flatnonzero(modes == 1), np.flatnonzero(modes == 2)])
    pairs, modes = pairs[order], modes[order]
    Ps, sets = [], []
    for wl in wls:
        P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL)
        cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=wl.raster_n <= 256)
        Ps.append(P)
        sets.append(cs)
    work = np.zeros(len(pairs), dtype=pcl.WORK_DTYPE)
    work["cls"], work["a"], work["b"], work["mode"] = pairs[:, 0], pairs[:, 1], pairs[:, 2], modes
    n_cos = int((modes == 1).sum())
    tw = torch.from_numpy(work.view(np.uint8).reshape(-1, 12)).to(dev)
    out = torch.empty((len(pairs), 40), dtype=torch.uint8, device=dev)

    def raster_all():
        for P, cs in zip(Ps, sets):
            pcl.pcl_rasterize(ctx, P, cs)

    raster_all()
    tune, tinfo = autotune.tune_mixed(ctx, Ps, sets, tw, n_cos, out, reset=raster_all)

    def step():
        raster_all()
        pcl.pcl_match_mixed(ctx, Ps, sets, tw, n_cos, out, tune)

    for _ in range(2):
        step()
    torch.cuda.synchronize()

    def timed(fn):
        ms = []
        for _ in range(max(steps, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))

    eager_ms = timed(step)
    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            step()
        torch.cuda.current_stream().wait_stream(cap)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cap, capture_error_mode="thread_local"):
            step()
        g.replay()
        torch.cuda.synchronize()
        graph_ms = timed(g.replay)
    except Exception as exc:  # capture not available: report eager only
        graph_ms = f"capture failed: {exc}"
    rec = pcl.records_to_numpy(out)
    aligned = int(((rec["flags"] & pcl.F_ALIGNED) > 0).sum())
    unsupported = int(((rec["flags"] & 15) == pcl.GATE_UNSUPPORTED).sum())
    best_ms = min(eager_ms, graph_ms) if isinstance(graph_ms, float) else eager_ms
    return {"config": f"batched recipe at {int(sum(w.n for w in wls)):,} clips ({clips_per_class:,} per size class; "
                      "the configured 1,000,000 clips: --batch-clips 250000)",
            "clips": int(sum(w.n for w in wls)), "sizes": [w.raster_n for w in wls], "pairs": int(len(pairs)),
            "cosine_pairs": n_cos, "aligned": aligned, "unsupported": unsupported,
            "ms_eager": eager_ms, "ms_graph": graph_ms, "pairs_per_s": len(pairs) / (best_ms / 1e3),
            "aligned_per_s": aligned / (best_ms / 1e3),
            "tuning": {"fft_radix": int(tune.fft_radix), "items_per_warp": int(tune.items_per_warp),
                       "candidates_ms": tinfo.get("ms")}}


def run_topo(pcl, ctx, dev, clips: int, seed: int):
    """The lossy topological pre-screen (PCL_P_TOPO_HASH: pairs of equal
    polygon count only) against the lossless screens on a scale-recipe set of
    `clips` clips: candidates kept, screen time, and the recall of the
    lossless screen's passing pairs (a pair it passes survives the
    pre-screen iff both clips have the same class, and the alignment engines
    are the same, so the recall needs one matching run).  Edge mode at the
    configured tolerance and at 8 dbu; cosine (tensor-core engine, no
    spectra) at the configured threshold."""
    import torch

    import synth
    k = clips
    wl = synth.preset("scale", seed=seed + 300, n_clips=k, n_seeds=k // 20, n_copies=7 * k // 10)
    cls = np.minimum(np.diff(wl.rect_off.astype(np.int64)), 63)
    out = {"clips": k, "workload": f"scale recipe at {k:,} clips (256^2 px)"}
    P0 = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL, cos_engine=pcl.ENGINE_TC_DIRECT)
    cs = pcl.alloc_clipset(P0, wl.rect_off, wl.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P0, cs)
    torch.cuda.synchronize()

    def timed_cand(P, mode):
        w, _ = pcl.candidates(ctx, P, mode, cs, cap=1 << 20)  # warm-up, gives the exact count
        m = int(w.shape[0])
        del w
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pairs, gates = pcl.candidates(ctx, P, mode, cs, cap=max(m, 1))
        e1.record()
        torch.cuda.synchronize()
        return pairs, gates, e0.elapsed_time(e1)

    dcls = torch.from_numpy(cls).to(dev)

    for name, mode, num, tol in (("edge_tol4", pcl.MODE_EDGE, COS_NUM, TOL), ("edge_tol8", pcl.MODE_EDGE, COS_NUM, 8),
                                 ("cosine_t95", pcl.MODE_COSINE, COS_NUM, TOL)):
        P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, num, COS_DEN, tol, cos_engine=pcl.ENGINE_TC_DIRECT)
        Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, num, COS_DEN, tol, cos_engine=pcl.ENGINE_TC_DIRECT,
                        flags=pcl.P_TOPO_HASH)
        lp, lg, lms = timed_cand(P, mode)
        tp, tg, tms = timed_cand(Pt, mode)
        rec = pcl.match(ctx, P, mode, cs, cs, lp)  # uint8 [m, 40]; the decision is byte 34
        passing = rec[:, 34] > 0
        la, lb = lp[:, 0].long(), lp[:, 1].long()
        n_pass = int(passing.sum().item())
        kept = int((passing & (dcls[la] == dcls[lb])).sum().item())
        out[name] = {"pairs": k * (k - 1) // 2, "lossless_candidates": int(len(lp)), "topo_candidates": int(len(tp)),
                     "lossless_ms": lms, "topo_ms": tms, "topo_rejected": int(tg[pcl.GATE_T0_TOPO]),
                     "passes": n_pass, "passes_kept": kept, "recall": kept / n_pass if n_pass else None,
                     "screened_out_by_topo_frac": float(tg[pcl.GATE_T0_TOPO]) / (k * (k - 1) // 2)}
        del lp, tp, rec
        torch.cuda.empty_cache()
    del cs
    torch.cuda.empty_cache()
    return out


def same_seed_pairs(wl) -> np.ndarray:
    """all pairs (a < b) of clips derived from the same seed, sorted"""
    lab = wl.label
    order = np.argsort(lab, kind="stable")
    ls = lab[order]
    out = []
    for s0 in np.flatnonzero(np.r_[True, ls[1:] != ls[:-1]]):
        if ls[s0] < 0:
            continue
        grp = np.sort(order[s0:s0 + int(np.sum(ls == ls[s0]))])
        i, j = np.triu_indices(len(grp), 1)
        out.append(np.stack([grp[i], grp[j]], 1))
    p = np.concatenate(out) if out else np.zeros((0, 2), np.int64)
    return p[np.lexsort((p[:, 1], p[:, 0]))].astype(np.int32)


def run_next(pcl, ctx, dev, wl, cs, P, steps: int, seed: int):
    """The rows beyond the plain path, measured on the scale recipe:
    re-extraction (the member's window moved at each shift, clips carrying a
    halo of M) on the same-seed pairs of a 100,000-clip set with halo;
    degrees / surprisal / first-step scores of a pass graph on the GPU; the
    coarse-to-fine loop with a low-resolution coarse stage (pitch x 2,
    relaxed thresholds) on the scale set; and the exact window scan that
    aligns 512^2 rasters."""
    import torch

    import synth
    from paper_2512_13133_gb300 import loop

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(max(reps, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))

    out = {}
    # 512^2 rasters: the exact window scan (S = 32) on the same-seed pairs of
    # a 10,000-clip set of the scale recipe at that size, gates off
    w5 = exact512_workload(seed, 10_000)
    P5 = pcl.params(w5.window_dbu, w5.pitch_dbu, w5.marker_dbu, COS_NUM, COS_DEN, TOL, flags=pcl.P_NO_GATES)
    cs5 = pcl.alloc_clipset(P5, w5.rect_off, w5.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, P5, cs5)
    p5 = torch.from_numpy(same_seed_pairs(w5)).to(dev)
    rec5 = torch.empty((p5.shape[0], 40), dtype=torch.uint8, device=dev)
    pcl.pcl_stats_get(ctx, reset=True)
    e_ms = timed(lambda: pcl.pcl_match_pairs(ctx, P5, pcl.MODE_COSINE, cs5, cs5, p5, rec5), steps)
    ev5, tot5 = pcl.pcl_stats_get(ctx, reset=True)  # groups of shifts counted / in the windows
    done5 = ev5 / tot5 if tot5 else 1.0
    K5, NW5 = 2 * cs5.S + 1, cs5.N // 64
    ops5 = 6.0 * K5 * K5 * cs5.N * NW5
    ach5 = p5.shape[0] * ops5 * done5 / (e_ms / 1e3) / 1e12
    out["exact_scan_512"] = {"clips": w5.n, "pairs": int(p5.shape[0]), "ms": e_ms,
                             "pairs_per_s": p5.shape[0] / (e_ms / 1e3),
                             "passes": int(pcl.records_to_numpy(rec5)["pass_"].sum()),
                             "window_counted": done5,
                             "roofline": {"bound": "alu", "achieved": ach5, "peak": alu_peak_tops(2070.0),
                                          "unit": "Tops/s", "frac": ach5 / alu_peak_tops(2070.0),
                                          "work": f"{ops5:.3g} int ops per pair (6 per shift, row and 64-bit word)"
                                                  f" x {done5:.4f} of the window counted"},
                             "popc_bound": popc_bound(int(p5.shape[0]), e_ms, K5, cs5.N, done5)}
    del cs5, p5, rec5
    # re-extraction
    hw = synth.preset("scale", seed=seed + 400, n_clips=wl.n, halo_dbu=wl.marker_dbu)
    Ph = pcl.params(hw.window_dbu, hw.pitch_dbu, hw.marker_dbu, COS_NUM, COS_DEN, TOL)
    hcs = pcl.alloc_clipset(Ph, hw.rect_off, hw.rects, with_spec=False)
    pcl.pcl_rasterize(ctx, Ph, hcs)
    hb, nb = pcl.alloc_halo(Ph, hcs)
    r_ms = timed(lambda: pcl.pcl_rasterize_halo(ctx, Ph, hcs, hb, nb), steps)
    hp = torch.from_numpy(same_seed_pairs(hw)).to(dev)
    hrec = torch.empty((hp.shape[0], 40), dtype=torch.uint8, device=dev)
    pcl.pcl_stats_get(ctx, reset=True, kernel="halo")
    m_ms = timed(lambda: pcl.pcl_match_halo(ctx, Ph, hcs, hcs, hb, nb, hp, hrec), steps)
    hev, htot = pcl.pcl_stats_get(ctx, reset=True, kernel="halo")
    hdone = hev / htot if htot else 1.0
    hr = pcl.records_to_numpy(hrec)
    K, NW = 2 * hcs.S + 1, hcs.N // 64
    ops = 6.0 * K * K * hcs.N * NW  # per pair: funnel shift, AND, popcount, add over every shift and word
    out["reextraction"] = {"clips": hw.n, "halo_dbu": hw.marker_dbu, "pairs": int(hp.shape[0]),
                           "halo_raster_ms": r_ms, "match_ms": m_ms,
                           "pairs_per_s": hp.shape[0] / (m_ms / 1e3), "passes": int(hr["pass_"].sum()),
                           "window_counted": hdone,
                           "roofline": {"bound": "alu", "achieved": hp.shape[0] * ops * hdone / (m_ms / 1e3) / 1e12,
                                        "peak": alu_peak_tops(2070.0), "unit": "Tops/s",
                                        "work": f"{ops:.3g} int ops per pair (6 per shift, row and word)"
                                                f" x {hdone:.4f} of the window counted"}}
    out["reextraction"]["roofline"]["frac"] = out["reextraction"]["roofline"]["achieved"] / alu_peak_tops(2070.0)
    out["reextraction"]["popc_bound"] = popc_bound(int(hp.shape[0]), m_ms, K, hcs.N, hdone)
    del hcs, hb, nb, hp, hrec
    # surprisal of a pass graph: 1,000,000 nodes, 16,000,000 random edges
    rng = np.random.default_rng(seed)
    n_nodes, n_edges = 1_000_000, 16_000_000
    e = torch.from_numpy(rng.integers(0, n_nodes, size=(n_edges, 2)).astype(np.int32)).to(dev)
    s_ms = timed(lambda: pcl.pcl_surprisal(ctx, e, n_nodes), steps)
    out["surprisal"] = {"nodes": n_nodes, "edges": n_edges, "ms": s_ms, "edges_per_s": n_edges / (s_ms / 1e3)}
    del e
    # coarse-to-fine loop, coarse stage at half the resolution
    t0 = time.perf_counter()
    rep, ncl, rounds, info = loop.coarse_to_fine(ctx, P, cs, wl.rect_off, wl.rects, mode=pcl.MODE_COSINE)
    out["coarse_to_fine_cosine"] = {"clips": wl.n, "coarse_pitch_dbu": 2 * wl.pitch_dbu, "clusters": ncl,
                                    "rounds": rounds, "wall_s": time.perf_counter() - t0, **info}
    torch.cuda.empty_cache()
    return out


def exact512_workload(seed: int, clips: int):
    """the scale recipe at 512^2 px (W = 2048 dbu, M = 128 dbu: S = 32)"""
    import synth
    return synth.generate(seed + 712, n_clips=clips, n_seeds=max(1, clips // 20), n_copies=7 * clips // 10,
                          window_dbu=2048, margin_dbu=128, min_rects=5, max_rects=40)


def workload(config: str, seed: int, clips: int = 0, **kw):
    import synth
    if not clips:
        return synth.preset(config, seed=seed, **kw)
    base = synth.PRESETS[config]
    f = clips / base["n_clips"]
    return synth.preset(config, seed=seed, n_clips=clips, n_seeds=max(1, int(base["n_seeds"] * f)),
                        n_copies=int(base["n_copies"] * f), **kw)


# ---------------------------------------------------------------- oracle arm

def cpu_model() -> str:
    """host CPU model name (lscpu, else /proc/cpuinfo, else platform)"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(wl, n_clips: int, threads: int = 0):
    """Time the CPU oracle, as it stands, on the first n_clips clips of the
    workload: rasters + signatures, exhaustive gate screens of both modes,
    brute-force alignment of the survivors.  Returns (aligned pairs, seconds,
    threads)."""
    import oracle
    sub = wl.subset(np.arange(min(n_clips, wl.n)))
    threads = threads or oracle.default_threads()
    t0 = time.perf_counter()
    cs = oracle.ClipSet(sub)
    pc, _ = cs.candidates(oracle.MODE_COSINE, threads=threads)
    pe, _ = cs.candidates(oracle.MODE_EDGE, threads=threads)
    rc = cs.match(pc, oracle.MODE_COSINE, threads=threads)
    re_ = cs.match(pe, oracle.MODE_EDGE, threads=threads)
    dt = time.perf_counter() - t0
    aligned = int(((rc["flags"] & oracle.F_ALIGNED) > 0).sum() + ((re_["flags"] & oracle.F_ALIGNED) > 0).sum())
    return aligned, dt, threads


def default_sample(config: str) -> int:
    return 4000 if config == "scale" else 1000


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload(args.config, args.seed, args.clips)
    n_s = args.cpu_sample or default_sample(args.config)
    for _ in range(args.warmup):
        oracle_sample(wl, n_s)
    tot_a, tot_t, thr = 0, 0.0, 1
    for _ in range(args.steps):
        a, t, thr = oracle_sample(wl, n_s)
        tot_a += a
        tot_t += t
    value = tot_a / tot_t if tot_t > 0 else 0.0
    sample = f"first {n_s} clips of the {args.config} set: all pairs screened, survivors aligned"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
        "data": "synthetic", "config": {"workload": f"{args.config} (oracle sample)", "sample_clips": n_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def reduce_over_ranks(aligned: int, ms_step: float, e2e_ms: float, world: int, device):
    """Whole-job figures: aligned pairs summed over ranks, step and end-to-end
    times maxed over ranks (each rank works on its own clip set, or on its
    shard of one self-join)."""
    if world <= 1:
        return aligned, ms_step, e2e_ms
    import torch
    a = torch.tensor([float(aligned)], dtype=torch.float64, device=device)
    t = torch.tensor([ms_step, e2e_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(a)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return int(a[0].item()), float(t[0].item()), float(t[1].item())

def run_ours(args, rank, world, local_rank):
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2512_13133_gb300 as pcl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    strong = args.scaling == "strong" and world > 1
    wl = workload(args.config, args.seed + (0 if strong else rank), args.clips)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL)
    ctx = pcl.Context(local_rank)
    h_off = torch.from_numpy(wl.rect_off.view(np.int32).copy()).pin_memory()
    h_rects = torch.from_numpy(wl.rects.reshape(-1).copy()).pin_memory()
    d_off = h_off.to(dev)
    d_rects = h_rects.to(dev)
    cs = pcl.alloc_clipset(P, d_off, d_rects)
    cap_c, cap_e = 1 << 22, 1 << 25
    pc = torch.empty((cap_c, 2), dtype=torch.int32, device=dev)
    pe = torch.empty((cap_e, 2), dtype=torch.int32, device=dev)
    rc = torch.empty((cap_c, 40), dtype=torch.uint8, device=dev)
    re_ = torch.empty((cap_e, 40), dtype=torch.uint8, device=dev)
    qc = torch.empty((cap_c, 2), dtype=torch.int32, device=dev)
    qe = torch.empty((cap_e, 2), dtype=torch.int32, device=dev)
    cnt = torch.zeros(4, dtype=torch.int64, device=dev)     # cand cos, cand edge, pass cos, pass edge
    gates = torch.zeros((2, 16), dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stages = ["raster", "cand_cos", "cand_edge", "match_cos", "match_edge", "compact"]

    def cand(mode, out, c, g):
        # strong scaling: this rank's shard of the one self-join
        if strong:
            pcl.pcl_candidates_shard(ctx, P, mode, cs, rank, world, out, c, g)
        else:
            pcl.pcl_candidates(ctx, P, mode, cs, out, c, g)

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record()
        mark(0)
        pcl.pcl_rasterize(ctx, P, cs)
        mark(1)
        cand(pcl.MODE_COSINE, pc, cnt[0:1], gates[0])
        mark(2)
        cand(pcl.MODE_EDGE, pe, cnt[1:2], gates[1])
        mark(3)
        pcl.pcl_match_pairs(ctx, P, pcl.MODE_COSINE, cs, cs, pc, rc, d_n=cnt[0:1])
        mark(4)
        pcl.pcl_match_pairs(ctx, P, pcl.MODE_EDGE, cs, cs, pe, re_, d_n=cnt[1:2])
        mark(5)
        pcl.pcl_compact_pass(ctx, rc, qc, cnt[2:3], d_n=cnt[0:1])
        pcl.pcl_compact_pass(ctx, re_, qe, cnt[3:4], d_n=cnt[1:2])
        mark(6)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    if c[0] > cap_c or c[1] > cap_e:
        raise RuntimeError(f"candidate capacity exceeded: {c[:2]}")
    aligned = int(c[0] + c[1])
    g = (gates.cpu().numpy() // max(args.warmup, 1))
    n = wl.n
    total_pairs = n * (n - 1) // 2

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    st_ms = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(6)] for k in range(args.steps)])
    ms_step = float(st_ms.sum(axis=1).mean())
    per_stage = {s: float(st_ms[:, i].mean()) for i, s in enumerate(stages)}

    # ---- end to end through the public API from pinned host memory, right
    # after the device-timed steps (the same GPU state; measured after the
    # serving and pre-screen sections it ran about 2 % slower)
    e2e = None
    if not args.no_e2e:
        h_cnt = torch.zeros(4, dtype=torch.int64).pin_memory()
        e2e_ms, bi, bo = [], 0, 0
        for k in range(max(args.steps, 1)):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            d_off.copy_(h_off, non_blocking=True)
            d_rects.copy_(h_rects, non_blocking=True)
            step()
            h_cnt.copy_(cnt, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            m_c, m_e = int(h_cnt[2]), int(h_cnt[3])
            out_c = qc[:m_c].cpu()
            out_e = qe[:m_e].cpu()
            e1.record()
            torch.cuda.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
            bi = h_off.numel() * 4 + h_rects.numel() * 4
            bo = 32 + (out_c.numel() + out_e.numel()) * 4
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
               "ms_per_step": float(np.mean(e2e_ms))}

    # ---- a11: the host set cover and coarse-to-fine loop on the last step's
    # records (outside the timed region).  Strict decisions are the records'
    # own; the relaxed ones use the loop's defaults: cosine threshold
    # (num - 2) / den by the integer rule, edge tolerance + 2 dbu.
    host_loop = None
    if rank == 0:
        pops = cs.pop.cpu().numpy().astype(np.int64)
        host_loop = {}
        for name, rec_t, m_k in (("edge", re_, int(c[1])), ("cosine", rc, int(c[0]))):
            r = pcl.records_to_numpy(rec_t[:m_k])
            al = (r["flags"] & pcl.F_ALIGNED) > 0
            if name == "edge":
                relaxed = al & ((r["flags"] & pcl.F_EDGE_VERIFY_FAIL) == 0) & (r["score"].astype(np.int64) <= TOL + 2)
            else:
                cc = r["score"].astype(np.int64)
                pp = pops[r["a"].astype(np.int64)] * pops[r["b"].astype(np.int64)]
                relaxed = al & (COS_DEN ** 2 * cc * cc > (COS_NUM - 2) ** 2 * pp)
            prs = np.stack([r["a"], r["b"]], 1).astype(np.uint32)
            t0 = time.perf_counter()
            _, ncl, nrd = pcl.pcl_cluster_loop(prs, r["pass_"].astype(np.uint8), relaxed.astype(np.uint8), n)
            t1 = time.perf_counter()
            order, _ = pcl.pcl_setcover(prs[relaxed], n)
            t2 = time.perf_counter()
            host_loop[name] = {"pairs": m_k, "relaxed": int(relaxed.sum()), "strict": int(r["pass_"].sum()),
                               "clusters": ncl, "rounds": nrd, "loop_ms": (t1 - t0) * 1e3,
                               "setcover_ms": (t2 - t1) * 1e3, "setcover_selected": int(len(order))}

    # ---- FFT phase-correlation engine on a fixed pair list: the same-seed
    # pairs of the workload (the pairs a looser coarse threshold would send
    # to alignment), gates off, spectra cached beforehand
    fft = None
    if not args.no_fft_engine:
        lab = wl.label
        order = np.argsort(lab, kind="stable")
        ls = lab[order]
        fp = []
        for s0 in np.flatnonzero(np.r_[True, ls[1:] != ls[:-1]]):
            e0 = s0
            while e0 < len(ls) and ls[e0] == ls[s0]:
                e0 += 1
            if ls[s0] < 0:
                continue
            grp = order[s0:e0]
            for x in range(len(grp)):
                for y in range(x + 1, len(grp)):
                    fp.append((min(grp[x], grp[y]), max(grp[x], grp[y])))
        fp = np.array(sorted(fp), dtype=np.int32).reshape(-1, 2)
        Pn = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL, flags=pcl.P_NO_GATES)
        tfp = torch.from_numpy(fp).to(dev)
        rfp = torch.empty((len(fp), 40), dtype=torch.uint8, device=dev)
        pcl.pcl_spectra(ctx, Pn, cs)
        for _ in range(2):
            pcl.pcl_match_pairs(ctx, Pn, pcl.MODE_COSINE, cs, cs, tfp, rfp)
        torch.cuda.synchronize()
        f_ms = []
        for _ in range(max(args.steps, 1)):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            pcl.pcl_match_pairs(ctx, Pn, pcl.MODE_COSINE, cs, cs, tfp, rfp)
            a1.record()
            torch.cuda.synchronize()
            f_ms.append(a0.elapsed_time(a1))
        recs = pcl.records_to_numpy(rfp)
        fms = float(np.mean(f_ms))
        L, Ls = cs.L, cs.Ls
        spec_b = L * Ls * 8
        fft = {"pairs": int(len(fp)), "ms": fms, "pairs_per_s": len(fp) / (fms / 1e3),
               "hbm_gbs_b_spectrum": len(fp) * spec_b / (fms / 1e3) / 1e9,
               "guard_rate": float(((recs["flags"] & pcl.F_FFT_GUARD) > 0).mean()) if len(recs) else 0.0,
               "pcm_agree_rate": float(((recs["flags"] & pcl.F_PCM_AGREES) > 0).mean()) if len(recs) else 0.0,
               "pass": int(recs["pass_"].sum())}
        # the tensor-core direct correlation on the same list and on a dense
        # list (32 members per representative: full items), FP16, BF16 and
        # E4M3 operands (all exact for 0/1 pixels); the roofline denominator is
        # the measured bf16 peak, times 2 for E4M3 (the nominal dense ratio)
        pk, _ = peaks()
        rngd = np.random.default_rng(5)
        reps = rngd.choice(wl.n, 4096, replace=False)
        dense = np.stack([np.repeat(reps, 32), rngd.integers(0, wl.n, 4096 * 32)], 1)
        dense = dense[dense[:, 0] != dense[:, 1]].astype(np.int32)
        # the FFT engine on the dense list too (like for like with the tensor-core rows)
        tdn = torch.from_numpy(np.ascontiguousarray(dense)).to(dev)
        rdn = torch.empty((len(dense), 40), dtype=torch.uint8, device=dev)
        pcl.pcl_match_pairs(ctx, Pn, pcl.MODE_COSINE, cs, cs, tdn, rdn)
        torch.cuda.synchronize()
        d_ms = []
        for _ in range(max(args.steps, 1)):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            pcl.pcl_match_pairs(ctx, Pn, pcl.MODE_COSINE, cs, cs, tdn, rdn)
            a1.record()
            torch.cuda.synchronize()
            d_ms.append(a0.elapsed_time(a1))
        dms = float(np.mean(d_ms))
        fft["dense32"] = {"pairs": int(len(dense)), "ms": dms, "pairs_per_s": len(dense) / (dms / 1e3),
                          "hbm_gbs_b_spectrum": len(dense) * spec_b / (dms / 1e3) / 1e9}
        dense_fft = pcl.records_to_numpy(rdn)
        del tdn, rdn
        tc = {}
        same_seed_recs = {"fft": recs}
        for eng_name, eng, peak_mult in (("f16", pcl.ENGINE_TC_DIRECT, 1.0), ("bf16", pcl.ENGINE_TC_DIRECT_BF16, 1.0),
                                         ("e4m3", pcl.ENGINE_TC_DIRECT_FP8, 2.0)):
            Pt = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL,
                            cos_engine=eng, flags=pcl.P_NO_GATES)
            for name, lst in (("same_seed", fp), ("dense32", dense)):
                tl = torch.from_numpy(np.ascontiguousarray(lst)).to(dev)
                rl = torch.empty((len(lst), 40), dtype=torch.uint8, device=dev)
                pcl.pcl_match_pairs(ctx, Pt, pcl.MODE_COSINE, cs, cs, tl, rl)
                torch.cuda.synchronize()
                t_ms = []
                for _ in range(max(args.steps, 1)):
                    flush.zero_()
                    a0 = torch.cuda.Event(enable_timing=True)
                    a1 = torch.cuda.Event(enable_timing=True)
                    a0.record()
                    pcl.pcl_match_pairs(ctx, Pt, pcl.MODE_COSINE, cs, cs, tl, rl)
                    a1.record()
                    torch.cuda.synchronize()
                    t_ms.append(a0.elapsed_time(a1))
                ms = float(np.mean(t_ms))
                flop = 2.0 * (2 * cs.S + 1) ** 2 * cs.N * cs.N * len(lst)
                key = f"{eng_name}_{name}"
                tc[key] = {"pairs": int(len(lst)), "ms": ms, "pairs_per_s": len(lst) / (ms / 1e3),
                           "tflops_useful": flop / (ms / 1e3) / 1e12,
                           "peak_tflops": pk["bf16_tflops"] * peak_mult,
                           "frac_of_peak": flop / (ms / 1e3) / 1e12 / (pk["bf16_tflops"] * peak_mult)}
                if name == "dense32":
                    rt = pcl.records_to_numpy(rl)
                    tc[key]["agrees_with_fft"] = bool((rt["score"] == dense_fft["score"]).all() and
                                                      (rt["dx_dbu"] == dense_fft["dx_dbu"]).all() and
                                                      (rt["dy_dbu"] == dense_fft["dy_dbu"]).all() and
                                                      (rt["pass_"] == dense_fft["pass_"]).all())
                    tc[key]["speedup_vs_fft"] = fft["dense32"]["ms"] / ms
                if name == "same_seed":
                    tc[key]["speedup_vs_fft"] = fms / ms
                    rt = pcl.records_to_numpy(rl)
                    same_seed_recs[f"tc_{eng_name}"] = rt
                    tc[key]["agrees_with_fft"] = bool((rt["score"] == recs["score"]).all() and
                                                      (rt["dx_dbu"] == recs["dx_dbu"]).all() and
                                                      (rt["dy_dbu"] == recs["dy_dbu"]).all() and
                                                      (rt["pass_"] == recs["pass_"]).all())
        tc["device_error"] = pcl.pcl_device_error(ctx)
        fft["tc_engine"] = tc
        # the bound-pruned exact window scan as a cosine engine (no spectra):
        # both lists, records against the FFT engine's, share of the window counted
        Pe = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL,
                        cos_engine=pcl.ENGINE_EXACT_SCAN, flags=pcl.P_NO_GATES)
        ex = {}
        for name, lst, ref, ref_ms in (("same_seed", fp, recs, fms), ("dense32", dense, dense_fft, dms)):
            tl = torch.from_numpy(np.ascontiguousarray(lst)).to(dev)
            rl = torch.empty((len(lst), 40), dtype=torch.uint8, device=dev)
            pcl.pcl_match_pairs(ctx, Pe, pcl.MODE_COSINE, cs, cs, tl, rl)
            torch.cuda.synchronize()
            pcl.pcl_stats_get(ctx, reset=True)
            x_ms = []
            for _ in range(max(args.steps, 1)):
                flush.zero_()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record()
                pcl.pcl_match_pairs(ctx, Pe, pcl.MODE_COSINE, cs, cs, tl, rl)
                a1.record()
                torch.cuda.synchronize()
                x_ms.append(a0.elapsed_time(a1))
            ev, tot = pcl.pcl_stats_get(ctx, reset=True)
            ms = float(np.mean(x_ms))
            rt = pcl.records_to_numpy(rl)
            ex[name] = {"pairs": int(len(lst)), "ms": ms, "pairs_per_s": len(lst) / (ms / 1e3),
                        "speedup_vs_fft": ref_ms / ms, "window_counted": ev / tot if tot else None,
                        "agrees_with_fft": bool((rt["score"] == ref["score"]).all() and
                                                (rt["dx_dbu"] == ref["dx_dbu"]).all() and
                                                (rt["dy_dbu"] == ref["dy_dbu"]).all() and
                                                (rt["pass_"] == ref["pass_"]).all())}
            del tl, rl
        fft["exact_scan_engine"] = ex
        # per-result error against the FP64 oracle (the precision form's report)
        if args.precision_sample and rank == 0:
            fft["precision_vs_fp64_oracle"] = precision_report(wl, fp.astype(np.int64), same_seed_recs,
                                                               args.precision_sample, pcl.F_NEAR_BAND)
        # the interval-competition shift (Sec. 3.2.1 (2)) on the same list:
        # speed, and what it loses against the exact argmax of the FFT engine
        Px = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL,
                        cos_engine=pcl.ENGINE_XYSEP, flags=pcl.P_NO_GATES)
        rx = torch.empty((len(fp), 40), dtype=torch.uint8, device=dev)
        for _ in range(2):
            pcl.pcl_match_pairs(ctx, Px, pcl.MODE_COSINE, cs, cs, tfp, rx)
        torch.cuda.synchronize()
        x_ms = []
        for _ in range(max(args.steps, 1)):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            pcl.pcl_match_pairs(ctx, Px, pcl.MODE_COSINE, cs, cs, tfp, rx)
            a1.record()
            torch.cuda.synchronize()
            x_ms.append(a0.elapsed_time(a1))
        xr = pcl.records_to_numpy(rx)
        xms = float(np.mean(x_ms))
        same_shift = (xr["dx_dbu"] == recs["dx_dbu"]) & (xr["dy_dbu"] == recs["dy_dbu"])
        fft["xysep_engine"] = {
            "pairs": int(len(fp)), "ms": xms, "pairs_per_s": len(fp) / (xms / 1e3),
            "speedup_vs_fft": fms / xms,
            "same_shift_as_exact": float(same_shift.mean()),
            "same_overlap_as_exact": float((xr["score"] == recs["score"]).mean()),
            "passes": int(xr["pass_"].sum()), "passes_exact": int(recs["pass_"].sum()),
            "passes_lost": int(((recs["pass_"] == 1) & (xr["pass_"] == 0)).sum()),
            "mean_sim_loss": float((recs["sim"].astype(np.float64) - xr["sim"].astype(np.float64)).mean()),
            "never_above_exact": bool((xr["score"] <= recs["score"]).all())}
        # spectra are per-step work of the main path again
        pcl.pcl_rasterize(ctx, P, cs)
        torch.cuda.synchronize()

    # ---- serving: continuous batching of query requests against the clip set
    # as a resident library (p50/p99 latency beside throughput)
    serving = serving_edge = serving_tc = serving_large = serving_classes = None
    if not args.no_serving and world == 1:
        pcl.pcl_rasterize(ctx, P, cs)
        serving = run_serving(pcl, ctx, P, cs, wl)
        serving_edge = run_serving(pcl, ctx, P, cs, wl, mode=pcl.MODE_EDGE)
        # the same library and requests on the tensor-core engine (no spectra)
        Ptc = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL,
                         cos_engine=pcl.ENGINE_TC_DIRECT)
        serving_tc = run_serving(pcl, ctx, Ptc, cs, wl)
        # the serving form's size mix: one resident library per raster size
        # class (64^2, 128^2 and 512^2 px sub-libraries of the scale recipe at
        # their size, W = 4N, S = N/16; the 256^2 class is this clip set),
        # requests drawing their class uniformly; cosine on the FFT engine
        # (spectra resident; the exact window scan at 512^2), and edge mode
        if args.config == "scale":
            import synth
            sub_w, sub_P, sub_cs = [], [], []
            for N in (64, 128, 256, 512):
                if N == 256:
                    w_, cs_ = wl, cs
                else:
                    k = args.class_library_clips
                    w_ = synth.generate(args.seed + 200 + N, n_clips=k, n_seeds=k // 20, n_copies=7 * k // 10,
                                        window_dbu=4 * N, margin_dbu=N // 4, min_rects=5, max_rects=40)
                    cs_ = None
                p_ = pcl.params(w_.window_dbu, w_.pitch_dbu, w_.marker_dbu, COS_NUM, COS_DEN, TOL)
                if cs_ is None:
                    cs_ = pcl.alloc_clipset(p_, w_.rect_off, w_.rects, with_spec=N < 512)
                pcl.pcl_rasterize(ctx, p_, cs_)
                sub_w.append(w_)
                sub_P.append(p_)
                sub_cs.append(cs_)
            serving_classes = {"cosine": run_serving(pcl, ctx, sub_P, sub_cs, sub_w),
                               "edge": run_serving(pcl, ctx, [pcl.params(w_.window_dbu, w_.pitch_dbu, w_.marker_dbu,
                                                                         COS_NUM, COS_DEN, TOL) for w_ in sub_w],
                                                   sub_cs, sub_w, mode=pcl.MODE_EDGE)}
            del sub_cs
            torch.cuda.empty_cache()
        if args.library_clips and args.config == "scale":
            # a resident library of the serving form's size: rasters and
            # signatures only (the tensor-core and exact-scan engines need no
            # spectra)
            import synth
            t0 = time.time()
            k = args.library_clips
            lib = synth.preset("scale", seed=args.seed + 100, n_clips=k, n_seeds=k // 20, n_copies=7 * k // 10)
            cs_lib = pcl.alloc_clipset(Ptc, lib.rect_off, lib.rects, with_spec=False)
            pcl.pcl_rasterize(ctx, Ptc, cs_lib)
            torch.cuda.synchronize()
            serving_large = {"library_clips": k, "library_device_gb": sum(
                t.numel() * t.element_size() for t in (cs_lib.rect_off, cs_lib.rects, cs_lib.bits, cs_lib.pop,
                                                       cs_lib.prof, cs_lib.blk, cs_lib.esig, cs_lib.occ,
                                                       cs_lib.rorder)) / 1e9,
                             "setup_s": time.time() - t0,
                             "cosine": run_serving(pcl, ctx, Ptc, cs_lib, lib, cand_per_query=256),
                             "cosine_exact_scan": run_serving(
                                 pcl, ctx, pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN,
                                                      TOL, cos_engine=pcl.ENGINE_EXACT_SCAN),
                                 cs_lib, lib, cand_per_query=256),
                             "edge": run_serving(pcl, ctx, P, cs_lib, lib, mode=pcl.MODE_EDGE,
                                                 cand_per_query=8192)}
            del cs_lib, lib
            torch.cuda.empty_cache()
        pcl.pcl_rasterize(ctx, P, cs)
        torch.cuda.synchronize()

    # ---- mixed batch: four raster sizes, Zipf candidate lists, both modes in
    # one persistent launch, eager and CUDA-graph replay
    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(pcl, ctx, dev, args.batch_clips, args.steps)
        torch.cuda.synchronize()

    # ---- the rows beyond the plain path (re-extraction, GPU surprisal,
    # low-resolution coarse stage)
    nxt = None
    if not args.no_next and world == 1 and args.config == "scale":
        pcl.pcl_rasterize(ctx, P, cs)
        nxt = run_next(pcl, ctx, dev, wl, cs, P, args.steps, args.seed)
        pcl.pcl_rasterize(ctx, P, cs)
        torch.cuda.synchronize()

    # ---- the lossy topological pre-screen against the lossless screens
    topo = None
    if args.topo_clips and world == 1:
        topo = run_topo(pcl, ctx, dev, args.topo_clips, args.seed)
        torch.cuda.synchronize()


    # ---- reduce over ranks
    tot_aligned, ms_max, e2e_max = reduce_over_ranks(aligned, ms_step, e2e["ms_per_step"] if e2e else 0.0,
                                                     world, dev)
    if rank != 0:
        return
    value = tot_aligned / (ms_max / 1e3)
    if e2e:
        e2e["value"] = tot_aligned / (e2e_max / 1e3)
        e2e["ms_per_step"] = e2e_max

    # ---- roofline of the dominant stage
    pk, pk_kind = peaks()
    dom = max(per_stage, key=per_stage.get)
    N, nb = cs.N, cs.N // 16
    sm_mhz = clk.get("sm_mhz") or 2070.0
    if dom == "raster":
        byts = n * (N * N / 8 + 4 + 4 * N + 4 * nb * nb + 32) + wl.rects.nbytes + wl.rect_off.nbytes
        ach = byts / (per_stage[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    elif dom == "cand_cos":
        band = int(g[0][0] + g[0][2] + g[0][3])
        ops = band * 4 * nb * nb
        ach = ops / (per_stage[dom] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak_tops(2070.0), "unit": "Tops/s"}
    elif dom == "cand_edge":
        # algorithmic work: the plain E1 procedure's overlap tests (8 integer
        # ops each: four compares, three ANDs, one count) plus 20 ops of
        # pre-alignment per pair; the kernel reaches the same decisions with
        # an occupancy-grid pre-check, so this is an effective rate
        tpp = plain_e1_tests_per_pair(wl)
        ops = total_pairs * (20 + 8 * tpp)
        ach = ops / (per_stage[dom] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak_tops(2070.0), "unit": "Tops/s",
                "work": f"{20 + 8 * tpp:.0f} int ops/pair (plain E1: {tpp:.1f} overlap tests/pair)"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": alu_peak_tops(2070.0), "unit": "Tops/s"}
    roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("achieved") else None
    roof["traffic"] = captured_traffic(dom, args.config == "scale" and not args.clips)
    roof["kernel"] = dom
    roof["peak_source"] = pk_kind

    # rooflines of the other stages and of the correlation engines, each
    # against its own bound (algorithmic work per launch / CUDA-event time)
    def frac(r):
        r["frac"] = r["achieved"] / r["peak"] if r.get("achieved") else None
        r["peak_source"] = pk_kind if r["unit"] != "Tops/s" else "derived: 152 SMs x 128 lanes x 2.07 GHz"
        return r

    rooflines = {}
    byts = n * (N * N / 8 + 4 + 4 * N + 4 * nb * nb + 32) + wl.rects.nbytes + wl.rect_off.nbytes
    rooflines["raster"] = frac({"bound": "hbm", "achieved": byts / (per_stage["raster"] / 1e3) / 1e9,
                                "peak": pk["hbm_gbs"], "unit": "GB/s",
                                "work": "N^2/8 + 4N + 4 nb^2 + 36 B written per clip + rectangles read"})
    band = int(g[0][0] + g[0][2] + g[0][3])
    rooflines["cand_cos"] = frac({"bound": "alu", "achieved": band * 4 * nb * nb / (per_stage["cand_cos"] / 1e3) / 1e12,
                                  "peak": alu_peak_tops(2070.0), "unit": "Tops/s",
                                  "work": f"{band} band pairs (G1 survivors) x 4 nb^2 integer ops (G3 both ways)",
                                  "traffic": captured_traffic("cand_cos", args.config == "scale" and not args.clips)})
    if dom == "cand_edge":
        rooflines["cand_edge"] = dict(roof)
    if fft:
        L, Ls = cs.L, cs.Ls
        rooflines["fft_pair"] = frac({"bound": "hbm", "achieved": fft["hbm_gbs_b_spectrum"], "peak": pk["hbm_gbs"],
                                      "unit": "GB/s",
                                      "work": f"B's spectrum per pair ({L * Ls * 8} B; A's from L2, the list sorted by "
                                              f"representative), {fft['pairs']} same-seed pairs",
                                      "traffic": captured_traffic("fft_pair", args.config == "scale" and not args.clips,
                                                                  fft["pairs"])})
        tcd = fft.get("tc_engine", {})
        for key in ("f16_dense32", "bf16_dense32", "f16_same_seed", "bf16_same_seed"):
            if key in tcd:
                t = tcd[key]
                rooflines[f"tc_corr_{key}"] = frac({"bound": "tensor", "achieved": t["tflops_useful"],
                                                    "peak": t["peak_tflops"], "unit": "TFLOP/s",
                                                    "work": "2 (2S+1)^2 N^2 useful FLOP per pair (bf16 burst peak)"})

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": args.scaling,
        "vs_baseline": None, "dtype": "u64/i32/f32", "data": "synthetic",
        "config": {"workload": f"{args.config}: {n} clips, {N}x{N} px, W={wl.window_dbu} dbu, "
                               f"M={wl.marker_dbu} dbu, T=0.95, tol=4 dbu, both modes",
                   "l2": "inputs > L2 and 512 MB flush between timed steps",
                   "pairs_screened": total_pairs, "aligned_cosine": int(c[0]), "aligned_edge": int(c[1]),
                   "passed_cosine": int(c[2]), "passed_edge": int(c[3]),
                   "gates_cosine": {"G1": int(g[0][1]), "G3": int(g[0][3]), "G2": int(g[0][2])},
                   "gates_edge": {"E2": int(g[1][5]), "E1": int(g[1][4])},
                   "stage_ms": per_stage, "screened_pairs_per_s": 2 * total_pairs * world / (ms_max / 1e3),
                   "wall_s_timed": wall},
        "roofline": roof, "rooflines": rooflines, "clocks": clk, "e2e": e2e, "gpu_launches": None, "fft_engine": fft,
        "host_loop": host_loop,
        "serving": serving,
        "serving_edge": serving_edge,
        "serving_tc": serving_tc,
        "serving_large_library": serving_large,
        "serving_size_classes": serving_classes,
        "batched": batched,
        "topo_prescreen": topo,
        "next": nxt,
    }
    # kernels launched per step: raster 1, band join 5, edge screen 2 (the screen and the
    # correspondence check of its list), cosine match 4 (mark, two spectra sweeps counted
    # once for a self-join, pair) -> 3, edge match 1, compact 2
    line["gpu_launches"] = args.steps * (1 + 5 + 2 + 3 + 1 + 2)
    if not args.no_cpu_baseline and world == 1:
        n_s = args.cpu_sample or default_sample(args.config)
        a, t, thr = oracle_sample(wl, n_s)
        n_1 = max(2, n_s // 4)  # single thread: a quarter of the clips (1/16 of the pairs)
        a1, t1, _ = oracle_sample(wl, n_1, threads=1)
        line["cpu_baseline"] = {"value": a / t, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "cpu_model": cpu_model(),
                                "sample": f"first {n_s} clips of the {args.config} set ({n_s*(n_s-1)//2} pairs "
                                          f"screened both modes, {a} aligned), {t:.1f} s on {thr} threads",
                                "single_thread": {"value": a1 / t1, "unit": UNIT, "cores": 1,
                                                  "sample": f"first {n_1} clips ({n_1*(n_1-1)//2} pairs screened "
                                                            f"both modes, {a1} aligned), {t1:.1f} s"}}
    print(json.dumps(line), flush=True)


def run_only(args):
    """One stage alone on the workload, with only the device buffers it needs
    (the command ncu captures of a single kernel run): edge screen, cosine
    band join, FFT engine on the same-seed list, the tensor-core engine
    (FP16) on the dense 32-member list, the exact window scan of 512^2
    rasters on the same-seed list of a 10,000-clip set (gates off), the
    exact-scan engine on the same-seed list of the workload (gates off), or
    re-extraction on the same-seed list of a set with halo.  Prints one JSON
    line with the mean CUDA-event time of the timed launches."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import synth
    import paper_2512_13133_gb300 as pcl
    dev = torch.device("cuda", 0)
    if args.only == "exact":
        wl = exact512_workload(args.seed, args.clips or 10_000)
    elif args.only == "halo":
        wl = workload(args.config, args.seed + 400, args.clips, halo_dbu=synth.PRESETS[args.config]["margin_dbu"])
    else:
        wl = workload(args.config, args.seed, args.clips)
    eng = {"tc": pcl.ENGINE_TC_DIRECT, "scan": pcl.ENGINE_EXACT_SCAN}.get(args.only, pcl.ENGINE_FFT_PCM)
    P = pcl.params(wl.window_dbu, wl.pitch_dbu, wl.marker_dbu, COS_NUM, COS_DEN, TOL, cos_engine=eng,
                   flags=pcl.P_NO_GATES if args.only in ("fft", "tc", "exact", "scan") else 0)
    ctx = pcl.Context(0)
    cs = pcl.alloc_clipset(P, wl.rect_off, wl.rects, with_spec=args.only == "fft")
    pcl.pcl_rasterize(ctx, P, cs)
    n = wl.n
    if args.only in ("edge", "band"):
        mode = pcl.MODE_EDGE if args.only == "edge" else pcl.MODE_COSINE
        out = torch.empty((1 << 24, 2), dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        fn = lambda: pcl.pcl_candidates(ctx, P, mode, cs, out, cnt)  # noqa: E731
        units, unit = n * (n - 1) // 2, "pairs screened"
    else:
        if args.only == "fft":
            pcl.pcl_spectra(ctx, P, cs)
            lst = same_seed_pairs(wl)
        elif args.only in ("exact", "halo", "scan"):
            lst = same_seed_pairs(wl)
        else:
            rng = np.random.default_rng(5)
            reps = rng.choice(n, min(4096, n), replace=False)
            lst = np.stack([np.repeat(reps, 32), rng.integers(0, n, len(reps) * 32)], 1)
            lst = lst[lst[:, 0] != lst[:, 1]].astype(np.int32)
        tl = torch.from_numpy(np.ascontiguousarray(lst)).to(dev)
        rec = torch.empty((len(lst), 40), dtype=torch.uint8, device=dev)
        if args.only == "halo":
            hb, nb = pcl.alloc_halo(P, cs)
            pcl.pcl_rasterize_halo(ctx, P, cs, hb, nb)
            fn = lambda: pcl.pcl_match_halo(ctx, P, cs, cs, hb, nb, tl, rec)  # noqa: E731
        else:
            fn = lambda: pcl.pcl_match_pairs(ctx, P, pcl.MODE_COSINE, cs, cs, tl, rec)  # noqa: E731
        units, unit = len(lst), "pairs aligned"
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    line = {"only": args.only, "clips": n, "units": units, "unit": unit, "ms": float(np.mean(ms)),
            "per_s": units / (float(np.mean(ms)) / 1e3)}
    if args.only in ("edge", "band"):
        line["candidates"] = int(cnt.item())
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.only:
        run_only(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
