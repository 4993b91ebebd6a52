"""Autotuner for the mixed-batch launch: picks the register DFT radix of the
FFT engine (2 or 4) and the cosine items each warp claims per round (8, 16
32 or 64: the pairs a CTA gates and aligns per round) by timing the candidates
on the batch itself, and remembers the choice in a JSON cache keyed by the
batch's size classes (raster side N, shift half-range S) and mode mix.  The
launch's shared memory fits one persistent CTA per SM, so CTAs per SM are
left at "as many as fit".

The cache lives next to the built library (``_lib/autotune.json``), so it is
per machine and per build.
"""
from __future__ import annotations

import json
import os

from . import Tuning, _build, pcl_match_mixed

CACHE = os.path.join(_build.OUTDIR, "autotune.json")
CANDIDATES = [(radix, items) for radix in (2, 4) for items in (8, 16, 32, 64)]


def _key(params_list, n_cosine: int, n: int) -> str:
    cls = "+".join(f"N{p.window_dbu // p.pitch_dbu}S{p.marker_dbu // p.pitch_dbu}" for p in params_list)
    mix = "cos" if n_cosine == n else ("edge" if n_cosine == 0 else "mixed")
    return f"{cls}|{mix}"


def load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(d: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_mixed(ctx, params_list, sets, work, n_cosine: int, out_rec, reps: int = 3, force: bool = False,
               reset=None) -> tuple[Tuning, dict]:
    """Time every candidate on the batch and return the fastest Tuning and the
    measurements (ms).  ``reset`` (optional callable) restores state that a
    launch changes (e.g. the spectra cache) before each timed launch."""
    import torch
    key = _key(params_list, n_cosine, int(work.shape[0])) + "|items"
    cache = load_cache()
    if not force and key in cache:
        c = cache[key]
        return Tuning(c["fft_radix"], 0, c["items_per_warp"]), c
    times = {}
    for radix, items in CANDIDATES:
        t = Tuning(radix, 0, items)
        best = None
        for _ in range(reps):
            if reset:
                reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pcl_match_mixed(ctx, params_list, sets, work, n_cosine, out_rec, t)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        times[f"r{radix}i{items}"] = best
    radix, items = min(CANDIDATES, key=lambda rc: times[f"r{rc[0]}i{rc[1]}"])
    entry = {"fft_radix": radix, "items_per_warp": items, "ms": times}
    cache[key] = entry
    save_cache(cache)
    return Tuning(radix, 0, items), entry
