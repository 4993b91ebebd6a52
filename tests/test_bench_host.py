"""Host logic of bench.py that needs no GPU: the per-result precision report
against the FP64 oracle counts every shift, overlap and decision mismatch it
is given and measures |sim - sim_fp64|, here on records that are the oracle's
own (rounded to FP32) with mistakes planted in known rows."""
import numpy as np

import oracle
import synth


def _same_seed_pairs(wl):
    lab = wl.label
    out = []
    for s in np.unique(lab[lab >= 0]):
        g = np.flatnonzero(lab == s)
        for x in range(len(g)):
            for y in range(x + 1, len(g)):
                out.append((g[x], g[y]))
    return np.array(sorted(out), dtype=np.int64)


def test_precision_report_counts_planted_mismatches():
    import bench
    wl = synth.preset("scale", seed=3, n_clips=400, n_seeds=40, n_copies=280)
    fp = _same_seed_pairs(wl)
    assert 500 < len(fp) < 4000
    o = oracle.ClipSet(wl).match(fp, oracle.MODE_COSINE, use_gates=False, cos_num=bench.COS_NUM,
                                 cos_den=bench.COS_DEN)
    f32 = o.copy()
    f32["sim"] = o["sim"].astype(np.float32).astype(np.float64)
    bad = o.copy()
    bad["dx_dbu"][3] += 4        # a shift
    bad["score"][5] -= 1         # an overlap
    bad["pass_"][7] ^= 1         # a decision
    bad["sim"][9] += 1e-3        # a similarity
    rep = bench.precision_report(wl, fp, {"f32": f32, "bad": bad}, sample=len(fp), near_bit=1 << 4)
    assert rep["sample_pairs"] == len(fp)
    g = rep["f32"]
    assert (g["shift_mismatch"], g["overlap_mismatch"], g["decision_mismatch"]) == (0, 0, 0)
    assert 0 < g["sim_abs_err_max"] < 1e-7
    b = rep["bad"]
    assert (b["shift_mismatch"], b["overlap_mismatch"], b["decision_mismatch"]) == (1, 1, 1)
    assert abs(b["sim_abs_err_max"] - 1e-3) < 1e-9
    # a smaller seeded sample takes whole seed groups and is reproducible
    r1 = bench.precision_report(wl, fp, {"f32": f32}, sample=300, near_bit=1 << 4)
    r2 = bench.precision_report(wl, fp, {"f32": f32}, sample=300, near_bit=1 << 4)
    assert r1["sample_pairs"] == r2["sample_pairs"] == 300 and r1["clips"] == r2["clips"]
