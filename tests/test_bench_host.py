"""Host logic of bench.py that needs no GPU: the per-result precision report
against the FP64 oracle counts every shift, overlap and decision mismatch it
is given and measures |sim - sim_fp64|, here on records that are the oracle's
own (rounded to FP32) with mistakes planted in known rows; the DRAM figures
count only for the sources they were captured on; the derived ALU peak."""
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


def test_captured_traffic_applies_only_to_the_captured_sources(tmp_path, monkeypatch):
    """A DRAM figure counts while its kernel's sources hash as at the capture,
    and only on the default workload; per-pair figures scale with the pairs."""
    import hashlib

    import bench
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {
        "whole": {"sources": {"k.cu": digest}, "bytes": 1.5e9},
        "per_pair": {"sources": {"k.cu": digest}, "bytes_per_pair": 1000.0},
        "missing": {"sources": {"gone.cu": digest}, "bytes": 1.0},
    })
    assert bench.captured_traffic("whole", True) == 1.5e9
    assert bench.captured_traffic("per_pair", True, pairs=7) == 7000.0
    assert bench.captured_traffic("whole", False) is None       # another workload
    assert bench.captured_traffic("missing", True) is None      # source not there
    assert bench.captured_traffic("unknown", True) is None
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.captured_traffic("whole", True) is None        # changed since the capture


def test_committed_traffic_figures_name_existing_sources():
    """Every DRAM figure the bench carries names sources of this repository,
    with sha256 digests and a positive byte count."""
    import os

    import bench
    for stage, t in bench.TRAFFIC.items():
        assert t["sources"], stage
        for rel, digest in t["sources"].items():
            assert os.path.exists(os.path.join(bench.ROOT, rel)), (stage, rel)
            assert len(digest) == 64 and int(digest, 16) >= 0
        v = t.get("bytes", t.get("bytes_per_pair"))
        assert v is not None and v > 0


def test_alu_peak_is_the_lane_count_times_the_clock():
    import bench
    # 152 SMs x 128 INT32 lanes at 2.07 GHz
    assert abs(bench.alu_peak_tops(2070.0) - 152 * 128 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.alu_peak_tops(2070.0) - 40.27392) < 1e-6
