"""Serving with one resident library per raster size class (64^2, 128^2,
256^2 and 512^2 px; W = 4N dbu, S = N/16): requests of every class share the
server's slots and memory budget and are in flight together.  Each request's
candidates, pass pairs and per-candidate records equal the oracle's, and equal
what the same request returns when served alone (records field by field,
|sim diff| <= 1e-5).  Cosine classes run the tensor-core engine (64^2, 256^2),
the FFT engine (128^2) and the exact window scan (512^2); edge mode runs every
class through the Min-Max procedure."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIZES = (64, 128, 256, 512)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _library(N, k):
    W = 4 * N
    return synth.generate(40 + N, n_clips=k, n_seeds=k // 10, n_copies=int(0.7 * k), window_dbu=W,
                          margin_dbu=W // 16, min_rects=5, max_rects=40)


def _queries(lib, idx, rng):
    W = lib.window_dbu
    clips = []
    for i in idx:
        r = lib.clip(int(i)).astype(np.int64).copy()
        t = 4 * rng.integers(-2, 3, size=2)
        r[:, [0, 2]] += t[0]
        r[:, [1, 3]] += t[1]
        r = np.clip(r, 0, W)
        r = r[(r[:, 0] < r[:, 2]) & (r[:, 1] < r[:, 3])]
        clips.append(r.tolist())
    return synth.from_lists(clips, W, lib.pitch_dbu, lib.marker_dbu)


def _wait(srv, ids, timeout=120.0):
    got, t0 = {}, time.time()
    while len(got) < len(ids):
        for c in srv.poll():
            got[c["id"]] = c
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.001)
    return got


def _sorted(r):
    return r[np.lexsort((r["b"], r["a"]))]


@pytest.fixture(scope="module")
def classes(torch_cuda):
    import paper_2512_13133_gb300 as pcl
    ctx = pcl.Context(0)
    rng = np.random.default_rng(21)
    libs, reqs = [], []
    for N in SIZES:
        lib = _library(N, 160 if N == 512 else 400)
        libs.append(lib)
        for n in (5, 23):
            reqs.append((len(libs) - 1, _queries(lib, rng.choice(lib.n, n, replace=False), rng)))
    return dict(pcl=pcl, ctx=ctx, libs=libs, reqs=reqs)


@pytest.mark.parametrize("mode", ["cosine", "edge"])
def test_size_classes_served_alone_and_mixed_equal_oracle(classes, mode):
    pcl, ctx, libs, reqs = classes["pcl"], classes["ctx"], classes["libs"], classes["reqs"]
    cosine = mode == "cosine"
    engines = {64: pcl.ENGINE_TC_DIRECT, 128: pcl.ENGINE_FFT_PCM, 256: pcl.ENGINE_TC_DIRECT_BF16,
               512: pcl.ENGINE_FFT_PCM}
    Ps, sets = [], []
    for lib in libs:
        N = lib.raster_n
        P = pcl.params(lib.window_dbu, lib.pitch_dbu, lib.marker_dbu, cos_num=80, edge_tol_dbu=8,
                       cos_engine=engines[N] if cosine else pcl.ENGINE_FFT_PCM)
        cs = pcl.alloc_clipset(P, lib.rect_off, lib.rects, with_spec=cosine and N == 128)
        pcl.pcl_rasterize(ctx, P, cs)
        Ps.append(P)
        sets.append(cs)
    srv = pcl.Server(ctx, Ps, sets, max_inflight=4, max_query_clips=64, cand_per_query=512, mem_budget=1 << 30,
                     mode=pcl.MODE_COSINE if cosine else pcl.MODE_EDGE)
    alone = {}
    for k, (c, q) in enumerate(reqs):
        assert srv.submit(q.rect_off, q.rects, 100 + k, cls=c)
        alone[k] = _wait(srv, [100 + k])[100 + k]
    # all requests, classes interleaved, up to four in flight
    order = [k for pair in zip(range(0, len(reqs), 2), range(1, len(reqs), 2)) for k in pair][::-1]
    pending, ids, got, nid = list(order), {}, {}, 200
    t0 = time.time()
    while pending or len(got) < len(ids):
        while pending:
            c, q = reqs[pending[0]]
            if not srv.submit(q.rect_off, q.rects, nid, cls=c):
                break
            ids[nid] = pending.pop(0)
            nid += 1
        for r in srv.poll():
            got[r["id"]] = r
        assert time.time() - t0 < 120
    srv.close()
    omode = oracle.MODE_COSINE if cosine else oracle.MODE_EDGE
    passes = 0
    for rid, res in got.items():
        k = ids[rid]
        c, q = reqs[k]
        a = alone[k]
        assert res["status"] == a["status"] == 0
        assert res["size_class"] == a["size_class"] == c
        assert res["n_candidates"] == a["n_candidates"] == len(res["records"])
        x, y = _sorted(res["records"]), _sorted(a["records"])
        for f in ("a", "b", "dx_dbu", "dy_dbu", "score", "flags", "pass_", "pcm_dx_dbu", "pcm_dy_dbu"):
            np.testing.assert_array_equal(x[f], y[f], err_msg=f"class {c} field {f}")
        assert np.abs(x["sim"].astype(np.float64) - y["sim"].astype(np.float64)).max(initial=0) <= 1e-5
        # against the oracle: every (query, library) pair of the class
        lib = libs[c]
        both = synth.concat(q, lib)
        pairs = np.array([(i, q.n + j) for i in range(q.n) for j in range(lib.n)], dtype=np.int64)
        o = oracle.ClipSet(both).match(pairs, omode, cos_num=80, edge_tol_dbu=8)
        cand = (o["flags"] & 15) == 0
        assert res["n_candidates"] == int(cand.sum()), f"class {c}"
        opass = {(int(i), int(j) - q.n) for i, j in pairs[o["pass_"] == 1]}
        assert set(map(tuple, res["pass_pairs"].astype(np.int64).tolist())) == opass, f"class {c}"
        oo = o[x["a"].astype(np.int64) * lib.n + x["b"].astype(np.int64)]
        np.testing.assert_array_equal(x["pass_"], oo["pass_"])
        al = (oo["flags"] & oracle.F_ALIGNED) > 0
        for f in ("dx_dbu", "dy_dbu"):
            np.testing.assert_array_equal(x[f][al], oo[f][al], err_msg=f"class {c} {f}")
        np.testing.assert_array_equal(x["score"][al].astype(np.int64), oo["score"][al])
        if cosine:
            assert np.abs(x["sim"][al].astype(np.float64) - oo["sim"][al]).max(initial=0) <= 1e-5
        passes += len(opass)
    assert len(got) == len(reqs)
    assert passes >= sum(q.n for _, q in reqs) // 2
