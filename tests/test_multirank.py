"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): weak scaling
with one clip set per rank, whole-job figures reduced over ranks, and the
oracle arm printing from rank 0 only."""
import contextlib
import io
import json
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.reduce_over_ranks(100 + rank, 10.0 * (rank + 1), 20.0 - rank, world, "cpu")
    q.put((rank, r))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (201, 20.0, 20.0)


def _reference_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                "--config", "small", "--cpu-sample", "150"]
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    q.put((rank, buf.getvalue()))


@pytest.mark.slow
def test_reference_arm_two_ranks_prints_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_reference_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[1].strip() == ""
    line = json.loads(out[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def _run_ranks(target, world=2, timeout=300):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=timeout) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def _sharded_join_worker(rank, world, port, q):
    """one self-join split over the ranks, the oracle standing in for each
    rank's device: rank r keeps the candidates of shard r, rank 0 gathers"""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle
    import synth
    from paper_2512_13133_gb300 import shard
    wl = synth.preset("small", seed=3, n_clips=300, n_seeds=30, n_copies=180)
    orc = oracle.ClipSet(wl)
    res = {}
    for mode in (shard.MODE_COSINE, shard.MODE_EDGE):
        full, _ = orc.candidates(mode, cos_num=80, edge_tol_dbu=12)
        full = full.astype(np.int64)
        mine = full[shard.pair_shard(full, wl.n, mode, world) == rank]
        got = shard.gather_pairs(mine)
        if rank == 0:
            res[mode] = (len(got), len(full),
                         sorted(map(tuple, got.tolist())) == sorted(map(tuple, full.tolist())))
    q.put((rank, res))
    dist.destroy_process_group()


def test_sharded_self_join_gather_gloo():
    """Shards of one self-join are disjoint and their gather on rank 0 is the
    whole candidate list (both modes)."""
    out = _run_ranks(_sharded_join_worker)
    assert out[1] == {}
    for mode, (n_got, n_full, same) in out[0].items():
        assert n_full > 0 and n_got == n_full and same


def _sharded_serving_worker(rank, world, port, q):
    """a library split by index range: rank 0 broadcasts the query batch,
    each rank matches it against its range (the oracle as its device), rank 0
    gathers the pass pairs with global library indices"""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle
    import synth
    from paper_2512_13133_gb300 import shard
    lib = synth.preset("small", seed=4, n_clips=240, n_seeds=24, n_copies=150)
    lo, hi = shard.library_ranges(lib.n, world)[rank]
    part = lib.subset(np.arange(lo, hi))

    def match_local(rect_off, rects):
        qs = synth.from_lists([rects[rect_off[i]:rect_off[i + 1]].tolist() for i in range(len(rect_off) - 1)],
                              lib.window_dbu, lib.pitch_dbu, lib.marker_dbu)
        both = synth.from_lists([qs.clip(i).tolist() for i in range(qs.n)] +
                                [part.clip(i).tolist() for i in range(part.n)], lib.window_dbu, lib.pitch_dbu,
                                lib.marker_dbu)
        a, b = np.meshgrid(np.arange(qs.n), np.arange(part.n), indexing="ij")
        pairs = np.stack([a.ravel(), qs.n + b.ravel()], 1)
        o = oracle.ClipSet(both).match(pairs, oracle.MODE_EDGE, edge_tol_dbu=12)
        pp = pairs[o["pass_"] == 1]
        return np.stack([pp[:, 0], pp[:, 1] - qs.n], 1) if len(pp) else np.zeros((0, 2), np.int64)

    request = None
    if rank == 0:
        qsrc = lib.subset(np.arange(0, lib.n, 7))  # library clips as queries: each passes against itself
        request = (qsrc.rect_off.astype(np.int64), qsrc.rects.astype(np.int64))
    merged = shard.serve_sharded(request, match_local, lo)
    res = None
    if rank == 0:
        ro, rr = request
        whole = synth.from_lists([rr[ro[i]:ro[i + 1]].tolist() for i in range(len(ro) - 1)] +
                                 [lib.clip(i).tolist() for i in range(lib.n)], lib.window_dbu, lib.pitch_dbu,
                                 lib.marker_dbu)
        nq = len(ro) - 1
        a, b = np.meshgrid(np.arange(nq), np.arange(lib.n), indexing="ij")
        pairs = np.stack([a.ravel(), nq + b.ravel()], 1)
        o = oracle.ClipSet(whole).match(pairs, oracle.MODE_EDGE, edge_tol_dbu=12)
        ref = pairs[o["pass_"] == 1]
        ref = np.stack([ref[:, 0], ref[:, 1] - nq], 1)
        ref = ref[np.lexsort((ref[:, 1], ref[:, 0]))]
        res = (merged.tolist() == ref.tolist(), len(ref), nq)
    q.put((rank, res))
    dist.destroy_process_group()


def test_sharded_serving_broadcast_gather_gloo():
    """Serving with the library split over two ranks returns exactly the pass
    pairs of the whole library."""
    out = _run_ranks(_sharded_serving_worker)
    assert out[1] is None
    same, n_pass, nq = out[0]
    assert same and n_pass >= nq
