"""Host side of running the path on several GPUs (one process per GPU, ranks
of a torch.distributed group).  Two ways to share work, neither with a
device collective:

* one self-join split over the ranks: every rank holds the whole clip set and
  screens shard `rank` of `world` of the pair space (pcl_candidates_shard);
  the candidate lists (or pass lists) of the ranks are disjoint and together
  equal the single-GPU result, so gathering them on rank 0 for the host set
  cover is the only exchange;
* a served library split by index range: each rank keeps clips
  [lo_r, hi_r) resident (ClipSet.view, no copy), rank 0 broadcasts each query
  batch, every rank matches it against its range, and rank 0 gathers the pass
  pairs with library indices shifted by lo_r.

The exchanges go through torch.distributed object collectives, so they run
over gloo (host TCP) as well as over NCCL groups.  pair_shard states the
partition pcl_candidates_shard uses, for checking and for host code that
must know which rank owns a pair.
"""
from __future__ import annotations

import numpy as np

MODE_COSINE = 1
MODE_EDGE = 2

# the edge screen's tile: 32 row clips i x 256 column clips j (i < j)
_ROWS, _COLS = 32, 256


def _tiles_before(by: np.ndarray, nbx: int) -> np.ndarray:
    """tiles numbered before column block `by` (row tiles 0 .. min(8 by + 8,
    nbx) - 1 per block, only those that hold a pair i < j)"""
    by = np.asarray(by, dtype=np.int64)
    y0 = nbx // 8
    head = 4 * by * (by + 1)
    tail = 4 * y0 * (y0 + 1) + (by - y0) * nbx
    return np.where(by <= y0, head, tail)


def pair_shard(pairs, n: int, mode: int, n_shards: int) -> np.ndarray:
    """Shard (0 .. n_shards - 1) that owns each pair (a, b), a != b, of a
    self-join of n clips, as pcl_candidates_shard partitions them: COSINE by
    min(a, b) mod S, EDGE by the screen tile of (min, max) modulo S."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if n_shards == 1:
        return np.zeros(len(p), np.int64)
    if mode == MODE_COSINE:
        return p.min(axis=1) % n_shards
    if mode != MODE_EDGE:
        raise ValueError("mode must be COSINE or EDGE")
    i, j = p.min(axis=1), p.max(axis=1)
    nbx = (n + _ROWS - 1) // _ROWS
    tile = _tiles_before(j // _COLS, nbx) + i // _ROWS
    return tile % n_shards


def library_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """contiguous clip ranges [lo, hi) of a library split over `world` ranks"""
    cut = [n * r // world for r in range(world + 1)]
    return [(cut[r], cut[r + 1]) for r in range(world)]


def gather_pairs(local: np.ndarray, offset_b: int = 0, dst: int = 0):
    """Concatenate every rank's (a, b) pairs on rank `dst` (b shifted by the
    rank's offset_b); other ranks get None."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    mine = np.asarray(local, dtype=np.int64).reshape(-1, 2).copy()
    mine[:, 1] += offset_b
    got = [None] * world if rank == dst else None
    dist.gather_object(mine, got, dst=dst)
    if rank != dst:
        return None
    return np.concatenate(got) if got else np.zeros((0, 2), np.int64)


def serve_sharded(request, match_local, lib_lo: int, src: int = 0):
    """One query batch against a library split by index range.  `request`
    (rect_off, rects) is read on rank `src` and broadcast; match_local(rect_off,
    rects) -> (query, local library index) pass pairs on every rank; returns
    the merged pass pairs (library indices global, sorted) on rank `src`,
    None elsewhere."""
    import torch.distributed as dist
    box = [request if dist.get_rank() == src else None]
    dist.broadcast_object_list(box, src=src)
    rect_off, rects = box[0]
    mine = match_local(rect_off, rects)
    allp = gather_pairs(mine, lib_lo, dst=src)
    if allp is None:
        return None
    return allp[np.lexsort((allp[:, 1], allp[:, 0]))]
