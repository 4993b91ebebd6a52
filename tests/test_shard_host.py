"""Host logic of sharing one problem over several GPUs (no GPU needed): the
partition that pcl_candidates_shard documents, restated in shard.pair_shard,
against a brute-force enumeration of the edge screen's tiles; every pair in
exactly one shard; library ranges that tile the library."""
import numpy as np
import pytest

from paper_2512_13133_gb300 import shard


def _tiles_brute(n):
    """tile index of every (row tile, column block), numbered column block
    after column block, row tiles 0 .. min(8 by + 8, ceil(n/32)) - 1"""
    nbx, nby = (n + 31) // 32, (n + 255) // 256
    idx, t = {}, 0
    for by in range(nby):
        for bx in range(min(8 * by + 8, nbx)):
            idx[(bx, by)] = t
            t += 1
    return idx


@pytest.mark.parametrize("n", [2, 3, 33, 256, 257, 300, 1000, 2600])
def test_edge_tile_numbering_matches_brute_force(n):
    i, j = np.triu_indices(n, 1)
    pairs = np.stack([i, j], 1)
    idx = _tiles_brute(n)
    expect = np.array([idx[(a // 32, b // 256)] for a, b in pairs])
    nbx = (n + 31) // 32
    got = shard._tiles_before(j // 256, nbx) + i // 32
    np.testing.assert_array_equal(got, expect)
    # the shard of a pair does not depend on the order of its clips
    for S in (2, 3, 7):
        np.testing.assert_array_equal(shard.pair_shard(pairs, n, shard.MODE_EDGE, S),
                                      shard.pair_shard(pairs[:, ::-1], n, shard.MODE_EDGE, S))


@pytest.mark.parametrize("mode", [shard.MODE_COSINE, shard.MODE_EDGE])
@pytest.mark.parametrize("S", [1, 2, 3, 5, 8])
def test_every_pair_in_exactly_one_shard(mode, S):
    n = 700
    i, j = np.triu_indices(n, 1)
    s = shard.pair_shard(np.stack([i, j], 1), n, mode, S)
    assert s.min() >= 0 and s.max() < S
    counts = np.bincount(s, minlength=S)
    assert counts.sum() == n * (n - 1) // 2
    if S > 1 and mode == shard.MODE_COSINE:  # min(a, b) mod S: shards within n pairs of each other
        assert counts.max() - counts.min() <= n


def test_library_ranges_tile_the_library():
    for n, w in [(0, 1), (1, 3), (10, 3), (2_000_000, 8)]:
        r = shard.library_ranges(n, w)
        assert len(r) == w and r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert all(hi - lo in (n // w, n // w + 1) for lo, hi in r)
