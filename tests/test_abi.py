"""CPU-side checks of the C ABI: the library loads, exports every entry point
declared in include/pcl.h, validates parameters, and its host set cover and
coarse-to-fine loop agree with the oracle's eager versions."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2512_13133_gb300 as pcl


def test_library_exports_every_declared_symbol():
    lib = pcl.load()
    names = pcl.exported_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_params_validation():
    lib = pcl.load()
    good = pcl.params(512)
    assert lib.pcl_params_validate(ctypes.byref(good)) == pcl.PCL_OK
    for bad in [pcl.params(500), pcl.params(512, pitch_dbu=3), pcl.params(512, marker_dbu=30),
                pcl.params(512, cos_num=100, cos_den=100), pcl.params(512, cos_num=0),
                pcl.params(512, edge_tol_dbu=-1), pcl.params(4096, pitch_dbu=4)]:
        assert lib.pcl_params_validate(ctypes.byref(bad)) == pcl.PCL_ERR_INVALID


def test_clipset_sizes():
    sz = pcl.clipset_sizes(pcl.params(1024, marker_dbu=64), 10)
    assert (sz.N, sz.S, sz.L) == (256, 16, 288)
    assert sz.bits == 10 * 256 * 4 * 8
    assert sz.spec == 10 * 288 * sz.Ls * 8 and sz.Ls >= 145


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert pcl.load().pcl_create(ctypes.byref(h), 0) == pcl.PCL_ERR_INVALID


def _random_graph(rng, n, m):
    e = rng.integers(0, n, size=(m, 2))
    e = e[e[:, 0] != e[:, 1]]
    e = np.unique(np.sort(e, axis=1), axis=0)
    return e


@pytest.mark.parametrize("seed", range(12))
def test_lazy_greedy_equals_eager(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 120))
    e = _random_graph(rng, n, int(rng.integers(0, 4 * n)))
    order, rep = pcl.pcl_setcover(e, n)
    o2, r2 = oracle.setcover_eager(n, e)
    assert order.tolist() == o2
    assert rep.tolist() == r2.tolist()


def test_lazy_greedy_star_and_duplicates():
    # duplicate edges and self loops must not change degrees
    e = np.array([(0, 1), (1, 0), (0, 2), (2, 2), (0, 3)])
    order, rep = pcl.pcl_setcover(e, 5)
    o2, r2 = oracle.setcover_eager(5, [(0, 1), (0, 2), (0, 3)])
    assert order.tolist() == o2 and rep.tolist() == r2.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_cluster_loop_equals_oracle(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(10, 200))
    pairs = _random_graph(rng, n, int(rng.integers(n, 6 * n)))
    relaxed = rng.random(len(pairs)) < 0.7
    strict = relaxed & (rng.random(len(pairs)) < 0.6)
    rep, ncl, rounds = pcl.pcl_cluster_loop(pairs, strict, relaxed, n)
    rep2, ncl2, rounds2 = oracle.cluster_loop(n, pairs, strict, relaxed)
    assert ncl == ncl2 and rounds == rounds2
    assert rep.tolist() == rep2.tolist()
