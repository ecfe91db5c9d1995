"""Lemma 3 on the GPU (wt_wt2wm_size / _build / wt_wt2wm): the WM position of a
WT position, against the oracle (oracle/lemma3.py) for every level and position
of small texts, on sampled positions of the full-size workloads, and for
out-of-range queries."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_wm, to_u64, torch_text

pytestmark = pytest.mark.gpu

NONE = np.uint64(2**64 - 1)


def _map(T, sigma):
    import paper_1702_07578_gb300 as wtg
    t = torch_text(T)
    bv = wtg.wt_build(t, sigma)
    idx = wtg.WtIndex(wtg.WT_TREE, bv, T.size, sigma)
    return bv, wtg.WtToWmMap(idx)


def _query(m, lv, pos):
    import torch
    dl = torch.from_numpy(lv.astype(np.uint32).view(np.int32)).cuda()
    dp = torch.from_numpy(pos.astype(np.uint64).view(np.int64)).cuda()
    return m(dl, dp).cpu().numpy().view(np.uint64)


def _bits(bv, l, idx):
    w = bv[l][idx >> 6]
    return (w >> (idx & 63).astype(np.uint64)) & np.uint64(1)


@pytest.mark.parametrize("n,sigma,dtype", [(1, 2, np.uint8), (1000, 3, np.uint8), (100003, 16, np.uint8),
                                           (70001, 256, np.uint8), (64 * 300, 256, np.uint8),
                                           (200000, 4096, np.uint16), (50000, 65536, np.uint16),
                                           (30011, 1 << 20, np.uint32), (5000, 1 << 24, np.uint32)])
def test_map_every_position(n, sigma, dtype):
    T = synth.zipf_text(n, sigma, 1.0, 55 + n, dtype) if sigma > 2 else synth.uniform_text(n, 2, 5, dtype)
    L = oracle.levels(sigma)
    bv, m = _map(T, sigma)
    lv = np.repeat(np.arange(L), n)
    pos = np.tile(np.arange(n), L)
    got = _query(m, lv, pos)
    exp = oracle.wt2wm(T, sigma, lv, pos).astype(np.uint64)
    assert np.array_equal(got, exp)
    # the lemma's claim, on the GPU-built WM: the bit at j is the WT's bit at i
    bm, _ = gpu_wm(T, sigma)
    bw = to_u64(bv)
    for l in range(L):
        j = got[l * n:(l + 1) * n].astype(np.int64)
        i = np.arange(n)
        assert np.array_equal(_bits(bw, l, i), _bits(bm, l, j)), l


def test_out_of_range_and_empty():
    T = synth.uniform_text(1000, 16, 3, np.uint8)
    _, m = _map(T, 16)
    got = _query(m, np.array([4, 0, 2, 1]), np.array([3, 1000, 5000, 999]))
    assert got.tolist() == [NONE, NONE, NONE, 999]
    _, m0 = _map(np.zeros(0, np.uint8), 16)
    assert _query(m0, np.array([2, 0]), np.array([0, 0])).tolist() == [NONE, NONE]


@pytest.mark.slow
@pytest.mark.parametrize("which", ["bytes", "large_alphabet"])
def test_map_fullsize_sampled(which):
    """2^30 uint8 (sigma 256) and 2^28 uint32 (sigma 2^20): 2^20 sampled (level, i)."""
    T, sigma = synth.workload_bytes() if which == "bytes" else synth.workload_large_alphabet()
    L = oracle.levels(sigma)
    _, m = _map(T, sigma)
    rng = np.random.default_rng(11)
    lv = rng.integers(0, L, 1 << 20)
    pos = rng.integers(0, T.size, 1 << 20)
    pos[:4] = [0, T.size - 1, 0, T.size - 1]
    lv[:4] = [L - 1, L - 1, 2, 2]
    got = _query(m, lv, pos)
    exp = oracle.wt2wm(T, sigma, lv, pos).astype(np.uint64)
    assert np.array_equal(got, exp)
