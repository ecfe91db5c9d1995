"""access / rank / select on built WT and WM (GPU) against direct counting on T."""
import numpy as np
import pytest

import synth
from tests.gpu_util import torch_text

pytestmark = pytest.mark.gpu

NONE = np.uint64(2**64 - 1)


def _brute(T, sigma, pos, sym, jj):
    """access = T[i]; rank = count of c in T[:i]; select = position of j-th c."""
    T64 = T.astype(np.int64)
    acc = T64[np.minimum(pos, T.size - 1)]
    rank = np.empty(len(sym), np.uint64)
    sel = np.empty(len(sym), np.uint64)
    cache = {}
    for k, (c, i, j) in enumerate(zip(sym.tolist(), pos.tolist(), jj.tolist())):
        if c not in cache:
            cache[c] = np.flatnonzero(T64 == c)
        occ = cache[c]
        rank[k] = np.searchsorted(occ, i, side="left")
        sel[k] = occ[j - 1] if 1 <= j <= occ.size else NONE
    return acc, rank, sel


@pytest.mark.parametrize("kind", ["wt", "wm"])
@pytest.mark.parametrize("n,sigma,dtype", [(1, 2, np.uint8), (1000, 2, np.uint8), (70001, 256, np.uint8),
                                           (200003, 13, np.uint8), (100000, 4096, np.uint16),
                                           (50000, 1 << 20, np.uint32), (64 * 300, 256, np.uint8)])
def test_queries_match_brute_force(kind, n, sigma, dtype):
    import torch

    import paper_1702_07578_gb300 as wtg
    T = synth.zipf_text(n, sigma, 1.0, 31 + n, dtype) if sigma > 2 else synth.uniform_text(n, 2, 7, dtype)
    t = torch_text(T)
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    if kind == "wt":
        bv, z = wtg.wt_build(t, sigma), None
    else:
        bv, z = wtg.wm_build(t, sigma)
    idx = wtg.WtIndex(k, bv, n, sigma, z)
    rng = np.random.default_rng(n)
    q = 3000
    pos = rng.integers(0, n, size=q).astype(np.uint64)
    sym = T[rng.integers(0, n, size=q)].astype(np.uint32)
    sym[::7] = rng.integers(0, sigma, size=len(sym[::7]))          # some absent symbols
    rpos = rng.integers(0, n + 1, size=q).astype(np.uint64)
    jj = rng.integers(1, max(2, n // max(1, min(sigma, 64))), size=q).astype(np.uint64)
    acc, rank, sel = _brute(T, sigma, pos, sym, jj)
    _, rank, _ = _brute(T, sigma, rpos, sym, jj)
    dpos = torch.from_numpy(pos.view(np.int64)).cuda()
    drpos = torch.from_numpy(rpos.view(np.int64)).cuda()
    dsym = torch.from_numpy(sym.view(np.int32)).cuda()
    dj = torch.from_numpy(jj.view(np.int64)).cuda()
    got_acc = idx.access(dpos).cpu().numpy().view(np.uint32)
    got_rank = idx.rank(dsym, drpos).cpu().numpy().view(np.uint64)
    got_sel = idx.select(dsym, dj).cpu().numpy().view(np.uint64)
    assert np.array_equal(got_acc, T.astype(np.uint32)[pos.astype(np.int64)])
    assert np.array_equal(got_rank, rank)
    assert np.array_equal(got_sel, sel)


def test_out_of_range_queries():
    import torch

    import paper_1702_07578_gb300 as wtg
    T = synth.uniform_text(1000, 16, 3, np.uint8)
    t = torch_text(T)
    bv, z = wtg.wm_build(t, 16)
    idx = wtg.WtIndex(wtg.WT_MATRIX, bv, 1000, 16, z)
    pos = torch.tensor([1000, 5000], dtype=torch.int64, device="cuda")
    assert idx.access(pos).cpu().numpy().view(np.uint32).tolist() == [0xFFFFFFFF] * 2
    sym = torch.tensor([16, 3], dtype=torch.int32, device="cuda")
    r = idx.rank(sym, torch.tensor([10, 1001], dtype=torch.int64, device="cuda"))
    assert r.cpu().numpy().view(np.uint64).tolist() == [2**64 - 1] * 2
    s = idx.select(sym, torch.tensor([1, 0], dtype=torch.int64, device="cuda"))
    assert s.cpu().numpy().view(np.uint64).tolist() == [2**64 - 1] * 2


def test_matrix_queries_32_levels():
    """The widest matrix (sigma = 2^32, 32 levels): access, rank and select against
    direct counting, with symbols spread over the whole 32-bit range."""
    import torch

    import paper_1702_07578_gb300 as wtg
    rng = np.random.default_rng(32)
    vals = rng.integers(0, 1 << 32, size=300, dtype=np.uint64).astype(np.uint32)
    T = vals[rng.integers(0, vals.size, size=40000)]
    n, sigma = T.size, 1 << 32
    bv, z = wtg.wm_build(torch_text(T), sigma)
    idx = wtg.WtIndex(wtg.WT_MATRIX, bv, n, sigma, z)
    q = 2000
    pos = rng.integers(0, n, size=q).astype(np.uint64)
    sym = T[rng.integers(0, n, size=q)].astype(np.uint32)
    jj = rng.integers(1, 300, size=q).astype(np.uint64)
    acc, rank, sel = _brute(T, sigma, pos, sym, jj)
    dpos = torch.from_numpy(pos.view(np.int64)).cuda()
    dsym = torch.from_numpy(sym.view(np.int32)).cuda()
    dj = torch.from_numpy(jj.view(np.int64)).cuda()
    assert np.array_equal(idx.access(dpos).cpu().numpy().view(np.uint32), T[pos.astype(np.int64)])
    assert np.array_equal(idx.rank(dsym, dpos).cpu().numpy().view(np.uint64), rank)
    assert np.array_equal(idx.select(dsym, dj).cpu().numpy().view(np.uint64), sel)
