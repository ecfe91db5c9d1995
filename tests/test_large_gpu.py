"""Texts of any length (wt_build_large): slices built on their own and merged
(domain decomposition, Sec. 3.3).  Small slice lengths force many slices on texts
the oracle checks bit for bit; at n > 2^32 the periodic text's closed form and
sampled access walks on a Zipf text (decoded on the host from the GPU levels)
check the 64-bit path."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_u64, torch_text

pytestmark = pytest.mark.gpu


def _build(kind, T, sigma, slice_len):
    import torch

    import paper_1702_07578_gb300 as wtg
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    t = torch_text(T) if T.size else torch.zeros(0, dtype=torch.uint8, device="cuda")
    ws = torch.empty((wtg.wt_large_workspace_size(k, T.dtype.itemsize, T.size, sigma, slice_len),),
                     dtype=torch.uint8, device="cuda")
    bv, z = wtg.build_large(k, t, sigma, slice_len, ws=ws)
    wtg.wt_sync_status(ws)
    return to_u64(bv), (z.cpu().numpy().astype(np.uint64) if z is not None else None)


@pytest.mark.parametrize("kind", ["wt", "wm"])
@pytest.mark.parametrize("n,sigma,slice_len,dtype", [
    (0, 256, 1000, np.uint8), (1, 2, 1000, np.uint8), (5000, 256, 1000, np.uint8),
    (100003, 256, 4097, np.uint8), (300000, 16, 32773, np.uint8), (200000, 3, 65536, np.uint8),
    (250000, 200, 100000, np.uint16), (123457, 256, 777, np.uint8), (70000, 256, 1 << 20, np.uint8),
    (90000, 1, 1000, np.uint8),
])
def test_large_matches_oracle(kind, n, sigma, slice_len, dtype):
    T = synth.zipf_text(n, sigma, 1.0, 3 + n, dtype) if sigma > 1 else np.zeros(n, dtype)
    bv, z = _build(kind, T, sigma, slice_len)
    if kind == "wt":
        assert np.array_equal(bv, oracle.wt(T, sigma))
    else:
        e, ez = oracle.wm(T, sigma)
        assert np.array_equal(bv, e)
        assert np.array_equal(z[: e.shape[0]], ez)


def test_large_reports_errors_of_any_slice():
    import torch

    import paper_1702_07578_gb300 as wtg
    T = synth.uniform_text(50000, 100, 4, np.uint8)
    T[45000] = 200                                   # in the last of five slices
    ws = torch.empty((wtg.wt_large_workspace_size(wtg.WT_TREE, 1, T.size, 100, 10000),), dtype=torch.uint8,
                     device="cuda")
    wtg.build_large(wtg.WT_TREE, torch_text(T), 100, 10000, ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2
    with pytest.raises(wtg.WtError):
        wtg.wt_large_workspace_size(wtg.WT_TREE, 1, 1 << 20, 1000, 0)     # sigma > 256


def _periodic_words(l, W):
    """Level l of T[i] = i mod 256 (n a multiple of 256): (0^h 1^h) repeated, h = 2^(7-l)."""
    h = 1 << (7 - l)
    if h >= 64:
        k = np.arange(W, dtype=np.int64)
        return np.where(((k * 64) // h) % 2 == 1, np.uint64(2**64 - 1), np.uint64(0))
    pat = 0
    for b in range(64):
        if (b // h) % 2:
            pat |= 1 << b
    return np.full(W, pat, dtype=np.uint64)


@pytest.mark.slow
def test_large_beyond_2_32_periodic_closed_form():
    import torch

    import paper_1702_07578_gb300 as wtg
    n = (1 << 32) + (1 << 16)
    t = torch.arange(256, dtype=torch.uint8, device="cuda").repeat(n // 256)
    for k in (wtg.WT_TREE, wtg.WT_MATRIX):
        bv, z = wtg.build_large(k, t, 256)
        W = bv.shape[1]
        for l in range(8):
            exp = torch.from_numpy(_periodic_words(l, W).view(np.int64)).cuda()
            assert torch.equal(bv[l], exp), l
        if z is not None:
            assert z.cpu().tolist() == [n // 2] * 8
        del bv, z
        torch.cuda.empty_cache()


_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)


def _popcount(words):
    """Set bits of every uint64 (byte table; works on numpy 1 and 2)."""
    b = np.ascontiguousarray(words).view(np.uint8).reshape(-1, 8)
    return _POP8[b].sum(axis=1, dtype=np.int64)


def _ranker(words):
    cum = np.concatenate(([0], np.cumsum(_popcount(words), dtype=np.int64)))

    def rank1(p):
        w, s = p >> 6, p & 63
        r = int(cum[w])
        if s:
            r += bin(int(words[w]) & ((1 << s) - 1)).count("1")
        return r

    def bit(p):
        return int((words[p >> 6] >> np.uint64(p & 63)) & np.uint64(1))
    return rank1, bit


@pytest.mark.slow
def test_large_beyond_2_32_sampled_access():
    """n = 2^32 + 12345 Zipf bytes: access(i) by the WT node walk and by the WM walk
    (Sec. 2, Sec. 5), on the host from the GPU levels, gives T[i] at sampled i."""
    import torch

    import paper_1702_07578_gb300 as wtg
    n = (1 << 32) + 12345
    T = synth.zipf_text(n, 256, 1.0, 77, np.uint8)
    t = torch.from_numpy(T).cuda()
    rng = np.random.default_rng(1)
    samples = [0, n - 1, (1 << 32) - 1, 1 << 32] + [int(x) for x in rng.integers(0, n, 60)]
    bw, _ = wtg.build_large(wtg.WT_TREE, t, 256)
    lev = bw.cpu().numpy().view(np.uint64)
    del bw
    rk = [_ranker(lev[l]) for l in range(8)]
    for i in samples:                                  # WT: node ranges
        s, e, k, a = 0, n, i, 0
        for l in range(8):
            rank1, bit = rk[l]
            b = bit(s + k)
            o_s, o_sk, o_e = rank1(s), rank1(s + k), rank1(e)
            z = (e - s) - (o_e - o_s)
            if b:
                s, k = s + z, o_sk - o_s
            else:
                e, k = s + z, (k - (o_sk - o_s))
            a = 2 * a + b
        assert a == int(T[i]), i
    del lev, rk
    bm, zm = wtg.build_large(wtg.WT_MATRIX, t, 256)
    lev = bm.cpu().numpy().view(np.uint64)
    Z = zm.cpu().numpy()
    del bm
    rk = [_ranker(lev[l]) for l in range(8)]
    for i in samples:                                  # WM: rank0 or Z[l] + rank1
        p, a = i, 0
        for l in range(8):
            rank1, bit = rk[l]
            b = bit(p)
            r1 = rank1(p)
            p = int(Z[l]) + r1 if b else p - r1
            a = 2 * a + b
        assert a == int(T[i]), i
