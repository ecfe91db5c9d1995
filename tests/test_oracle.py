"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * the paper's running example, worked out by hand from the definitions;
  * brute-force decoders (access / rank / select) that reconstruct T;
  * the sorted-order characterisations of Obs. 1 and Obs. 2, computed with
    Python's stable sort;
  * closed forms (identity text, constant text, sigma = 2, zero text);
  * invariants stated in the paper (levels 0 and 1 of WT and WM agree, equal
    interval sizes, Z[l] = zeros of level l);
  * exhaustive enumeration of all texts with n <= 6 over sigma <= 4 and
    n <= 5 over sigma = 5, plus Algorithm 1 and Algorithm 2 as two further
    independent routes.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from tests import bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _golden():
    g = {"wt": {}, "wm": {}}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "text":
            g["text"] = [int(x) for x in f[1:]]
        elif f[0] == "sigma":
            g["sigma"] = int(f[1])
        elif f[0] in ("wt", "wm"):
            g[f[0]][int(f[1])] = f[2]
        else:
            g[f[0]] = [int(x) for x in f[1:]]
    return g


def _strings(bv, n):
    return {l: oracle.bits_string(bv[l], n) for l in range(bv.shape[0])}


def test_worked_example_all_routes():
    g = _golden()
    T = np.array(g["text"], dtype=np.uint8)
    n = T.size
    assert _strings(oracle.wt(T, g["sigma"]), n) == g["wt"]
    bv, Z = oracle.wm(T, g["sigma"])
    assert _strings(bv, n) == g["wm"]
    assert list(Z) == g["z"]
    assert _strings(oracle.pc("wt", T, g["sigma"]), n) == g["wt"]
    bv, Z = oracle.pc("wm", T, g["sigma"])
    assert _strings(bv, n) == g["wm"] and list(Z) == g["z"]
    for p in (1, 2, 3, 10):
        assert _strings(oracle.ps("wt", T, g["sigma"], p), n) == g["wt"]
        bv, Z = oracle.ps("wm", T, g["sigma"], p)
        assert _strings(bv, n) == g["wm"] and list(Z) == g["z"]


def test_worked_example_intermediates():
    """Level-2 histogram and interval starts of Alg. 1 (id and pi_2 order)."""
    g = _golden()
    L = 3
    hist2 = [0] * 4
    for a in g["text"]:
        hist2[bf.prefix(a, 2, L)] += 1
    assert hist2 == g["hist2"]
    spos_wt = [sum(hist2[:p]) for p in range(4)]
    spos_wm = [sum(hist2[q] for q in range(4) if bf.rev(q, 2) < bf.rev(p, 2)) for p in range(4)]
    assert spos_wt == g["spos2_wt"] and spos_wm == g["spos2_wm"]
    # the interval starts are where each prefix's bits begin in the levels
    T = np.array(g["text"], dtype=np.uint8)
    srt_wt = sorted(g["text"], key=lambda a: bf.prefix(a, 2, L))
    srt_wm = sorted(g["text"], key=lambda a: bf.rev(bf.prefix(a, 2, L), 2))
    for p in range(4):
        if hist2[p]:
            assert bf.prefix(srt_wt[spos_wt[p]], 2, L) == p
            assert bf.prefix(srt_wm[spos_wm[p]], 2, L) == p
    assert oracle.wt(T, 8).shape == (3, 1)


def _check_all(T, sigma, decoders=True):
    """Every route and every brute-force property for one text."""
    n = len(T)
    L = bf.levels_of(sigma)
    arr = np.array(T, dtype=np.uint32)
    wt = oracle.wt(arr, sigma)
    wm, Z = oracle.wm(arr, sigma)
    assert wt.shape == (L, (n + 63) // 64) and wm.shape == wt.shape
    exp_wt = bf.sorted_levels(T, L, matrix=False)
    exp_wm = bf.sorted_levels(T, L, matrix=True)
    for l in range(L):
        assert bf.level_bits(wt[l], n) == exp_wt[l]
        assert bf.level_bits(wm[l], n) == exp_wm[l]
        # tail bits beyond n are zero
        if n % 64:
            assert int(wt[l][-1]) >> (n % 64) == 0 and int(wm[l][-1]) >> (n % 64) == 0
        assert int(Z[l]) == n - sum(exp_wm[l])
    assert np.array_equal(oracle.pc("wt", arr, sigma), wt)
    pz = oracle.pc("wm", arr, sigma)
    assert np.array_equal(pz[0], wm) and np.array_equal(pz[1], Z)
    for p in (1, 2, 3):
        assert np.array_equal(oracle.ps("wt", arr, sigma, p), wt)
        sz = oracle.ps("wm", arr, sigma, p)
        assert np.array_equal(sz[0], wm) and np.array_equal(sz[1], Z)
    if decoders and L > 0:
        lv_wt = [bf.level_bits(wt[l], n) for l in range(L)]
        lv_wm = [bf.level_bits(wm[l], n) for l in range(L)]
        for i in range(n):
            assert bf.wt_access(lv_wt, n, L, i) == T[i]
            assert bf.wm_access(lv_wm, Z, L, i) == T[i]
    return wt, wm, Z


def test_exhaustive_tiny_texts():
    count = 0
    for sigma in range(1, 6):
        nmax = 6 if sigma <= 4 else 5
        for n in range(0, nmax + 1):
            for T in itertools.product(range(sigma), repeat=n):
                _check_all(list(T), sigma, decoders=(n <= 4))
                count += 1
    assert count > 5000


@pytest.mark.parametrize("sigma,n,seed", [
    (2, 1000, 1), (3, 777, 2), (5, 4096, 3), (8, 3001, 4), (256, 4096, 5),
    (4096, 2500, 6), (1 << 20, 700, 7), (1000, 1500, 8)])
def test_random_against_sorted_definitions(sigma, n, seed):
    rng = np.random.default_rng(seed)
    T = rng.integers(0, sigma, size=n).tolist()
    _check_all(T, sigma, decoders=False)


@pytest.mark.parametrize("sigma", [4, 8, 16, 23])
def test_rank_select_by_decoders(sigma):
    """rank/select through the WT and WM walks equal direct counting on T."""
    rng = np.random.default_rng(sigma)
    n = 97
    T = rng.integers(0, sigma, size=n).tolist()
    L = bf.levels_of(sigma)
    arr = np.array(T, dtype=np.uint32)
    wt = oracle.wt(arr, sigma)
    wm, Z = oracle.wm(arr, sigma)
    lv_wt = [bf.level_bits(wt[l], n) for l in range(L)]
    lv_wm = [bf.level_bits(wm[l], n) for l in range(L)]
    for c in range(sigma):
        for i in range(0, n + 1, 7):
            exp = sum(1 for x in T[:i] if x == c)
            assert bf.wt_rank(lv_wt, n, L, c, i) == exp
            assert bf.wm_rank(lv_wm, Z, n, L, c, i) == exp
        occ = [p for p, x in enumerate(T) if x == c]
        for j, p in enumerate(occ[:3], start=1):
            assert bf.select_by_rank(lambda cc, ii: bf.wt_rank(lv_wt, n, L, cc, ii), c, j, n) == p
            assert bf.select_by_rank(lambda cc, ii: bf.wm_rank(lv_wm, Z, n, L, cc, ii), c, j, n) == p


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 11])
def test_identity_text_closed_form(L):
    """T = 0..2^L-1: every level of WT and WM is (0^h 1^h)^(2^l), h = 2^(L-l-1)."""
    n = 1 << L
    T = np.arange(n, dtype=np.uint32)
    wt = oracle.wt(T, n)
    wm, Z = oracle.wm(T, n)
    for l in range(L):
        h = 1 << (L - l - 1)
        exp = ([0] * h + [1] * h) * (1 << l)
        assert bf.level_bits(wt[l], n) == exp
        assert bf.level_bits(wm[l], n) == exp
        assert int(Z[l]) == n // 2


@pytest.mark.parametrize("a,sigma,n", [(0, 2, 100), (5, 8, 130), (255, 256, 64), (1000, 1024, 65),
                                       (0, 256, 300)])
def test_constant_text_closed_form(a, sigma, n):
    T = np.full(n, a, dtype=np.uint32)
    L = bf.levels_of(sigma)
    wt = oracle.wt(T, sigma)
    wm, Z = oracle.wm(T, sigma)
    for l in range(L):
        exp = [bf.bit(a, l, L)] * n
        assert bf.level_bits(wt[l], n) == exp
        assert bf.level_bits(wm[l], n) == exp
        assert int(Z[l]) == (n if exp[0] == 0 else 0)


def test_sigma_two_is_the_text():
    rng = np.random.default_rng(11)
    T = rng.integers(0, 2, size=1000).astype(np.uint8)
    wt = oracle.wt(T, 2)
    wm, Z = oracle.wm(T, 2)
    assert wt.shape[0] == 1
    assert bf.level_bits(wt[0], 1000) == T.tolist() == bf.level_bits(wm[0], 1000)
    assert int(Z[0]) == 1000 - int(T.sum())


def test_sigma_one_and_empty():
    assert oracle.wt(np.zeros(10, np.uint8), 1).shape == (0, 1)
    bv, Z = oracle.wm(np.zeros(0, np.uint8), 256)
    assert bv.shape == (8, 0) and list(Z) == [0] * 8


def test_invariants_wt_vs_wm():
    """Levels 0 and 1 agree; every level has the same ones count (Sec. 5.1, 5.2)."""
    rng = np.random.default_rng(3)
    T = rng.integers(0, 256, size=5000).astype(np.uint8)
    wt = oracle.wt(T, 256)
    wm, Z = oracle.wm(T, 256)
    assert np.array_equal(wt[0], wm[0]) and np.array_equal(wt[1], wm[1])
    for l in range(8):
        ones_wt = sum(bin(int(x)).count("1") for x in wt[l])
        ones_wm = sum(bin(int(x)).count("1") for x in wm[l])
        assert ones_wt == ones_wm == 5000 - int(Z[l])
        assert ones_wt == int(sum((int(a) >> (7 - l)) & 1 for a in T))


def test_symbol_out_of_range_rejected():
    with pytest.raises(ValueError):
        oracle.wt(np.array([0, 8], dtype=np.uint8), 8)
    with pytest.raises(ValueError):
        oracle.wm(np.array([300], dtype=np.uint16), 256)


def test_planted_mistakes_are_caught():
    """Plausible oracle mistakes (planted in copies of its output) fail the pins."""
    rng = np.random.default_rng(5)
    T = rng.integers(0, 16, size=200).tolist()
    n, L = len(T), 4
    arr = np.array(T, dtype=np.uint32)
    wt = oracle.wt(arr, 16)
    wm, Z = oracle.wm(arr, 16)
    exp_wt = bf.sorted_levels(T, L, matrix=False)
    exp_wm = bf.sorted_levels(T, L, matrix=True)
    # a transposed pair of levels
    bad = wt[[0, 2, 1, 3]]
    assert any(bf.level_bits(bad[l], n) != exp_wt[l] for l in range(L))
    # WT order used for the WM (missing bit reversal) differs from Obs. 2 at level 2+
    assert any(bf.level_bits(wt[l], n) != exp_wm[l] for l in range(2, L))
    # an off-by-one Z breaks access()
    lv_wm = [bf.level_bits(wm[l], n) for l in range(L)]
    Zbad = Z.copy()
    Zbad[1] += 1
    assert any(bf.wm_access(lv_wm, Zbad, L, i) != T[i] for i in range(n))
    # one flipped bit breaks access()
    lv_wt = [bf.level_bits(wt[l], n) for l in range(L)]
    lv_wt[3][57] ^= 1
    assert any(bf.wt_access(lv_wt, n, L, i) != T[i] for i in range(n))
