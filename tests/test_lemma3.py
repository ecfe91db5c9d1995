"""Pins for the Lemma 3 oracle (WT position -> WM position, Sec. 5.2), no GPU.

* brute force: the WT and WM levels as stable sorts of the text positions
  (Obs. 1 / Obs. 2), so j must be the WM position of the very symbol that sits
  at WT position i; compared for every level and position on small random texts;
* the lemma's own claim: WT level bit i equals WM level bit j, read from the
  (separately pinned) construction oracles;
* j is a permutation of [0, n) on every level;
* a hand-derived example on the paper's running text (tests/golden);
* the statement's index X[2^(l-1) - 2 + bp] fails the brute force, the proof's
  X[2^l - 2 + bp] passes (the two forms disagree in the paper).
"""
import os

import numpy as np
import pytest

import oracle
from tests import bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lemma3_example.txt")


def brute_map(T, sigma):
    """level -> list j[i], from stable sorts of the text positions."""
    L = bf.levels_of(sigma)
    T = [int(x) for x in T]
    n = len(T)
    res = {}
    for l in range(L):
        wt = sorted(range(n), key=lambda k: bf.prefix(T[k], l, L))
        wm = sorted(range(n), key=lambda k: bf.rev(bf.prefix(T[k], l, L), l))
        where = {k: j for j, k in enumerate(wm)}
        res[l] = [where[wt[i]] for i in range(n)]
    return res


def all_levels(T, sigma, base="proof"):
    L = bf.levels_of(sigma)
    n = len(T)
    lv = np.repeat(np.arange(L), n)
    pos = np.tile(np.arange(n), L)
    return oracle.wt2wm(T, sigma, lv, pos, base=base).reshape(L, n) if L else np.zeros((0, n), np.int64)


@pytest.mark.parametrize("seed", range(6))
def test_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        sigma = int(rng.integers(1, 70))
        n = int(rng.integers(0, 90))
        # skewed draws leave characters out, so U has empty runs
        T = np.minimum(rng.geometric(0.25, n) - 1, sigma - 1).astype(np.uint16) if seed % 2 else \
            rng.integers(0, sigma, n).astype(np.uint16)
        got = all_levels(T, sigma)
        exp = brute_map(T, sigma)
        for l in range(bf.levels_of(sigma)):
            assert got[l].tolist() == exp[l], (sigma, n, l)


def test_bits_agree_with_construction_oracles():
    rng = np.random.default_rng(7)
    for sigma in (3, 5, 8, 17, 256, 1000):
        T = rng.integers(0, sigma, 3000).astype(np.uint16)
        wt = oracle.wt(T, sigma)
        wm, _ = oracle.wm(T, sigma)
        got = all_levels(T, sigma)
        for l in range(got.shape[0]):
            bt = np.array(bf.level_bits(wt[l], T.size))
            bm = np.array(bf.level_bits(wm[l], T.size))
            assert np.array_equal(bt, bm[got[l]]), (sigma, l)
            assert np.array_equal(np.sort(got[l]), np.arange(T.size)), (sigma, l)


def test_worked_example():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    T = np.array([int(x) for x in rows[0][1:]], np.uint8)
    sigma = int(rows[1][1])
    got = all_levels(T, sigma)
    for r in rows[2:]:
        l = int(r[0])
        assert got[l].tolist() == [int(x) for x in r[1:]], l


def test_statement_index_fails_proof_index_passes():
    rng = np.random.default_rng(3)
    fails = 0
    for _ in range(20):
        T = rng.integers(0, 16, 40).astype(np.uint8)
        exp = brute_map(T, 16)
        st = all_levels(T, 16, base="statement")
        pr = all_levels(T, 16, base="proof")
        for l in range(2, 4):
            assert pr[l].tolist() == exp[l]
            fails += st[l].tolist() != exp[l]
    assert fails > 0
