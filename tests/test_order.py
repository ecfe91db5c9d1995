"""Pins for the stable-order oracle (oracle/order.py), no GPU.

* Python's stable ``sorted`` with the key written from Obs. 1 / Obs. 2
  (tests/bf.py), on small random texts;
* the levels: the last level of the (separately pinned) construction oracles is
  the last code bit of the level-(L-1) sequence, and splitting that sequence
  stably by that bit gives the returned order;
* hand-derived values on the paper's running example;
* permutation, stability and sortedness invariants.
"""
import numpy as np
import pytest

import oracle
from tests import bf


def test_matches_python_sorted():
    rng = np.random.default_rng(12)
    for _ in range(300):
        sigma = int(rng.integers(1, 40))
        n = int(rng.integers(0, 50))
        T = rng.integers(0, sigma, n).astype(np.uint16)
        L = bf.levels_of(sigma)
        for kind in ("wt", "wm"):
            perm, srt = oracle.stable_order(T, sigma, kind)
            if kind == "wt":
                key = lambda i: int(T[i])
            else:
                key = lambda i: bf.rev(int(T[i]), L)
            exp = sorted(range(n), key=key)
            assert perm.tolist() == exp, (sigma, n, kind)
            assert srt.tolist() == [int(T[i]) for i in exp]


def test_running_example():
    """T = 0167154263, sigma = 8.  WT: positions of 0,1,1,2,3,4,5,6,6,7.  WM: codes
    reversed (0->0, 4->1, 2->2, 6->3, 1->4, 5->5, 3->6, 7->7), so the order is
    0 | 4 | 2 | 6 6 | 1 1 | 5 | 3 | 7."""
    T = np.array([0, 1, 6, 7, 1, 5, 4, 2, 6, 3], np.uint8)
    p, s = oracle.stable_order(T, 8, "wt")
    assert p.tolist() == [0, 1, 4, 7, 9, 6, 5, 2, 8, 3]
    assert s.tolist() == [0, 1, 1, 2, 3, 4, 5, 6, 6, 7]
    p, s = oracle.stable_order(T, 8, "wm")
    assert s.tolist() == [0, 4, 2, 6, 6, 1, 1, 5, 3, 7]
    assert p.tolist() == [0, 6, 7, 2, 8, 1, 4, 5, 9, 3]


@pytest.mark.parametrize("sigma", [2, 5, 16, 256, 1000])
def test_last_split_of_the_levels(sigma):
    """The returned order is the stable split, by the last code bit, of the sequence
    whose last bit the construction oracles store as their last level: within each
    node for the WT, over the whole level (zeros first) for the WM."""
    rng = np.random.default_rng(sigma)
    T = rng.integers(0, sigma, 3000).astype(np.uint16)
    L = bf.levels_of(sigma)
    for kind in ("wt", "wm"):
        if kind == "wt":
            key = lambda a: bf.prefix(a, L - 1, L)
            lev = oracle.wt(T, sigma)
        else:
            key = lambda a: bf.rev(bf.prefix(a, L - 1, L), L - 1)
            lev = oracle.wm(T, sigma)[0]
        last = sorted((int(x) for x in T), key=key)               # level L-1 sequence (Obs. 1 / 2)
        assert [a & 1 for a in last] == bf.level_bits(lev[L - 1], T.size)
        if kind == "wm":
            exp = [a for a in last if a & 1 == 0] + [a for a in last if a & 1]
        else:
            exp = []
            for p in range(1 << (L - 1)):
                node = [a for a in last if a >> 1 == p]
                exp += [a for a in node if a & 1 == 0] + [a for a in node if a & 1]
        _, srt = oracle.stable_order(T, sigma, kind)
        assert srt.tolist() == exp, kind


def test_invariants():
    rng = np.random.default_rng(4)
    T = (rng.zipf(1.3, 20000) % 300).astype(np.uint16)
    for kind in ("wt", "wm"):
        p, s = oracle.stable_order(T, 300, kind)
        assert np.array_equal(np.sort(p), np.arange(T.size))
        assert np.array_equal(s, T[p])
        key = s.astype(np.int64) if kind == "wt" else np.array([bf.rev(int(x), 9) for x in s])
        assert np.all(np.diff(key) >= 0)
        same = np.diff(key) == 0
        assert np.all(np.diff(p.astype(np.int64))[same] > 0)       # stable: equal keys keep text order
