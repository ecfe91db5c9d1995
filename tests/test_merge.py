"""Pins for the domain-decomposition merge of the oracle (oracle/merge.py), no GPU:
merging the (separately pinned) oracle WT / WM of consecutive slices gives the oracle
WT / WM of the whole text, for slice counts 1 to many, empty and one-symbol slices,
slice borders off word boundaries, and alphabets of one to eight levels; merging the
WM's intervals in id order instead of bit-reversal order fails."""
import numpy as np
import pytest

import oracle


def _slices(T, sigma, cuts, kind):
    L = oracle.levels(sigma)
    out = []
    for a, b in zip([0] + cuts, cuts + [T.size]):
        part = T[a:b]
        hist = np.bincount(part.astype(np.int64), minlength=1 << L)[: 1 << L] if L else np.array([part.size])
        if kind == "wt":
            lev, z = oracle.wt(part, sigma), None
        else:
            lev, z = oracle.wm(part, sigma)
        out.append((part.size, lev, hist, z))
    return out


@pytest.mark.parametrize("kind", ["wt", "wm"])
@pytest.mark.parametrize("sigma", [2, 3, 8, 100, 256])
def test_merge_equals_whole_text(kind, sigma):
    rng = np.random.default_rng(sigma)
    for trial in range(6):
        n = int(rng.integers(0, 3000))
        T = rng.integers(0, sigma, n).astype(np.uint8)
        k = int(rng.integers(0, 6))
        cuts = sorted(int(x) for x in rng.integers(0, n + 1, size=k)) if n else []
        got, z = oracle.merge(kind, oracle.levels(sigma), _slices(T, sigma, cuts, kind))
        if kind == "wt":
            assert np.array_equal(got, oracle.wt(T, sigma)), (n, cuts)
        else:
            e, ez = oracle.wm(T, sigma)
            assert np.array_equal(got, e), (n, cuts)
            assert np.array_equal(z, ez)


def test_wm_needs_bit_reversal_order():
    """Planted mistake: the WM merged in id order differs from the whole text's WM."""
    import importlib
    om = importlib.import_module("oracle.merge")      # the module (the package exports the function)
    rng = np.random.default_rng(5)
    T = rng.integers(0, 16, 500).astype(np.uint8)
    sl = _slices(T, 16, [123, 300], "wm")
    saved = om._rho
    try:
        om._rho = lambda l: np.arange(1 << l)
        got, _ = om.merge("wm", 4, sl)
    finally:
        om._rho = saved
    assert not np.array_equal(got, oracle.wm(T, 16)[0])
