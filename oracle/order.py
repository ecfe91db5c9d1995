"""The stable order behind the levels: the permutation that the last level's split
leaves the text in, and the text in that order.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.  It
shares no code with the CUDA library; numpy's stable argsort is the one primitive.

Definitions (Obs. 1 and Obs. 2 taken one level past the last, l = L):
  * WT: the level-l sequence is T stably sorted by prefix(l, .); at l = L that is
    T stably sorted by the whole L-bit code, i.e. by the symbol (the sorted text
    T_sorted that psWT builds level by level, Sec. 3.2.1).
  * WM: the level-l sequence is T stably sorted by the bit-reversed prefix
    rho_l(prefix(l, .)) (Sec. 5.1); at l = L, by the reversed L-bit code.
perm[j] is the text position of the j-th symbol of that sequence; sorted[j] =
T[perm[j]].  The alphabet is [0, 2^L), L = ceil(lg sigma), as for the levels.
"""
from __future__ import annotations

import numpy as np


def _levels(sigma: int) -> int:
    L = 0
    while (1 << L) < sigma:
        L += 1
    return L


def _rev(a: np.ndarray, L: int) -> np.ndarray:
    """rho_L: the L-bit reversal of every code."""
    out = np.zeros_like(a)
    for b in range(L):
        out |= ((a >> b) & 1) << (L - 1 - b)
    return out


def stable_order(T, sigma, kind: str):
    """(perm, sorted) for kind 'wt' or 'wm'."""
    T = np.asarray(T)
    L = _levels(int(sigma))
    key = T.astype(np.int64)
    if kind == "wm":
        key = _rev(key, L)
    elif kind != "wt":
        raise ValueError(kind)
    perm = np.argsort(key, kind="stable").astype(np.uint32)
    return perm, T[perm]
