"""Lemma 3 (Sec. 5.2): the position in the wavelet matrix of a wavelet tree position.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.  It
shares no code with the CUDA library; numpy's cumsum / flatnonzero / bincount are
the only primitives, used as the plain definitions of rank, select and counting.

The construction, in the order of the proof of Lemma 3:

1. X[c] = |{j : T[j] = c}| for every character c (the histogram).
2. U = 1^X[0] 0 1^X[1] 0 ... 1^X[2^L - 1] 0, the unary histogram (length n + 2^L),
   with rank and select.
3. For l = L-1 down to 1: the counts of the l-bit prefixes from the (l+1)-bit ones
   (count[b] = count[2b] + count[2b+1]); then the zero-based prefix sum of those
   counts taken in bit-reversal order rho_l (the order of the WM's intervals on
   level l, Sec. 5.1) gives the start of each interval of level l in the WM; the
   start of prefix bp is stored at X[2^l - 2 + bp].
4. Query (l, i): j = i for l <= 1; otherwise
       c'  = rank0(U, select1(U, i + 1))          (a character with i's l-prefix)
       bp  = prefix(l, c')
       r   = select0(U, bp << (L - l))
       off = i - rank1(U, r)
       j   = X[2^l - 2 + bp] + off.

Readings (each also listed in the design notes of the repository):
  - The lemma's statement reads X[2^(l-1) - 2 + bp]; its proof stores level l at
    X[2^l - 2 ...] and reads X[2^l - 2 + bp].  Under the statement's form the
    levels overlap (level 2 would use X[0, 4), level 3 X[2, 10)), so the proof's
    index is taken; ``base="statement"`` keeps the other form so that a brute-force
    test can show it fails.
  - The alphabet is [0, 2^L) with L = ceil(lg sigma), as for every other oracle
    function: U has a run (possibly empty) and a closing zero for each of the
    2^L characters, and X has 2^l entries on each level l in [1, L).  Characters
    in [sigma, 2^L) never occur, so no query result changes.
  - select is 1-based as in the lemma; select0(U, 0) is taken as position 0, so
    that rank1(U, select0(U, 0)) = 0 (no character precedes character 0).
  - The in-place reuse of X for counting (a space bound, not a result) is not
    reproduced: the counts of each level live in their own array.
"""
from __future__ import annotations

import numpy as np


def _levels(sigma: int) -> int:
    L = 0
    while (1 << L) < sigma:
        L += 1
    return L


def _rho(l: int) -> np.ndarray:
    """rho_l(r): the l-bit reversal of r, for r in [0, 2^l)  (Sec. 5.1)."""
    r = np.arange(1 << l, dtype=np.int64)
    out = np.zeros_like(r)
    for b in range(l):
        out |= ((r >> b) & 1) << (l - 1 - b)
    return out


def _x_base(l: int, base: str) -> int:
    return (1 << l) - 2 if base == "proof" else (1 << (l - 1)) - 2


def wt2wm_tables(T, sigma, base: str = "proof"):
    """U (uint8 bits, length n + 2^L) and X (int64, 2^L entries) of Lemma 3."""
    T = np.asarray(T)
    L = _levels(int(sigma))
    if T.size and int(T.max()) >= (1 << L) and L > 0:
        raise ValueError("symbol out of range")
    # step 1: the histogram (counted in slices only to bound the memory of the copy)
    hist = np.zeros(1 << L, dtype=np.int64)
    for k in range(0, T.size, 1 << 24):
        hist += np.bincount(T[k:k + (1 << 24)], minlength=1 << L)[: 1 << L]
    # step 2: a run of X[c] ones, then one zero, for every character c
    runs = np.empty(2 * hist.size, dtype=np.int64)
    runs[0::2] = hist
    runs[1::2] = 1
    U = np.repeat(np.tile(np.array([1, 0], dtype=np.uint8), hist.size), runs)
    # step 3: interval starts of the WM, level by level from the leaves up
    X = np.zeros(max(1 << L, 1), dtype=np.int64)
    count = hist
    for l in range(L - 1, 0, -1):
        count = count[0::2] + count[1::2]          # counts of the l-bit prefixes
        order = _rho(l)                            # interval order of WM level l
        sizes = count[order]
        starts = np.concatenate(([0], np.cumsum(sizes)[:-1]))
        if _x_base(l, base) >= 0:                  # level 1 is never read (j = i there)
            X[_x_base(l, base) + order] = starts
    return U, X


def wt2wm(T, sigma, level, pos, base: str = "proof"):
    """j for every (level[k], pos[k]): WT level position -> WM level position."""
    U, X = wt2wm_tables(T, sigma, base)
    L = _levels(int(sigma))
    level = np.asarray(level, dtype=np.int64)
    pos = np.asarray(pos, dtype=np.int64)
    rank1 = np.concatenate(([0], np.cumsum(U, dtype=np.int64)))     # rank1(U, p) = rank1[p]
    ones = np.flatnonzero(U == 1)                                    # select1(U, k) = ones[k - 1]
    zeros = np.flatnonzero(U == 0)                                   # select0(U, k) = zeros[k - 1]
    out = pos.copy()
    deep = level > 1
    if not deep.any():
        return out
    l = level[deep]
    i = pos[deep]
    s1 = ones[i]                                   # select1(U, i + 1)
    c = s1 - rank1[s1]                             # rank0(U, s1)
    bp = c >> (L - l)
    m = bp << (L - l)
    r = np.where(m > 0, zeros[np.maximum(m, 1) - 1], 0)             # select0(U, m)
    off = i - rank1[r]
    xb = (np.int64(1) << l) - 2 if base == "proof" else (np.int64(1) << (l - 1)) - 2
    out[deep] = X[xb + bp] + off
    return out
