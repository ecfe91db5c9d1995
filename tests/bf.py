"""Brute-force helpers for the tests: decoders and definitions written without
any of the construction code (oracle or CUDA).

* ``level_bits``     unpack one packed level (LSB-first words) into a list of bits
* ``wt_access``      WT access(i): walk down with node ranges (Sec. 2)
* ``wm_access``      WM access(i): i <- rank0 or Z[l] + rank1 (Sec. 5)
* ``wt_rank`` / ``wm_rank``  rank_c(i) by the same walks
* ``sorted_levels``  level l as bit l of T stably sorted by a key (Obs. 1 / Obs. 2),
                     using Python's stable ``sorted`` as the primitive
* ``rev``            bit reversal of a k-bit integer (Sec. 5)
"""
from __future__ import annotations

import numpy as np


def levels_of(sigma: int) -> int:
    L = 0
    while (1 << L) < sigma:
        L += 1
    return L


def level_bits(words, n):
    words = [int(x) for x in words]
    return [(words[j >> 6] >> (j & 63)) & 1 for j in range(n)]


def pack_bits(bits):
    n = len(bits)
    out = np.zeros((n + 63) // 64, dtype=np.uint64)
    for j, b in enumerate(bits):
        if b:
            out[j >> 6] |= np.uint64(1 << (j & 63))
    return out


def bit(a, k, L):
    return (a >> (L - 1 - k)) & 1


def prefix(a, k, L):
    return a >> (L - k) if k > 0 else 0


def rev(x, k):
    r = 0
    for b in range(k):
        r |= ((x >> b) & 1) << (k - 1 - b)
    return r


def sorted_levels(T, L, matrix):
    """Level l = bit l of T stably sorted by prefix(l) (WT) or rev(prefix(l)) (WM)."""
    T = [int(x) for x in T]
    out = []
    for l in range(L):
        if matrix:
            key = lambda a, l=l: rev(prefix(a, l, L), l)
        else:
            key = lambda a, l=l: prefix(a, l, L)
        s = sorted(T, key=key)
        out.append([bit(a, l, L) for a in s])
    return out


def _rank(bits, b, e, v):
    return sum(1 for j in range(b, e) if bits[j] == v)


def wt_access(levels, n, L, i):
    s, e, a = 0, n, 0
    for l in range(L):
        bits = levels[l]
        z = _rank(bits, s, e, 0)
        b = bits[s + i]
        a = (a << 1) | b
        if b == 0:
            i = _rank(bits, s, s + i, 0)
            e = s + z
        else:
            i = _rank(bits, s, s + i, 1)
            s = s + z
    return a


def wm_access(levels, Z, L, i):
    a = 0
    for l in range(L):
        bits = levels[l]
        b = bits[i]
        a = (a << 1) | b
        i = (int(Z[l]) + _rank(bits, 0, i, 1)) if b else _rank(bits, 0, i, 0)
    return a


def wt_rank(levels, n, L, c, i):
    """Number of c in T[0, i) using the WT alone."""
    s, e = 0, n
    for l in range(L):
        bits = levels[l]
        z = _rank(bits, s, e, 0)
        b = bit(c, l, L)
        if b == 0:
            i = _rank(bits, s, s + i, 0)
            e = s + z
        else:
            i = _rank(bits, s, s + i, 1)
            s = s + z
    return i


def wm_rank(levels, Z, n, L, c, i):
    """Number of c in T[0, i) using the WM alone (Sec. 5 navigation)."""
    s = 0                       # start of c's interval on the current level
    for l in range(L):
        bits = levels[l]
        b = bit(c, l, L)
        if b == 0:
            s, i = _rank(bits, 0, s, 0), _rank(bits, 0, i, 0)
        else:
            s = int(Z[l]) + _rank(bits, 0, s, 1)
            i = int(Z[l]) + _rank(bits, 0, i, 1)
    return i - s


def select_by_rank(rank_fn, c, j, n):
    """Position of the j-th (1-based) c, from a rank function, or None."""
    for p in range(n):
        if rank_fn(c, p + 1) == j:
            return p
    return None
