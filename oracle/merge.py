"""Merging the partial wavelet trees / matrices of consecutive slices of a text
(domain decomposition, Sec. 3.3).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.  It
shares no code with the CUDA library; numpy's unpackbits / packbits / cumsum are the
only primitives.

In the order of the paper's description: every slice's levels are a partial WT (or
WM) whose level l consists of one interval per l-bit prefix, in id order (WT) or in
the bit-reversal order rho_l (WM, Sec. 5.1), each holding that prefix's symbols in
text order.  The merged level l concatenates, prefix by prefix in the same order, the
intervals of all slices in slice order; a zero-based prefix sum of the interval sizes
gives where each lands.  The WM's Z[l] is the sum of the slices' Z[l].

Readings (listed in the design notes):
  - the WM is merged like the WT with the prefixes in rho_l order, which Sec. 3.3
    does not spell out (it treats the WT); the merged intervals are then the
    intervals of the whole text's WM because each is the prefix's symbols in text
    order;
  - interval sizes come from each slice's leaf histogram (2^L entries, folded).
"""
from __future__ import annotations

import numpy as np


def _rho(l: int) -> np.ndarray:
    r = np.arange(1 << l, dtype=np.int64)
    out = np.zeros_like(r)
    for b in range(l):
        out |= ((r >> b) & 1) << (l - 1 - b)
    return out


def _bits(words: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(np.asarray(words, dtype=np.uint64).view(np.uint8), bitorder="little")[:n]


def _words(bits: np.ndarray) -> np.ndarray:
    pad = (-bits.size) % 64
    b = np.concatenate([bits.astype(np.uint8), np.zeros(pad, np.uint8)])
    return np.packbits(b, bitorder="little").view(np.uint64)


def merge(kind: str, L: int, slices):
    """slices: list of (n_c, levels_c (L, W_c) uint64, leaf_hist_c (2^L,), Z_c or None).
    Returns (levels (L, W) uint64, Z or None) of the whole text."""
    n = sum(s[0] for s in slices)
    out = np.zeros((L, (n + 63) // 64), dtype=np.uint64)
    for l in range(L):
        order = _rho(l) if kind == "wm" else np.arange(1 << l)
        pieces = []
        per_slice = []
        for n_c, lev, hist, _ in slices:
            cnt = np.asarray(hist, dtype=np.int64).reshape(1 << l, -1).sum(axis=1)   # l-bit prefixes
            start = np.zeros(1 << l, dtype=np.int64)
            start[order] = np.concatenate(([0], np.cumsum(cnt[order])[:-1]))       # interval starts
            per_slice.append((_bits(lev[l], n_c), cnt, start))
        for q in order:
            for bits, cnt, start in per_slice:
                pieces.append(bits[start[q]:start[q] + cnt[q]])
        merged = np.concatenate(pieces) if pieces else np.zeros(0, np.uint8)
        assert merged.size == n
        out[l] = _words(merged)[: out.shape[1]]
    Z = None
    if kind == "wm":
        Z = np.sum([np.asarray(s[3], dtype=np.uint64) for s in slices], axis=0) if slices else np.zeros(L, np.uint64)
    return out, Z
