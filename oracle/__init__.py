"""CPU oracle for wavelet tree / wavelet matrix construction (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.

The arithmetic lives in ``wt_oracle.c`` (plain single-threaded C, compiled here
with gcc into ``oracle/_build/``).  This module only marshals numpy arrays.

Functions (all return numpy arrays; ``bv`` has shape ``(L, ceil(n/64))`` of
uint64, level-major, bit j of a level at bit ``j & 63`` of word ``j >> 6``):

``wt(T, sigma)``            WT from the node definition (Sec. 2, Obs. 1)
``wm(T, sigma)``            WM and Z from the definition (Sec. 5)
``pc(kind, T, sigma)``      Algorithm 1, pcWT / pcWM (Sec. 3.1, Sec. 5.1)
``ps(kind, T, sigma, p)``   Algorithm 2, psWT / psWM with p slices (Sec. 3.2.1)
``wt2wm(T, sigma, l, i)``   Lemma 3: WT position -> WM position (``lemma3.py``, numpy)
``stable_order(T, sigma, kind)``  the order after the last level, as a permutation and
                            as the sorted text (``order.py``, numpy)
``merge(kind, L, slices)``  merge of the partial WT/WM of consecutive slices, Sec. 3.3
                            (``merge.py``, numpy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no vectorisation flags, no threads)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            vp = ctypes.c_void_p
            lib.oracle_levels.argtypes = [ctypes.c_uint64]
            lib.oracle_levels.restype = ctypes.c_uint32
            lib.oracle_wt_topdown.argtypes = [vp, ctypes.c_int, ctypes.c_uint64,
                                              ctypes.c_uint32, u64p]
            lib.oracle_wm_topdown.argtypes = [vp, ctypes.c_int, ctypes.c_uint64,
                                              ctypes.c_uint32, u64p, u64p]
            lib.oracle_pc.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint32, u64p, u64p]
            lib.oracle_ps.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_uint32, u64p, u64p]
            for f in (lib.oracle_wt_topdown, lib.oracle_wm_topdown, lib.oracle_pc,
                      lib.oracle_ps):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def levels(sigma: int) -> int:
    """L = ceil(lg sigma); 0 for sigma <= 1."""
    return int(_load().oracle_levels(int(sigma)))


def _prep(T):
    T = np.ascontiguousarray(T)
    if T.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError("text must be uint8, uint16 or uint32")
    return T, T.dtype.itemsize


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


_ERR = {-1: "invalid argument", -2: "symbol out of range", -3: "out of memory"}


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")


def _outputs(n, L):
    W = (n + 63) // 64
    return np.zeros((max(L, 0), W), dtype=np.uint64), np.zeros(max(L, 1), dtype=np.uint64)


def wt(T, sigma):
    """Level-wise wavelet tree bit vectors, shape (L, ceil(n/64))."""
    T, w = _prep(T)
    L = levels(sigma)
    bv, _ = _outputs(T.size, L)
    _check(_load().oracle_wt_topdown(T.ctypes.data, w, T.size, L, _u64p(bv)))
    return bv


def wm(T, sigma):
    """Wavelet matrix bit vectors and zero counts Z (length L)."""
    T, w = _prep(T)
    L = levels(sigma)
    bv, Z = _outputs(T.size, L)
    _check(_load().oracle_wm_topdown(T.ctypes.data, w, T.size, L, _u64p(bv), _u64p(Z)))
    return bv, Z[:L]


def pc(kind, T, sigma):
    """Algorithm 1 (kind 'wt' or 'wm').  Returns bv (and Z for 'wm')."""
    T, w = _prep(T)
    L = levels(sigma)
    bv, Z = _outputs(T.size, L)
    m = 1 if kind == "wm" else 0
    _check(_load().oracle_pc(m, T.ctypes.data, w, T.size, L, _u64p(bv), _u64p(Z)))
    return (bv, Z[:L]) if m else bv


def ps(kind, T, sigma, p):
    """Algorithm 2 with p slices (kind 'wt' or 'wm').  Returns bv (and Z for 'wm')."""
    T, w = _prep(T)
    L = levels(sigma)
    bv, Z = _outputs(T.size, L)
    m = 1 if kind == "wm" else 0
    _check(_load().oracle_ps(m, T.ctypes.data, w, T.size, L, int(p), _u64p(bv), _u64p(Z)))
    return (bv, Z[:L]) if m else bv


def bits_string(bv_level, n):
    """Render the first n bits of one packed level as a '0'/'1' string (position order)."""
    out = []
    for j in range(n):
        out.append("1" if (int(bv_level[j >> 6]) >> (j & 63)) & 1 else "0")
    return "".join(out)


from .lemma3 import wt2wm, wt2wm_tables  # noqa: E402,F401
from .order import stable_order  # noqa: E402,F401
from .merge import merge  # noqa: E402,F401
