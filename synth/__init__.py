"""Seeded synthetic inputs for the tests and the benchmark.

The draws are made by ``synth.c`` (SplitMix64, counter based, so any number of
threads gives the same bytes).  This package holds no wavelet tree / matrix
arithmetic; the oracle and the CUDA library both consume the arrays it returns.

Workloads (stand-ins for the byte texts and the integer-alphabet text of the
paper's Table 1, whose data is not available here):

``uniform_text``        i.i.d. uniform symbols over [0, sigma)
``zipf_text``           Zipf(s) ranks over sigma symbols mapped through a seeded
                        permutation (byte-text-like skew)
``uniform_markov_text`` first half i.i.d. uniform, second half an order-1
                        Markov chain with 64 hash-defined successors per state
``batch_specs`` / ``batch_texts``  many texts of log-uniform length with mixed
                        alphabets (uint16 storage), Zipf symbols
``request_specs``       a served request stream (Poisson arrivals)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT, "libsynth.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 0x5EED0000


def build(force: bool = False) -> str:
    os.makedirs(_OUT, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u32, vp, ci = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
            lib.synth_splitmix64.argtypes = [u64, u64]
            lib.synth_splitmix64.restype = u64
            lib.synth_permutation.argtypes = [u64, u32, vp]
            lib.synth_uniform.argtypes = [u64, u64, u64, u32, vp, ci, ci]
            lib.synth_zipf.argtypes = [u64, u64, u64, u32, ctypes.c_double, vp, ci, ci]
            lib.synth_markov.argtypes = [u64, u64, u64, u32, u32, vp, ci]
            for f in (lib.synth_permutation, lib.synth_uniform, lib.synth_zipf,
                      lib.synth_markov):
                f.restype = ci
            _lib = lib
    return _lib


def _threads():
    return max(1, min(64, os.cpu_count() or 1))


def _dtype_for(sigma: int):
    if sigma <= 1 << 8:
        return np.uint8
    if sigma <= 1 << 16:
        return np.uint16
    return np.uint32


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"synth: error {rc}")


def splitmix64(seed: int, i: int) -> int:
    return int(_load().synth_splitmix64(seed & (2**64 - 1), i))


def uniform01(seed: int, i: int) -> float:
    return (splitmix64(seed, i) >> 11) * (1.0 / 9007199254740992.0)


def permutation(seed: int, k: int) -> np.ndarray:
    p = np.empty(k, dtype=np.uint32)
    _check(_load().synth_permutation(seed, k, p.ctypes.data))
    return p


def uniform_text(n: int, sigma: int, seed: int, dtype=None, offset: int = 0) -> np.ndarray:
    dtype = dtype or _dtype_for(sigma)
    out = np.empty(n, dtype=dtype)
    _check(_load().synth_uniform(seed, offset, n, sigma, out.ctypes.data,
                                 out.itemsize, _threads()))
    return out


def zipf_text(n: int, sigma: int, s: float, seed: int, dtype=None) -> np.ndarray:
    dtype = dtype or _dtype_for(sigma)
    out = np.empty(n, dtype=dtype)
    _check(_load().synth_zipf(seed, seed ^ 0xA5A5A5A5, n, sigma, float(s),
                              out.ctypes.data, out.itemsize, _threads()))
    return out


def uniform_markov_text(n: int, sigma: int, seed: int, dtype=None) -> np.ndarray:
    """First half uniform over [0, sigma); second half a Markov chain started at
    the last uniform symbol (sigma must be a power of two)."""
    dtype = dtype or _dtype_for(sigma)
    out = np.empty(n, dtype=dtype)
    h = n // 2
    _check(_load().synth_uniform(seed, 0, h, sigma, out.ctypes.data, out.itemsize,
                                 _threads()))
    start = int(out[h - 1]) if h > 0 else 0
    tail = out[h:]
    _check(_load().synth_markov(seed ^ 0x1234567, seed ^ 0x7654321, n - h, sigma, start,
                                tail.ctypes.data, out.itemsize))
    return out


# ---- named workloads ------------------------------------------------------

def workload_small():
    """n = 2^20 uint8, sigma = 256, i.i.d. uniform."""
    return uniform_text(1 << 20, 256, SEED_BASE + 0, np.uint8), 256


def workload_bytes(n: int = 1 << 30):
    """n = 2^30 uint8, sigma = 256, Zipf(1.0) over a seeded permutation."""
    return zipf_text(n, 256, 1.0, SEED_BASE + 1, np.uint8), 256


def workload_large_alphabet(n: int = 1 << 28):
    """n = 2^28 uint32, sigma = 2^20, half uniform, half Markov."""
    return uniform_markov_text(n, 1 << 20, SEED_BASE + 2, np.uint32), 1 << 20


def batch_specs(count: int = 4096, seed: int = SEED_BASE + 3,
                min_log: int = 10, max_log: int = 20,
                sigmas=(1 << 4, 1 << 8, 1 << 12, 1 << 16)):
    """(length, sigma, text seed) per text: length floor(2^(min+(max-min)u))."""
    specs = []
    for t in range(count):
        u = uniform01(seed, 3 * t)
        n = int(math.floor(2.0 ** (min_log + (max_log - min_log) * u)))
        sg = sigmas[int(uniform01(seed, 3 * t + 1) * len(sigmas))]
        specs.append((n, sg, (seed * 1000003 + t) & (2**63 - 1)))
    return specs


def batch_texts(specs, s: float = 0.8):
    """Zipf(s) texts, uint16 storage, one seeded permutation per text."""
    return [zipf_text(n, sg, s, ts, np.uint16) for (n, sg, ts) in specs]


def request_specs(count: int, rate_hz: float, seed: int = SEED_BASE + 4,
                  min_log: int = 12, max_log: int = 26):
    """Served stream: (arrival time s, n, sigma, zipf?, kind, text seed)."""
    t = 0.0
    out = []
    for r in range(count):
        u = uniform01(seed, 6 * r)
        t += -math.log(1.0 - u) / rate_hz
        n = int(math.floor(2.0 ** (min_log + (max_log - min_log) * uniform01(seed, 6 * r + 1))))
        sg = (1 << 8) if uniform01(seed, 6 * r + 2) < 0.5 else (1 << 16)
        zipf = uniform01(seed, 6 * r + 3) < 0.5
        kind = "wt" if uniform01(seed, 6 * r + 4) < 0.5 else "wm"
        out.append((t, n, sg, zipf, kind, (seed * 7919 + r) & (2**63 - 1)))
    return out


def request_text(n: int, sigma: int, zipf: bool, seed: int) -> np.ndarray:
    dt = np.uint8 if sigma <= 256 else np.uint16
    if zipf:
        return zipf_text(n, sigma, 1.0, seed, dt)
    return uniform_text(n, sigma, seed, dt)
