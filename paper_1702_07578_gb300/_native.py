"""Build and load the in-tree CUDA library ``libwt_gb300.so`` (sm_103a).

``build()`` compiles every ``csrc/*.cu`` with nvcc (one -gencode, in parallel)
and links them into ``_build/libwt_gb300.so``.  ``lib()`` loads it with ctypes
and declares the C ABI of ``include/wt_gb300.h``.  There is no fallback: if the
library is missing or fails to load, every call raises.

With ``WT_DEBUG_BOUNDS=1`` in the environment (or ``build(debug_bounds=True)``)
the same sources are compiled with ``-DWT_DEBUG_BOUNDS`` into
``_build_dbg/libwt_gb300_dbg.so``, the build whose construction kernels check
their indexes (``wt_debug_bounds_read``), and ``lib()`` loads that one.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT, "libwt_gb300.so")
OUT_DBG = os.path.join(HERE, "_build_dbg")
LIB_PATH_DBG = os.path.join(OUT_DBG, "libwt_gb300_dbg.so")
DEBUG_ENV = "WT_DEBUG_BOUNDS"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = _sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    files.append(os.path.join(INCLUDE, "wt_gb300.h"))
    return files


def _debug_wanted(debug_bounds):
    return os.environ.get(DEBUG_ENV) == "1" if debug_bounds is None else bool(debug_bounds)


def _stale(lib_path):
    if not os.path.exists(lib_path):
        return True
    t = os.path.getmtime(lib_path)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, debug_bounds=None) -> str:
    """Compile the library for sm_103a (no-op when up to date).  debug_bounds:
    the build with the kernels' bounds checks (None: the environment decides)."""
    debug = _debug_wanted(debug_bounds)
    out_dir, lib_path = (OUT_DBG, LIB_PATH_DBG) if debug else (OUT, LIB_PATH)
    with _lock:
        if not force and not _stale(lib_path):
            return lib_path
        os.makedirs(out_dir, exist_ok=True)
        nvcc = _nvcc()
        common = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "--expt-relaxed-constexpr", "-I", INCLUDE]
        if debug:
            common += ["-DWT_DEBUG_BOUNDS"]
        if verbose:
            common += ["-Xptxas", "-v"]

        def compile_one(src):
            obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
            r = subprocess.run([nvcc, *common, "-c", src, "-o", obj],
                               capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            return obj, r.stderr

        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(compile_one, _sources()))
        objs = [o for o, _ in results]
        if verbose:
            for _, err in results:
                print(err)
        tmp = lib_path + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                            "-lpthread"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib_path)
        return lib_path


class WtTextDesc(ctypes.Structure):
    _fields_ = [("d_text", ctypes.c_void_p), ("n", ctypes.c_uint64), ("sigma", ctypes.c_uint64),
                ("d_bv", ctypes.c_void_p), ("d_zeros", ctypes.c_void_p)]


class WtServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_uint32),
                ("streams", ctypes.c_uint32), ("device", ctypes.c_int),
                ("max_pending", ctypes.c_uint32)]


class WtRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("type", ctypes.c_int), ("h_text", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("sigma", ctypes.c_uint64)]


class WtResult(ctypes.Structure):
    _fields_ = [("d_bv", ctypes.c_void_p), ("d_zeros", ctypes.c_void_p), ("levels", ctypes.c_uint32),
                ("words_per_level", ctypes.c_uint64), ("n", ctypes.c_uint64),
                ("status", ctypes.c_int), ("latency_us", ctypes.c_double)]


class WtServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("in_flight", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("symbols_per_s", ctypes.c_double), ("hbm_in_use", ctypes.c_size_t)]


class WtProfile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_uint64 * 4)]


class WtBoundsReport(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_uint32), ("failures", ctypes.c_uint32), ("site", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("index", ctypes.c_uint64), ("bound", ctypes.c_uint64)]


# name -> (restype, argtypes); must cover every function of include/wt_gb300.h
_C = ctypes
SIGNATURES = {
    "wt_levels": (_C.c_uint32, [_C.c_uint64]),
    "wt_words_per_level": (_C.c_uint64, [_C.c_uint64]),
    "wt_status_string": (_C.c_char_p, [_C.c_int]),
    "wt_workspace_size": (_C.c_int, [_C.c_int, _C.c_int, _C.c_uint64, _C.c_uint64,
                                     _C.POINTER(_C.c_size_t)]),
    "wt_build": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p,
                            _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wm_build": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p,
                            _C.c_void_p, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_sync_status": (_C.c_int, [_C.c_void_p, _C.c_void_p]),
    "wt_batched_workspace_size": (_C.c_int, [_C.c_int, _C.c_int, _C.POINTER(WtTextDesc),
                                             _C.c_uint32, _C.POINTER(_C.c_size_t)]),
    "wt_build_batched": (_C.c_int, [_C.c_int, _C.c_int, _C.POINTER(WtTextDesc), _C.c_uint32,
                                    _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_server_create": (_C.c_int, [_C.POINTER(WtServerConfig), _C.POINTER(_C.c_void_p)]),
    "wt_server_submit": (_C.c_int, [_C.c_void_p, _C.POINTER(WtRequest), _C.POINTER(_C.c_uint64)]),
    "wt_server_submit_pinned": (_C.c_int, [_C.c_void_p, _C.POINTER(WtRequest), _C.POINTER(_C.c_uint64)]),
    "wt_server_wait": (_C.c_int, [_C.c_void_p, _C.c_uint64, _C.c_int64, _C.POINTER(WtResult)]),
    "wt_server_release": (_C.c_int, [_C.c_void_p, _C.c_uint64]),
    "wt_server_read": (_C.c_int, [_C.c_void_p, _C.c_uint64, _C.c_void_p, _C.c_void_p]),
    "wt_server_get_stats": (_C.c_int, [_C.c_void_p, _C.POINTER(WtServerStats)]),
    "wt_server_destroy": (None, [_C.c_void_p]),
    "wt_build_static_ws": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64,
                                      _C.c_void_p, _C.c_void_p]),
    "wt_batch_plan_create": (_C.c_int, [_C.c_int, _C.c_int, _C.POINTER(WtTextDesc), _C.c_uint32,
                                        _C.c_uint32, _C.c_void_p, _C.c_size_t, _C.c_void_p,
                                        _C.POINTER(_C.c_void_p)]),
    "wt_batch_plan_update": (_C.c_int, [_C.c_void_p, _C.POINTER(WtTextDesc), _C.c_void_p]),
    "wt_batch_plan_launch": (_C.c_int, [_C.c_void_p, _C.c_void_p]),
    "wt_batch_plan_symbols_per_block": (_C.c_uint32, [_C.c_void_p]),
    "wt_batch_plan_destroy": (None, [_C.c_void_p]),
    "wt_autotune_batched": (_C.c_int, [_C.c_int, _C.c_int, _C.POINTER(WtTextDesc), _C.c_uint32,
                                       _C.c_void_p, _C.c_size_t, _C.c_void_p,
                                       _C.POINTER(_C.c_uint32)]),
    "wt_rank_support_size": (_C.c_int, [_C.c_int, _C.c_uint64, _C.c_uint64, _C.POINTER(_C.c_size_t)]),
    "wt_rank_support_build": (_C.c_int, [_C.c_int, _C.c_void_p, _C.c_void_p, _C.c_uint64, _C.c_uint64,
                                         _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_access": (_C.c_int, [_C.c_int, _C.c_void_p, _C.c_void_p, _C.c_void_p, _C.c_uint64, _C.c_uint64,
                             _C.c_void_p, _C.c_uint32, _C.c_void_p, _C.c_void_p]),
    "wt_rank": (_C.c_int, [_C.c_int, _C.c_void_p, _C.c_void_p, _C.c_void_p, _C.c_uint64, _C.c_uint64,
                           _C.c_void_p, _C.c_void_p, _C.c_uint32, _C.c_void_p, _C.c_void_p]),
    "wt_select": (_C.c_int, [_C.c_int, _C.c_void_p, _C.c_void_p, _C.c_void_p, _C.c_uint64, _C.c_uint64,
                             _C.c_void_p, _C.c_void_p, _C.c_uint32, _C.c_void_p, _C.c_void_p]),
    "wt_large_workspace_size": (_C.c_int, [_C.c_int, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_uint64,
                                           _C.POINTER(_C.c_size_t)]),
    "wt_build_large": (_C.c_int, [_C.c_int, _C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_uint64,
                                  _C.c_void_p, _C.c_void_p, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_order_workspace_size": (_C.c_int, [_C.c_int, _C.c_int, _C.c_uint64, _C.c_uint64,
                                           _C.POINTER(_C.c_size_t)]),
    "wt_build_order": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p, _C.c_void_p,
                                  _C.c_void_p, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wm_build_order": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p, _C.c_void_p,
                                  _C.c_void_p, _C.c_void_p, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_wm_workspace_size": (_C.c_int, [_C.c_int, _C.c_uint64, _C.c_uint64, _C.POINTER(_C.c_size_t)]),
    "wt_wm_build": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p, _C.c_void_p,
                               _C.c_void_p, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_host_workspace_size": (_C.c_int, [_C.c_int, _C.c_uint64, _C.c_uint64, _C.POINTER(_C.c_size_t)]),
    "wt_build_host": (_C.c_int, [_C.c_void_p, _C.c_int, _C.c_uint64, _C.c_uint64, _C.c_void_p, _C.c_void_p,
                                 _C.c_void_p, _C.c_int, _C.c_void_p, _C.c_size_t, _C.c_void_p]),
    "wt_wt2wm_size": (_C.c_int, [_C.c_uint64, _C.c_uint64, _C.POINTER(_C.c_size_t)]),
    "wt_wt2wm_build": (_C.c_int, [_C.c_void_p, _C.c_void_p, _C.c_uint64, _C.c_uint64, _C.c_void_p,
                                  _C.c_size_t, _C.c_void_p]),
    "wt_wt2wm": (_C.c_int, [_C.c_void_p, _C.c_uint64, _C.c_uint64, _C.c_void_p, _C.c_void_p, _C.c_uint32,
                            _C.c_void_p, _C.c_void_p]),
    "wt_profile_enable": (None, [_C.c_int]),
    "wt_profile_read": (_C.c_int, [_C.POINTER(WtProfile), _C.c_int]),
    "wt_debug_bounds_read": (_C.c_int, [_C.POINTER(WtBoundsReport), _C.c_int]),
    "wt_debug_bounds_selftest": (_C.c_int, [_C.c_void_p]),
}


def lib():
    """The loaded library (built first if needed).  Raises if it cannot load."""
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib
