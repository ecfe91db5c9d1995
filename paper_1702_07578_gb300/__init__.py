"""Python binding of ``libwt_gb300`` (bottom-up wavelet tree / matrix construction).

Same names as the C ABI in ``include/wt_gb300.h``; these functions only marshal
arguments: PyTorch supplies device memory and streams, every step of the
construction runs in the library's CUDA kernels.  There is no CPU path: if the
library cannot be built or loaded, every call raises.

Bit vectors come back as int64 tensors of shape (L, ceil(n/64)) holding the
uint64 words (bit j of a level is bit j & 63 of word j >> 6).
"""
from __future__ import annotations

import ctypes

from . import _native

WT_TREE, WT_MATRIX = 0, 1
WT_U8, WT_U16, WT_U32 = 1, 2, 4

STATUS = {0: "ok", 1: "invalid argument", 2: "symbol out of range", 3: "out of memory",
          4: "CUDA error", 5: "timeout", 6: "busy", 7: "not found"}


class WtError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


def _check(code, where):
    if code != 0:
        raise WtError(code, where)


def build():
    """Compile the CUDA library (sm_103a) in-tree."""
    return _native.build()


def lib():
    return _native.lib()


def _torch():
    import torch
    return torch


def _symtype(t):
    torch = _torch()
    m = {torch.uint8: WT_U8, torch.int16: WT_U16, torch.int32: WT_U32}
    if hasattr(torch, "uint16"):
        m[torch.uint16] = WT_U16
    if hasattr(torch, "uint32"):
        m[torch.uint32] = WT_U32
    if t.dtype not in m:
        raise TypeError(f"unsupported text dtype {t.dtype}")
    return m[t.dtype]


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def wt_levels(sigma: int) -> int:
    return int(lib().wt_levels(int(sigma)))


def wt_words_per_level(n: int) -> int:
    return int(lib().wt_words_per_level(int(n)))


def wt_status_string(code: int) -> str:
    return lib().wt_status_string(int(code)).decode()


def wt_workspace_size(kind: int, symtype: int, n: int, sigma: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().wt_workspace_size(kind, symtype, int(n), int(sigma), ctypes.byref(out)),
           "wt_workspace_size")
    return out.value


def _alloc(text, sigma, bv, zeros, ws, kind):
    torch = _torch()
    n = text.numel()
    L = wt_levels(sigma)
    W = wt_words_per_level(n)
    dev = text.device
    if bv is None:
        bv = torch.empty((L, W), dtype=torch.int64, device=dev)
    if kind == WT_MATRIX and zeros is None:
        zeros = torch.empty((max(L, 1),), dtype=torch.int64, device=dev)
    if ws is None:
        ws = torch.empty((max(wt_workspace_size(kind, _symtype(text), n, sigma), 1),),
                         dtype=torch.uint8, device=dev)
    return bv, zeros, ws


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


def wt_build(text, sigma: int, bv=None, ws=None, stream=None):
    """Wavelet tree of a device text; returns the (L, W) int64 bit-vector tensor."""
    if not text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA tensor")
    bv, _, ws = _alloc(text, sigma, bv, None, ws, WT_TREE)
    _check(lib().wt_build(_ptr(text), _symtype(text), text.numel(), int(sigma), _ptr(bv), _ptr(ws),
                          ws.numel(), _stream(stream)), "wt_build")
    return bv


def wm_build(text, sigma: int, bv=None, zeros=None, ws=None, stream=None):
    """Wavelet matrix of a device text; returns (bit vectors, Z)."""
    if not text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA tensor")
    bv, zeros, ws = _alloc(text, sigma, bv, zeros, ws, WT_MATRIX)
    _check(lib().wm_build(_ptr(text), _symtype(text), text.numel(), int(sigma), _ptr(bv),
                          _ptr(zeros), _ptr(ws), ws.numel(), _stream(stream)), "wm_build")
    return bv, zeros[:wt_levels(sigma)]


def wt_large_workspace_size(kind: int, symtype: int, n: int, sigma: int, slice_len: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().wt_large_workspace_size(kind, symtype, int(n), int(sigma), int(slice_len), ctypes.byref(out)),
           "wt_large_workspace_size")
    return out.value


def build_large(kind: int, text, sigma: int, slice_len: int = 0, bv=None, zeros=None, ws=None, stream=None):
    """WT or WM of a device text of any length (slices built separately, then merged);
    returns (bit vectors, Z or None)."""
    torch = _torch()
    if not text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA tensor")
    n = text.numel()
    L = wt_levels(sigma)
    dev = text.device
    if bv is None:
        bv = torch.empty((L, wt_words_per_level(n)), dtype=torch.int64, device=dev)
    if kind == WT_MATRIX and zeros is None:
        zeros = torch.empty((max(L, 1),), dtype=torch.int64, device=dev)
    if ws is None:
        ws = torch.empty((max(wt_large_workspace_size(kind, _symtype(text), n, sigma, slice_len), 1),),
                         dtype=torch.uint8, device=dev)
    _check(lib().wt_build_large(kind, _ptr(text), _symtype(text), n, int(sigma), int(slice_len), _ptr(bv),
                                _ptr(zeros), _ptr(ws), ws.numel(), _stream(stream)), "wt_build_large")
    return bv, (zeros[:L] if zeros is not None else None)


def wt_order_workspace_size(kind: int, symtype: int, n: int, sigma: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().wt_order_workspace_size(kind, symtype, int(n), int(sigma), ctypes.byref(out)),
           "wt_order_workspace_size")
    return out.value


def build_order(kind: int, text, sigma: int, sorted_text: bool = True, ws=None, stream=None):
    """WT (kind WT_TREE) or WM (WT_MATRIX) of a device text plus the stable order
    after the last level: returns (bit vectors, Z or None, perm, sorted text or None)."""
    torch = _torch()
    if not text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA tensor")
    n = text.numel()
    L = wt_levels(sigma)
    dev = text.device
    bv = torch.empty((L, wt_words_per_level(n)), dtype=torch.int64, device=dev)
    zeros = torch.empty((max(L, 1),), dtype=torch.int64, device=dev) if kind == WT_MATRIX else None
    perm = torch.empty((n,), dtype=torch.int32, device=dev)
    srt = torch.empty_like(text) if sorted_text else None
    if ws is None:
        ws = torch.empty((max(wt_order_workspace_size(kind, _symtype(text), n, sigma), 1),), dtype=torch.uint8,
                         device=dev)
    if kind == WT_TREE:
        _check(lib().wt_build_order(_ptr(text), _symtype(text), n, int(sigma), _ptr(bv), _ptr(perm), _ptr(srt),
                                    _ptr(ws), ws.numel(), _stream(stream)), "wt_build_order")
    else:
        _check(lib().wm_build_order(_ptr(text), _symtype(text), n, int(sigma), _ptr(bv), _ptr(zeros), _ptr(perm),
                                    _ptr(srt), _ptr(ws), ws.numel(), _stream(stream)), "wm_build_order")
    return bv, (zeros[:L] if zeros is not None else None), perm, srt


def wt_wm_workspace_size(symtype: int, n: int, sigma: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().wt_wm_workspace_size(symtype, int(n), int(sigma), ctypes.byref(out)), "wt_wm_workspace_size")
    return out.value


def wt_wm_build(text, sigma: int, bv_wt=None, bv_wm=None, zeros=None, ws=None, stream=None):
    """WT and WM of the same device text in one call; returns (WT bits, WM bits, Z)."""
    torch = _torch()
    if not text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA tensor")
    n = text.numel()
    L = wt_levels(sigma)
    W = wt_words_per_level(n)
    dev = text.device
    if bv_wt is None:
        bv_wt = torch.empty((L, W), dtype=torch.int64, device=dev)
    if bv_wm is None:
        bv_wm = torch.empty((L, W), dtype=torch.int64, device=dev)
    if zeros is None:
        zeros = torch.empty((max(L, 1),), dtype=torch.int64, device=dev)
    if ws is None:
        ws = torch.empty((max(wt_wm_workspace_size(_symtype(text), n, sigma), 1),), dtype=torch.uint8, device=dev)
    _check(lib().wt_wm_build(_ptr(text), _symtype(text), n, int(sigma), _ptr(bv_wt), _ptr(bv_wm), _ptr(zeros),
                             _ptr(ws), ws.numel(), _stream(stream)), "wt_wm_build")
    return bv_wt, bv_wm, zeros[:L]


_HOST_DUMMY = ctypes.c_uint64(0)      # stands for an empty host output (nothing is written to it)


def _hptr(t):
    """Host pointer of an output that is asked for, even when it has no elements."""
    if t.numel() > 0:
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(ctypes.addressof(_HOST_DUMMY))


def wt_host_workspace_size(symtype: int, n: int, sigma: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().wt_host_workspace_size(symtype, int(n), int(sigma), ctypes.byref(out)), "wt_host_workspace_size")
    return out.value


def wt_build_host(text, sigma: int, wt=True, wm=True, one_pass=False, out_wt=None, out_wm=None, out_zeros=None,
                  ws=None, stream=None):
    """Host text in, host levels out (wt_build_host): returns (WT bits or None, WM bits or None, Z or None).

    text and the outputs are contiguous CPU tensors; page-locked ones make the
    call asynchronous on `stream` (synchronise before reading them)."""
    torch = _torch()
    if text.is_cuda or not text.is_contiguous():
        raise ValueError("text must be a contiguous CPU tensor")
    if not (wt or wm):
        raise ValueError("ask for the WT, the WM or both")
    n = text.numel()
    L = wt_levels(sigma)
    W = wt_words_per_level(n)
    pin = text.is_pinned()
    if wt and out_wt is None:
        out_wt = torch.empty((L, W), dtype=torch.int64, pin_memory=pin)
    if wm and out_wm is None:
        out_wm = torch.empty((L, W), dtype=torch.int64, pin_memory=pin)
    if wm and out_zeros is None:
        out_zeros = torch.empty((max(L, 1),), dtype=torch.int64, pin_memory=pin)
    for o in (out_wt, out_wm, out_zeros):
        if o is not None and (o.is_cuda or not o.is_contiguous()):
            raise ValueError("outputs must be contiguous CPU tensors")
    if ws is None:
        ws = torch.empty((wt_host_workspace_size(_symtype(text), n, sigma),), dtype=torch.uint8, device="cuda")
    _check(lib().wt_build_host(_ptr(text), _symtype(text), n, int(sigma), _hptr(out_wt) if wt else None,
                               _hptr(out_wm) if wm else None, _hptr(out_zeros) if wm else None, 1 if one_pass else 0,
                               _ptr(ws), ws.numel(), _stream(stream)), "wt_build_host")
    return out_wt if wt else None, out_wm if wm else None, out_zeros[:L] if wm else None


def wt_sync_status(ws, stream=None):
    """Synchronise and raise WtError if the device recorded an error in ws."""
    _check(lib().wt_sync_status(_ptr(ws), _stream(stream)), "device")


def _descs(texts, sigmas, bvs, zeros):
    arr = (_native.WtTextDesc * len(texts))()
    for i, t in enumerate(texts):
        arr[i].d_text = t.data_ptr() if t.numel() else 0
        arr[i].n = t.numel()
        arr[i].sigma = int(sigmas[i])
        arr[i].d_bv = bvs[i].data_ptr() if bvs is not None and bvs[i].numel() else 0
        arr[i].d_zeros = zeros[i].data_ptr() if zeros is not None and zeros[i].numel() else 0
    return arr


def wt_batched_workspace_size(kind: int, symtype: int, lengths, sigmas) -> int:
    arr = (_native.WtTextDesc * len(lengths))()
    for i, (n, s) in enumerate(zip(lengths, sigmas)):
        arr[i].n = int(n)
        arr[i].sigma = int(s)
    out = ctypes.c_size_t(0)
    _check(lib().wt_batched_workspace_size(kind, symtype, arr, len(lengths), ctypes.byref(out)),
           "wt_batched_workspace_size")
    return out.value


def wt_build_batched(kind: int, texts, sigmas, bvs=None, zeros=None, ws=None, stream=None):
    """Build many texts in one call.  Returns (bvs, zeros or None)."""
    torch = _torch()
    if not texts:
        return [], ([] if kind == WT_MATRIX else None)
    st = _symtype(texts[0])
    dev = texts[0].device
    if bvs is None:
        bvs = [torch.empty((wt_levels(s), wt_words_per_level(t.numel())), dtype=torch.int64,
                           device=dev) for t, s in zip(texts, sigmas)]
    if kind == WT_MATRIX and zeros is None:
        zeros = [torch.empty((max(wt_levels(s), 1),), dtype=torch.int64, device=dev) for s in sigmas]
    if ws is None:
        sz = wt_batched_workspace_size(kind, st, [t.numel() for t in texts], sigmas)
        ws = torch.empty((max(sz, 1),), dtype=torch.uint8, device=dev)
    arr = _descs(texts, sigmas, bvs, zeros if kind == WT_MATRIX else None)
    _check(lib().wt_build_batched(kind, st, arr, len(texts), _ptr(ws), ws.numel(), _stream(stream)),
           "wt_build_batched")
    return bvs, (zeros if kind == WT_MATRIX else None)


PROFILE_FAMILIES = ("build", "hist", "scan", "jobs")


def wt_profile_enable(on: bool = True):
    lib().wt_profile_enable(1 if on else 0)


def wt_profile_read(reset: bool = False):
    """{family: (milliseconds, launches)} since the last reset (waits for the events)."""
    p = _native.WtProfile()
    _check(lib().wt_profile_read(ctypes.byref(p), 1 if reset else 0), "wt_profile_read")
    return {f: (p.ms[i], int(p.launches[i])) for i, f in enumerate(PROFILE_FAMILIES)}


BOUNDS_SITES = {0: "selftest", 1: "text", 2: "level", 3: "table", 4: "shared", 5: "next"}


def wt_debug_bounds_read(reset: bool = False):
    """Report of the kernels' bounds checks (the WT_DEBUG_BOUNDS build): enabled,
    failures and the first failure's site, index and bound."""
    r = _native.WtBoundsReport()
    _check(lib().wt_debug_bounds_read(ctypes.byref(r), 1 if reset else 0), "wt_debug_bounds_read")
    return {"enabled": bool(r.enabled), "failures": int(r.failures),
            "site": BOUNDS_SITES.get(int(r.site), int(r.site)), "index": int(r.index), "bound": int(r.bound)}


def wt_debug_bounds_selftest(stream=None):
    """One failing and one holding check on the device, with no access behind them."""
    _check(lib().wt_debug_bounds_selftest(_stream(stream)), "wt_debug_bounds_selftest")


class WtServer:
    """Serving loop (wt_server_*): submit host texts, wait, read or keep results on the device."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 64, streams: int = 2,
                 device: int = 0, max_pending: int = 0):
        cfg = _native.WtServerConfig(int(hbm_budget_bytes), int(max_batch), int(streams),
                                     int(device), int(max_pending))
        h = ctypes.c_void_p()
        _check(lib().wt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "wt_server_create")
        self._h = h
        self._keep = {}

    def submit(self, kind: int, text, sigma: int) -> int:
        """Queue a host text.  A numpy array is copied during the call
        (wt_server_submit); a page-locked torch CPU tensor (``pin_memory()``) is
        read in place (wt_server_submit_pinned) and is kept referenced here until
        the request is released."""
        import numpy as np
        if hasattr(text, "is_pinned"):
            if text.device.type != "cpu" or not text.is_pinned() or not text.is_contiguous():
                raise ValueError("a tensor text must be a contiguous page-locked CPU tensor")
            n, width, ptr, fn, keep = text.numel(), text.element_size(), text.data_ptr(), \
                lib().wt_server_submit_pinned, text
        else:
            text = np.ascontiguousarray(text)
            n, width, ptr, fn, keep = text.size, text.dtype.itemsize, text.ctypes.data, \
                lib().wt_server_submit, None
        st = {1: WT_U8, 2: WT_U16, 4: WT_U32}[width]
        req = _native.WtRequest(kind, st, ptr if n else 0, n, int(sigma))
        t = ctypes.c_uint64(0)
        _check(fn(self._h, ctypes.byref(req), ctypes.byref(t)), "wt_server_submit")
        self._keep[t.value] = (kind, n, int(sigma), keep)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        r = _native.WtResult()
        _check(lib().wt_server_wait(self._h, ticket, int(timeout_us), ctypes.byref(r)), "wt_server_wait")
        return {"levels": r.levels, "words_per_level": r.words_per_level, "n": r.n,
                "status": r.status, "latency_us": r.latency_us, "d_bv": r.d_bv, "d_zeros": r.d_zeros}

    def read(self, ticket: int):
        import numpy as np
        kind, n, sigma, _ = self._keep[ticket]
        L = wt_levels(sigma)
        bv = np.zeros((L, wt_words_per_level(n)), dtype=np.uint64)
        z = np.zeros(max(L, 1), dtype=np.uint64)
        _check(lib().wt_server_read(self._h, ticket, ctypes.c_void_p(bv.ctypes.data),
                                    ctypes.c_void_p(z.ctypes.data)), "wt_server_read")
        return bv, (z[:L] if kind == WT_MATRIX else None)

    def release(self, ticket: int):
        _check(lib().wt_server_release(self._h, ticket), "wt_server_release")
        self._keep.pop(ticket, None)

    def stats(self):
        st = _native.WtServerStats()
        _check(lib().wt_server_get_stats(self._h, ctypes.byref(st)), "wt_server_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self._h:
            lib().wt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WtBatchPlan:
    """wt_batch_plan_*: a batched build recorded once into a CUDA graph, then replayed.

    ``stream`` must be a non-default torch.cuda.Stream (graph capture).  The texts,
    outputs and workspace must stay alive while the plan is used.
    """

    def __init__(self, kind, texts, sigmas, bvs, zeros=None, ws=None, stream=None,
                 symbols_per_block=0):
        torch = _torch()
        self.kind = kind
        self.stream = stream if stream is not None else torch.cuda.Stream()
        st = _symtype(texts[0]) if texts else WT_U8
        if ws is None:
            sz = wt_batched_workspace_size(kind, st, [t.numel() for t in texts], sigmas)
            ws = torch.empty((max(sz, 1),), dtype=torch.uint8, device="cuda")
        self.ws = ws
        self._refs = (texts, bvs, zeros)
        arr = _descs(texts, sigmas, bvs, zeros if kind == WT_MATRIX else None)
        h = ctypes.c_void_p()
        _check(lib().wt_batch_plan_create(kind, st, arr, len(texts), int(symbols_per_block),
                                          _ptr(ws), ws.numel(), _stream(self.stream),
                                          ctypes.byref(h)), "wt_batch_plan_create")
        self._h = h
        self._sigmas = list(sigmas)

    @property
    def symbols_per_block(self):
        return int(lib().wt_batch_plan_symbols_per_block(self._h))

    def update(self, texts, bvs, zeros=None):
        self._refs = (texts, bvs, zeros)
        arr = _descs(texts, self._sigmas, bvs, zeros if self.kind == WT_MATRIX else None)
        _check(lib().wt_batch_plan_update(self._h, arr, _stream(self.stream)), "wt_batch_plan_update")

    def launch(self):
        _check(lib().wt_batch_plan_launch(self._h, _stream(self.stream)), "wt_batch_plan_launch")

    def close(self):
        if getattr(self, "_h", None):
            lib().wt_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wt_autotune_batched(kind, texts, sigmas, bvs, zeros=None, ws=None, stream=None):
    """Times the candidate symbols-per-block values on this batch; returns the best."""
    torch = _torch()
    st = _symtype(texts[0])
    if ws is None:
        sz = wt_batched_workspace_size(kind, st, [t.numel() for t in texts], sigmas)
        ws = torch.empty((max(sz, 1),), dtype=torch.uint8, device="cuda")
    arr = _descs(texts, sigmas, bvs, zeros if kind == WT_MATRIX else None)
    best = ctypes.c_uint32(0)
    _check(lib().wt_autotune_batched(kind, st, arr, len(texts), _ptr(ws), ws.numel(), _stream(stream),
                                     ctypes.byref(best)), "wt_autotune_batched")
    return best.value


class WtIndex:
    """access / rank / select on a built WT or WM (wt_rank_support_* and queries).

    ``bv`` (and ``zeros`` for the WM) are the device tensors a build returned; they
    must stay unchanged while the index is used.
    """

    def __init__(self, kind, bv, n, sigma, zeros=None, stream=None):
        torch = _torch()
        self.kind, self.bv, self.zeros, self.n, self.sigma = kind, bv, zeros, int(n), int(sigma)
        size = ctypes.c_size_t(0)
        _check(lib().wt_rank_support_size(kind, self.n, self.sigma, ctypes.byref(size)),
               "wt_rank_support_size")
        self.rs = torch.empty((max(size.value, 1),), dtype=torch.uint8, device=bv.device)
        _check(lib().wt_rank_support_build(kind, _ptr(bv), _ptr(zeros), self.n, self.sigma,
                                           _ptr(self.rs), self.rs.numel(), _stream(stream)),
               "wt_rank_support_build")

    def _common(self):
        return (self.kind, _ptr(self.bv), _ptr(self.zeros), _ptr(self.rs), self.n, self.sigma)

    def access(self, pos, stream=None):
        torch = _torch()
        out = torch.empty(pos.numel(), dtype=torch.int32, device=pos.device)
        _check(lib().wt_access(*self._common(), _ptr(pos), pos.numel(), _ptr(out), _stream(stream)),
               "wt_access")
        return out

    def rank(self, sym, pos, stream=None):
        torch = _torch()
        out = torch.empty(pos.numel(), dtype=torch.int64, device=pos.device)
        _check(lib().wt_rank(*self._common(), _ptr(sym), _ptr(pos), pos.numel(), _ptr(out),
                             _stream(stream)), "wt_rank")
        return out

    def select(self, sym, j, stream=None):
        torch = _torch()
        out = torch.empty(j.numel(), dtype=torch.int64, device=j.device)
        _check(lib().wt_select(*self._common(), _ptr(sym), _ptr(j), j.numel(), _ptr(out),
                               _stream(stream)), "wt_select")
        return out


class WtToWmMap:
    """Lemma 3: position i of WT level l -> position j of WM level l (wt_wt2wm_*).

    Built from a WT's ``WtIndex`` (its bit vectors and rank support, which must
    stay unchanged while the map is built).
    """

    def __init__(self, index, stream=None):
        torch = _torch()
        if index.kind != WT_TREE:
            raise ValueError("WtToWmMap needs the rank support of a wavelet tree")
        self.n, self.sigma = index.n, index.sigma
        size = ctypes.c_size_t(0)
        _check(lib().wt_wt2wm_size(self.n, self.sigma, ctypes.byref(size)), "wt_wt2wm_size")
        self.map = torch.empty((max(size.value, 1),), dtype=torch.uint8, device=index.bv.device)
        _check(lib().wt_wt2wm_build(_ptr(index.bv), _ptr(index.rs), self.n, self.sigma, _ptr(self.map),
                                    self.map.numel(), _stream(stream)), "wt_wt2wm_build")

    def __call__(self, level, pos, stream=None):
        torch = _torch()
        if level.numel() != pos.numel():
            raise ValueError("level and pos must have the same length")
        out = torch.empty(pos.numel(), dtype=torch.int64, device=pos.device)
        _check(lib().wt_wt2wm(_ptr(self.map), self.n, self.sigma, _ptr(level), _ptr(pos), pos.numel(),
                              _ptr(out), _stream(stream)), "wt_wt2wm")
        return out
