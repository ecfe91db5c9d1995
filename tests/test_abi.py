"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/wt_gb300.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import paper_1702_07578_gb300 as wtg
from paper_1702_07578_gb300 import _native

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "wt_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\b((?:wt|wm)_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("wt_build", "wm_build", "wt_build_batched", "wt_workspace_size",
                 "wt_server_create", "wt_server_submit", "wt_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = _native.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    assert set(declared_functions()) <= exported
    assert set(_native.SIGNATURES) == set(declared_functions())


def test_host_only_calls():
    assert wtg.wt_levels(1) == 0 and wtg.wt_levels(2) == 1 and wtg.wt_levels(256) == 8
    assert wtg.wt_levels(257) == 9 and wtg.wt_levels(1 << 20) == 20
    assert wtg.wt_words_per_level(0) == 0 and wtg.wt_words_per_level(65) == 2
    assert wtg.wt_status_string(2) == "symbol out of range"
    assert wtg.wt_workspace_size(wtg.WT_TREE, wtg.WT_U8, 1 << 20, 256) > 0
    import pytest
    with pytest.raises(wtg.WtError):
        wtg.wt_workspace_size(wtg.WT_TREE, wtg.WT_U8, 10, 0)
    with pytest.raises(wtg.WtError):
        wtg.wt_workspace_size(wtg.WT_TREE, wtg.WT_U8, 10, 300)
    with pytest.raises(wtg.WtError):
        wtg.wt_workspace_size(wtg.WT_TREE, wtg.WT_U32, 10, 1 << 25)
    assert wtg.wt_workspace_size(wtg.WT_MATRIX, wtg.WT_U32, 10, 1 << 32) > 0
    sz = wtg.wt_batched_workspace_size(wtg.WT_TREE, wtg.WT_U16, [1000, 5000], [16, 65536])
    assert sz > 0


def test_compiled_for_sm103a_only():
    """The build uses exactly one -gencode, for sm_103a."""
    assert _native.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


def test_host_build_argument_errors():
    """wt_build_host rejects bad arguments before it touches the device."""
    lib = wtg.lib()
    n, sigma = 100000, 256
    need = wtg.wt_host_workspace_size(wtg.WT_U8, n, sigma)
    text_bytes = n
    levels = 8 * ((n + 63) // 64) * 8
    # the build workspace, the text, two sets of levels and Z, each 256-byte aligned
    assert need >= wtg.wt_wm_workspace_size(wtg.WT_U8, n, sigma) + text_bytes + 2 * levels + 64
    assert wtg.wt_host_workspace_size(wtg.WT_U32, n, 1 << 25) > 0      # the WM alone may be asked for
    buf = (ctypes.c_uint8 * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    fake_ws = ctypes.c_void_p(1 << 40)        # never dereferenced: every call below fails first
    call = lib.wt_build_host
    assert call(p, wtg.WT_U8, n, sigma, None, None, None, 0, fake_ws, need, None) == 1     # no output
    assert call(p, wtg.WT_U8, n, sigma, p, None, None, 0, None, need, None) == 1           # no workspace
    assert call(p, wtg.WT_U8, n, sigma, p, None, None, 0, fake_ws, need - 1, None) == 3    # workspace short
    assert call(None, wtg.WT_U8, n, sigma, p, None, None, 0, fake_ws, need, None) == 1     # no text
    assert call(p, wtg.WT_U8, n, sigma, None, p, None, 0, fake_ws, need, None) == 1        # WM without Z
    assert call(p, wtg.WT_U8, n, 300, p, None, None, 0, fake_ws, need, None) == 1          # sigma > 2^8
    big = wtg.wt_host_workspace_size(wtg.WT_U32, n, 1 << 25)
    assert call(p, wtg.WT_U32, n, 1 << 25, p, None, None, 0, fake_ws, big, None) == 1      # WT beyond 2^24


def test_bounds_report_of_the_default_build():
    """The default build compiles no bounds checks: the report says so and the
    self-test is refused, both without touching a device."""
    r = wtg.wt_debug_bounds_read()
    assert r == {"enabled": False, "failures": 0, "site": "selftest", "index": 0, "bound": 0}
    assert wtg.lib().wt_debug_bounds_selftest(None) == 1


def test_bounds_checked_build_compiles_and_exports_the_boundary():
    path = _native.build(debug_bounds=True)
    assert path == _native.LIB_PATH_DBG and path != _native.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(declared_functions()) <= set(re.findall(r"\bT\s+(\w+)", out))
