"""wt_build_static_ws: the wavelet tree build for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Called through
the C ABI and compared word for word with wt_build on the same texts, twice in a
row (the shared scratch keeps the previous call's contents, which must not leak
into the next result).  Collected last so a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _static_build(t, sigma, bv):
    import torch

    import paper_1702_07578_gb300 as wtg
    rc = wtg.lib().wt_build_static_ws(ctypes.c_void_p(t.data_ptr()), t.element_size(), t.numel(),
                                       sigma, ctypes.c_void_p(bv.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_static_scratch_build_matches_wt_build_twice():
    import torch

    import paper_1702_07578_gb300 as wtg
    from tests.gpu_util import torch_text
    cases = [(synth.zipf_text(3_000_001, 256, 1.0, 21, np.uint8), 256),
             (synth.uniform_text(1_000_003, 200, 22, np.uint8), 200)]
    for T, sigma in cases:
        t = torch_text(T)
        ref = wtg.wt_build(t, sigma)
        for _ in range(2):
            bv = torch.full_like(ref, -1)
            assert _static_build(t, sigma, bv) == 0
            torch.cuda.synchronize()
            assert torch.equal(bv, ref)


def test_static_scratch_rejects_texts_beyond_capacity():
    import torch

    import paper_1702_07578_gb300 as wtg
    n = 1 << 26                       # needs more than the 1 MiB scratch
    t = torch.zeros(n, dtype=torch.uint8, device="cuda")
    bv = torch.empty((8, n // 64), dtype=torch.int64, device="cuda")
    assert _static_build(t, 256, bv) == 3       # WT_ERR_OUT_OF_MEMORY, nothing launched
