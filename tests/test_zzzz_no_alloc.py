"""wt_build_static_ws: the wavelet tree build for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Called through
the C ABI and compared word for word with wt_build and with the oracle on the same
texts, twice in a row (the shared scratch keeps the previous call's contents, which
must not leak into the next result), at the largest accepted sizes, and with the
first sizes past the capacity rejected.  The file name sorts after every other test
file, so pytest collects it last and a failure here comes after every other test
has run."""
import ctypes

import numpy as np
import pytest

import oracle
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


# largest accepted text per alphabet: wt_workspace_size(WT_TREE, ...) <= 1 MiB
EDGES = [(11_010_048, 256, np.uint8), (948_736, 257, np.uint16), (882_688, 4096, np.uint16)]


@pytest.mark.parametrize("n,sigma,dtype", EDGES)
def test_static_scratch_edge_sizes_match_oracle_twice(n, sigma, dtype):
    """The largest text that fits (one round for bytes, two rounds with a re-sorted
    text in the scratch for the larger alphabets), twice in a row, against the
    oracle and against wt_build; one symbol more is rejected."""
    import torch

    import paper_1702_07578_gb300 as wtg
    from tests.gpu_util import torch_text
    assert wtg.wt_workspace_size(wtg.WT_TREE, np.dtype(dtype).itemsize, n, sigma) <= 1 << 20
    assert wtg.wt_workspace_size(wtg.WT_TREE, np.dtype(dtype).itemsize, n + 1, sigma) > 1 << 20
    T = synth.zipf_text(n, sigma, 1.0, 23 + sigma, dtype)
    t = torch_text(T)
    exp = oracle.wt(T, sigma)
    ref = wtg.wt_build(t, sigma)
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy().view(np.uint64), exp)
    for _ in range(2):
        bv = torch.full_like(ref, -1)
        assert _static_build(t, sigma, bv) == 0
        torch.cuda.synchronize()
        assert np.array_equal(bv.cpu().numpy().view(np.uint64), exp)
    t1 = torch_text(np.concatenate([T, T[:1]]))
    bv1 = torch.empty((wtg.wt_levels(sigma), wtg.wt_words_per_level(n + 1)), dtype=torch.int64, device="cuda")
    assert _static_build(t1, sigma, bv1) == 3   # WT_ERR_OUT_OF_MEMORY


def test_static_scratch_rejects_three_round_alphabets():
    """sigma = 2^17 (three rounds) needs more than the array for any text."""
    import torch

    import paper_1702_07578_gb300 as wtg
    t = torch.zeros(1000, dtype=torch.int32, device="cuda")
    bv = torch.empty((17, 16), dtype=torch.int64, device="cuda")
    assert _static_build(t, 1 << 17, bv) == 3
