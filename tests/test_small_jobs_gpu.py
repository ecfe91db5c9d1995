"""Small jobs at the edges of their kernels: jobs of at most 256 symbols are built
by one thread each, jobs of 257 to 1024 and of 1025 to 4096 symbols by one warp in
the one-row and four-row instantiations, larger ones by the tile kernel.  Wavelet
trees whose second round has subtrees of exactly 1, 255, 256, 257, 1024, 1025, 4096
and 4097 symbols, single-round texts of 1 to 8 levels with at most 256 symbols, both
kinds (the WM's Z too), must equal the oracle bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_wm, gpu_wt

pytestmark = pytest.mark.gpu


def _subtree_text(sizes, low_bits, seed):
    """A text whose first-round classes (the top code bits above low_bits) have the
    given sizes: class c holds sizes[c] symbols, mixed in a seeded random order."""
    rng = np.random.default_rng(seed)
    parts = [(c << low_bits) + rng.integers(0, 1 << low_bits, size=k) for c, k in enumerate(sizes)]
    T = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    rng.shuffle(T)
    return T.astype(np.uint16 if len(sizes) << low_bits <= 1 << 16 else np.uint32)


# the short round goes first, so a text of L = r0 + 8 levels has 2^r0 subtrees in its
# last round, each one job: their sizes are the sizes of the r0-bit classes
CASES = [
    (4, [1, 255, 256, 257, 1024, 1025, 4096, 4097, 0, 3, 2000, 7, 7, 7, 128, 4095]),
    (1, [256, 257]),
    (1, [1, 4096]),
    (2, [0, 0, 256, 0]),
]


@pytest.mark.parametrize("r0,sizes", CASES)
def test_wt_subtrees_at_kernel_edges(r0, sizes):
    assert len(sizes) == 1 << r0
    sigma = 1 << (r0 + 8)
    T = _subtree_text(sizes, 8, 100 + r0 + len(sizes))
    assert T.size == sum(sizes)
    assert np.array_equal(gpu_wt(T, sigma), oracle.wt(T, sigma))
    bm, z = gpu_wm(T, sigma)
    em, ez = oracle.wm(T, sigma)
    assert np.array_equal(bm, em) and np.array_equal(z, ez)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 255, 256])
@pytest.mark.parametrize("sigma", [2, 3, 16, 200, 256])
def test_tiny_texts_both_kinds(n, sigma):
    T = synth.uniform_text(n, sigma, 7 * n + sigma, np.uint8)
    assert np.array_equal(gpu_wt(T, sigma), oracle.wt(T, sigma))
    bm, z = gpu_wm(T, sigma)
    em, ez = oracle.wm(T, sigma)
    assert np.array_equal(bm, em)
    assert np.array_equal(z, ez)


def test_many_tiny_subtrees_of_a_large_alphabet():
    # 65536 symbols over 2^16: 256 subtrees of about 256 symbols each, on both sides of
    # the one-thread limit; a skewed text adds subtrees of a few symbols
    for seed, gen in ((1, "uniform"), (2, "zipf")):
        T = (synth.uniform_text(65536, 1 << 16, seed, np.uint16) if gen == "uniform"
             else synth.zipf_text(65536, 1 << 16, 1.2, seed, np.uint16))
        assert np.array_equal(gpu_wt(T, 1 << 16), oracle.wt(T, 1 << 16)), gen
        bm, z = gpu_wm(T, 1 << 16)
        em, ez = oracle.wm(T, 1 << 16)
        assert np.array_equal(bm, em) and np.array_equal(z, ez), gen


def _status_after_build(kind, T, sigma):
    import torch

    import paper_1702_07578_gb300 as wtg
    from tests.gpu_util import torch_text
    t = torch_text(T)
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    ws = torch.empty((wtg.wt_workspace_size(k, T.dtype.itemsize, t.numel(), sigma),), dtype=torch.uint8,
                     device="cuda")
    if kind == "wt":
        wtg.wt_build(t, sigma, ws=ws)
    else:
        wtg.wm_build(t, sigma, ws=ws)
    try:
        wtg.wt_sync_status(ws)
        first = 0
    except wtg.WtError as e:
        first = e.code
    wtg.wt_sync_status(ws)                 # cleared after being reported
    return first


@pytest.mark.parametrize("n", [100, 256, 1000, 3000])
@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_small_text_symbol_out_of_range_is_reported(kind, n):
    """Texts of at most 4096 symbols in one round are built by the small-job kernels
    alone (no histogram pass): they report a symbol >= sigma too."""
    T = synth.uniform_text(n, 200, 5 + n, np.uint8)
    assert _status_after_build(kind, T, 200) == 0
    T[n // 2] = 230
    assert _status_after_build(kind, T, 200) == 2


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_small_text_beyond_the_code_bits_is_reported(kind):
    """A 16-bit stored text over sigma = 16 with a value of 300: beyond the 4 code
    bits, so out of range, though its low byte would be a valid class."""
    T = synth.uniform_text(500, 16, 9, np.uint16)
    T[123] = 300
    assert _status_after_build(kind, T, 16) == 2
