"""CUDA path vs. the oracle, bit-exact word for word (GPU).

Integer and bit work: every word of every level and every Z entry must be equal.
Sizes span several tiles/groups and ragged tails; edge cases cover empty and
one-symbol texts, word and tile boundaries, constant / sorted / reverse-sorted
texts, non-power-of-two alphabets and every storage width.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import first_diff, gpu_wm, gpu_wt

pytestmark = pytest.mark.gpu

TILE8 = 512 * 32          # u8 tile (symbols)
GROUP8 = TILE8 * 4        # symbols per build block for u8
TILE16 = 512 * 16


def _check(T, sigma):
    bw = gpu_wt(T, sigma)
    ew = oracle.wt(T, sigma)
    assert bw.shape == ew.shape
    assert np.array_equal(bw, ew), f"WT differs at {first_diff(bw, ew)}"
    bm, zm = gpu_wm(T, sigma)
    em, ez = oracle.wm(T, sigma)
    assert np.array_equal(bm, em), f"WM differs at {first_diff(bm, em)}"
    assert np.array_equal(zm, ez)


def _dt(sigma):
    return np.uint8 if sigma <= 256 else (np.uint16 if sigma <= 65536 else np.uint32)


def test_worked_example():
    T = np.array([0, 1, 6, 7, 1, 5, 4, 2, 6, 3], dtype=np.uint8)
    _check(T, 8)


@pytest.mark.parametrize("n", [0, 1, 2, 63, 64, 65, 127, 1000, TILE8 - 1, TILE8, TILE8 + 1,
                               GROUP8 - 1, GROUP8, GROUP8 + 1, 3 * GROUP8 + 12345])
def test_lengths_u8_sigma256(n):
    T = synth.uniform_text(n, 256, 100 + n, np.uint8)
    _check(T, 256)


@pytest.mark.parametrize("sigma", [1, 2, 3, 5, 17, 100, 255, 256])
def test_alphabets_u8(sigma):
    T = synth.zipf_text(70001, sigma, 1.0, 7 + sigma, np.uint8) if sigma > 1 else np.zeros(70001, np.uint8)
    _check(T, sigma)


@pytest.mark.parametrize("sigma,dtype", [(257, np.uint16), (4096, np.uint16), (65536, np.uint16),
                                         (300, np.uint32), (1 << 20, np.uint32), (1 << 24, np.uint32)])
def test_large_alphabets(sigma, dtype):
    T = synth.uniform_text(200003, sigma, 11, dtype)
    _check(T, sigma)


@pytest.mark.parametrize("sigma,dtype", [(16, np.uint16), (256, np.uint16), (256, np.uint32),
                                         (16, np.uint32)])
def test_wide_storage_small_alphabet(sigma, dtype):
    T = synth.uniform_text(100000, sigma, 13, dtype)
    _check(T, sigma)


def test_matrix_up_to_32_levels():
    sigma = 1 << 32
    T = synth.uniform_text(50000, 1 << 31, 17, np.uint32)
    T[::7] |= np.uint32(1 << 31)
    bm, zm = gpu_wm(T, sigma)
    em, ez = oracle.wm(T, sigma)
    assert np.array_equal(bm, em) and np.array_equal(zm, ez)


@pytest.mark.parametrize("shape", ["constant", "sorted", "reverse", "alternating", "zeros"])
def test_structured_texts(shape):
    n = 2 * GROUP8 + 777
    if shape == "constant":
        T = np.full(n, 201, np.uint8)
    elif shape == "zeros":
        T = np.zeros(n, np.uint8)
    elif shape == "sorted":
        T = np.sort(synth.uniform_text(n, 256, 3, np.uint8))
    elif shape == "reverse":
        T = np.sort(synth.uniform_text(n, 256, 4, np.uint8))[::-1].copy()
    else:
        T = (np.arange(n) % 2 * 255).astype(np.uint8)
    _check(T, 256)


def test_sorted_large_alphabet_deep_levels():
    n = 300000
    T = np.sort(synth.uniform_text(n, 1 << 20, 5, np.uint32))
    _check(T, 1 << 20)


def test_small_workload_full():
    """n = 2^20 uint8 i.i.d. uniform over 256 symbols, full parity."""
    T, sigma = synth.workload_small()
    _check(T, sigma)


def test_symbol_out_of_range_is_reported():
    import torch

    import paper_1702_07578_gb300 as wtg
    from tests.gpu_util import torch_text
    T = synth.uniform_text(100000, 200, 3, np.uint8)
    T[4321] = 250
    t = torch_text(T)
    ws = torch.empty((wtg.wt_workspace_size(wtg.WT_TREE, 1, t.numel(), 200),), dtype=torch.uint8,
                     device="cuda")
    wtg.wt_build(t, 200, ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2
    wtg.wt_sync_status(ws)          # cleared after being reported


def test_argument_errors_are_immediate():
    import torch

    import paper_1702_07578_gb300 as wtg
    t = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(wtg.WtError):
        wtg.wt_build(t, 0)                    # sigma = 0
    with pytest.raises(wtg.WtError):
        wtg.wt_build(t, 300)                  # does not fit uint8
    with pytest.raises(wtg.WtError):
        wtg.wt_build(t, 1 << 25)              # WT alphabet limit
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(wtg.WtError):
        wtg.wt_build(t, 256, ws=small)        # workspace too small
