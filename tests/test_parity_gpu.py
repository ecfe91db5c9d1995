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

TILE = 512 * 2 * 32       # symbols per tile of the split kernel (512 threads x 2 words x 32)
GROUP = 2 * TILE          # symbols per build block (default)
SMALL = 4096              # largest job built by one warp


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


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 63, 64, 65, 127, 1000, SMALL - 1, SMALL, SMALL + 1,
                               TILE - 1, TILE, TILE + 1, GROUP - 1, GROUP, GROUP + 1, 3 * GROUP + 12345])
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
    n = 2 * GROUP + 777
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


def _random_text(rng, n, sigma, dtype):
    kind = int(rng.integers(0, 4))
    if kind == 0:
        return synth.uniform_text(n, sigma, int(rng.integers(1, 1 << 30)), dtype)
    if kind == 1:
        return synth.zipf_text(n, sigma, float(rng.uniform(0.5, 1.5)), int(rng.integers(1, 1 << 30)), dtype)
    if kind == 2:                                    # long runs of equal symbols
        runs = rng.integers(1, 5000, size=max(1, n // 100))
        vals = rng.integers(0, sigma, size=runs.size)
        return np.resize(np.repeat(vals, runs), n).astype(dtype)
    return (np.arange(n, dtype=np.int64) * int(rng.integers(1, 97)) % sigma).astype(dtype)   # periodic


@pytest.mark.parametrize("seed", range(8))
def test_random_shapes(seed):
    """Seeded sweep: lengths around tile and group edges and in between, alphabets
    from 2 to 2^20 (one to three rounds), every storage width that holds them,
    uniform / Zipf / long runs / periodic texts."""
    rng = np.random.default_rng(9000 + seed)
    edges = [SMALL, TILE, GROUP, 2 * GROUP, 5 * TILE]
    for _ in range(5):
        if rng.random() < 0.5:
            n = int(rng.choice(edges)) + int(rng.integers(-3, 4))
        else:
            n = int(rng.integers(0, 400000))
        sigma = int(rng.choice([2, 3, 7, 64, 200, 256, 257, 1000, 4096, 40000, 65536, 1 << 18, 1 << 20]))
        widths = [np.uint8, np.uint16, np.uint32]
        ok = [w for w in widths if sigma <= (1 << (8 * np.dtype(w).itemsize))]
        dtype = ok[int(rng.integers(0, len(ok)))]
        T = _random_text(rng, max(n, 0), sigma, dtype)
        _check(T, sigma)
