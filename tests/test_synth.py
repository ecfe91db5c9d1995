"""The seeded generators: determinism, thread independence, distribution shape."""
import numpy as np

import synth


def test_splitmix64_published_values():
    # SplitMix64 seeded with 0: first outputs of the published generator
    assert synth.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert synth.splitmix64(0, 1) == 0x6E789E6AA1B965F4


def test_thread_count_does_not_change_bytes():
    lib = synth._load()
    a = np.empty(300000, np.uint8)
    b = np.empty(300000, np.uint8)
    lib.synth_zipf(9, 10, a.size, 256, 1.0, a.ctypes.data, 1, 1)
    lib.synth_zipf(9, 10, b.size, 256, 1.0, b.ctypes.data, 1, 7)
    assert np.array_equal(a, b)


def test_zipf_skew_and_range():
    T = synth.zipf_text(1 << 20, 256, 1.0, 3, np.uint8)
    c = np.bincount(T, minlength=256)
    assert 0.15 < c.max() / T.size < 0.18      # 1 / H_256 = 0.163
    assert (c > 0).sum() == 256


def test_markov_half_has_64_successors():
    T = synth.uniform_markov_text(1 << 16, 1 << 20, 5, np.uint32)
    assert T.max() < (1 << 20)
    tail = T[(1 << 15):]
    succ = {}
    for x, y in zip(tail[:-1].tolist(), tail[1:].tolist()):
        succ.setdefault(x, set()).add(y)
    assert max(len(s) for s in succ.values()) <= 64


def test_batch_specs_ranges():
    specs = synth.batch_specs(500)
    assert all(1024 <= n <= (1 << 20) for n, _, _ in specs)
    assert {s for _, s, _ in specs} == {16, 256, 4096, 65536}
