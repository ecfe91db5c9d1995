"""Build blocks of several tiles: a block builds a group of consecutive tiles of a
job, and a word of a level shared by two tiles' runs of one class is finished by
the later tile.  Texts built with fixed symbols-per-block values (1 to 8 tiles per
block) must equal the oracle bit for bit, including classes that are empty in many
tiles, runs shorter than a word spread over several tiles, and ragged last groups."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_u64, torch_text

pytestmark = pytest.mark.gpu

TILE = 32768


def _text(n, sigma, dist, seed, dtype):
    if dist == "zipf":
        return synth.zipf_text(n, sigma, 1.0, seed, dtype)
    if dist == "uniform":
        return synth.uniform_text(n, sigma, seed, dtype)
    if dist == "lowtail":
        # the last tile holds only the lower half of the alphabet: at every level
        # below the first, the last interval's class (all ones) is empty there and
        # its run ends at n inside an earlier tile of the last group
        T = synth.uniform_text(n, sigma, seed, dtype)
        k = (n - 1) // TILE * TILE
        T[k:] = synth.uniform_text(n - k, max(1, sigma // 2), seed + 1, dtype)
        return T
    # half uniform, then a long run of one symbol, then sparse rare symbols: most
    # classes are empty in many consecutive tiles
    T = synth.uniform_text(n, sigma, seed, dtype)
    T[n // 3: 2 * n // 3] = sigma // 3
    tail = T[2 * n // 3:]
    tail[:] = sigma - 1
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, tail.size, size=max(1, tail.size // 5000))
    tail[pos] = rng.integers(0, sigma, size=pos.size).astype(dtype)
    return T


CASES = [
    (1_000_003, 256, "zipf", np.uint8),
    (300_000, 256, "uniform", np.uint8),
    (700_001, 256, "runs", np.uint8),
    (500_001, 16, "zipf", np.uint8),
    (200_000, 2, "uniform", np.uint8),
    (400_003, 4096, "zipf", np.uint16),
    (262_144, 97, "zipf", np.uint8),
    (3 * 32768 + 1000, 256, "lowtail", np.uint8),
    (6 * 32768 + 77, 256, "lowtail", np.uint16),
    (5 * 32768 + 4001, 4096, "lowtail", np.uint16),
]


@pytest.mark.parametrize("spb", [TILE * 2, TILE * 3, TILE * 4, TILE * 8])
@pytest.mark.parametrize("n,sigma,dist,dtype", CASES)
@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_groups_match_oracle(kind, n, sigma, dist, dtype, spb):
    import torch

    import paper_1702_07578_gb300 as wtg
    T = _text(n, sigma, dist, 11 + n % 97, dtype)
    t = torch_text(T)
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    L = wtg.wt_levels(sigma)
    bv = torch.full((L, wtg.wt_words_per_level(n)), -1, dtype=torch.int64, device="cuda")   # stale bits everywhere
    z = torch.full((max(L, 1),), -1, dtype=torch.int64, device="cuda")
    plan = wtg.WtBatchPlan(k, [t], [sigma], [bv], [z] if kind == "wm" else None, symbols_per_block=spb)
    assert plan.symbols_per_block == spb
    plan.launch()
    plan.stream.synchronize()
    wtg.wt_sync_status(plan.ws, stream=plan.stream)
    got = to_u64(bv)
    if kind == "wt":
        exp = oracle.wt(T, sigma)
    else:
        exp, ez = oracle.wm(T, sigma)
        assert np.array_equal(z[:L].cpu().numpy().astype(np.uint64), ez)
    bad = np.argwhere(got != exp)
    assert bad.size == 0, f"first differing (level, word): {tuple(bad[0])}"
    plan.close()
