"""Stable order as a by-product (wt_build_order / wm_build_order): the permutation
and the sorted text equal the oracle's stable order, and the levels equal the
oracle's, for one, two and three rounds, ragged tiles and tiny jobs."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_u64, torch_text

pytestmark = pytest.mark.gpu


def _text(n, sigma, dtype, seed):
    if sigma == 1:
        return np.zeros(n, dtype)
    return synth.zipf_text(n, sigma, 1.0, seed, dtype)


@pytest.mark.parametrize("kind", ["wt", "wm"])
@pytest.mark.parametrize("n,sigma,dtype", [
    (1, 2, np.uint8), (1000, 3, np.uint8), (4096, 256, np.uint8), (100003, 256, np.uint8),
    (32768 * 2 + 5, 97, np.uint8), (70001, 4096, np.uint16), (200000, 65536, np.uint16),
    (60000, 1 << 20, np.uint32), (3000, 1 << 24, np.uint32), (5000, 1, np.uint8), (0, 256, np.uint8),
])
def test_order_matches_oracle(kind, n, sigma, dtype):
    import torch

    import paper_1702_07578_gb300 as wtg
    T = _text(n, sigma, dtype, 41 + n)
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    bv, z, perm, srt = wtg.build_order(k, torch_text(T), sigma)
    torch.cuda.synchronize()
    ep, es = oracle.stable_order(T, sigma, kind)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), ep)
    got_s = srt.cpu().numpy().view(T.dtype)
    assert np.array_equal(got_s, es)
    if kind == "wt":
        assert np.array_equal(to_u64(bv), oracle.wt(T, sigma))
    else:
        e, ez = oracle.wm(T, sigma)
        assert np.array_equal(to_u64(bv), e)
        assert np.array_equal(z.cpu().numpy().astype(np.uint64), ez)


def test_order_without_sorted_text_and_errors():
    import torch

    import paper_1702_07578_gb300 as wtg
    T = synth.uniform_text(10000, 16, 2, np.uint8)
    bv, _, perm, srt = wtg.build_order(wtg.WT_TREE, torch_text(T), 16, sorted_text=False)
    torch.cuda.synchronize()
    assert srt is None
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), oracle.stable_order(T, 16, "wt")[0])
    T[77] = 16
    t = torch_text(T)
    ws = torch.empty((wtg.wt_order_workspace_size(wtg.WT_TREE, 1, T.size, 16),), dtype=torch.uint8, device="cuda")
    wtg.build_order(wtg.WT_TREE, t, 16, ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2
