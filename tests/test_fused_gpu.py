"""wt_wm_build: the WT and the WM of one text in one call, bit-identical to the
oracle (and to wt_build + wm_build) for the fused pass (sigma <= 256, n > 4096)
and for the texts it hands to the separate builds."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_wm, gpu_wt, to_u64, torch_text

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,sigma,dtype,dist", [
    (4097, 256, np.uint8, "zipf"),            # smallest fused text
    (32768 * 3 + 17, 256, np.uint8, "zipf"),  # several tiles and a ragged tail
    (200003, 256, np.uint8, "uniform"),
    (65536 * 5, 97, np.uint8, "zipf"),        # sigma not a power of two
    (150001, 2, np.uint8, "uniform"),         # one level
    (100000, 16, np.uint16, "zipf"),
    (300000, 256, np.uint32, "markovish"),
    (4096, 256, np.uint8, "zipf"),            # small: separate builds
    (0, 256, np.uint8, "zipf"),
    (70000, 4096, np.uint16, "zipf"),         # two rounds: separate builds
    (9000, 1, np.uint8, "zero"),
])
def test_fused_matches_oracle(n, sigma, dtype, dist):
    import paper_1702_07578_gb300 as wtg
    if dist == "zero":
        T = np.zeros(n, dtype)
    elif dist == "uniform":
        T = synth.uniform_text(n, sigma, 17 + n, dtype)
    elif dist == "markovish":
        T = np.sort(synth.uniform_text(n, sigma, 5, dtype))          # long runs of equal symbols
    else:
        T = synth.zipf_text(n, sigma, 1.0, 23 + n, dtype)
    t = torch_text(T)
    bw, bm, z = wtg.wt_wm_build(t, sigma)
    import torch
    torch.cuda.synchronize()
    L = oracle.levels(sigma)
    ew = oracle.wt(T, sigma)
    em, ez = oracle.wm(T, sigma)
    assert np.array_equal(to_u64(bw), ew)
    assert np.array_equal(to_u64(bm), em)
    assert np.array_equal(z.cpu().numpy().astype(np.uint64)[:L], ez)


def test_fused_equals_separate_on_byte_workload_slice():
    import paper_1702_07578_gb300 as wtg
    T, sigma = synth.workload_bytes(1 << 24)
    t = torch_text(T)
    ws = __import__("torch").empty((wtg.wt_wm_workspace_size(wtg.WT_U8, T.size, sigma),),
                                   dtype=__import__("torch").uint8, device="cuda")
    bw, bm, z = wtg.wt_wm_build(t, sigma, ws=ws)
    wtg.wt_sync_status(ws)
    assert np.array_equal(to_u64(bw), gpu_wt(T, sigma))
    pb, pz = gpu_wm(T, sigma)
    assert np.array_equal(to_u64(bm), pb)
    assert np.array_equal(z.cpu().numpy().astype(np.uint64), pz)


def test_fused_symbol_range_error():
    import torch

    import paper_1702_07578_gb300 as wtg
    T = synth.uniform_text(50000, 200, 3, np.uint8)
    T[4321] = 230
    t = torch_text(T)
    ws = torch.empty((wtg.wt_wm_workspace_size(wtg.WT_U8, T.size, 200),), dtype=torch.uint8, device="cuda")
    wtg.wt_wm_build(t, 200, ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2
