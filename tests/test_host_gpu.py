"""wt_build_host: host text in, host levels out, in one C-ABI call.  The levels
and Z must be bit-identical to the oracle (and to the device builds), for
page-locked and pageable host buffers, the WT alone, the WM alone, both from
separate builds and both from one pass."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_wm, gpu_wt

pytestmark = pytest.mark.gpu


def _host_text(T, pinned):
    import torch
    T = np.ascontiguousarray(T)
    view = {np.dtype(np.uint8): np.uint8, np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[T.dtype]
    t = torch.from_numpy(T.view(view).copy())
    return t.pin_memory() if pinned else t


def _u64(t):
    return t.numpy().view(np.uint64)


@pytest.mark.parametrize("n,sigma,dtype", [
    (0, 256, np.uint8),
    (1, 2, np.uint8),
    (9000, 1, np.uint8),                  # one symbol value: no levels
    (1000, 3, np.uint8),
    (32768 * 3 + 17, 256, np.uint8),      # several tiles and a ragged tail
    (200000, 4096, np.uint16),            # two rounds
    (30011, 1 << 20, np.uint32),          # three rounds, small wavelet-tree jobs
])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("what", ["wt", "wm", "both", "one_pass"])
def test_host_build_matches_oracle(n, sigma, dtype, pinned, what):
    import torch
    import paper_1702_07578_gb300 as wtg
    T = synth.zipf_text(n, sigma, 1.0, 91 + n, dtype) if sigma > 2 else synth.uniform_text(n, max(sigma, 1), 7, dtype)
    t = _host_text(T, pinned)
    ws = torch.empty((wtg.wt_host_workspace_size(T.dtype.itemsize, n, sigma),), dtype=torch.uint8, device="cuda")
    bw, bm, z = wtg.wt_build_host(t, sigma, wt=what != "wm", wm=what != "wt", one_pass=what == "one_pass", ws=ws)
    wtg.wt_sync_status(ws)
    L = oracle.levels(sigma)
    if what != "wm":
        assert bw.shape == (L, (n + 63) // 64)
        assert np.array_equal(_u64(bw), oracle.wt(T, sigma))
    else:
        assert bw is None
    if what != "wt":
        em, ez = oracle.wm(T, sigma)
        assert np.array_equal(_u64(bm), em)
        assert np.array_equal(z.numpy().astype(np.uint64), ez)
    else:
        assert bm is None and z is None


def test_host_build_equals_device_builds_on_byte_workload_slice():
    """2^24 symbols of the bench's byte workload; three calls reuse one workspace
    and their outputs, on a side stream."""
    import torch
    import paper_1702_07578_gb300 as wtg
    T, sigma = synth.workload_bytes(1 << 24)
    t = _host_text(T, True)
    ws = torch.empty((wtg.wt_host_workspace_size(1, T.size, sigma),), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    bw, bm, z = wtg.wt_build_host(t, sigma, ws=ws, stream=s)
    for one_pass in (True, False):
        bw2, bm2, z2 = wtg.wt_build_host(t, sigma, one_pass=one_pass, out_wt=bw, out_wm=bm, out_zeros=z, ws=ws,
                                         stream=s)
    wtg.wt_sync_status(ws, stream=s)
    assert bw2.data_ptr() == bw.data_ptr()
    assert np.array_equal(_u64(bw), gpu_wt(T, sigma))
    pb, pz = gpu_wm(T, sigma)
    assert np.array_equal(_u64(bm), pb)
    assert np.array_equal(z.numpy().astype(np.uint64), pz)


def test_host_build_errors():
    import torch
    import paper_1702_07578_gb300 as wtg
    T = synth.zipf_text(50000, 200, 1.0, 3, np.uint8)
    t = _host_text(T, False)
    need = wtg.wt_host_workspace_size(1, T.size, 256)
    small = torch.empty((need - 256,), dtype=torch.uint8, device="cuda")
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_build_host(t, 256, ws=small)
    assert e.value.code == 3
    with pytest.raises(ValueError):
        wtg.wt_build_host(t, 256, wt=False, wm=False)
    ws = torch.empty((need,), dtype=torch.uint8, device="cuda")
    # sigma = 2^25 is beyond the WT's limit; the WM alone is built
    _, bm, _ = wtg.wt_build_host(_host_text(T.astype(np.uint32), False), 1 << 25, wt=False,
                                 ws=torch.empty((wtg.wt_host_workspace_size(4, T.size, 1 << 25),),
                                                dtype=torch.uint8, device="cuda"))
    assert bm.shape[0] == 25
    with pytest.raises(wtg.WtError):
        wtg.wt_build_host(_host_text(T.astype(np.uint32), False), 1 << 25, wm=False,
                          ws=torch.empty((wtg.wt_host_workspace_size(4, T.size, 1 << 25),),
                                         dtype=torch.uint8, device="cuda"))
    # a symbol >= sigma is found on the device and reported by wt_sync_status
    wtg.wt_build_host(t, 100, ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2
