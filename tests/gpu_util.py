"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding
and bring results back as numpy arrays comparable with the oracle."""
import numpy as np

import paper_1702_07578_gb300 as wtg


def torch_text(T):
    import torch
    T = np.ascontiguousarray(T)
    if T.dtype == np.uint8:
        t = torch.from_numpy(T)
    elif T.dtype == np.uint16:
        t = torch.from_numpy(T.view(np.int16))
    elif T.dtype == np.uint32:
        t = torch.from_numpy(T.view(np.int32))
    else:
        raise TypeError(T.dtype)
    return t.cuda()


def to_u64(bv):
    return bv.cpu().numpy().view(np.uint64)


def gpu_wt(T, sigma):
    import torch
    t = torch_text(T)
    n = t.numel()
    ws = torch.empty((max(wtg.wt_workspace_size(wtg.WT_TREE, T.dtype.itemsize, n, sigma), 1),),
                     dtype=torch.uint8, device="cuda")
    bv = wtg.wt_build(t, sigma, ws=ws)
    wtg.wt_sync_status(ws)
    return to_u64(bv)


def gpu_wm(T, sigma):
    import torch
    t = torch_text(T)
    n = t.numel()
    ws = torch.empty((max(wtg.wt_workspace_size(wtg.WT_MATRIX, T.dtype.itemsize, n, sigma), 1),),
                     dtype=torch.uint8, device="cuda")
    bv, z = wtg.wm_build(t, sigma, ws=ws)
    wtg.wt_sync_status(ws)
    return to_u64(bv), z.cpu().numpy().astype(np.uint64)


def first_diff(a, b):
    """(level, word) of the first differing word, for messages."""
    d = np.argwhere(a != b)
    return tuple(d[0]) if len(d) else None
