"""Serving loop shutdown: wt_server_destroy with requests in every state returns,
and the device stays usable."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_close_with_requests_in_flight():
    """Destroying the server with requests finished but never released, running, and
    queued behind a budget those unreleased results hold (they could never be
    admitted) returns: launched batches finish, the rest is dropped; the device
    stays usable and a new server's results equal the oracle.
    The close runs in a watchdog thread so that a regression fails instead of
    hanging the suite."""
    import threading

    import torch

    import paper_1702_07578_gb300 as wtg
    srv = wtg.WtServer(hbm_budget_bytes=64 << 20, max_batch=2, streams=2)
    T = synth.uniform_text(1 << 22, 256, 13, np.uint8)
    tickets = [srv.submit(wtg.WT_TREE if i % 2 else wtg.WT_MATRIX, T, 256) for i in range(10)]
    assert len(set(tickets)) == 10
    assert srv.wait(tickets[0], 60_000_000)["status"] == 0
    closer = threading.Thread(target=srv.close, daemon=True)
    closer.start()
    closer.join(120)
    hung = closer.is_alive()
    if hung:
        srv._h = None          # the blocked call still owns the server: never destroy it twice
    assert not hung, "wt_server_destroy did not return"
    torch.cuda.synchronize()
    srv2 = wtg.WtServer(hbm_budget_bytes=1 << 30, max_batch=2, streams=2)
    U = synth.zipf_text(300001, 200, 1.0, 17, np.uint8)
    t = srv2.submit(wtg.WT_MATRIX, U, 200)
    assert srv2.wait(t, 60_000_000)["status"] == 0
    bv, z = srv2.read(t)
    e, ez = oracle.wm(U, 200)
    assert np.array_equal(bv, e) and np.array_equal(z, ez)
    srv2.release(t)
    srv2.close()
