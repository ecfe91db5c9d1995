"""Serving loop: results equal the oracle, and each result is the same built
alone and built in a mix of concurrent requests (tolerance 0: bit-exact)."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _requests(count, seed, max_log=18):
    specs = synth.request_specs(count, 1000.0, seed=seed, max_log=max_log)
    return [(kind, synth.request_text(n, sg, zipf, ts), sg) for (_, n, sg, zipf, kind, ts) in specs]


def test_served_results_match_oracle_and_solo():
    import paper_1702_07578_gb300 as wtg
    reqs = _requests(24, 77)
    srv = wtg.WtServer(hbm_budget_bytes=4 << 30, max_batch=8, streams=3)
    tickets = [srv.submit(wtg.WT_TREE if k == "wt" else wtg.WT_MATRIX, T, sg) for k, T, sg in reqs]
    mixed = []
    for t in tickets:
        r = srv.wait(t, timeout_us=60_000_000)
        assert r["status"] == 0
        mixed.append(srv.read(t))
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_us"] >= st["p50_us"] > 0
    srv.close()
    solo = wtg.WtServer(hbm_budget_bytes=4 << 30, max_batch=1, streams=1)
    for (k, T, sg), (bv, z) in zip(reqs, mixed):
        t = solo.submit(wtg.WT_TREE if k == "wt" else wtg.WT_MATRIX, T, sg)
        solo.wait(t)
        bv1, z1 = solo.read(t)
        solo.release(t)
        assert np.array_equal(bv, bv1)
        if k == "wt":
            assert np.array_equal(bv, oracle.wt(T, sg))
        else:
            e, ez = oracle.wm(T, sg)
            assert np.array_equal(bv, e) and np.array_equal(z, ez) and np.array_equal(z1, ez)
    solo.close()


def test_admission_budget_and_errors():
    import paper_1702_07578_gb300 as wtg
    srv = wtg.WtServer(hbm_budget_bytes=8 << 20, max_batch=4, streams=2)
    big = np.zeros(64 << 20, dtype=np.uint8)
    with pytest.raises(wtg.WtError) as e:
        srv.submit(wtg.WT_TREE, big, 256)            # alone exceeds the budget
    assert e.value.code == 6
    with pytest.raises(wtg.WtError) as e:
        srv.wait(12345, 0)
    assert e.value.code == 7
    # many requests that fit only a few at a time still all complete
    T = synth.uniform_text(300000, 256, 5, np.uint8)
    ts = [srv.submit(wtg.WT_MATRIX, T, 256) for _ in range(12)]
    exp, ez = oracle.wm(T, 256)
    for t in ts:
        assert srv.wait(t, 60_000_000)["status"] == 0
        bv, z = srv.read(t)
        assert np.array_equal(bv, exp) and np.array_equal(z, ez)
        srv.release(t)
    assert srv.stats()["hbm_in_use"] == 0
    srv.close()


def test_wait_timeout_returns():
    import paper_1702_07578_gb300 as wtg
    srv = wtg.WtServer(hbm_budget_bytes=2 << 30, max_batch=2, streams=1)
    T = synth.uniform_text(1 << 22, 256, 9, np.uint8)
    t = srv.submit(wtg.WT_TREE, T, 256)
    try:
        srv.wait(t, 0)
    except wtg.WtError as e:
        assert e.code == 5
    assert srv.wait(t, 60_000_000)["status"] == 0
    srv.release(t)
    srv.close()


def test_pinned_submit_matches_copy_submit():
    """wt_server_submit_pinned reads page-locked client buffers in place; results
    equal the copying submit and the oracle; a pageable tensor is refused."""
    import torch

    import paper_1702_07578_gb300 as wtg
    reqs = _requests(12, 91, max_log=17)
    srv = wtg.WtServer(hbm_budget_bytes=2 << 30, max_batch=4, streams=2)
    pinned = [torch.from_numpy(T.view(np.int16) if T.dtype == np.uint16 else T).pin_memory()
              for _, T, _ in reqs]
    tp = [srv.submit(wtg.WT_TREE if k == "wt" else wtg.WT_MATRIX, P, sg)
          for (k, _, sg), P in zip(reqs, pinned)]
    tc = [srv.submit(wtg.WT_TREE if k == "wt" else wtg.WT_MATRIX, T, sg) for k, T, sg in reqs]
    for (k, T, sg), a, b in zip(reqs, tp, tc):
        assert srv.wait(a)["status"] == 0 and srv.wait(b)["status"] == 0
        bva, za = srv.read(a)
        bvb, zb = srv.read(b)
        srv.release(a)
        srv.release(b)
        assert np.array_equal(bva, bvb)
        if k == "wt":
            assert np.array_equal(bva, oracle.wt(T, sg))
        else:
            e, ez = oracle.wm(T, sg)
            assert np.array_equal(bva, e) and np.array_equal(za, ez) and np.array_equal(zb, ez)
    pageable = torch.from_numpy(reqs[0][1].astype(np.uint8) if reqs[0][2] <= 256 else reqs[0][1].view(np.int16))
    with pytest.raises(ValueError):
        srv.submit(wtg.WT_TREE, pageable, reqs[0][2])
    srv.close()


def test_concurrent_submitters():
    """Four host threads submit, wait, read and release at the same time (the C calls
    run without the interpreter lock); every result equals the oracle."""
    import threading

    import paper_1702_07578_gb300 as wtg
    reqs = _requests(32, 123, max_log=16)
    srv = wtg.WtServer(hbm_budget_bytes=1 << 30, max_batch=6, streams=3)
    errors = []

    def worker(part):
        try:
            for k, T, sg in part:
                kind = wtg.WT_TREE if k == "wt" else wtg.WT_MATRIX
                t = srv.submit(kind, T, sg)
                r = srv.wait(t, timeout_us=60_000_000)
                assert r["status"] == 0
                bv, z = srv.read(t)
                srv.release(t)
                if k == "wt":
                    assert np.array_equal(bv, oracle.wt(T, sg))
                else:
                    e, ez = oracle.wm(T, sg)
                    assert np.array_equal(bv, e) and np.array_equal(z, ez)
        except Exception as exc:          # reported on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(reqs[i::4],)) for i in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    st = srv.stats()
    srv.close()
    assert not errors, errors[0]
    assert st["completed"] == len(reqs)

