"""Full-size parity: the benchmark workloads, every word compared with the oracle.

  * n = 2^30 uint8, sigma = 256, Zipf(1.0) over a seeded permutation
  * n = 2^28 uint32, sigma = 2^20, half uniform / half order-1 Markov (20 levels,
    three rounds, deep sparse histograms)

Same launch configuration as bench.py (wt_build / wm_build on the current stream).
The oracle runs in worker processes (spawned before the first GPU call) that
regenerate the seeded text themselves, while the GPU builds.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _oracle_job(which, kind):
    import oracle
    import synth as s
    if which == "bytes":
        T, sigma = s.workload_bytes()
    else:
        T, sigma = s.workload_large_alphabet()
    if kind == "wt":
        return oracle.wt(T, sigma), None
    return oracle.wm(T, sigma)


@pytest.fixture(scope="module")
def oracle_results():
    ex = ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn"))
    futs = {(w, k): ex.submit(_oracle_job, w, k)
            for w in ("bytes", "large_alphabet") for k in ("wt", "wm")}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.mark.parametrize("which", ["bytes", "large_alphabet"])
def test_fullsize_parity(which, oracle_results):
    from tests.gpu_util import first_diff, gpu_wm, gpu_wt
    if which == "bytes":
        T, sigma = synth.workload_bytes()
    else:
        T, sigma = synth.workload_large_alphabet()
    bw = gpu_wt(T, sigma)
    bm, zm = gpu_wm(T, sigma)
    ew, _ = oracle_results[(which, "wt")].result()
    assert np.array_equal(bw, ew), f"WT differs at {first_diff(bw, ew)}"
    del ew
    em, ez = oracle_results[(which, "wm")].result()
    assert np.array_equal(bm, em), f"WM differs at {first_diff(bm, em)}"
    assert np.array_equal(zm, ez)
