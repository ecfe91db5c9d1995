"""Batched construction (wt_build_batched): every text bit-exact with the oracle
and with a plain single-text build of the same text."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_wm, gpu_wt, to_u64, torch_text

pytestmark = pytest.mark.gpu


def _batch(specs, dtype):
    texts = []
    for n, sigma, seed in specs:
        if sigma == 1:
            texts.append(np.zeros(n, dtype))
        else:
            texts.append(synth.zipf_text(n, sigma, 0.8, seed, dtype))
    return texts


SPECS_MIXED = [(1000, 16, 1), (0, 256, 2), (70000, 256, 3), (1, 4096, 4), (300000, 4096, 5),
               (65536, 65536, 6), (123457, 65536, 7), (5000, 1, 8), (64, 2, 9), (200001, 16, 10),
               (131072, 257, 11), (777, 65536, 12)]


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_batched_matches_oracle_and_plain(kind):
    import paper_1702_07578_gb300 as wtg
    texts = _batch(SPECS_MIXED, np.uint16)
    sigmas = [s for _, s, _ in SPECS_MIXED]
    dts = [torch_text(t) for t in texts]
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    bvs, zs = wtg.wt_build_batched(k, dts, sigmas)
    import torch
    torch.cuda.synchronize()
    for i, (T, sigma) in enumerate(zip(texts, sigmas)):
        got = to_u64(bvs[i])
        if kind == "wt":
            exp = oracle.wt(T, sigma)
            assert np.array_equal(got, exp), f"text {i}"
            assert np.array_equal(got, gpu_wt(T, sigma)), f"text {i} vs plain"
        else:
            exp, ez = oracle.wm(T, sigma)
            L = exp.shape[0]
            assert np.array_equal(got, exp), f"text {i}"
            assert np.array_equal(zs[i][:L].cpu().numpy().astype(np.uint64), ez), f"Z {i}"
            pb, pz = gpu_wm(T, sigma)
            assert np.array_equal(got, pb)


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_batched_workload_sample(kind):
    """A slice of the 4096-text batched workload (log-uniform lengths, mixed sigma)."""
    import torch

    import paper_1702_07578_gb300 as wtg
    specs = synth.batch_specs(256, max_log=17)
    texts = synth.batch_texts(specs)
    sigmas = [s for _, s, _ in specs]
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    bvs, zs = wtg.wt_build_batched(k, [torch_text(t) for t in texts], sigmas)
    torch.cuda.synchronize()
    for i in range(0, len(texts), 7):
        T, sigma = texts[i], sigmas[i]
        if kind == "wt":
            assert np.array_equal(to_u64(bvs[i]), oracle.wt(T, sigma)), f"text {i}"
        else:
            e, ez = oracle.wm(T, sigma)
            assert np.array_equal(to_u64(bvs[i]), e), f"text {i}"
            assert np.array_equal(zs[i][:e.shape[0]].cpu().numpy().astype(np.uint64), ez)


def test_batched_symbol_range_error():
    import torch

    import paper_1702_07578_gb300 as wtg
    a = synth.uniform_text(5000, 100, 1, np.uint16)
    b = synth.uniform_text(5000, 100, 2, np.uint16)
    b[17] = 100
    ts = [torch_text(a), torch_text(b)]
    sz = wtg.wt_batched_workspace_size(wtg.WT_TREE, 2, [5000, 5000], [100, 100])
    ws = torch.empty((sz,), dtype=torch.uint8, device="cuda")
    wtg.wt_build_batched(wtg.WT_TREE, ts, [100, 100], ws=ws)
    with pytest.raises(wtg.WtError) as e:
        wtg.wt_sync_status(ws)
    assert e.value.code == 2


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_graph_plan_replay_and_update(kind, tmp_path, monkeypatch):
    """One graph replay builds the whole batch; after an in-place descriptor update
    the same graph builds other texts of the same shapes; the autotuner's choice is
    cached and picked up by a new plan."""
    import torch

    import paper_1702_07578_gb300 as wtg
    monkeypatch.setenv("WT_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = synth.batch_specs(64, max_log=16)
    sigmas = [s for _, s, _ in specs]
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    A = synth.batch_texts(specs)
    B = [synth.zipf_text(n, sg, 1.0, ts + 99, np.uint16) for n, sg, ts in specs]
    ta = [torch_text(t) for t in A]
    tb = [torch_text(t) for t in B]

    def outs():
        bv = [torch.empty((wtg.wt_levels(s), wtg.wt_words_per_level(t.numel())), dtype=torch.int64,
                          device="cuda") for t, s in zip(ta, sigmas)]
        zz = [torch.empty((max(wtg.wt_levels(s), 1),), dtype=torch.int64, device="cuda")
              for s in sigmas] if kind == "wm" else None
        return bv, zz

    bva, za = outs()
    bvb, zb = outs()
    stream = torch.cuda.Stream()
    best = wtg.wt_autotune_batched(k, ta, sigmas, bva, za, stream=stream)
    assert best in (32768, 65536, 131072, 262144)
    plan = wtg.WtBatchPlan(k, ta, sigmas, bva, za, stream=stream)
    assert plan.symbols_per_block == best
    for _ in range(2):
        plan.launch()
    plan.update(tb, bvb, zb)
    plan.launch()
    stream.synchronize()
    for i in range(0, len(A), 5):
        for T, bv, zz in ((A[i], bva, za), (B[i], bvb, zb)):
            if kind == "wt":
                assert np.array_equal(to_u64(bv[i]), oracle.wt(T, sigmas[i])), i
            else:
                e, ez = oracle.wm(T, sigmas[i])
                assert np.array_equal(to_u64(bv[i]), e), i
                assert np.array_equal(zz[i][:e.shape[0]].cpu().numpy().astype(np.uint64), ez)
    plan.close()


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_batched_mixed_round_geometry(kind):
    """One batch whose texts have 1, 2 and 3 rounds of different first-round lengths
    (L = 2, 9, 12, 13, 17, 20, 24): round r mixes texts with different prefixes done,
    different children per parent and texts that are already finished."""
    import torch

    import paper_1702_07578_gb300 as wtg
    rng = np.random.default_rng(2024)
    sigmas = [3, 300, 4096, 5000, 70000, 1 << 20, 1 << 24, 300, 5000, 1 << 20]
    lengths = [1000, 50000, 70001, 12345, 90000, 130000, 60000, 0, 1, 4097]
    texts = [synth.zipf_text(n, s, 0.9, int(rng.integers(1, 1 << 30)), np.uint32) if n else np.zeros(0, np.uint32)
             for n, s in zip(lengths, sigmas)]
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    bvs, zs = wtg.wt_build_batched(k, [torch_text(t) if t.size else torch.zeros(0, dtype=torch.int32, device="cuda")
                                       for t in texts], sigmas)
    torch.cuda.synchronize()
    for i, (T, sigma) in enumerate(zip(texts, sigmas)):
        if kind == "wt":
            assert np.array_equal(to_u64(bvs[i]), oracle.wt(T, sigma)), f"text {i} sigma {sigma}"
        else:
            e, ez = oracle.wm(T, sigma)
            assert np.array_equal(to_u64(bvs[i]), e), f"text {i} sigma {sigma}"
            assert np.array_equal(zs[i][:e.shape[0]].cpu().numpy().astype(np.uint64), ez)


@pytest.mark.parametrize("kind", ["wt", "wm"])
def test_batched_workload_slice_full_lengths(kind):
    """A 512-text slice of the batched workload with its full length range (2^10 to
    2^20 symbols, sigma 2^4 .. 2^16), built by one graph replay with the default
    block size: every text equal to the oracle."""
    import torch

    import paper_1702_07578_gb300 as wtg
    specs = synth.batch_specs(512)
    assert max(n for n, _, _ in specs) > 1 << 19
    texts = synth.batch_texts(specs)
    sigmas = [s for _, s, _ in specs]
    k = wtg.WT_TREE if kind == "wt" else wtg.WT_MATRIX
    dts = [torch_text(t) for t in texts]
    bv = [torch.full((wtg.wt_levels(s), wtg.wt_words_per_level(t.size)), -1, dtype=torch.int64, device="cuda")
          for t, s in zip(texts, sigmas)]
    zz = [torch.empty((max(wtg.wt_levels(s), 1),), dtype=torch.int64, device="cuda") for s in sigmas]
    stream = torch.cuda.Stream()
    plan = wtg.WtBatchPlan(k, dts, sigmas, bv, zz if kind == "wm" else None, stream=stream)
    plan.launch()
    stream.synchronize()
    for i, (T, sigma) in enumerate(zip(texts, sigmas)):
        if kind == "wt":
            assert np.array_equal(to_u64(bv[i]), oracle.wt(T, sigma)), f"text {i} n {T.size} sigma {sigma}"
        else:
            e, ez = oracle.wm(T, sigma)
            assert np.array_equal(to_u64(bv[i]), e), f"text {i} n {T.size} sigma {sigma}"
            assert np.array_equal(zz[i][:e.shape[0]].cpu().numpy().astype(np.uint64), ez), f"Z {i}"
    plan.close()
