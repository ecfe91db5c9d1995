"""The bounds-checked build of the library (-DWT_DEBUG_BOUNDS): its construction
kernels compare their indexes with the sizes of the buffers they address and
record every failure.  A child process loads that build (WT_DEBUG_BOUNDS=1),
checks that a failure is recorded at all (a self-test kernel that evaluates one
failing check with no memory access behind it), then builds texts that reach
every kernel and code path of the construction (byte rounds, rounds that cut,
three rounds, small jobs, groups of several tiles, ragged tails, the one-pass
WT+WM build, the stable order, a batch) and compares each with the oracle: the
outputs must match bit for bit and no check may fail."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import torch
import paper_1702_07578_gb300 as wtg
import oracle, synth
from tests.gpu_util import torch_text, to_u64

out = {{"cases": []}}
rep = wtg.wt_debug_bounds_read(reset=True)
out["enabled"] = rep["enabled"]
wtg.wt_debug_bounds_selftest()
out["selftest"] = wtg.wt_debug_bounds_read(reset=True)
out["after_reset"] = wtg.wt_debug_bounds_read()

def record(name, ok):
    r = wtg.wt_debug_bounds_read(reset=True)
    out["cases"].append({{"case": name, "match": bool(ok), "failures": r["failures"], "site": r["site"],
                          "index": r["index"], "bound": r["bound"]}})

def text(n, sigma, dist, seed, dt):
    if dist == "zipf":
        return synth.zipf_text(n, sigma, 1.0, seed, dt)
    if dist == "markov":
        return synth.uniform_markov_text(n, sigma, seed, dt)
    return synth.uniform_text(n, sigma, seed, dt)

CASES = [(3 * 32768 + 777, 256, "zipf", np.uint8), (100003, 200, "uniform", np.uint8),
         (5000, 256, "zipf", np.uint8), (777, 16, "uniform", np.uint8),
         (300001, 4096, "zipf", np.uint16), (200001, 1 << 20, "markov", np.uint32),
         (120000, 65536, "uniform", np.uint16), (9 * 32768 + 5, 2, "uniform", np.uint8)]
for i, (n, sigma, dist, dt) in enumerate(CASES):
    T = text(n, sigma, dist, 101 + i, dt)
    t = torch_text(T)
    bv = wtg.wt_build(t, sigma)
    torch.cuda.synchronize()
    record(f"wt n={{n}} sigma={{sigma}}", np.array_equal(to_u64(bv), oracle.wt(T, sigma)))
    bm, z = wtg.wm_build(t, sigma)
    torch.cuda.synchronize()
    em, ez = oracle.wm(T, sigma)
    record(f"wm n={{n}} sigma={{sigma}}",
           np.array_equal(to_u64(bm), em) and np.array_equal(z.cpu().numpy().astype(np.uint64), ez))

# groups of several tiles (carried words between the tiles of a group)
T = text(6 * 32768 + 77, 256, "zipf", 7, np.uint8)
t = torch_text(T)
for kind in (wtg.WT_TREE, wtg.WT_MATRIX):
    bv = [torch.full((8, wtg.wt_words_per_level(T.size)), -1, dtype=torch.int64, device="cuda")]
    zz = [torch.empty((8,), dtype=torch.int64, device="cuda")]
    plan = wtg.WtBatchPlan(kind, [t], [256], bv, zz if kind else None, symbols_per_block=3 * 32768)
    plan.launch()
    torch.cuda.synchronize()
    exp = oracle.wt(T, 256) if kind == wtg.WT_TREE else oracle.wm(T, 256)[0]
    record(f"group of 3 tiles kind={{kind}}", np.array_equal(to_u64(bv[0]), exp))
    plan.close()

# one pass for both structures
T = text(200000, 256, "zipf", 9, np.uint8)
t = torch_text(T)
bt, bm, z = wtg.wt_wm_build(t, 256)
torch.cuda.synchronize()
record("wt_wm_build", np.array_equal(to_u64(bt), oracle.wt(T, 256)) and np.array_equal(to_u64(bm), oracle.wm(T, 256)[0]))

# the stable order (ranks written by the cut pass)
T = text(150001, 4096, "zipf", 10, np.uint16)
t = torch_text(T)
res = wtg.build_order(wtg.WT_MATRIX, t, 4096)
torch.cuda.synchronize()
record("wm_build_order", np.array_equal(to_u64(res[0]), oracle.wm(T, 4096)[0]))

# a small batch of uneven texts
specs = synth.batch_specs(48)
texts_h = synth.batch_texts(specs)
sig = [s for _, s, _ in specs]
texts = [torch.from_numpy(x.view(np.int16)).cuda() for x in texts_h]
for kind in (wtg.WT_TREE, wtg.WT_MATRIX):
    bvs, _ = wtg.wt_build_batched(kind, texts, sig)
    torch.cuda.synchronize()
    ok = all(np.array_equal(to_u64(b), (oracle.wt(x, s) if kind == wtg.WT_TREE else oracle.wm(x, s)[0]))
             for b, x, s in zip(bvs, texts_h, sig))
    record(f"batched kind={{kind}}", ok)
print("RESULT " + json.dumps(out), flush=True)
"""


def test_bounds_checked_build_matches_oracle_with_no_failed_check():
    import paper_1702_07578_gb300 as wtg
    from paper_1702_07578_gb300 import _native
    assert wtg.wt_debug_bounds_read()["enabled"] is False      # the default build has no checks
    _native.build(debug_bounds=True)
    env = dict(os.environ, WT_DEBUG_BOUNDS="1")
    code = CHILD.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = next(x for x in r.stdout.splitlines() if x.startswith("RESULT "))
    out = json.loads(line[len("RESULT "):])
    assert out["enabled"] is True
    st = out["selftest"]
    assert (st["failures"], st["site"], st["index"], st["bound"]) == (1, "selftest", 1, 1), st
    assert out["after_reset"]["failures"] == 0
    assert len(out["cases"]) >= 20
    for c in out["cases"]:
        assert c["match"], c
        assert c["failures"] == 0, c
