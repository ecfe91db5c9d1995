"""The C oracle and the C input generators built with AddressSanitizer and
UndefinedBehaviorSanitizer (gcc -fsanitize=address,undefined, every report fatal)
and run on small cases in a child process with the sanitizer runtimes preloaded.
The child must exit cleanly and give the same bytes as the normal builds.  Host
code only: no GPU."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (n, sigma, dtype, generator): byte, 16-bit and 32-bit texts, sigma not a power of
# two, one level, no level, empty and one-symbol texts, several tiles of 64 words
CASES = [(0, 256, "uint8", "zipf"), (1, 2, "uint8", "uniform"), (777, 1, "uint8", "uniform"),
         (1000, 3, "uint8", "zipf"), (5003, 256, "uint8", "zipf"), (4097, 97, "uint8", "uniform"),
         (3001, 4096, "uint16", "zipf"), (2000, 65536, "uint16", "uniform"),
         (1500, 1 << 20, "uint32", "markov"), (700, 1 << 24, "uint32", "uniform")]

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import oracle, synth
oracle.build = lambda force=False: {oracle_so!r}
synth.build = lambda force=False: {synth_so!r}
out = {{}}
for i, (n, sigma, dt, gen) in enumerate({cases!r}):
    dt = np.dtype(dt).type
    if gen == "zipf":
        T = synth.zipf_text(n, sigma, 1.0, 11 + i, dt)
    elif gen == "markov":
        T = synth.uniform_markov_text(n, sigma, 5 + i, dt)
    else:
        T = synth.uniform_text(n, sigma, 3 + i, dt)
    out["T%d" % i] = T
    out["wt%d" % i] = oracle.wt(T, sigma)
    out["wm%d" % i], out["z%d" % i] = oracle.wm(T, sigma)
    out["pcwt%d" % i] = oracle.pc("wt", T, sigma)
    out["pcwm%d" % i], _ = oracle.pc("wm", T, sigma)
    out["pswt%d" % i] = oracle.ps("wt", T, sigma, 3)
    out["pswm%d" % i], _ = oracle.ps("wm", T, sigma, 5)
out["perm"] = synth.permutation(7, 1000)
np.savez({out!r}, **out)
"""


def _runtime(name):
    p = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def _sanitized(src, out, extra):
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-shared", "-fPIC", "-fno-omit-frame-pointer",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-o", out, src] + extra)
    return out


def test_oracle_and_generators_under_asan_ubsan(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if asan is None or ubsan is None:
        pytest.skip("gcc sanitizer runtimes not installed")
    oracle_so = _sanitized(os.path.join(ROOT, "oracle", "wt_oracle.c"), str(tmp_path / "liboracle_san.so"), [])
    synth_so = _sanitized(os.path.join(ROOT, "synth", "synth.c"), str(tmp_path / "libsynth_san.so"),
                          ["-pthread", "-lm"])
    out = str(tmp_path / "san.npz")
    script = CHILD.format(root=ROOT, oracle_so=oracle_so, synth_so=synth_so, cases=CASES, out=out)
    env = dict(os.environ, LD_PRELOAD=asan + " " + ubsan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    got = np.load(out)
    for i, (n, sigma, dt, gen) in enumerate(CASES):
        T = got["T%d" % i]
        ref = synth.zipf_text(n, sigma, 1.0, 11 + i, np.dtype(dt).type) if gen == "zipf" else (
            synth.uniform_markov_text(n, sigma, 5 + i, np.dtype(dt).type) if gen == "markov"
            else synth.uniform_text(n, sigma, 3 + i, np.dtype(dt).type))
        assert np.array_equal(T, ref)
        assert np.array_equal(got["wt%d" % i], oracle.wt(T, sigma))
        bm, z = oracle.wm(T, sigma)
        assert np.array_equal(got["wm%d" % i], bm) and np.array_equal(got["z%d" % i], z)
        for k in ("pcwt", "pswt"):
            assert np.array_equal(got["%s%d" % (k, i)], got["wt%d" % i])
        for k in ("pcwm", "pswm"):
            assert np.array_equal(got["%s%d" % (k, i)], got["wm%d" % i])
    assert np.array_equal(got["perm"], synth.permutation(7, 1000))
