"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU, no GPU).

compute-sanitizer is not available for the CUDA side, so memory safety is checked where it can be:
the oracle's C source is compiled with -fsanitize=address,undefined and driven through every entry
point on small and degenerate inputs (a single point, single-point leaves with empty right
children, a single leaf, ties, the priority search with and without eps, reflections) in a child
process that preloads the sanitizer runtime.  Any out-of-bounds access, use after free or undefined
behaviour aborts the child.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOAD = r"""
import numpy as np
import oracle
from oracle import screen

rng = np.random.default_rng(0)
for n, d, T, p in ((1, 3, 2, 1), (9, 2, 3, 1), (300, 7, 3, 5), (257, 5, 4, 300), (64, 4, 2, 4)):
    X = rng.standard_normal((n, d)).astype(np.float32)
    if n == 64:
        X = np.round(X * 2) / 2          # many equal coordinates
    Q = rng.standard_normal((11, d)).astype(np.float32)
    for scope in (0, 1):
        for shuffle in (0, 1):
            F = oracle.build_forest(X, T, p, t=min(5, d), shuffle=shuffle, var_scope=scope, seed=3)
    k = min(4, n)
    leaf = oracle.descend(F, Q)
    offs, ids = oracle.candidates(F, leaf)
    oracle.topk(X, Q, offs, ids, k + 2)
    oracle.search(F, X, Q, k, return_ncand=True)
    nleaves = F.T << F.L
    for c, eps in ((F.T, 0.0), (F.T + 3, 0.0), (nleaves, 0.5), (nleaves + 5, 0.0)):
        oracle.search_priority(F, X, Q, k, c, eps, return_leaves=True)
    oracle.bruteforce(X, Q, k)
    oracle.variance(X)
    oracle.top_dims(oracle.variance(X), min(3, d))
    U = rng.standard_normal((T, d)).astype(np.float32)
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    G = oracle.build_forest(X, T, p, t=min(5, d), seed=5, U=U)
    oracle.search(G, X, Q, k)
    oracle.reflect(X[0], U[0])
    screen.screened_search(F, X, Q, k, 2 * k, "bf16")
    screen.screened_search(F, X, Q, k, 2 * k, "fp8")
print("sanitized oracle ok")
"""


def _runtime(name):
    try:
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    except OSError:
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_under_asan_and_ubsan(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("gcc has no AddressSanitizer runtime here")
    so = str(tmp_path / "libgforacle_san.so")
    r = subprocess.run(["gcc", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                        "-fPIC", "-o", so, os.path.join(ROOT, "oracle", "gf_oracle.c"), "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"sanitizer build unavailable: {r.stderr[-300:]}")
    env = dict(os.environ, GF_ORACLE_LIB=so, LD_PRELOAD=asan, PYTHONPATH=ROOT,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-c", WORKLOAD], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    assert p.returncode == 0 and "sanitized oracle ok" in p.stdout, p.stderr[-3000:]
    assert "AddressSanitizer" not in p.stderr and "runtime error" not in p.stderr, p.stderr[-3000:]
