"""The cached exact nearest neighbours the benchmark reads (oracle/exact/, written by
oracle/exact_cache.py) are what the oracle's brute force gives: the tiny workload in full, the
10^5-point one on a few of its queries (the brute force of all of them takes minutes)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import exact_cache


def _check(w, rows):
    law, n, d, seed, qseed, m, nq, k = w
    got = exact_cache.load(*w)
    if got is None:
        pytest.skip(f"no cache file for {w}")
    ids, d2 = got
    assert ids.shape == (nq, k) and d2.shape == (nq, k)
    X, Q = synth.mixture(n, d, m, law, seed=seed, qseed=qseed)
    ri, rd = oracle.bruteforce(X, np.ascontiguousarray(Q[rows]), k)
    assert np.array_equal(ids[rows], ri)
    assert np.array_equal(d2[rows], rd)


def test_tiny_cache_is_the_oracle_brute_force():
    w = next(w for w in exact_cache.WORKLOADS if w[1] == 10_000)
    _check(w, np.arange(w[6]))


def test_gist100k_cache_on_sampled_queries():
    w = next(w for w in exact_cache.WORKLOADS if w[1] == 100_000)
    _check(w, np.array([0, 517, 999]))
