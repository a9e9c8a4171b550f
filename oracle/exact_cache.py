"""Exact nearest neighbours of the benchmark's recall samples, by the oracle's float64 brute force --
TEST INFRASTRUCTURE (see oracle/__init__.py).

Recall (Sec. 4: a query is a miss unless its answer lies at the exact nearest distance) and the
distance error of the returned results need the exact k nearest neighbours of every sampled query.
They cost a brute-force pass over all n points per query, so they are computed once per workload
(law, sizes, seeds) by oracle.bruteforce and kept as text files under oracle/exact/.  This script
writes them; bench.py only reads them:

    python oracle/exact_cache.py            # every workload bench.py samples

A file holds the workload's description, the ids and the float64 squared distances, ordered by
(distance, id) as the oracle returns them.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

CACHE = os.path.join(HERE, "exact")

# (law, n, d, data seed, query seed, queries drawn, queries in the sample, k): the recall samples of
# bench.py -- the first `sample` of the `m` queries the workload draws
WORKLOADS = [
    ("A", 10_000, 128, 0, 1, 100, 100, 10),          # 10^4 x 128 (tiny)
    ("B", 1_000_000, 960, 0, 1, 10_000, 1000, 10),   # the 10^6 x 960 headline workload
    ("B", 100_000, 960, 0, 1, 10_000, 1000, 10),     # 10^5 x 960
    ("C", 200_000, 10_000, 0, 1, 2_000, 200, 10),    # 2 x 10^5 x 10^4
]


def path_of(law: str, n: int, d: int, seed: int, qseed: int, m: int, nq: int, k: int) -> str:
    return os.path.join(CACHE, f"law{law}_n{n}_d{d}_s{seed}_q{qseed}_m{m}_first{nq}_k{k}.json")


def load(law: str, n: int, d: int, seed: int, qseed: int, m: int, nq: int, k: int):
    """(ids int64 [nq, k], squared distances float64 [nq, k]) of the first nq of the m queries, or None."""
    p = path_of(law, n, d, seed, qseed, m, nq, k)
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    return np.array(j["ids"], dtype=np.int64), np.array(j["dist2"], dtype=np.float64)


def compute(law: str, n: int, d: int, seed: int, qseed: int, m: int, nq: int, k: int) -> str:
    import oracle
    import synth
    X, Q = synth.mixture(n, d, m, law, seed=seed, qseed=qseed)
    t0 = time.time()
    ids, dist = oracle.bruteforce(X, np.ascontiguousarray(Q[:nq]), k)
    p = path_of(law, n, d, seed, qseed, m, nq, k)
    os.makedirs(CACHE, exist_ok=True)
    with open(p, "w") as f:
        json.dump({"law": law, "n": n, "d": d, "seed": seed, "qseed": qseed, "m": m, "queries": nq, "k": k,
                   "how": "oracle.bruteforce (float64 distances of the float32 points), first nq of m queries",
                   "seconds": round(time.time() - t0, 1), "threads": oracle.num_threads(),
                   "ids": ids.tolist(), "dist2": [[float(v) for v in row] for row in dist]}, f)
    return p


if __name__ == "__main__":
    only = sys.argv[1:]
    for w in WORKLOADS:
        if only and w[0] + str(w[1]) not in only:
            continue
        if load(*w) is None:
            print(compute(*w), flush=True)
