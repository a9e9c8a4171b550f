"""CPU oracle for the kd-GeRaF search path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  The GPU library and its Python binding never import it, and it shares no code with them.

The arithmetic lives in ``gf_oracle.c`` (plain C, double precision, one function per step of
Alg. 1-3 of the paper); this module compiles it with gcc and marshals numpy arrays into it.
The precision-screening references (bfloat16 / FP8-E4M3 rounding) are plain numpy in
``oracle/screen.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_LIB = os.path.join(_HERE, "libgforacle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over trees and queries)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # GF_ORACLE_LIB: a prebuilt copy of the same source (e.g. a sanitizer build) to load instead
        path = os.environ.get("GF_ORACLE_LIB") or build()
        L = C.CDLL(path)
        i32, i64, u32, u64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        P = C.c_void_p
        L.gfo_splitmix64_at.argtypes = [u64, u64]; L.gfo_splitmix64_at.restype = u64
        L.gfo_fmix32.argtypes = [u32]; L.gfo_fmix32.restype = u32
        L.gfo_tree_key.argtypes = [u64, i32]; L.gfo_tree_key.restype = u64
        L.gfo_rank.argtypes = [u64, i32, i32, u32]; L.gfo_rank.restype = u32
        L.gfo_node_draw.argtypes = [u64, i32, i64]; L.gfo_node_draw.restype = u64
        L.gfo_depth.argtypes = [i64, i32]; L.gfo_depth.restype = i32
        L.gfo_variance.argtypes = [P, i32, P, i64, P]; L.gfo_variance.restype = None
        L.gfo_top_dims.argtypes = [P, i32, i32, P]; L.gfo_top_dims.restype = None
        L.gfo_build.argtypes = [P, i64, i32, i32, i32, i32, i32, i32, u64, P, P, P]
        L.gfo_build.restype = i32
        L.gfo_descend.argtypes = [P, P, i32, i32, P, i64, i32, P]; L.gfo_descend.restype = None
        L.gfo_candidates.argtypes = [P, i64, i32, i32, P, i64, P, P]; L.gfo_candidates.restype = i64
        L.gfo_dist2.argtypes = [P, P, i32]; L.gfo_dist2.restype = C.c_double
        L.gfo_topk.argtypes = [P, i32, P, i64, P, P, i32, P, P]; L.gfo_topk.restype = None
        L.gfo_search.argtypes = [P, i64, i32, P, P, P, i32, i32, P, i64, i32, P, P, P]
        L.gfo_search.restype = None
        L.gfo_bruteforce.argtypes = [P, i64, i32, P, i64, i32, P, P]; L.gfo_bruteforce.restype = None
        L.gfo_search_priority.argtypes = [P, i64, i32, P, P, P, i32, i32, P, i64, i32, i64, C.c_double,
                                          P, P, P, P, P, i64, P]
        L.gfo_reflect.argtypes = [P, P, i32, P]; L.gfo_reflect.restype = None
        L.gfo_build_reflected.argtypes = [P, i64, i32, i32, i32, i32, i32, i32, u64, P, P, P, P]
        L.gfo_build_reflected.restype = i32
        L.gfo_descend_reflected.argtypes = [P, P, i32, i32, P, i64, i32, P, P]
        L.gfo_descend_reflected.restype = None
        L.gfo_search_reflected.argtypes = [P, i64, i32, P, P, P, i32, i32, P, i64, i32, P, P, P, P]
        L.gfo_search_reflected.restype = None
        L.gfo_search_priority.restype = None
        L.gfo_search_f32.argtypes = [P, i64, i32, P, P, P, i32, i32, P, i64, i32, P, P]
        L.gfo_search_f32.restype = None
        L.gfo_num_threads.argtypes = []; L.gfo_num_threads.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------- random numbers

def splitmix64_at(s0: int, i: int) -> int:
    return lib().gfo_splitmix64_at(s0 & (2**64 - 1), i)


def fmix32(h: int) -> int:
    return lib().gfo_fmix32(h & 0xFFFFFFFF)


def rank(seed: int, tree: int, shuffle: int, i: int) -> int:
    return lib().gfo_rank(seed, tree, shuffle, i)


def node_draw(seed: int, tree: int, j: int) -> int:
    return lib().gfo_node_draw(seed, tree, j)


def num_threads() -> int:
    return lib().gfo_num_threads()


# ---------------------------------------------------------------- build

def depth(n: int, p: int) -> int:
    return lib().gfo_depth(n, p)


def variance(X: np.ndarray, idx: np.ndarray | None = None) -> np.ndarray:
    """Alg. 3 variance of rows X[idx] (all rows if idx is None), float64 [d]."""
    X = _f32(X)
    if idx is None:
        idx = np.arange(X.shape[0], dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(X.shape[1], dtype=np.float64)
    lib().gfo_variance(_p(X), X.shape[1], _p(idx), idx.shape[0], _p(out))
    return out


def top_dims(var: np.ndarray, t: int) -> np.ndarray:
    var = np.ascontiguousarray(var, dtype=np.float64)
    D = np.empty(t, dtype=np.int32)
    lib().gfo_top_dims(_p(var), var.shape[0], t, _p(D))
    return D


@dataclass
class Forest:
    """A forest in the flat layout both sides use: heap-ordered internal nodes and leaf perms."""
    n: int
    d: int
    T: int
    leaf_size: int
    L: int
    split_dim: np.ndarray  # int32 [T, 2^L - 1]
    split_val: np.ndarray  # float32 [T, 2^L - 1]
    perm: np.ndarray       # int32 [T, n]
    U: np.ndarray | None = None  # float32 [T, d]: per-tree Householder vectors (Sec. 2.2), or None

    def leaf_range(self, b: int) -> tuple[int, int]:
        return (b * self.n) >> self.L, ((b + 1) * self.n) >> self.L


def build_forest(X: np.ndarray, T: int, leaf_size: int, t: int = 5, shuffle: int = 1,
                 var_scope: int = 0, seed: int = 0, U: np.ndarray | None = None) -> Forest:
    """Alg. 1: T randomized trees on X (readings R1-R5 of gf_oracle.c); with U [T, d] each tree is
    built on its Householder-reflected points (Sec. 2.2)."""
    X = _f32(X)
    n, d = X.shape
    L = depth(n, leaf_size)
    nn = (1 << L) - 1
    sd = np.zeros((T, nn), dtype=np.int32)
    sv = np.zeros((T, nn), dtype=np.float32)
    pm = np.zeros((T, n), dtype=np.int32)
    Up = None
    if U is not None:
        U = _f32(U)
        assert U.shape == (T, d)
        Up = _p(U)
    r = lib().gfo_build_reflected(_p(X), n, d, T, leaf_size, t, shuffle, var_scope, seed, Up, _p(sd), _p(sv),
                                  _p(pm))
    if r < 0:
        raise ValueError("gfo_build: invalid arguments")
    assert r == L
    return Forest(n, d, T, leaf_size, L, sd, sv, pm, U)


def reflect(x: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Px = x - 2 (u^T x) u (Sec. 2.2), with the rounding steps gfo_reflect fixes."""
    x, u = _f32(x), _f32(u)
    if x.ndim != 1 or x.shape != u.shape:
        raise ValueError("reflect takes one vector x and a vector u of the same length")
    out = np.empty_like(x)
    lib().gfo_reflect(_p(x), _p(u), x.shape[0], _p(out))
    return out


def _Up(F: "Forest"):
    return _p(np.ascontiguousarray(F.U, dtype=np.float32)) if F.U is not None else None


# ---------------------------------------------------------------- search

def descend(F: Forest, Q: np.ndarray) -> np.ndarray:
    """leaf[i, t]: the leaf of tree t reached by query i (Alg. 2 "descend", Eq. 1)."""
    Q = _f32(Q)
    m = Q.shape[0]
    leaf = np.empty((m, F.T), dtype=np.int32)
    lib().gfo_descend_reflected(_p(np.ascontiguousarray(F.split_dim)), _p(np.ascontiguousarray(F.split_val)),
                                F.L, F.T, _p(Q), m, F.d, _Up(F), _p(leaf))
    return leaf


def candidates(F: Forest, leaf: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sorted, de-duplicated union of each query's T leaves, as CSR (offs int64, ids int32)."""
    leaf = np.ascontiguousarray(leaf, dtype=np.int32)
    m = leaf.shape[0]
    cap = ((F.n + (1 << F.L) - 1) >> F.L) * F.T
    offs = np.empty(m + 1, dtype=np.int64)
    ids = np.empty(max(1, m * cap), dtype=np.int32)
    tot = lib().gfo_candidates(_p(np.ascontiguousarray(F.perm)), F.n, F.L, F.T, _p(leaf), m,
                               _p(offs), _p(ids))
    return offs, ids[:tot].copy()


def topk(X: np.ndarray, Q: np.ndarray, offs: np.ndarray, ids: np.ndarray, k: int):
    """k nearest (distance, id) among each query's candidates, float64 distances."""
    X, Q = _f32(X), _f32(Q)
    m = Q.shape[0]
    oi = np.empty((m, k), dtype=np.int64)
    od = np.empty((m, k), dtype=np.float64)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    ids = np.ascontiguousarray(ids if ids.size else np.zeros(1, np.int32), dtype=np.int32)
    lib().gfo_topk(_p(X), X.shape[1], _p(Q), m, _p(offs), _p(ids), k, _p(oi), _p(od))
    return oi, od


def search(F: Forest, X: np.ndarray, Q: np.ndarray, k: int, return_ncand: bool = False):
    """Whole search (Alg. 2 with c = T): ids int64 [m, k], dists float64 [m, k]."""
    X, Q = _f32(X), _f32(Q)
    m = Q.shape[0]
    oi = np.empty((m, k), dtype=np.int64)
    od = np.empty((m, k), dtype=np.float64)
    nc = np.empty(m, dtype=np.int64)
    lib().gfo_search_reflected(_p(X), F.n, F.d, _p(np.ascontiguousarray(F.split_dim)),
                               _p(np.ascontiguousarray(F.split_val)), _p(np.ascontiguousarray(F.perm)),
                               F.L, F.T, _p(Q), m, k, _Up(F), _p(oi), _p(od), _p(nc))
    return (oi, od, nc) if return_ncand else (oi, od)


def search_f32(F: Forest, X: np.ndarray, Q: np.ndarray, k: int):
    """The same search with float32 distance arithmetic in a plain loop (a CPU baseline to time,
    not a reference): ids int64 [m, k], dists [m, k] (float32 values)."""
    if F.U is not None:
        raise ValueError("search_f32 takes plain forests only")
    X, Q = _f32(X), _f32(Q)
    m = Q.shape[0]
    oi = np.empty((m, k), dtype=np.int64)
    od = np.empty((m, k), dtype=np.float64)
    lib().gfo_search_f32(_p(X), F.n, F.d, _p(np.ascontiguousarray(F.split_dim)),
                         _p(np.ascontiguousarray(F.split_val)), _p(np.ascontiguousarray(F.perm)),
                         F.L, F.T, _p(Q), m, k, _p(oi), _p(od))
    return oi, od


def search_priority(F: Forest, X: np.ndarray, Q: np.ndarray, k: int, c: int, eps: float = 0.0,
                    return_leaves: bool = False):
    """Alg. 2 with the shared priority queue: at least the T first leaves, then leaves in order of
    |q_s - v| until c / (1 + eps) were checked.  Returns ids, dists, candidates, leaves checked (and
    with return_leaves the leaf sequence, (tree << L) | leaf, -1 padded)."""
    X, Q = _f32(X), _f32(Q)
    m = Q.shape[0]
    oi = np.empty((m, k), dtype=np.int64)
    od = np.empty((m, k), dtype=np.float64)
    nc = np.empty(m, dtype=np.int64)
    nl = np.empty(m, dtype=np.int64)
    cap = max(int(c / (1.0 + eps)) + 1, F.T)
    seq = np.full((m, cap), -1, dtype=np.int64)
    lib().gfo_search_priority(_p(X), F.n, F.d, _p(np.ascontiguousarray(F.split_dim)),
                              _p(np.ascontiguousarray(F.split_val)), _p(np.ascontiguousarray(F.perm)),
                              F.L, F.T, _p(Q), m, k, c, eps, _p(oi), _p(od), _p(nc), _p(nl), _p(seq), cap,
                              _Up(F))
    return (oi, od, nc, nl, seq) if return_leaves else (oi, od, nc, nl)


def bruteforce(X: np.ndarray, Q: np.ndarray, k: int):
    """Exact k-NN by brute force, float64 distances, ordered by (distance, id)."""
    X, Q = _f32(X), _f32(Q)
    m = Q.shape[0]
    oi = np.empty((m, k), dtype=np.int64)
    od = np.empty((m, k), dtype=np.float64)
    lib().gfo_bruteforce(_p(X), X.shape[0], X.shape[1], _p(Q), m, k, _p(oi), _p(od))
    return oi, od


def dist2(q: np.ndarray, x: np.ndarray) -> float:
    q, x = _f32(q), _f32(x)
    return lib().gfo_dist2(_p(q), _p(x), q.shape[0])


# ---------------------------------------------------------------- metrics

def recall_at_1(ids: np.ndarray, exact_d: np.ndarray, X: np.ndarray, Q: np.ndarray) -> float:
    """Share of queries whose first result lies at the exact NN distance (ties accepted, Sec. 4)."""
    hit = 0
    for i in range(ids.shape[0]):
        if ids[i, 0] < 0:
            continue
        if dist2(Q[i], X[ids[i, 0]]) <= exact_d[i, 0]:
            hit += 1
    return hit / max(1, ids.shape[0])


def recall_at_k(ids: np.ndarray, exact_ids: np.ndarray) -> float:
    k = exact_ids.shape[1]
    tot = 0
    for i in range(ids.shape[0]):
        tot += len(set(ids[i].tolist()) & set(exact_ids[i].tolist()) - {-1})
    return tot / (k * max(1, ids.shape[0]))
