"""Pins for the CPU oracle: each check comes from something other than the oracle itself.

Sources of truth used here: published generator outputs, a hand-derived forest, numpy's two-pass
variance and sorts, closed-form variances, brute force in numpy, and invariants the paper's
construction implies (Alg. 1: every tree partitions all points; Alg. 2 / Eq. 1: the query takes the
side of the sign of q_s - v).  Every test here runs on the CPU.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from parity import check_forest as _check_forest


# ------------------------------------------------------------------ random numbers

def test_splitmix64_known_answer(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "rng.json")))
    sm = g["splitmix64"]
    assert oracle.splitmix64_at(sm["state0"], 0) == int(sm["first_output_hex"], 16)


def test_fmix32_known_answers(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "rng.json")))
    for x, y in g["fmix32"]["cases"]:
        assert oracle.fmix32(int(x, 16)) == int(y, 16)


def test_splitmix64_output_is_invertible():
    # The output mix is a bijection: undo each xor-shift and odd multiply (inverses derived from
    # the definition, not from the oracle), recovering the stream state s0 + (i+1) * gamma.
    M = 2**64
    gamma = 0x9E3779B97F4A7C15

    def unxorshift(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x

    inv1 = pow(0xBF58476D1CE4E5B9, -1, M)
    inv2 = pow(0x94D049BB133111EB, -1, M)
    for s0, i in [(0, 0), (12345, 7), (2**63 + 5, 1000)]:
        z = oracle.splitmix64_at(s0, i)
        z = unxorshift(z, 31)
        z = (z * inv2) % M
        z = unxorshift(z, 27)
        z = (z * inv1) % M
        z = unxorshift(z, 30)
        assert z == (s0 + (i + 1) * gamma) % M


def test_rank_is_a_permutation_per_tree():
    # R2: rk_t must give distinct tie-break keys to distinct points.
    ids = range(4096)
    for tree in range(3):
        r = [oracle.rank(7, tree, 1, i) for i in ids]
        assert len(set(r)) == len(r)
    assert [oracle.rank(7, 0, 0, i) for i in range(10)] == list(range(10))
    assert [oracle.rank(7, 0, 1, i) for i in range(10)] != [oracle.rank(7, 1, 1, i) for i in range(10)]


def test_node_draw_is_roughly_uniform_mod_t():
    draws = np.array([oracle.node_draw(0, 0, j) % 5 for j in range(5000)])
    counts = np.bincount(draws, minlength=5)
    assert counts.min() > 850 and counts.max() < 1150


# ------------------------------------------------------------------ Alg. 3 variance

@pytest.mark.parametrize("n,d", [(2, 3), (17, 5), (1000, 64)])
def test_variance_matches_two_pass(n, d):
    rng = np.random.default_rng(n)
    X = (rng.standard_normal((n, d)) * 3 + 10).astype(np.float32)
    v = oracle.variance(X)
    ref = X.astype(np.float64).var(axis=0, ddof=1)
    np.testing.assert_allclose(v, ref, rtol=1e-12, atol=0)


def test_variance_subset_and_special_cases():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 4)).astype(np.float32)
    idx = np.array([3, 9, 1, 44, 20], dtype=np.int32)
    np.testing.assert_allclose(oracle.variance(X, idx), X[idx].astype(np.float64).var(0, ddof=1),
                               rtol=1e-12)
    assert np.all(oracle.variance(X, np.array([5], np.int32)) == 0)      # fewer than two vectors
    assert np.all(oracle.variance(X, np.array([], np.int32)) == 0)
    C = np.full((30, 3), 2.5, dtype=np.float32)
    assert np.all(oracle.variance(C) == 0)                                # constant data


def test_variance_closed_form():
    # values 0..n-1: variance n(n+1)/12
    n = 1001
    X = np.arange(n, dtype=np.float32)[:, None]
    assert oracle.variance(X)[0] == pytest.approx(n * (n + 1) / 12, rel=1e-13)


def test_top_dims_order_and_ties():
    rng = np.random.default_rng(4)
    var = rng.random(100)
    var[[10, 20, 30]] = 5.0                  # three-way tie at the top
    D = oracle.top_dims(var, 5)
    ref = np.lexsort((np.arange(100), -var))[:5]
    assert D.tolist() == ref.tolist()
    assert D[:3].tolist() == [10, 20, 30]


# ------------------------------------------------------------------ tree shape

def test_depth_values():
    # L = min{l : ceil(n / 2^l) <= p}, worked by hand for the workload shapes
    assert oracle.depth(10_000, 32) == 9        # 10000/512 = 19.5 -> 20 <= 32; /256 -> 40 > 32
    assert oracle.depth(100_000, 64) == 11      # /2048 -> 49; /1024 -> 98
    assert oracle.depth(1_000_000, 64) == 14    # /16384 -> 62; /8192 -> 123
    assert oracle.depth(200_000, 32) == 13      # /8192 -> 25; /4096 -> 49
    assert oracle.depth(5, 5) == 0 and oracle.depth(5, 100) == 0 and oracle.depth(6, 5) == 1


# ------------------------------------------------------------------ hand-derived forest

def test_hand_built_forest(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_2d.json")))
    X = np.array(g["X"], dtype=np.float32)
    F = oracle.build_forest(X, g["T"], g["leaf_size"], t=g["t"], shuffle=g["shuffle"],
                            var_scope=g["var_scope"], seed=0)
    assert F.L == g["L"]
    assert F.split_dim[0].tolist() == g["split_dim"]
    assert F.split_val[0].tolist() == g["split_val"]
    assert F.perm[0].tolist() == g["perm"]
    np.testing.assert_allclose(oracle.variance(X), g["root_variance"], rtol=1e-14)
    Qh = np.array(g["queries"], dtype=np.float32)
    assert oracle.descend(F, Qh)[:, 0].tolist() == g["leaf"]
    ids, d = oracle.search(F, X, Qh, 1)
    assert ids[:, 0].tolist() == g["nn1_ids"]
    np.testing.assert_allclose(d[:, 0], g["nn1_dist"], rtol=1e-6)
    ei, _ = oracle.bruteforce(X, Qh, 1)
    assert ei[:, 0].tolist() == g["exact_nn1_ids"]


# ------------------------------------------------------------------ forest invariants

@pytest.mark.parametrize("var_scope", [0, 1])
def test_forest_invariants_mixture(var_scope):
    X, _ = synth.mixture(600, 16, 1, "A", seed=2)
    F = oracle.build_forest(X, 3, 20, t=5, shuffle=1, var_scope=var_scope, seed=11)
    _check_forest(F, X, 5, 11, 1, var_scope)


def test_forest_invariants_quantized_ties():
    # Byte-valued data: many equal split coordinates, broken by the per-tree order (Sec. 2.1).
    X, _ = synth.mixture(500, 8, 1, "B", seed=3)
    X = synth.quantize_u8(X, 4.0)
    F1 = oracle.build_forest(X, 2, 16, t=3, shuffle=1, seed=5)
    _check_forest(F1, X, 3, 5, 1, 0, check_dims=False)
    F0 = oracle.build_forest(X, 2, 16, t=3, shuffle=0, seed=5)
    _check_forest(F0, X, 3, 5, 0, 0, check_dims=False)
    assert not np.array_equal(F0.perm, F1.perm)


@pytest.mark.parametrize("n", [5, 13, 64])
def test_single_point_leaves(n):
    # p = 1 (Table 4's smallest leaf): perfect trees may leave a leaf empty, never misplace a point
    X, Q = synth.mixture(n, 4, 6, "A", seed=n)
    F = oracle.build_forest(X, 2, 1, t=2, seed=3)
    _check_forest(F, X, 2, 3, 1, 0)
    leaf = oracle.descend(F, X)
    for tr in range(F.T):
        for i in range(n):
            lo, hi = F.leaf_range(int(leaf[i, tr]))
            assert i in F.perm[tr, lo:hi].tolist()


def test_trees_are_independent_of_forest_size():
    X, _ = synth.mixture(800, 12, 1, "A", seed=4)
    F4 = oracle.build_forest(X, 4, 25, seed=9)
    F7 = oracle.build_forest(X, 7, 25, seed=9)
    assert np.array_equal(F4.perm, F7.perm[:4])
    assert np.array_equal(F4.split_dim, F7.split_dim[:4])


# ------------------------------------------------------------------ search

def _np_bruteforce(X, Q, k):
    D = ((Q[:, None, :].astype(np.float64) - X[None, :, :].astype(np.float64)) ** 2).sum(-1)
    ids = np.lexsort((np.broadcast_to(np.arange(X.shape[0]), D.shape), D), axis=1)[:, :k]
    return ids, np.take_along_axis(D, ids, 1)


def test_bruteforce_matches_numpy():
    X, Q = synth.mixture(700, 20, 15, "A", seed=6)
    ids, d = oracle.bruteforce(X, Q, 5)
    rid, rd = _np_bruteforce(X, Q, 5)
    np.testing.assert_allclose(d, rd, rtol=1e-12)
    assert np.array_equal(ids, rid)


def test_leaf_size_at_least_n_is_exact_knn():
    # c = n reduces the search to brute force (Sec. 4, approximate search evaluation)
    X, Q = synth.mixture(300, 10, 20, "A", seed=7)
    F = oracle.build_forest(X, 3, 300, seed=0)
    assert F.L == 0
    ids, d = oracle.search(F, X, Q, 7)
    rid, rd = _np_bruteforce(X, Q, 7)
    assert np.array_equal(ids, rid)
    np.testing.assert_allclose(d, rd, rtol=1e-12)


def test_float32_search_is_the_float64_search_up_to_its_rounding():
    # the float32 CPU baseline: same candidates, distances within (d + 2) 2^-24 of float64 (a sum of
    # non-negative terms), ids equal except where two candidates lie within that bound
    X, Q = synth.mixture(3000, 96, 60, "B", seed=9, qseed=10)
    F = oracle.build_forest(X, 6, 24, seed=2)
    oi, od = oracle.search(F, X, Q, 8)
    fi, fd = oracle.search_f32(F, X, Q, 8)
    tol = (X.shape[1] + 2) * 2.0 ** -24
    fin = oi >= 0
    assert np.array_equal(fi >= 0, fin)
    assert np.all(np.abs(fd[fin] - od[fin]) <= tol * od[fin])
    for i, j in zip(*np.nonzero((fi != oi) & fin)):
        assert abs(oracle.dist2(Q[i], X[fi[i, j]]) - od[i, j]) <= 2 * tol * od[i, j]
    # with one leaf holding everything it is a brute force in float32
    F1 = oracle.build_forest(X[:500], 2, 500, seed=0)
    bi, bd = oracle.search_f32(F1, X[:500], Q, 3)
    ri, rd = _np_bruteforce(X[:500], Q, 3)
    assert np.mean(bi == ri) >= 0.99


def test_descent_follows_sign_of_eq1():
    X, Q = synth.mixture(1000, 16, 40, "A", seed=8)
    F = oracle.build_forest(X, 4, 30, seed=3)
    leaf = oracle.descend(F, Q)
    for i in range(Q.shape[0]):
        for tr in range(F.T):
            b = int(leaf[i, tr])
            j = 0
            for l in range(F.L):
                bit = (b >> (F.L - 1 - l)) & 1
                s, v = F.split_dim[tr, j], F.split_val[tr, j]
                assert (Q[i, s] - v < 0) == (bit == 0)
                j = 2 * j + 1 + bit


def test_data_point_query_reaches_its_own_leaf():
    # Continuous data has no ties, so a data point used as a query lands in the leaf holding it.
    X, _ = synth.mixture(1200, 24, 1, "B", seed=9)
    F = oracle.build_forest(X, 5, 40, seed=1)
    leaf = oracle.descend(F, X)
    for tr in range(F.T):
        for b in range(1 << F.L):
            lo, hi = F.leaf_range(b)
            for i in F.perm[tr, lo:hi]:
                assert leaf[i, tr] == b


def test_candidates_and_topk_against_sets():
    X, Q = synth.mixture(2000, 32, 25, "A", seed=10)
    F = oracle.build_forest(X, 6, 40, seed=2)
    leaf = oracle.descend(F, Q)
    offs, cid = oracle.candidates(F, leaf)
    ids, d, nc = oracle.search(F, X, Q, 4, return_ncand=True)
    for i in range(Q.shape[0]):
        u = set()
        for tr in range(F.T):
            lo, hi = F.leaf_range(int(leaf[i, tr]))
            u |= set(F.perm[tr, lo:hi].tolist())
        got = cid[offs[i]:offs[i + 1]]
        assert got.tolist() == sorted(u)
        assert nc[i] == len(u)
        cl = np.array(sorted(u))
        rid, rd = _np_bruteforce(X[cl], Q[i:i + 1], 4)
        assert ids[i].tolist() == cl[rid[0]].tolist()
        np.testing.assert_allclose(d[i], rd[0], rtol=1e-12)
    oi, od = oracle.topk(X, Q, offs, cid, 4)
    assert np.array_equal(oi, ids) and np.array_equal(od, d)


def test_topk_pads_when_fewer_candidates():
    X, Q = synth.mixture(64, 8, 3, "A", seed=12)
    F = oracle.build_forest(X, 1, 4, seed=0)       # leaves of 4 points, one tree
    ids, d = oracle.search(F, X, Q, 6)
    assert np.all(ids[:, 4:] == -1) and np.all(np.isinf(d[:, 4:]))
    assert np.all(ids[:, :4] >= 0)


def test_more_trees_never_hurt():
    X, Q = synth.mixture(3000, 32, 60, "A", seed=13)
    F = oracle.build_forest(X, 8, 32, seed=4)
    best_prev = np.full(Q.shape[0], np.inf)
    for T in (1, 2, 4, 8):
        sub = oracle.Forest(F.n, F.d, T, F.leaf_size, F.L, F.split_dim[:T], F.split_val[:T], F.perm[:T])
        _, d = oracle.search(sub, X, Q, 1)
        assert np.all(d[:, 0] <= best_prev)
        best_prev = d[:, 0]


def test_recall_metrics():
    X, Q = synth.mixture(500, 8, 30, "A", seed=14)
    ei, ed = oracle.bruteforce(X, Q, 3)
    assert oracle.recall_at_1(ei, ed, X, Q) == 1.0
    assert oracle.recall_at_k(ei, ei) == 1.0
    wrong = ei.copy()
    wrong[:, 0] = ei[:, 2]
    assert oracle.recall_at_1(wrong, ed, X, Q) < 1.0


# ------------------------------------------------------------------ Alg. 2 priority search

def test_priority_search_hand_order(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_2d.json")))
    X = np.array(g["X"], dtype=np.float32)
    F = oracle.build_forest(X, 1, 2, t=1, shuffle=0, seed=0)
    q = np.array([g["priority_query"]], dtype=np.float32)
    for c, e in g["priority_expect"].items():
        ids, d, nc, nl = oracle.search_priority(F, X, q, 1, int(c))
        assert (nl[0], nc[0], ids[0, 0]) == (e["leaves"], e["cand"], e["id"])


def test_priority_search_with_c_equal_T_is_one_leaf_per_tree():
    X, Q = synth.mixture(3000, 24, 40, "B", seed=21)
    F = oracle.build_forest(X, 6, 30, seed=2)
    ids, d, nc = oracle.search(F, X, Q, 5, return_ncand=True)
    pi, pd, pnc, pnl = oracle.search_priority(F, X, Q, 5, F.T)
    assert np.array_equal(pi, ids) and np.array_equal(pd, d) and np.array_equal(pnc, nc)
    assert np.all(pnl == F.T)


def test_priority_search_all_leaves_is_exact():
    X, Q = synth.mixture(600, 12, 30, "A", seed=22)
    F = oracle.build_forest(X, 2, 20, seed=1)
    ids, d, nc, nl = oracle.search_priority(F, X, Q, 4, F.T << F.L)
    ei, ed = oracle.bruteforce(X, Q, 4)
    assert np.array_equal(ids, ei) and np.all(nc == 600)


def test_priority_search_budget_and_monotonicity():
    X, Q = synth.mixture(4000, 32, 50, "B", seed=23)
    F = oracle.build_forest(X, 4, 25, seed=3)
    prev = np.full(Q.shape[0], np.inf)
    for c in (4, 8, 16, 40, 100):
        ids, d, nc, nl = oracle.search_priority(F, X, Q, 1, c)
        assert np.all(nl == c)
        assert np.all(d[:, 0] <= prev)
        prev = d[:, 0]
    # c / (1 + eps) leaves: eps = 1 halves the budget (Sec. 2.3)
    _, _, _, nl = oracle.search_priority(F, X, Q, 1, 40, eps=1.0)
    assert np.all(nl == 20)


def test_priority_pop_order_across_trees(golden_dir):
    # a hand-made two-tree forest: the queue mixes both trees and breaks a key tie by tree
    g = json.load(open(os.path.join(golden_dir, "hand_prio_2trees.json")))
    X = np.array(g["X"], dtype=np.float32)
    F = oracle.Forest(8, 2, 2, 2, g["L"], np.array(g["split_dim"], dtype=np.int32),
                      np.array(g["split_val"], dtype=np.float32), np.array(g["perm"], dtype=np.int32))
    q = np.array([g["query"]], dtype=np.float32)
    _, _, nc, nl, seq = oracle.search_priority(F, X, q, 1, 8, return_leaves=True)
    assert seq[0, :8].tolist() == g["sequence"]
    for c, cand in g["candidates_after_c"].items():
        _, _, nc, nl = oracle.search_priority(F, X, q, 1, int(c))
        assert (nl[0], nc[0]) == (int(c), cand)


# ------------------------------------------------------------------ Householder reflection (Sec. 2.2)

def _units(T, d, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((T, d))
    return (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)


def test_reflection_basis_vector_flips_one_coordinate():
    x = np.float32([1.5, -2.25, 3.0, 0.5])
    u = np.float32([0, 0, 1, 0])
    assert oracle.reflect(x, u).tolist() == [1.5, -2.25, -3.0, 0.5]


def test_reflection_is_an_involutive_isometry():
    rng = np.random.default_rng(31)
    u = _units(1, 50, 32)[0]
    x, y = rng.standard_normal((2, 50)).astype(np.float32)
    px, py = oracle.reflect(x, u), oracle.reflect(y, u)
    # float32 arithmetic: within a few units of rounding of the exact reflection
    np.testing.assert_allclose(oracle.reflect(px, u), x, atol=1e-4)
    assert np.linalg.norm(px - py) == pytest.approx(np.linalg.norm(x - y), rel=1e-4)
    assert np.dot(px.astype(np.float64), u) == pytest.approx(-np.dot(x.astype(np.float64), u), abs=1e-4)


def test_reflected_tree_is_the_tree_of_reflected_points():
    X, _ = synth.mixture(900, 10, 1, "B", seed=33)
    U = _units(3, 10, 34)
    F = oracle.build_forest(X, 3, 20, seed=5, U=U)
    for t in range(3):
        Xt = np.stack([oracle.reflect(x, U[t]) for x in X])
        Ft = oracle.build_forest(Xt, 3, 20, seed=5)
        assert np.array_equal(F.split_dim[t], Ft.split_dim[t])
        assert np.array_equal(F.split_val[t], Ft.split_val[t])
        assert np.array_equal(F.perm[t], Ft.perm[t])


def test_reflected_forest_data_point_reaches_its_leaf():
    # queries are reflected before descending (Sec. 2.3) with the same arithmetic as the points
    X, _ = synth.mixture(1000, 16, 1, "B", seed=35)
    U = _units(4, 16, 36)
    F = oracle.build_forest(X, 4, 30, seed=2, U=U)
    leaf = oracle.descend(F, X)
    for tr in range(F.T):
        for b in range(1 << F.L):
            lo, hi = F.leaf_range(b)
            for i in F.perm[tr, lo:hi]:
                assert leaf[i, tr] == b


def test_reflected_single_leaf_is_exact_on_original_distances():
    X, Q = synth.mixture(200, 8, 15, "A", seed=37)
    F = oracle.build_forest(X, 2, 200, seed=0, U=_units(2, 8, 38))
    ids, d = oracle.search(F, X, Q, 5)
    ei, ed = oracle.bruteforce(X, Q, 5)
    assert np.array_equal(ids, ei)
    np.testing.assert_allclose(d, ed, rtol=1e-12)
