"""Comparison rules shared by the GPU parity tests.

Floating point: float32 GPU distances must lie within RTOL (1e-5) relative of the float64 oracle.
Integers (leaves, candidate ids) must match exactly.  k-NN ids must match exactly except inside a
near-tie: where the GPU's id differs from the oracle's at a position, the GPU's point must be a
candidate whose float64 distance lies within RTOL * (largest distance of the row) of the oracle's
distance at that position -- an equally good answer (Sec. 4 accepts any point at the same
distance as correct).
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL = 1e-5


def assert_topk_close(X, Q, g_ids, g_d, o_ids, o_d, cand_sets=None, max_tie_frac=0.02, rtol=RTOL):
    """Compare GPU (g_*) and oracle (o_*) top-k results row by row."""
    g_ids = np.asarray(g_ids)
    g_d = np.asarray(g_d, dtype=np.float64)
    o_ids = np.asarray(o_ids)
    o_d = np.asarray(o_d, dtype=np.float64)
    assert g_ids.shape == o_ids.shape
    m, k = o_ids.shape
    pad_o = o_ids < 0
    assert np.array_equal(g_ids < 0, pad_o), "padding (-1) positions differ"
    assert np.all(np.isinf(g_d[pad_o])), "padded distances must be +inf"
    fin = ~pad_o
    scale = np.where(fin, o_d, 0).max(axis=1, keepdims=True)
    scale = np.maximum(scale, 1e-30)
    err = np.abs(g_d - o_d) / scale
    assert np.all(err[fin] <= rtol), f"distance error {err[fin].max():.3g} > {rtol}"
    mism = (g_ids != o_ids) & fin
    rows = np.unique(np.nonzero(mism)[0])
    for i in rows:
        for j in np.nonzero(mism[i])[0]:
            gid = int(g_ids[i, j])
            if cand_sets is not None:
                assert gid in cand_sets[i], f"query {i}: id {gid} is not a candidate"
            true = oracle.dist2(Q[i], X[gid])
            assert abs(true - o_d[i, j]) <= rtol * scale[i, 0], \
                f"query {i} pos {j}: id {gid} at {true} is not a near-tie of {o_ids[i, j]} at {o_d[i, j]}"
        assert len(set(g_ids[i][fin[i]].tolist())) == int(fin[i].sum()), f"query {i}: repeated id"
    assert len(rows) <= max(1, int(max_tie_frac * m)), f"{len(rows)} of {m} rows differ"
    return len(rows)


def assert_screened_close(X, Q, gi, gd, oi, od, cands, max_frac=0.03):
    """Like assert_topk_close, but a row may also differ where the float32 screen and the float64
    screen order the shortlist boundary differently; every reported id must still be a candidate
    reported with its exact distance, and such rows must be rare."""
    m, k = oi.shape
    bad = 0
    for i in range(m):
        fin = oi[i] >= 0
        assert np.array_equal(gi[i] >= 0, fin)
        if np.array_equal(gi[i], oi[i]):
            np.testing.assert_allclose(gd[i][fin], od[i][fin], rtol=RTOL)
            continue
        bad += 1
        for j in np.nonzero(fin)[0]:
            gid = int(gi[i, j])
            assert gid in cands[i]
            true = oracle.dist2(Q[i], X[gid])
            assert abs(true - gd[i, j]) <= RTOL * max(true, 1e-30)
        assert np.all(np.diff(gd[i][fin]) >= 0)
    assert bad <= max(1, int(max_frac * m)), f"{bad} of {m} rows differ"


def candidate_sets(offs, ids):
    return [set(ids[offs[i]:offs[i + 1]].tolist()) for i in range(len(offs) - 1)]


# ------------------------------------------------------------------ forest invariants

def _node_points(F, tree, l, a):
    lo, hi = (a * F.n) >> l, ((a + 1) * F.n) >> l
    return F.perm[tree, lo:hi]


def check_forest(F, X, t, seed, shuffle, var_scope, check_dims=True):
    n, L = F.n, F.L
    Xd = X.astype(np.float64)
    gvar = Xd.var(0, ddof=1) if n > 1 else np.zeros(X.shape[1])
    for tree in range(F.T):
        assert np.array_equal(np.sort(F.perm[tree]), np.arange(n))        # partition of all points
        rk = np.array([oracle.rank(seed, tree, shuffle, i) for i in range(n)], dtype=np.uint64)
        for b in range(1 << L):
            lo, hi = F.leaf_range(b)
            assert (1 if F.leaf_size > 1 else 0) <= hi - lo <= F.leaf_size
            assert np.all(np.diff(F.perm[tree, lo:hi]) > 0)                # ascending ids (R2)
        for l in range(L):
            for a in range(1 << l):
                j = (1 << l) - 1 + a
                pts = _node_points(F, tree, l, a)
                s, v = int(F.split_dim[tree, j]), float(F.split_val[tree, j])
                # split dimension among the top-t by numpy's two-pass variance (tolerant to near-ties)
                var = Xd[pts].var(0, ddof=1) if var_scope == 0 else gvar
                if var_scope == 0 and len(pts) < 2:
                    var = np.zeros_like(var)
                order = np.lexsort((np.arange(len(var)), -var))
                D = order[:t]
                if check_dims:
                    thr = var[D[-1]]
                    assert var[s] >= thr * (1 - 1e-9)
                    if var[order[t - 1]] > var[order[t]] * (1 + 1e-9) and \
                            all(var[D[i]] > var[D[i + 1]] * (1 + 1e-9) for i in range(t - 1)):
                        assert s == D[oracle.node_draw(seed, tree, j) % t]
                # median split by the key (x_s, rk), h fixed by the perfect shape (R1, R5)
                xs = X[pts, s].astype(np.float32) + np.float32(0.0)
                key_order = np.lexsort((rk[pts], xs))
                lo = (a * n) >> l
                h = ((2 * a + 1) * n >> (l + 1)) - lo
                left_ref = np.sort(pts[key_order[:h]])
                assert v == (xs[key_order[h]] if h < len(pts) else np.inf)
                left = _node_points(F, tree, l + 1, 2 * a)
                assert np.array_equal(np.sort(left), left_ref)
                right = _node_points(F, tree, l + 1, 2 * a + 1)
                assert np.all(X[left, s] <= v) and np.all(X[right, s] >= v)
