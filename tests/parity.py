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
from oracle import screen

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


U32 = 2.0 ** -24  # unit roundoff of float32


def screen_bounds(X, q, c, precision, form):
    """Float64 screened distances sd_c of the candidates c to query q (the oracle's screen, Sec. 3
    "Distance computation": the distance to the rounded points) and, per candidate, a bound eps_c on
    how far the GPU's float32 screened score of c can lie from sd_c.  Both forms rank candidates of
    one query; the norm form drops the query's |q|^2, common to all of them, so only differences
    between candidates matter and eps bounds the score up to that constant.

    form "direct" (streaming and sort kernels): sum_j (q_j - x~_j)^2 with the float32 query; every
    difference is one rounding (q - x~ for bf16, fma(-scale, code, q) for fp8, the product exact),
    every square-and-add one more, then a short sum tree.  All terms are non-negative, so the
    error is relative: at most (chain + tree + 2) u sd_c; (ceil(d/32) + 16) u covers any lane layout
    of the kernels (u = 2^-24).

    form "norm" (leaf-major on the tensor cores): |x~|^2 - 2 x~.q~ with q~ the query's parts.
      bf16: q~ = hi + lo, hi = bf16(q), lo = bf16(q - hi), so |q_j - q~_j| <= 2^-16 |q_j|;
      fp8:  q~ = c (p0 + p1/16 + p2/256) in E4M3 parts, c the smallest power of two with
            max|q| / c <= 448, so |q_j - q~_j| <= 2^-12 |q_j| + 2^-18 c.
    With A = sum_j |x~_j| |q_j|: the query parts cost at most 2 sum_j |x~_j| |q_j - q~_j|; the tensor
    core's float32 accumulation of one K step (16 bf16 or 32 E4M3 values) at most 4 ulps (2^-21
    relative) of a running sum bounded by A, for ceil(d/K) steps plus a few, doubled by the factor
    2 and taken over all parts (x 1.1); |x~|^2 is a float64 sum rounded once (u), and the parts'
    sum and the final fused multiply-add round a few times more."""
    deq = screen.dequantized_rows(X, c, precision)
    q64 = np.asarray(q, dtype=np.float64)
    sd = ((deq - q64) ** 2).sum(axis=1)
    d = X.shape[1]
    if form == "direct":
        eps = (np.ceil(d / 32) + 16) * U32 * sd
    elif form == "norm":
        ax = np.abs(deq)
        A = ax @ np.abs(q64)
        xn = (deq ** 2).sum(axis=1)
        if precision == "bf16":
            qerr, steps = 2.0 ** -16 * np.abs(q64), np.ceil(d / 16)
        elif precision == "fp8":
            mx = np.abs(q64).max()
            c = 2.0 ** np.ceil(np.log2(mx / 448.0)) if mx > 0 else 1.0
            qerr, steps = 2.0 ** -12 * np.abs(q64) + 2.0 ** -18 * c, np.ceil(d / 32)
        else:
            raise ValueError(precision)
        eps = 2 * U32 * xn + 2 * (ax @ qerr) + A * (2.2 * (steps + 4) * 2.0 ** -21 + 6 * U32)
    else:
        raise ValueError(form)
    return sd, eps


def screened_sets(sd, eps, R):
    """Which candidates the GPU's shortlist of R (the R smallest screened scores) may hold and which
    it must hold, when each GPU score lies within [sd - eps, sd + eps].  c may be on the list unless
    R others certainly score below it (sd_j + eps_j < sd_c - eps_c); c must be on it when fewer than
    R others can score at or below it (sd_j - eps_j <= sd_c + eps_c)."""
    lo, hi = sd - eps, sd + eps
    may = np.searchsorted(np.sort(hi), lo, side="left") < R
    must = np.searchsorted(np.sort(lo), hi, side="right") - 1 < R
    return may, must


def gpu_screen_scores(gf, G, Q, offs, ids, precision):
    """The GPU's own float32 screened distances (gf_score_screened, the same arithmetic as the
    streaming and sort kernels) and float32 exact distances of every candidate, [m][width]."""
    import torch
    m = len(offs) - 1
    nc = np.diff(offs).astype(np.int32)
    width = max(1, int(nc.max()))
    cand = np.zeros((m, width), dtype=np.int32)
    for i in range(m):
        cand[i, :nc[i]] = ids[offs[i]:offs[i + 1]]
    Qg, cg, ng = (torch.from_numpy(np.ascontiguousarray(Q)).cuda(), torch.from_numpy(cand).cuda(),
                  torch.from_numpy(nc).cuda())
    gs = gf.gf_score_screened(G, Qg, cg, ng, gf.PRECISIONS[precision]).cpu().numpy()
    ge = gf.gf_score_screened(G, Qg, cg, ng, gf.GF_FP32).cpu().numpy()
    return gs, ge


def assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, precision, R, form="direct", gpu_scores=None,
                          max_frac=0.03):
    """GPU screened search (gi, gd) against the oracle's (oi, od: float64 screen of the rounded
    points, R best, exact rerank, k best) on the candidates offs/ids.

    A row equal to the oracle's must carry its distances (1e-5 relative).  A row that differs is
    held to what any screen within the error bound of screen_bounds can return:
      - exactly min(k, R, candidates) results, distinct, each a candidate the shortlist may hold,
        reported with its exact distance (1e-5 relative), in (distance, id) order;
      - nothing better left out: a candidate the shortlist must hold and that is not reported lies
        no closer than the last reported one (up to 2e-5 relative, the float32 rerank's rounding);
    and such rows must be rare (max_frac).  With gpu_scores (gpu_screen_scores) every row must also
    equal, bit for bit, the exact top-k of the shortlist those scores make: the R smallest by
    (screened score, id), ordered by (float32 exact distance, id)."""
    m, k = oi.shape
    bad = 0
    for i in range(m):
        c = np.asarray(ids[offs[i]:offs[i + 1]], dtype=np.int64)
        nexp = min(k, R, len(c))
        fin = gi[i] >= 0
        assert int(fin.sum()) == nexp and fin[:nexp].all(), f"query {i}: {int(fin.sum())} results, {nexp} expected"
        assert np.all(np.isinf(gd[i][~fin]))
        if gpu_scores is not None:
            gs, ge = gpu_scores[0][i, :len(c)], gpu_scores[1][i, :len(c)]
            sl = np.lexsort((c, gs))[:R]
            top = sl[np.lexsort((c[sl], ge[sl]))[:k]]
            assert np.array_equal(gi[i][:nexp], c[top]), f"query {i}: not the top-k of the GPU's own shortlist"
            assert np.array_equal(gd[i][:nexp], ge[top]), f"query {i}: distances differ from the GPU's own"
        if np.array_equal(gi[i], oi[i]):
            np.testing.assert_allclose(gd[i][fin], od[i][fin], rtol=RTOL)
            continue
        bad += 1
        rep = gi[i][:nexp].astype(np.int64)
        assert len(set(rep.tolist())) == nexp, f"query {i}: repeated id"
        pos = np.searchsorted(c, rep)
        assert np.all(pos < len(c)) and np.array_equal(c[np.minimum(pos, len(c) - 1)], rep), \
            f"query {i}: a reported id is not a candidate"
        sd, eps = screen_bounds(X, Q[i], c, precision, form)
        may, must = screened_sets(sd, eps, R)
        assert may[pos].all(), f"query {i}: ids {rep[~may[pos]]} cannot be on a shortlist of {R}"
        ed = ((X[c].astype(np.float64) - np.asarray(Q[i], dtype=np.float64)) ** 2).sum(axis=1)
        gdr = gd[i][:nexp].astype(np.float64)
        assert np.all(np.abs(gdr - ed[pos]) <= RTOL * ed[pos]), f"query {i}: reported distances are not exact"
        assert np.all((np.diff(gdr) > 0) | ((np.diff(gdr) == 0) & (np.diff(rep) > 0))), \
            f"query {i}: not in (distance, id) order"
        left = must.copy()
        left[pos] = False
        if nexp < k:
            assert not left.any(), f"query {i}: a candidate the shortlist must hold is missing"
        else:
            assert np.all(ed[left] >= gdr[-1] * (1 - 2 * RTOL)), \
                f"query {i}: a closer candidate the shortlist must hold was left out"
    assert bad <= max(1, int(max_frac * m)), f"{bad} of {m} rows differ"
    return bad


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
