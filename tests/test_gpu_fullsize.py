"""Parity at the full workload sizes, in the launch configuration the benchmark times.

The oracle cannot rebuild 10^6-point forests in seconds, so at these sizes the GPU-built forest is
checked on properties that hold at any size and on sampled outputs the oracle computes one by one:
  * every tree's permutation is a permutation of 0..n-1;
  * sampled nodes: split dimension among the float64 top-t of the node's points (the draw picks it
    when there is no variance near-tie), split value = the rank-h key, left child = the h smallest
    keys (Alg. 1 with readings R1-R5);
  * sampled queries: the oracle searches the GPU forest itself; candidate counts must match
    exactly, distances within 1e-5, ids except at near-ties; the bf16 / fp8 screens against the
    float64 screen of the same rounded points within the screen's rounding bound, and (direct
    form) against the top-k of the GPU's own shortlist.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import screen
from parity import assert_screened_close, assert_topk_close, candidate_sets, gpu_screen_scores

pytestmark = pytest.mark.gpu

# (name, n, d, m, T, leaf_size, law, k)
FULL = {
    "gist100k": (100_000, 960, 10_000, 16, 64, "B", 10),
    "gist1m_p64": (1_000_000, 960, 10_000, 32, 64, "B", 10),
    "gist1m_p1024": (1_000_000, 960, 10_000, 32, 1024, "B", 10),
    "highd": (200_000, 10_000, 2_000, 24, 32, "C", 10),
}
_data = {}


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


def data(name):
    n, d, m, T, p, law, k = FULL[name]
    key = (n, d, law)
    if key not in _data:
        _data.clear()
        _data[key] = synth.mixture(n, d, m, law, seed=0, qseed=1)
    return _data[key]


def gpu_forest(gf, name):
    n, d, m, T, p, law, k = FULL[name]
    X, Q = data(name)
    Xg = torch.from_numpy(X).cuda()
    G = gf.gf_build(Xg, T, p, seed=0)
    del Xg
    sd, sv, pm = gf.gf_forest_export(G)
    inf = G.info
    return G, oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm)


def check_sampled_nodes(X, F, t, seed, rng, per_level=3, max_pts=25_000):
    for tree in range(F.T):
        assert np.array_equal(np.sort(F.perm[tree]), np.arange(F.n))
    checked = 0
    for l in range(F.L):
        if (F.n >> l) > max_pts:
            continue
        for _ in range(per_level):
            tree = int(rng.integers(F.T))
            a = int(rng.integers(1 << l))
            j = (1 << l) - 1 + a
            lo, hi = (a * F.n) >> l, ((a + 1) * F.n) >> l
            pts = F.perm[tree, lo:hi]
            var = X[pts].astype(np.float64).var(0, ddof=1)
            order = np.lexsort((np.arange(len(var)), -var))
            s = int(F.split_dim[tree, j])
            assert var[s] >= var[order[t - 1]] * (1 - 1e-9)
            D = order[:t]
            gaps_ok = all(var[order[i]] > var[order[i + 1]] * (1 + 1e-9) for i in range(t))
            if gaps_ok:
                assert s == D[oracle.node_draw(seed, tree, j) % t]
            rk = np.array([oracle.rank(seed, tree, 1, int(i)) for i in pts], dtype=np.uint64)
            xs = X[pts, s] + np.float32(0.0)
            ko = np.lexsort((rk, xs))
            h = (((2 * a + 1) * F.n) >> (l + 1)) - lo
            assert F.split_val[tree, j] == xs[ko[h]]
            left = F.perm[tree, lo:lo + h]
            assert np.array_equal(np.sort(left), np.sort(pts[ko[:h]]))
            checked += 1
    assert checked > 0


def check_sampled_queries(gf, G, F, X, Q, k, idx, precisions=("fp32", "bf16")):
    Qs = Q[idx]
    Qg = torch.from_numpy(Qs).cuda()
    offs, ids = oracle.candidates(F, oracle.descend(F, Qs))
    cs = candidate_sets(offs, ids)
    nc = torch.empty(len(idx), dtype=torch.int32, device="cuda")
    gi, gd = gf.gf_query(G, Qg, k, algo=gf.GF_ALGO_STREAM, ncand_out=nc)
    assert np.array_equal(nc.cpu().numpy(), np.diff(offs))
    oi, od = oracle.topk(X, Qs, offs, ids, k)
    assert_topk_close(X, Qs, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, cs)
    for prec in precisions:
        if prec == "fp32":
            continue
        gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
        R = 32
        gi, gd = gf.gf_query(G, Qg, k, precision=gf.PRECISIONS[prec], rerank_R=R)
        si, sd, _ = screen.screened_search(F, X, Qs, k, R, prec, offs, ids)
        assert_screened_close(X, Qs, gi.cpu().numpy(), gd.cpu().numpy(), si, sd, offs, ids, prec, R, "direct",
                              gpu_scores=gpu_screen_scores(gf, G, Qs, offs, ids, prec))


@pytest.mark.parametrize("name", ["gist100k", "gist1m_p64", "gist1m_p1024"])
def test_full_size_gist_like(gf, name):
    n, d, m, T, p, law, k = FULL[name]
    X, Q = data(name)
    G, F = gpu_forest(gf, name)
    rng = np.random.default_rng(0)
    check_sampled_nodes(X, F, 5, 0, rng)
    idx = np.sort(rng.choice(m, 200, replace=False))
    check_sampled_queries(gf, G, F, X, Q, k, idx)
    G.free()


def test_full_size_gist100k_forest_equals_oracle(gf):
    # 10^5 points are cheap enough for the oracle to rebuild the whole forest
    X, Q = data("gist100k")
    G, F = gpu_forest(gf, "gist100k")
    Fo = oracle.build_forest(X, 16, 64, seed=0)
    assert np.array_equal(F.split_dim, Fo.split_dim)
    assert np.array_equal(F.split_val, Fo.split_val)
    assert np.array_equal(F.perm, Fo.perm)
    G.free()


def test_full_size_high_d(gf):
    n, d, m, T, p, law, k = FULL["highd"]
    X, Q = data("highd")
    G, F = gpu_forest(gf, "highd")
    rng = np.random.default_rng(1)
    check_sampled_nodes(X, F, 5, 0, rng, per_level=2, max_pts=3000)
    idx = np.sort(rng.choice(m, 60, replace=False))
    check_sampled_queries(gf, G, F, X, Q, k, idx, precisions=("fp32", "bf16", "fp8"))
    G.free()


def test_full_size_leaf_major_batch(gf):
    # the headline launch: the whole 10^4-query batch through the leaf-major path (bf16 screen with
    # R = 16, and float32), sampled rows checked against the oracle on the same GPU-built forest
    n, d, m, T, p, law, k = FULL["gist1m_p1024"]
    X, Q = data("gist1m_p1024")
    G, F = gpu_forest(gf, "gist1m_p1024")
    gf.gf_forest_add_screen(G, gf.GF_BF16_RERANK)
    Qg = torch.from_numpy(Q).cuda()
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(m, 200, replace=False))
    Qs = Q[idx]
    offs, ids = oracle.candidates(F, oracle.descend(F, Qs))
    cs = candidate_sets(offs, ids)
    # float32
    gi, gd = gf.gf_query(G, Qg, k, algo=gf.GF_ALGO_LEAF)
    oi, od = oracle.topk(X, Qs, offs, ids, k)
    assert_topk_close(X, Qs, gi.cpu().numpy()[idx], gd.cpu().numpy()[idx], oi, od, cs)
    # bf16 screen, R = 16
    gi, gd = gf.gf_query(G, Qg, k, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_LEAF)
    si, sd, _ = screen.screened_search(F, X, Qs, k, 16, "bf16", offs, ids)
    assert_screened_close(X, Qs, gi.cpu().numpy()[idx], gd.cpu().numpy()[idx], si, sd, offs, ids, "bf16", 16, "norm")
    assert gf.gf_kernel_status() == 0
    G.free()
