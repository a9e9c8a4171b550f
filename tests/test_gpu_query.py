"""GPU query path against the CPU oracle on the same forest (Alg. 2 with one leaf per tree).

The forest is built by the oracle and imported into the GPU library, so both sides search the
identical structure.  Leaves and candidate sets must match bit for bit; float32 distances within
1e-5 relative of float64; k-NN ids exactly except at near-ties.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import screen
from parity import RTOL, assert_screened_close, assert_topk_close, candidate_sets, gpu_screen_scores

pytestmark = pytest.mark.gpu

# (name, n, d, m, T, leaf_size, law): the tiny workload, ragged sizes (d not a multiple of 4/8/16,
# m and n odd), more trees than a warp, a row longer than the register-resident query, the
# 960-d GIST-like law, and a noisy Klein bottle in R^100 (low intrinsic dimension).
CASES = [
    ("tiny", 10_000, 128, 100, 8, 32, "A"),
    ("ragged", 3001, 37, 57, 5, 9, "B"),
    ("manytrees", 5000, 64, 40, 40, 16, "A"),
    ("long_rows", 3000, 2000, 30, 6, 40, "C"),
    ("gist_like", 20_000, 960, 200, 16, 64, "B"),
    ("klein", 10_000, 100, 100, 8, 32, "klein"),   # the paper's Klein-bottle set (Sec. 4)
]


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


_cache = {}


def case(name):
    if name not in _cache:
        spec = next(c for c in CASES if c[0] == name)
        _, n, d, m, T, p, law = spec
        if law in ("klein", "sphere"):
            X, Q = synth.manifold(n, d, m, law, seed=0, qseed=1)
        else:
            X, Q = synth.mixture(n, d, m, law, seed=0, qseed=1)
        F = oracle.build_forest(X, T, p, t=min(5, d), seed=7)
        _cache[name] = (X, Q, F)
    return _cache[name]


def gpu_forest(gf, X, F):
    Xg = torch.from_numpy(X).cuda()
    return gf.gf_forest_import(Xg, F.T, F.leaf_size, F.split_dim, F.split_val, F.perm), Xg


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_descend_bit_exact(gf, name):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    leaf = gf.gf_descend(G, torch.from_numpy(Q).cuda()).cpu().numpy()
    assert np.array_equal(leaf, oracle.descend(F, Q))


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_candidates_bit_exact(gf, name):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    leaf = oracle.descend(F, Q)
    cand, nc = gf.gf_candidates(G, torch.from_numpy(leaf).cuda())
    cand, nc = cand.cpu().numpy(), nc.cpu().numpy()
    offs, ids = oracle.candidates(F, leaf)
    assert np.array_equal(nc, np.diff(offs))
    for i in range(Q.shape[0]):
        assert np.array_equal(cand[i, :nc[i]], ids[offs[i]:offs[i + 1]])


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_score_topk(gf, name):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    m = Q.shape[0]
    width = int(np.diff(offs).max())
    cand = np.zeros((m, width), dtype=np.int32)
    for i in range(m):
        cand[i, :offs[i + 1] - offs[i]] = ids[offs[i]:offs[i + 1]]
    k = 10
    gi, gd = gf.gf_score_topk(G, torch.from_numpy(Q).cuda(), torch.from_numpy(cand).cuda(),
                              torch.from_numpy(np.diff(offs).astype(np.int32)).cuda(), k)
    oi, od = oracle.topk(X, Q, offs, ids, k)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, candidate_sets(offs, ids))


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("k", [1, 10])
def test_query_fused_fp32(gf, name, k):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k)
    torch.cuda.synchronize()
    oi, od = oracle.search(F, X, Q, k)
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, candidate_sets(offs, ids))


@pytest.mark.parametrize("warps,cps", [(1, 1), (4, 2), (8, 3), (16, 1)])
def test_query_kernel_shapes_agree(gf, warps, cps):
    X, Q, F = case("gist_like")
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    ref_i, ref_d = gf.gf_query(G, Qg, 10)
    gi, gd = gf.gf_query(G, Qg, 10, warps_per_cta=warps, ctas_per_sm=cps)
    # the distance of a row does not depend on the CTA shape: bit-identical results
    assert torch.equal(gi, ref_i) and torch.equal(gd, ref_d)


def test_query_pads_short_candidate_lists(gf):
    X, Q = synth.mixture(64, 8, 5, "A", seed=3)
    F = oracle.build_forest(X, 1, 4, seed=0)
    G, _ = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 6)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = oracle.search(F, X, Q, 6)
    assert np.all(gi[:, 4:] == -1) and np.all(np.isinf(gd[:, 4:]))
    assert_topk_close(X, Q, gi, gd, oi, od)


def test_query_single_leaf_is_exact_knn(gf):
    # leaf_size >= n: one leaf holds every point, so the search is brute force
    X, Q = synth.mixture(500, 33, 25, "B", seed=4)
    F = oracle.build_forest(X, 2, 500, seed=0)
    G, _ = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 7)
    ei, ed = oracle.bruteforce(X, Q, 7)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), ei, ed)


def test_query_edge_sizes(gf):
    X, Q, F = case("ragged")
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    e = gf.gf_query(G, Qg[:0], 3)
    assert e[0].shape == (0, 3)
    gi, gd = gf.gf_query(G, Qg[:1], 3)
    oi, od = oracle.search(F, X, Q[:1], 3)
    assert_topk_close(X, Q[:1], gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    with pytest.raises(gf.GFError):
        gf.gf_query(G, Qg, 0)


def test_query_on_side_stream(gf):
    X, Q, F = case("tiny")
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gi, gd = gf.gf_query(G, Qg, 5, stream=s)
    s.synchronize()
    oi, od = oracle.search(F, X, Q, 5)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


# ---------------------------------------------------------------- screened precisions

@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("name", ["tiny", "ragged", "long_rows", "gist_like"])
def test_query_screened(gf, prec, name):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
    R, k = 32, 10
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k, precision=gf.PRECISIONS[prec], rerank_R=R)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    oi, od, _ = screen.screened_search(F, X, Q, k, R, prec, offs, ids)
    assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, prec, R, "direct",
                          gpu_scores=gpu_screen_scores(gf, G, Q, offs, ids, prec))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_screened_full_shortlist_equals_fp32(gf, prec):
    # R >= every candidate count: the rerank sees every candidate, so the answer is the float32 one
    X, Q, F = case("tiny")
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
    Qg = torch.from_numpy(Q).cuda()
    fi, fd = gf.gf_query(G, Qg, 10)
    si, sd = gf.gf_query(G, Qg, 10, precision=gf.PRECISIONS[prec], rerank_R=G.info.cand_cap)
    assert torch.equal(fi, si) and torch.equal(fd, sd)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("name", ["ragged", "long_rows", "gist_like"])
def test_screened_distances_elementwise(gf, prec, name):
    # every candidate's screened distance against the float64 value of the same rounded points
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    if prec != "fp32":
        gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    m = Q.shape[0]
    width = int(np.diff(offs).max())
    cand = np.zeros((m, width), dtype=np.int32)
    for i in range(m):
        cand[i, :offs[i + 1] - offs[i]] = ids[offs[i]:offs[i + 1]]
    nc = np.diff(offs).astype(np.int32)
    dist = gf.gf_score_screened(G, torch.from_numpy(Q).cuda(), torch.from_numpy(cand).cuda(),
                                torch.from_numpy(nc).cuda(), gf.PRECISIONS[prec]).cpu().numpy()
    for i in range(m):
        c = cand[i, :nc[i]]
        ref = ((screen.dequantized_rows(X, c, prec) - Q[i].astype(np.float64)) ** 2).sum(axis=1)
        np.testing.assert_allclose(dist[i, :nc[i]], ref, rtol=RTOL, atol=RTOL * ref.max())


# ---------------------------------------------------------------- streaming kernel (bitmap dedupe)

@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("k", [1, 10])
def test_stream_matches_oracle_and_counts(gf, name, k):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    nc = torch.full((Q.shape[0],), -1, dtype=torch.int32, device="cuda")
    gi, gd = gf.gf_query(G, Qg, k, algo=gf.GF_ALGO_STREAM, ncand_out=nc)
    oi, od, onc = oracle.search(F, X, Q, k, return_ncand=True)
    assert np.array_equal(nc.cpu().numpy(), onc)        # the bitmap admits each candidate once
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, candidate_sets(offs, ids))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("name", ["tiny", "ragged", "gist_like"])
def test_stream_equals_sort_kernel(gf, prec, name):
    # same row arithmetic in both kernels: bit-identical ids and distances
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    p = gf.PRECISIONS[prec]
    if p:
        gf.gf_forest_add_screen(G, p)
    Qg = torch.from_numpy(Q).cuda()
    a = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_SORT)
    for g in (2, 4):
        b = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_STREAM, rows_in_flight=g)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_stream_caller_workspace_is_left_zero(gf):
    X, Q, F = case("tiny")
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    nbytes = gf.gf_query_workspace_size(G, Q.shape[0], ctas_per_sm=2)
    ws = torch.zeros(nbytes // 4, dtype=torch.int32, device="cuda")
    ref = gf.gf_query(G, Qg, 5, algo=gf.GF_ALGO_STREAM, ctas_per_sm=2)
    for _ in range(2):
        got = gf.gf_query(G, Qg, 5, algo=gf.GF_ALGO_STREAM, ctas_per_sm=2, workspace=ws)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
        assert int(torch.count_nonzero(ws)) == 0
    with pytest.raises(gf.GFError):
        gf.gf_query(G, Qg, 5, algo=gf.GF_ALGO_STREAM, ctas_per_sm=2, workspace=ws[:10])


_big = {}


def big_case():
    # leaves of 782 points in 16 trees: up to 12.5k candidates per query, beyond the sort kernel
    if not _big:
        X, Q = synth.mixture(50_000, 64, 60, "B", seed=5, qseed=6)
        F = oracle.build_forest(X, 16, 1000, seed=2)
        _big["c"] = (X, Q, F)
    return _big["c"]


@pytest.mark.parametrize("k", [1, 10, 300])
def test_stream_large_candidate_sets(gf, k):
    # k = 300 keeps a large best set, so the shared buffer is cut back many times per query
    X, Q, F = big_case()
    G, _ = gpu_forest(gf, X, F)
    assert G.info.cand_cap > 4096
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k)
    oi, od = oracle.search(F, X, Q, k)
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, candidate_sets(offs, ids))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("R", [16, 256])
def test_stream_large_screened(gf, prec, R):
    X, Q, F = big_case()
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, precision=gf.PRECISIONS[prec], rerank_R=R)
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    oi, od, _ = screen.screened_search(F, X, Q, 10, R, prec, offs, ids)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, offs, ids, prec, R, "direct",
                          gpu_scores=gpu_screen_scores(gf, G, Q, offs, ids, prec))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_locality_order_changes_no_result(gf, prec):
    # CTAs taking the queries sorted by their tree-0 leaf: every answer (and candidate count) stays
    # at its query's row and is bit-identical to the batch taken as given
    X, Q, F = case("gist_like")
    G, _ = gpu_forest(gf, X, F)
    p = gf.PRECISIONS[prec]
    if p:
        gf.gf_forest_add_screen(G, p)
    Qg = torch.from_numpy(Q).cuda()
    res = {}
    for order in (gf.GF_ORDER_GIVEN, gf.GF_ORDER_LOCALITY, gf.GF_ORDER_AUTO):
        nc = torch.full((Q.shape[0],), -1, dtype=torch.int32, device="cuda")
        i, d = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_STREAM, ctas_per_sm=1,
                           order=order, ncand_out=nc)
        res[order] = (i, d, nc)
    a = res[gf.GF_ORDER_GIVEN]
    for order in (gf.GF_ORDER_LOCALITY, gf.GF_ORDER_AUTO):
        b = res[order]
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


# ---------------------------------------------------------------- Alg. 2 priority search

@pytest.mark.parametrize("name,c", [("tiny", 24), ("ragged", 23), ("manytrees", 100), ("gist_like", 64),
                                    ("klein", 32), ("gist_like", 512), ("manytrees", 300)])
def test_priority_leaf_order_bit_exact(gf, name, c):
    # (budgets of hundreds of leaves move the queue's small array into its large one many times)
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    leaves, nl = gf.gf_prio_leaves(G, torch.from_numpy(Q).cuda(), c)
    leaves = leaves.cpu().numpy().view(np.uint32).astype(np.int64)
    _, _, _, onl, oseq = oracle.search_priority(F, X, Q, 1, c, return_leaves=True)
    assert np.array_equal(nl.cpu().numpy(), onl)
    for i in range(Q.shape[0]):
        assert np.array_equal(leaves[i, :onl[i]], oseq[i, :onl[i]])


@pytest.mark.parametrize("name,c,eps", [("tiny", 24, 0.0), ("ragged", 23, 0.0), ("manytrees", 100, 0.5),
                                        ("gist_like", 64, 0.0), ("klein", 32, 0.1)])
@pytest.mark.parametrize("k", [1, 10])
def test_priority_search_matches_oracle(gf, name, c, eps, k):
    X, Q, F = case(name)
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    nc = torch.full((Q.shape[0],), -1, dtype=torch.int32, device="cuda")
    gi, gd = gf.gf_query(G, Qg, k, checks=c, eps=eps, ncand_out=nc)
    oi, od, onc, onl = oracle.search_priority(F, X, Q, k, c, eps)
    assert np.array_equal(nc.cpu().numpy(), onc)   # the same leaves, each id admitted once
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


def test_priority_with_c_equal_T_is_the_one_leaf_search(gf):
    X, Q, F = case("gist_like")
    G, _ = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    a = gf.gf_query(G, Qg, 10, algo=gf.GF_ALGO_STREAM)
    b = gf.gf_query(G, Qg, 10, checks=F.T)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_priority_with_screening(gf, prec):
    X, Q, F = case("gist_like")
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_add_screen(G, gf.PRECISIONS[prec])
    Qg = torch.from_numpy(Q).cuda()
    full = gf.gf_query(G, Qg, 10, checks=48)
    # a shortlist of every candidate gives the float32 answer exactly
    scr = gf.gf_query(G, Qg, 10, checks=48, precision=gf.PRECISIONS[prec], rerank_R=2048)
    assert torch.equal(full[0], scr[0]) and torch.equal(full[1], scr[1])


def test_exact_neighbours_by_one_leaf_forest(gf):
    # leaf_size >= n: the library's own kernel scans every point, which is exact k-NN
    from paper_1603_09596_gb300 import autotune
    X, Q, F = case("ragged")
    ids, d = autotune.exact_neighbours(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), 3)
    ei, ed = oracle.bruteforce(X, Q, 3)
    assert_topk_close(X, Q, ids.cpu().numpy(), d.cpu().numpy(), ei, ed)


def test_configure_meets_recall_target(gf):
    from paper_1603_09596_gb300 import autotune
    X, Q = synth.manifold(20_000, 100, 200, "klein", seed=5, qseed=6)
    res = autotune.configure(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), target_recall=0.9,
                             grid=[(8, 32, 0), (16, 64, 0), (16, 64, 64), (32, 256, 0)])
    assert res["met_target"] and res["choice"]["recall_at_1"] >= 0.9
    assert len(res["tried"]) == 4


# ---------------------------------------------------------------- Householder reflections (Sec. 2.2)

def _units(T, d, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((T, d))
    return (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)


_refl = {}


def reflected_case(name):
    if name not in _refl:
        X, Q, F0 = case(name)
        U = _units(F0.T, F0.d, 77)
        _refl[name] = (X, Q, oracle.build_forest(X, F0.T, F0.leaf_size, t=min(5, F0.d), seed=7, U=U), U)
    return _refl[name]


@pytest.mark.parametrize("name", ["tiny", "ragged", "gist_like"])
def test_reflected_descent_and_candidates_bit_exact(gf, name):
    X, Q, F, U = reflected_case(name)
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_set_reflections(G, U)
    Qg = torch.from_numpy(Q).cuda()
    leaf = gf.gf_descend(G, Qg).cpu().numpy()
    assert np.array_equal(leaf, oracle.descend(F, Q))
    nc = torch.empty(Q.shape[0], dtype=torch.int32, device="cuda")
    gf.gf_query(G, Qg, 1, algo=gf.GF_ALGO_STREAM, ncand_out=nc)
    offs, _ = oracle.candidates(F, leaf)
    assert np.array_equal(nc.cpu().numpy(), np.diff(offs))


@pytest.mark.parametrize("name", ["tiny", "ragged", "gist_like"])
@pytest.mark.parametrize("algo", ["sort", "stream"])
def test_reflected_query_matches_oracle(gf, name, algo):
    X, Q, F, U = reflected_case(name)
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_set_reflections(G, U)
    a = gf.GF_ALGO_SORT if algo == "sort" else gf.GF_ALGO_STREAM
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, algo=a)
    oi, od = oracle.search(F, X, Q, 10)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


@pytest.mark.parametrize("name,c", [("tiny", 24), ("gist_like", 48)])
def test_reflected_priority_search_matches_oracle(gf, name, c):
    X, Q, F, U = reflected_case(name)
    G, _ = gpu_forest(gf, X, F)
    gf.gf_forest_set_reflections(G, U)
    Qg = torch.from_numpy(Q).cuda()
    leaves, nl = gf.gf_prio_leaves(G, Qg, c)
    oi, od, onc, onl, oseq = oracle.search_priority(F, X, Q, 10, c, return_leaves=True)
    leaves = leaves.cpu().numpy().view(np.uint32).astype(np.int64)
    for i in range(Q.shape[0]):
        assert np.array_equal(leaves[i, :onl[i]], oseq[i, :onl[i]])
    gi, gd = gf.gf_query(G, Qg, 10, checks=c)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)


@pytest.mark.parametrize("prec,algo", [("bf16", "stream"), ("bf16", "sort"), ("bf16", "leaf"),
                                       ("fp8", "stream"), ("fp8", "sort")])
def test_screen_reorders_the_hand_worked_pair_as_the_oracle(gf, prec, algo):
    """The pair of test_screen_pins.SCREEN_FLIPS: a shortlist of one keeps the point the screen ranks
    first (reported with its exact distance), a shortlist of two the exact nearest, on every path."""
    from test_screen_pins import SCREEN_FLIPS
    X, screen_first, exact_first = SCREEN_FLIPS[prec]
    p = {"bf16": gf.GF_BF16_RERANK, "fp8": gf.GF_FP8_RERANK}[prec]
    a = {"stream": gf.GF_ALGO_STREAM, "sort": gf.GF_ALGO_SORT, "leaf": gf.GF_ALGO_LEAF}[algo]
    G = gf.gf_build(torch.from_numpy(X).cuda(), 1, 2, t=2, seed=0)
    assert G.info.L == 0
    gf.gf_forest_add_screen(G, p)
    Q = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    exact = (X.astype(np.float64) ** 2).sum(axis=1)
    for R, want in ((1, screen_first), (2, exact_first)):
        ids, d = gf.gf_query(G, Q, 1, precision=p, rerank_R=R, algo=a)
        assert int(ids[0, 0]) == want, (R, ids)
        assert abs(float(d[0, 0]) - exact[want]) <= RTOL * exact[want]
