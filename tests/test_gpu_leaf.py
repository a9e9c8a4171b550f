"""The leaf-major batched path (GF_ALGO_LEAF) against the CPU oracle's screened search.

The forest is built by the oracle and imported, so both sides search the same trees.  The oracle's
bf16 (fp8) screen ranks the candidate union of every query by the float64 distance to the
bf16-rounded (E4M3-coded, row-scaled) points, keeps the R best and reranks them exactly; the GPU
screen ranks the same union by |x~|^2 - 2 x~.q~ on the tensor cores, q~ the query's bf16 or E4M3
parts, and is held to the rounding bound of that form (parity.screen_bounds).  As for the other
screened kernels: every reported id must be a candidate reported with its float32 distance (1e-5
relative), and a row may differ from the oracle only where the two screens order the shortlist
boundary differently, which must be rare.  Where
the shortlist holds every candidate the screen decides nothing, and the answer must equal the
float32 search bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import screen
from parity import assert_screened_close, assert_topk_close

pytestmark = pytest.mark.gpu

# (name, n, d, m, T, leaf_size, law)
CASES = [
    ("tiny", 10_000, 128, 100, 8, 32, "A"),
    ("ragged", 3001, 37, 57, 5, 9, "B"),          # d not a multiple of 8 or 64; odd n and m
    ("manytrees", 5000, 64, 40, 40, 16, "A"),     # T above a warp
    ("long_rows", 3000, 2000, 30, 6, 40, "C"),    # 32 k-steps per row tile
    ("gist_like", 20_000, 960, 200, 16, 64, "B"),
    ("shared", 20_000, 96, 3000, 8, 300, "B"),    # ~23 queries per leaf, leaves of 156: two row tiles
    ("crowded", 8000, 64, 4000, 4, 1000, "A"),    # 500 queries per leaf: many chunks; 8 row tiles each
    ("klein", 10_000, 100, 100, 8, 32, "klein"),
]


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


_cache = {}


def case(name):
    if name not in _cache:
        _, n, d, m, T, p, law = next(c for c in CASES if c[0] == name)
        if law == "klein":
            X, Q = synth.manifold(n, d, m, law, seed=0, qseed=1)
        else:
            X, Q = synth.mixture(n, d, m, law, seed=0, qseed=1)
        F = oracle.build_forest(X, T, p, t=min(5, d), seed=7)
        _cache[name] = (X, Q, F)
    return _cache[name]


def gpu_forest(gf, X, F):
    G = gf.gf_forest_import(torch.from_numpy(X).cuda(), F.T, F.leaf_size, F.split_dim, F.split_val, F.perm)
    gf.gf_forest_add_screen(G, gf.GF_BF16_RERANK)
    gf.gf_forest_add_screen(G, gf.GF_FP8_RERANK)
    return G


def oracle_screen(F, X, Q, k, R, prec="bf16"):
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    oi, od, _ = screen.screened_search(F, X, Q, k, R, prec, offs, ids)
    return oi, od, (offs, ids)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("R", [16, 32])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_matches_oracle(gf, name, R, prec):
    X, Q, F = case(name)
    G = gpu_forest(gf, X, F)
    k = 10
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k, precision=gf.PRECISIONS[prec], rerank_R=R,
                         algo=gf.GF_ALGO_LEAF)
    oi, od, cands = oracle_screen(F, X, Q, k, R, prec)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, prec, R, "norm")
    assert gf.gf_kernel_status() == 0


@pytest.mark.parametrize("name", ["ragged", "long_rows", "shared", "crowded"])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_one_cta_shape_matches_oracle(gf, name, prec):
    # the kernel's other shape (one CTA per SM, a deeper ring of k-slices): the oracle's answer
    # within the screen's bound, and bit for bit the default shape's answer (the shortlist of every
    # (query, leaf) is the same set whatever order the chunks ran in)
    X, Q, F = case(name)
    G = gpu_forest(gf, X, F)
    k, R = 10, 32
    Qg = torch.from_numpy(Q).cuda()
    p = gf.PRECISIONS[prec]
    gi, gd = gf.gf_query(G, Qg, k, precision=p, rerank_R=R, algo=gf.GF_ALGO_LEAF, ctas_per_sm=1)
    di, dd = gf.gf_query(G, Qg, k, precision=p, rerank_R=R, algo=gf.GF_ALGO_LEAF)
    oi, od, cands = oracle_screen(F, X, Q, k, R, prec)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, prec, R, "norm")
    assert torch.equal(gi, di) and torch.equal(gd, dd)
    assert gf.gf_kernel_status() == 0


@pytest.mark.parametrize("m", [1001, 3000])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_paired_chunks_at_the_limit(gf, m, prec):
    # leaves of exactly 64 rows (4096 points, 2^6 leaves): two chunks share every row tile; 1001
    # queries give buckets of one or two chunks (a wave may end on an unpaired chunk), 3000 give
    # three or more (two chunks of one leaf share a tile); both shapes, against the oracle
    X, Q = synth.mixture(4096, 96, m, "B", seed=5, qseed=6)
    F = oracle.build_forest(X, 5, 64, t=5, seed=3)
    assert F.L == 6 and (F.n >> F.L) == 64
    G = gpu_forest(gf, X, F)
    k, R = 10, 16
    Qg = torch.from_numpy(Q).cuda()
    p = gf.PRECISIONS[prec]
    oi, od, cands = oracle_screen(F, X, Q, k, R, prec)
    res = []
    for cps in (0, 1):
        gi, gd = gf.gf_query(G, Qg, k, precision=p, rerank_R=R, algo=gf.GF_ALGO_LEAF, ctas_per_sm=cps)
        assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, prec, R, "norm")
        res.append((gi, gd))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert gf.gf_kernel_status() == 0


@pytest.mark.parametrize("k,R", [(1, 1), (1, 16), (5, 16), (7, 7)])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_small_k(gf, k, R, prec):
    # shortlists shorter than a power of two and of length one
    X, Q, F = case("shared")
    G = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k, precision=gf.PRECISIONS[prec], rerank_R=R,
                         algo=gf.GF_ALGO_LEAF)
    oi, od, cands = oracle_screen(F, X, Q, k, R, prec)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, prec, R, "norm")


@pytest.mark.parametrize("m", [1, 33])
def test_leaf_tiny_batches(gf, m):
    # a batch of one query, and one that does not fill a chunk
    X, Q, F = case("tiny")
    G = gpu_forest(gf, X, F)
    Qs = np.ascontiguousarray(Q[:m])
    for prec in ("bf16", "fp8"):
        gi, gd = gf.gf_query(G, torch.from_numpy(Qs).cuda(), 10, precision=gf.PRECISIONS[prec], rerank_R=16,
                             algo=gf.GF_ALGO_LEAF)
        oi, od, cands = oracle_screen(F, X, Qs, 10, 16, prec)
        assert_screened_close(X, Qs, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, prec, 16, "norm")
    fi, fd = gf.gf_query(G, torch.from_numpy(Qs).cuda(), 10, algo=gf.GF_ALGO_LEAF)
    oi, od = oracle.search(F, X, Qs, 10)
    assert_topk_close(X, Qs, fi.cpu().numpy(), fd.cpu().numpy(), oi, od)


def test_leaf_full_shortlist_equals_fp32(gf):
    # at most 32 candidates per query and R = 32: every candidate is reranked, so the answer is
    # the float32 search's, bit for bit
    X, Q = synth.mixture(1000, 40, 300, "B", seed=3, qseed=4)
    F = oracle.build_forest(X, 4, 8, t=5, seed=7)
    G = gpu_forest(gf, X, F)
    assert G.info.cand_cap <= 32
    Qg = torch.from_numpy(Q).cuda()
    fi, fd = gf.gf_query(G, Qg, 10, algo=gf.GF_ALGO_STREAM)
    for p in (gf.GF_BF16_RERANK, gf.GF_FP8_RERANK):
        li, ld = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_LEAF)
        assert torch.equal(fi, li) and torch.equal(fd, ld)


def test_leaf_order_changes_no_result(gf):
    X, Q, F = case("shared")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    for p in (gf.GF_BF16_RERANK, gf.GF_FP8_RERANK):
        a = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_LEAF, order=gf.GF_ORDER_GIVEN)
        b = gf.gf_query(G, Qg, 10, precision=p, rerank_R=32, algo=gf.GF_ALGO_LEAF, order=gf.GF_ORDER_LOCALITY)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_leaf_caller_workspace_is_left_zero(gf):
    X, Q, F = case("crowded")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    nb = gf.gf_query_workspace_size(G, Q.shape[0], precision=gf.GF_BF16_RERANK, rerank_R=16,
                                    algo=gf.GF_ALGO_LEAF)
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    a = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_LEAF, workspace=ws)
    b = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_LEAF)
    torch.cuda.synchronize()
    assert int(ws.count_nonzero()) == 0
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # the same workspace then serves the streaming kernel, which needs it zero
    ns = gf.gf_query_workspace_size(G, Q.shape[0], precision=gf.GF_BF16_RERANK, rerank_R=16)
    ws2 = torch.zeros(max(nb, ns), dtype=torch.uint8, device="cuda")
    gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_LEAF, workspace=ws2)
    s = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_STREAM, workspace=ws2)
    t = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=16, algo=gf.GF_ALGO_STREAM)
    assert torch.equal(s[0], t[0]) and torch.equal(s[1], t[1])


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_leaf_in_a_cuda_graph(gf, prec):
    # the benchmark's launch: captured once with a caller workspace (nothing allocates inside the
    # capture), replayed; the replays equal a direct call
    X, Q, F = case("shared")
    G = gpu_forest(gf, X, F)
    p = gf.PRECISIONS[prec]
    Qg = torch.from_numpy(Q).cuda()
    m, k = Q.shape[0], 10
    ws = torch.zeros(gf.gf_query_workspace_size(G, m, precision=p, rerank_R=16, algo=gf.GF_ALGO_LEAF),
                     dtype=torch.uint8, device="cuda")
    ids = torch.empty((m, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((m, k), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    kw = dict(precision=p, rerank_R=16, algo=gf.GF_ALGO_LEAF, workspace=ws, stream=s, out=(ids, dd))
    with torch.cuda.stream(s):
        gf.gf_query(G, Qg, k, **kw)  # warm-up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        gf.gf_query(G, Qg, k, **kw)
    ref = gf.gf_query(G, Qg, k, precision=p, rerank_R=16, algo=gf.GF_ALGO_LEAF)
    torch.cuda.synchronize()
    for _ in range(2):
        ids.fill_(-7)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref[0]) and torch.equal(dd, ref[1])
    assert int(ws.count_nonzero()) == 0


def test_leaf_agrees_with_streaming_screen(gf):
    # two float32 screens of the same candidates: they may order the shortlist boundary
    # differently, so a few rows can differ; every answer is within the other's tolerance
    X, Q, F = case("gist_like")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    a = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=32, algo=gf.GF_ALGO_LEAF)
    b = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=32, algo=gf.GF_ALGO_STREAM)
    same = (a[0] == b[0]).all(dim=1).float().mean().item()
    assert same >= 0.97


def test_leaf_reflected_forest(gf):
    X, Q, F0 = case("tiny")
    rng = np.random.default_rng(77)
    U = rng.standard_normal((F0.T, F0.d))
    U = (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)
    F = oracle.build_forest(X, F0.T, F0.leaf_size, t=5, seed=7, U=U)
    G = gpu_forest(gf, X, F)
    gf.gf_forest_set_reflections(G, U)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, precision=gf.GF_BF16_RERANK, rerank_R=32,
                         algo=gf.GF_ALGO_LEAF)
    oi, od, cands = oracle_screen(F, X, Q, 10, 32)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, "bf16", 32, "norm")


@pytest.mark.parametrize("c", [0, 24])
def test_leaf_reflected_fp32_one_leaf_and_priority(gf, c):
    # a reflected forest (Sec. 2.2) through the float32 leaf-major path: one leaf per tree (c = 0)
    # and the priority search, against the oracle's reflected search
    X, Q, F0 = case("tiny")
    rng = np.random.default_rng(78)
    U = rng.standard_normal((F0.T, F0.d))
    U = (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)
    F = oracle.build_forest(X, F0.T, F0.leaf_size, t=5, seed=9, U=U)
    G = gpu_forest(gf, X, F)
    gf.gf_forest_set_reflections(G, U)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, checks=c, algo=gf.GF_ALGO_LEAF)
    if c:
        oi, od, _, _ = oracle.search_priority(F, X, Q, 10, c)
    else:
        oi, od = oracle.search(F, X, Q, 10)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    assert gf.gf_kernel_status() == 0


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("k", [1, 10])
def test_leaf_fp32_matches_oracle(gf, name, k):
    # the plain float32 search through the leaf-major path: exact distances, ids up to near-ties
    X, Q, F = case(name)
    G = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), k, algo=gf.GF_ALGO_LEAF)
    oi, od = oracle.search(F, X, Q, k)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    assert gf.gf_kernel_status() == 0


def test_leaf_fp32_agrees_with_streaming(gf):
    # the same float32 search by two kernels: distances within 1e-5 relative, ids equal up to ties
    X, Q, F = case("shared")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    a = gf.gf_query(G, Qg, 10, algo=gf.GF_ALGO_LEAF)
    b = gf.gf_query(G, Qg, 10, algo=gf.GF_ALGO_STREAM)
    assert_topk_close(X, Q, a[0].cpu().numpy(), a[1].cpu().numpy(), b[0].cpu().numpy(),
                      b[1].cpu().numpy().astype(np.float64))


def priority_candidates(F, seq, nl):
    """Sorted distinct point ids of the leaves each query checked (the oracle's leaf sequence)."""
    offs, ids = [0], []
    for i in range(seq.shape[0]):
        pts = set()
        for code in seq[i, :nl[i]]:
            t, b = int(code) >> F.L, int(code) & ((1 << F.L) - 1)
            lo, hi = (b * F.n) >> F.L, ((b + 1) * F.n) >> F.L
            pts.update(F.perm[t, lo:hi].tolist())
        ids.extend(sorted(pts))
        offs.append(len(ids))
    return np.asarray(offs, dtype=np.int64), np.asarray(ids, dtype=np.int64)


# Alg. 2 with the shared priority queue through the leaf-major path: each query's list of leaves
# from the priority kernel, the (query, slot) pairs grouped by leaf
PRIO_CASES = [("tiny", 24), ("shared", 20), ("gist_like", 48), ("crowded", 9)]


@pytest.mark.parametrize("name,c", PRIO_CASES)
def test_leaf_priority_fp32_matches_oracle(gf, name, c):
    X, Q, F = case(name)
    G = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, checks=c, algo=gf.GF_ALGO_LEAF)
    oi, od, _, _ = oracle.search_priority(F, X, Q, 10, c)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    assert gf.gf_kernel_status() == 0


@pytest.mark.parametrize("name,c", PRIO_CASES)
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_priority_screened_matches_oracle(gf, name, c, prec):
    X, Q, F = case(name)
    G = gpu_forest(gf, X, F)
    R = 16
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 10, precision=gf.PRECISIONS[prec], rerank_R=R,
                         checks=c, algo=gf.GF_ALGO_LEAF)
    _, _, _, nl, seq = oracle.search_priority(F, X, Q, 10, c, return_leaves=True)
    offs, ids = priority_candidates(F, seq, nl)
    oi, od, _ = screen.screened_search(F, X, Q, 10, R, prec, offs, ids)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, offs, ids, prec, R, "norm")


def test_leaf_priority_agrees_with_streaming(gf):
    # the same priority search, float32, by the streaming kernel and the leaf-major path
    X, Q, F = case("shared")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    a = gf.gf_query(G, Qg, 10, checks=20, algo=gf.GF_ALGO_LEAF)
    b = gf.gf_query(G, Qg, 10, checks=20, algo=gf.GF_ALGO_STREAM)
    assert_topk_close(X, Q, a[0].cpu().numpy(), a[1].cpu().numpy(), b[0].cpu().numpy(),
                      b[1].cpu().numpy().astype(np.float64))


def test_leaf_at_its_limits(gf):
    # the largest per-query key count the merge takes (T R = 256 x 32 = 8192 keys) and the largest
    # bucket count the regrouping takes (T 2^L = 64 x 2^16 = 2^22 leaves), against the oracle
    X, Q = synth.mixture(2000, 16, 300, "B", seed=5, qseed=6)
    F = oracle.build_forest(X, 256, 16, t=5, seed=11)
    assert F.T * 32 == 8192
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    gi, gd = gf.gf_query(G, Qg, 32, algo=gf.GF_ALGO_LEAF)
    oi, od = oracle.search(F, X, Q, 32)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    gi, gd = gf.gf_query(G, Qg, 10, precision=gf.GF_BF16_RERANK, rerank_R=32, algo=gf.GF_ALGO_LEAF)
    oi, od, cands = oracle_screen(F, X, Q, 10, 32)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, *cands, "bf16", 32, "norm")

    X, Q = synth.mixture(65_536, 8, 2000, "A", seed=7, qseed=8)
    F = oracle.build_forest(X, 64, 1, t=5, seed=13)
    assert F.L == 16 and F.T << F.L == 1 << 22
    G = gpu_forest(gf, X, F)
    gi, gd = gf.gf_query(G, torch.from_numpy(Q).cuda(), 5, algo=gf.GF_ALGO_LEAF)
    oi, od = oracle.search(F, X, Q, 5)
    assert_topk_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od)
    assert gf.gf_kernel_status() == 0


def test_leaf_rejects_what_it_does_not_run(gf):
    X, Q, F = case("tiny")
    G = gpu_forest(gf, X, F)
    Qg = torch.from_numpy(Q).cuda()
    for kw in (dict(precision=gf.GF_FP8_RERANK, rerank_R=33),                # shortlist above 32
               dict(precision=gf.GF_BF16_RERANK, rerank_R=33),
               dict(precision=gf.GF_BF16_RERANK, rerank_R=16, checks=1024)):  # 1024 leaves x R > 8192
        with pytest.raises(gf.GFError) as e:
            gf.gf_query(G, Qg, 10, algo=gf.GF_ALGO_LEAF, **kw)
        assert e.value.code == gf.GF_EUNSUPPORTED
    assert gf.gf_kernel_status() == 0
