"""Continuous-batching server: every answer equals the query run alone (streaming kernel) or the
oracle's search within tolerance (large batches on the leaf-major path); admission by HBM budget."""
import threading

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


@pytest.fixture(scope="module")
def forests(gf):
    specs = [(8000, 128, 8, 64, "A"), (20_000, 512, 12, 256, "B"), (30_000, 960, 16, 512, "B")]
    out = []
    for i, (n, d, T, p, law) in enumerate(specs):
        X, Q = synth.mixture(n, d, 64, law, seed=10 + i, qseed=20 + i)
        F = gf.gf_build(torch.from_numpy(X).cuda(), T, p, seed=i)
        gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
        out.append((F, Q))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_alone_equals_mixed(gf, forests, prec):
    p = gf.PRECISIONS[prec]
    S = gf.Server([F for F, _ in forests], max_batch=16, slots=3, k_max=10, precision=p, rerank_R=32)
    k = 10
    # alone: one request at a time
    alone = {}
    for f, (F, Q) in enumerate(forests):
        for i in range(Q.shape[0]):
            alone[(f, i)] = S.poll(S.submit(f, Q[i], k), k)
    # the same queries through gf_query, one batch per forest
    for f, (F, Q) in enumerate(forests):
        gi, gd = gf.gf_query(F, torch.from_numpy(Q).cuda(), k, precision=p, rerank_R=32)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        for i in range(Q.shape[0]):
            assert np.array_equal(alone[(f, i)][0], gi[i]) and np.array_equal(alone[(f, i)][1], gd[i])
    # mixed: four threads submit interleaved requests for all forests at once
    got = {}
    lock = threading.Lock()

    def worker(tid):
        tickets = []
        for f, (F, Q) in enumerate(forests):
            for i in range(tid, Q.shape[0], 4):
                tickets.append(((f, i), S.submit(f, Q[i], k)))
        for key, t in tickets:
            r = S.poll(t, k)
            with lock:
                got[key] = r

    th = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert set(got) == set(alone)
    for key, (ids, d) in got.items():
        assert np.array_equal(ids, alone[key][0]) and np.array_equal(d, alone[key][1])
    st = S.stats()
    assert st["completed"] > 0 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["leaf_batches"] == 0  # batches of at most 16 share no leaves: all streamed
    S.close()


def test_smaller_k_is_a_prefix(gf, forests):
    F, Q = forests[1]
    S = gf.Server([F], max_batch=8, slots=2, k_max=10)
    t3 = [S.submit(0, Q[i], 3) for i in range(8)]
    t10 = [S.submit(0, Q[i], 10) for i in range(8)]
    for a, b in zip(t3, t10):
        i3, d3 = S.poll(a, 3)
        i10, d10 = S.poll(b, 10)
        assert np.array_equal(i3, i10[:3]) and np.array_equal(d3, d10[:3])
    S.close()


def test_hbm_budget_limits_slots(gf, forests):
    F, _ = forests[2]
    big = gf.Server([F], max_batch=256, slots=8, hbm_budget_bytes=8 << 30)
    assert big.slots == 8
    # a slot holds a full batch's queries and results and the larger scratch of the two kernels a
    # batch may take (the leaf-major path's, when a full batch would take it)
    one = gf.gf_query_workspace_size(F, 256, algo=gf.GF_ALGO_AUTO) + 256 * F.info.d * 4 + 256 * 10 * 12
    S = gf.Server([F], max_batch=256, slots=8, hbm_budget_bytes=3 * one + 100)
    assert S.slots == 3
    S.close()
    big.close()


def test_budget_without_room_is_rejected(gf, forests):
    F, _ = forests[0]
    with pytest.raises(gf.GFError) as e:
        gf.Server([F], max_batch=64, slots=2, hbm_budget_bytes=1024)
    assert e.value.code == gf.GF_ENOMEM


def test_bad_requests(gf, forests):
    F, Q = forests[0]
    S = gf.Server([F], max_batch=4, slots=1, k_max=5)
    with pytest.raises(gf.GFError):
        S.submit(0, Q[0], 6)
    with pytest.raises(gf.GFError):
        S.submit(1, Q[0], 1)
    with pytest.raises(gf.GFError):
        S.poll(12345, 1, timeout_us=0)
    S.close()


def test_poisson_load_reports_latency(gf, forests):
    S = gf.Server([F for F, _ in forests], max_batch=64, slots=4, k_max=10)
    st = S.run_poisson([Q for _, Q in forests], rate_qps=5000, duration_s=0.5, k=10, seed=1)
    assert st["completed"] > 1000
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    S.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_large_batches_take_the_leaf_path(gf, prec):
    """A forest of two leaves a tree: batches of 8 queries or more share leaves enough for the
    leaf-major path (the rule of GF_ALGO_AUTO), which the server then runs; with one slot, requests
    pile up while a batch runs.  Every answer must be the oracle's search on the same forest, within
    the tolerance of the kernel that served it."""
    import oracle
    from oracle import screen
    from parity import assert_screened_close, assert_topk_close
    X, Q = synth.mixture(8000, 64, 1024, "B", seed=31, qseed=32)
    F = gf.gf_build(torch.from_numpy(X).cuda(), 8, 4000, seed=3)
    assert F.info.L == 1
    gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
    p = gf.PRECISIONS[prec]
    S = gf.Server([F], max_batch=512, slots=1, k_max=10, precision=p, rerank_R=32)
    tickets = [S.submit(0, Q[i], 10) for i in range(Q.shape[0])]
    res = [S.poll(t, 10) for t in tickets]
    st = S.stats()
    S.close()
    assert st["mean_batch"] >= 8, st
    assert st["leaf_batches"] >= 1, st  # the server says which path its batches took
    gi = np.stack([r[0] for r in res])
    gd = np.stack([r[1] for r in res])
    sd, sv, pm = gf.gf_forest_export(F)
    inf = F.info
    Fo = oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm)
    offs, ids = oracle.candidates(Fo, oracle.descend(Fo, Q))
    if prec == "fp32":
        oi, od = oracle.topk(X, Q, offs, ids, 10)
        assert_topk_close(X, Q, gi, gd, oi, od)
    else:
        oi, od, _ = screen.screened_search(Fo, X, Q, 10, 32, "bf16", offs, ids)
        # the norm form's bound is the wider one: it covers a batch served by either kernel
        assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, "bf16", 32, "norm")
    assert gf.gf_kernel_status() == 0
