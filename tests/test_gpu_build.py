"""GPU forest build (Alg. 1, Alg. 3) against the CPU oracle.

With the same data, parameters and seed both sides make the same random draws, so the forests
must agree node for node; the only admissible difference is a near-tie in the variance ranking
(compensated float32 sums combined in float64 on the GPU, Welford's float64 recurrence in the
oracle; both within 1e-10 relative of the exact variance), which is checked explicitly.  Every
GPU forest must also satisfy the partition invariants on its own.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import check_forest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


def gpu_build(gf, X, T, p, **kw):
    G = gf.gf_build(torch.from_numpy(X).cuda(), T, p, **kw)
    sd, sv, pm = gf.gf_forest_export(G)
    inf = G.info
    return G, oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm)


def first_divergence(Fg, Fo):
    """(tree, heap index) of the first node, in level order, where the forests differ."""
    out = []
    for tr in range(Fo.T):
        for l in range(Fo.L):
            done = False
            for a in range(1 << l):
                j = (1 << l) - 1 + a
                lo, hi = (a * Fo.n) >> l, ((a + 1) * Fo.n) >> l
                if (Fg.split_dim[tr, j] != Fo.split_dim[tr, j] or Fg.split_val[tr, j] != Fo.split_val[tr, j]
                        or not np.array_equal(np.sort(Fg.perm[tr, lo:hi]), np.sort(Fo.perm[tr, lo:hi]))):
                    out.append((tr, l, a, j))
                    done = True
                    break
            if done:
                break
    return out


def assert_same_forest(X, Fg, Fo, t):
    assert Fg.L == Fo.L
    for tr, l, a, j in first_divergence(Fg, Fo):
        # admissible only as a variance near-tie among the top-t at that node
        lo, hi = (a * Fo.n) >> l, ((a + 1) * Fo.n) >> l
        pts = Fo.perm[tr, lo:hi]
        var = oracle.variance(X, np.sort(pts).astype(np.int32))
        sg, so = Fg.split_dim[tr, j], Fo.split_dim[tr, j]
        order = np.lexsort((np.arange(len(var)), -var))
        # the GPU's compensated float32 sums are within ~cnt * 2^-48 (< 1e-10) of float64
        near = np.abs(var - var[order[t - 1]]) <= 1e-10 * abs(var[order[t - 1]]) + 1e-300
        assert near.sum() > 1 or sg == so, f"tree {tr} node {j}: GPU split {sg}, oracle {so}, no variance tie"
    assert len(first_divergence(Fg, Fo)) <= max(1, Fo.T // 8)


CASES = [
    # (n, d, T, p, law, t, shuffle, var_scope)
    (10_000, 128, 8, 32, "A", 5, 1, 0),     # the tiny workload (level 0 is a chunked level)
    (50_000, 48, 4, 16, "B", 5, 1, 0),      # three chunked levels
    (3001, 37, 5, 9, "B", 3, 1, 0),         # ragged sizes, d not a multiple of 4
    (20_000, 64, 3, 20, "A", 5, 0, 0),      # no shuffling
    (20_000, 64, 3, 20, "A", 5, 1, 1),      # Alg. 1 literal: variance of the whole set
    (257, 1500, 2, 8, "C", 7, 1, 0),        # d above one dimension block
    (13, 4, 3, 1, "A", 2, 1, 0),            # leaf_size 1: empty leaves
    (40, 6, 2, 64, "A", 5, 1, 0),           # n <= p: a single leaf
]


@pytest.mark.parametrize("n,d,T,p,law,t,shuffle,scope", CASES + [(12_000, 100, 4, 32, "klein", 5, 1, 0)])
def test_build_matches_oracle(gf, n, d, T, p, law, t, shuffle, scope):
    if law == "klein":
        X, _ = synth.manifold(n, d, 1, "klein", seed=n)
    else:
        X, _ = synth.mixture(n, d, 1, law, seed=n)
    G, Fg = gpu_build(gf, X, T, p, t=t, shuffle=shuffle, var_scope=scope, seed=3)
    Fo = oracle.build_forest(X, T, p, t=t, shuffle=shuffle, var_scope=scope, seed=3)
    assert_same_forest(X, Fg, Fo, t)
    if n * T <= 60_000:
        check_forest(Fg, X, t, 3, shuffle, scope)


def test_build_quantized_ties(gf):
    # byte-valued data: coordinate ties everywhere; exact variance ties possible, so only the
    # invariants (which hold for any admissible tie order) are required
    X, _ = synth.mixture(4000, 16, 1, "B", seed=2)
    X = synth.quantize_u8(X, 4.0)
    G, Fg = gpu_build(gf, X, 3, 16, t=3, seed=9)
    check_forest(Fg, X, 3, 9, 1, 0, check_dims=False)


def test_build_is_deterministic(gf):
    X, _ = synth.mixture(30_000, 96, 1, "B", seed=5)
    _, F1 = gpu_build(gf, X, 6, 32, seed=11)
    _, F2 = gpu_build(gf, X, 6, 32, seed=11)
    assert np.array_equal(F1.perm, F2.perm) and np.array_equal(F1.split_dim, F2.split_dim)
    assert np.array_equal(F1.split_val, F2.split_val)


def test_build_rejects_bad_input(gf):
    X, _ = synth.mixture(100, 8, 1, "A", seed=1)
    Xg = torch.from_numpy(X).cuda()
    with pytest.raises(gf.GFError) as e:
        gf.gf_build(Xg, 2, 4, t=9)
    assert e.value.code == gf.GF_EINVAL
    with pytest.raises(gf.GFError) as e:
        gf.gf_build(Xg, 2, 4, householder=1)          # reflections need their vectors
    assert e.value.code == gf.GF_EINVAL
    Xn = Xg.clone()
    Xn[7, 3] = float("nan")
    with pytest.raises(gf.GFError) as e:
        gf.gf_build(Xn, 2, 4)
    assert e.value.code == gf.GF_EINVAL


def test_build_recall_matches_oracle_forest(gf):
    # the GIST-like law at 10^5 x 960, T=16, p=64: recall@1 of the GPU-built forest equals the
    # oracle-built forest's within 0.5 points (identical forests give identical recall)
    X, Q = synth.mixture(100_000, 960, 300, "B", seed=0, qseed=1)
    G, Fg = gpu_build(gf, X, 16, 64, seed=0)
    Fo = oracle.build_forest(X, 16, 64, seed=0)
    ei, ed = oracle.bruteforce(X, Q, 1)
    gi, _ = gf.gf_query(G, torch.from_numpy(Q).cuda(), 1)
    oi, _ = oracle.search(Fo, X, Q, 1)
    rg = oracle.recall_at_1(gi.cpu().numpy(), ed, X, Q)
    ro = oracle.recall_at_1(oi, ed, X, Q)
    assert abs(rg - ro) <= 0.005, (rg, ro)


# ---------------------------------------------------------------- Householder reflections (Sec. 2.2)

def _units(T, d, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((T, d))
    return (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)


@pytest.mark.parametrize("n,d,T,p", [(10_000, 64, 4, 32), (30_000, 37, 3, 16), (3000, 300, 2, 40)])
def test_reflected_build_matches_oracle(gf, n, d, T, p):
    X, _ = synth.mixture(n, d, 1, "B", seed=n + 1)
    U = _units(T, d, n)
    G = gf.gf_build(torch.from_numpy(X).cuda(), T, p, seed=4, U=U)
    sd, sv, pm = gf.gf_forest_export(G)
    inf = G.info
    Fg = oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm, U)
    Fo = oracle.build_forest(X, T, p, seed=4, U=U)
    assert np.array_equal(Fg.split_dim, Fo.split_dim)
    assert np.array_equal(Fg.split_val, Fo.split_val)
    assert np.array_equal(Fg.perm, Fo.perm)


def test_reflected_global_scope_is_rejected(gf):
    X, _ = synth.mixture(500, 8, 1, "A", seed=2)
    with pytest.raises(gf.GFError) as e:
        gf.gf_build(torch.from_numpy(X).cuda(), 2, 16, var_scope=gf.GF_VAR_GLOBAL, U=_units(2, 8, 1))
    assert e.value.code == gf.GF_EINVAL
