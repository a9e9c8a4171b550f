"""Failure handling on the GPU, driven by the library's injection hooks -- no device fault, trap or
hang is caused.

  * A device allocation made to fail (gf_debug_fail_alloc) at every point of a forest build: the
    build returns GF_ENOMEM, leaves no forest behind and no device memory allocated, and the next
    build, with nothing injected, equals a build that never failed.  The same for a screening copy
    added to a live forest, which stays usable.
  * The tensor-core scoring kernel's pipeline waits given a limit of a few hundred nanoseconds
    (gf_debug_set_wait_limit) on an ordinary launch: they run out, gf_kernel_status reports
    GF_ETIMEOUT, the kernel drains and frees its tensor memory, and the next query on the same
    context, with the default limit, agrees with the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import screen
from parity import assert_screened_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    yield g
    g.gf_debug_fail_alloc(-1)
    g.gf_debug_set_wait_limit(0)


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_build_allocation_failure_at_every_point(gf):
    X, _ = synth.mixture(20_000, 48, 1, "B", seed=21, qseed=22)
    Xg = torch.from_numpy(X).cuda()
    ref = gf.gf_build(Xg, 8, 40, seed=3)  # also loads the build's kernels before memory is watched
    want = gf.gf_forest_export(ref)
    ref.free()
    free0 = free_bytes()
    failed = 0
    for after in range(64):
        gf.gf_debug_fail_alloc(after)
        try:
            F = gf.gf_build(Xg, 8, 40, seed=3)
        except gf.GFError as e:
            assert e.code == gf.GF_ENOMEM, str(e)
            assert "gf_debug_fail_alloc" in str(e)
            assert free_bytes() == free0, f"allocation {after} failed and device memory leaked"
            failed += 1
            continue
        gf.gf_debug_fail_alloc(-1)
        got = gf.gf_forest_export(F)
        assert all(np.array_equal(a, b) for a, b in zip(got, want)), "a build after failed ones differs"
        F.free()
        break
    else:
        pytest.fail("the build never got past the injected failures")
    assert failed >= 3  # the forest's storage and the build's scratch: several allocations
    assert free_bytes() == free0


def test_screen_allocation_failure_keeps_the_forest(gf):
    X, Q = synth.mixture(5000, 32, 50, "A", seed=23, qseed=24)
    F = gf.gf_build(torch.from_numpy(X).cuda(), 4, 32, seed=5)
    Qg = torch.from_numpy(Q).cuda()
    before = gf.gf_query(F, Qg, 5)
    for prec in (gf.GF_BF16_RERANK, gf.GF_FP8_RERANK):
        for after in (0, 1):
            gf.gf_debug_fail_alloc(after)
            with pytest.raises(gf.GFError) as e:
                gf.gf_forest_add_screen(F, prec)
            assert e.value.code == gf.GF_ENOMEM
            assert not (F.info.screens >> prec) & 1
        gf.gf_debug_fail_alloc(-1)
        after_ids, after_d = gf.gf_query(F, Qg, 5)
        assert torch.equal(before[0], after_ids) and torch.equal(before[1], after_d)
        gf.gf_forest_add_screen(F, prec)
        assert (F.info.screens >> prec) & 1
    F.free()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_leaf_wait_runs_out_then_the_next_query_is_right(gf, prec):
    X, Q = synth.mixture(20_000, 96, 3000, "B", seed=25, qseed=26)
    F = oracle.build_forest(X, 8, 300, t=5, seed=7)
    G = gf.gf_forest_import(torch.from_numpy(X).cuda(), F.T, F.leaf_size, F.split_dim, F.split_val, F.perm)
    p = gf.PRECISIONS[prec]
    gf.gf_forest_add_screen(G, p)
    Qg = torch.from_numpy(Q).cuda()
    assert gf.gf_kernel_status() == 0
    gf.gf_debug_set_wait_limit(300)
    try:
        gf.gf_query(G, Qg, 10, precision=p, rerank_R=16, algo=gf.GF_ALGO_LEAF)
        status = gf.gf_kernel_status()
    finally:
        gf.gf_debug_set_wait_limit(0)
    assert status == gf.GF_ETIMEOUT
    # the context survived: the same query with the default limit is right
    gi, gd = gf.gf_query(G, Qg, 10, precision=p, rerank_R=16, algo=gf.GF_ALGO_LEAF)
    assert gf.gf_kernel_status() == 0
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    oi, od, _ = screen.screened_search(F, X, Q, 10, 16, prec, offs, ids)
    assert_screened_close(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, offs, ids, prec, 16, "norm")
