"""gf_query_noalloc, the query entry point for callers that may not allocate device memory.

It is called here through the C ABI directly (ctypes), twice in a row on the same inputs -- the
second call finds the shared static scratch as the first left it -- and each answer is checked
against gf_query_ex (which allocates its scratch) within the tolerance the other GPU tests use:
distances within 1e-5 relative, ids equal.  One case is small enough for a single launch; the other
has so many points that the queries must be split over several launches to fit the scratch.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from parity import RTOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    L = g.lib()
    f = L.gf_query_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int32
    return g


def noalloc(gf, F, Qg, k, precision, R):
    m = Qg.shape[0]
    ids = torch.full((m, k), -7, dtype=torch.int64, device="cuda")
    d = torch.full((m, k), -1.0, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = gf.lib().gf_query_noalloc(F.handle, Qg.data_ptr(), m, k, precision, R, st, ids.data_ptr(),
                                   d.data_ptr())
    assert rc == 0, gf.lib().gf_last_error().decode()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy()


def check_against_query_ex(gf, F, Qg, k, precision, R):
    ref_i, ref_d = gf.gf_query(F, Qg, k, precision=precision, rerank_R=R, algo=gf.GF_ALGO_STREAM)
    ref_i, ref_d = ref_i.cpu().numpy(), ref_d.cpu().numpy()
    for _ in range(2):  # two calls in a row share the static scratch
        ids, d = noalloc(gf, F, Qg, k, precision, R)
        fin = ref_i >= 0
        np.testing.assert_allclose(d[fin], ref_d[fin], rtol=RTOL)
        assert np.array_equal(ids, ref_i)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_single_launch(gf, prec):
    X, Q = synth.mixture(5000, 64, 300, "B", seed=41, qseed=42)
    F = gf.gf_build(torch.from_numpy(X).cuda(), 6, 40, seed=3)
    p = gf.PRECISIONS[prec]
    if p:
        gf.gf_forest_add_screen(F, p)
    check_against_query_ex(gf, F, torch.from_numpy(Q).cuda(), 10, p, 32)


def test_noalloc_splits_launches_to_fit_the_scratch(gf):
    # 10^6 points: one bitmap is 125,000 bytes, so a launch may use at most 536 CTAs of the
    # 64 MiB scratch and 1500 queries take three launches
    X, Q = synth.mixture(1_000_000, 16, 1500, "A", seed=43, qseed=44)
    F = gf.gf_build(torch.from_numpy(X).cuda(), 4, 512, seed=5)
    per_cta = ((F.info.n + 31) // 32) * 4
    assert (64 << 20) // per_cta < Q.shape[0]
    check_against_query_ex(gf, F, torch.from_numpy(Q).cuda(), 5, gf.GF_FP32, 0)
