"""gf_query_noalloc, the query entry point for callers that may not allocate device memory.

It is called here through the C ABI directly (ctypes), twice in a row on the same inputs -- the
second call finds the shared static scratch as the first left it -- and each answer is checked
against gf_query_ex (which allocates its scratch) within the tolerance the other GPU tests use:
distances within 1e-5 relative, ids equal.  The cases:
  - a batch small enough for a single launch;
  - so many points that the queries must be split over several launches to fit the scratch;
  - a forest tuned to launch far more CTAs than the SMs hold, sized so that its bitmaps leave
    less room than the locality order of a launch needs: the entry point must still find launches
    that fit rather than refuse the call;
  - a call on another forest in between, whose leftovers (bitmaps of another size, locality keys)
    must not leak into the next call's answers.
The entry point's one promise -- no device allocation -- is checked on the device's default
memory pool (where stream-ordered allocations land) and on the device's free memory, for every call
after the first (the first loads the library's module, and with it the array, on the device).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from parity import RTOL

pytestmark = pytest.mark.gpu

SCRATCH = 64 << 20  # GF_NOALLOC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    L = g.lib()
    f = L.gf_query_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int32
    # The array is device memory of the library's own module: the driver sets it aside when it loads
    # that module on the device, which with lazy module loading is the first call.  One call here,
    # so that the calls the tests watch come after it.
    X, Q = synth.mixture(64, 8, 2, "A", seed=1, qseed=2)
    F = g.gf_build(torch.from_numpy(X).cuda(), 2, 16, seed=1)
    Qg = torch.from_numpy(Q).cuda()
    ids = torch.empty((2, 1), dtype=torch.int64, device="cuda")
    d = torch.empty((2, 1), dtype=torch.float32, device="cuda")
    assert f(F.handle, Qg.data_ptr(), 2, 1, 0, 0, None, ids.data_ptr(), d.data_ptr()) == 0
    torch.cuda.synchronize()
    return g


def _cudart():
    """The CUDA runtime the library and torch share (already loaded), or None."""
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            pass
    return None


class PoolWatch:
    """Used-memory high-water mark of the current device's default memory pool."""
    USED_CURRENT, USED_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent / cudaMemPoolAttrUsedMemHigh

    def __init__(self):
        self.rt = _cudart()
        self.pool = C.c_void_p()
        if self.rt is not None:
            rc = self.rt.cudaDeviceGetDefaultMemPool(C.byref(self.pool), C.c_int(torch.cuda.current_device()))
            if rc != 0:
                self.rt = None

    def _get(self, attr):
        v = C.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, C.c_int(attr), C.byref(v)) == 0
        return v.value

    def reset(self):
        if self.rt is None:
            return None
        zero = C.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, C.c_int(self.USED_HIGH), C.byref(zero)) == 0
        return self._get(self.USED_CURRENT)

    def high(self):
        return None if self.rt is None else self._get(self.USED_HIGH)


def noalloc(gf, F, Qg, k, precision, R):
    m = Qg.shape[0]
    ids = torch.full((m, k), -7, dtype=torch.int64, device="cuda")
    d = torch.full((m, k), -1.0, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    watch = PoolWatch()
    used0 = watch.reset()
    free0 = torch.cuda.mem_get_info()[0]
    rc = gf.lib().gf_query_noalloc(F.handle, Qg.data_ptr(), m, k, precision, R, st, ids.data_ptr(),
                                   d.data_ptr())
    assert rc == 0, gf.lib().gf_last_error().decode()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    if used0 is not None:
        assert watch.high() == used0, "the call allocated from the default memory pool"
    assert free1 >= free0, f"device free memory fell by {free0 - free1} bytes during the call"
    return ids.cpu().numpy(), d.cpu().numpy()


def reference(gf, F, Qg, k, precision, R):
    ref_i, ref_d = gf.gf_query(F, Qg, k, precision=precision, rerank_R=R, algo=gf.GF_ALGO_STREAM)
    return ref_i.cpu().numpy(), ref_d.cpu().numpy()


def same(ids, d, ref_i, ref_d):
    fin = ref_i >= 0
    np.testing.assert_allclose(d[fin], ref_d[fin], rtol=RTOL)
    assert np.array_equal(ids, ref_i)


def check_against_query_ex(gf, F, Qg, k, precision, R, between=None):
    ref_i, ref_d = reference(gf, F, Qg, k, precision, R)
    for call in range(2):  # two calls in a row share the static scratch
        ids, d = noalloc(gf, F, Qg, k, precision, R)
        same(ids, d, ref_i, ref_d)
        if call == 0 and between is not None:
            between()


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
    assert SCRATCH // per_cta < Q.shape[0]
    check_against_query_ex(gf, F, torch.from_numpy(Q).cuda(), 5, gf.GF_FP32, 0)


def test_noalloc_many_ctas_leave_room_for_the_locality_order(gf):
    """32 CTAs per SM, and a bitmap sized so that one more CTA's bitmap would not fit: a launch with
    one query more than it has CTAs takes the queries in locality order, which needs 12 bytes a
    query after the bitmaps.  The call must still succeed, in launches that fit."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid = sms * 32
    words = SCRATCH // (grid + 1) // 4
    n = words * 32  # ceil(n / 32) words per bitmap; SCRATCH // per_cta == grid + 1 (or just above)
    X, Q = synth.mixture(n, 8, grid + 3000, "A", seed=45, qseed=46)
    F = gf.gf_build(torch.from_numpy(X).cuda(), 4, 256, seed=7)
    gf.gf_forest_set_tuning(F, gf.GF_FP32, 8, 32, 0, 0)
    per_cta = words * 4
    assert grid * per_cta + 12 * (grid + 1) > SCRATCH  # the old bitmap-only sizing would not fit
    check_against_query_ex(gf, F, torch.from_numpy(Q).cuda(), 4, gf.GF_FP32, 0)


def test_noalloc_after_a_call_on_another_forest(gf):
    """Between two calls on forest A, a call on forest B with a different bitmap size and a batch
    reordered for locality leaves its keys and bitmaps in the shared array; A's answers must not
    change."""
    XA, QA = synth.mixture(20_000, 32, 700, "B", seed=47, qseed=48)
    XB, QB = synth.mixture(3_000, 16, 5000, "A", seed=49, qseed=50)
    A = gf.gf_build(torch.from_numpy(XA).cuda(), 8, 64, seed=9)
    B = gf.gf_build(torch.from_numpy(XB).cuda(), 6, 32, seed=11)
    QAg, QBg = torch.from_numpy(QA).cuda(), torch.from_numpy(QB).cuda()
    ref_bi, ref_bd = reference(gf, B, QBg, 6, gf.GF_FP32, 0)

    def call_b():
        ids, d = noalloc(gf, B, QBg, 6, gf.GF_FP32, 0)
        same(ids, d, ref_bi, ref_bd)

    check_against_query_ex(gf, A, QAg, 10, gf.GF_FP32, 0, between=call_b)
