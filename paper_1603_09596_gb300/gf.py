"""Python binding of the C ABI in include/gf.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device buffers are torch CUDA
tensors (allocation and streams come from PyTorch); all computation runs in the library's CUDA
kernels.  If the compiled library is missing, importing this module raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import _build

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ETIMEOUT, GF_EUNSUPPORTED, GF_EIO = 0, -1, -2, -3, -4, -5, -6
GF_FP32, GF_BF16_RERANK, GF_FP8_RERANK = 0, 1, 2
GF_VAR_NODE, GF_VAR_GLOBAL = 0, 1
PRECISIONS = {"fp32": GF_FP32, "bf16": GF_BF16_RERANK, "fp8": GF_FP8_RERANK}


class GFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gf error {code}: {msg}")
        self.code = code


class RandParams(C.Structure):
    _fields_ = [("t", C.c_int32), ("shuffle", C.c_int32), ("var_scope", C.c_int32),
                ("householder", C.c_int32)]


GF_ALGO_AUTO, GF_ALGO_SORT, GF_ALGO_STREAM, GF_ALGO_LEAF = 0, 1, 2, 3
GF_ORDER_AUTO, GF_ORDER_GIVEN, GF_ORDER_LOCALITY = 0, 1, 2


class QueryOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rerank_R", C.c_int32), ("warps_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("stream", C.c_void_p), ("algo", C.c_int32),
                ("rows_in_flight", C.c_int32), ("workspace", C.c_void_p), ("workspace_bytes", C.c_int64),
                ("ncand_out", C.c_void_p), ("order", C.c_int32), ("checks", C.c_int32), ("eps", C.c_double),
                ("events", C.c_void_p)]


class ServerOpts(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("slots", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("k_max", C.c_int32), ("precision", C.c_int32), ("rerank_R", C.c_int32),
                ("checks", C.c_int32), ("eps", C.c_double), ("algo", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("mean_batch", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("span_s", C.c_double), ("qps", C.c_double), ("slots", C.c_int32),
                ("leaf_batches", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ForestInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("T", C.c_int32), ("leaf_size", C.c_int32),
                ("L", C.c_int32), ("max_leaf", C.c_int32), ("cand_cap", C.c_int32),
                ("screens", C.c_int32), ("device_bytes", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"CUDA library {_build.LIB} is not built; run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        P, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        sig = {
            "gf_build": ([P, i64, i32, i32, i32, P, u64, P], i32),
            "gf_build_ex": ([P, i64, i32, i32, i32, P, u64, i32, P, P], i32),
            "gf_build_reflected": ([P, i64, i32, i32, i32, P, u64, P, i32, P, P], i32),
            "gf_forest_set_reflections": ([P, P], i32),
            "gf_forest_import": ([P, i64, i32, i32, i32, P, P, P, P], i32),
            "gf_forest_export": ([P, P, P, P], i32),
            "gf_forest_get_info": ([P, P], i32),
            "gf_forest_save": ([P, C.c_char_p], i32),
            "gf_forest_load": ([C.c_char_p, P], i32),
            "gf_forest_add_screen": ([P, i32, P], i32),
            "gf_forest_set_tuning": ([P, i32, i32, i32, i32, i32], i32),
            "gf_forest_free": ([P], i32),
            "gf_query": ([P, P, i64, i32, P, P], i32),
            "gf_query_ex": ([P, P, i64, i32, P, P, P], i32),
            "gf_query_workspace_size": ([P, i64, P, P], i32),
            "gf_descend": ([P, P, i64, P, P], i32),
            "gf_candidates": ([P, P, i64, P, P, P], i32),
            "gf_score_topk": ([P, P, i64, P, P, i32, i32, P, P, P], i32),
            "gf_score_screened": ([P, P, i64, P, P, i32, i32, P, P], i32),
            "gf_prio_leaves": ([P, P, i64, i32, C.c_double, P, P, i32, P], i32),
            "gf_server_opts_default": ([P], None),
            "gf_server_create": ([P, i32, P, P], i32),
            "gf_server_slots": ([P], i32),
            "gf_server_submit": ([P, i32, P, i32, P], i32),
            "gf_server_poll": ([P, u64, P, P, i32], i32),
            "gf_server_get_stats": ([P, P], i32),
            "gf_server_reset_stats": ([P], i32),
            "gf_server_run_poisson": ([P, P, P, C.c_double, C.c_double, i32, u64, i32, P], i32),
            "gf_server_destroy": ([P], i32),
            "gf_kernel_status": ([P], i32),
            "gf_debug_fail_alloc": ([i32], i32),
            "gf_debug_set_wait_limit": ([u64], i32),
            "gf_last_error": ([], C.c_char_p),
            "gf_version": ([], i32),
            "gf_rand_params_default": ([P], None),
            "gf_query_opts_default": ([P], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(code: int) -> None:
    if code != GF_OK:
        raise GFError(code, lib().gf_last_error().decode())


def _dptr(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Forest:
    """Owner of a gf_forest handle."""

    def __init__(self, handle: C.c_void_p):
        self.handle = handle
        self._info = None

    @property
    def info(self) -> ForestInfo:
        inf = ForestInfo()
        _check(lib().gf_forest_get_info(self.handle, C.byref(inf)))
        return inf

    def free(self) -> None:
        if self.handle:
            _check(lib().gf_forest_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gf_rand_params(t: int = 5, shuffle: int = 1, var_scope: int = GF_VAR_NODE,
                   householder: int = 0) -> RandParams:
    return RandParams(t, shuffle, var_scope, householder)


def gf_build(X: torch.Tensor, T: int, leaf_size: int, t: int = 5, shuffle: int = 1,
             var_scope: int = GF_VAR_NODE, seed: int = 0, householder: int = 0,
             borrow_x: bool = False, stream=None, U=None) -> Forest:
    """Build a forest on the GPU; with U (host [T, d] float32) every tree is built on its
    Householder-reflected points (gf_build_reflected)."""
    n, d = X.shape
    rp = gf_rand_params(t, shuffle, var_scope, 1 if U is not None else householder)
    h = C.c_void_p()
    if U is not None:
        import numpy as np
        Uh = np.ascontiguousarray(U, dtype=np.float32)
        if Uh.shape != (T, d):
            raise ValueError("U must be [T, d]")
        _check(lib().gf_build_reflected(_dptr(X, torch.float32, "X"), n, d, T, leaf_size, C.byref(rp),
                                        seed & (2**64 - 1), Uh.ctypes.data, int(borrow_x), _stream(stream),
                                        C.byref(h)))
    else:
        _check(lib().gf_build_ex(_dptr(X, torch.float32, "X"), n, d, T, leaf_size, C.byref(rp),
                                 seed & (2**64 - 1), int(borrow_x), _stream(stream), C.byref(h)))
    f = Forest(h)
    if borrow_x:
        f._x = X  # keep the borrowed points alive
    return f


def gf_forest_import(X: torch.Tensor, T: int, leaf_size: int, split_dim, split_val, perm) -> Forest:
    import numpy as np
    n, d = X.shape
    sd = np.ascontiguousarray(split_dim, dtype=np.int32)
    sv = np.ascontiguousarray(split_val, dtype=np.float32)
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().gf_forest_import(_dptr(X, torch.float32, "X"), n, d, T, leaf_size,
                                  sd.ctypes.data, sv.ctypes.data, pm.ctypes.data, C.byref(h)))
    return Forest(h)


def gf_forest_set_reflections(F: Forest, U) -> None:
    import numpy as np
    Uh = np.ascontiguousarray(U, dtype=np.float32)
    _check(lib().gf_forest_set_reflections(F.handle, Uh.ctypes.data))


def gf_forest_export(F: Forest):
    import numpy as np
    inf = F.info
    nn = (1 << inf.L) - 1
    sd = np.empty((inf.T, nn), dtype=np.int32)
    sv = np.empty((inf.T, nn), dtype=np.float32)
    pm = np.empty((inf.T, inf.n), dtype=np.int32)
    _check(lib().gf_forest_export(F.handle, sd.ctypes.data, sv.ctypes.data, pm.ctypes.data))
    return sd, sv, pm


def gf_forest_save(F: Forest, path) -> None:
    _check(lib().gf_forest_save(F.handle, os.fsencode(path)))


def gf_forest_load(path) -> Forest:
    h = C.c_void_p()
    _check(lib().gf_forest_load(os.fsencode(path), C.byref(h)))
    return Forest(h)


def gf_forest_add_screen(F: Forest, precision: int, stream=None) -> None:
    _check(lib().gf_forest_add_screen(F.handle, precision, _stream(stream)))


def gf_forest_set_tuning(F: Forest, precision: int, warps_per_cta: int, ctas_per_sm: int,
                         rerank_R: int, rows_in_flight: int = 0) -> None:
    _check(lib().gf_forest_set_tuning(F.handle, precision, warps_per_cta, ctas_per_sm, rerank_R,
                                      rows_in_flight))


def _opts(precision, rerank_R, warps_per_cta, ctas_per_sm, stream, algo, workspace, ncand_out,
          rows_in_flight=0, order=GF_ORDER_AUTO, checks=0, eps=0.0):
    o = QueryOpts(precision, rerank_R, warps_per_cta, ctas_per_sm, _stream(stream), algo, rows_in_flight,
                  None, 0, None, order, checks, eps)
    if workspace is not None:
        o.workspace = _dptr(workspace, workspace.dtype, "workspace")
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if ncand_out is not None:
        o.ncand_out = _dptr(ncand_out, torch.int32, "ncand_out")
    return o


def gf_query(F: Forest, Q: torch.Tensor, k: int, precision: int = GF_FP32, rerank_R: int = 0,
             warps_per_cta: int = 0, ctas_per_sm: int = 0, stream=None, algo: int = GF_ALGO_AUTO,
             workspace: torch.Tensor | None = None, ncand_out: torch.Tensor | None = None,
             rows_in_flight: int = 0, order: int = GF_ORDER_AUTO, checks: int = 0, eps: float = 0.0,
             out: tuple[torch.Tensor, torch.Tensor] | None = None, events=None):
    """k nearest neighbours of the rows of Q: (ids int64 [m, k], dists float32 [m, k]).  events: two
    torch.cuda.Event the query records just before and after its scoring kernel's launches."""
    qp = _dptr(Q, torch.float32, "Q")
    m = Q.shape[0]
    if out is None:
        ids = torch.empty((m, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((m, k), dtype=torch.float32, device=Q.device)
    else:
        ids, dists = out
    o = _opts(precision, rerank_R, warps_per_cta, ctas_per_sm, stream, algo, workspace, ncand_out,
              rows_in_flight, order, checks, eps)
    if events is not None:
        raw = []
        for ev in events:
            if not ev.cuda_event:  # torch creates an event at its first record
                ev.record(stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.current_stream())
            raw.append(ev.cuda_event)
        handles = (C.c_void_p * 2)(*raw)
        o.events = C.cast(handles, C.c_void_p)
    _check(lib().gf_query_ex(F.handle, qp, m, k, C.byref(o),
                             _dptr(ids, torch.int64, "ids"), _dptr(dists, torch.float32, "dists")))
    return ids, dists


def gf_query_workspace_size(F: Forest, m: int, precision: int = GF_FP32, rerank_R: int = 0,
                            warps_per_cta: int = 0, ctas_per_sm: int = 0, order: int = GF_ORDER_AUTO,
                            checks: int = 0, eps: float = 0.0, algo: int = GF_ALGO_STREAM) -> int:
    o = _opts(precision, rerank_R, warps_per_cta, ctas_per_sm, None, algo, None, None, 0, order,
              checks, eps)
    b = C.c_int64()
    _check(lib().gf_query_workspace_size(F.handle, m, C.byref(o), C.byref(b)))
    return b.value


def gf_descend(F: Forest, Q: torch.Tensor, stream=None) -> torch.Tensor:
    m = Q.shape[0]
    leaf = torch.empty((m, F.info.T), dtype=torch.int32, device=Q.device)
    _check(lib().gf_descend(F.handle, _dptr(Q, torch.float32, "Q"), m, _dptr(leaf, torch.int32, "leaf"),
                            _stream(stream)))
    return leaf


def gf_candidates(F: Forest, leaf: torch.Tensor, stream=None):
    m = leaf.shape[0]
    cap = F.info.cand_cap
    cand = torch.empty((m, cap), dtype=torch.int32, device=leaf.device)
    ncand = torch.empty((m,), dtype=torch.int32, device=leaf.device)
    _check(lib().gf_candidates(F.handle, _dptr(leaf, torch.int32, "leaf"), m,
                               _dptr(cand, torch.int32, "cand"), _dptr(ncand, torch.int32, "ncand"),
                               _stream(stream)))
    return cand, ncand


def gf_score_topk(F: Forest, Q: torch.Tensor, cand: torch.Tensor, ncand: torch.Tensor, k: int,
                  stream=None):
    m = Q.shape[0]
    ids = torch.empty((m, k), dtype=torch.int64, device=Q.device)
    dists = torch.empty((m, k), dtype=torch.float32, device=Q.device)
    _check(lib().gf_score_topk(F.handle, _dptr(Q, torch.float32, "Q"), m,
                               _dptr(cand, torch.int32, "cand"), _dptr(ncand, torch.int32, "ncand"),
                               cand.shape[1], k, _dptr(ids, torch.int64, "ids"),
                               _dptr(dists, torch.float32, "dists"), _stream(stream)))
    return ids, dists


def gf_score_screened(F: Forest, Q: torch.Tensor, cand: torch.Tensor, ncand: torch.Tensor,
                      precision: int, stream=None) -> torch.Tensor:
    m = Q.shape[0]
    dist = torch.full(cand.shape, float("nan"), dtype=torch.float32, device=Q.device)
    _check(lib().gf_score_screened(F.handle, _dptr(Q, torch.float32, "Q"), m,
                                   _dptr(cand, torch.int32, "cand"), _dptr(ncand, torch.int32, "ncand"),
                                   cand.shape[1], precision, _dptr(dist, torch.float32, "dist"),
                                   _stream(stream)))
    return dist


class Server:
    """Continuous-batching request loop over resident forests (gf_server_* in the C ABI)."""

    def __init__(self, forests, max_batch: int = 1024, slots: int = 4, hbm_budget_bytes: int = 4 << 30,
                 k_max: int = 10, precision: int = GF_FP32, rerank_R: int = 0, checks: int = 0,
                 eps: float = 0.0, algo: int = GF_ALGO_AUTO):
        self.forests = list(forests)      # keep the forests alive while the server runs
        arr = (C.c_void_p * len(self.forests))(*[f.handle for f in self.forests])
        o = ServerOpts(max_batch, slots, hbm_budget_bytes, k_max, precision, rerank_R, checks, eps, algo)
        self.handle = C.c_void_p()
        _check(lib().gf_server_create(arr, len(self.forests), C.byref(o), C.byref(self.handle)))
        self.dims = [f.info.d for f in self.forests]

    @property
    def slots(self) -> int:
        return lib().gf_server_slots(self.handle)

    def submit(self, forest: int, q, k: int) -> int:
        import numpy as np
        q = np.ascontiguousarray(q, dtype=np.float32)
        if 0 <= forest < len(self.dims) and q.shape != (self.dims[forest],):
            raise ValueError("query has the wrong length")
        t = C.c_uint64()
        _check(lib().gf_server_submit(self.handle, forest, q.ctypes.data, k, C.byref(t)))
        return t.value

    def poll(self, ticket: int, k: int, timeout_us: int = 10_000_000):
        import numpy as np
        ids = np.empty(k, dtype=np.int64)
        d = np.empty(k, dtype=np.float32)
        _check(lib().gf_server_poll(self.handle, ticket, ids.ctypes.data, d.ctypes.data, timeout_us))
        return ids, d

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().gf_server_get_stats(self.handle, C.byref(st)))
        return st.as_dict()

    def reset_stats(self) -> None:
        _check(lib().gf_server_reset_stats(self.handle))

    def run_poisson(self, queries, rate_qps: float, duration_s: float, k: int, seed: int = 0,
                    timeout_ms: int = 60_000) -> dict:
        import numpy as np
        qs = [np.ascontiguousarray(q, dtype=np.float32) for q in queries]
        ptrs = (C.c_void_p * len(qs))(*[q.ctypes.data for q in qs])
        nq = (C.c_int64 * len(qs))(*[q.shape[0] for q in qs])
        st = ServerStats()
        _check(lib().gf_server_run_poisson(self.handle, ptrs, nq, rate_qps, duration_s, k, seed,
                                           timeout_ms, C.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if self.handle:
            _check(lib().gf_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def leaf_budget(F: Forest, checks: int, eps: float = 0.0) -> int:
    """Leaves the priority search checks per query: max(T, ceil(c / (1 + eps)))."""
    T = F.info.T
    if checks <= T:
        return T
    b = checks / (1.0 + eps)
    nl = T
    while nl < b:
        nl += 1
    return nl


def gf_prio_leaves(F: Forest, Q: torch.Tensor, checks: int, eps: float = 0.0, stream=None):
    m = Q.shape[0]
    nb = leaf_budget(F, checks, eps)
    leaves = torch.zeros((m, nb), dtype=torch.int32, device=Q.device)
    nl = torch.empty((m,), dtype=torch.int32, device=Q.device)
    _check(lib().gf_prio_leaves(F.handle, _dptr(Q, torch.float32, "Q"), m, checks, eps,
                                _dptr(leaves, torch.int32, "leaves"), _dptr(nl, torch.int32, "nleaves"),
                                nb, _stream(stream)))
    return leaves, nl


def gf_kernel_status() -> int:
    """First error code a library kernel recorded since the last call (0: none); synchronizes."""
    v = C.c_int32(0)
    _check(lib().gf_kernel_status(C.byref(v)))
    return v.value


def gf_debug_fail_alloc(after: int) -> None:
    """Failure injection for tests: the (after + 1)-th library device allocation from now fails
    with GF_ENOMEM (once); after < 0 disarms."""
    _check(lib().gf_debug_fail_alloc(after))


def gf_debug_set_wait_limit(ns: int) -> None:
    """Failure injection for tests: time limit (ns, 0 = default) of the tensor-core scoring
    kernel's pipeline waits; a short one makes them run out (GF_ETIMEOUT in gf_kernel_status)."""
    _check(lib().gf_debug_set_wait_limit(ns))


def gf_version() -> int:
    return lib().gf_version()
