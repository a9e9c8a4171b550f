"""Autotuner for the query kernel: CTA shape per precision and the screening shortlist R.

For a resident forest and a sample of queries it
  1. times every (warps per CTA, CTAs per SM) shape of the query kernel in each precision and
     keeps the fastest (the leaf-major tensor-core kernel: one or two CTAs per SM, i.e. a ring of
     eight or nine k-slices per SM against two rings of three or four);
  2. for a screened precision, picks the shortest shortlist R that costs the search no accuracy
     (the screen only decides which candidates get the exact float32 rerank, so this is what R
     trades away): given the points X, the shortest R whose recall@1 and recall@10 on the sample,
     against the exact neighbours (the library's own exact scan), are within `tol` of the float32
     search's; without X, the shortest R whose answers agree with the float32 search on at least
     `agree` of the sample's top-k entries;
and stores the choice in the forest (gf_forest_set_tuning), where gf_query picks it up.
Results are cached per (n, d, T, leaf_size, k, precision, batch) for the process.
"""
from __future__ import annotations

import torch

from . import gf

_cache: dict = {}

# (warps per CTA, CTAs per SM (0 = occupancy), rows in flight per warp (0 = default))
SHAPES = [(w, c, g) for w in (4, 8) for c in (0, 2, 3) for g in (0, 2, 4)] + [(16, 0, 0), (16, 1, 0)]
R_CHOICES = [16, 24, 32, 48, 64, 128, 256]


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _recalls(ids: torch.Tensor, dists: torch.Tensor, ex_ids: torch.Tensor, ex_d: torch.Tensor):
    """recall@1 (the first answer at the exact nearest distance; equal distances count, Sec. 4) and
    recall@k of a result against exact neighbours."""
    # (float32 distances of the same point from two kernels may differ in the last bits)
    r1 = float(((dists[:, 0] <= ex_d[:, 0] * (1 + 2e-6)) & (ids[:, 0] >= 0)).float().mean())
    rk = float((ids[:, :, None] == ex_ids[:, None, :]).any(-1).float().mean())
    return r1, rk


def tune(F: gf.Forest, Q: torch.Tensor, k: int, precision: int, agree: float = 0.995,
         shapes=SHAPES, r_choices=R_CHOICES, checks: int = 0, X: torch.Tensor | None = None,
         tol: float = 0.005, algo: int = gf.GF_ALGO_AUTO, r_max: int = 0,
         Qt: torch.Tensor | None = None) -> dict:
    """Qt: the batch the shapes are timed on (default Q); the best shape depends on how many
    queries share a leaf, so time it on a batch of the size that will run."""
    inf = F.info
    Qt = Q if Qt is None else Qt
    key = (inf.n, inf.d, inf.T, inf.leaf_size, k, precision, Q.shape[0], checks, X is not None, algo, r_max,
           Qt.shape[0])
    if key in _cache:
        res = _cache[key]
        gf.gf_forest_set_tuning(F, precision, res["warps"], res["ctas_per_sm"], res.get("R", 0),
                                res["rows_in_flight"])
        return res
    res: dict = {"precision": precision}
    R = 0
    if precision != gf.GF_FP32:
        choices = [r for r in r_choices if r >= k and (r_max <= 0 or r <= r_max)]
        if r_max > 0 and r_max not in choices and r_max >= k:
            choices.append(r_max)
        R = choices[-1]
        ref_ids, ref_d = gf.gf_query(F, Q, k, checks=checks)
        if X is not None:
            # accuracy parity with the float32 search against the exact neighbours
            ex_ids, ex_d = _exact(X, Q, k)
            ref = _recalls(ref_ids, ref_d, ex_ids, ex_d)
            res["criterion"] = f"recall@1 and recall@{k} within {tol} of float32's {ref}"
            for r in choices:
                ids, d = gf.gf_query(F, Q, k, precision=precision, rerank_R=r, checks=checks, algo=algo)
                got = _recalls(ids, d, ex_ids, ex_d)
                res.setdefault("recall", {})[r] = got
                if got[0] >= ref[0] - tol and got[1] >= ref[1] - tol:
                    R = r
                    break
        else:
            res["criterion"] = f"top-{k} ids agree with float32's on {agree} of entries"
            for r in choices:
                ids, _ = gf.gf_query(F, Q, k, precision=precision, rerank_R=r, checks=checks, algo=algo)
                hit = (ids[:, :, None] == ref_ids[:, None, :]).any(-1).float().mean().item()
                res.setdefault("agreement", {})[r] = hit
                if hit >= agree:
                    R = r
                    break
        res["R"] = R
    timings = {}
    if algo == gf.GF_ALGO_LEAF:
        # the leaf-major tensor-core kernel: two CTAs per SM (0, the default) or one with a deeper
        # ring (1); the float32 one has a single shape
        shapes = [(8, 0, 0)] + ([(8, 1, 0)] if precision != gf.GF_FP32 else [])
    for w, c, g in shapes:
        try:
            t = _time(lambda: gf.gf_query(F, Qt, k, precision=precision, rerank_R=R, warps_per_cta=w,
                                          ctas_per_sm=c, rows_in_flight=g, checks=checks, algo=algo))
        except gf.GFError:
            continue
        timings[(w, c, g)] = t
    (w, c, g), t = min(timings.items(), key=lambda kv: kv[1])
    res.update(warps=w, ctas_per_sm=c, rows_in_flight=g, ms=t,
               timings={f"{a}x{b}x{e}": v for (a, b, e), v in timings.items()})
    gf.gf_forest_set_tuning(F, precision, w, c, R, g)
    _cache[key] = res
    return res


# ---------------------------------------------------------------- forest configuration
#
# Sec. 3 ("Configuration") sets the leaf size p, the leaf checks c, the split-dimension count t and
# the number of trees from (epsilon, n, d, the top-5 variances) with piecewise-constant rules whose
# constants the paper does not print.  configure() is the hook in their place: it measures.  For a
# grid of (T, leaf_size, c) it builds the forest on the GPU, runs the query sample, and scores
# recall@1 against the exact nearest neighbours -- computed by this library itself on a one-leaf
# forest (leaf_size >= n makes every query scan all points exactly).  It returns the fastest
# configuration whose recall@1 reaches the target.

DEFAULT_GRID = [(T, p, c) for T in (16, 32) for p in (64, 256, 1024) for c in (0,)]


_exact_cache: dict = {}


def _exact(X: torch.Tensor, Q: torch.Tensor, k: int):
    key = (X.data_ptr(), tuple(X.shape), Q.data_ptr(), tuple(Q.shape), k)
    if key not in _exact_cache:
        _exact_cache.clear()
        _exact_cache[key] = exact_neighbours(X, Q, k)
    return _exact_cache[key]


def exact_neighbours(X: torch.Tensor, Q: torch.Tensor, k: int = 1):
    """Exact k-NN by the library's own kernel: one tree whose single leaf holds every point."""
    F1 = gf.gf_build(X, 1, X.shape[0], seed=0)
    ids, d = gf.gf_query(F1, Q, k, algo=gf.GF_ALGO_STREAM)
    torch.cuda.synchronize()
    F1.free()
    return ids, d


def recall_at_1(F: gf.Forest, Q: torch.Tensor, exact_d: torch.Tensor, checks: int = 0) -> float:
    ids, d = gf.gf_query(F, Q, 1, checks=checks)
    return float((d[:, 0] <= exact_d[:, 0]).float().mean())


def configure(X: torch.Tensor, Q: torch.Tensor, target_recall: float = 0.9, grid=DEFAULT_GRID,
              t: int = 5, seed: int = 0) -> dict:
    """Fastest (T, leaf_size, checks) on the grid whose recall@1 on Q reaches target_recall."""
    _, ed = exact_neighbours(X, Q)
    tried = []
    for T, p, c in grid:
        F = gf.gf_build(X, T, p, t=min(t, X.shape[1]), seed=seed)
        r = recall_at_1(F, Q, ed, checks=c)
        ms = _time(lambda: gf.gf_query(F, Q, 10, checks=c))
        tried.append({"T": T, "leaf_size": p, "checks": c, "recall_at_1": r, "ms": ms})
        F.free()
    ok = [e for e in tried if e["recall_at_1"] >= target_recall]
    best = min(ok, key=lambda e: e["ms"]) if ok else max(tried, key=lambda e: e["recall_at_1"])
    return {"choice": best, "met_target": bool(ok), "tried": tried}
