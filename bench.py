"""Throughput of batched kd-GeRaF queries on one GB300 (and N replicas under torchrun).

Workload (synthetic, seeded; stands in for GIST-1M, which is not available): n = 10^6 points,
d = 960, the GIST-like Gaussian-mixture law "B" (100 components, per-dimension std
1/sqrt(1 + j/32), shifted non-negative); m = 10^4 queries from the same mixture; k = 10.

A step is one batch of m queries through the whole search (descent, gather + de-duplication,
screened scoring, float32 rerank, top-k) with the forest and the points resident in HBM.  The
forest is built once per run on the GPU (its time is reported separately).  The headline number is
queries/s of the bfloat16 screen + float32 rerank at the operating point whose recall@1 >= 0.9;
the float32-only path and the tree parameters T=32, leaf_size=64 are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--small]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "queries/s at 1M×960, k=10, recall@1≥0.9: BF16-screen vs FP32 plain; p99 ms"
UNIT = "queries/s"

# operating points on the 10^6 x 960 law-B workload
HEADLINE = dict(T=32, leaf_size=1024)   # recall@1 >= 0.9 (one leaf per tree)
SPEC = dict(T=32, leaf_size=64)         # the tree parameters quoted with the workload


# the query kernels' sources and the committed ncu traffic record of each headline algorithm
# (the files that define the timed kernels; the C header's prose does not change them)
_COMMON = ["paper_1603_09596_gb300/csrc/gf_internal.cuh", "paper_1603_09596_gb300/csrc/gf_device.cuh",
           "paper_1603_09596_gb300/csrc/gf_score.cuh"]
KERNEL_SOURCES = {"stream": ["paper_1603_09596_gb300/csrc/gf_query.cu"] + _COMMON,
                  "leaf": ["paper_1603_09596_gb300/csrc/gf_leaf.cu"] + _COMMON}
TRAFFIC_FILES = {"stream": os.path.join(ROOT, "profiles", "k_query_stream_traffic.json"),
                 "leaf": os.path.join(ROOT, "profiles", "k_leaf_score_traffic.json")}


def kernel_source_hash(algo: str = "leaf") -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[algo]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def recorded_traffic(algo: str):
    """DRAM bytes per step of the headline algorithm from the committed ncu record, or None when the
    kernel sources changed since the counters were taken."""
    f = TRAFFIC_FILES[algo]
    if not os.path.exists(f):
        return None
    j = json.load(open(f))
    if j.get("source_sha256") != kernel_source_hash(algo):
        return None
    return j


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms_local: float, m_local: int, world: int, device=None):
    """Whole-job throughput over N replicas: every rank answered m_local queries; the job's time is
    the slowest rank's (max over ranks).  Returns (queries/s, max ms)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * m_local / (ms / 1e3), ms


def exact_cached(law, n, d, seed, qseed, m, nq, k):
    """Exact neighbours of the first nq of the m queries from the committed cache the oracle's
    brute force wrote (oracle/exact/, see oracle/exact_cache.py): (ids [nq, k], float64 squared
    distances [nq, k]), or None.  Only the file is read here."""
    p = os.path.join(ROOT, "oracle", "exact", f"law{law}_n{n}_d{d}_s{seed}_q{qseed}_m{m}_first{nq}_k{k}.json")
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    return np.array(j["ids"], dtype=np.int64), np.array(j["dist2"], dtype=np.float64)


def exact_scan(gf, Xg, Qs, k):
    """Exact neighbours by the library's own float32 scan (a forest of one tree whose single leaf
    holds every point), for workloads without an oracle cache: (ids, float64 distances)."""
    from paper_1603_09596_gb300 import autotune
    ids, _ = autotune.exact_neighbours(Xg, Qs, k)
    ids = ids.cpu().numpy()
    X = Xg.cpu().numpy()
    Q = Qs.cpu().numpy().astype(np.float64)
    d2 = ((X[ids].astype(np.float64) - Q[:, None, :]) ** 2).sum(-1)
    return ids, d2


def accuracy(X, Qs, ids, dists, exact):
    """Recall and distance error of a result against the exact neighbours (Sec. 4: a query is a
    miss unless its answer lies at the nearest distance; equal distances count as hits).
      recall_at_1, recall_at_10: as usual (ids);
      dist_rel_err_max / _median: |returned float32 distance - float64 distance of the returned id|
        relative to the latter, over all returned results (the arithmetic's error);
      approx_ratio_mean / _max: float64 distance of the i-th result over the i-th exact distance,
        minus 1 (the search's approximation, the paper's epsilon, per result)."""
    ids = np.asarray(ids)
    dists = np.asarray(dists, dtype=np.float64)
    ei, ed = exact
    nq, k = ei.shape
    ids, dists = ids[:nq, :k], dists[:nq, :k]
    Q = np.asarray(Qs[:nq], dtype=np.float64)
    valid = ids >= 0
    d64 = ((X[np.where(valid, ids, 0)].astype(np.float64) - Q[:, None, :]) ** 2).sum(-1)
    # (the two float64 sums add the same terms in different orders: equal up to ~1e-15)
    r1 = float(np.mean(valid[:, 0] & (d64[:, 0] <= ed[:, 0] * (1 + 1e-12))))
    r10 = float(np.mean([len(set(ids[i][valid[i]].tolist()) & set(ei[i].tolist())) / k for i in range(nq)]))
    rel = np.abs(dists - d64)[valid] / np.maximum(d64[valid], 1e-30)
    ratio = (d64 / np.maximum(ed, 1e-30) - 1.0)[valid]
    return {"recall_at_1": r1, "recall_at_10": r10,
            "dist_rel_err_max": float(rel.max()) if rel.size else None,
            "dist_rel_err_median": float(np.median(rel)) if rel.size else None,
            "approx_ratio_mean": float(ratio.mean()) if ratio.size else None,
            "approx_ratio_max": float(ratio.max()) if ratio.size else None,
            "sample": nq}


def time_batch(gf, F, Qg, k, prec, steps, warmup, dev, world=1, local=0, no_graph=False, checks=0, algo=0, R=0):
    """Time `steps` launches of the batch Qg; the launch is captured once in a CUDA graph (with a
    caller workspace, so nothing allocates inside the capture) and replayed per step."""
    import torch
    m = Qg.shape[0]
    ids = torch.empty((m, k), dtype=torch.int64, device=dev)
    dd = torch.empty((m, k), dtype=torch.float32, device=dev)
    ws = torch.zeros(gf.gf_query_workspace_size(F, m, precision=prec, rerank_R=R, checks=checks, algo=algo) // 4 + 1,
                     dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)

    def launch():
        gf.gf_query(F, Qg, k, precision=prec, rerank_R=R, out=(ids, dd), workspace=ws, stream=s, checks=checks,
                    algo=algo)

    with torch.cuda.stream(s):
        for _ in range(warmup):
            launch()
    torch.cuda.synchronize()
    graph = None
    if not no_graph:
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                launch()
            torch.cuda.synchronize()
            with torch.cuda.stream(s):
                graph.replay()
            torch.cuda.synchronize()
        except Exception as e:  # capture not possible here: time direct launches
            print(f"cuda graph capture failed, timing direct launches: {e}", file=sys.stderr)
            graph = None
            torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with Clocks(local) as ck:
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            for a, b in evs:
                a.record(s)
                graph.replay() if graph is not None else launch()
                b.record(s)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return ids, dd, ms, dict(ck.summary(), launch="cuda_graph" if graph is not None else "direct")


def query_bytes(gf, F, prec, C, R, d, k, leaves=0):
    """Algorithmic bytes of one query: candidate rows in the scored precision, the float32 rerank
    rows, the query, the leaf ids read from the permutations and the results."""
    inf = F.info
    positions = (leaves or inf.T) * (inf.n / (1 << inf.L))
    b = {gf.GF_FP32: 4, gf.GF_BF16_RERANK: 2, gf.GF_FP8_RERANK: 1}[prec]
    rows = C * (d * b + (4 if prec == gf.GF_FP8_RERANK else 0))
    rerank = R * d * 4 if prec != gf.GF_FP32 else 0
    return rows + rerank + d * 4 + positions * 4 + 12 * k


QP = {"fp32": 0, "bf16": 2, "fp8": 3}  # query parts of the tensor-core screens (MMA N = 16 QP)


def leaf_stats(gf, F, Qg, R, k, prec, checks=0):
    """One leaf-major step, from the batch's own leaves (the descents, or the priority search's
    lists with `checks`): chunks (a (tree, leaf) bucket cut into groups of at most 16 queries),
    128-row tiles (two chunks a tile when no leaf exceeds 64 rows), (row, query) pairs scored, MMAs
    issued, and the algorithmic bytes -- every chunk reads its leaf's rows once (the screen's copy
    with its ids and |x~|^2, and the E4M3 row scale), plus the queries (read, split), the (query,
    leaf) lists written and merged, the float32 rerank rows and the results.  The query parts
    re-read per row tile come from L2 and are not counted."""
    import torch
    inf = F.info
    m, T, L, n, d = Qg.shape[0], inf.T, inf.L, inf.n, inf.d
    if checks:
        codes, nl = gf.gf_prio_leaves(F, Qg, checks)
        S = codes.shape[1]
        live = torch.arange(S, device=Qg.device)[None, :] < nl[:, None]
        u = codes.long()[live]
    else:
        S = T
        leaf = gf.gf_descend(F, Qg).long()
        u = (leaf + (torch.arange(T, device=Qg.device) << L)).flatten()
    cnt = torch.bincount(u, minlength=T << L)
    chunks = (cnt + 15) // 16
    b = torch.arange(T << L, device=Qg.device) & ((1 << L) - 1)
    rows = ((b + 1) * n >> L) - (b * n >> L)
    ch = 2 if (n + (1 << L) - 1) >> L <= 64 else 1
    tiles = int((chunks * ((rows + 127) // 128)).sum()) if ch == 1 else (int(chunks.sum()) + 1) // 2
    pairs = int((cnt * rows).sum())
    ldx, ldb, ld8 = (d + 3) // 4 * 4, (d + 7) // 8 * 8, (d + 15) // 16 * 16
    crow = int((chunks * rows).sum())
    if prec == "fp32":
        row_b, other = ldx * 4 + 4, m * d * 4 + m * ldx * 4 * 2 + m * S * k * 8 * 2 + m * k * 12
    else:
        row_b = (ldb * 2 + 8) if prec == "bf16" else (ld8 + 12)
        qb = ldb * 2 if prec == "bf16" else ld8
        other = m * d * 4 * 2 + m * qb * QP[prec] + m * S * R * 8 * 2 + m * R * ldx * 4 + m * k * 12
    esz = {"bf16": 2, "fp8": 1}.get(prec, 4)
    mmas_per_tile = -(-d * esz // 32)  # one MMA per 32 bytes of the row (K = 16 bf16 or 32 E4M3)
    return {"chunks": int(chunks.sum()), "tiles": tiles, "chunks_per_tile": ch, "pairs": pairs,
            "bytes": crow * row_b + other, "useful_flops": 2.0 * pairs * d * QP[prec],
            "issued_flops": 2.0 * tiles * 128 * 16 * ch * QP[prec] * mmas_per_tile * (32 // esz) if QP[prec] else 0.0}


def time_kernel(gf, F, Qg, k, prec, algo, R, steps, dev, checks=0):
    """Mean time per step of the path's scoring kernel alone (both launches on the leaf-major
    path), from CUDA events the library records around its launches on the launching stream;
    direct launches after a warm-up, one event pair per step."""
    import torch
    m = Qg.shape[0]
    ids = torch.empty((m, k), dtype=torch.int64, device=dev)
    dd = torch.empty((m, k), dtype=torch.float32, device=dev)
    ws = torch.zeros(gf.gf_query_workspace_size(F, m, precision=prec, rerank_R=R, checks=checks, algo=algo) // 4 + 1,
                     dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kw = dict(precision=prec, rerank_R=R, out=(ids, dd), workspace=ws, stream=s, checks=checks, algo=algo)
    with torch.cuda.stream(s):
        for _ in range(2):
            gf.gf_query(F, Qg, k, **kw)
        for e in evs:
            gf.gf_query(F, Qg, k, events=e, **kw)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def tensor_peaks():
    """Dense bf16 TFLOP/s (burst, sustained) of the GB300s, and where the figure comes from."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["bf16_tflops"]), float(j.get("bf16_tflops_sustained", j["bf16_tflops"])), "measured"
    return 1900.0, 1700.0, "fallback"


def ours(args):
    import torch
    import paper_1603_09596_gb300 as gf
    from paper_1603_09596_gb300 import autotune

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import synth

    n, d, m, k = (args.n, args.d, args.m, 10)
    t0 = time.time()
    X, Q = synth.mixture(n, d, m, "B", seed=0, qseed=1 + rank)
    gen_s = time.time() - t0
    Xg = torch.from_numpy(X).to(dev)
    Qg = torch.from_numpy(Q).to(dev)
    stream = torch.cuda.current_stream(dev)
    hbm_peak, peak_kind = peaks()
    bf16_peak, bf16_sust, tpeak_kind = tensor_peaks()

    # the exact neighbours of the recall sample: the oracle's float64 brute force, cached per seed
    S = min(m, args.recall_sample)
    exact = exact_cached("B", n, d, 0, 1 + rank, m, S, k)
    exact_src = "oracle float64 brute force (oracle/exact cache)"
    if exact is None:
        exact = exact_scan(gf, Xg, Qg[:S], k)
        exact_src = "library float32 exact scan (no oracle cache for this workload)"

    def evaluate(ids, dd):
        return accuracy(X, Q, ids[:S].cpu().numpy(), dd[:S].cpu().numpy(), exact)

    def bytes_per_query(F, prec, C, R, leaves=0):
        return query_bytes(gf, F, prec, C, R, d, k, leaves)

    algos = {gf.GF_ALGO_STREAM: "stream", gf.GF_ALGO_LEAF: "leaf"}

    def run_forest(T, p, tune_sample, checks=0, F=None):
        entry = {"T": T, "leaf_size": p}
        if F is None:
            torch.cuda.synchronize()
            tb = time.time()
            F = gf.gf_build(Xg, T, p, seed=0)
            torch.cuda.synchronize()
            entry["build_s"] = round(time.time() - tb, 3)
            gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
            gf.gf_forest_add_screen(F, gf.GF_FP8_RERANK)
        entry["L"] = F.info.L
        if checks:
            entry["checks"] = checks
        nc = torch.empty((m,), dtype=torch.int32, device=dev)
        gf.gf_query(F, Qg, k, algo=gf.GF_ALGO_STREAM, ncand_out=nc, checks=checks)
        C = float(nc.double().mean())
        entry["cand_per_query"] = round(C, 1)
        leaves = gf.leaf_budget(F, checks) if checks else 0
        runs = [("fp32_stream", "fp32", gf.GF_ALGO_STREAM), ("bf16_stream", "bf16", gf.GF_ALGO_STREAM)]
        # the leaf-major path: one leaf per tree, or the priority search's lists (the screens; its
        # float32 kernel's 256-row tiles would stay mostly empty on the priority search's small leaves)
        runs += ([("fp32_leaf", "fp32", gf.GF_ALGO_LEAF)] if not checks else []) + \
            [("bf16_leaf", "bf16", gf.GF_ALGO_LEAF), ("fp8_leaf", "fp8", gf.GF_ALGO_LEAF)]
        for name, pn, algo in runs:
            prec = gf.PRECISIONS[pn]
            # kernel shape and shortlist: R is the shortest whose recall@1 and recall@10 on the tuning
            # sample stay within 0.5 points of the float32 search's (the leaf-major path keeps at most
            # 32, and its merge at most 8192 keys a query: (leaves per query) x R); the shape is the
            # fastest on the whole batch
            tr = autotune.tune(F, Qg[:tune_sample], k, prec, checks=checks, X=Xg, algo=algo,
                               r_max=min(32, 8192 // max(leaves, T)) if algo == gf.GF_ALGO_LEAF else 0, Qt=Qg)
            R = tr.get("R", 0)
            ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, world, local,
                                         args.no_graph, checks, algo=algo, R=R)
            mean_ms = statistics.mean(ms)
            if algo == gf.GF_ALGO_LEAF:
                st = leaf_stats(gf, F, Qg, R if pn != "fp32" else k, k, pn, checks)
                bpq = st["bytes"] / m
            else:
                st, bpq = None, bytes_per_query(F, prec, C, R, leaves)
            e = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4),
                 "ms_min": round(min(ms), 4), "clocks": ck, "R": R, "algo": algos[algo],
                 "bytes_per_query": round(bpq), "achieved_gbs": round(bpq * m / (mean_ms / 1e3) / 1e9, 1)}
            e.update(evaluate(ids, dd))
            if "recall" in tr:
                e["tuning_recall"] = {str(r): v for r, v in tr["recall"].items()}
            if st:
                e["chunks"] = st["chunks"]
                if pn != "fp32":  # the autotuner's shape of the tensor-core kernel
                    e["ctas_per_sm"] = tr["ctas_per_sm"] or 2
                    e["shape_ms"] = {("1 CTA/SM" if key.split("x")[1] == "1" else "2 CTAs/SM"): round(v, 3)
                                     for key, v in tr["timings"].items()}
            elif "warps" in tr:
                e.update(warps_per_cta=tr["warps"], ctas_per_sm=tr["ctas_per_sm"], rows_in_flight=tr["rows_in_flight"])
            entry[name] = e
        if not checks and (T, p) == (HEADLINE["T"], HEADLINE["leaf_size"]):
            # k = 1 at the same point (the workload asks for k = 1 and 10), with the shortlist the
            # k = 10 tuning chose
            for name, pn in (("fp32_leaf_k1", "fp32"), ("bf16_leaf_k1", "bf16")):
                R1 = entry[pn + "_leaf"]["R"]
                ids, dd, ms, ck = time_batch(gf, F, Qg, 1, gf.PRECISIONS[pn], args.steps, args.warmup, dev, world,
                                             local, args.no_graph, 0, algo=gf.GF_ALGO_LEAF, R=R1)
                mean_ms = statistics.mean(ms)
                acc = accuracy(X, Q, ids[:S].cpu().numpy(), dd[:S].cpu().numpy(), (exact[0][:, :1], exact[1][:, :1]))
                entry[name] = {"k": 1, "qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4),
                               "R": R1, "algo": "leaf", "clocks": ck,
                               **{key: acc[key] for key in ("recall_at_1", "dist_rel_err_max", "approx_ratio_mean",
                                                            "sample")}}
        for pn in ("fp32", "bf16", "fp8"):
            cands = [entry[nm] for nm in (pn + "_stream", pn + "_leaf") if nm in entry]
            if cands:
                entry[pn] = max(cands, key=lambda e: e["qps"])
        return F, entry

    Fh, head = run_forest(HEADLINE["T"], HEADLINE["leaf_size"], args.tune_sample)
    spec = prio = Fs = None
    if not args.skip_spec:
        Fs, spec = run_forest(SPEC["T"], SPEC["leaf_size"], args.tune_sample)
        if args.prio_checks > 0:
            # Alg. 2 proper on the same forest: the shared priority queue over all trees, c leaves
            _, prio = run_forest(SPEC["T"], SPEC["leaf_size"], args.tune_sample, checks=args.prio_checks, F=Fs)
    # headline: the fastest bf16 operating point whose recall@1 reaches 0.9
    points = [("one_leaf_T32_p1024", "one leaf per tree (Alg. 2 with c = T), T=32, leaf_size=1024", head)]
    if prio:
        points.append(("priority_T32_p64_c%d" % args.prio_checks,
                       "Alg. 2 shared priority queue, T=32, leaf_size=64, c=%d leaf checks" % args.prio_checks, prio))
    ok = [pt for pt in points if pt[2]["bf16"]["recall_at_1"] >= 0.9]
    point_id, point_desc, chosen = max(ok or points[:1], key=lambda pt: pt[2]["bf16"]["qps"])
    best = chosen["bf16"]
    Fc, cc = (Fh, 0) if point_id.startswith("one_leaf") else (Fs, args.prio_checks)
    value, mean_ms = aggregate(best["ms_per_step"], m, world, device=dev)
    algo = best["algo"]

    # roofline of the dominant kernel, timed alone with CUDA events on its stream
    gal = gf.GF_ALGO_LEAF if algo == "leaf" else gf.GF_ALGO_STREAM
    kms = time_kernel(gf, Fc, Qg, k, gf.GF_BF16_RERANK, gal, best["R"], args.steps, dev, checks=cc)
    tr = recorded_traffic(algo)
    if tr and (tr.get("point") != point_id or tr.get("ctas_per_sm", 2) != best.get("ctas_per_sm", 2)):
        tr = None  # taken on another workload or kernel shape
    traffic = (tr.get("bytes_per_step") or tr.get("bytes_per_launch")) if tr else None
    alg_bytes = best["bytes_per_query"] * m
    if algo == "leaf":
        st = leaf_stats(gf, Fc, Qg, best["R"], k, "bf16", cc)
        kernel = ("k_leaf_score<bf16> (tcgen05 kind::f16 screen; 2 launches per step: the chunks of tree 0, then the "
                  "rest), timed alone; bytes and flops of those launches")
        per_query = bytes_per_query(Fc, gf.GF_BF16_RERANK, chosen["cand_per_query"], best["R"])
        tensor = {"useful_tflops": round(st["useful_flops"] / (kms / 1e3) / 1e12, 2),
                  "issued_tflops": round(st["issued_flops"] / (kms / 1e3) / 1e12, 2),
                  "peak": bf16_peak, "unit": "TFLOP/s",
                  "frac_useful": round(st["useful_flops"] / (kms / 1e3) / 1e12 / bf16_peak, 4),
                  "frac_issued": round(st["issued_flops"] / (kms / 1e3) / 1e12 / bf16_peak, 4),
                  "peak_kind": f"{tpeak_kind} cuBLAS bf16 burst (MEASURED_PEAKS bf16_tflops)",
                  "note": "useful = (row, query) pairs x d x 2 flops x 2 query parts (hi, lo); issued adds the "
                          "padding of chunks to 16 queries and of leaves to 128-row tiles"}
    else:
        st, tensor, per_query = None, None, None
        kernel = ("k_query_stream<bf16> (leaves + bitmap dedupe + bf16 screen + fp32 rerank + top-k), "
                  + ("k_prio_leaves + " if "priority" in point_id else "") + "1 query launch per step")
    if traffic is not None:
        dram_gbs = traffic / (kms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(dram_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(dram_gbs / hbm_peak, 4), "traffic": traffic,
                "basis": "DRAM bytes of the kernel's launches in one step (ncu, committed record) / the kernel's "
                         "live CUDA-event time"}
    else:
        alg_gbs = (st["bytes"] if st else alg_bytes) / (kms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(alg_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(alg_gbs / hbm_peak, 4), "traffic": None,
                "basis": "algorithmic bytes / the kernel's live CUDA-event time (no ncu record for the current "
                         "kernel sources)"}
    roof.update({"peak_kind": f"{peak_kind} STREAM copy (MEASURED_PEAKS hbm_gbs)", "kernel": kernel,
                 "kernel_ms": round(kms, 4), "step_ms": round(best["ms_per_step"], 4)})
    if st:
        roof["algorithmic"] = {"bytes": st["bytes"], "gbs": round(st["bytes"] / (kms / 1e3) / 1e9, 1),
                               "frac": round(st["bytes"] / (kms / 1e3) / 1e9 / hbm_peak, 4),
                               "note": "L2-assisted: each chunk's leaf rows counted once per chunk; most of them "
                                       "come from L2 (the DRAM figure above is what HBM serves)"}
        roof["per_query_model"] = {"bytes_per_query": round(per_query),
                                   "gbs": round(per_query * m / (kms / 1e3) / 1e9, 1),
                                   "note": "each query reading its own candidates' rows, as the streaming kernel "
                                           "does; the leaf-major kernel shares every leaf read among the queries "
                                           "that reach it"}
        roof["tensor"] = tensor
        roof["chunks"], roof["tiles"] = st["chunks"], st["tiles"]

    # end to end through the public API with host buffers.  Every step copies its queries from
    # pinned host memory and reads its ids and distances back; the copy of step j + 1's queries
    # (on a copy stream, into the other of two device buffers) overlaps the query of step j.
    Qh = torch.from_numpy(Q).pin_memory()
    ih = torch.empty((m, k), dtype=torch.int64).pin_memory()
    dh = torch.empty((m, k), dtype=torch.float32).pin_memory()
    Qd = [torch.empty_like(Qg), torch.empty_like(Qg)]
    ids = torch.empty((m, k), dtype=torch.int64, device=dev)
    dd = torch.empty((m, k), dtype=torch.float32, device=dev)
    copy_stream = torch.cuda.Stream(device=dev)
    h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
    q_done = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d(j):  # step j's queries into buffer j % 2, once the query that last read it is done
        bi = j % 2
        copy_stream.wait_event(q_done[bi])
        with torch.cuda.stream(copy_stream):
            Qd[bi].copy_(Qh, non_blocking=True)
        h2d_done[bi].record(copy_stream)

    def e2e_step(j):
        bi = j % 2
        stream.wait_event(h2d_done[bi])
        gf.gf_query(Fc, Qd[bi], k, precision=gf.GF_BF16_RERANK, rerank_R=best["R"], out=(ids, dd), checks=cc,
                    stream=stream)
        q_done[bi].record(stream)
        with torch.cuda.stream(stream):
            ih.copy_(ids, non_blocking=True)
            dh.copy_(dd, non_blocking=True)

    def e2e_run(nsteps, start=None):
        if start is not None:
            copy_stream.wait_event(start)  # the first copy starts inside the timed region
        h2d(0)
        for j in range(nsteps):
            if j + 1 < nsteps:
                h2d(j + 1)
            e2e_step(j)

    e2e_run(args.warmup)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    e2e_run(args.steps, start=a)
    b.record(stream)
    torch.cuda.synchronize()
    e_ms = a.elapsed_time(b) / args.steps
    e2e = {"value": round(world * m / (e_ms / 1e3), 1), "unit": UNIT, "h2d_bytes_per_step": m * d * 4,
           "d2h_bytes_per_step": m * k * 12}

    # latency under load: single-query requests to the headline forest with continuous batching
    # (batches of at most 1024, 4 slots).  The server's capacity is measured first (arrivals far
    # above it for half a second); latency is then taken at Poisson arrivals of half that capacity.
    # Batches of at most 1024 stay on the streaming kernel (on this forest the leaf-major path needs
    # about 4 * 2^L = 4096 queries a batch); batches of up to 16,384 let a saturated server take it.
    lat = lat_big = None

    def serve_point(max_batch):
        srv = gf.Server([Fc], max_batch=max_batch, slots=4, hbm_budget_bytes=8 << 30, k_max=k,
                        precision=gf.GF_BF16_RERANK, rerank_R=best["R"], checks=cc)
        srv.run_poisson([Q[:4096]], rate_qps=5000, duration_s=0.3, k=k, seed=3)
        st_cap = srv.run_poisson([Q], rate_qps=4.0 * chosen["bf16"]["qps"], duration_s=0.5, k=k, seed=5)
        rate = 0.5 * st_cap["qps"]
        st_srv = srv.run_poisson([Q], rate_qps=rate, duration_s=args.serve_seconds, k=k, seed=4)
        srv.close()
        return {"max_batch": max_batch, "capacity_qps": round(st_cap["qps"], 1),
                "capacity_mean_batch": round(st_cap["mean_batch"], 1),
                "capacity_leaf_batches": f"{st_cap['leaf_batches']} of {st_cap['batches']}",
                "offered_qps": round(rate, 1), "qps": round(st_srv["qps"], 1),
                "p50_ms": round(st_srv["p50_ms"], 3), "p99_ms": round(st_srv["p99_ms"], 3),
                "mean_batch": round(st_srv["mean_batch"], 1),
                "leaf_batches": f"{st_srv['leaf_batches']} of {st_srv['batches']}", "completed": st_srv["completed"]}

    if not args.no_serve:
        lat = serve_point(1024)
        lat_big = serve_point(16384)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(X, Q, Fc, gf, k, budget_s=args.cpu_budget, checks=cc)

    configs = None
    if not args.no_configs:
        del Xg
        torch.cuda.empty_cache()
        configs = other_configs(args, gf, dev, X, Q, Fh)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(mean_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"law-B Gaussian mixture n={n} d={d}, m={m} queries, k={k}",
                   "search": point_desc, "T": chosen["T"], "leaf_size": chosen["leaf_size"],
                   "checks": chosen.get("checks", chosen["T"]),
                   "precision": "bf16 screen + fp32 rerank", "R": best["R"],
                   "recall_at_1": best["recall_at_1"], "recall_sample": S, "exact_neighbours": exact_src,
                   "l2": "inputs larger than L2 (points 3.84 GB fp32 + 1.92 GB bf16 + 0.96 GB e4m3)",
                   "parallelism": f"replicas x{world}"},
        "accuracy": {key: best[key] for key in ("recall_at_1", "recall_at_10", "dist_rel_err_max",
                                                "dist_rel_err_median", "approx_ratio_mean", "approx_ratio_max",
                                                "sample")},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        # library kernels per step: leaf-major = descend, 6 regrouping kernels, query split, 2 scoring
        # launches, merge; streaming = the 2 locality-order kernels and the query kernel (+ the
        # priority-queue kernel for the priority point)
        "gpu_launches": args.steps * (11 if algo == "leaf" else 3 + (1 if "priority" in point_id else 0)),
        "clocks": best["clocks"],
        "fp32_plain": chosen["fp32"],
        "bf16_screen": chosen["bf16"],
        "fp8_screen": chosen.get("fp8"),
        "paths": {name: {key: chosen[name][key] for key in ("qps", "algo", "R", "achieved_gbs", "recall_at_1",
                                                             "recall_at_10", "dist_rel_err_max")}
                  for name in ("fp32_stream", "bf16_stream", "fp32_leaf", "bf16_leaf", "fp8_leaf") if name in chosen},
        "operating_points": {pid: {"bf16_qps": pt["bf16"]["qps"], "fp32_qps": pt["fp32"]["qps"],
                                   "recall_at_1": pt["bf16"]["recall_at_1"], "cand_per_query": pt["cand_per_query"]}
                             for pid, _, pt in points},
        "headline_forest": {kk: head[kk] for kk in ("T", "leaf_size", "L", "build_s", "cand_per_query")},
        "k1": {name: head[name] for name in ("fp32_leaf_k1", "bf16_leaf_k1") if name in head},
        "at_T32_p64": spec,
        "at_T32_p64_priority": prio,
        "configs": configs,
        "gen_s": round(gen_s, 2),
        "serving": lat,
        "serving_large_batches": lat_big,
        "p99_ms": lat["p99_ms"] if lat else None,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(X, Q, F, gf, k, budget_s=15.0, checks=0):
    """The oracle search, as it stands, on this host's cores over a bounded query sample, and beside
    it the same search with float32 distances in a plain loop (a fairer CPU figure)."""
    import oracle
    sd, sv, pm = gf.gf_forest_export(F)
    inf = F.info
    Fo = oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm)

    def timed(fn, budget):
        done, t0, bs = 0, time.time(), 64
        while time.time() - t0 < budget and done < Q.shape[0]:
            fn(Q[done:done + bs])
            done += min(bs, Q.shape[0] - done)
            bs = min(bs * 2, 1024)
        return done, time.time() - t0

    if checks:
        done, el = timed(lambda q: oracle.search_priority(Fo, X, q, k, checks), budget_s)
    else:
        done, el = timed(lambda q: oracle.search(Fo, X, q, k), budget_s)
    search = f"priority search, c={checks}" if checks else "one leaf per tree"
    out = {"value": round(done / el, 2), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{done} of the {Q.shape[0]} queries, same forest (T={inf.T}, leaf_size={inf.leaf_size}), "
                     f"{search}, float64"}
    if not checks:
        d32, e32 = timed(lambda q: oracle.search_f32(Fo, X, q, k), budget_s / 2)
        out["fp32_loop"] = {"value": round(d32 / e32, 2), "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "float32 plain loop (oracle/gf_oracle.c gfo_search_f32)",
                            "sample": f"{d32} of the {Q.shape[0]} queries, same forest, one leaf per tree"}
    return out


def run_config(gf, dev, args, name, law, n, d, m, T, p, ks=(10,), precs=("fp32", "bf16"), sample=1000,
               shapes=None):
    """One workload: build its forest, time every precision's search (CUDA graph, AUTO kernel), and
    measure recall and distance error against the oracle's cached exact neighbours."""
    import torch
    import synth
    from paper_1603_09596_gb300 import autotune
    t0 = time.time()
    X, Q = synth.mixture(n, d, m, law, seed=0, qseed=1)
    gen_s = time.time() - t0
    Xg, Qg = torch.from_numpy(X).to(dev), torch.from_numpy(Q).to(dev)
    torch.cuda.synchronize()
    tb = time.time()
    F = gf.gf_build(Xg, T, p, t=min(5, d), seed=0)
    torch.cuda.synchronize()
    out = {"workload": f"law-{law} Gaussian mixture n={n} d={d}, m={m} queries", "T": T, "leaf_size": p,
           "L": F.info.L, "build_s": round(time.time() - tb, 3), "gen_s": round(gen_s, 1)}
    for pn in precs:
        if pn != "fp32":
            gf.gf_forest_add_screen(F, gf.PRECISIONS[pn])
    for k in ks:
        nq = min(sample, m)
        exact = exact_cached(law, n, d, 0, 1, m, nq, 10)
        src = "oracle float64 brute force (cached)"
        if exact is None:
            exact = exact_scan(gf, Xg, Qg[:nq], 10)
            src = "library float32 exact scan"
        exact = (exact[0][:, :k], exact[1][:, :k])
        for pn in precs:
            prec = gf.PRECISIONS[pn]
            tr = autotune.tune(F, Qg[:min(m, 500 if d > 2000 else 2000)], k, prec, X=Xg,
                               **({"shapes": shapes} if shapes else {}))
            R = tr.get("R", 0)
            ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, R=R)
            mean_ms = statistics.mean(ms)
            e = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4), "R": R,
                 "exact_neighbours": src}
            if "recall" in tr:
                e["tuning_recall"] = {str(r): v for r, v in tr["recall"].items()}
            e.update(accuracy(X, Q, ids[:nq].cpu().numpy(), dd[:nq].cpu().numpy(), exact))
            out[f"{pn}_k{k}"] = e
    F.free()
    del Xg, Qg
    torch.cuda.empty_cache()
    return out


def serve_config(gf, dev, args, Xh, Qh, Fh):
    """Six resident forests of uneven size under Poisson arrivals at 5k-200k queries/s (targets
    uniform over the forests), k = 10: throughput and p50/p99 latency per rate.  The 10^6 x 960
    forest is the headline's."""
    import torch
    import synth
    forests, queries = [], []
    t0 = time.time()
    for i, (n, d, T, p) in enumerate(SERVE_FORESTS):
        if (n, d) == (Xh.shape[0], Xh.shape[1]) and Fh is not None:
            forests.append(Fh)
            queries.append(Qh[:2048])
            continue
        X, Q = synth.mixture(n, d, 2048, "B", seed=100 + i, qseed=200 + i)
        F = gf.gf_build(torch.from_numpy(X).to(dev), T, p, seed=i)
        gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
        forests.append(F)
        queries.append(Q)
    setup_s = time.time() - t0
    S = gf.Server(forests, max_batch=1024, slots=args.serve_slots, hbm_budget_bytes=args.serve_budget << 30,
                  k_max=10, precision=gf.GF_BF16_RERANK, rerank_R=32)
    S.run_poisson(queries, rate_qps=5000, duration_s=0.3, k=10, seed=1)  # warm-up
    rates = []
    for rate in SERVE_RATES:
        st = S.run_poisson(queries, rate_qps=rate, duration_s=args.serve_seconds, k=10, seed=rate)
        rates.append({"offered_qps": rate, "qps": round(st["qps"], 1), "p50_ms": round(st["p50_ms"], 3),
                      "p99_ms": round(st["p99_ms"], 3), "max_ms": round(st["max_ms"], 3),
                      "mean_batch": round(st["mean_batch"], 1), "completed": st["completed"]})
    out = {"forests": [dict(n=n, d=d, T=T, leaf_size=p) for n, d, T, p in SERVE_FORESTS], "slots": S.slots,
           "precision": "bf16 screen + fp32 rerank, R=32", "setup_s": round(setup_s, 1), "rates": rates}
    S.close()
    for F in forests:
        if F is not Fh:
            F.free()
    return out


def other_configs(args, gf, dev, Xh, Qh, Fh):
    """The workloads beside the headline: tiny 10^4 x 128 (k = 1 and 10), batched 10^5 x 960,
    high-d 2 x 10^5 x 10^4 (float32 / bf16 / E4M3 screens) and the six-forest serving load."""
    out = {}
    t0 = time.time()
    out["tiny_1e4x128"] = run_config(gf, dev, args, "tiny", "A", 10_000, 128, 100, 8, 32, ks=(1, 10),
                                     precs=("fp32",), sample=100)
    out["batched_1e5x960"] = run_config(gf, dev, args, "batched", "B", 100_000, 960, 10_000, 16, 64,
                                        precs=("fp32", "bf16"))
    out["highd_2e5x1e4"] = run_config(gf, dev, args, "highd", "C", 200_000, 10_000, 2_000, 24, 32,
                                      precs=("fp32", "bf16", "fp8"), sample=200,
                                      shapes=[(8, 0, 0), (4, 0, 0), (8, 2, 0), (4, 2, 0)])
    if not args.no_serve:
        out["serving_6_forests"] = serve_config(gf, dev, args, Xh, Qh, Fh)
    out["seconds"] = round(time.time() - t0, 1)
    return out


def profile(args):
    """Fixed launches for ncu: build, one warm-up query, then --steps query launches."""
    import torch
    import paper_1603_09596_gb300 as gf
    import synth
    X, Q = synth.mixture(args.n, args.d, args.m, "B", seed=0, qseed=1)
    Xg, Qg = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    F = gf.gf_build(Xg, args.T, args.leaf_size, seed=0)
    prec = gf.PRECISIONS[args.precision]
    if prec:
        gf.gf_forest_add_screen(F, prec)
    algo = {"stream": gf.GF_ALGO_STREAM, "sort": gf.GF_ALGO_SORT, "leaf": gf.GF_ALGO_LEAF}[args.profile_algo]
    kw = dict(precision=prec, rerank_R=args.profile_R, warps_per_cta=args.profile_warps,
              ctas_per_sm=args.profile_ctas, algo=algo, rows_in_flight=args.profile_rows,
              checks=args.profile_checks)
    gf.gf_query(F, Qg, 10, **kw)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        gf.gf_query(F, Qg, 10, **kw)
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": True, "n": args.n, "d": args.d, "m": args.m, "T": args.T,
                      "leaf_size": args.leaf_size, "precision": args.precision, "algo": args.profile_algo,
                      "checks": args.profile_checks,
                      "ms_per_launch": a.elapsed_time(b) / args.steps, "kernel_status": gf.gf_kernel_status()}))


def highd(args):
    """The d = 10^4 workload alone: float32 vs bf16 vs FP8-E4M3 screening (+ float32 rerank)."""
    import torch
    import paper_1603_09596_gb300 as gf
    out = run_config(gf, torch.device("cuda", 0), args, "highd", "C", 200_000, 10_000, 2_000, 24, 32,
                     precs=("fp32", "bf16", "fp8"), sample=200)
    print(json.dumps({"metric": "queries/s at 2e5 x 1e4, k=10: fp8 / bf16 screen + fp32 rerank vs fp32",
                      "unit": "queries/s", **out}))


def klein(args):
    """Low-intrinsic-dimension workload: a noisy Klein bottle in R^100 (the paper's Klein set, Sec. 4,
    at 10^6 points), one leaf per tree; recall and the epsilon-miss rate of Sec. 4."""
    import torch
    import paper_1603_09596_gb300 as gf
    from paper_1603_09596_gb300 import autotune
    import synth
    n, d, m, T, p, k = 1_000_000, 100, 10_000, 32, 64, 10
    X, Q = synth.manifold(n, d, m, "klein", seed=0, qseed=1)
    dev = torch.device("cuda", 0)
    Xg, Qg = torch.from_numpy(X).to(dev), torch.from_numpy(Q).to(dev)
    S = min(m, args.recall_sample)
    exact = exact_scan(gf, Xg, Qg[:S], k)
    tb = time.time()
    F = gf.gf_build(Xg, T, p, seed=0)
    torch.cuda.synchronize()
    build_s = time.time() - tb
    gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
    out = {}
    for name in ("fp32", "bf16"):
        prec = gf.PRECISIONS[name]
        tr = autotune.tune(F, Qg[:min(m, 2000)], k, prec)
        ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, no_graph=args.no_graph)
        acc = accuracy(X, Q, ids[:S].cpu().numpy(), dd[:S].cpu().numpy(), exact)
        # the epsilon-miss rate of Sec. 4: the first answer farther than (1 + eps) times the nearest
        idn = ids[:S, 0].cpu().numpy()
        dr = np.sqrt(((X[np.maximum(idn, 0)].astype(np.float64) - Q[:S].astype(np.float64)) ** 2).sum(1))
        de = np.sqrt(exact[1][:, 0])
        eps_miss = {str(e): float(np.mean((dr > (1 + e) * de) | (idn < 0))) for e in (0.0, 0.1, 0.5, 0.9)}
        mean_ms = statistics.mean(ms)
        out[name] = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4), **acc,
                     "eps_miss": eps_miss, "R": tr.get("R", 0), "clocks": ck}
    print(json.dumps({"metric": "queries/s, noisy Klein bottle in R^100, n=10^6, k=10", "unit": "queries/s",
                      "n": n, "d": d, "m": m, "T": T, "leaf_size": p, "build_s": round(build_s, 2),
                      "results": out}))


def householder(args):
    """NEXT-4: the headline workload on a forest with a Householder reflection per tree (Sec. 2.2)."""
    import torch
    import paper_1603_09596_gb300 as gf
    from paper_1603_09596_gb300 import autotune
    import synth
    n, d, m, k = args.n, args.d, args.m, 10
    T, p = HEADLINE["T"], HEADLINE["leaf_size"]
    X, Q = synth.mixture(n, d, m, "B", seed=0, qseed=1)
    dev = torch.device("cuda", 0)
    Xg, Qg = torch.from_numpy(X).to(dev), torch.from_numpy(Q).to(dev)
    rng = np.random.default_rng(12345)
    U = rng.standard_normal((T, d))
    U = (U / np.linalg.norm(U, axis=1, keepdims=True)).astype(np.float32)
    S = min(m, args.recall_sample)
    exact = exact_cached("B", n, d, 0, 1, m, S, k) or exact_scan(gf, Xg, Qg[:S], k)
    out = {}
    for name, UU in (("plain", None), ("reflected", U)):
        torch.cuda.synchronize()
        tb = time.time()
        F = gf.gf_build(Xg, T, p, seed=0, U=UU)
        torch.cuda.synchronize()
        build_s = time.time() - tb
        gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
        res = {"build_s": round(build_s, 3)}
        for pn in ("fp32", "bf16"):
            prec = gf.PRECISIONS[pn]
            tr = autotune.tune(F, Qg[:min(m, 2000)], k, prec)
            ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, no_graph=args.no_graph)
            acc = accuracy(X, Q, ids[:S].cpu().numpy(), dd[:S].cpu().numpy(), exact)
            res[pn] = {"qps": round(m / (statistics.mean(ms) / 1e3), 1), **acc, "R": tr.get("R", 0)}
        out[name] = res
        F.free()
    print(json.dumps({"metric": "Householder reflection per tree (Sec. 2.2) vs none, headline workload",
                      "unit": "queries/s", "n": n, "d": d, "m": m, "T": T, "leaf_size": p, "results": out}))


SERVE_FORESTS = [  # (n, d, T, leaf_size): six resident forests of uneven size
    (10_000, 128, 16, 256), (50_000, 512, 16, 256), (100_000, 960, 24, 256),
    (500_000, 960, 32, 512), (1_000_000, 960, 32, 1024), (100_000, 4096, 16, 256)]
SERVE_RATES = [5_000, 20_000, 50_000, 100_000, 200_000]


def serve(args):
    """Continuous batching over six resident forests under Poisson load (k=10)."""
    import torch
    import paper_1603_09596_gb300 as gf
    import synth
    forests, queries = [], []
    t0 = time.time()
    for i, (n, d, T, p) in enumerate(SERVE_FORESTS):
        X, Q = synth.mixture(n, d, 2048, "B", seed=100 + i, qseed=200 + i)
        F = gf.gf_build(torch.from_numpy(X).cuda(), T, p, seed=i)
        if args.precision != "fp32":
            gf.gf_forest_add_screen(F, gf.PRECISIONS[args.precision])
        forests.append(F)
        queries.append(Q)
        del X
    setup_s = time.time() - t0
    S = gf.Server(forests, max_batch=1024, slots=args.serve_slots, hbm_budget_bytes=args.serve_budget << 30,
                  k_max=10, precision=gf.PRECISIONS[args.precision], rerank_R=32)
    S.run_poisson(queries, rate_qps=5000, duration_s=0.3, k=10, seed=1)  # warm-up
    out = []
    for rate in SERVE_RATES:
        st = S.run_poisson(queries, rate_qps=rate, duration_s=args.serve_seconds, k=10, seed=rate)
        out.append({"offered_qps": rate, "qps": round(st["qps"], 1), "p50_ms": round(st["p50_ms"], 3),
                    "p99_ms": round(st["p99_ms"], 3), "max_ms": round(st["max_ms"], 3),
                    "mean_batch": round(st["mean_batch"], 1), "completed": st["completed"]})
    line = {"metric": "serving: q/s and p50/p99 latency, 6 resident forests, Poisson arrivals, k=10",
            "unit": "queries/s", "precision": args.precision, "slots": S.slots,
            "forests": [dict(n=n, d=d, T=T, leaf_size=p) for n, d, T, p in SERVE_FORESTS],
            "setup_s": round(setup_s, 1), "rates": out}
    S.close()
    print(json.dumps(line))


def reference(args):
    """The oracle, timed on the host cores on the same workload (bounded query sample per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    n, d, m, k = args.n, args.d, args.m, 10
    X, Q = synth.mixture(n, d, m, "B", seed=0, qseed=1)
    tb = time.time()
    F = oracle.build_forest(X, HEADLINE["T"], HEADLINE["leaf_size"], seed=0)
    build_s = time.time() - tb
    per_step = args.ref_queries
    for w in range(args.warmup):
        oracle.search(F, X, Q[:min(m, 16)], k)
    times = []
    for s in range(args.steps):
        lo = (s * per_step) % m
        qs = Q[lo:lo + per_step]
        t = time.time()
        oracle.search(F, X, qs, k)
        times.append((time.time() - t) / qs.shape[0])
    sec_per_q = statistics.mean(times)
    value = 1.0 / sec_per_q
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec_per_q * per_step * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"law-B Gaussian mixture n={n} d={d}, m={m} queries, k={k}",
                   "T": HEADLINE["T"], "leaf_size": HEADLINE["leaf_size"], "precision": "float64 oracle",
                   "build_s": round(build_s, 1)},
        "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{per_step} queries per step"},
        "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=960)
    ap.add_argument("--m", type=int, default=10_000)
    ap.add_argument("--recall-sample", type=int, default=1000)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-queries", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--skip-spec", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the workloads beside the headline")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--prio-checks", type=int, default=512, help="leaf checks c of the priority-search point")
    ap.add_argument("--tune-sample", type=int, default=2000)
    ap.add_argument("--profile", action="store_true", help="fixed query launches for ncu")
    ap.add_argument("--T", type=int, default=HEADLINE["T"])
    ap.add_argument("--leaf-size", type=int, default=HEADLINE["leaf_size"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--profile-R", type=int, default=16)
    ap.add_argument("--profile-warps", type=int, default=8)
    ap.add_argument("--profile-rows", type=int, default=0)
    ap.add_argument("--source-hash", action="store_true", help="print the query kernel's source hash")
    ap.add_argument("--profile-ctas", type=int, default=0)
    ap.add_argument("--profile-algo", default="stream", choices=["stream", "sort", "leaf"])
    ap.add_argument("--profile-checks", type=int, default=0, help="leaf checks c (priority search) of the profile launches")
    ap.add_argument("--serve", action="store_true", help="serving workload (six forests, Poisson load)")
    ap.add_argument("--highd", action="store_true", help="d = 10^4 workload: fp8 / bf16 / fp32")
    ap.add_argument("--klein", action="store_true", help="noisy Klein bottle in R^100, 10^6 points")
    ap.add_argument("--householder", action="store_true", help="reflected vs plain forest on the headline workload")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget", type=int, default=8, help="GiB for batch slots")
    args = ap.parse_args()
    if args.source_hash:
        print(json.dumps({a: kernel_source_hash(a) for a in KERNEL_SOURCES}))
    elif args.profile:
        profile(args)
    elif args.serve:
        serve(args)
    elif args.highd:
        highd(args)
    elif args.klein:
        klein(args)
    elif args.householder:
        householder(args)
    elif args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
