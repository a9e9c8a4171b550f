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
_COMMON = ["paper_1603_09596_gb300/csrc/gf_internal.cuh", "paper_1603_09596_gb300/csrc/gf_device.cuh",
           "paper_1603_09596_gb300/csrc/gf_score.cuh", "include/gf.h"]
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


def exact_nn(torch, Xg, Qs, k):
    """Exact k-NN of the sample Qs (evaluation only): float32 GEMM shortlist, float64 recheck."""
    xn = (Xg * Xg).sum(1)
    out_i, out_d = [], []
    for s in range(0, Qs.shape[0], 128):
        q = Qs[s:s + 128]
        D = xn[None, :] - 2.0 * (q @ Xg.T)
        cand = torch.topk(D, 64, dim=1, largest=False).indices
        diff = Xg[cand].double() - q.double()[:, None, :]
        ed = (diff * diff).sum(-1)
        o = torch.argsort(ed, dim=1)[:, :k]
        out_i.append(torch.gather(cand, 1, o))
        out_d.append(torch.gather(ed, 1, o))
    return torch.cat(out_i), torch.cat(out_d)


def recall(torch, Xg, Qs, ids, exact_i, exact_d):
    ids = ids[:, :exact_i.shape[1]]
    valid = ids[:, 0] >= 0
    x0 = Xg[ids[:, 0].clamp(min=0)].double()
    d0 = ((x0 - Qs.double()) ** 2).sum(1)
    r1 = float(((d0 <= exact_d[:, 0]) & valid).double().mean())
    k = exact_i.shape[1]
    hits = (ids[:, :, None] == exact_i[:, None, :]).any(-1).double().sum(1) / k
    return r1, float(hits.mean())


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


def leaf_bytes(gf, F, Qg, R, k, fp32=False):
    """Algorithmic bytes of one leaf-major batch: every chunk (a (tree, leaf) bucket cut into groups
    of at most 16 queries) reads its leaf's rows once -- bf16 with their ids and |x~|^2, or float32
    with their ids; plus the query (read, split or padded), the (query, tree) lists written and
    merged, the float32 rerank rows (bf16 screen) and the results.  The query rows re-read per row
    tile come from L2 (a few tens of MB in all) and are not counted."""
    import torch
    inf = F.info
    m, T, L = Qg.shape[0], inf.T, inf.L
    leaf = gf.gf_descend(F, Qg).long()
    u = (leaf + (torch.arange(T, device=Qg.device) << L)).flatten()
    cnt = torch.bincount(u, minlength=T << L)
    chunks = (cnt + 15) // 16
    b = torch.arange(T << L, device=Qg.device) & ((1 << L) - 1)
    rows = ((b + 1) * inf.n >> L) - (b * inf.n >> L)
    ldb, ldx = (inf.d + 7) // 8 * 8, (inf.d + 3) // 4 * 4
    if fp32:
        row_bytes = int((chunks * rows).sum()) * (ldx * 4 + 4)
        other = m * inf.d * 4 + m * ldx * 4 * 2 + m * T * R * 8 * 2 + m * k * 12
    else:
        row_bytes = int((chunks * rows).sum()) * (ldb * 2 + 8)
        other = m * inf.d * 4 * 2 + m * ldb * 2 * 2 + m * T * R * 8 * 2 + m * R * ldx * 4 + m * k * 12
    return row_bytes + other, int(chunks.sum())


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

    S = min(m, args.recall_sample)
    ei, ed = exact_nn(torch, Xg, Qg[:S], k)

    def time_query(F, prec, steps, warmup):
        return time_batch(gf, F, Qg, k, prec, steps, warmup, dev, world, local, args.no_graph)

    def bytes_per_query(F, prec, C, R, leaves=0):
        return query_bytes(gf, F, prec, C, R, d, k, leaves)

    def run_forest(T, p, tune_sample, checks=0, F=None):
        entry = {"T": T, "leaf_size": p}
        if F is None:
            torch.cuda.synchronize()
            tb = time.time()
            F = gf.gf_build(Xg, T, p, seed=0)
            torch.cuda.synchronize()
            entry["build_s"] = round(time.time() - tb, 3)
            gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
        entry["L"] = F.info.L
        if checks:
            entry["checks"] = checks
        nc = torch.empty((m,), dtype=torch.int32, device=dev)
        gf.gf_query(F, Qg, k, algo=gf.GF_ALGO_STREAM, ncand_out=nc, checks=checks)
        C = float(nc.double().mean())
        entry["cand_per_query"] = round(C, 1)
        leaves = gf.leaf_budget(F, checks) if checks else 0
        runs = [("fp32_stream", gf.GF_FP32, gf.GF_ALGO_STREAM), ("bf16_stream", gf.GF_BF16_RERANK, gf.GF_ALGO_STREAM)]
        if not checks:  # the leaf-major path runs the one-leaf-per-tree search
            runs += [("fp32_leaf", gf.GF_FP32, gf.GF_ALGO_LEAF), ("bf16_leaf", gf.GF_BF16_RERANK, gf.GF_ALGO_LEAF)]
        tuned = {}
        for name, prec, algo in runs:
            if prec not in tuned:
                tuned[prec] = autotune.tune(F, Qg[:tune_sample], k, prec, checks=checks)
            tr = tuned[prec]
            R = tr.get("R", 0)
            if algo == gf.GF_ALGO_LEAF and R > 32:  # the leaf-major path keeps at most 32
                continue
            ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, world, local,
                                         args.no_graph, checks, algo=algo, R=R)
            r1, rk = recall(torch, Xg, Qg[:S], ids[:S], ei, ed)
            mean_ms = statistics.mean(ms)
            if algo == gf.GF_ALGO_LEAF:
                lb, nchunks = leaf_bytes(gf, F, Qg, R if prec != gf.GF_FP32 else k, k, prec == gf.GF_FP32)
                bpq = lb / m
            else:
                bpq, nchunks = bytes_per_query(F, prec, C, R, leaves), None
            entry[name] = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4),
                           "ms_min": round(min(ms), 4), "recall_at_1": r1, "recall_at_10": rk, "clocks": ck,
                           "R": R, "algo": {gf.GF_ALGO_STREAM: "stream", gf.GF_ALGO_LEAF: "leaf"}[algo],
                           "bytes_per_query": round(bpq),
                           "achieved_gbs": round(bpq * m / (mean_ms / 1e3) / 1e9, 1)}
            if algo == gf.GF_ALGO_LEAF:
                entry[name]["chunks"] = nchunks
            else:
                entry[name].update(warps_per_cta=tr["warps"], ctas_per_sm=tr["ctas_per_sm"],
                                   rows_in_flight=tr["rows_in_flight"])
        for prec_name in ("fp32", "bf16"):
            cands = [entry[nm] for nm in (prec_name + "_stream", prec_name + "_leaf") if nm in entry]
            entry[prec_name] = max(cands, key=lambda e: e["qps"])
        return F, entry

    Fh, head = run_forest(HEADLINE["T"], HEADLINE["leaf_size"], args.tune_sample)
    spec = prio = None
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
    achieved = best["bytes_per_query"] * m / (mean_ms / 1e3) / 1e9
    algo = best["algo"]
    tr = recorded_traffic(algo)
    if tr and tr.get("point") != point_id:
        tr = None
    kernel = ("k_leaf_score (2 launches: tree 0, then the rest; tcgen05 bf16 screen) dominant, with the "
              "regrouping kernels and k_leaf_merge (dedupe + fp32 rerank + top-k); bytes and time of the whole step"
              if algo == "leaf" else
              "k_query_stream<bf16> (leaves + bitmap dedupe + bf16 screen + fp32 rerank + top-k), "
              + ("k_prio_leaves + " if "priority" in point_id else "") + "1 query launch/step")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": tr["bytes_per_launch"] if tr else None,
            "traffic_note": tr["note"] if tr else "no ncu record for the current kernel sources",
            "peak_kind": f"{peak_kind} STREAM copy (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "kernel": kernel, "bytes_per_query": best["bytes_per_query"]}

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
        gf.gf_query(Fc, Qd[bi], k, precision=gf.GF_BF16_RERANK, out=(ids, dd), checks=cc, stream=stream)
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
    # (batches of at most 1024 through the streaming kernel, 4 slots).  The server's capacity is
    # measured first (arrivals far above it for half a second); latency is then taken at Poisson
    # arrivals of half that capacity.
    lat = None
    if not args.no_serve:
        srv = gf.Server([Fc], max_batch=1024, slots=4, hbm_budget_bytes=8 << 30, k_max=k,
                        precision=gf.GF_BF16_RERANK, rerank_R=best["R"], checks=cc)
        srv.run_poisson([Q[:4096]], rate_qps=5000, duration_s=0.3, k=k, seed=3)
        cap = srv.run_poisson([Q], rate_qps=4.0 * chosen["bf16_stream"]["qps"], duration_s=0.5, k=k, seed=5)["qps"]
        rate = 0.5 * cap
        st = srv.run_poisson([Q], rate_qps=rate, duration_s=args.serve_seconds, k=k, seed=4)
        lat = {"capacity_qps": round(cap, 1), "offered_qps": round(rate, 1), "qps": round(st["qps"], 1),
               "p50_ms": round(st["p50_ms"], 3),
               "p99_ms": round(st["p99_ms"], 3), "mean_batch": round(st["mean_batch"], 1),
               "completed": st["completed"]}
        srv.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(X, Q, Fc, gf, k, budget_s=args.cpu_budget, checks=cc)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(mean_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"law-B Gaussian mixture n={n} d={d}, m={m} queries, k={k}",
                   "search": point_desc, "T": chosen["T"], "leaf_size": chosen["leaf_size"],
                   "checks": chosen.get("checks", chosen["T"]),
                   "precision": "bf16 screen + fp32 rerank", "R": best["R"],
                   "recall_at_1": best["recall_at_1"], "recall_sample": S,
                   "l2": "inputs larger than L2 (points 3.84 GB fp32 + 1.92 GB bf16)",
                   "parallelism": f"replicas x{world}"},
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
        "paths": {name: {key: chosen[name][key] for key in ("qps", "algo", "R", "achieved_gbs", "recall_at_1")}
                  for name in ("fp32_stream", "bf16_stream", "fp32_leaf", "bf16_leaf") if name in chosen},
        "operating_points": {pid: {"bf16_qps": pt["bf16"]["qps"], "fp32_qps": pt["fp32"]["qps"],
                                   "recall_at_1": pt["bf16"]["recall_at_1"], "cand_per_query": pt["cand_per_query"]}
                             for pid, _, pt in points},
        "headline_forest": {kk: head[kk] for kk in ("T", "leaf_size", "L", "build_s", "cand_per_query")},
        "at_T32_p64": spec,
        "at_T32_p64_priority": prio,
        "gen_s": round(gen_s, 2),
        "serving": lat,
        "p99_ms": lat["p99_ms"] if lat else None,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(X, Q, F, gf, k, budget_s=15.0, checks=0):
    """The oracle search, as it stands, on this host's cores over a bounded query sample."""
    import oracle
    sd, sv, pm = gf.gf_forest_export(F)
    inf = F.info
    Fo = oracle.Forest(inf.n, inf.d, inf.T, inf.leaf_size, inf.L, sd, sv, pm)
    done, t0, bs = 0, time.time(), 64
    while time.time() - t0 < budget_s and done < Q.shape[0]:
        if checks:
            oracle.search_priority(Fo, X, Q[done:done + bs], k, checks)
        else:
            oracle.search(Fo, X, Q[done:done + bs], k)
        done += min(bs, Q.shape[0] - done)
        bs = min(bs * 2, 1024)
    el = time.time() - t0
    search = f"priority search, c={checks}" if checks else "one leaf per tree"
    return {"value": round(done / el, 2), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} of the {Q.shape[0]} queries, same forest (T={inf.T}, leaf_size={inf.leaf_size}), "
                      f"{search}, float64"}


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
    """The d = 10^4 workload: float32 vs bf16 vs FP8-E4M3 screening (+ float32 rerank)."""
    import torch
    import paper_1603_09596_gb300 as gf
    from paper_1603_09596_gb300 import autotune
    import synth
    n, d, m, T, p, k = 200_000, 10_000, 2_000, 24, 32, 10
    X, Q = synth.mixture(n, d, m, "C", seed=0, qseed=1)
    dev = torch.device("cuda", 0)
    Xg, Qg = torch.from_numpy(X).to(dev), torch.from_numpy(Q).to(dev)
    del X
    S = min(m, args.recall_sample)
    ei, ed = exact_nn(torch, Xg, Qg[:S], k)
    tb = time.time()
    F = gf.gf_build(Xg, T, p, seed=0)
    torch.cuda.synchronize()
    build_s = time.time() - tb
    gf.gf_forest_add_screen(F, gf.GF_BF16_RERANK)
    gf.gf_forest_add_screen(F, gf.GF_FP8_RERANK)
    nc = torch.empty((m,), dtype=torch.int32, device=dev)
    gf.gf_query(F, Qg, k, algo=gf.GF_ALGO_STREAM, ncand_out=nc)
    C = float(nc.double().mean())
    hbm_peak, _ = peaks()
    out = {}
    for name in ("fp32", "bf16", "fp8"):
        prec = gf.PRECISIONS[name]
        tr = autotune.tune(F, Qg[:min(m, 1000)], k, prec)
        ids, dd, ms, ck = time_batch(gf, F, Qg, k, prec, args.steps, args.warmup, dev, no_graph=args.no_graph)
        r1, rk = recall(torch, Xg, Qg[:S], ids[:S], ei, ed)
        mean_ms = statistics.mean(ms)
        bpq = query_bytes(gf, F, prec, C, tr.get("R", 0), d, k)
        out[name] = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4),
                     "recall_at_1": r1, "recall_at_10": rk, "R": tr.get("R", 0),
                     "achieved_gbs": round(bpq * m / (mean_ms / 1e3) / 1e9, 1),
                     "frac_of_hbm": round(bpq * m / (mean_ms / 1e3) / 1e9 / hbm_peak, 4), "clocks": ck}
    print(json.dumps({"metric": "queries/s at 2e5 x 1e4, k=10: fp8 / bf16 screen + fp32 rerank vs fp32",
                      "unit": "queries/s", "n": n, "d": d, "m": m, "T": T, "leaf_size": p,
                      "cand_per_query": round(C, 1), "build_s": round(build_s, 2), "results": out}))


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
    ei, ed = exact_nn(torch, Xg, Qg[:S], k)
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
        r1, rk = recall(torch, Xg, Qg[:S], ids[:S], ei, ed)
        got = Xg[ids[:S, 0].clamp(min=0)].double()
        dr = ((got - Qg[:S].double()) ** 2).sum(1).sqrt()
        de = ed[:, 0].sqrt()
        eps_miss = {str(e): float(((dr > (1 + e) * de) | (ids[:S, 0] < 0)).double().mean()) for e in (0.0, 0.1, 0.5, 0.9)}
        mean_ms = statistics.mean(ms)
        out[name] = {"qps": round(m / (mean_ms / 1e3), 1), "ms_per_step": round(mean_ms, 4), "recall_at_1": r1,
                     "recall_at_10": rk, "eps_miss": eps_miss, "R": tr.get("R", 0), "clocks": ck}
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
    ei, ed = exact_nn(torch, Xg, Qg[:S], k)
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
            r1, rk = recall(torch, Xg, Qg[:S], ids[:S], ei, ed)
            res[pn] = {"qps": round(m / (statistics.mean(ms) / 1e3), 1), "recall_at_1": r1, "recall_at_10": rk,
                       "R": tr.get("R", 0)}
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
