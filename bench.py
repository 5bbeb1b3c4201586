"""Benchmark: query throughput of MRPT with voting on one GB300.

Workload (default): 60,000 x 784 stroke images with integer pixel values
0..255 and about 80 % zeros (the MNIST shape of Table II), 10,000 held-out
queries, k = 10, trees of depth 8.  The number of trees T (50/100/200, taken
as prefixes of one 200-tree index) and the vote threshold v (1..10) are
picked by a sweep: the fastest (T, v) whose recall@10 reaches 0.9.  A step
is one query pass over the 10,000 queries (projection, routing, voting,
candidate distances, top-k), inputs resident in HBM; L2 is flushed before
every timed step.

Prints one JSON line (see the keys below).  ``--impl reference`` times the
CPU oracle instead, on a bounded sample of the same workload.
Multi-GPU (torchrun, N > 1): every rank holds a replica of the index and
answers its own 10,000 queries (weak scaling; no collective on the path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = dict(name="mnist-like 60000x784 u8-valued fp32, 10000 queries, k=10, depth 8",
                n=60000, d=784, m=10000, k=10, l=8, T_max=200, T_grid=(50, 100, 200),
                v_grid=tuple(range(1, 11)), seed=0, target_recall=0.9)
METRIC = "queries/sec at recall@10>=0.9 (mnist-like 60000x784, k=10)"


# ----------------------------------------------------------------- utils --

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_ms: float, units_per_rank: int, steps: int, world: int, device=None):
    """Replicas: every rank answers its own batch.  The job's time is the
    slowest rank's (max over ranks, over the default process group when
    world > 1); the job's throughput counts every rank's units."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * units_per_rank * steps / (total_ms / 1e3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


HEADLINE_MAX_BYTES = 2048
# optional keys dropped, in this order, if a headline would not fit
_DROPPABLE = (("stage_ms",), ("config", "fp32_best"), ("config", "knobs"), ("clocks", "samples"),
              ("roofline", "peak_kind"), ("cpu_baseline", "single_thread"))


def emit_line(out: dict, limit: int = HEADLINE_MAX_BYTES) -> str:
    """Print `out` as one compact JSON line (the last line of stdout, which
    the result is read from) and return it.  Optional keys are dropped in a
    fixed order if the line would be longer than `limit` bytes."""
    line = json.dumps(out, separators=(",", ":"))
    for path in _DROPPABLE:
        if len(line.encode()) <= limit:
            break
        node = out
        for key in path[:-1]:
            node = node.get(key) if isinstance(node, dict) else None
        if isinstance(node, dict):
            node.pop(path[-1], None)
        line = json.dumps(out, separators=(",", ":"))
    print(line, flush=True)
    return line


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha(kernel: str, path: str) -> str:
    """Hash of one kernel's source: the lines from its `__global__`
    declaration to the next top-level closing brace."""
    lines = open(path).read().split("\n")
    start = None
    for i, ln in enumerate(lines):
        if "__global__" in ln and (kernel + "(") in " ".join(lines[i:i + 2]):
            start = i
            break
    if start is None:
        return ""
    end = start
    while end < len(lines) and lines[end] != "}":
        end += 1
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()[:16]


def search_kernel_name(prec: int, d: int) -> str:
    """The candidate-search kernel the library launches for rows of `d`
    values in precision `prec` (0 float32, 1 bfloat16, 2 e4m3): per-lane
    cp.async rows (k_cand_knn_rows) for rows of at least 8 16-byte chunks
    of values and at most 1,024 padded values, whole-row bulk copies
    (k_cand_knn) otherwise."""
    dpad = (d + 7) & ~7
    nchunk = (dpad + 15) // 16 if prec == 2 else dpad // (8 if prec == 1 else 4)
    return "k_cand_knn_rows" if nchunk >= 8 and dpad <= 1024 else "k_cand_knn"


def load_traffic(kernel: str, src: str, key: str = "dram_bytes_per_launch"):
    """A figure (DRAM bytes per launch by default) from the committed ncu
    summary of `kernel`, if it was taken on the kernel's current source
    (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    entry = json.load(open(p)).get(kernel)
    if not entry or entry.get("source_sha") != kernel_source_sha(kernel, src):
        return None
    return entry.get(key)


# ------------------------------------------------------- ground truth -----

def exact_knn_gpu(X, Q, k, torch):
    """Exact k-NN in float64 on the GPU (ground truth for recall only).
    Returns (ids, kth distance^2) with ids ordered by (distance, id)."""
    Xd = X.double()
    xn = (Xd * Xd).sum(1)
    ids_out, kth_out = [], []
    for s in range(0, Q.shape[0], 512):
        q = Q[s:s + 512].double()
        d2 = (q * q).sum(1, keepdim=True) + xn[None, :] - 2.0 * (q @ Xd.T)
        vals, idx = torch.topk(d2, k + 8, dim=1, largest=False, sorted=True)
        # order by (distance, id) among the k + 8 smallest
        key = torch.argsort(idx, dim=1)
        vals, idx = torch.gather(vals, 1, key), torch.gather(idx, 1, key)
        key = torch.argsort(vals, dim=1, stable=True)
        vals, idx = torch.gather(vals, 1, key), torch.gather(idx, 1, key)
        ids_out.append(idx[:, :k])
        kth_out.append(vals[:, k - 1])
    return torch.cat(ids_out), torch.cat(kth_out)


def recall_at_k(ids, X, Q, gt_ids, gt_kth, torch):
    """Recall |A n K| / k (Sec. I-A): strict (K ordered by (distance, id))
    and tie-aware (a returned point counts when its exact distance is at
    most the true k-th distance)."""
    m, k = gt_ids.shape
    strict = 0
    for s in range(0, m, 2048):
        a = ids[s:s + 2048].long()
        g = gt_ids[s:s + 2048].long()
        strict += (a[:, :, None] == g[:, None, :]).any(2).sum().item()
    valid = ids >= 0
    a = ids.clamp(min=0).long()
    ta = 0
    for s in range(0, m, 1024):
        rows = X[a[s:s + 1024]].double()                       # b x k x d
        q = Q[s:s + 1024].double()[:, None, :]
        d2 = ((rows - q) ** 2).sum(2)
        ok = (d2 <= gt_kth[s:s + 1024, None] * (1 + 1e-12)) & valid[s:s + 1024]
        ta += ok.sum().item()
    return strict / (m * k), ta / (m * k)


# ------------------------------------------------------------- GPU arm ----

def run_gpu(args):
    import torch
    import paper_1509_06957_gb300 as mr

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = WORKLOAD
    X_np, Q_np = workloads.mnist_like(W["n"], W["m"], seed=W["seed"])
    X = torch.from_numpy(X_np).to(dev)
    Q = torch.from_numpy(Q_np).to(dev)
    n, d, m, k, l = W["n"], W["d"], W["m"], W["k"], W["l"]

    # ---- build (timed once)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    index = mr.mrpt_build(X, W["T_max"], l, 0.0, seed=W["seed"])
    build_s = time.perf_counter() - t0

    gt_ids, gt_kth = exact_knn_gpu(X, Q, k, torch)
    ids = torch.empty((m, k), dtype=torch.int32, device=dev)
    dists = torch.empty((m, k), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    mr.mrpt_add_lowp(index, mr.MRPT_PREC_BF16)
    mr.mrpt_add_lowp(index, mr.MRPT_PREC_FP8)

    knobs = dict(chunk=0, ring=0)

    def query(T_use, v, stage=None, prec=0, margin=0):
        mr.mrpt_query_ex(index, Q, k, v, n_trees=T_use, out_ids=ids, out_dists=dists,
                         stage_ms=stage, path=args.path, precision=prec, margin=margin,
                         chunk=knobs["chunk"], ring=knobs["ring"])

    # ---- sweep (T, v): fastest with recall >= target (tie-aware), unless
    # the operating point is given
    sweep = []
    stage = np.zeros(4, np.float32)
    grid = [(args.T, args.v)] if args.T and args.v else \
        [(T_, v_) for T_ in W["T_grid"] for v_ in W["v_grid"] if v_ <= T_]
    bf16 = [(1, m_) for m_ in (0, 8, 32)]
    fp8 = [(2, m_) for m_ in (8, 32)]
    precs = {"fp32": [(0, 0)], "bf16": bf16, "fp8": fp8,
             "auto": [(0, 0)] + bf16 + fp8}[args.precision]
    if args.path == 1:
        precs = [(0, 0)]
    for T_use, v in grid:
        for prec, margin in precs:
            query(T_use, v, prec=prec, margin=margin)  # warm
            flush.zero_()
            query(T_use, v, stage, prec=prec, margin=margin)
            rs, rt = recall_at_k(ids, X, Q, gt_ids, gt_kth, torch)
            sweep.append(dict(T=T_use, v=v, precision=("fp32", "bf16", "fp8")[prec], margin=margin,
                              ms=float(stage[3]), recall=round(rt, 4), recall_strict=round(rs, 4)))
    ok = [s for s in sweep if s["recall"] >= W["target_recall"]]
    best = min(ok, key=lambda s: s["ms"]) if ok else max(sweep, key=lambda s: s["recall"])
    T_use, v = best["T"], best["v"]
    prec, margin = ("fp32", "bf16", "fp8").index(best["precision"]), best["margin"]
    ok32 = [s for s in ok if s["precision"] == "fp32"]
    best32 = min(ok32, key=lambda s: s["ms"]) if ok32 else None

    # ---- launch knobs (work-item chunk, staged rows, path) for that setting
    from paper_1509_06957_gb300 import autotune
    knobs = autotune.tune_kernels(index, Q, k, v, T_use, prec, margin, reps=3)["best"] \
        if args.path == 0 else dict(path=1, chunk=0, ring=0, ms=None)
    args.path = knobs["path"]

    # ---- mean |S| at the operating point (untimed debug pass)
    _, _, dbg = mr.mrpt_query_ex(index, Q[:2000], k, v, n_trees=T_use, debug=True, cand_cap=1)
    mean_S = float(dbg["n_cand"].double().mean().item())
    del dbg

    # ---- timed steps (device-resident inputs)
    for _ in range(args.warmup):
        query(T_use, v, prec=prec, margin=margin)
    torch.cuda.synchronize()
    per_step, vote_ms, route_ms, search_ms = [], [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            query(T_use, v, stage, prec=prec, margin=margin)
            route_ms.append(float(stage[0]))
            vote_ms.append(float(stage[1]))
            search_ms.append(float(stage[2]))
            per_step.append(float(stage[3]))
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.summary()
    total_ms, value = aggregate(sum(per_step), m, args.steps, world, dev)
    recall_strict, recall_ta = recall_at_k(ids, X, Q, gt_ids, gt_kth, torch)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(mr, index, Q, k, v, T_use, flush, args, world, torch, prec, margin, knobs)

    # ---- rooflines: voting (leaf ids, L2-resident) and candidate search
    # (candidate rows); "roofline" reports the kernel that takes longer
    peak, peak_kind = load_peaks()
    L = 1 << l
    leaf_bytes = T_use * math.ceil(n / L) * 4
    # candidate rows in the precision used, plus the float32 rows of the
    # re-rank (the library skips it only for a lossless bfloat16 copy)
    bf16_exact = bool(torch.equal(X, X.bfloat16().float()))
    vbytes = (4, 2, 1)[prec]
    rerank = prec == 2 or (prec == 1 and not bf16_exact)
    rerank_rows = min(k + margin, mean_S) if rerank else 0
    row_bytes = mean_S * (d * vbytes + (16 if prec == 2 else 0)) + rerank_rows * d * 4
    vote_avg = statistics.mean(vote_ms)
    search_avg = statistics.mean(search_ms)
    if args.path == 1:
        # one fused kernel reads both
        vote_bytes = leaf_bytes + row_bytes + d * 4 + T_use * 4 + k * 8
        search_bytes = 0.0
    else:
        vote_bytes = leaf_bytes + T_use * 4 + mean_S * 4 + 4
        search_bytes = row_bytes + mean_S * 4 + d * 4 + k * 8 + 4
    src = os.path.join(ROOT, "paper_1509_06957_gb300", "csrc", "mrpt_query.cu")

    def roof(name, per_query, ms):
        achieved = per_query * m / (ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": load_traffic(name, src),
                "l2_sectors_pct": load_traffic(name, src, "l2_sectors_pct_of_peak"),
                "peak_kind": f"{peak_kind} hbm_gbs", "kernel": name,
                "bytes_per_query": round(per_query, 1), "avg_ms": round(ms, 4)}

    # ids of at most 65,536 points fit one counter array: the vote kernel
    # then reads the padded leaf layout (k_vote_flat)
    vote_kernel = "k_vote_search" if args.path == 1 else ("k_vote_flat" if n <= 65536 else "k_vote_emit")
    r_vote = roof(vote_kernel, vote_bytes, vote_avg)
    rooflines = [r_vote]
    if args.path == 0:
        r_search = roof(search_kernel_name(prec, d), search_bytes, search_avg)
        # each candidate row once per step (rows reused across queries)
        uniq = min(n, mean_S * m) * d * 4
        r_search["frac_rows_once"] = round(
            (uniq + (search_bytes - row_bytes) * m) / (search_avg / 1e3) / 1e9 / peak, 4)
        rooflines.append(r_search)
    roofline = max(rooflines, key=lambda r: r["avg_ms"])
    others = [r for r in rooflines if r is not roofline]
    # whole query path: B_q = T ceil(n/2^l) 4 (leaf ids) + |S| d b (candidate
    # rows, b bytes per value) + d 4 (query) + k 8 (output) [+ re-rank rows],
    # over the step's device time
    path_bytes = leaf_bytes + row_bytes + d * 4 + k * 8
    step_ms = total_ms / args.steps
    path_roofline = {"achieved": round(path_bytes * m / (step_ms / 1e3) / 1e9, 1),
                     "frac": round(path_bytes * m / (step_ms / 1e3) / 1e9 / peak, 4),
                     "bytes_per_query": round(path_bytes, 1)}

    out = None
    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline(X_np, Q_np, T_use, v, k, l)
        detail = {"sweep": sweep, "roofline_other_kernels": others, "tuned_knobs": knobs,
                  "bf16_exact": bf16_exact}
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                json.dump(detail, f)
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32", "bf16 rows, f32 accumulate" + ("" if rerank else " (lossless copy: no re-rank)"),
                      "e4m3 rows + per-row scale, f32 accumulate + f32 re-rank")[prec],
            "data": "synthetic",
            "config": {"workload": W["name"], "n": n, "d": d, "queries_per_step": m, "k": k,
                       "depth": l, "T": T_use, "v": v, "density": "1/sqrt(d)",
                       "precision": ("fp32", "bf16", "fp8")[prec], "rerank_margin": margin,
                       "knobs": {kk: knobs.get(kk) for kk in ("path", "chunk", "ring")},
                       "fp32_best": None if best32 is None else
                       {kk: best32[kk] for kk in ("T", "v", "ms", "recall")},
                       "recall_at_10": round(recall_ta, 4),
                       "recall_at_10_strict": round(recall_strict, 4),
                       "mean_candidates": round(mean_S, 1), "build_s_T200": round(build_s, 3),
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}",
                       "path": "fused" if args.path == 1 else "vote-emit + candidate-search"},
            "e2e": e2e,
            "gpu_launches": (2 if args.path == 1 else 3) * args.steps,
            "roofline": roofline,
            "path_roofline": path_roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "stage_ms": {"route": round(statistics.mean(route_ms), 4),
                         "vote": round(vote_avg, 4), "search": round(search_avg, 4)},
        }
        emit_line(out)
    index.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def run_e2e(mr, index, Q, k, v, T_use, flush, args, world, torch, prec=0, margin=0, knobs=None):
    knobs = knobs or {}
    """The same metric through the public call with pinned host buffers:
    every step copies the queries in and the results out."""
    m, d = Q.shape
    Qh = Q.cpu().pin_memory().numpy()
    ids_h = torch.empty((m, k), dtype=torch.int32).pin_memory().numpy()
    dists_h = torch.empty((m, k), dtype=torch.float32).pin_memory().numpy()
    def call():
        mr.mrpt_query_ex(index, Qh, k, v, n_trees=T_use, out_ids=ids_h, out_dists=dists_h,
                         precision=prec, margin=margin, path=args.path, chunk=knobs.get("chunk", 0),
                         ring=knobs.get("ring", 0))
    call()
    el = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        el += time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([el], device=Q.device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    return {"value": round(world * m * args.steps / el, 1), "unit": "queries/s",
            "h2d_bytes_per_step": int(m * d * 4), "d2h_bytes_per_step": int(m * k * 8)}


def run_stream(args):
    """Uneven query stream on the 60k x 784 index: 100,000 queries in batches
    of floor(exp(U(0, ln 4097))) clamped to [1, 4096], k in {1, 10, 100} and
    v in {2, 5, 8} drawn per batch.  Every batch is one plan run (a CUDA
    graph); the same stream through plain mrpt_query_ex calls is timed too.
    Reports queries/s and p50/p99 batch latency (device events)."""
    import torch
    import paper_1509_06957_gb300 as mr
    W = WORKLOAD
    dev = torch.device("cuda", 0)
    X_np, Q_np = workloads.mnist_like(W["n"], W["m"], seed=W["seed"])
    X = torch.from_numpy(X_np).to(dev)
    Q = torch.from_numpy(Q_np).to(dev)
    T_use = args.T or 100
    index = mr.mrpt_build(X, T_use, W["l"], 0.0, seed=W["seed"])
    mr.mrpt_add_lowp(index)
    batches = workloads.uneven_batches(args.stream_queries, seed=1)
    mmax = max(b for b, _, _ in batches)
    out_ids = torch.empty((mmax, 100), dtype=torch.int32, device=dev)
    out_d = torch.empty((mmax, 100), dtype=torch.float32, device=dev)
    res = {}
    for prec in (0, 1):
        plans = {}
        for kk in (1, 10, 100):
            for vv in (2, 5, 8):
                plans[(kk, vv)] = mr.Plan(index, mmax, kk, vv, precision=prec)
        for mode in ("graph", "calls"):
            def one(bi, b, kk, vv):
                s0 = (bi * 977) % (Q.shape[0] - b + 1)
                q = Q[s0:s0 + b]
                oi = out_ids[:b, :kk]
                od = out_d[:b, :kk]
                if mode == "graph":
                    plans[(kk, vv)].run(q, oi.contiguous(), od.contiguous())
                else:
                    mr.mrpt_query_ex(index, q, kk, vv, precision=prec)
            for bi, (b, kk, vv) in enumerate(batches[:20]):
                one(bi, b, kk, vv)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in batches]
            t0 = time.perf_counter()
            for bi, (b, kk, vv) in enumerate(batches):
                evs[bi][0].record()
                one(bi, b, kk, vv)
                evs[bi][1].record()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            lat = np.array([a.elapsed_time(z) for a, z in evs])
            res[f"{'bf16' if prec else 'fp32'}_{mode}"] = {
                "queries_per_s": round(args.stream_queries / wall, 1),
                "p50_batch_ms": round(float(np.percentile(lat, 50)), 4),
                "p99_batch_ms": round(float(np.percentile(lat, 99)), 4),
                "mean_batch_ms": round(float(lat.mean()), 4)}
        for p_ in plans.values():
            p_.close()
    best = max(res.values(), key=lambda r: r["queries_per_s"])
    out = {"metric": "queries/sec on an uneven batch stream (mnist-like 60000x784 index, batches 1..4096)",
           "value": best["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic",
           "config": {"workload": "uneven stream: 100k queries, batch sizes log-uniform 1..4096, "
                                  "k in {1,10,100}, v in {2,5,8}", "T": T_use, "depth": W["l"],
                      "batches": len(batches)},
           "modes": res}
    print(json.dumps(out), flush=True)
    index.close()
    return out


def run_build(args):
    """Index build time (Algorithms 1-2) for the 1M-point shapes, data
    already on the device: 1M x 128 (T = 100, l = 12) and 1M x 960
    (T = 200, l = 10).  Each build is timed around the synchronous
    mrpt_build call (host-visible wall time, device-resident input)."""
    import torch
    import paper_1509_06957_gb300 as mr
    dev = torch.device("cuda", 0)
    rows = []
    shapes = [("lognormal-int 1000000x128", workloads.lognormal_int, 128, 100, 12),
              ("latent-factor 1000000x960", workloads.latent_factor, 960, 200, 10)]
    for name, gen, d, T, l in shapes[: args.build_shapes]:
        X_np, _ = gen(1_000_000, d, 1, seed=0)
        X = torch.from_numpy(X_np).to(dev)
        del X_np
        times = []
        for rep in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            idx = mr.mrpt_build(X, T, l, 0.0, seed=rep)
            el = time.perf_counter() - t0
            idx.close()
            if rep >= args.warmup:
                times.append(el)
        flops = 2.0 * 1_000_000 * T * l * (d ** 0.5)   # projections: a d nonzeros per vector
        rows.append({"workload": name, "T": T, "depth": l, "build_s_median": round(float(np.median(times)), 4),
                     "build_s_min": round(min(times), 4), "projection_gflop": round(flops / 1e9, 1)})
        del X
        torch.cuda.empty_cache()
    out = {"metric": "index build seconds (all trees, data on the device)", "value": rows[-1]["build_s_median"],
           "unit": "s", "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "builds": rows}
    print(json.dumps(out), flush=True)
    return out


def lowp_copy(X, prec, torch):
    """Host-side float64 values of the library's reduced-precision copy of X
    (mrpt_add_lowp): bfloat16 round-to-nearest-even, or e4m3 of
    x / (max|x| / 448) per row times that scale."""
    if prec == 1:
        return X.bfloat16().double()
    mx = X.abs().amax(1, keepdim=True)
    scale = torch.where(mx > 0, mx / 448.0, torch.ones_like(mx))
    q = (X * (1.0 / scale)).clamp(-448.0, 448.0).to(torch.float8_e4m3fn)
    return q.double() * scale.double()


def lowp_distance_error(X, Xl, Q, ids, torch):
    """Relative error of the squared distances computed from the reduced
    copy Xl (in float64, so only its rounding counts) against the exact
    float64 squared distances, over the returned neighbours (ids >= 0):
    (max, mean)."""
    errs = []
    for s0 in range(0, Q.shape[0], 256):
        a = ids[s0:s0 + 256].long()
        ok = a >= 0
        a = a.clamp(min=0)
        q = Q[s0:s0 + 256].double()[:, None, :]
        d64 = ((X[a].double() - q) ** 2).sum(2)
        dl = ((Xl[a] - q) ** 2).sum(2)
        good = ok & (d64 > 0)
        errs.append(((dl - d64).abs() / d64.clamp(min=1e-300))[good])
    e = torch.cat(errs)
    return (float(e.max()), float(e.mean())) if e.numel() else (0.0, 0.0)


def run_large(args):
    """--workload large: the v sweep per precision on the synthetic stand-ins.
    - mnist-like 60,000 x 784 (integers 0..255, exact in bfloat16),
      10,000 queries, k = 10, T = 100, l = 8;
    - 1M x 128 heavy-tailed integers (lognormal-int), 10,000 queries,
      k = 100, T = 100, l = 12;
    - 1M x 960 rank-64 factors (latent-factor), 1,000 queries, k = 10,
      T = 200, l = 10.
    Precisions: float32, bfloat16 and e4m3 rows, each with a float32 re-rank
    of the k + 32 nearest (skipped for a lossless bfloat16 copy).  Each point
    reports tie-aware recall@k against a float64 brute force, the recall loss
    against float32 at the same v, the relative error of the reduced copy's
    squared distances against float64 at the returned neighbours (max, mean),
    queries/s of device time (L2 flushed before the timed pass), the
    candidate search's time, the mean |S| and the search's algorithmic bytes
    per second (rows in the precision used, lists, queries, outputs and
    re-rank rows)."""
    import torch
    import paper_1509_06957_gb300 as mr
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stage = np.zeros(4, np.float32)
    confs = [("mnist-like 60000x784, 10000 queries", lambda n, d, m, seed: workloads.mnist_like(n, m, seed=seed),
              60000, 784, 10000, 10, 100, 8),
             ("lognormal-int 1000000x128, 10000 queries", workloads.lognormal_int, 1_000_000, 128, 10000, 100, 100, 12),
             ("latent-factor 1000000x960, 1000 queries", workloads.latent_factor, 1_000_000, 960, 1000, 10, 200, 10)]
    precs = [(0, 0), (1, 32), (2, 32)]
    out = {"metric": "queries/s, tie-aware recall@k and reduced-precision distance error per v (device time)",
           "data": "synthetic", "configs": []}
    for name, gen, n, d, m, k, T, l in confs[: args.large_configs]:
        X_np, Q_np = gen(n, d, m, seed=0)
        X, Q = torch.from_numpy(X_np).to(dev), torch.from_numpy(Q_np).to(dev)
        del X_np, Q_np
        gt_ids, _ = exact_knn_gpu(X, Q, k, torch)
        kth = torch.cat([((X[gt_ids[s:s + 64, k - 1].long()].double() - Q[s:s + 64].double()) ** 2).sum(1).sqrt()
                         for s in range(0, m, 64)]).float()[:, None]
        index = mr.mrpt_build(X, T, l, 0.0, seed=0)
        mr.mrpt_add_lowp(index, mr.MRPT_PREC_BF16)
        mr.mrpt_add_lowp(index, mr.MRPT_PREC_FP8)
        bf16_exact = bool(torch.equal(X, X.bfloat16().float()))
        lows = {1: lowp_copy(X, 1, torch), 2: lowp_copy(X, 2, torch)}
        rows = []
        for v in range(1, 11):
            rec32 = None
            ncand = torch.empty(m, dtype=torch.int64, device=dev)
            mr.mrpt_query_ex(index, Q, k, v, n_cand_out=ncand)
            mean_S = float(ncand.double().mean())
            for prec, margin in precs:
                mr.mrpt_query_ex(index, Q, k, v, precision=prec, margin=margin)  # warm
                flush.zero_()
                ids, dists = mr.mrpt_query_ex(index, Q, k, v, precision=prec, margin=margin, stage_ms=stage)
                rec = float(((dists <= kth * (1 + 1e-5)) & torch.isfinite(dists)).sum()) / (m * k)
                # the search's algorithmic bytes per query: candidate rows
                # (+ e4m3 scale chunk), list, query, output, re-rank rows
                reranked = prec == 2 or (prec == 1 and not bf16_exact)
                sbytes = (mean_S * (d * (4, 2, 1)[prec] + (16 if prec == 2 else 0) + 4) + d * 4 + k * 8
                          + (min(k + margin, mean_S) * d * 4 if reranked else 0))
                row = dict(v=v, precision=("fp32", "bf16", "fp8")[prec], margin=margin,
                           recall=round(rec, 4), qps=round(m / (float(stage[3]) / 1e3), 1),
                           ms=round(float(stage[3]), 3), search_ms=round(float(stage[2]), 3),
                           mean_S=round(mean_S, 1),
                           search_gbs=round(sbytes * m / (float(stage[2]) / 1e3) / 1e9, 1))
                if prec == 0:
                    rec32 = rec
                else:
                    emax, emean = lowp_distance_error(X, lows[prec], Q, ids, torch)
                    row.update(recall_loss_vs_fp32=round(rec32 - rec, 4), dist2_rel_err_max=float(f"{emax:.3g}"),
                               dist2_rel_err_mean=float(f"{emean:.3g}"),
                               rerank=not (prec == 1 and bf16_exact))
                rows.append(row)
        index.close()
        out["configs"].append({"workload": name, "T": T, "depth": l, "k": k, "bf16_exact": bf16_exact,
                               "rows": rows})
        del X, Q, lows
        torch.cuda.empty_cache()
    if args.detail_out:
        with open(args.detail_out, "w") as f:
            json.dump(out, f)
    print(json.dumps(out), flush=True)
    return out


# ------------------------------------------------------- CPU (oracle) -----

def _oracle_index(X, T, l, seed):
    """The oracle's own index (Algorithm 1), trees grown on a thread pool."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    d = X.shape[1]
    dens = float(np.float32(1.0 / np.sqrt(d)))
    R = oracle.random_matrix(T, l, d, dens, seed)
    P = oracle.project_threads(X, R) if hasattr(oracle, "project_threads") else oracle.project(X, R)
    L = 1 << l
    split = np.zeros((T, L - 1), np.float32)
    leaf_off = np.zeros((T, L + 1), np.int32)
    leaf_ids = np.zeros((T, X.shape[0]), np.int32)

    def one(t):
        s, o, i = oracle.grow_tree(P, t * l, l)
        split[t], leaf_off[t], leaf_ids[t] = s, o, i

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        list(ex.map(one, range(T)))
    return oracle.Index(X, T, l, R, P, split, leaf_off, leaf_ids)


def _time_oracle(ref, Q, k, v, threads, target_s):
    """Queries/s of the oracle's query path (float32 distances) with
    `threads` threads on the first queries of Q, repeated (bounded) until
    about target_s of work has been timed.  Returns (qps, sample text)."""
    import oracle
    probe = Q[: max(threads, 8)]
    t0 = time.perf_counter()
    oracle.query(ref, probe, k, v, mode=1, nthreads=threads)
    per_q = (time.perf_counter() - t0) / len(probe)
    ns = int(min(len(Q), max(len(probe), target_s / max(per_q, 1e-6))))
    sample = Q[:ns]
    el, done, reps = 0.0, 0, 0
    while el < target_s and reps < 4096:
        t0 = time.perf_counter()
        oracle.query(ref, sample, k, v, mode=1, nthreads=threads)
        el += time.perf_counter() - t0
        done += ns
        reps += 1
    return done / el, f"first {ns} of the {len(Q)} queries x{reps}, {el:.1f} s"


def cpu_baseline(X, Q, T, v, k, l, target_s=15.0, single_s=5.0):
    """The oracle's query path (float32 distances) on a bounded sample of
    the queries: OpenMP over queries on all host cores, and single-threaded."""
    import oracle
    ref = _oracle_index(X, T, l, WORKLOAD["seed"])
    threads = oracle.max_threads()
    qps, sample = _time_oracle(ref, Q, k, v, threads, target_s)
    qps1, sample1 = _time_oracle(ref, Q, k, v, 1, single_s)
    return {"value": round(qps, 2), "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{sample}, T={T}, v={v}, float32 distances",
            "single_thread": {"value": round(qps1, 2), "cores": 1, "sample": sample1}}


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload, metric and
    operating point, each step a bounded sample of the queries."""
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    W = WORKLOAD
    X, Q = workloads.mnist_like(W["n"], W["m"], seed=W["seed"])
    T, v = args.ref_T, args.ref_v
    ref = _oracle_index(X, T, W["l"], W["seed"])
    threads = oracle.max_threads()
    probe = Q[:threads]
    t0 = time.perf_counter()
    oracle.query(ref, probe, W["k"], v, mode=1, nthreads=threads)
    per_q = (time.perf_counter() - t0) / len(probe)
    budget = args.ref_budget_s / max(1, args.steps + args.warmup)
    ns = int(min(len(Q), max(threads, budget / max(per_q, 1e-6))))
    for i in range(args.warmup):
        oracle.query(ref, Q[:ns], W["k"], v, mode=1, nthreads=threads)
    el = 0.0
    for i in range(args.steps):
        s = (i * ns) % len(Q)
        sample = np.ascontiguousarray(np.roll(Q, -s, axis=0)[:ns])
        t0 = time.perf_counter()
        oracle.query(ref, sample, W["k"], v, mode=1, nthreads=threads)
        el += time.perf_counter() - t0
    qps = ns * args.steps / el
    out = {"metric": METRIC, "value": round(qps, 2), "unit": "queries/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": W["name"], "n": W["n"], "d": W["d"], "k": W["k"],
                      "depth": W["l"], "T": T, "v": v, "queries_per_step": ns},
           "cpu_baseline": {"value": round(qps, 2), "unit": "queries/s", "cores": threads,
                            "kind": "oracle",
                            "sample": f"{ns} queries per step of the {len(Q)}"},
           "e2e": {"value": round(qps, 2), "unit": "queries/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    emit_line(out)
    return out


# ----------------------------------------------------- Pareto / ablation --

def _front(points):
    """Non-dominated (recall up, queries/s up) points, by recall."""
    front = []
    for p in sorted(points, key=lambda p: (-p["qps"], -p["recall"])):
        if not front or p["recall"] > front[-1]["recall"]:
            front.append(p)
    return sorted(front, key=lambda p: p["recall"])


def run_pareto(args):
    """--workload pareto: the paper's parameter search (Sec. IV-B: grid over
    T, depth and v with a = 1/sqrt(d)) as Pareto fronts of queries/s against
    recall@k for k in {1, 10, 100}, for MRPT and the ablations of Table III:
    fixed-count sparse vectors (exactly ceil(a d) nonzeros, the Sec. II-D
    footnote), sparse trees without voting (v = 1), and classic dense RP
    trees (a = 1, v = 1).  Also MRPT on the "Random" set (unit-length
    N(0, I), 50,000 x 4096, Sec. IV-A).  Time is the library's device time of
    one query pass (L2 flushed before it); recall is tie-aware."""
    import torch
    import paper_1509_06957_gb300 as mr

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stage = np.zeros(4, np.float32)
    T_grid = (10, 25, 50, 100, 200)

    def sweep(X, Q, variants, depths, ks):
        m = Q.shape[0]
        kmax = max(ks)
        gt_ids, _ = exact_knn_gpu(X, Q, kmax, torch)
        gt_d = torch.cat([((X[gt_ids[s:s + 256].long()].double() - Q[s:s + 256].double()[:, None, :]) ** 2)
                          .sum(2).sqrt() for s in range(0, m, 256)])
        n = X.shape[0]
        out = {}
        for name, density, sparsity, v_grid in variants:
            pts = {k: [] for k in ks}
            for l in depths:
                index = mr.mrpt_build(X, max(T_grid), l, density, seed=0, sparsity=sparsity)
                leaf = -(-n // (1 << l))
                for T_use in T_grid:
                    for v in v_grid:
                        # |S| <= T ceil(n / 2^l) / v; settings with more than
                        # 40,000 candidates per query are left out (seconds per pass)
                        if v > T_use or T_use * leaf / v > 40000:
                            continue
                        for k in ks:
                            mr.mrpt_query_ex(index, Q, k, v, n_trees=T_use)  # warm
                            flush.zero_()
                            _, dists = mr.mrpt_query_ex(index, Q, k, v, n_trees=T_use, stage_ms=stage)
                            kth = gt_d[:, k - 1:k].float()
                            rec = float(((dists <= kth * (1 + 1e-5)) & torch.isfinite(dists)).sum()) / (m * k)
                            pts[k].append(dict(T=T_use, l=l, v=v, recall=round(rec, 4),
                                               qps=round(m / (float(stage[3]) / 1e3), 1)))
                index.close()
            out[name] = {}
            for k in ks:
                ok = [p for p in pts[k] if p["recall"] >= 0.9]
                out[name][f"k={k}"] = {"best_at_recall_0.9": max(ok, key=lambda p: p["qps"]) if ok else None,
                                       "front": _front(pts[k])}
        return out

    result = {"metric": "Pareto fronts: queries/s vs tie-aware recall@k (device time, L2 flushed)",
              "T_grid": T_grid, "data": "synthetic"}
    X_np, Q_np = workloads.mnist_like(60000, 10000, seed=0)
    X, Q = torch.from_numpy(X_np).to(dev), torch.from_numpy(Q_np).to(dev)
    variants = [("MRPT (a = 1/sqrt(d), voting)", 0.0, 0, range(1, 11)),
                ("MRPT, exactly ceil(a d) nonzeros per vector", 0.0, 1, range(1, 11)),
                ("sparse RP trees, no voting (v = 1)", 0.0, 0, (1,)),
                ("dense RP trees (a = 1), no voting (v = 1)", 1.0, 0, (1,))]
    result["mnist-like 60000x784, 10000 queries"] = sweep(X, Q, variants, (6, 7, 8, 9), (1, 10, 100))
    del X, Q
    X_np, Q_np = workloads.unit_gaussian(50000, 4096, 1000, seed=0)
    X, Q = torch.from_numpy(X_np).to(dev), torch.from_numpy(Q_np).to(dev)
    result["Random: unit-length N(0, I) 50000x4096, 1000 queries"] = sweep(
        X, Q, [("MRPT (a = 1/sqrt(d), voting)", 0.0, 0, range(1, 11))], (6, 8, 10), (10,))
    print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--build-shapes", type=int, default=2, help="build workload: how many shapes")
    ap.add_argument("--workload", choices=["batch", "stream", "build", "pareto", "large"], default="batch",
                    help="batch: the 10,000-query benchmark; stream: uneven batches through plans")
    ap.add_argument("--stream-queries", type=int, default=100000)
    ap.add_argument("--large-configs", type=int, default=3, help="large workload: how many configurations")
    ap.add_argument("--precision", choices=["auto", "fp32", "bf16", "fp8"], default="auto",
                    help="candidate-distance precision (auto: the faster at the recall target)")
    ap.add_argument("--path", type=int, default=0, choices=[0, 1],
                    help="0: vote/emit + candidate search kernels, 1: one fused kernel")
    ap.add_argument("--T", type=int, default=0, help="fix the number of trees (with --v)")
    ap.add_argument("--v", type=int, default=0, help="fix the vote threshold (with --T)")
    ap.add_argument("--ref-T", type=int, default=100, help="reference arm: trees (the GPU arm's operating point)")
    ap.add_argument("--ref-v", type=int, default=10, help="reference arm: vote threshold (the GPU arm's operating point)")
    ap.add_argument("--ref-budget-s", type=float, default=120.0,
                    help="reference arm: seconds of oracle work over all warm-up and timed steps")
    ap.add_argument("--detail-out", default="",
                    help="write the (T, v, precision) sweep and per-kernel rooflines to this JSON file")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "stream":
        run_stream(args)
    elif args.workload == "build":
        run_build(args)
    elif args.workload == "pareto":
        run_pareto(args)
    elif args.workload == "large":
        run_large(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
