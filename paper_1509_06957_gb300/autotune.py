"""Autotuning of query parameters to a recall target.

The paper tunes T, l and v by grid search with the sparsity a = 1/sqrt(d)
fixed and reports the fastest setting at each recall level (Sec. IV-B).
Here, on a built index and a sample of queries:

1. :func:`tune` sweeps the number of trees used (prefixes of the index --
   trees are prefix-stable), the vote threshold v and the candidate-distance
   precision (float32; bfloat16 / e4m3 with re-rank margins) and returns the
   fastest setting whose recall@k reaches the target, together with the
   Pareto front of (recall, device time).
2. :func:`tune_kernels` then sweeps the launch knobs of that setting (work
   items per candidate list, staged rows per warp, one- or two-kernel path).

Recall is |A n K| / k (Sec. I-A) with ties counted: a returned point counts
when its distance is at most the true k-th distance.  The true neighbours
come from the library itself: an index with T = 1 and l = 0 has one leaf
holding every point, so with v = 1 its answer is exact k-NN.

Results can be cached in a JSON file keyed by the index shape, k and the
target.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import (MRPT_PREC_BF16, MRPT_PREC_FP8, MRPT_PREC_FP32, mrpt_build, mrpt_query_ex)


def exact_knn(X, Q, k):
    """Exact k-NN of the rows of Q among the rows of X (torch CUDA tensors)
    through a one-leaf index (T = 1, l = 0, v = 1)."""
    one = mrpt_build(X, 1, 0, 1.0, 0)
    try:
        ids, dists = mrpt_query_ex(one, Q, k, 1, path=1)
    finally:
        one.close()
    return ids, dists


def recall(dists, true_dists, rel=1e-5) -> float:
    """Tie-aware recall@k from returned and true distance rows."""
    import torch
    kth = true_dists[:, -1:].clamp(min=0)
    ok = torch.isfinite(dists) & (dists <= kth * (1 + rel) + 1e-30)
    return float(ok.sum().item()) / float(true_dists.numel())


def _time(index, Q, k, v, reps, **opts):
    st = np.zeros(4, np.float32)
    mrpt_query_ex(index, Q, k, v, **opts)  # warm
    ts = []
    for _ in range(reps):
        ids, d = mrpt_query_ex(index, Q, k, v, stage_ms=st, **opts)
        ts.append(float(st[3]))
    return float(np.median(ts)), ids, d


def pareto(points):
    """Non-dominated (recall up, time down) subset of dicts with keys
    'recall' and 'ms', sorted by recall."""
    front = []
    for p in sorted(points, key=lambda p: (p["ms"], -p["recall"])):
        if not front or p["recall"] > front[-1]["recall"]:
            front.append(p)
    return sorted(front, key=lambda p: p["recall"])


def tune(index, X, Q, k, target=0.9, tree_grid=None, v_grid=range(1, 11),
         precisions=((MRPT_PREC_FP32, 0), (MRPT_PREC_BF16, 0), (MRPT_PREC_FP8, 32)),
         reps=3, cache_path=None):
    """Fastest (n_trees, v, precision, margin) reaching `target` recall@k on
    the query sample Q (torch CUDA tensor; the index's data X, same device).
    Reduced precisions need the index's copies (mrpt_add_lowp); those
    missing are skipped.  Returns dict(best=..., pareto=[...], table=[...])."""
    key = f"n{index.n}_d{index.d}_T{index.T}_l{index.l}_k{k}_r{target}"
    if cache_path and os.path.exists(cache_path):
        cached = json.load(open(cache_path)).get(key)
        if cached:
            return cached
    _, true_d = exact_knn(X, Q, k)
    trees = tree_grid or sorted({max(1, index.T // 4), max(1, index.T // 2), index.T})
    table = []
    for T_use in trees:
        for v in v_grid:
            if v > T_use:
                continue
            for prec, margin in precisions:
                try:
                    ms, _, d = _time(index, Q, k, v, reps, n_trees=T_use, precision=prec,
                                     margin=margin)
                except Exception:  # precision copy not present
                    continue
                table.append(dict(n_trees=T_use, v=v, precision=prec, margin=margin, ms=ms,
                                  recall=recall(d, true_d)))
    ok = [r for r in table if r["recall"] >= target]
    best = min(ok, key=lambda r: r["ms"]) if ok else max(table, key=lambda r: r["recall"])
    out = dict(best=best, pareto=pareto(table), table=table, target=target, reached=bool(ok))
    if cache_path:
        db = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        db[key] = out
        json.dump(db, open(cache_path, "w"), indent=1)
    return out


def tune_kernels(index, Q, k, v, n_trees=0, precision=MRPT_PREC_FP32, margin=0,
                 chunks=(32, 64, 128), rings=(2, 3, 4), reps=5):
    """Fastest launch knobs for one setting: (path, chunk, ring) by median
    device time over `reps` runs.  Returns dict(best=..., table=[...])."""
    table = []
    paths = (0, 1) if precision == MRPT_PREC_FP32 else (0,)
    for path in paths:
        knob_sets = [(c, r) for c in chunks for r in rings] if path == 0 else [(0, 0)]
        for chunk, ring in knob_sets:
            ms, _, _ = _time(index, Q, k, v, reps, n_trees=n_trees, precision=precision,
                             margin=margin, path=path, chunk=chunk, ring=ring)
            table.append(dict(path=path, chunk=chunk, ring=ring, ms=ms))
    return dict(best=min(table, key=lambda r: r["ms"]), table=table)
