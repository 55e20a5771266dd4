"""Probed-item / recall curves (the protocol of Figure 2 and Figure 3 of the
paper) and bucket-balance statistics, run through the library.

* SIMPLE-LSH is norm-ranging LSH with one sub-dataset (m = 1): one global U.
* Codes are compared at equal total code length: as in Section 5, the
  ceil(log2 m) bits that address a sub-dataset count against RANGE-LSH's
  length, so it hashes L - ceil(log2 m) bits while SIMPLE-LSH hashes L.
* Buckets are probed whole (NRLSH_WHOLE_BUCKETS) at budgets 2^i, so the probed
  count can overshoot the budget exactly as the paper's x-values do; the
  x-value reported is the mean number of probed items per query.
* recall@10 = |returned top-10 and exact top-10| / 10, averaged over queries;
  the exact top-10 is the library's own result at B = n (the full re-rank,
  which the parity tests pin to exact MIPS).
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np
import torch

from . import nrlsh as N


def exact_topk(idx: "N.Index", Q: torch.Tensor, k: int = 10, chunk: int = 256) -> np.ndarray:
    out = []
    for i in range(0, Q.shape[0], chunk):
        ids, _ = N.nrlsh_query_ex(idx, Q[i:i + chunk], k, idx.n)
        out.append(ids.cpu().numpy())
    return np.concatenate(out)


def recall(found: np.ndarray, truth: np.ndarray) -> float:
    k = truth.shape[1]
    return float(np.mean([len(set(found[i][found[i] >= 0]) & set(truth[i]))
                          for i in range(len(truth))])) / k


def probed_counts(idx: "N.Index", Q: torch.Tensor, B: int, chunk: int = 64) -> np.ndarray:
    counts = []
    for i in range(0, Q.shape[0], chunk):
        _, c = N.nrlsh_query_candidates(idx, Q[i:i + chunk], B, flags=N.NRLSH_WHOLE_BUCKETS,
                                        cap=idx.n)
        counts.append(c.cpu().numpy())
    return np.concatenate(counts)


def curve(items: torch.Tensor, Q: torch.Tensor, truth: np.ndarray, m: int, L_hash: int, seed: int,
          eps: float, budgets: List[int], partition: int = None) -> List[Dict]:
    idx = N.nrlsh_build_ex(items, m, L_hash, seed, eps=eps, partition=partition)
    pts = []
    for B in budgets:
        ids, _ = N.nrlsh_query_ex(idx, Q, 10, B, flags=N.NRLSH_WHOLE_BUCKETS)
        pts.append({"budget": int(B), "probed": float(probed_counts(idx, Q, B).mean()),
                    "recall": recall(ids.cpu().numpy(), truth)})
        if pts[-1]["recall"] >= 0.999:
            break
    pts_stats = bucket_stats(idx)
    idx.free()
    return [{"points": pts, **pts_stats}]


def bucket_stats(idx: "N.Index") -> Dict:
    """Number of non-empty buckets (sub-dataset, code) and the largest bucket
    (the bucket-balance figures of Sections 3.1 and 3.2)."""
    codes = N.nrlsh_get_codes(idx).numpy().view(np.uint64)
    sub, _, _ = N.nrlsh_get_partition(idx)
    # (sub-dataset, code) pairs as rows: a code may use all 64 bits, so the pair
    # does not fit one 64-bit key
    pairs = np.stack([sub.numpy().astype(np.uint64), codes], axis=1)
    _, counts = np.unique(pairs, axis=0, return_counts=True)
    return {"buckets": int(counts.size), "largest_bucket": int(counts.max())}


def compare(items: torch.Tensor, Q: torch.Tensor, L: int, m: int, seed: int, eps: float,
            truth: np.ndarray = None) -> Dict:
    """RANGE-LSH (m sub-datasets, L - ceil(log2 m) hash bits) versus SIMPLE-LSH
    (m = 1, L hash bits) at total code length L."""
    n = items.shape[0]
    if truth is None:
        idx = N.nrlsh_build_ex(items, 1, 8, seed)
        truth = exact_topk(idx, Q)
        idx.free()
    budgets = [2 ** i for i in range(4, int(math.ceil(math.log2(n))) + 1)]
    L_range = L - int(math.ceil(math.log2(m)))
    return {"L": L, "m": m, "L_hash_range": L_range,
            "range_lsh": curve(items, Q, truth, m, L_range, seed, eps, budgets)[0],
            "simple_lsh": curve(items, Q, truth, 1, L, seed, eps, budgets)[0]}


def compare_partitions(items: torch.Tensor, Q: torch.Tensor, L: int, m: int, seed: int,
                       eps: float, truth: np.ndarray) -> Dict:
    """Percentile partitioning (Algorithm 1) versus uniform norm ranges (Section 5,
    Figure 3a), both RANGE-LSH with m sub-datasets at total code length L."""
    n = items.shape[0]
    budgets = [2 ** i for i in range(4, int(math.ceil(math.log2(n))) + 1)]
    L_range = L - int(math.ceil(math.log2(m)))
    return {"L": L, "m": m, "L_hash_range": L_range,
            "percentile": curve(items, Q, truth, m, L_range, seed, eps, budgets,
                                N.NRLSH_PARTITION_PERCENTILE)[0],
            "uniform": curve(items, Q, truth, m, L_range, seed, eps, budgets,
                             N.NRLSH_PARTITION_UNIFORM)[0]}


def multitable_curve(items: torch.Tensor, Q: torch.Tensor, truth: np.ndarray, m: int, L: int,
                     seed: int, eps: float, tables: List[int], partition: int = None) -> Dict:
    """Algorithm 2 with T single-probe tables of L/T bits each, for T in `tables`:
    mean probed items |C(q)|, recall@10 and device time per query."""
    idx = N.nrlsh_build_ex(items, m, L, seed, eps=eps, partition=partition)
    pts = []
    for T in tables:
        N.nrlsh_query_multitable(idx, Q[:8], T, 10)         # warm-up
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        ids, _, probed = N.nrlsh_query_multitable(idx, Q, T, 10)
        t1.record()
        torch.cuda.synchronize()
        pts.append({"tables": int(T), "bits_per_table": L // T,
                    "probed": float(probed.float().mean().item()),
                    "recall": recall(ids.cpu().numpy(), truth),
                    "us_per_query": t0.elapsed_time(t1) * 1e3 / Q.shape[0]})
    idx.free()
    return {"m": m, "L": L, "points": pts}


def probed_at_recall(points: List[Dict], target: float = 0.9):
    """First point (probed, recall) with recall >= target, like the paper's tables."""
    for p in points:
        if p["recall"] >= target:
            return p["probed"], p["recall"]
    return None, None
