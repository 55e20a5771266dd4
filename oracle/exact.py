"""Exact maximum inner product search (Eq. 1) and recall.  TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def exact_scores(X: np.ndarray, q: np.ndarray) -> list:
    """q^T x for every item as an exact rational (fp32/bf16/fp64 inputs are exact)."""
    qf = [Fraction(float(v)) for v in np.asarray(q, dtype=np.float64)]
    out = []
    for row in np.asarray(X, dtype=np.float64):
        out.append(sum((Fraction(float(a)) * b for a, b in zip(row, qf)), Fraction(0)))
    return out


def exact_topk(X: np.ndarray, q: np.ndarray, k: int) -> np.ndarray:
    """Eq. 1 extended to top-k: the k items with the largest exact q^T x, ties by id."""
    sc = exact_scores(X, q)
    order = sorted(range(len(sc)), key=lambda i: (-sc[i], i))
    return np.array(order[:k], dtype=np.int64)


def brute_topk_fp64(X: np.ndarray, Q: np.ndarray, k: int) -> np.ndarray:
    """Top-k ids by FP64 matrix product (ties by id) for recall at larger sizes,
    where exact rationals are too slow; near-ties below 1e-12 are not resolved."""
    S = np.asarray(Q, dtype=np.float64) @ np.asarray(X, dtype=np.float64).T
    ids = np.arange(S.shape[1])
    out = np.empty((S.shape[0], k), dtype=np.int64)
    for i in range(S.shape[0]):
        out[i] = np.lexsort((ids, -S[i]))[:k]
    return out


def recall_at_k(found: np.ndarray, truth: np.ndarray) -> float:
    """Mean over queries of |found_i intersect truth_i| / k (the probed-item recall of
    Figure 2, measured on the returned top-k)."""
    found = np.asarray(found)
    truth = np.asarray(truth)
    k = truth.shape[1]
    hits = [len(set(found[i][found[i] >= 0].tolist()) & set(truth[i].tolist()))
            for i in range(truth.shape[0])]
    return float(np.mean(hits)) / k
