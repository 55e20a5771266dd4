"""SIMPLE-LSH with one global normaliser (Eq. 8), written separately from
``oracle.nrlsh``.  TEST INFRASTRUCTURE ONLY.

It forms P(x) = [x / U; sqrt(1 - ||x / U||^2)] explicitly with U the largest
2-norm in the dataset, hashes with sign random projection (Eq. 4) and ranks items
by Hamming ranking (more identical bits first, ties by id), which is what
norm-ranging LSH reduces to with a single sub-dataset.
"""
from __future__ import annotations

import numpy as np


def transform_items(X: np.ndarray, U: float) -> np.ndarray:
    """P(x) = [x/U; sqrt(1 - ||x/U||^2)] (Eq. 8)."""
    Xs = np.asarray(X, dtype=np.float64) / U
    tail = np.sqrt(np.maximum(0.0, 1.0 - np.einsum("ij,ij->i", Xs, Xs)))
    return np.concatenate([Xs, tail[:, None]], axis=1)


def transform_queries(Q: np.ndarray) -> np.ndarray:
    """P(q) = [q; 0] (Eq. 8)."""
    Q = np.asarray(Q, dtype=np.float64)
    return np.concatenate([Q, np.zeros((Q.shape[0], 1))], axis=1)


def srp_bits(V: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Sign random projection h_a(v) = sign(a^T v) (Eq. 4); True for a^T v >= 0."""
    return (V @ A) >= 0.0


def candidates(X: np.ndarray, q: np.ndarray, A: np.ndarray, B: int) -> np.ndarray:
    """First min(B, n) items by Hamming ranking of the SIMPLE-LSH codes."""
    X = np.asarray(X, dtype=np.float64)
    U = float(np.sqrt(np.max(np.einsum("ij,ij->i", X, X))))
    bx = srp_bits(transform_items(X, U), A)
    bq = srp_bits(transform_queries(np.asarray(q, dtype=np.float64)[None, :]), A)[0]
    same = (bx == bq[None, :]).sum(axis=1)
    ids = np.arange(X.shape[0])
    order = np.lexsort((ids, -same))
    return order[:min(int(B), X.shape[0])]
