"""Algorithm 2 with several hash tables and a single probe per table.
TEST INFRASTRUCTURE ONLY.

The index of ``oracle.nrlsh`` holds L = T * L_t sign-random-projection bits per
item (Eq. 4 on the Eq. 8 transform of each sub-dataset, Algorithm 1).  Read as T
hash tables, table t uses bits [t L_t, (t + 1) L_t) of the code.  A single probe
of table t visits the bucket whose code equals the query's code in that table.
For every sub-dataset S_j, Algorithm 2 searches the index I_j: its probed items are

    C_j(q) = { x in S_j : code_t(x) = code_t(q) for some table t },

and the answer is the best item over all the C_j(q).  With top-k instead of the
single best item, the result is the k largest q^T x over C(q) = union of the
C_j(q) (FP64 sequential scores, ties by smaller id, exactly as in the
multi-probe query).  The probed-item count is |C(q)|.
"""
from __future__ import annotations

import numpy as np

from . import nrlsh as O


def table_fields(codes: np.ndarray, T: int, L: int) -> np.ndarray:
    """(n, T) array: the L/T-bit code of every item in every table."""
    if T < 1 or L % T:
        raise ValueError("need T >= 1 dividing L")
    Lt = L // T
    mask = np.uint64((1 << Lt) - 1) if Lt < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    codes = np.asarray(codes, dtype=np.uint64)
    return np.stack([(codes >> np.uint64(t * Lt)) & mask for t in range(T)], axis=1)


def candidates(idx: "O.Index", cq: int, T: int) -> np.ndarray:
    """C(q) in storage order (sub-dataset, then id): items that share the query's
    bucket in at least one of the T tables."""
    fx = table_fields(idx.codes, T, idx.L)
    fq = table_fields(np.array([cq], dtype=np.uint64), T, idx.L)[0]
    hit = (fx == fq[None, :]).any(axis=1)
    ids = np.flatnonzero(hit)
    return ids[np.lexsort((ids, idx.sub[ids]))].astype(np.int64)


def per_subdataset_best(idx: "O.Index", q: np.ndarray, cq: int, T: int):
    """Algorithm 2 literally: x*_j per sub-dataset (None where C_j(q) is empty)."""
    cand = candidates(idx, cq, T)
    q = np.asarray(q, dtype=np.float64)
    best = []
    for j in range(idx.m):
        cj = cand[idx.sub[cand] == j]
        if cj.size == 0:
            best.append(None)
            continue
        sc = O.scores_fp64(idx.X[cj], q)
        ids, _ = O.topk(cj, sc, 1)
        best.append(int(ids[0]))
    return best


def query(idx: "O.Index", Q, k: int, T: int, cap: int = 0):
    """Top-k over C(q) for every query; with cap > 0 only the first cap items of
    C(q) in storage order are scored.  Returns (ids, scores, probed) with probed
    = |C(q)| before the cap."""
    Q = np.asarray(Q, dtype=np.float64)
    nq = Q.shape[0]
    cqs = O.query_codes(Q, idx.A)
    out_ids = np.full((nq, k), -1, dtype=np.int64)
    out_sc = np.full((nq, k), -np.inf, dtype=np.float32)
    probed = np.zeros(nq, dtype=np.int64)
    for i in range(nq):
        cand = candidates(idx, int(cqs[i]), T)
        probed[i] = cand.size
        if cap > 0:
            cand = cand[:cap]
        sc = O.scores_fp64(idx.X[cand], Q[i])
        out_ids[i], out_sc[i] = O.topk(cand, sc, k)
    return out_ids, out_sc, probed
