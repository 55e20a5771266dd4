"""Norm-ranging LSH, step by step in FP64.  TEST INFRASTRUCTURE ONLY.

Plain, slow and meant to be read against the paper.  Every floating-point value
that decides an integer (a code bit, a bucket order, a top-k order) is computed
in FP64 in a fixed order, which the CUDA library's last precision tier also
uses, so the two must agree bit for bit:

* s_x = ||x||^2: the exact sum of the x_k * x_k (each exact in FP64 for fp32/bf16
  items) rounded once to FP64, round-to-nearest-even.       (Algorithm 1)
* partition: rank items by (s_x, id) ascending (ties broken by id, one valid
  way to "break ties arbitrarily"); sub-dataset j holds ranks
  [floor(j n / m), floor((j+1) n / m)).  U_j^2 = max s_x over S_j.
                                                             (Algorithm 1)
  Or uniform norm ranges: j = min(m-1, floor(((nu - nu_min) / w) * m)) with
  nu = sqrt(s_x), w = nu_max - nu_min, all FP64 round-to-nearest; empty S_j
  have U_j^2 = 0.                                      (Section 5, Figure 3a)
* code bit b of item x in S_j: [v >= 0] with
      v = fl(A_b + fl(a_{d,b} * tau_x)),  A_b = sum_{k<d} a_{k,b} x_k  (in order),
      tau_x = fl(sqrt(fl(U_j^2 - s_x)))  (tau_x = 1 when U_j^2 = 0).
  This is sign(a^T P(x)) of Eq. 4 applied to the SIMPLE-LSH transform of Eq. 8
  with U = U_j, multiplied through by U_j > 0 (which leaves the sign unchanged),
  so no division is needed.                           (Eq. 8, Eq. 4, Algorithm 1)
* query bit b: [sum_{k<d} a_{k,b} q_k >= 0], i.e. P(q) = [q; 0] (Eq. 8).
* l(q, x) = number of identical hash bits = L - popcount(c_q xor c_x). (Section 3.3)
* bucket score s_hat(j, l) = fl(U_j * c_l), U_j = fl(sqrt(U_j^2)),
  c_l = cos(pi (1 - eps) (L - l) / L) correctly rounded to FP64.  Buckets are
  probed in descending s_hat, ties by larger l, then larger j.     (Eq. 12)
* candidates: the first min(B, n) items in the order (bucket rank, id).
* score = FP64 sum of q_k x_k in order k = 0..d-1; top-k by (score desc, id asc);
  the returned score is the score rounded to fp32.                 (Eq. 1)
"""
from __future__ import annotations

import dataclasses
import decimal
from fractions import Fraction
from typing import Optional

import numpy as np

from . import philox


# ---------------------------------------------------------------- index build

def sq_norms(X: np.ndarray) -> np.ndarray:
    """s_x = ||x||^2 correctly rounded to FP64 (Algorithm 1, "rank the items
    according to their 2-norms": s_x orders items exactly as ||x|| does).  Every
    x_k^2 of an fp32/bf16 value is exact in FP64; math.fsum returns their sum
    rounded once, so s_x does not depend on a summation order."""
    import math
    X = np.asarray(X, dtype=np.float64)
    sq = X * X
    return np.array([math.fsum(row) for row in sq.tolist()], dtype=np.float64)


def percentile_bounds(n: int, m: int) -> list:
    """Start ranks of the m sub-datasets plus n: S_j = ranks [floor(jn/m), floor((j+1)n/m))
    (Algorithm 1, partition by 2-norm percentiles)."""
    return [(j * n) // m for j in range(m + 1)]


def partition(s: np.ndarray, m: int):
    """Algorithm 1: rank by norm (ties by id), split into m percentile ranges and take
    U_j^2 = max_{x in S_j} ||x||^2.  Returns (sub_of_id, U2, bounds, rank_order)."""
    n = s.shape[0]
    if not 1 <= m <= n:
        raise ValueError("need 1 <= m <= n")
    ids = np.arange(n)
    order = np.lexsort((ids, s))             # primary key s ascending, then id
    bounds = percentile_bounds(n, m)
    sub = np.empty(n, dtype=np.int32)
    U2 = np.empty(m, dtype=np.float64)
    for j in range(m):
        members = order[bounds[j]:bounds[j + 1]]
        sub[members] = j
        U2[j] = s[members].max()
    return sub, U2, bounds, order


def partition_uniform(s: np.ndarray, m: int):
    """The alternative partition of Section 5 (Figure 3a): the domain of 2-norms
    [nu_min, nu_max], nu_x = sqrt(s_x), is cut into m equally wide ranges and
    S_j holds the items whose norm falls in range j:

        j(x) = min(m - 1, floor(((nu_x - nu_min) / w) * m)),  w = nu_max - nu_min,

    every operation in FP64, rounded to nearest, in this order (all items in
    S_0 when w = 0).  Ranges may be empty; an empty S_j has U_j^2 = 0.  Returns
    (sub_of_id, U2, bounds) with bounds the m+1 storage offsets of the
    sub-datasets in (sub-dataset, id) order."""
    n = s.shape[0]
    if not 1 <= m <= n:
        raise ValueError("need 1 <= m <= n")
    nu = np.sqrt(np.asarray(s, dtype=np.float64))
    lo, hi = nu.min(), nu.max()
    w = hi - lo
    if w > 0.0:
        t = ((nu - lo) / w) * np.float64(m)
        sub = np.minimum(np.floor(t), m - 1).astype(np.int32)
    else:
        sub = np.zeros(n, dtype=np.int32)
    U2 = np.zeros(m, dtype=np.float64)
    counts = np.zeros(m, dtype=np.int64)
    for j in range(m):
        members = np.flatnonzero(sub == j)
        counts[j] = members.size
        if members.size:
            U2[j] = s[members].max()
    bounds = [0] + np.cumsum(counts).tolist()
    return sub, U2, bounds


def tail_component(s: np.ndarray, sub: np.ndarray, U2: np.ndarray) -> np.ndarray:
    """tau_x = sqrt(U_j^2 - s_x): U_j times the last entry sqrt(1 - ||x/U_j||^2) of P(x)
    in Eq. 8.  A sub-dataset of zero vectors (U_j = 0) gets tau = 1, i.e. P(x) = [0; 1]."""
    U2x = U2[sub]
    tau = np.sqrt(U2x - s)
    tau[U2x == 0.0] = 1.0
    return tau


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack an (n, L) boolean array into uint64 codes, bit b at position b."""
    n, L = bits.shape
    weights = np.left_shift(np.uint64(1), np.arange(L, dtype=np.uint64))
    return (bits.astype(np.uint64) * weights[None, :]).sum(axis=1, dtype=np.uint64)


def projection_values(X: np.ndarray, A: np.ndarray, tau: Optional[np.ndarray]) -> np.ndarray:
    """v = a^T [x; tau] in FP64 with the fixed order of the module docstring
    (tau None: the query transform P(q) = [q; 0] of Eq. 8)."""
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[1]
    acc = np.zeros((X.shape[0], A.shape[1]), dtype=np.float64)
    for k in range(d):
        acc = acc + X[:, k:k + 1] * A[k][None, :]
    if tau is None:
        return acc
    return acc + A[d][None, :] * np.asarray(tau, dtype=np.float64)[:, None]


def item_codes(X, A, tau) -> np.ndarray:
    """Sign random projection (Eq. 4) of the transformed items (Eq. 8), packed."""
    return pack_bits(projection_values(X, A, tau) >= 0.0)


def query_codes(Q, A) -> np.ndarray:
    """Sign random projection of P(q) = [q; 0] (Eq. 8), packed."""
    return pack_bits(projection_values(Q, A, None) >= 0.0)


# ------------------------------------------------------- Eq. 12 bucket scores

_DEC_PREC = 80


def _dec_pi() -> decimal.Decimal:
    """pi by Machin's formula, pi = 16 atan(1/5) - 4 atan(1/239), in Decimal."""
    def atan_inv(x: int) -> decimal.Decimal:
        x2 = x * x
        term = decimal.Decimal(1) / x
        total = term
        k = 1
        while True:
            term = term / x2
            t = term / (2 * k + 1)
            if t == 0 or abs(t) < decimal.Decimal(10) ** (-(_DEC_PREC + 5)):
                break
            total = total - t if k % 2 else total + t
            k += 1
        return total
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def cos_class(L: int, l: int, eps: float) -> float:
    """c_l = cos(pi (1 - eps) (L - l) / L) correctly rounded to FP64 (Eq. 12 with the
    eps adjustment).  Taylor series in 80-digit Decimal; the angle is exactly pi/2
    only when 2 (1 - eps) (L - l) = L, and cos is then exactly 0 (Niven: 0, +-1/2 and
    +-1 are the only rational values, all representable, so no other case needs care)."""
    fe = Fraction(eps)
    if 2 * (1 - fe) * (L - l) == L:
        return 0.0
    with decimal.localcontext() as ctx:
        ctx.prec = _DEC_PREC
        theta = _dec_pi() * (1 - decimal.Decimal(eps)) * (L - l) / L
        x2 = theta * theta
        total = decimal.Decimal(1)
        term = decimal.Decimal(1)
        i = 1
        while True:
            term = -term * x2 / ((2 * i - 1) * (2 * i))
            total += term
            if abs(term) < decimal.Decimal(10) ** (-(_DEC_PREC - 2)):
                break
            i += 1
        return float(total)                 # Decimal -> float rounds to nearest


def class_table(U2: np.ndarray, L: int, eps: float):
    """The sorted (U_j, l) structure of Section 3.3: all m(L+1) buckets ordered by
    s_hat = U_j cos[pi (1 - eps)(1 - l/L)] descending, ties by larger l then larger j.
    Returns (list of (j, l) in probing order, s_hat array (m, L+1), c array (L+1))."""
    m = U2.shape[0]
    c = np.array([cos_class(L, l, eps) for l in range(L + 1)], dtype=np.float64)
    U = np.sqrt(U2)
    shat = np.empty((m, L + 1), dtype=np.float64)
    for j in range(m):
        for l in range(L + 1):
            shat[j, l] = float(U[j]) * float(c[l]) + 0.0   # + 0.0 turns -0 into +0
    keys = [(-shat[j, l], -l, -j, j, l) for j in range(m) for l in range(L + 1)]
    keys.sort()
    table = [(kk[3], kk[4]) for kk in keys]
    return table, shat, c


# ------------------------------------------------------------------ the index

@dataclasses.dataclass
class Index:
    n: int
    d: int
    m: int
    L: int
    eps: float
    A: np.ndarray            # (d+1, L)
    s: np.ndarray            # (n,) squared norms
    sub: np.ndarray          # (n,) sub-dataset of each id
    U2: np.ndarray           # (m,)
    bounds: list             # m+1 start ranks
    tau: np.ndarray          # (n,)
    codes: np.ndarray        # (n,) uint64, id order
    table: list              # [(j, l)] probing order
    shat: np.ndarray         # (m, L+1)
    class_rank: np.ndarray   # (m, L+1) position of (j, l) in the probing order
    X: np.ndarray            # (n, d) float64 copy of the items


def build(X, m: int, L: int, seed: int, eps: float = 0.1, A: Optional[np.ndarray] = None,
          partition_scheme: str = "percentile") -> Index:
    """Algorithm 1: partition by norm percentiles (or, with partition_scheme="uniform",
    by the uniform norm ranges of Section 5), normalise each S_j by its own U_j,
    and hash with SIMPLE-LSH (Eq. 8 + Eq. 4) into L-bit codes."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if not (1 <= L <= 64 and 0.0 < eps < 1.0):
        raise ValueError("need 1 <= L <= 64 and 0 < eps < 1")
    if A is None:
        A = philox.projections(seed, d, L)
    s = sq_norms(X)
    if partition_scheme == "percentile":
        sub, U2, bounds, _ = partition(s, m)
    elif partition_scheme == "uniform":
        sub, U2, bounds = partition_uniform(s, m)
    else:
        raise ValueError("partition_scheme is 'percentile' or 'uniform'")
    tau = tail_component(s, sub, U2)
    codes = item_codes(X, A, tau)
    table, shat, _ = class_table(U2, L, eps)
    class_rank = np.empty((m, L + 1), dtype=np.int64)
    for t, (j, l) in enumerate(table):
        class_rank[j, l] = t
    return Index(n, d, m, L, eps, A, s, sub, U2, bounds, tau, codes, table, shat,
                 class_rank, X)


def storage_order(idx: Index) -> np.ndarray:
    """Ids sorted by (sub-dataset, id): the order in which candidates are reported."""
    return np.lexsort((np.arange(idx.n), idx.sub))


# ---------------------------------------------------------------- query path

def matches(idx: Index, cq: int) -> np.ndarray:
    """l(q, x) for every item x (id order): identical bits among the L hash bits."""
    ham = np.bitwise_count(idx.codes ^ np.uint64(cq)).astype(np.int64)
    return idx.L - ham


def histogram(idx: Index, cq: int) -> np.ndarray:
    """H[j, l] = number of items of S_j with l identical bits (bucket sizes per class)."""
    H = np.zeros((idx.m, idx.L + 1), dtype=np.int64)
    np.add.at(H, (idx.sub, matches(idx, cq)), 1)
    return H


def threshold(idx: Index, H: np.ndarray, B: int, whole_class: bool = False):
    """Walk the probing order until B items are reached (Section 3.3).  Returns
    (lam, j_star, l_star, r, full): buckets before the boundary bucket (j*, l*) are
    probed whole, so S_j contributes the items with l >= lam[j]; r items of the
    boundary bucket complete the budget; full = items in the whole buckets."""
    Bp = min(int(B), idx.n)
    lam = [idx.L + 1] * idx.m
    cum = 0
    for (j, l) in idx.table:
        c = int(H[j, l])
        if cum + c >= Bp:
            r = c if whole_class else Bp - cum
            return lam, j, l, r, cum
        cum += c
        lam[j] = min(lam[j], l)
    raise AssertionError("histogram counts do not add up to n")


def candidates(idx: Index, cq: int, B: int, whole_class: bool = False) -> np.ndarray:
    """Probed items, by definition: the first min(B, n) items in the order
    (bucket rank, id), or with whole_class, every item of the buckets reached."""
    l = matches(idx, cq)
    rank = idx.class_rank[idx.sub, l]
    ids = np.arange(idx.n)
    order = np.lexsort((ids, rank))
    Bp = min(int(B), idx.n)
    if whole_class:
        last = rank[order[Bp - 1]]
        return order[rank[order] <= last]
    return order[:Bp]


def candidates_reported(idx: Index, cq: int, B: int, whole_class: bool = False) -> np.ndarray:
    """The candidate ids in the order the library reports them: items of whole buckets
    first, in storage order (sub-dataset, then id), then the boundary bucket's items
    by id."""
    cand = candidates(idx, cq, B, whole_class)
    l = matches(idx, cq)
    rank = idx.class_rank[idx.sub, l]
    last = rank[cand].max()
    full = cand[rank[cand] < last]
    bnd = cand[rank[cand] == last]
    full = full[np.lexsort((full, idx.sub[full]))]
    bnd = np.sort(bnd)
    return np.concatenate([full, bnd]).astype(np.int64)


def scores_fp64(X64: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Inner products q^T x, summed over k = 0..d-1 in order in FP64 (products exact)."""
    q = np.asarray(q, dtype=np.float64)
    acc = np.zeros(X64.shape[0], dtype=np.float64)
    for k in range(X64.shape[1]):
        acc = acc + X64[:, k] * q[k]
    return acc


def topk(ids: np.ndarray, scores: np.ndarray, k: int):
    """k largest scores, ties by smaller id; padded with (-1, -inf) if fewer than k."""
    order = np.lexsort((ids, -scores))[:k]
    out_ids = np.full(k, -1, dtype=np.int64)
    out_sc = np.full(k, -np.inf, dtype=np.float32)
    out_ids[:order.size] = ids[order]
    out_sc[:order.size] = scores[order].astype(np.float32)
    return out_ids, out_sc


def query(idx: Index, Q, k: int, B, whole_class: bool = False):
    """Section 3.3 multi-probe query + exact re-rank + top-k.  B may be a scalar or a
    per-query array; k likewise (output padded to max k).  Returns (ids, scores)."""
    Q = np.asarray(Q, dtype=np.float64)
    nq = Q.shape[0]
    Bs = np.broadcast_to(np.asarray(B, dtype=np.int64), (nq,))
    ks = np.broadcast_to(np.asarray(k, dtype=np.int64), (nq,))
    kmax = int(ks.max()) if nq else int(np.max(k))
    cq = query_codes(Q, idx.A)
    out_ids = np.full((nq, kmax), -1, dtype=np.int64)
    out_sc = np.full((nq, kmax), -np.inf, dtype=np.float32)
    for i in range(nq):
        cand = candidates(idx, int(cq[i]), int(Bs[i]), whole_class)
        sc = scores_fp64(idx.X[cand], Q[i])
        ii, ss = topk(cand.astype(np.int64), sc, int(ks[i]))
        out_ids[i, :ks[i]] = ii
        out_sc[i, :ks[i]] = ss
    return out_ids, out_sc
