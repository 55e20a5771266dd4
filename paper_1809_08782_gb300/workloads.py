"""Seeded synthetic workloads shaped like the paper's datasets (Section 5).

This module only draws inputs.  It holds none of the method's arithmetic, so the
CUDA path (through the binding) and the CPU oracle can both be fed from it.

The paper evaluates on Netflix and Yahoo!Music item embeddings (n = 17,770 and
n = 136,736, d = 300, user embeddings as queries) and on about 2.34M ImageNet
SIFT descriptors (Section 5).  None of those datasets is used here; the presets
below are synthetic stand-ins of the same sizes:

* directions: i.i.d. N(0,1) rows, normalised to unit length (FP64);
* norms: lognormal(0, sigma) or 1 + Pareto(alpha) (classical, x_m = 1), which gives
  the long-tailed 2-norm distributions that motivate the method (Section 3.1);
* items = direction * norm, rounded to the stored dtype (fp32 RN, or bf16 RNE
  from the fp32 value);
* queries: i.i.d. N(0,1) rows normalised to unit length, fp32.

Directions and norms come from two independent PCG64 streams, so generating the
rows chunk by chunk gives the same values as generating them at once.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

__all__ = [
    "Workload", "PRESETS", "make_workload", "gen_items", "gen_queries",
    "bf16_bits_from_f32", "bf16_bits_to_f64", "items_to_f64", "to_torch",
    "per_query_budgets_and_k",
]


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    d: int
    m: int
    L: int
    nq: int
    k: int
    budget: int               # default probe budget B (items)
    dtype: str                # "f32" or "bf16"
    norm_dist: str            # "lognormal" or "pareto"
    norm_param: float         # sigma or alpha
    item_seed: int
    query_seed: int
    index_seed: int
    budget_sweep: tuple = ()  # candidate budgets for a recall sweep
    items: Optional[np.ndarray] = None    # (n, d) float32, or uint16 bf16 bit patterns
    queries: Optional[np.ndarray] = None  # (nq, d) float32


# Presets.  Sizes follow the paper's three datasets and two larger forms;
# the seeds are fixed so every consumer sees the same inputs.
PRESETS = {
    # small plain case: n=10,000, d=64 fp32, lognormal(0,0.5), m=8, L=16, B=1,000
    "small-n10k-d64": dict(n=10_000, d=64, m=8, L=16, nq=1_000, k=10, budget=1_000,
                           dtype="f32", norm_dist="lognormal", norm_param=0.5, cfg=1),
    # Netflix-sized: n=17,770, d=300 fp32, lognormal(0,0.8), m=32, L=32
    "netflix-n17770-d300": dict(n=17_770, d=300, m=32, L=32, nq=1_000, k=10,
                                budget=3_554, dtype="f32", norm_dist="lognormal",
                                norm_param=0.8, cfg=2,
                                sweep_frac=(0.01, 0.015, 0.02, 0.03, 0.04, 0.05, 0.075, 0.10, 0.15, 0.20)),
    # Yahoo!Music-sized: n=136,736, d=300, lognormal(0,1.0), m=32, L=64
    "yahoo-n136736-d300": dict(n=136_736, d=300, m=32, L=64, nq=10_000, k=10,
                               budget=4_096, dtype="f32", norm_dist="lognormal",
                               norm_param=1.0, cfg=3),
    # ImageNet-SIFT-sized: n=2,340,373, d=150 bf16, Pareto(3) norms, m=64, L=64
    "imagenet-n2340373-d150": dict(n=2_340_373, d=150, m=64, L=64, nq=100_000, k=10,
                                   budget=65_536, dtype="bf16", norm_dist="pareto",
                                   norm_param=3.0, cfg=4),
    # resident serving index: n=10M, d=128 bf16, lognormal(0,1.0), m=64, L=64
    "serving-n10m-d128": dict(n=10_000_000, d=128, m=64, L=64, nq=10_000, k=10,
                              budget=10_000, dtype="bf16", norm_dist="lognormal",
                              norm_param=1.0, cfg=5),
}


def bf16_bits_from_f32(x32: np.ndarray) -> np.ndarray:
    """Round fp32 values to bfloat16 (round to nearest, ties to even); uint16 bits."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact float64 values of bfloat16 bit patterns."""
    u32 = bits.astype(np.uint32) << 16
    return u32.view(np.float32).astype(np.float64)


def items_to_f64(items: np.ndarray, dtype: str) -> np.ndarray:
    """Exact float64 copy of stored items (fp32 array or bf16 bit patterns)."""
    if dtype == "bf16":
        return bf16_bits_to_f64(items)
    return np.asarray(items, dtype=np.float32).astype(np.float64)


def _norms(rng: np.random.Generator, count: int, dist: str, param: float) -> np.ndarray:
    if dist == "lognormal":
        return rng.lognormal(mean=0.0, sigma=param, size=count)
    if dist == "pareto":
        return 1.0 + rng.pareto(param, size=count)
    raise ValueError(f"unknown norm distribution {dist!r}")


def gen_items(n: int, d: int, seed: int, dist: str, param: float, dtype: str = "f32",
              rows: Optional[slice] = None, chunk: int = 1 << 18) -> np.ndarray:
    """Items (n, d): Gaussian unit directions scaled by long-tailed norms.

    ``rows`` selects a contiguous row range without materialising the rest
    (the streams are consumed in row order, so row r is the same either way).
    """
    start, stop = (0, n) if rows is None else (rows.start or 0, rows.stop)
    dir_rng = np.random.Generator(np.random.PCG64([seed, 0]))
    nrm_rng = np.random.Generator(np.random.PCG64([seed, 1]))
    out = np.empty((stop - start, d), dtype=np.uint16 if dtype == "bf16" else np.float32)
    r = 0
    while r < stop:
        c = min(chunk, stop - r)
        dirs = dir_rng.standard_normal((c, d))
        nrm = _norms(nrm_rng, c, dist, param)
        lo, hi = max(r, start), min(r + c, stop)
        if hi > lo:
            sl = slice(lo - r, hi - r)
            dd = dirs[sl]
            dd /= np.sqrt(np.einsum("ij,ij->i", dd, dd))[:, None]
            x32 = (dd * nrm[sl][:, None]).astype(np.float32)
            out[lo - start:hi - start] = bf16_bits_from_f32(x32) if dtype == "bf16" else x32
        r += c
    return out


def gen_queries(nq: int, d: int, seed: int) -> np.ndarray:
    """Unit-norm Gaussian queries (nq, d), fp32."""
    rng = np.random.Generator(np.random.PCG64([seed, 2]))
    q = rng.standard_normal((nq, d))
    q /= np.sqrt(np.einsum("ij,ij->i", q, q))[:, None]
    return q.astype(np.float32)


def per_query_budgets_and_k(nq: int, n: int, lo_frac: float, hi_frac: float,
                            seed: int, ks=(1, 10, 100)):
    """Uneven per-query probe budgets, uniform in [lo_frac, hi_frac] * n, and k."""
    rng = np.random.Generator(np.random.PCG64([seed, 3]))
    b = np.rint(rng.uniform(lo_frac, hi_frac, size=nq) * n).astype(np.int64)
    b = np.maximum(b, 1)
    k = rng.choice(np.asarray(ks, dtype=np.int32), size=nq)
    return b, k


def make_workload(name: str, n: Optional[int] = None, nq: Optional[int] = None,
                  with_data: bool = True) -> Workload:
    """Build a preset (optionally shrunk in n or nq; the draw recipe is unchanged)."""
    p = dict(PRESETS[name])
    cfg = p.pop("cfg")
    sweep_frac = p.pop("sweep_frac", ())
    if n is not None:
        p["n"] = n
    if nq is not None:
        p["nq"] = nq
    w = Workload(name=name, item_seed=1000 + cfg, query_seed=2000 + cfg,
                 index_seed=3000 + cfg, **p)
    if sweep_frac:
        w.budget_sweep = tuple(max(1, int(round(f * w.n))) for f in sweep_frac)
    if with_data:
        w.items = gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
        w.queries = gen_queries(w.nq, w.d, w.query_seed)
    return w


def to_torch(arr: np.ndarray, dtype: str = "f32", device: str = "cpu"):
    """Items/queries as a torch tensor (fp32, or bf16 from uint16 bit patterns)."""
    import torch
    if dtype == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32))
    return t.to(device)
