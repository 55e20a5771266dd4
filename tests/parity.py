"""Shared helpers for the GPU-versus-oracle parity tests."""
import numpy as np
import torch

import paper_1809_08782_gb300.nrlsh as N
from oracle import nrlsh as O

DEV = "cuda:0"


def f32(x: float) -> float:
    """The float32 value the C ABI receives for eps."""
    return float(np.float32(x))


def to_dev_items(items: np.ndarray, dtype: str):
    if dtype == "bf16":
        return torch.from_numpy(np.ascontiguousarray(items).view(np.int16)).view(torch.bfloat16).to(DEV)
    return torch.from_numpy(np.ascontiguousarray(items, dtype=np.float32)).to(DEV)


def build_pair(items: np.ndarray, dtype: str, m: int, L: int, seed: int, eps: float,
               projection=None, partition: str = "percentile"):
    """(library index, oracle index) on the same inputs; projection forces the
    projection path (N.NRLSH_PROJECT_SIMT / N.NRLSH_PROJECT_TENSOR), partition
    selects percentile or uniform norm ranges."""
    from paper_1809_08782_gb300 import workloads as W
    eps = f32(eps)
    part = {"percentile": None, "uniform": N.NRLSH_PARTITION_UNIFORM}[partition]
    lib = N.nrlsh_build_ex(to_dev_items(items, dtype), m, L, seed, eps=eps, projection=projection,
                           partition=part)
    ref = O.build(W.items_to_f64(items, dtype), m, L, seed, eps=eps, partition_scheme=partition)
    return lib, ref


def check_index(lib, ref, projection=None):
    info = N.nrlsh_get_info(lib)
    assert info["device_error"] == 0, "a bounded device wait ran out"
    if projection is not None:
        assert info["projection"] == projection
    A = N.nrlsh_get_projections(lib).numpy().astype(np.float64)
    assert np.array_equal(A, ref.A), "projection matrix differs"
    sub, U2, s = N.nrlsh_get_partition(lib)
    assert np.array_equal(s.numpy(), ref.s), "squared norms differ"
    assert np.array_equal(sub.numpy(), ref.sub), "partition differs"
    assert np.array_equal(U2.numpy(), ref.U2), "U_j^2 differs"
    assert N.nrlsh_get_segments(lib).tolist() == list(ref.bounds), "segment offsets differ"
    codes = N.nrlsh_get_codes(lib).numpy().view(np.uint64)
    bad = np.flatnonzero(codes != ref.codes)
    assert bad.size == 0, f"{bad.size} codes differ, first ids {bad[:8]}"
    bj, bl, sh = N.nrlsh_get_buckets(lib)
    order = list(zip(bj.tolist(), bl.tolist()))
    assert order == [tuple(t) for t in ref.table], "bucket order differs"
    exp_sh = np.array([ref.shat[j, l] for j, l in ref.table])
    assert np.array_equal(sh.numpy(), exp_sh), "s_hat differs"


def check_queries(lib, ref, Q: np.ndarray, k: int, B: int, flags: int = 0,
                  check_hist: bool = True):
    Qd = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).to(DEV)
    Q64 = Q.astype(np.float32).astype(np.float64)
    cq = O.query_codes(Q64, ref.A)
    got_cq = N.nrlsh_hash_queries(lib, Qd).cpu().numpy().view(np.uint64)
    assert np.array_equal(got_cq, cq), "query codes differ"
    whole = bool(flags & N.NRLSH_WHOLE_BUCKETS)
    if check_hist:
        H = N.nrlsh_query_histograms(lib, Qd).cpu().numpy()
        for i in range(Q.shape[0]):
            assert np.array_equal(H[i], O.histogram(ref, int(cq[i]))), f"histogram {i} differs"
    cand, count = N.nrlsh_query_candidates(lib, Qd, B, flags=flags)
    cand = cand.cpu().numpy()
    count = count.cpu().numpy()
    for i in range(Q.shape[0]):
        exp = O.candidates_reported(ref, int(cq[i]), B, whole_class=whole)
        assert count[i] == exp.size, f"query {i}: {count[i]} candidates, expected {exp.size}"
        assert np.array_equal(cand[i, :count[i]], exp), f"candidates of query {i} differ"
    ids, sc = N.nrlsh_query_ex(lib, Qd, k, B, flags=flags)
    rids, rsc = O.query(ref, Q64, k, B, whole_class=whole)
    ids = ids.cpu().numpy()
    sc = sc.cpu().numpy()
    bad = np.flatnonzero((ids != rids).any(axis=1))
    assert bad.size == 0, f"top-k ids differ for queries {bad[:8]}"
    assert np.array_equal(sc, rsc), "top-k scores differ"


def check_queries_tc(lib, ref, Q: np.ndarray, k: int, B: int, flags: int = 0,
                     check_hist: bool = True):
    """The tensor-core query path against the oracle: histograms element by
    element, candidate sets (the path groups them by sub-dataset, in no order
    inside one), then top-k ids and scores bit for bit."""
    T = N.NRLSH_QUERY_TENSOR
    Qd = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).to(DEV)
    Q64 = Q.astype(np.float32).astype(np.float64)
    cq = O.query_codes(Q64, ref.A)
    whole = bool(flags & N.NRLSH_WHOLE_BUCKETS)
    if check_hist:
        H = N.nrlsh_query_histograms(lib, Qd, flags=T).cpu().numpy()
        for i in range(Q.shape[0]):
            assert np.array_equal(H[i], O.histogram(ref, int(cq[i]))), f"TC histogram {i} differs"
    cand, count = N.nrlsh_query_candidates(lib, Qd, B, flags=flags | T)
    cand = cand.cpu().numpy()
    count = count.cpu().numpy()
    order = O.storage_order(ref)
    rank_of = np.empty(ref.n, dtype=np.int64)
    rank_of[order] = np.arange(ref.n)
    for i in range(Q.shape[0]):
        exp = O.candidates(ref, int(cq[i]), B, whole_class=whole)
        assert count[i] == exp.size, f"query {i}: {count[i]} TC candidates, expected {exp.size}"
        got = cand[i, :count[i]].astype(np.int64)
        assert np.array_equal(np.sort(got), np.sort(exp)), f"TC candidates of query {i} differ"
        subs = ref.sub[got]
        assert np.all(np.diff(subs) >= 0), f"TC candidates of query {i} not grouped by sub-dataset"
    ids, sc = N.nrlsh_query_ex(lib, Qd, k, B, flags=flags | T)
    rids, rsc = O.query(ref, Q64, k, B, whole_class=whole)
    ids = ids.cpu().numpy()
    sc = sc.cpu().numpy()
    bad = np.flatnonzero((ids != rids).any(axis=1))
    assert bad.size == 0, f"TC top-k ids differ for queries {bad[:8]}"
    assert np.array_equal(sc, rsc), "TC top-k scores differ"
    info = N.nrlsh_get_info(lib)
    assert info["query_error"] == 0, f"tensor-core query kernel error {info['query_error']}"
