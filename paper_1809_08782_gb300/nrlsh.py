"""Python binding of libnrlsh.so (ctypes).  Argument marshalling only: every
step of index building and query processing runs in the library's CUDA
kernels.  Functions carry the names of the C entry points in include/nrlsh.h.

Tensors may live on the GPU (the usual case: calls are then asynchronous on
PyTorch's current stream) or on the CPU (the library stages them through device
memory and synchronises).  There is no CPU fallback: if the library has not been
built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnrlsh.so")

NRLSH_F32 = 0
NRLSH_BF16 = 1
NRLSH_WHOLE_BUCKETS = 0x1
NRLSH_QUERY_GRAPH = 0x2
NRLSH_QUERY_NO_TUNE = 0x4
NRLSH_QUERY_TENSOR = 0x8
NRLSH_QUERY_FP32 = 0x10
NRLSH_QUERY_BF16 = 0x20
NRLSH_QUERY_ASYNC_INPUT = 0x40

_STATUS = {0: "NRLSH_OK", -1: "NRLSH_ERR_ARG", -2: "NRLSH_ERR_OOM", -3: "NRLSH_ERR_CUDA",
           -4: "NRLSH_ERR_TIMEOUT", -5: "NRLSH_ERR_UNSUPPORTED"}

# Names and ctypes signatures of every entry point declared in include/nrlsh.h.
_P = ctypes.c_void_p
_I32, _I64, _U32, _U64, _F32 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_float)
SIGNATURES = {
    "nrlsh_build": (_I32, [_P, _I64, _I32, _I32, _I32, _U64, _P]),
    "nrlsh_build_ex": (_I32, [_P, _I64, _I32, _I32, _I32, _U64, _I32, _F32, _P, _P]),
    "nrlsh_build_opts": (_I32, [_P, _I64, _I32, _I32, _I32, _U64, _P, _P]),
    "nrlsh_query": (_I32, [_P, _P, _I64, _I32, _I64, _P, _P]),
    "nrlsh_query_ex": (_I32, [_P, _P, _I64, _I32, _I64, _U32, _P, _P, _P]),
    "nrlsh_query_noalloc": (_I32, [_P, _P, _I64, _I32, _I64, _P, _P, _P]),
    "nrlsh_query_batched": (_I32, [_P, _P, _I64, _P, _P, _I32, _I64, _U32, _P, _P, _P]),
    "nrlsh_get_tuning": (_I32, [_P, _P, _P, _P]),
    "nrlsh_batched_scratch_bytes": (_I32, [_P, _I64, _I32, _I64, _U32, _P]),
    "nrlsh_hash_queries": (_I32, [_P, _P, _I64, _P, _P]),
    "nrlsh_query_histograms": (_I32, [_P, _P, _I64, _P, _U32, _P]),
    "nrlsh_query_candidates": (_I32, [_P, _P, _I64, _I64, _U32, _I64, _P, _P, _P]),
    "nrlsh_query_multitable": (_I32, [_P, _P, _I64, _I32, _I32, _I64, _P, _P, _P, _P]),
    "nrlsh_multitable_candidates": (_I32, [_P, _P, _I64, _I32, _I64, _P, _P, _P]),
    "nrlsh_get_codes": (_I32, [_P, _P]),
    "nrlsh_get_partition": (_I32, [_P, _P, _P, _P]),
    "nrlsh_get_segments": (_I32, [_P, _P]),
    "nrlsh_get_projections": (_I32, [_P, _P]),
    "nrlsh_get_buckets": (_I32, [_P, _P, _P, _P]),
    "nrlsh_get_info": (_I32, [_P, _P]),
    "nrlsh_free": (None, [_P]),
    "nrlsh_last_error": (ctypes.c_char_p, []),
    "nrlsh_launch_count": (_U64, []),
    "nrlsh_read_bandwidth": (_I32, [_P, _I64, _I32, _P, _P]),
    "nrlsh_set_profiling": (_I32, [_I32]),
    "nrlsh_profile_read": (_I32, [_P, _I64, _P, _P, _I32, _P]),
}


class NrlshInfo(ctypes.Structure):
    _fields_ = [("n", _I64), ("d", _I32), ("m", _I32), ("L", _I32), ("dtype", _I32),
                ("eps", _F32), ("seed", _U64), ("code_bytes", _I32), ("row_stride", _I32),
                ("device_bytes", _I64), ("ambiguous_bits", _I64), ("projection", _I32),
                ("device_error", _I32), ("partition", _I32), ("norm_fallbacks", _I32),
                ("query_error", _I32)]


class NrlshBuildOptions(ctypes.Structure):
    _fields_ = [("dtype", _I32), ("eps", _F32), ("projection", _I32), ("partition", _I32),
                ("stream", _P), ("flags", ctypes.c_uint32)]


NRLSH_PROJECT_AUTO = 0
NRLSH_PROJECT_SIMT = 1
NRLSH_PROJECT_TENSOR = 2
NRLSH_PARTITION_PERCENTILE = 0
NRLSH_PARTITION_UNIFORM = 1
NRLSH_BUILD_ASYNC_INPUT = 0x1


class NrlshError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnrlsh.so (built in-tree by paper_1809_08782_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1809_08782_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise NrlshError(status, load().nrlsh_last_error().decode())


def _stream(t: torch.Tensor, stream) -> Optional[int]:
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    if t.is_cuda:
        return int(torch.cuda.current_stream(t.device).cuda_stream)
    return None


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Index:
    """Owner of an nrlsh_index handle; freed with nrlsh_free when collected."""

    def __init__(self, handle: ctypes.c_void_p, n: int, d: int, m: int, L: int, device):
        self.handle = handle
        self.n, self.d, self.m, self.L = n, d, m, L
        self.device = device

    def free(self):
        if self.handle:
            load().nrlsh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # conveniences that mirror the C calls
    def query(self, queries, k, probe_budget, flags=0, stream=None):
        return nrlsh_query_ex(self, queries, k, probe_budget, flags, stream)

    def info(self):
        return nrlsh_get_info(self)


def _items_dtype(items: torch.Tensor) -> int:
    if items.dtype == torch.float32:
        return NRLSH_F32
    if items.dtype == torch.bfloat16:
        return NRLSH_BF16
    raise TypeError("items must be float32 or bfloat16")


def nrlsh_build_ex(items: torch.Tensor, m: int, L: int, seed: int, eps: float = 0.1,
                   stream=None, projection: Optional[int] = None,
                   partition: Optional[int] = None, build_flags: int = 0) -> Index:
    """Index building (Algorithm 1).  items: (n, d) float32 or bfloat16, row-major.
    projection selects the projection path, partition the split into sub-datasets
    and build_flags the NRLSH_BUILD_* flags (nrlsh_build_opts) when any is given."""
    lib = load()
    if items.dim() != 2:
        raise ValueError("items must be 2-D (n, d)")
    items = items.contiguous()
    n, d = items.shape
    out = ctypes.c_void_p()
    if projection is None and partition is None and not build_flags:
        _check(lib.nrlsh_build_ex(_ptr(items), n, d, m, L, seed, _items_dtype(items), eps,
                                  _stream(items, stream), ctypes.byref(out)))
    else:
        st = _stream(items, stream)
        opts = NrlshBuildOptions(_items_dtype(items), eps,
                                 NRLSH_PROJECT_AUTO if projection is None else projection,
                                 NRLSH_PARTITION_PERCENTILE if partition is None else partition, st,
                                 build_flags)
        _check(lib.nrlsh_build_opts(_ptr(items), n, d, m, L, seed, ctypes.byref(opts),
                                    ctypes.byref(out)))
    return Index(out, n, d, m, L, _index_device(items))


def _index_device(items: torch.Tensor) -> torch.device:
    """The GPU an index lives on: the items' device, or for host items the current one."""
    if items.is_cuda:
        return items.device
    return torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else items.device


def nrlsh_build(items: torch.Tensor, m: int, L: int, seed: int) -> Index:
    """Short form: fp32 items, eps = 0.1, legacy default stream."""
    lib = load()
    if items.dtype != torch.float32 or items.dim() != 2:
        raise TypeError("nrlsh_build takes a 2-D float32 tensor")
    items = items.contiguous()
    n, d = items.shape
    out = ctypes.c_void_p()
    _check(lib.nrlsh_build(_ptr(items), n, d, m, L, seed, ctypes.byref(out)))
    return Index(out, n, d, m, L, _index_device(items))


def _queries(index: Index, queries: torch.Tensor) -> torch.Tensor:
    if queries.dtype != torch.float32 or queries.dim() != 2 or queries.shape[1] != index.d:
        raise ValueError(f"queries must be float32 of shape (nq, {index.d})")
    return queries.contiguous()


def _out_devices(index: "Index", queries: torch.Tensor) -> tuple:
    """Where the outputs of a query call may live: host memory or the index's GPU
    (the C ABI takes either for every argument)."""
    dev = index.device if index.device.type == "cuda" else queries.device
    return tuple({torch.device("cpu"), dev, queries.device})


def _check_out(t: torch.Tensor, name: str, dtype: torch.dtype, shape: tuple, device):
    """A caller-supplied output tensor must be exactly what the kernels write: they
    store rows of shape[1] elements at that stride, so another dtype, a smaller
    shape or a strided view would be written past its end."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    devices = device if isinstance(device, tuple) else (device,)
    if t.device not in devices:
        raise ValueError(f"{name} must be on one of {[str(x) for x in devices]}, got {t.device}")


def nrlsh_query_ex(index: Index, queries: torch.Tensor, k: int, probe_budget: int,
                   flags: int = 0, stream=None, ids: Optional[torch.Tensor] = None,
                   scores: Optional[torch.Tensor] = None):
    """Multi-probe query + exact re-rank + top-k.  Returns (ids int64, scores fp32),
    both (nq, k), on the queries' device unless output tensors are given."""
    queries = _queries(index, queries)
    nq = queries.shape[0]
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
    else:
        _check_out(ids, "ids", torch.int64, (nq, k), _out_devices(index, queries))
    if scores is None:
        scores = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    else:
        _check_out(scores, "scores", torch.float32, (nq, k), _out_devices(index, queries))
    lib = load()
    _check(lib.nrlsh_query_ex(index.handle, _ptr(queries), nq, k, probe_budget, flags,
                              _ptr(ids), _ptr(scores), _stream(queries, stream)))
    return ids, scores


def nrlsh_query(index: Index, queries: torch.Tensor, k: int, probe_budget: int):
    """Short form on the legacy default stream."""
    lib = load()
    queries = _queries(index, queries)
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
    scores = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    _check(lib.nrlsh_query(index.handle, _ptr(queries), nq, k, probe_budget, _ptr(ids),
                           _ptr(scores)))
    return ids, scores


def nrlsh_query_noalloc(index: Index, queries: torch.Tensor, k: int, probe_budget: int,
                        ids: torch.Tensor, scores: torch.Tensor, stream=None):
    """The query path without device allocation (for callers that cannot
    allocate while querying).  queries, ids (nq, k) int64 and scores (nq, k) fp32
    must be GPU tensors; the library's fixed 32 MiB scratch array is shared by
    every call, so calls must not overlap on the GPU."""
    queries = _queries(index, queries)
    nq = queries.shape[0]
    _check_out(ids, "ids", torch.int64, (nq, k), queries.device)
    _check_out(scores, "scores", torch.float32, (nq, k), queries.device)
    if not queries.is_cuda:
        raise ValueError("nrlsh_query_noalloc takes GPU tensors only")
    lib = load()
    _check(lib.nrlsh_query_noalloc(index.handle, _ptr(queries), nq, k,
                                   probe_budget, _ptr(ids), _ptr(scores),
                                   _stream(queries, stream)))
    return ids, scores


def nrlsh_query_batched(index: Index, queries: torch.Tensor, ks: torch.Tensor,
                        budgets: torch.Tensor, k_max: int, budget_max: int, flags: int = 0,
                        stream=None, ids: Optional[torch.Tensor] = None,
                        scores: Optional[torch.Tensor] = None):
    """Batched queries with per-query k (int32) and budgets (int64): persistent fused
    probe/re-rank kernel, autotuned tiles, optional CUDA-graph replay
    (NRLSH_QUERY_GRAPH).  Returns (ids, scores), rows k_max wide."""
    queries = _queries(index, queries)
    nq = queries.shape[0]
    if ks.numel() != nq or budgets.numel() != nq:
        raise ValueError(f"ks and budgets must hold {nq} entries")
    ks = ks.to(torch.int32).contiguous()
    budgets = budgets.to(torch.int64).contiguous()
    if ids is None:
        ids = torch.empty((nq, k_max), dtype=torch.int64, device=queries.device)
    else:
        _check_out(ids, "ids", torch.int64, (nq, k_max), _out_devices(index, queries))
    if scores is None:
        scores = torch.empty((nq, k_max), dtype=torch.float32, device=queries.device)
    else:
        _check_out(scores, "scores", torch.float32, (nq, k_max), _out_devices(index, queries))
    lib = load()
    _check(lib.nrlsh_query_batched(index.handle, _ptr(queries), nq, _ptr(ks), _ptr(budgets),
                                   k_max, budget_max, flags, _ptr(ids), _ptr(scores),
                                   _stream(queries, stream)))
    return ids, scores


def nrlsh_batched_scratch_bytes(index: Index, nq: int, k_max: int, budget_max: int,
                                flags: int = 0) -> int:
    """Device scratch of one nrlsh_query_batched call with these sizes and flags."""
    out = ctypes.c_int64()
    _check(load().nrlsh_batched_scratch_bytes(index.handle, nq, k_max, budget_max, flags,
                                              ctypes.byref(out)))
    return out.value


def nrlsh_get_tuning(index: Index):
    """The autotuned batched configuration: popcount histogram tile, persistent
    CTAs per SM, whether the histograms / the re-rank run on tensor cores, and
    whether the FP32 re-rank gathers a bf16 copy of the rows."""
    qb, cps, tc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().nrlsh_get_tuning(index.handle, ctypes.byref(qb), ctypes.byref(cps),
                                   ctypes.byref(tc)))
    return {"hist_queries_per_block": qb.value, "ctas_per_sm": cps.value,
            "hist_tensor": bool(tc.value & 1), "rerank_tensor": bool(tc.value & 2),
            "rows_bf16": bool(tc.value & 4)}


def nrlsh_hash_queries(index: Index, queries: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    queries = _queries(index, queries)
    codes = torch.empty(queries.shape[0], dtype=torch.int64, device=queries.device)
    _check(lib.nrlsh_hash_queries(index.handle, _ptr(queries), queries.shape[0], _ptr(codes),
                                  _stream(queries, stream)))
    return codes


def nrlsh_query_histograms(index: Index, queries: torch.Tensor, flags: int = 0,
                           stream=None) -> torch.Tensor:
    """H (nq, m, L+1): items of sub-dataset j sharing exactly l bits with each query
    (flags NRLSH_QUERY_TENSOR: counted on tensor cores)."""
    lib = load()
    queries = _queries(index, queries)
    H = torch.empty((queries.shape[0], index.m, index.L + 1), dtype=torch.int32,
                    device=queries.device)
    _check(lib.nrlsh_query_histograms(index.handle, _ptr(queries), queries.shape[0], _ptr(H),
                                      flags, _stream(queries, stream)))
    return H


def nrlsh_query_candidates(index: Index, queries: torch.Tensor, probe_budget: int,
                           flags: int = 0, cap: Optional[int] = None, stream=None):
    """Probed item ids (nq, cap) int32 (rows valid up to count) and count (nq,) int64."""
    lib = load()
    queries = _queries(index, queries)
    nq = queries.shape[0]
    if cap is None:
        cap = index.n if flags & NRLSH_WHOLE_BUCKETS else min(probe_budget, index.n)
    cand = torch.full((nq, cap), -1, dtype=torch.int32, device=queries.device)
    count = torch.empty(nq, dtype=torch.int64, device=queries.device)
    _check(lib.nrlsh_query_candidates(index.handle, _ptr(queries), nq, probe_budget, flags, cap,
                                      _ptr(cand), _ptr(count), _stream(queries, stream)))
    return cand, count


def nrlsh_query_multitable(index: Index, queries: torch.Tensor, tables: int, k: int,
                           max_candidates: int = 0, stream=None):
    """Algorithm 2 with `tables` hash tables of L / tables bits, one probe each:
    (ids (nq, k) int64, scores (nq, k) float32, probed (nq,) int64 = |C(q)|)."""
    lib = load()
    queries = _queries(index, queries)
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
    scores = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    probed = torch.empty(nq, dtype=torch.int64, device=queries.device)
    _check(lib.nrlsh_query_multitable(index.handle, _ptr(queries), nq, tables, k, max_candidates,
                                      _ptr(ids), _ptr(scores), _ptr(probed),
                                      _stream(queries, stream)))
    return ids, scores, probed


def nrlsh_multitable_candidates(index: Index, queries: torch.Tensor, tables: int,
                                cap: Optional[int] = None, stream=None):
    """The single-probe candidates C(q) as ids (nq, cap) int32 in storage order (rows
    valid up to min(count, cap)) and count (nq,) int64 = |C(q)|."""
    lib = load()
    queries = _queries(index, queries)
    nq = queries.shape[0]
    cap = index.n if cap is None else cap
    cand = torch.full((nq, cap), -1, dtype=torch.int32, device=queries.device)
    count = torch.empty(nq, dtype=torch.int64, device=queries.device)
    _check(lib.nrlsh_multitable_candidates(index.handle, _ptr(queries), nq, tables, cap,
                                           _ptr(cand), _ptr(count), _stream(queries, stream)))
    return cand, count


def nrlsh_get_codes(index: Index) -> torch.Tensor:
    out = torch.empty(index.n, dtype=torch.int64)
    _check(load().nrlsh_get_codes(index.handle, _ptr(out)))
    return out


def nrlsh_get_partition(index: Index):
    sub = torch.empty(index.n, dtype=torch.int32)
    U2 = torch.empty(index.m, dtype=torch.float64)
    s = torch.empty(index.n, dtype=torch.float64)
    _check(load().nrlsh_get_partition(index.handle, _ptr(sub), _ptr(U2), _ptr(s)))
    return sub, U2, s


def nrlsh_get_segments(index: Index) -> torch.Tensor:
    """Storage offsets: S_j occupies positions [seg[j], seg[j+1])."""
    seg = torch.empty(index.m + 1, dtype=torch.int64)
    _check(load().nrlsh_get_segments(index.handle, _ptr(seg)))
    return seg


def nrlsh_get_projections(index: Index) -> torch.Tensor:
    A = torch.empty((index.d + 1, index.L), dtype=torch.float32)
    _check(load().nrlsh_get_projections(index.handle, _ptr(A)))
    return A


def nrlsh_get_buckets(index: Index):
    c = index.m * (index.L + 1)
    bj = torch.empty(c, dtype=torch.int32)
    bl = torch.empty(c, dtype=torch.int32)
    sh = torch.empty(c, dtype=torch.float64)
    _check(load().nrlsh_get_buckets(index.handle, _ptr(bj), _ptr(bl), _ptr(sh)))
    return bj, bl, sh


def nrlsh_get_info(index: Index, check: bool = True) -> dict:
    """Sizes and statistics of the index.  The library reports a run-out device
    wait as NRLSH_ERR_TIMEOUT; with check=False the statistics (device_error,
    query_error) are returned instead of raising."""
    info = NrlshInfo()
    st = load().nrlsh_get_info(index.handle, ctypes.byref(info))
    if check or st not in (0, -4, -3) or (st == -3 and info.query_error != 15):
        _check(st)
    return {name: getattr(info, name) for name, _ in NrlshInfo._fields_}


def nrlsh_free(index: Index):
    index.free()


def nrlsh_last_error() -> str:
    return load().nrlsh_last_error().decode()


def nrlsh_launch_count() -> int:
    return int(load().nrlsh_launch_count())


def nrlsh_read_bandwidth(buf: torch.Tensor, reps: int = 10, stream=None) -> float:
    """GB/s of reading the device tensor buf (bytes a multiple of 16) with every SM."""
    out = ctypes.c_double()
    _check(load().nrlsh_read_bandwidth(_ptr(buf), buf.numel() * buf.element_size(), reps,
                                       _stream(buf, stream), ctypes.byref(out)))
    return out.value


def nrlsh_set_profiling(enable: bool):
    _check(load().nrlsh_set_profiling(1 if enable else 0))


def nrlsh_profile_read() -> dict:
    """{kernel name: (total ms, launches)} since the last read."""
    lib = load()
    cap = 256
    names = ctypes.create_string_buffer(1 << 16)
    ms = (ctypes.c_double * cap)()
    la = (ctypes.c_int64 * cap)()
    cnt = ctypes.c_int32()
    _check(lib.nrlsh_profile_read(names, len(names), ms, la, cap, ctypes.byref(cnt)))
    keys = [k for k in names.value.decode().split("\n") if k]
    return {k: (ms[i], int(la[i])) for i, k in enumerate(keys[:cap])}
