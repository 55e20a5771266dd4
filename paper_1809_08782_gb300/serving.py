"""Continuous-batching query server over a resident norm-ranging LSH index.

Requests (one query vector, its k and its probe budget) are admitted in arrival
order into batches as soon as a slot (a CUDA stream) is free and the batch's
device scratch fits the memory left in the budget; the scratch size is the
library's own figure (``nrlsh_batched_scratch_bytes``).  Batches on different
slots run concurrently on the device.  Each batch goes through
``nrlsh_query_batched`` (the tensor-core path or the persistent FP32 re-rank), with its
inputs copied from pinned host memory and its results copied back on the slot's
stream; a request completes when its batch's event has fired.

Results do not depend on which requests share a batch: every query is
processed independently, with the same arithmetic, so a request returns the
same ids and scores alone or in any mix.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import nrlsh as N


@dataclasses.dataclass
class Request:
    rid: int
    query: np.ndarray            # (d,) float32
    k: int
    budget: int
    t_arrival: float = 0.0       # perf_counter seconds
    t_admit: float = 0.0
    t_done: float = 0.0
    ids: Optional[np.ndarray] = None
    scores: Optional[np.ndarray] = None

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_arrival) * 1e3


@dataclasses.dataclass
class _Batch:
    reqs: List[Request]
    event: torch.cuda.Event
    nbytes: int
    k_max: int
    host_ids: torch.Tensor
    host_scores: torch.Tensor
    keep: tuple                  # device tensors alive until the batch completes


class Server:
    """Continuous batching with memory-based admission.

    index          a built ``nrlsh.Index`` (kept resident)
    slots          concurrent batches (one CUDA stream each)
    memory_budget  bytes of device scratch all in-flight batches may use
    max_batch      requests per batch at most
    path           "auto": the configuration the index's autotuner chose last;
                   "tensor": the tensor-core path; "fp32": the FP32 re-rank over the
                   stored rows; "bf16": bf16 operands (tensor cores or bf16 rows)
    """

    _PATH_FLAGS = {"auto": 0, "tensor": N.NRLSH_QUERY_TENSOR, "fp32": N.NRLSH_QUERY_FP32,
                   "bf16": N.NRLSH_QUERY_BF16}

    def __init__(self, index: "N.Index", slots: int = 3, memory_budget: int = 1 << 30,
                 max_batch: int = 4096, path: str = "auto"):
        if path not in self._PATH_FLAGS:
            raise ValueError(f"path must be one of {sorted(self._PATH_FLAGS)}")
        self.flags = N.NRLSH_QUERY_NO_TUNE | self._PATH_FLAGS[path]
        self.index = index
        self.d = index.d
        self.device = index.device if index.device.type == "cuda" else torch.device("cuda")
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.busy: List[Optional[_Batch]] = [None] * slots
        self.pending: collections.deque = collections.deque()
        self.memory_budget = int(memory_budget)
        self.in_flight_bytes = 0
        self.max_batch = max_batch
        self.lock = threading.Lock()
        self.completed: List[Request] = []
        self.max_concurrent = 0
        self.batches = 0
        self._thread = None
        self._stop = threading.Event()

    # -------------------------------------------------------------- admission

    def submit(self, req: Request) -> Request:
        if req.t_arrival == 0.0:
            req.t_arrival = time.perf_counter()
        with self.lock:
            self.pending.append(req)
        return req

    def _batch_bytes(self, nq: int, k_max: int, budget_max: int) -> int:
        scratch = N.nrlsh_batched_scratch_bytes(self.index, nq, k_max, budget_max, self.flags)
        io = nq * (self.d * 4 + 4 + 8) + nq * k_max * (8 + 4)     # device inputs and outputs
        return scratch + io

    def _take_batch(self) -> Optional[List[Request]]:
        """Largest FIFO prefix of the pending requests whose scratch fits."""
        with self.lock:
            if not self.pending:
                return None
            free = self.memory_budget - self.in_flight_bytes
            reqs: List[Request] = []
            k_max = budget_max = 0
            for r in self.pending:
                if len(reqs) == self.max_batch:
                    break
                k2, b2 = max(k_max, r.k), max(budget_max, min(r.budget, self.index.n))
                if self._batch_bytes(len(reqs) + 1, k2, b2) > free:
                    break
                reqs.append(r)
                k_max, budget_max = k2, b2
            if not reqs and self.in_flight_bytes == 0:
                reqs = [self.pending[0]]        # larger than the budget alone: run it alone
            for _ in reqs:
                self.pending.popleft()
            return reqs or None

    # --------------------------------------------------------------- the loop

    def _launch(self, slot: int, reqs: List[Request]):
        now = time.perf_counter()
        nq = len(reqs)
        k_max = max(r.k for r in reqs)
        budget_max = max(min(r.budget, self.index.n) for r in reqs)
        nbytes = self._batch_bytes(nq, k_max, budget_max)
        q_h = torch.from_numpy(np.stack([r.query for r in reqs]).astype(np.float32)).pin_memory()
        k_h = torch.tensor([r.k for r in reqs], dtype=torch.int32).pin_memory()
        b_h = torch.tensor([r.budget for r in reqs], dtype=torch.int64).pin_memory()
        ids_h = torch.empty((nq, k_max), dtype=torch.int64).pin_memory()
        sc_h = torch.empty((nq, k_max), dtype=torch.float32).pin_memory()
        st = self.streams[slot]
        with torch.cuda.stream(st):
            q_d = q_h.to(self.device, non_blocking=True)
            k_d = k_h.to(self.device, non_blocking=True)
            b_d = b_h.to(self.device, non_blocking=True)
            ids_d = torch.empty((nq, k_max), dtype=torch.int64, device=self.device)
            sc_d = torch.empty((nq, k_max), dtype=torch.float32, device=self.device)
            N.nrlsh_query_batched(self.index, q_d, k_d, b_d, k_max, budget_max,
                                  flags=self.flags, stream=st, ids=ids_d, scores=sc_d)
            ids_h.copy_(ids_d, non_blocking=True)
            sc_h.copy_(sc_d, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        for r in reqs:
            r.t_admit = now
        self.in_flight_bytes += nbytes
        self.busy[slot] = _Batch(reqs, ev, nbytes, k_max, ids_h, sc_h,
                                 (q_h, k_h, b_h, q_d, k_d, b_d, ids_d, sc_d))
        self.batches += 1
        self.max_concurrent = max(self.max_concurrent, sum(b is not None for b in self.busy))

    def _reap(self):
        for slot, b in enumerate(self.busy):
            if b is None or not b.event.query():
                continue
            now = time.perf_counter()
            ids = b.host_ids.numpy()
            sc = b.host_scores.numpy()
            for i, r in enumerate(b.reqs):
                r.ids = ids[i, :r.k].copy()
                r.scores = sc[i, :r.k].copy()
                r.t_done = now
            self.completed.extend(b.reqs)
            self.in_flight_bytes -= b.nbytes
            self.busy[slot] = None

    def step(self) -> bool:
        """One pass: complete finished batches, admit new ones.  True if busy."""
        self._reap()
        for slot in range(len(self.busy)):
            if self.busy[slot] is None:
                reqs = self._take_batch()
                if reqs is None:
                    break
                self._launch(slot, reqs)
        return any(b is not None for b in self.busy) or bool(self.pending)

    def serve(self, requests: Sequence[Request], arrivals: Sequence[float]) -> List[Request]:
        """Open-loop run: request i arrives arrivals[i] seconds after the start
        (non-decreasing); returns the requests once all have completed."""
        order = np.argsort(np.asarray(arrivals), kind="stable")
        t0 = time.perf_counter()
        i = 0
        while i < len(order) or self.step():
            now = time.perf_counter() - t0
            while i < len(order) and arrivals[order[i]] <= now:
                r = requests[order[i]]
                r.t_arrival = t0 + arrivals[order[i]]
                self.submit(r)
                i += 1
            self.step()
        return list(requests)

    # ------------------------------------------------------ background thread

    def start(self):
        """Serve submitted requests from a background thread until stop()."""
        def run():
            while not self._stop.is_set():
                if not self.step():
                    time.sleep(20e-6)
        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join()
        while self.step():
            pass


def latency_summary(reqs: Sequence[Request]) -> dict:
    lat = np.array([r.latency_ms for r in reqs])
    span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "queries_per_s": len(reqs) / span if span > 0 else float("inf")}
