"""Benchmark: queries/s of the norm-ranging LSH hot path at recall@10 >= 0.9.

One step = one pass of the whole path over one batch of synthetic input:
index build (norms, percentile partition, SIMPLE-LSH transform, sign-random-
projection codes, bucket order) over the resident items, then the query batch
(hash, Hamming histograms, bucket walk, candidate selection, exact re-rank,
top-k).  Workload: the Netflix-sized preset (n = 17,770 items, d = 300 fp32,
lognormal(0, 0.8) norms, m = 32, L = 32, 1,000 unit queries per GPU, top-10);
the probe budget B and eps are calibrated (untimed) as the smallest B of the
1%..20% sweep (and the smallest eps of 0.1/0.2/0.3) that reaches recall@10 >= 0.9
against the exact top-10 (the same library at B = n, which the parity tests pin
to exact MIPS).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU: each rank builds its own replica of
the index and answers its own query batch (weak scaling, no data-path
collective).  --impl reference times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1809_08782_gb300 import workloads as W  # noqa: E402

METRIC = "queries/s at recall@10>=0.9, plain FP32 vs BF16-batched; HBM GB/s; p50/p99 ms"
WORKLOAD = "netflix-n17770-d300"
EPS_CHOICES = (0.1, 0.2, 0.3)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP32 CUDA-core rate for the ALU roofline: 152 SMs x 128 FMA lanes x 2 flop x clock
SMS, FP32_LANES = 152, 128
# DRAM bytes per launch (read + write) from the ncu captures summarised in profiles/;
# reported only while the kernel's source file is byte-identical to the captured one.
TRAFFIC = {"probe_rerank": ("query.cu", "0043717274ad1b76", 5.9584e6)}


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(value: float, device=None) -> float:
    """Max of a per-rank value over all ranks (identity without a process group).
    Each rank times its own replica; the job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(prefix="nrlsh_clocks_", suffix=".csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ GPU arm

def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_1809_08782_gb300.nrlsh as N

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_1809_08782_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    N.load()

    w = W.make_workload(WORKLOAD)
    Qh = W.gen_queries(w.nq, w.d, w.query_seed + 7919 * rank)
    X = torch.from_numpy(w.items).to(dev)
    Q = torch.from_numpy(Qh).to(dev)
    stream = torch.cuda.current_stream(dev)

    # -------- calibration (untimed): exact top-10 and the (eps, B) operating point
    idx = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=0.1)
    truth, _ = N.nrlsh_query_ex(idx, Q, w.k, w.n)
    truth = truth.cpu().numpy()
    idx.free()

    def recall(ids):
        ids = ids.cpu().numpy()
        return float(np.mean([len(set(ids[i]) & set(truth[i])) for i in range(len(ids))])) / w.k

    chosen = None
    best = (0.0, None, None)
    if args.eps is not None and args.budget is not None:
        idx = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=float(np.float32(args.eps)))
        ids, _ = N.nrlsh_query_ex(idx, Q, w.k, args.budget)
        chosen = (args.eps, args.budget, recall(ids))
        idx.free()
    for eps in (EPS_CHOICES if chosen is None else ()):
        idx = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=float(np.float32(eps)))
        for B_ in w.budget_sweep:
            ids, _ = N.nrlsh_query_ex(idx, Q, w.k, B_)
            r = recall(ids)
            if r > best[0]:
                best = (r, eps, B_)
            if r >= 0.9:
                if chosen is None or B_ < chosen[1]:
                    chosen = (eps, B_, r)
                break
        idx.free()
    if chosen is None:
        chosen = (best[1], best[2], best[0])
    eps, budget, rec = chosen
    eps = float(np.float32(eps))

    forms = {"plain_fp32": N.NRLSH_PROJECT_SIMT, "bf16_tc": N.NRLSH_PROJECT_TENSOR}
    if args.form != "both":
        forms = {k: v for k, v in forms.items() if k == args.form}

    def step(proj):
        ix = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=proj)
        ids, sc = N.nrlsh_query_ex(ix, Q, w.k, budget)
        return ix, ids

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def timed(proj):
        for _ in range(args.warmup):
            ix, _ = step(proj)
            ix.free()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches0 = N.nrlsh_launch_count()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ix, ids = step(proj)
            e1.record(stream)
            ix.free()                       # synchronises; outside the timed region
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        return times, N.nrlsh_launch_count() - launches0

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    per_form = {}
    for name, proj in forms.items():
        times, launches = timed(proj)
        per_form[name] = (reduce_max(float(np.mean(times)), dev), times, launches, proj)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else None
    best = min(per_form, key=lambda k: per_form[k][0])
    ms_max, times, launches, best_proj = per_form[best]
    value = job_throughput(w.nq, world, ms_max)

    # -------- per-kernel times: the same steps again with event brackets on
    N.nrlsh_set_profiling(True)
    N.nrlsh_profile_read()
    for _ in range(args.steps):
        flush.zero_()
        ix, _ = step(best_proj)
        ix.free()
    torch.cuda.synchronize()
    prof = N.nrlsh_profile_read()
    N.nrlsh_set_profiling(False)

    # -------- end to end through the public API with host buffers
    Xh = torch.from_numpy(w.items).pin_memory()
    Qp = torch.from_numpy(Qh).pin_memory()
    ids_h = torch.empty((w.nq, w.k), dtype=torch.int64).pin_memory()
    sc_h = torch.empty((w.nq, w.k), dtype=torch.float32).pin_memory()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = N.nrlsh_build_ex(Xh, w.m, w.L, w.index_seed, eps=eps, projection=best_proj)
        N.nrlsh_query_ex(ix, Qp, w.k, budget, ids=ids_h, scores=sc_h)
        t1 = time.perf_counter()
        ix.free()
        if i >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_value = job_throughput(w.nq, world, reduce_max(float(np.mean(e2e_t)) * 1e3, dev))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded Gaussian directions, lognormal norms)",
            "form": best,
            "forms": {k: {"queries_per_s": job_throughput(w.nq, world, v[0]), "ms_per_step": v[0],
                          "p50_ms": float(np.percentile(v[1], 50)),
                          "p99_ms": float(np.percentile(v[1], 99))}
                      for k, v in per_form.items()},
            "config": {"workload": WORKLOAD, "n": w.n, "d": w.d, "m": w.m, "L": w.L,
                       "queries_per_gpu": w.nq, "k": w.k, "probe_budget": budget,
                       "eps": eps, "recall_at_10": rec,
                       "step": "index build + query batch",
                       "l2": "flushed (512 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(times, 50)),
                           "p99": float(np.percentile(times, 99))},
            "e2e": {"value": e2e_value, "unit": "queries/s",
                    "h2d_bytes_per_step": int(w.items.nbytes + Qh.nbytes),
                    "d2h_bytes_per_step": int(w.nq * w.k * (8 + 4))},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        line["roofline"] = roofline(prof, w, budget, args.steps)
        line["kernels_ms_per_step"] = {k: v[0] / args.steps for k, v in
                                       sorted(prof.items(), key=lambda kv: -kv[1][0])}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, Qh, eps, budget)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def algorithmic(name: str, w, budget: int):
    """(kind, units per launch) for the kernels whose roofline is stated:
    bytes for HBM-bound kernels, flops for ALU-bound ones (per launch of one step)."""
    n, d, L, nq, k = w.n, w.d, w.L, w.nq, w.k
    cb = 4 if L <= 32 else 8
    if name.startswith("probe_rerank") or name.startswith("rerank_fp32"):
        # candidate rows + their ids, the lower/upper bounds, the histogram row
        return "hbm", float(nq * (budget * (4 * d + 4 + 8) + w.m * (L + 1) * 4))
    if name.startswith("project_fp32"):
        return "hbm", float(n * d * 4 + n * cb + n * 12)
    if name.startswith("hist"):
        return "hbm", float(n * cb * -(-nq // 128) + nq * w.m * (L + 1) * 4)
    if name.startswith("select"):
        return "hbm", float(nq * (n * cb + budget * 4))
    if name.startswith("topk"):
        return "hbm", float(nq * budget * 8)
    if name.startswith("sqnorm"):
        return "hbm", float(n * d * 4 + n * 8)
    return None, None


def roofline(prof: dict, w, budget: int, steps: int):
    hbm, sm_mhz, src = peaks()
    if not prof:
        return None
    name, (ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    kind, units = algorithmic(name, w, budget)
    per_launch_ms = ms / max(launches, 1)
    if kind is None:
        return {"kernel": name, "bound": None, "note": "no algorithmic model for this kernel"}
    launches_per_step = launches / steps
    units_per_launch = units / launches_per_step
    if kind == "hbm":
        achieved = units_per_launch / (per_launch_ms * 1e-3) / 1e9
        peak = hbm
        unit = "GB/s"
        peak_src = f"hbm_gbs of {src} peaks"
    else:
        achieved = units_per_launch / (per_launch_ms * 1e-3) / 1e12
        peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        unit = "TFLOP/s"
        peak_src = f"FP32 FMA rate at {sm_mhz:.0f} MHz (152 SMs x 128 lanes)"
    traffic = None
    key = next((k for k in TRAFFIC if name.startswith(k)), None)
    if key:
        import hashlib
        src, digest, nbytes = TRAFFIC[key]
        path = os.path.join(ROOT, "paper_1809_08782_gb300", "csrc", src)
        if hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] == digest:
            traffic = nbytes
    return {"kernel": name, "bound": kind, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
            "launch_ms": per_launch_ms,
            "algorithmic_units_per_launch": units_per_launch}


# ------------------------------------------------------------ CPU oracle arm

def cpu_baseline(w, Qh, eps, budget, target_s: float = 12.0):
    """The oracle as it stands, single-threaded NumPy on the host: one full index
    build plus as many queries as fit in about `target_s` seconds; scaled to a step
    (build + the whole query batch)."""
    from oracle import nrlsh as O
    X64 = W.items_to_f64(w.items, w.dtype)
    t0 = time.perf_counter()
    ref = O.build(X64, w.m, w.L, w.index_seed, eps=eps)
    t_build = time.perf_counter() - t0
    done = 0
    t1 = time.perf_counter()
    while done < w.nq and time.perf_counter() - t1 < target_s:
        O.query(ref, Qh[done:done + 10].astype(np.float64), w.k, budget)
        done += min(10, w.nq - done)
    t_q = (time.perf_counter() - t1) / done
    step_s = t_build + t_q * w.nq
    return {"value": w.nq / step_s, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"index build over all {w.n} items + {done} of {w.nq} queries, "
                      f"scaled to build + {w.nq} queries"}


def reference_arm(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from oracle import nrlsh as O
    w = W.make_workload(WORKLOAD)
    Qh = W.gen_queries(w.nq, w.d, w.query_seed)
    X64 = W.items_to_f64(w.items, w.dtype)
    eps, budget = float(np.float32(0.3)), int(round(0.03 * w.n))   # the GPU arm's calibrated point
    sample_q = 40
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ref = O.build(X64, w.m, w.L, w.index_seed, eps=eps)
        O.query(ref, Qh[:sample_q].astype(np.float64), w.k, budget)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    step_s = float(np.mean(times))
    value = sample_q / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": w.n, "d": w.d, "m": w.m, "L": w.L,
                       "queries_per_step": sample_q, "k": w.k, "probe_budget": budget,
                       "eps": eps, "step": "index build + query sample"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"index build over all {w.n} items + {sample_q} queries per step"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Kernel-level timing run (not a bench line): builds (or queries) the named
    preset a few times with the library's per-kernel event timing on, and prints
    {kernel: ms per launch}.  Used for the ncu captures summarised in profiles/."""
    import torch

    import paper_1809_08782_gb300.nrlsh as N
    from paper_1809_08782_gb300 import build as B
    B.build()
    N.load()
    kw = {"n": args.n} if args.n else {}
    w = W.make_workload(args.workload, nq=args.queries, with_data=False, **kw)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
    X = W.to_torch(items, w.dtype, "cuda")
    Q = torch.from_numpy(W.gen_queries(w.nq, w.d, w.query_seed)).cuda()
    proj = {"plain_fp32": N.NRLSH_PROJECT_SIMT, "bf16_tc": N.NRLSH_PROJECT_TENSOR,
            "both": N.NRLSH_PROJECT_TENSOR}[args.form]
    eps = float(np.float32(args.eps if args.eps is not None else 0.2))
    budget = args.budget if args.budget is not None else w.budget
    ix = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=proj)
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            N.nrlsh_set_profiling(True)
            N.nrlsh_profile_read()
        if args.profile_case == "build":
            ix.free()
            ix = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=proj)
        else:
            N.nrlsh_query_ex(ix, Q, w.k, budget, flags=N.NRLSH_QUERY_TENSOR if args.tensor else 0)
    torch.cuda.synchronize()
    prof = N.nrlsh_profile_read()
    info = N.nrlsh_get_info(ix)
    print(json.dumps({"profile_case": args.profile_case, "workload": w.name, "form": args.form,
                      "n": w.n, "d": w.d, "L": w.L, "queries": w.nq, "budget": budget,
                      "ambiguous_bits": info["ambiguous_bits"],
                      "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in prof.items()},
                      "launches": {k: v[1] for k, v in prof.items()}}))


def serve_sweep(args):
    """Serving run (not the bench line): the resident serving preset, Poisson
    arrivals at geometrically increasing rates through the continuous-batching
    server, p50/p99 latency and achieved queries/s per rate; and, as the plain
    comparison, the same requests one at a time through nrlsh_query_ex."""
    import torch

    import paper_1809_08782_gb300.nrlsh as N
    from paper_1809_08782_gb300 import build as B
    from paper_1809_08782_gb300.serving import Request, Server, latency_summary
    B.build()
    N.load()
    w = W.make_workload("serving-n10m-d128", n=args.serve_n, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
    X = W.to_torch(items, w.dtype, "cuda")
    del items
    eps = float(np.float32(0.2))
    idx = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=N.NRLSH_PROJECT_TENSOR)
    torch.cuda.synchronize()
    nreq = args.serve_requests
    Q = W.gen_queries(nreq, w.d, w.query_seed)
    budgets, ks = W.per_query_budgets_and_k(nreq, w.n, 0.0005, 0.01, seed=5000)
    # plain: one request at a time, single-query path, synchronous
    plain_n = min(nreq, 300)
    t0 = time.perf_counter()
    for i in range(plain_n):
        ids, sc = N.nrlsh_query_ex(idx, torch.from_numpy(Q[i:i + 1]).cuda(), int(ks[i]),
                                   int(budgets[i]))
        ids.cpu()
    plain_qps = plain_n / (time.perf_counter() - t0)
    # tune the batched tiles once on a full-size batch
    N.nrlsh_query_batched(idx, torch.from_numpy(Q[:1024]).cuda(), torch.from_numpy(ks[:1024]).cuda(),
                          torch.from_numpy(budgets[:1024]).cuda(), 100, int(budgets.max()))
    torch.cuda.synchronize()
    print(json.dumps({"serving": "plain_one_at_a_time", "n": w.n, "d": w.d,
                      "queries_per_s": plain_qps, "requests": plain_n}), flush=True)
    rng = np.random.default_rng(5001)
    rate = args.serve_rate0
    for _ in range(args.serve_rates):
        reqs = [Request(i, Q[i], int(ks[i]), int(budgets[i])) for i in range(nreq)]
        arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
        srv = Server(idx, slots=4, memory_budget=args.serve_memory << 20, max_batch=4096)
        srv.serve(reqs, arrivals)
        summ = latency_summary(reqs)
        summ.update({"serving": "continuous_batching", "offered_queries_per_s": rate, "n": w.n,
                     "d": w.d, "batches": srv.batches, "max_concurrent_batches": srv.max_concurrent,
                     "memory_budget_mb": args.serve_memory,
                     "tuning": N.nrlsh_get_tuning(idx)})
        print(json.dumps(summ), flush=True)
        if summ["p99_ms"] > 1000.0:
            break
        rate *= 2


def batched_run(args):
    """Batching form (not the bench line): the ImageNet-sized preset, 100,000
    queries with per-query budgets uniform in [0.1%, 5%] of n and k in {1, 10, 100},
    one nrlsh_query_batched call replayed as a CUDA graph; queries/s, recall@10 on
    a subset, and the plain single-query path on a subset at the mean budget."""
    import torch

    import paper_1809_08782_gb300.nrlsh as N
    from paper_1809_08782_gb300 import build as B
    from paper_1809_08782_gb300 import curves as C
    B.build()
    N.load()
    w = W.make_workload("imagenet-n2340373-d150", nq=args.queries, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
    X = W.to_torch(items, w.dtype, "cuda")
    del items
    eps = float(np.float32(args.eps if args.eps is not None else 0.3))
    idx = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=N.NRLSH_PROJECT_TENSOR)
    Qh = W.gen_queries(w.nq, w.d, w.query_seed)
    budgets, ks = W.per_query_budgets_and_k(w.nq, w.n, 0.001, 0.05, seed=4000)
    Q = torch.from_numpy(Qh).cuda()
    ksd = torch.from_numpy(ks).cuda()
    bd = torch.from_numpy(budgets).cuda()
    k_max, bmax = int(ks.max()), int(budgets.max())
    ids = torch.empty((w.nq, k_max), dtype=torch.int64, device="cuda")
    sc = torch.empty((w.nq, k_max), dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    times = []
    with torch.cuda.stream(st):
        for i in range(args.warmup + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            N.nrlsh_query_batched(idx, Q, ksd, bd, k_max, bmax, flags=N.NRLSH_QUERY_GRAPH, ids=ids,
                                  scores=sc)
            e1.record(st)
            e1.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    sub = min(w.nq, 500)
    truth = C.exact_topk(idx, Q[:sub])
    got = ids[:sub, :10].cpu().numpy()
    mask = ks[:sub] >= 10
    rec = C.recall(got[mask], truth[mask])
    # plain comparison: single-query path (FP32 CUDA-core projection index) at the mean budget
    idx_plain = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=N.NRLSH_PROJECT_SIMT)
    mb = int(budgets.mean())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    N.nrlsh_query_ex(idx_plain, Q[:2000], 10, mb)
    torch.cuda.synchronize()
    plain_qps = 2000 / (time.perf_counter() - t0)
    print(json.dumps({"batched": True, "workload": w.name, "n": w.n, "d": w.d, "queries": w.nq,
                      "ms_per_batch": ms, "queries_per_s": w.nq / (ms / 1e3),
                      "recall_at_10_subset": rec, "eps": eps, "mean_budget": mb,
                      "tuning": N.nrlsh_get_tuning(idx),
                      "plain_single_query_path_queries_per_s_at_mean_budget": plain_qps}),
          flush=True)


def curves_run(args):
    """Probed items vs recall@10 (Figure 2 protocol) on the synthetic stand-ins:
    RANGE-LSH vs SIMPLE-LSH at L = 16/32/64 with m = 32/64/128 (Section 5), an
    m sweep at L = 32 (Figure 3b) and percentile vs uniform partitioning at L = 32,
    m = 32 (Figure 3a).  Prints JSON lines (not the bench line)."""
    import torch

    import paper_1809_08782_gb300.nrlsh as N
    from paper_1809_08782_gb300 import build as B
    from paper_1809_08782_gb300 import curves as C
    B.build()
    N.load()
    for name in args.curve_workloads.split(","):
        w = W.make_workload(name, nq=args.queries, with_data=False)
        items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
        X = W.to_torch(items, w.dtype, "cuda")
        Q = torch.from_numpy(W.gen_queries(w.nq, w.d, w.query_seed)).cuda()
        idx = N.nrlsh_build_ex(X, 1, 8, w.index_seed)
        truth = C.exact_topk(idx, Q)
        idx.free()
        eps = float(np.float32(args.eps if args.eps is not None else 0.1))
        sets = args.curve_sets.split(",")
        for L, m in (((16, 32), (32, 64), (64, 128)) if "fig2" in sets else ()):
            r = C.compare(X, Q, L, m, w.index_seed, eps, truth)
            r.update({"workload": name, "queries": w.nq, "eps": eps})
            print(json.dumps(r), flush=True)
        if name.startswith("yahoo") and "fig3b" in sets:
            for m in (32, 64, 128, 256):
                r = C.compare(X, Q, 32, m, w.index_seed, eps, truth)
                r.update({"workload": name, "queries": w.nq, "eps": eps, "m_sweep": True})
                print(json.dumps(r), flush=True)
        # Figure 3a: percentile versus uniform norm ranges, code length 32, m = 32
        if "fig3a" in sets:
            r = C.compare_partitions(X, Q, 32, 32, w.index_seed, eps, truth)
            r.update({"workload": name, "queries": w.nq, "eps": eps, "partitions": True})
            print(json.dumps(r), flush=True)


def multitable_run(args):
    """Algorithm 2 with several single-probe tables (the variant of the paper's
    supplementary comparison): probed items, recall@10 and device time per query as
    the code is split into more, shorter tables; RANGE-LSH (m = 32) vs SIMPLE-LSH
    (m = 1) at L = 32 and 64.  Prints JSON lines (not the bench line)."""
    import torch

    import paper_1809_08782_gb300.nrlsh as N
    from paper_1809_08782_gb300 import build as B
    from paper_1809_08782_gb300 import curves as C
    B.build()
    N.load()
    for name in args.curve_workloads.split(","):
        w = W.make_workload(name, nq=args.queries, with_data=False)
        items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, w.dtype)
        X = W.to_torch(items, w.dtype, "cuda")
        Q = torch.from_numpy(W.gen_queries(w.nq, w.d, w.query_seed)).cuda()
        idx = N.nrlsh_build_ex(X, 1, 8, w.index_seed)
        truth = C.exact_topk(idx, Q)
        idx.free()
        eps = float(np.float32(args.eps if args.eps is not None else 0.1))
        for L in (32, 64):
            tables = [t for t in (1, 2, 4, 8, 16, 32, 64) if L % t == 0 and L // t >= 2]
            for m in (32, 1):
                r = C.multitable_curve(X, Q, truth, m, L, w.index_seed, eps, tables)
                r.update({"workload": name, "queries": w.nq, "eps": eps,
                          "method": "range_lsh" if m > 1 else "simple_lsh"})
                print(json.dumps(r), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="both", choices=["both", "plain_fp32", "bf16_tc"],
                    help="projection path(s) to time")
    ap.add_argument("--eps", type=float, default=None, help="skip calibration: fixed eps")
    ap.add_argument("--budget", type=int, default=None, help="skip calibration: fixed B")
    ap.add_argument("--profile-case", default=None, choices=["build", "query"],
                    help="kernel timing run of one phase instead of the bench line")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.PRESETS))
    ap.add_argument("--queries", type=int, default=1000, help="queries (profile runs)")
    ap.add_argument("--n", type=int, default=None, help="profile runs: items of the preset")
    ap.add_argument("--tensor", action="store_true",
                    help="profile runs: queries through the tensor-core path")
    ap.add_argument("--serve", action="store_true", help="serving sweep instead of the bench line")
    ap.add_argument("--curves", action="store_true", help="probed-item/recall curves")
    ap.add_argument("--batched", action="store_true", help="batching-form run (ImageNet-sized)")
    ap.add_argument("--multitable", action="store_true",
                    help="multi-table single-probe curves (Algorithm 2)")
    ap.add_argument("--curve-workloads", default="netflix-n17770-d300,yahoo-n136736-d300")
    ap.add_argument("--curve-sets", default="fig2,fig3a,fig3b",
                    help="which curve families --curves runs")
    ap.add_argument("--serve-n", type=int, default=10_000_000)
    ap.add_argument("--serve-requests", type=int, default=20_000)
    ap.add_argument("--serve-rate0", type=float, default=25_000.0)
    ap.add_argument("--serve-rates", type=int, default=7)
    ap.add_argument("--serve-memory", type=int, default=8192, help="admission budget, MB")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        profile_case(args)
        return
    if args.serve:
        serve_sweep(args)
        return
    if args.curves:
        curves_run(args)
        return
    if args.batched:
        batched_run(args)
        return
    if args.multitable:
        multitable_run(args)
        return
    if args.impl == "reference":
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
