"""The continuous-batching server: every request returns exactly what it returns
when run alone, while batches of mixed requests overlap on several streams;
admission respects the memory budget."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from paper_1809_08782_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1809_08782_gb300.nrlsh as N
    w = W.make_workload("small-n10k-d64", n=30_000, nq=600, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, 1.0, "f32")
    idx = N.nrlsh_build_ex(torch.from_numpy(items).cuda(), 16, 32, 5, eps=float(np.float32(0.2)))
    Q = W.gen_queries(w.nq, w.d, w.query_seed)
    budgets, ks = W.per_query_budgets_and_k(w.nq, w.n, 0.0005, 0.01, seed=9)
    return N, idx, Q, ks, budgets


def alone(N, idx, q, k, b):
    ids, sc = N.nrlsh_query_ex(idx, torch.from_numpy(q[None, :]).cuda(), int(k), int(b))
    torch.cuda.synchronize()
    return ids.cpu().numpy()[0], sc.cpu().numpy()[0]


@pytest.mark.parametrize("path", ["auto", "tensor", "bf16"])
def test_results_equal_alone_and_in_the_mix(setup, path):
    from paper_1809_08782_gb300.serving import Request, Server, latency_summary
    N, idx, Q, ks, budgets = setup
    reqs = [Request(i, Q[i], int(ks[i]), int(budgets[i])) for i in range(len(Q))]
    rng = np.random.default_rng(3)
    arrivals = np.cumsum(rng.exponential(1.0 / 50_000.0, len(reqs)))   # Poisson, 50k q/s
    srv = Server(idx, slots=3, memory_budget=256 << 20, max_batch=64, path=path)
    done = srv.serve(reqs, arrivals)
    assert all(r.ids is not None for r in done)
    assert srv.batches < len(reqs)            # requests were batched together
    for r in done[::7]:
        ids, sc = alone(N, idx, r.query, r.k, r.budget)
        assert np.array_equal(r.ids, ids) and np.array_equal(r.scores, sc), r.rid
    s = latency_summary(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_memory_admission_limits_concurrency(setup):
    from paper_1809_08782_gb300.serving import Request, Server
    N, idx, Q, ks, budgets = setup
    bmax = int(budgets.max())             # every request at the largest budget: one batch of
    one = N.nrlsh_batched_scratch_bytes(idx, 8, 100, bmax)   # 8 needs about `one` bytes
    reqs = [Request(i, Q[i], 100, bmax) for i in range(200)]
    srv = Server(idx, slots=4, memory_budget=int(one * 1.5), max_batch=8)
    done = srv.serve(reqs, np.zeros(len(reqs)))
    assert srv.max_concurrent == 1            # a second batch never fits beside the first
    for r in done[::11]:
        ids, sc = alone(N, idx, r.query, r.k, r.budget)
        assert np.array_equal(r.ids, ids)


def test_background_thread_mode(setup):
    from paper_1809_08782_gb300.serving import Request, Server
    N, idx, Q, ks, budgets = setup
    srv = Server(idx, slots=2, memory_budget=512 << 20, max_batch=32)
    srv.start()
    reqs = [srv.submit(Request(i, Q[i], int(ks[i]), int(budgets[i]))) for i in range(100)]
    srv.stop()
    assert len(srv.completed) == 100
    r = reqs[42]
    ids, _ = alone(N, idx, r.query, r.k, r.budget)
    assert np.array_equal(r.ids, ids)


def test_admission_budget_smaller_than_one_request(setup):
    """A memory budget below any single request's scratch: the server still makes
    progress by running each request alone (never two batches at once), and every
    result equals the request run alone."""
    from paper_1809_08782_gb300.serving import Request, Server
    N, idx, Q, ks, budgets = setup
    reqs = [Request(i, Q[i], int(ks[i]), int(budgets[i])) for i in range(40)]
    srv = Server(idx, slots=3, memory_budget=1, max_batch=16)
    done = srv.serve(reqs, np.zeros(len(reqs)))
    assert srv.max_concurrent == 1 and srv.batches == len(reqs)
    for r in done[::5]:
        ids, sc = alone(N, idx, r.query, r.k, r.budget)
        assert np.array_equal(r.ids, ids) and np.array_equal(r.scores, sc)


def test_server_rejects_unknown_path(setup):
    from paper_1809_08782_gb300.serving import Server
    _, idx, _, _, _ = setup
    with pytest.raises(ValueError):
        Server(idx, path="fp16")
