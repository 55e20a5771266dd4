"""Parity where the large configurations run: k up to NRLSH_MAX_K with many equal
scores (every branch of the exact top-k), probe budgets of 10^4 and 10^5
candidates, a query subset of the full ImageNet-sized index (n = 2,340,373) and
a 10^6-item serving index -- each against the CPU oracle, element by element, on
the FP32 path and on the tensor-core path."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair, check_queries, check_queries_tc  # noqa: E402


@pytest.fixture(scope="module")
def N():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1809_08782_gb300.nrlsh as nrlsh
    return nrlsh


def rand_items(n, d, seed, sigma=1.0, dtype="f32"):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x32 = (x * rng.lognormal(0, sigma, n)[:, None]).astype(np.float32)
    return W.bf16_bits_from_f32(x32) if dtype == "bf16" else x32


def check_batched(N, lib, ref, Q, ks, budgets, flags):
    k_max = int(ks.max())
    ids, sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                                    torch.from_numpy(budgets).cuda(), k_max, int(budgets.max()),
                                    flags=flags)
    torch.cuda.synchronize()
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i in range(Q.shape[0]):
        k = int(ks[i])
        assert np.array_equal(ids[i, :k], rids[i, :k]), f"query {i} (k={k}, B={budgets[i]})"
        assert np.array_equal(sc[i, :k], rsc[i, :k]), f"query {i}"
        assert np.all(ids[i, k:] == -1) and np.all(np.isneginf(sc[i, k:]))
    assert N.nrlsh_get_info(lib)["query_error"] == 0


# ------------------------------------------------------------------- large k

@pytest.fixture(scope="module")
def tied(N):
    """20,000 items: 2,500 distinct rows, each stored 8 times, so the top-k of a
    query holds groups of exactly equal scores (ties go to the smaller id) and the
    contender set near the k-th score is wide."""
    base = rand_items(2_500, 32, 17)
    rng = np.random.default_rng(18)
    items = np.repeat(base, 8, axis=0)[rng.permutation(20_000)]
    return build_pair(items, "f32", 16, 32, seed=3, eps=0.3)


@pytest.mark.parametrize("k", [256, 600, 1024])
def test_large_k_with_equal_scores(N, tied, k):
    """k = 256 (compensated tier), 600 (more than 512 contenders: canonical FP64
    for every contender, ranked by counting) and 1,024 (more than 1,024
    contenders: block arg-max rounds), budget 8,000 and n."""
    lib, ref = tied
    Q = W.gen_queries(12, 32, 5)
    for B in (8_000, 20_000):
        check_queries(lib, ref, Q, k, B, check_hist=False)
        check_queries_tc(lib, ref, Q, k, B, check_hist=False)


def test_large_k_batched(N, tied):
    lib, ref = tied
    Q = W.gen_queries(40, 32, 6)
    rng = np.random.default_rng(4)
    ks = rng.choice([1, 100, 600, 1024], 40).astype(np.int32)
    budgets = rng.integers(1_024, 20_001, 40).astype(np.int64)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_FP32)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_BF16 | N.NRLSH_QUERY_NO_TUNE)
    assert N.nrlsh_get_tuning(lib)["rows_bf16"]
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_TENSOR)


# ------------------------------------------------------------- large budgets

@pytest.fixture(scope="module")
def big(N):
    items = rand_items(200_000, 16, 23, sigma=1.0)
    return build_pair(items, "f32", 16, 32, seed=8, eps=0.2)


@pytest.mark.parametrize("B", [10_000, 100_000])
def test_large_budgets(N, big, B):
    lib, ref = big
    Q = W.gen_queries(16, 16, 31)
    check_queries(lib, ref, Q, 100, B, check_hist=False)
    check_queries_tc(lib, ref, Q, 100, B, check_hist=False)


def test_large_budgets_batched(N, big):
    lib, ref = big
    Q = W.gen_queries(48, 16, 32)
    rng = np.random.default_rng(33)
    budgets = rng.choice([1, 500, 10_000, 60_000, 100_000, 200_000], 48).astype(np.int64)
    ks = rng.choice([1, 10, 100], 48).astype(np.int32)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_FP32)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_BF16 | N.NRLSH_QUERY_NO_TUNE)
    assert N.nrlsh_get_tuning(lib)["rows_bf16"]
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_TENSOR)


# ---------------------------------------------------- the ImageNet-sized index

@pytest.fixture(scope="module")
def imagenet(N):
    w = W.make_workload("imagenet-n2340373-d150", with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, "bf16")
    eps = float(np.float32(0.3))
    lib = N.nrlsh_build_ex(W.to_torch(items, "bf16", "cuda"), w.m, w.L, w.index_seed, eps=eps,
                           projection=N.NRLSH_PROJECT_TENSOR)
    ref = O.build(W.items_to_f64(items, "bf16"), w.m, w.L, w.index_seed, eps=eps)
    return w, lib, ref


def test_full_size_imagenet_queries(N, imagenet):
    """24 queries of the full n = 2,340,373 x 150 bf16 index with budgets up to 5% of
    n and k in {1, 10, 100}: ids and scores of both batched paths, and the probed
    candidates of four queries (FP32 path in reported order, tensor path as sets),
    against the oracle."""
    w, lib, ref = imagenet
    assert N.nrlsh_get_info(lib)["device_error"] == 0
    assert np.array_equal(N.nrlsh_get_codes(lib).numpy().view(np.uint64), ref.codes)
    Q = W.gen_queries(24, w.d, w.query_seed + 1)
    budgets, ks = W.per_query_budgets_and_k(24, w.n, 0.001, 0.05, seed=4001)
    ks[:6] = 100
    budgets[:6] = int(0.05 * w.n)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_FP32)
    check_batched(N, lib, ref, Q, ks, budgets, N.NRLSH_QUERY_TENSOR)
    Qd = torch.from_numpy(Q[:4]).cuda()
    cq = O.query_codes(Q[:4].astype(np.float64), ref.A)
    B = int(budgets[0])
    cand, count = N.nrlsh_query_candidates(lib, Qd, B)
    cand_t, count_t = N.nrlsh_query_candidates(lib, Qd, B, flags=N.NRLSH_QUERY_TENSOR)
    cand, count = cand.cpu().numpy(), count.cpu().numpy()
    cand_t, count_t = cand_t.cpu().numpy(), count_t.cpu().numpy()
    for i in range(4):
        exp = O.candidates_reported(ref, int(cq[i]), B)
        assert count[i] == exp.size and np.array_equal(cand[i, :count[i]], exp)
        assert count_t[i] == exp.size
        assert np.array_equal(np.sort(cand_t[i, :count_t[i]]), np.sort(exp))


# ----------------------------------------------------------------- serving

def test_serving_million_item_index_against_oracle(N):
    """50 requests through the continuous-batching server over a 10^6 x 128 bf16
    index (lognormal(0, 1) norms, m = 64, L = 64), budgets uniform in [0.05%, 1%]
    of n and k in {1, 10, 100}: every result equals the oracle's, on the
    tensor-core path and on the autotuned one."""
    from paper_1809_08782_gb300.serving import Request, Server
    n, d = 1_000_000, 128
    items = W.gen_items(n, d, 1005, "lognormal", 1.0, "bf16")
    eps = float(np.float32(0.2))
    lib = N.nrlsh_build_ex(W.to_torch(items, "bf16", "cuda"), 64, 64, 3005, eps=eps,
                           projection=N.NRLSH_PROJECT_TENSOR)
    ref = O.build(W.items_to_f64(items, "bf16"), 64, 64, 3005, eps=eps)
    Q = W.gen_queries(50, d, 2005)
    budgets, ks = W.per_query_budgets_and_k(50, n, 0.0005, 0.01, seed=5005)
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    # tune once on a batch shaped like the requests, so the server has a choice
    N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                          torch.from_numpy(budgets).cuda(), 100, int(budgets.max()))
    for path in ("tensor", "auto"):
        reqs = [Request(i, Q[i], int(ks[i]), int(budgets[i])) for i in range(50)]
        rng = np.random.default_rng(7)
        srv = Server(lib, slots=3, memory_budget=4 << 30, max_batch=16, path=path)
        done = srv.serve(reqs, np.cumsum(rng.exponential(1.0 / 20_000.0, 50)))
        for r in done:
            k = int(ks[r.rid])
            assert np.array_equal(r.ids, rids[r.rid, :k]), (path, r.rid)
            assert np.array_equal(r.scores, rsc[r.rid, :k]), (path, r.rid)
    assert N.nrlsh_get_info(lib)["query_error"] == 0
