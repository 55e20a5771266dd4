"""The tensor-core query path (NRLSH_QUERY_TENSOR: match counts from +-1 sign
products and bf16 score intervals on tcgen05, then the exact top-k) against the
CPU oracle, element by element: histograms, candidate sets, top-k ids and
scores, on the presets and on ragged and degenerate shapes; and the batched
entry point on that path."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair, check_index, check_queries_tc  # noqa: E402

SIMT, TENSOR = 1, 2


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


@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_tc_small_preset(N, proj):
    """n=10,000, d=64 fp32, m=8, L=16, B=1,000: 300 queries (three 128-query tiles,
    the last one ragged), then all 1,000 without the histogram check."""
    w = W.make_workload("small-n10k-d64")
    lib, ref = build_pair(w.items, w.dtype, w.m, w.L, w.index_seed, 0.1, projection=proj)
    check_index(lib, ref, proj)
    check_queries_tc(lib, ref, w.queries[:300], w.k, w.budget)
    check_queries_tc(lib, ref, w.queries, w.k, w.budget, check_hist=False)


@pytest.mark.parametrize("frac", [0.01, 0.03, 0.20])
def test_tc_netflix_preset(N, frac):
    """n=17,770, d=300 fp32 (five score chunks), m=32, L=32."""
    w = W.make_workload("netflix-n17770-d300", nq=200)
    lib, ref = build_pair(w.items, w.dtype, w.m, w.L, w.index_seed, 0.3, projection=SIMT)
    check_queries_tc(lib, ref, w.queries, w.k, int(round(frac * w.n)))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tc_yahoo_preset(N, dtype):
    """n=136,736, d=300, m=32, L=64, both stored dtypes; 64 queries."""
    w = W.make_workload("yahoo-n136736-d300", nq=64, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, dtype)
    Q = W.gen_queries(w.nq, w.d, w.query_seed)
    lib, ref = build_pair(items, dtype, w.m, w.L, w.index_seed, 0.1, projection=TENSOR)
    check_queries_tc(lib, ref, Q, 10, w.budget)


@pytest.mark.parametrize("n,d,m,L", [
    (1, 3, 1, 8), (2, 5, 2, 1), (37, 9, 37, 17), (1000, 37, 7, 63), (1031, 64, 13, 64),
    (4099, 8, 64, 32), (5000, 130, 1, 24), (700, 190, 3, 16),
])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tc_ragged_shapes(N, n, d, m, L, dtype):
    items = rand_items(n, d, n + d + m + L, dtype=dtype)
    lib, ref = build_pair(items, dtype, m, L, seed=5, eps=0.2)
    Q = W.gen_queries(131, d, 7)
    for B in sorted({1, max(1, n // 3), n, n + 5}):
        check_queries_tc(lib, ref, Q, min(10, n + 2), B, check_hist=(B == 1))


def test_tc_duplicates_zero_vectors_and_zero_query(N):
    rng = np.random.default_rng(3)
    base = rng.standard_normal((20, 16)).astype(np.float32)
    items = np.concatenate([np.zeros((300, 16), np.float32), np.repeat(base, 40, axis=0)])
    rng.shuffle(items)
    lib, ref = build_pair(items, "f32", 16, 32, seed=9, eps=0.1)
    assert ref.U2[0] == 0.0
    Q = W.gen_queries(12, 16, 4)
    Q[0] = 0.0          # zero query: every bit is 1
    for B in (1, 50, 333, 1100):
        check_queries_tc(lib, ref, Q, 25, B)


@pytest.mark.parametrize("eps", [1e-9, 0.5, 0.9])
def test_tc_eps_extremes(N, eps):
    items = rand_items(3000, 24, 11)
    lib, ref = build_pair(items, "f32", 8, 32, seed=2, eps=eps)
    check_queries_tc(lib, ref, W.gen_queries(20, 24, 12), 10, 400)


def test_tc_whole_bucket_probing(N):
    items = rand_items(4000, 32, 21)
    lib, ref = build_pair(items, "f32", 8, 16, seed=3, eps=0.2)
    check_queries_tc(lib, ref, W.gen_queries(16, 32, 22), 10, 300, flags=N.NRLSH_WHOLE_BUCKETS)


def test_tc_budget_below_k_and_full_budget(N):
    from oracle import exact
    items = rand_items(2000, 20, 8)
    lib, ref = build_pair(items, "f32", 8, 32, seed=4, eps=0.1)
    Q = W.gen_queries(10, 20, 9)
    check_queries_tc(lib, ref, Q, 20, 7)
    ids, _ = N.nrlsh_query_ex(lib, torch.from_numpy(Q).cuda(), 10, 2000, flags=N.NRLSH_QUERY_TENSOR)
    assert np.array_equal(ids.cpu().numpy(), exact.brute_topk_fp64(items.astype(np.float64), Q, 10))


def test_tc_host_buffers_and_other_stream(N):
    """Host tensors are staged; a second stream waits for the index's sign matrix
    made on the first call's stream."""
    items = rand_items(3000, 40, 31)
    Q = W.gen_queries(16, 40, 32)
    lib, ref = build_pair(items, "f32", 8, 32, seed=7, eps=0.2)
    T = N.NRLSH_QUERY_TENSOR
    ids_h, sc_h = N.nrlsh_query_ex(lib, torch.from_numpy(Q), 10, 500, flags=T)
    assert ids_h.device.type == "cpu"
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ids_d, sc_d = N.nrlsh_query_ex(lib, torch.from_numpy(Q).cuda(), 10, 500, flags=T)
    s.synchronize()
    assert torch.equal(ids_h, ids_d.cpu()) and torch.equal(sc_h, sc_d.cpu())
    rids, rsc = O.query(ref, Q.astype(np.float64), 10, 500)
    assert np.array_equal(ids_h.numpy(), rids) and np.array_equal(sc_h.numpy(), rsc)


def _check_batched(ids, sc, ref, Q, ks, budgets):
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    ids = ids.cpu().numpy()
    sc = sc.cpu().numpy()
    for i in range(Q.shape[0]):
        k = int(ks[i])
        assert np.array_equal(ids[i, :k], rids[i, :k]), f"query {i}"
        assert np.array_equal(sc[i, :k], rsc[i, :k]), f"query {i}"
        assert np.all(ids[i, k:] == -1) and np.all(np.isneginf(sc[i, k:]))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tc_batched_uneven_budgets_and_k(N, dtype):
    n, d, m, L = 20_000, 48, 16, 64
    items = rand_items(n, d, 3, dtype=dtype)
    lib, ref = build_pair(items, dtype, m, L, seed=7, eps=0.2)
    Q = W.gen_queries(300, d, 11)
    budgets, ks = W.per_query_budgets_and_k(300, n, 0.001, 0.05, seed=12)
    k_max = int(ks.max())
    ids, sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                                    torch.from_numpy(budgets).cuda(), k_max, int(budgets.max()),
                                    flags=N.NRLSH_QUERY_TENSOR)
    torch.cuda.synchronize()
    _check_batched(ids, sc, ref, Q, ks, budgets)
    tun = N.nrlsh_get_tuning(lib)
    assert tun["rerank_tensor"]
    assert N.nrlsh_get_info(lib)["query_error"] == 0


def test_tc_batched_graph_replay_and_autotuned_choice(N):
    n, d, m, L = 12_000, 32, 8, 32
    items = rand_items(n, d, 5)
    lib, ref = build_pair(items, "f32", m, L, seed=3, eps=0.3)
    nq = 200
    rng = np.random.default_rng(1)
    Q1 = W.gen_queries(nq, d, 21)
    Q2 = W.gen_queries(nq, d, 22)
    budgets = rng.integers(1, 900, nq).astype(np.int64)
    ks = rng.integers(1, 25, nq).astype(np.int32)
    k_max, bmax = 24, 600                      # ks above k_max and budgets above bmax clamp
    s = torch.cuda.Stream()
    Qd = torch.from_numpy(Q1).cuda()
    ksd = torch.from_numpy(ks).cuda()
    bd = torch.from_numpy(budgets).cuda()
    ids = torch.empty((nq, k_max), dtype=torch.int64, device="cuda")
    sc = torch.empty((nq, k_max), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    flags = N.NRLSH_QUERY_GRAPH | N.NRLSH_QUERY_TENSOR
    with torch.cuda.stream(s):
        for _ in range(2):                     # capture, then replay
            N.nrlsh_query_batched(lib, Qd, ksd, bd, k_max, bmax, flags=flags, ids=ids, scores=sc)
    s.synchronize()
    ks_eff = np.minimum(ks, k_max)
    b_eff = np.minimum(budgets, bmax)
    _check_batched(ids, sc, ref, Q1, ks_eff, b_eff)
    Qd.copy_(torch.from_numpy(Q2))
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        N.nrlsh_query_batched(lib, Qd, ksd, bd, k_max, bmax, flags=flags, ids=ids, scores=sc)
    s.synchronize()
    _check_batched(ids, sc, ref, Q2, ks_eff, b_eff)
    # without a path restriction the autotuner picks one; the results are the same
    ids_a, sc_a = N.nrlsh_query_batched(lib, torch.from_numpy(Q2).cuda(), ksd, bd, k_max, bmax)
    torch.cuda.synchronize()
    assert torch.equal(ids_a, ids) and torch.equal(sc_a, sc)
    ids_f, sc_f = N.nrlsh_query_batched(lib, torch.from_numpy(Q2).cuda(), ksd, bd, k_max, bmax,
                                        flags=N.NRLSH_QUERY_FP32)
    torch.cuda.synchronize()
    assert torch.equal(ids_f, ids) and torch.equal(sc_f, sc)
    assert not N.nrlsh_get_tuning(lib)["rerank_tensor"]


def test_score_intervals_cover_worst_case_bf16_rounding(N):
    """Round to nearest bf16 (an 8-bit significand) moves a value by up to 2^-8 of
    itself.  Item 0's coordinates and the query's on them sit just below the
    midpoint 1 + 2^-8 (both round down); item 1's and the query's on them just
    above it (both round up), so the bf16 products err by about -2^-7 and +2^-7 in
    opposite directions while item 0's exact score is the larger by 2^-13.  An
    interval taken with 2^-9 per rounding puts item 0's entirely below item 1's
    and drops the true top-1 before the exact rescoring; both bf16 paths (tensor
    cores, and the FP32 re-rank over a bf16 copy of the rows) must return the
    oracle's top-2."""
    n, d = 1000, 129
    a = np.float32(1 + 2**-8 - 2**-20)
    b = np.float32(1 + 2**-8 + 2**-20)
    X = np.random.default_rng(5).standard_normal((n, d)).astype(np.float32) * np.float32(1e-3)
    X[0] = 0
    X[0, :64] = a
    X[0, 128] = np.float32(3 * 2**-13)
    X[1] = 0
    X[1, 64:128] = b
    q = np.zeros((1, d), np.float32)
    q[0, :64] = a
    q[0, 64:128] = b
    q[0, 128] = 1
    lib, ref = build_pair(X, "f32", 4, 32, 9, 0.1)
    rids, rsc = O.query(ref, q.astype(np.float64), 2, n)
    assert rids[0].tolist() == [0, 1]
    Qd = torch.from_numpy(q).cuda()
    ks = torch.full((1,), 2, dtype=torch.int32, device="cuda")
    bs = torch.full((1,), n, dtype=torch.int64, device="cuda")
    runs = {"tensor": N.nrlsh_query_ex(lib, Qd, 2, n, flags=N.NRLSH_QUERY_TENSOR),
            "fp32": N.nrlsh_query_ex(lib, Qd, 2, n)}
    runs["bf16_rows"] = N.nrlsh_query_batched(lib, Qd, ks, bs, 2, n,
                                              flags=N.NRLSH_QUERY_BF16 | N.NRLSH_QUERY_NO_TUNE)
    assert N.nrlsh_get_tuning(lib)["rows_bf16"]
    runs["tensor_batched"] = N.nrlsh_query_batched(lib, Qd, ks, bs, 2, n,
                                                   flags=N.NRLSH_QUERY_TENSOR | N.NRLSH_QUERY_NO_TUNE)
    torch.cuda.synchronize()
    for name, (ids, sc) in runs.items():
        assert ids.cpu().numpy().tolist() == rids.tolist(), name
        assert np.array_equal(sc.cpu().numpy(), rsc), name
