"""Batched queries (per-query probe budgets and k, persistent fused kernel,
autotuned tiles, CUDA-graph replay) against the CPU oracle, plus sampled
checks of a full-size ImageNet-shaped index."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair, check_index  # noqa: E402


@pytest.fixture(scope="module")
def N():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1809_08782_gb300.nrlsh as nrlsh
    return nrlsh


def rand_items(n, d, seed, dtype="f32"):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x32 = (x * rng.lognormal(0, 1.0, n)[:, None]).astype(np.float32)
    return W.bf16_bits_from_f32(x32) if dtype == "bf16" else x32


def check_batched(ids, sc, ref, Q, ks, budgets, k_max):
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    ids = ids.cpu().numpy()
    sc = sc.cpu().numpy()
    for i in range(Q.shape[0]):
        k = int(ks[i])
        assert np.array_equal(ids[i, :k], rids[i, :k]), f"query {i}"
        assert np.array_equal(sc[i, :k], rsc[i, :k]), f"query {i}"
        assert np.all(ids[i, k:] == -1) and np.all(np.isneginf(sc[i, k:]))


@pytest.mark.parametrize("path", ["auto", "bf16"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_uneven_budgets_and_k(N, dtype, path):
    n, d, m, L = 20_000, 48, 16, 64
    items = rand_items(n, d, 3, dtype)
    lib, ref = build_pair(items, dtype, m, L, seed=7, eps=0.2)
    check_index(lib, ref)
    Q = W.gen_queries(300, d, 11)
    budgets, ks = W.per_query_budgets_and_k(300, n, 0.001, 0.05, seed=12)
    k_max = int(ks.max())
    flags = {"auto": 0, "bf16": N.NRLSH_QUERY_BF16}[path]
    ids, sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                                    torch.from_numpy(budgets).cuda(), k_max, int(budgets.max()),
                                    flags=flags)
    torch.cuda.synchronize()
    check_batched(ids, sc, ref, Q, ks, budgets, k_max)
    tun = N.nrlsh_get_tuning(lib)
    assert tun["hist_queries_per_block"] in (32, 64, 128) and tun["ctas_per_sm"] in (1, 2, 4)
    if path == "bf16" and dtype == "f32":
        assert tun["rerank_tensor"] or tun["rows_bf16"]


def test_batched_graph_replay_and_clamping(N):
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
    with torch.cuda.stream(s):
        for _ in range(2):                     # capture, then replay
            N.nrlsh_query_batched(lib, Qd, ksd, bd, k_max, bmax, flags=N.NRLSH_QUERY_GRAPH,
                                  ids=ids, scores=sc)
    s.synchronize()
    ks_eff = np.minimum(ks, k_max)
    b_eff = np.minimum(budgets, bmax)
    check_batched(ids, sc, ref, Q1, ks_eff, b_eff, k_max)
    # the replay reads the buffers' current contents
    Qd.copy_(torch.from_numpy(Q2))
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        N.nrlsh_query_batched(lib, Qd, ksd, bd, k_max, bmax, flags=N.NRLSH_QUERY_GRAPH,
                              ids=ids, scores=sc)
    s.synchronize()
    check_batched(ids, sc, ref, Q2, ks_eff, b_eff, k_max)
    # the same results without the graph and from host buffers
    ids_h, sc_h = N.nrlsh_query_batched(lib, torch.from_numpy(Q2), torch.from_numpy(ks),
                                        torch.from_numpy(budgets), k_max, bmax)
    assert torch.equal(ids_h, ids.cpu()) and torch.equal(sc_h, sc.cpu())


def test_tuning_is_shared_by_indexes_of_the_same_shape(N):
    """The autotuner's choice is kept per device and index shape for the process: a
    rebuilt index of the same shape answers its first batched call without tuning
    again (far fewer launches) and with the same configuration and results."""
    n, d = 9_000, 48
    items = rand_items(n, d, 13)
    Q = torch.from_numpy(W.gen_queries(300, d, 14)).cuda()
    ks = torch.full((300,), 10, dtype=torch.int32, device="cuda")
    bs = torch.full((300,), 450, dtype=torch.int64, device="cuda")
    runs = []
    for _ in range(2):
        lib, _ = build_pair(items, "f32", 8, 32, seed=6, eps=0.2)
        torch.cuda.synchronize()
        c0 = N.nrlsh_launch_count()
        ids, sc = N.nrlsh_query_batched(lib, Q, ks, bs, 10, 450)
        torch.cuda.synchronize()
        runs.append((N.nrlsh_launch_count() - c0, N.nrlsh_get_tuning(lib), ids.cpu(), sc.cpu()))
        lib.free()
    (l0, t0, i0, s0), (l1, t1, i1, s1) = runs
    assert l1 < l0, (l0, l1)
    assert t0 == t1
    assert torch.equal(i0, i1) and torch.equal(s0, s1)


def test_batched_matches_single_query_path(N):
    n, d = 8_000, 64
    items = rand_items(n, d, 9)
    lib, _ = build_pair(items, "f32", 8, 32, seed=2, eps=0.2)
    Q = torch.from_numpy(W.gen_queries(64, d, 4)).cuda()
    ids1, sc1 = N.nrlsh_query_ex(lib, Q, 10, 333)
    ids2, sc2 = N.nrlsh_query_batched(lib, Q, torch.full((64,), 10, dtype=torch.int32).cuda(),
                                      torch.full((64,), 333, dtype=torch.int64).cuda(), 10, 333)
    torch.cuda.synchronize()
    assert torch.equal(ids1, ids2) and torch.equal(sc1, sc2)


def test_full_size_imagenet_shape_sampled(N):
    """n = 2,340,373, d = 150 bf16, Pareto(3) norms, m = 64, L = 64, tensor-core
    projection: the partition in full, codes of sampled items against the oracle,
    and properties of a batched query run that hold at any size."""
    w = W.make_workload("imagenet-n2340373-d150", with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, "bf16")
    X64 = W.items_to_f64(items, "bf16")
    eps = float(np.float32(0.2))
    lib = N.nrlsh_build_ex(W.to_torch(items, "bf16", "cuda"), w.m, w.L, w.index_seed, eps=eps,
                           projection=N.NRLSH_PROJECT_TENSOR)
    info = N.nrlsh_get_info(lib)
    assert info["device_error"] == 0
    # partition, in full
    s = O.sq_norms(X64)
    sub, U2, _, _ = O.partition(s, w.m)
    gsub, gU2, gs = N.nrlsh_get_partition(lib)
    assert np.array_equal(gs.numpy(), s)
    assert np.array_equal(gsub.numpy(), sub) and np.array_equal(gU2.numpy(), U2)
    # codes of sampled items
    A = N.nrlsh_get_projections(lib).numpy().astype(np.float64)
    from oracle import philox
    assert np.array_equal(A, philox.projections(w.index_seed, w.d, w.L))
    rng = np.random.default_rng(0)
    ids = rng.choice(w.n, 4000, replace=False)
    tau = O.tail_component(s, sub, U2)
    codes = N.nrlsh_get_codes(lib).numpy().view(np.uint64)
    assert np.array_equal(codes[ids], O.item_codes(X64[ids], A, tau[ids]))
    # a batched run: counts, padding and ordering properties
    nq = 512
    Q = W.gen_queries(nq, w.d, w.query_seed)
    budgets, ks = W.per_query_budgets_and_k(nq, w.n, 0.001, 0.05, seed=4000)
    k_max = 100
    out_ids, out_sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(),
                                            torch.from_numpy(ks).cuda(),
                                            torch.from_numpy(budgets).cuda(), k_max,
                                            int(budgets.max()))
    out_ids = out_ids.cpu().numpy()
    out_sc = out_sc.cpu().numpy()
    for i in range(0, nq, 37):
        k = int(ks[i])
        assert np.all(out_ids[i, :k] >= 0) and np.all(out_ids[i, k:] == -1)
        assert np.all(np.diff(out_sc[i, :k]) <= 0)              # best first
        # returned scores are the FP64 inner products rounded to fp32
        ref = O.scores_fp64(X64[out_ids[i, :k]], Q[i].astype(np.float64)).astype(np.float32)
        assert np.array_equal(out_sc[i, :k], ref)
    lib.free()
