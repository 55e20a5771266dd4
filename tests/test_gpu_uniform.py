"""Uniform norm-range partitioning (Section 5, Figure 3a) through the C ABI
against the oracle: sub-dataset of every item, U_j^2 (0 for empty ranges),
segment offsets, codes, bucket order, histograms, candidates and top-k, all
bit for bit, on both projection paths, with empty sub-datasets, equal norms,
zero vectors and ragged shapes."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair, check_index, check_queries  # noqa: E402

SIMT, TENSOR = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def rand_items(n, d, seed, sigma=1.0, dtype="f32"):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x32 = (x * rng.lognormal(0, sigma, n)[:, None]).astype(np.float32)
    return W.bf16_bits_from_f32(x32) if dtype == "bf16" else x32


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_yahoo_shape_uniform(dtype, proj):
    """n=136,736, d=300, lognormal(0, 1) norms, m=32, L=64: a long tail leaves the
    top ranges sparse or empty."""
    w = W.make_workload("yahoo-n136736-d300", nq=48, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, dtype)
    Q = W.gen_queries(w.nq, w.d, w.query_seed)
    lib, ref = build_pair(items, dtype, w.m, w.L, w.index_seed, 0.1, projection=proj,
                          partition="uniform")
    assert (np.diff(ref.bounds) == 0).any()          # this draw has empty ranges
    check_index(lib, ref, proj)
    check_queries(lib, ref, Q, 10, w.budget)


@pytest.mark.parametrize("n,d,m,L", [
    (1, 3, 1, 8), (2, 5, 2, 1), (37, 9, 37, 17), (1031, 64, 13, 64), (4099, 8, 64, 32),
    (9000, 300, 32, 32),
])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_ragged_shapes_uniform(n, d, m, L, dtype):
    items = rand_items(n, d, 3 * n + d + m + L, dtype=dtype)
    lib, ref = build_pair(items, dtype, m, L, seed=6, eps=0.2, projection=SIMT,
                          partition="uniform")
    check_index(lib, ref, SIMT)
    Q = W.gen_queries(7, d, 8)
    for B in sorted({1, max(1, n // 3), n, n + 5}):
        check_queries(lib, ref, Q, min(10, n + 2), B)


@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_gaps_zero_vectors_and_duplicates(proj):
    """Two norm clusters far apart (the ranges between them are empty), zero
    vectors (S_0) and repeated rows."""
    rng = np.random.default_rng(21)
    d = 24
    dirs = rng.standard_normal((600, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    norms = np.concatenate([rng.uniform(0.5, 1.0, 300), rng.uniform(20.0, 25.0, 300)])
    items = (dirs * norms[:, None]).astype(np.float32)
    items = np.concatenate([items, np.zeros((50, d), np.float32), np.repeat(items[:10], 20, 0)])
    rng.shuffle(items)
    lib, ref = build_pair(items, "f32", 16, 32, seed=4, eps=0.1, projection=proj,
                          partition="uniform")
    assert (np.diff(ref.bounds) == 0).sum() >= 8
    check_index(lib, ref, proj)
    Q = W.gen_queries(10, d, 5)
    for B in (1, 77, 400, 850):
        check_queries(lib, ref, Q, 12, B)


def test_equal_norms_put_everything_in_the_first_range():
    rng = np.random.default_rng(2)
    base = rng.standard_normal(16).astype(np.float32)
    items = (rng.choice([-1.0, 1.0], size=(700, 16)) * base[None, :]).astype(np.float32)
    assert len(set(O.sq_norms(items.astype(np.float64)))) == 1
    lib, ref = build_pair(items, "f32", 8, 16, seed=3, eps=0.2, partition="uniform")
    import paper_1809_08782_gb300.nrlsh as N
    assert N.nrlsh_get_segments(lib).tolist() == [0] + [700] * 8
    sub, _, _ = N.nrlsh_get_partition(lib)
    assert np.all(sub.numpy() == 0)
    check_index(lib, ref)
    check_queries(lib, ref, W.gen_queries(6, 16, 1), 10, 100)


def test_batched_and_whole_buckets_on_uniform_index():
    import paper_1809_08782_gb300.nrlsh as N
    items = rand_items(20_000, 48, 14)
    lib, ref = build_pair(items, "f32", 16, 64, seed=7, eps=0.2, partition="uniform")
    check_index(lib, ref)
    Q = W.gen_queries(200, 48, 15)
    check_queries(lib, ref, Q[:16], 10, 300, flags=N.NRLSH_WHOLE_BUCKETS)
    budgets, ks = W.per_query_budgets_and_k(200, 20_000, 0.001, 0.05, seed=16)
    k_max = int(ks.max())
    ids, sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                                    torch.from_numpy(budgets).cuda(), k_max, int(budgets.max()))
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    ids = ids.cpu().numpy()
    sc = sc.cpu().numpy()
    for i in range(200):
        k = int(ks[i])
        assert np.array_equal(ids[i, :k], rids[i, :k]), i
        assert np.array_equal(sc[i, :k], rsc[i, :k]), i


def test_info_reports_the_partition():
    import paper_1809_08782_gb300.nrlsh as N
    items = rand_items(500, 8, 1)
    lib, _ = build_pair(items, "f32", 4, 8, seed=1, eps=0.1, partition="uniform")
    assert N.nrlsh_get_info(lib)["partition"] == N.NRLSH_PARTITION_UNIFORM
    lib2, _ = build_pair(items, "f32", 4, 8, seed=1, eps=0.1)
    assert N.nrlsh_get_info(lib2)["partition"] == N.NRLSH_PARTITION_PERCENTILE
    with pytest.raises(N.NrlshError):
        N.nrlsh_build_ex(torch.from_numpy(items).cuda(), 4, 8, 1, partition=7)
