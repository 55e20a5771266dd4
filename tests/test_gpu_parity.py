"""GPU (through the C ABI) versus the CPU oracle, element by element.

Codes, partitions, bucket order, query codes, Hamming histograms, candidate
lists and top-k ids must be identical; returned scores are the FP64 inner
product rounded to fp32 on both sides, so they must be identical too (a tighter
bar than the 1e-5 relative tolerance allowed for FP32 scores)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair, check_index, check_queries, f32  # noqa: E402


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


def rand_q(nq, d, seed):
    return W.gen_queries(nq, d, seed)


# ------------------------------------------------------------ presets

SIMT, TENSOR = 1, 2


@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_small_preset_full(proj):
    """n=10,000, d=64 fp32, m=8, L=16, 1,000 queries, B=1,000, top-10."""
    w = W.make_workload("small-n10k-d64")
    lib, ref = build_pair(w.items, w.dtype, w.m, w.L, w.index_seed, 0.1, projection=proj)
    check_index(lib, ref, proj)
    check_queries(lib, ref, w.queries[:300], w.k, w.budget)
    check_queries(lib, ref, w.queries, w.k, w.budget, check_hist=False)


@pytest.mark.parametrize("frac,proj", [(0.01, SIMT), (0.03, TENSOR), (0.20, SIMT)])
def test_netflix_preset(frac, proj):
    """n=17,770, d=300 fp32, m=32, L=32; budget swept 1%..20% of n."""
    w = W.make_workload("netflix-n17770-d300", nq=200)
    lib, ref = build_pair(w.items, w.dtype, w.m, w.L, w.index_seed, 0.3, projection=proj)
    check_index(lib, ref, proj)
    check_queries(lib, ref, w.queries, w.k, int(round(frac * w.n)))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_yahoo_preset(dtype, proj):
    """n=136,736, d=300, m=32, L=64, stored fp32 and bf16; a 64-query subset."""
    w = W.make_workload("yahoo-n136736-d300", nq=64, with_data=False)
    items = W.gen_items(w.n, w.d, w.item_seed, w.norm_dist, w.norm_param, dtype)
    Q = W.gen_queries(w.nq, w.d, w.query_seed)
    lib, ref = build_pair(items, dtype, w.m, w.L, w.index_seed, 0.1, projection=proj)
    check_index(lib, ref, proj)
    check_queries(lib, ref, Q, 10, w.budget)


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("n,d,m,L", [
    (1, 3, 1, 8), (2, 5, 2, 1), (37, 9, 37, 17), (1000, 37, 7, 63), (1031, 64, 13, 64),
    (4099, 8, 64, 32), (5000, 130, 1, 24),
])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_ragged_shapes(n, d, m, L, dtype, proj):
    items = rand_items(n, d, n + d + m + L, dtype=dtype)
    lib, ref = build_pair(items, dtype, m, L, seed=5, eps=0.2, projection=proj)
    check_index(lib, ref, proj)
    Q = rand_q(9, d, 7)
    for B in sorted({1, max(1, n // 3), n, n + 5}):
        check_queries(lib, ref, Q, min(10, n + 2), B)


@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_duplicates_zero_vectors_and_zero_subdatasets(proj):
    rng = np.random.default_rng(3)
    base = rng.standard_normal((20, 16)).astype(np.float32)
    items = np.concatenate([np.zeros((300, 16), np.float32), np.repeat(base, 40, axis=0)])
    rng.shuffle(items)
    lib, ref = build_pair(items, "f32", 16, 32, seed=9, eps=0.1, projection=proj)
    assert ref.U2[0] == 0.0
    check_index(lib, ref, proj)
    Q = rand_q(12, 16, 4)
    Q[0] = 0.0          # zero query: every bit is 1
    for B in (1, 50, 333, 1100):
        check_queries(lib, ref, Q, 25, B)


@pytest.mark.parametrize("eps", [1e-9, 0.5, 0.9])
def test_eps_extremes(eps):
    items = rand_items(3000, 24, 11)
    lib, ref = build_pair(items, "f32", 8, 32, seed=2, eps=eps)
    check_index(lib, ref)
    check_queries(lib, ref, rand_q(20, 24, 12), 10, 400)


def test_whole_bucket_probing():
    items = rand_items(4000, 32, 21)
    lib, ref = build_pair(items, "f32", 8, 16, seed=3, eps=0.2)
    import paper_1809_08782_gb300.nrlsh as N
    check_queries(lib, ref, rand_q(16, 32, 22), 10, 300, flags=N.NRLSH_WHOLE_BUCKETS)


def test_budget_below_k_pads_with_minus_one():
    items = rand_items(500, 16, 5)
    lib, ref = build_pair(items, "f32", 4, 16, seed=3, eps=0.1)
    check_queries(lib, ref, rand_q(5, 16, 6), 20, 7)


def test_full_budget_is_exact_mips():
    from oracle import exact
    items = rand_items(2000, 20, 8)
    lib, ref = build_pair(items, "f32", 8, 32, seed=4, eps=0.1)
    Q = rand_q(10, 20, 9)
    import paper_1809_08782_gb300.nrlsh as N
    ids, _ = N.nrlsh_query_ex(lib, torch.from_numpy(Q).cuda(), 10, 2000)
    truth = exact.brute_topk_fp64(items.astype(np.float64), Q, 10)
    assert np.array_equal(ids.cpu().numpy(), truth)


def test_host_buffers_and_streams():
    """CPU tensors are staged by the library; a side stream gives the same result."""
    import paper_1809_08782_gb300.nrlsh as N
    items = rand_items(3000, 40, 31)
    Q = rand_q(16, 40, 32)
    eps = f32(0.2)
    lib_h = N.nrlsh_build_ex(torch.from_numpy(items), 8, 32, 7, eps=eps)
    lib_d = N.nrlsh_build_ex(torch.from_numpy(items).cuda(), 8, 32, 7, eps=eps)
    assert torch.equal(N.nrlsh_get_codes(lib_h), N.nrlsh_get_codes(lib_d))
    ids_h, sc_h = N.nrlsh_query_ex(lib_h, torch.from_numpy(Q), 10, 500)
    assert ids_h.device.type == "cpu"
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ids_d, sc_d = N.nrlsh_query_ex(lib_d, torch.from_numpy(Q).cuda(), 10, 500)
    s.synchronize()
    assert torch.equal(ids_h, ids_d.cpu()) and torch.equal(sc_h, sc_d.cpu())
    ids_s, sc_s = N.nrlsh_query(lib_d, torch.from_numpy(Q).cuda(), 10, 500)
    torch.cuda.synchronize()
    assert torch.equal(ids_s.cpu(), ids_h)


def test_async_host_input_build_and_device_outputs_of_host_queries():
    """NRLSH_BUILD_ASYNC_INPUT: the build returns with the pinned items' copy still
    queued on its stream; host queries with device outputs return once the queries
    have landed (with NRLSH_QUERY_ASYNC_INPUT, at once).  All give what the
    synchronous calls give, on two streams."""
    import paper_1809_08782_gb300.nrlsh as N
    items = rand_items(3000, 40, 33)
    Q = rand_q(16, 40, 34)
    eps = f32(0.2)
    ref = N.nrlsh_build_ex(torch.from_numpy(items).cuda(), 8, 32, 7, eps=eps)
    ids_r, sc_r = N.nrlsh_query_ex(ref, torch.from_numpy(Q).cuda(), 10, 500)
    torch.cuda.synchronize()
    Xh = torch.from_numpy(items).pin_memory()
    Qh = torch.from_numpy(Q).pin_memory()
    sb, sq = torch.cuda.Stream(), torch.cuda.Stream()
    ix = N.nrlsh_build_ex(Xh, 8, 32, 7, eps=eps, stream=sb, build_flags=N.NRLSH_BUILD_ASYNC_INPUT)
    ids = torch.empty((16, 10), dtype=torch.int64, device="cuda")
    sc = torch.empty((16, 10), dtype=torch.float32, device="cuda")
    N.nrlsh_query_ex(ix, Qh, 10, 500, ids=ids, scores=sc, stream=sq)
    sq.synchronize()
    assert torch.equal(N.nrlsh_get_codes(ix), N.nrlsh_get_codes(ref))
    assert torch.equal(ids, ids_r) and torch.equal(sc, sc_r)
    ks = torch.full((16,), 10, dtype=torch.int32)
    bs = torch.full((16,), 500, dtype=torch.int64)
    ids_b = torch.empty((16, 10), dtype=torch.int64, device="cuda")
    sc_b = torch.empty((16, 10), dtype=torch.float32, device="cuda")
    N.nrlsh_query_batched(ix, Qh, ks, bs, 10, 500, ids=ids_b, scores=sc_b, stream=sq)
    sq.synchronize()
    assert torch.equal(ids_b, ids_r) and torch.equal(sc_b, sc_r)
    # NRLSH_QUERY_ASYNC_INPUT: the queries' copy is left queued on the stream
    ids_a = torch.empty_like(ids)
    sc_a = torch.empty_like(sc)
    N.nrlsh_query_ex(ix, Qh, 10, 500, flags=N.NRLSH_QUERY_ASYNC_INPUT, ids=ids_a, scores=sc_a,
                     stream=sq)
    ids_c = torch.empty_like(ids_b)
    sc_c = torch.empty_like(sc_b)
    N.nrlsh_query_batched(ix, Qh, ks, bs, 10, 500, flags=N.NRLSH_QUERY_ASYNC_INPUT, ids=ids_c,
                          scores=sc_c, stream=sq)
    sq.synchronize()
    assert torch.equal(ids_a, ids_r) and torch.equal(sc_a, sc_r)
    assert torch.equal(ids_c, ids_r) and torch.equal(sc_c, sc_r)


def test_empty_query_batch_and_launch_count():
    import paper_1809_08782_gb300.nrlsh as N
    items = rand_items(100, 8, 1)
    lib, _ = build_pair(items, "f32", 2, 8, 1, 0.1)
    before = N.nrlsh_launch_count()
    ids, sc = N.nrlsh_query_ex(lib, torch.zeros((0, 8), device="cuda"), 5, 10)
    assert ids.shape == (0, 5) and N.nrlsh_launch_count() == before
    N.nrlsh_query_ex(lib, torch.zeros((2, 8), device="cuda"), 5, 10)
    assert N.nrlsh_launch_count() > before


@pytest.mark.parametrize("n,m", [
    (65_536, 16),     # 64 tiles, ranges of 4,096: the tile-rank path at its limits
    (65_537, 17),     # 65 tiles: the radix path
    (40_000, 9),      # ranges of 4,445: the radix path
    (1_000, 900),     # ranges of one or two items
])
def test_ranking_paths_and_their_limits(n, m):
    rng = np.random.default_rng(n + m)
    items = rand_items(n, 16, n + 3 * m)
    items[rng.choice(n, n // 5, replace=False)] = items[0]     # many equal norms
    lib, ref = build_pair(items, "f32", m, 16, seed=5, eps=0.2, projection=SIMT)
    check_index(lib, ref, SIMT)
    check_queries(lib, ref, rand_q(8, 16, 3), 10, 700)


@pytest.mark.parametrize("d,L", [(1000, 64), (1000, 32), (1030, 16), (700, 64)])
def test_wide_rows(d, L):
    """Rows up to 1,024 columns go through the warp-per-row projection while A^T
    fits in shared memory (L = 32 at d = 1,000), else through the register-tiled
    one (L = 64 at d = 1,000; d > 1,024)."""
    items = rand_items(2500, d, d + L)
    lib, ref = build_pair(items, "f32", 8, L, seed=3, eps=0.2, projection=SIMT)
    check_index(lib, ref, SIMT)
    check_queries(lib, ref, rand_q(6, d, 4), 10, 300)


def _window_tie_row(t, d=15):
    """A row built for the squared-norm kernels' 128-bit window: W0 = top +
    bitlen(d) + 1 - 128 with top = 1 for the term 1.0 (W0 = -122 for
    8 <= d <= 15, even whenever bitlen(d) is).  The in-window part is
    1 + 2^-53 - 2^W0 (one unit below the half-way point); t terms of 2^(W0 - 2)
    each (dropped by the window) decide it."""
    import math
    W0 = 1 + d.bit_length() + 1 - 128
    assert W0 % 2 == 0
    row = [1.0, 11863283 * 2.0 ** -50]
    rem = 4817239 * 2 ** (-100 - W0) - 1                # in units of 2^W0
    while rem > 0:
        j = max(0, (rem.bit_length() - 46) // 2)       # M^2 = rem / 4^j below 2^48
        M = min(math.isqrt(rem // 4 ** j), 2 ** 24 - 1)
        row.append(M * 2.0 ** (j + W0 // 2))
        rem -= M * M * 4 ** j
    row += [2.0 ** ((W0 - 2) // 2)] * t
    assert len(row) <= d
    row += [0.0] * (d - len(row))
    return np.array(row, dtype=np.float32)


@pytest.mark.parametrize("d", [
    15,     # a warp per row, one value per load
    32,     # 16 lanes per row, 2 groups of 4 per lane
    200,    # 16 lanes per row, 4 groups per lane
    512,    # 16 lanes per row at its limit, 8 groups per lane
    516,    # a warp per row, four values per load
])
def test_exact_squared_norms_and_the_slow_path(d):
    """s_x is the exact sum of squares rounded once: rows with a wide exponent
    range, rows of subnormal values (alone and beside normal ones), and rows built
    to land next to a rounding tie inside the kernels' window (those take the
    exact slow path), against the oracle."""
    from oracle import nrlsh as O
    import paper_1809_08782_gb300.nrlsh as N
    rng = np.random.default_rng(77 + d)
    wide = (rng.standard_normal((500, d)) * 2.0 ** rng.integers(-60, 60, (500, d))).astype(np.float32)
    ties = np.stack([_window_tie_row(t, d) for t in (0, 3, 4, 5, 9)] * 4)
    sub = (rng.standard_normal((6, d)) * 2.0 ** -135).astype(np.float32)
    sub[3:, 0] = 2.0 ** -125                                 # one normal value beside them
    assert np.all(np.abs(sub[:3]) < 2.0 ** -126) and np.any(sub[:3] != 0)
    items = np.concatenate([wide, ties, sub, np.zeros((3, d), np.float32)])
    s_ref = O.sq_norms(items.astype(np.float64))
    assert list(s_ref[500:505]) == [1.0, 1.0, 1.0, 1.0 + 2.0 ** -52, 1.0 + 2.0 ** -52]
    lib = N.nrlsh_build_ex(torch.from_numpy(items).cuda(), 4, 16, 3, eps=f32(0.2),
                           projection=SIMT)
    _, _, s = N.nrlsh_get_partition(lib)
    assert np.array_equal(s.numpy(), s_ref)
    assert N.nrlsh_get_info(lib)["norm_fallbacks"] >= 12   # the tie rows with t > 0


def _hyperplane_queries(A, d, bits, seed):
    """Queries on and next to the hyperplanes a_b^T q = 0 (Eq. 4 with P(q) = [q; 0]):
    q_k1 = a_k2b, q_k2 = -a_k1b (bf16 values, so q^T a_b = 0 exactly) plus
    delta at k3 > k2 with |delta a_k3b| = r ||q|| ||a_b||.  r = 0 and 2^-60 reach the
    canonical sequential sum, 2^-42 the FP64 tier, 2^-30 the compensated FP32
    tier; in-order partial sums are exact here, so the canonical sign is the
    exact one."""
    rng = np.random.default_rng(seed)
    rows = []
    for b in bits:
        for r in (0.0, 2.0 ** -60, 2.0 ** -42, 2.0 ** -30):
            for sign in (1.0, -1.0):
                k1, k2, k3 = sorted(rng.choice(d, 3, replace=False))
                q = np.zeros(d)
                q[k1], q[k2] = A[k2, b], -A[k1, b]
                scale = np.linalg.norm(q) * np.linalg.norm(A[:d, b])
                q[k3] = np.float32(sign * r * scale / A[k3, b])
                rows.append(q)
    return np.array(rows, dtype=np.float32)


@pytest.mark.parametrize("proj", [SIMT, TENSOR])
def test_code_bits_on_and_near_the_hyperplanes(proj):
    """Bits that only the later precision tiers can decide: query codes on and
    next to a_b^T q = 0, and an item with a_b^T x = 0 exactly and tau = 0 (the
    largest norm, so U = ||x||): its canonical value is 0 and the bit is 1."""
    import paper_1809_08782_gb300.nrlsh as N
    from oracle import nrlsh as O, philox
    d, L, seed = 40, 32, 9
    A = philox.projections(seed, d, L)
    items = rand_items(300, d, 5)
    planted = np.zeros(d, np.float32)
    planted[3], planted[17] = A[17, 0] * 64.0, -A[3, 0] * 64.0
    assert np.linalg.norm(planted) > np.linalg.norm(items, axis=1).max()
    items = np.concatenate([items, planted[None, :]])
    lib, ref = build_pair(items, "f32", 4, L, seed, 0.2, projection=proj)
    assert np.array_equal(ref.A, A)
    check_index(lib, ref, proj)
    assert int(ref.codes[300]) & 1                       # canonical value 0 -> bit 1
    Q = _hyperplane_queries(A, d, [0, 5, 31], 11)
    got = N.nrlsh_hash_queries(lib, torch.from_numpy(Q).cuda()).cpu().numpy().view(np.uint64)
    want = O.query_codes(Q.astype(np.float64), A)
    assert np.array_equal(got, want)
    check_queries(lib, ref, Q, 5, 120)


def test_queries_opposite_to_every_item():
    """Queries opposite to a tight cluster of items: every item matches few bits,
    so the walk reaches the buckets of few matching bits before it has B items.
    Results equal the oracle's, through the single-budget and the batched entry
    points."""
    import paper_1809_08782_gb300.nrlsh as N
    from oracle import nrlsh as O
    rng = np.random.default_rng(41)
    d = 24
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    items = (u[None, :] + 0.05 * rng.standard_normal((3000, d))) * rng.lognormal(0, 0.5, (3000, 1))
    items = items.astype(np.float32)
    lib, ref = build_pair(items, "f32", 8, 32, seed=3, eps=0.2)
    check_index(lib, ref)
    Q = np.concatenate([np.tile(-u, (6, 1)) + 0.01 * rng.standard_normal((6, d)),
                        rng.standard_normal((6, d))]).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    for B in (1, 40, 700):
        check_queries(lib, ref, Q, 10, B)
    ks = np.array([10] * 12, np.int32)
    budgets = np.array([40, 700, 5, 3000, 1, 90] * 2, np.int64)
    ids, sc = N.nrlsh_query_batched(lib, torch.from_numpy(Q).cuda(), torch.from_numpy(ks).cuda(),
                                    torch.from_numpy(budgets).cuda(), 10, int(budgets.max()))
    rids, rsc = O.query(ref, Q.astype(np.float64), ks, budgets)
    assert np.array_equal(ids.cpu().numpy(), rids) and np.array_equal(sc.cpu().numpy(), rsc)


@pytest.mark.parametrize("L", [16, 64])
def test_bucket_stats_count_sub_dataset_code_pairs(L):
    """curves.bucket_stats (the bucket-balance figures of Sections 3.1-3.2) equals a
    count of the distinct (sub-dataset, code) pairs of the oracle's index, for
    codes of all 64 bits too."""
    from paper_1809_08782_gb300 import curves
    items = rand_items(6000, 24, 41)
    lib, ref = build_pair(items, "f32", 16, L, seed=4, eps=0.2)
    got = curves.bucket_stats(lib)
    pairs = {}
    for j, c in zip(ref.sub.tolist(), ref.codes.tolist()):
        pairs[(j, c)] = pairs.get((j, c), 0) + 1
    assert got == {"buckets": len(pairs), "largest_bucket": max(pairs.values())}
