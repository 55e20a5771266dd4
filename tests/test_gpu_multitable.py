"""Multi-table single probe (Algorithm 2 with T tables of L/T bits) through the C
ABI against the oracle: candidate sets in storage order, probed counts, top-k ids
and scores bit for bit, the cap, host buffers, and the extreme table counts."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import multitable as MT, nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402
from tests.parity import build_pair  # noqa: E402


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


def check(N, lib, ref, Q, T, k, cap=0):
    Qd = torch.from_numpy(Q).cuda()
    cand, count = N.nrlsh_multitable_candidates(lib, Qd, T)
    cand = cand.cpu().numpy()
    count = count.cpu().numpy()
    cqs = O.query_codes(Q.astype(np.float64), ref.A)
    for i in range(Q.shape[0]):
        exp = MT.candidates(ref, int(cqs[i]), T)
        assert count[i] == exp.size, (T, i)
        assert np.array_equal(cand[i, :exp.size], exp), (T, i)
    ids, sc, probed = N.nrlsh_query_multitable(lib, Qd, T, k, max_candidates=cap)
    rids, rsc, rprobed = MT.query(ref, Q.astype(np.float64), k, T, cap=cap)
    assert np.array_equal(probed.cpu().numpy(), rprobed)
    assert np.array_equal(ids.cpu().numpy(), rids), T
    assert np.array_equal(sc.cpu().numpy(), rsc), T


@pytest.mark.parametrize("T", [1, 2, 4, 8, 16, 32])
def test_netflix_shape_tables(N, T):
    """n=17,770, d=300 fp32, m=32, L=32 read as T tables."""
    w = W.make_workload("netflix-n17770-d300", nq=40)
    lib, ref = build_pair(w.items, w.dtype, w.m, w.L, w.index_seed, 0.3)
    check(N, lib, ref, w.queries, T, 10)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("L,T", [(64, 1), (64, 4), (64, 16), (64, 64), (48, 6), (7, 7), (1, 1)])
def test_code_widths_and_dtypes(N, dtype, L, T):
    items = rand_items(6000, 40, L * 10 + T, dtype=dtype)
    lib, ref = build_pair(items, dtype, 16, L, seed=3, eps=0.2)
    check(N, lib, ref, W.gen_queries(24, 40, 2), T, 7)


@pytest.mark.parametrize("partition", ["percentile", "uniform"])
def test_cap_and_simple_lsh(N, partition):
    items = rand_items(8000, 32, 5)
    for m in (1, 8):             # m = 1: SIMPLE-LSH's single table set
        lib, ref = build_pair(items, "f32", m, 32, seed=4, eps=0.2, partition=partition)
        Q = W.gen_queries(20, 32, 6)
        check(N, lib, ref, Q, 8, 10)
        check(N, lib, ref, Q, 8, 10, cap=25)
        check(N, lib, ref, Q, 32, 10, cap=1)


def test_no_candidates_pads_and_host_buffers(N):
    items = rand_items(300, 16, 7)
    lib, ref = build_pair(items, "f32", 4, 64, seed=8, eps=0.2)
    Q = W.gen_queries(30, 16, 9)
    ids, sc, probed = N.nrlsh_query_multitable(lib, torch.from_numpy(Q), 1, 5)  # host in and out
    rids, rsc, rprobed = MT.query(ref, Q.astype(np.float64), 5, 1)
    assert (rprobed == 0).any()              # 64-bit single table: most queries probe nothing
    assert np.array_equal(probed.numpy(), rprobed)
    assert np.array_equal(ids.numpy(), rids) and np.array_equal(sc.numpy(), rsc)
    with pytest.raises(N.NrlshError):
        N.nrlsh_query_multitable(lib, torch.from_numpy(Q).cuda(), 3, 5)   # 64 % 3 != 0
