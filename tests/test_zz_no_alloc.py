"""nrlsh_query_noalloc: the query path for callers that cannot allocate device
memory while they query (for instance a serving process whose GPU memory is held
by another allocator).  It must return exactly what nrlsh_query_ex returns, on
consecutive calls that reuse the library's one fixed scratch array.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1809_08782_gb300.nrlsh as nrlsh
    return nrlsh


def _items(n, d, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return torch.from_numpy((x * rng.lognormal(0, 0.8, n)[:, None]).astype(np.float32))


def _queries(nq, d, seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((nq, d))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return torch.from_numpy(q.astype(np.float32)).cuda()


@pytest.mark.parametrize("n,d,m,L,nq,k,budget", [
    (20_000, 48, 16, 32, 700, 10, 900),        # one chunk
    (200_000, 16, 8, 16, 40, 25, 100_000),     # several chunks of the 32 MiB array
])
def test_noalloc_matches_query_ex_on_consecutive_calls(N, n, d, m, L, nq, k, budget):
    idx = N.nrlsh_build_ex(_items(n, d, n).cuda(), m, L, 11, eps=float(np.float32(0.2)))
    Q = _queries(nq, d, 5)
    ref_ids, ref_sc = N.nrlsh_query_ex(idx, Q, k, budget)
    for _ in range(2):
        ids = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
        sc = torch.full((nq, k), 7.0, dtype=torch.float32, device="cuda")
        N.nrlsh_query_noalloc(idx, Q, k, budget, ids, sc)
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        assert torch.equal(sc, ref_sc)
    idx.free()


def test_noalloc_rejects_oversized_budget_and_host_pointers(N):
    idx = N.nrlsh_build_ex(_items(1_500_000, 4, 3).cuda(), 1, 8, 2)
    Q = _queries(2, 4, 1)
    ids = torch.empty((2, 5), dtype=torch.int64, device="cuda")
    sc = torch.empty((2, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(N.NrlshError) as e:
        N.nrlsh_query_noalloc(idx, Q, 5, 1_500_000, ids, sc)
    assert e.value.status == -1 and "32 MiB" in str(e.value)
    with pytest.raises(ValueError):                  # the binding refuses host queries
        N.nrlsh_query_noalloc(idx, Q.cpu(), 5, 100, ids.cpu(), sc.cpu())
    # and so does the C entry point itself, before any work is queued
    import ctypes
    Qh = Q.cpu().contiguous()
    st = N.load().nrlsh_query_noalloc(idx.handle, ctypes.c_void_p(Qh.data_ptr()), 2, 5, 100,
                                      ctypes.c_void_p(ids.data_ptr()),
                                      ctypes.c_void_p(sc.data_ptr()), None)
    assert st == -1 and "device pointers" in N.nrlsh_last_error()
    N.nrlsh_query_noalloc(idx, Q, 5, 1000, ids, sc)    # a budget that fits still works
    ref_ids, _ = N.nrlsh_query_ex(idx, Q, 5, 1000)
    torch.cuda.synchronize()
    assert torch.equal(ids, ref_ids)
    idx.free()
