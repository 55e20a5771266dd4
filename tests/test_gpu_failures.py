"""Failure detection without a GPU fault: the tensor-core kernels' bounded waits
are made to run out on purpose (the NRLSH_TEST_SPIN_FIRST hook gives the MMA
thread's first wait zero polls), and the library must report NRLSH_ERR_TIMEOUT
while the context stays usable: the next index and query on the same device
give the oracle's results."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import nrlsh as O  # noqa: E402
from paper_1809_08782_gb300 import workloads as W  # noqa: E402

HOOK = "NRLSH_TEST_SPIN_FIRST"


@pytest.fixture(scope="module")
def N():
    from paper_1809_08782_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1809_08782_gb300.nrlsh as nrlsh
    return nrlsh


@pytest.fixture()
def hook():
    os.environ[HOOK] = "0"
    yield
    os.environ.pop(HOOK, None)


def _data():
    w = W.make_workload("small-n10k-d64", n=4000, nq=40)
    return w, torch.from_numpy(w.items).cuda(), torch.from_numpy(w.queries).cuda()


def _still_works(N, w, X, Q):
    eps = float(np.float32(0.2))
    lib = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=eps, projection=N.NRLSH_PROJECT_TENSOR)
    ids, sc = N.nrlsh_query_ex(lib, Q, 10, 400, flags=N.NRLSH_QUERY_TENSOR)
    ref = O.build(W.items_to_f64(w.items, w.dtype), w.m, w.L, w.index_seed, eps=eps)
    rids, rsc = O.query(ref, w.queries.astype(np.float64), 10, 400)
    assert np.array_equal(ids.cpu().numpy(), rids) and np.array_equal(sc.cpu().numpy(), rsc)
    info = N.nrlsh_get_info(lib)
    assert info["device_error"] == 0 and info["query_error"] == 0


def test_projection_wait_that_runs_out_is_reported(N, hook):
    w, X, Q = _data()
    lib = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=float(np.float32(0.2)),
                           projection=N.NRLSH_PROJECT_TENSOR)
    info = N.nrlsh_get_info(lib, check=False)
    assert info["device_error"] != 0
    with pytest.raises(N.NrlshError) as e:
        N.nrlsh_get_info(lib)
    assert e.value.status == -4
    with pytest.raises(N.NrlshError) as e:
        N.nrlsh_get_codes(lib)
    assert e.value.status == -4
    lib.free()
    os.environ.pop(HOOK)
    _still_works(N, w, X, Q)


def test_tensor_query_wait_that_runs_out_is_reported(N, hook):
    w, X, Q = _data()
    os.environ.pop(HOOK)
    lib = N.nrlsh_build_ex(X, w.m, w.L, w.index_seed, eps=float(np.float32(0.2)))
    assert N.nrlsh_get_info(lib)["query_error"] == 0
    os.environ[HOOK] = "0"
    N.nrlsh_query_ex(lib, Q, 10, 400, flags=N.NRLSH_QUERY_TENSOR)
    torch.cuda.synchronize()
    info = N.nrlsh_get_info(lib, check=False)
    assert info["query_error"] != 0 and info["device_error"] == 0
    with pytest.raises(N.NrlshError) as e:
        N.nrlsh_get_info(lib)
    assert e.value.status == -4
    lib.free()
    os.environ.pop(HOOK)
    _still_works(N, w, X, Q)
