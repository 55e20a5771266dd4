"""The C-ABI library builds, loads and exports every entry point that
include/nrlsh.h declares; argument errors are reported before any GPU work
(so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nrlsh.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"NRLSH_API\s+[\w\s\*]+?\b(nrlsh_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_08782_gb300 import build
    build.build()
    import paper_1809_08782_gb300.nrlsh as N
    return N.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("nrlsh_build", "nrlsh_query", "nrlsh_build_ex", "nrlsh_query_ex",
                     "nrlsh_free", "nrlsh_last_error", "nrlsh_get_codes"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_exactly_the_header():
    import paper_1809_08782_gb300.nrlsh as N
    assert sorted(N.SIGNATURES) == header_functions()


def test_exports_are_only_the_c_abi(lib):
    out = os.popen(f"nm -D --defined-only {lib._name}").read().split("\n")
    syms = {line.split()[-1] for line in out if line.strip() and " T " in line}
    ours = {s for s in syms if s.startswith("nrlsh_")}
    assert ours == set(header_functions())


def _build(lib, items, n, d, m, L, seed=1, dtype=0, eps=0.1):
    out = ctypes.c_void_p()
    st = lib.nrlsh_build_ex(items, n, d, m, L, seed, dtype, eps, None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("n,d,m,L,eps,dtype", [
    (0, 4, 1, 8, 0.1, 0),       # n < 1
    (10, 0, 1, 8, 0.1, 0),      # d < 1
    (10, 4, 11, 8, 0.1, 0),     # m > n
    (10, 4, 0, 8, 0.1, 0),      # m < 1
    (10, 4, 2, 0, 0.1, 0),      # L < 1
    (10, 4, 2, 65, 0.1, 0),     # L > 64
    (100000, 4, 300, 64, 0.1, 0),  # m (L+1) > 16384
    (10, 4, 2, 8, 0.0, 0),      # eps <= 0
    (10, 4, 2, 8, 1.0, 0),      # eps >= 1
    (10, 4, 2, 8, 0.1, 7),      # unknown dtype
])
def test_build_rejects_bad_arguments(lib, n, d, m, L, eps, dtype):
    buf = np.zeros(16, dtype=np.float32)
    st, out = _build(lib, buf.ctypes.data, n, d, m, L, eps=eps, dtype=dtype)
    assert st == -1
    assert out.value is None
    assert lib.nrlsh_last_error()


def test_null_arguments(lib):
    st, out = _build(lib, None, 10, 4, 2, 8)
    assert st == -1
    assert lib.nrlsh_build_ex(np.zeros(4, np.float32).ctypes.data, 1, 1, 1, 8, 1, 0, 0.1, None,
                              None) == -1
    assert lib.nrlsh_query(None, None, 1, 10, 10, None, None) == -1
    assert lib.nrlsh_get_codes(None, None) == -1
    lib.nrlsh_free(None)   # no-op
