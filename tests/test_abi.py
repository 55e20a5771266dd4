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


def test_build_opts_rejects_unknown_partition_and_projection(lib):
    import paper_1809_08782_gb300.nrlsh as N
    buf = np.zeros(64, dtype=np.float32)
    for proj, part in ((0, 7), (0, -1), (9, 0)):
        opts = N.NrlshBuildOptions(0, 0.1, proj, part, None, 0)
        out = ctypes.c_void_p()
        st = lib.nrlsh_build_opts(buf.ctypes.data, 16, 4, 2, 8, 1, ctypes.byref(opts),
                                  ctypes.byref(out))
        assert st == -1 and out.value is None
    opts = N.NrlshBuildOptions(0, 0.1, 0, 0, None, 0x2)     # an unknown build flag
    assert lib.nrlsh_build_opts(buf.ctypes.data, 16, 4, 2, 8, 1, ctypes.byref(opts),
                                ctypes.byref(out)) == -1
    assert lib.nrlsh_build_opts(buf.ctypes.data, 16, 4, 2, 8, 1, None, ctypes.byref(out)) == -1


def test_struct_layouts_match_the_header(tmp_path):
    """Offsets and sizes of the public structs, as a C compiler lays them out
    from include/nrlsh.h, equal the binding's ctypes structures."""
    import shutil
    import subprocess
    import paper_1809_08782_gb300.nrlsh as N
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"nrlsh_info": N.NrlshInfo, "nrlsh_build_options": N.NrlshBuildOptions}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nrlsh.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_binding_rejects_output_tensors_the_kernels_would_overrun():
    """Caller-supplied ids/scores must be (nq, k) int64 / float32, contiguous and on
    the queries' device: anything else raises ValueError before the library is
    called (the index handle here is NULL, which the library would reject with
    NrlshError instead)."""
    import torch
    import paper_1809_08782_gb300.nrlsh as N
    fake = N.Index(None, n=100, d=8, m=2, L=16, device=torch.device("cpu"))
    Q = torch.zeros((3, 8), dtype=torch.float32)
    good_ids = torch.empty((3, 5), dtype=torch.int64)
    good_sc = torch.empty((3, 5), dtype=torch.float32)
    bad = [
        (torch.empty((3, 5), dtype=torch.int32), good_sc),        # int32 ids
        (good_ids, torch.empty((3, 5), dtype=torch.float64)),     # float64 scores
        (torch.empty((3, 4), dtype=torch.int64), good_sc),        # k' < k
        (torch.empty((2, 5), dtype=torch.int64), good_sc),        # fewer rows
        (torch.empty((5, 3), dtype=torch.int64).t(), good_sc),    # strided view
        (good_ids, torch.empty((3, 5), dtype=torch.float32, device="meta")),  # other device
    ]
    for ids, sc in bad:
        with pytest.raises(ValueError):
            N.nrlsh_query_ex(fake, Q, 5, 10, ids=ids, scores=sc)
        with pytest.raises(ValueError):
            N.nrlsh_query_noalloc(fake, Q, 5, 10, ids, sc)
    with pytest.raises(ValueError, match="GPU tensors only"):
        N.nrlsh_query_noalloc(fake, Q, 5, 10, good_ids, good_sc)
    ks = torch.ones(3, dtype=torch.int32)
    bs = torch.ones(3, dtype=torch.int64)
    with pytest.raises(ValueError):
        N.nrlsh_query_batched(fake, Q, ks, bs, 5, 10, ids=torch.empty((3, 4), dtype=torch.int64))
    with pytest.raises(ValueError):
        N.nrlsh_query_batched(fake, Q, ks[:2], bs, 5, 10)
    fake.handle = None
