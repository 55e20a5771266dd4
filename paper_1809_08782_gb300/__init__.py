"""GB300-native norm-ranging LSH for maximum inner product search.

The compute path is libnrlsh.so (hand-written CUDA for sm_103a behind a C ABI,
declared in include/nrlsh.h); ``paper_1809_08782_gb300.nrlsh`` is its ctypes
binding and ``paper_1809_08782_gb300.workloads`` draws seeded synthetic inputs.
Importing this package loads nothing; the binding loads the library on first use.
"""
__all__ = ["nrlsh", "workloads", "build"]
