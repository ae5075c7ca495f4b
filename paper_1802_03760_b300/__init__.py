"""B300-native Generic Join: the prefix-extension step (count, propose,
intersect) of worst-case optimal subgraph-query evaluation and its delta
queries, as CUDA kernels for sm_103a behind the C ABI in include/gj.h.

Submodules: ``gj`` (ctypes binding of libgj.so), ``inputs`` (seeded
synthetic workloads), ``build`` (nvcc build of libgj.so).
"""
