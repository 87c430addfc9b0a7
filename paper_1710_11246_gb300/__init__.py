"""GB300 (sm_103a) slab hash: WCWS slab lists with SlabAlloc behind a C ABI.

``slabhash`` is the ctypes binding of ``libslabhash.so`` (declared in
include/slabhash.h); ``build`` compiles it with nvcc; ``workload`` draws the
seeded synthetic inputs of the paper's benchmarks.
"""
