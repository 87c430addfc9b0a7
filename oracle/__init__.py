"""CPU oracle for the slab hash. Test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The product path never does.
"""
from .oracle import (OracleTable, build_oracle, check_alloc, fit_points, hash_of, learn_model,  # noqa: F401
                     learned_buckets, load_oracle)
