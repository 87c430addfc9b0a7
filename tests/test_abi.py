"""The C-ABI library builds, loads and exports every symbol include/slabhash.h declares.

CPU only: nothing here launches a kernel.
"""
import ctypes as C
import os
import re

import pytest
import torch

from paper_1710_11246_gb300 import build as B
from paper_1710_11246_gb300 import slabhash as sh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slabhash.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(slab_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sh.load_library(build_if_stale=False)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("slab_create", "slab_insert_batch", "slab_delete_batch", "slab_search_batch",
                 "slab_mixed_batch", "slab_destroy"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_binding_covers_the_header():
    assert sorted(sh.EXPORTED) == declared_functions()


def test_library_built_for_sm103a():
    # the build pins one -gencode for sm_103a and nothing else
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(B.LIB)


def test_error_strings(lib):
    for rc in range(8):
        assert lib.slab_error_string(rc) and lib.slab_error_string(rc) != b"unknown error"
    assert sh.slab_error_string(sh.SLAB_ERR_OUT_OF_SLABS) == "SlabAlloc pool exhausted"


def test_host_argument_checks(lib):
    h = C.c_void_p()
    P = sh.SLAB_HASH_PRIME
    bad = [(0, 0, 1, 0, 1024), (8, 2, 1, 0, 1024), (8, 0, 0, 0, 1024), (8, 0, P, 0, 1024),
           (8, 0, 1, P, 1024), (8, 0, 1, 0, 0), (8, 0, 1, 0, 1 << 32)]
    for args in bad:
        assert lib.slab_create(*args, C.byref(h)) == sh.SLAB_ERR_INVALID_ARG, args
    assert lib.slab_insert_batch(None, None, None, None, 0, None) == sh.SLAB_ERR_INVALID_ARG
    assert lib.slab_status(None, None, None) == sh.SLAB_ERR_INVALID_ARG
    sv = C.c_void_p()
    assert lib.slab_server_create(None, 4, 1024, 0.9, 0, C.byref(sv)) == sh.SLAB_ERR_INVALID_ARG
    assert lib.slab_server_submit(None, None, None, None, 1, None) == sh.SLAB_ERR_INVALID_ARG
    assert lib.slab_server_collect(None, 1, None, None, 1) == sh.SLAB_ERR_INVALID_ARG
    assert lib.slab_server_run(None, 0, None, None, None, None, None, None, None, None, None, None,
                               None) == sh.SLAB_ERR_INVALID_ARG


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_create_without_device_fails_cleanly(lib):
    h = C.c_void_p()
    assert lib.slab_create(8, 0, 1, 0, 1024, C.byref(h)) == sh.SLAB_ERR_CUDA
    assert not h.value


def test_binding_rejects_host_tensors(lib):
    with pytest.raises(ValueError):
        sh.slab_search_batch(1, torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.int32))


def test_seeded_hash_parameters(lib):
    """slab_hash_params draws a = 1 + x1 mod (p - 1), b = x2 mod p from the first two
    SplitMix64 outputs; for seed 0 those are the generator's published reference
    values 0xE220A8397B1DCDAF and 0x6E789E6AA1B965F4."""
    P = sh.SLAB_HASH_PRIME
    a, b = sh.slab_hash_params(0)
    assert a == 1 + 0xE220A8397B1DCDAF % (P - 1) and b == 0x6E789E6AA1B965F4 % P
    seen = set()
    for seed in range(200):
        a, b = sh.slab_hash_params(seed)
        assert 1 <= a < P and 0 <= b < P and (a, b) == sh.slab_hash_params(seed)
        seen.add((a, b))
    assert len(seen) == 200
    assert lib.slab_hash_params(1, None, None) == sh.SLAB_ERR_INVALID_ARG
