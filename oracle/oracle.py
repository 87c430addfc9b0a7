"""ctypes wrapper over the plain-C slab-hash oracle (slab_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product path never imports it. It shares no code
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slab_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NOT_FOUND = 0xFFFFFFFF


def build_oracle(force: bool = False) -> str:
    """Compile slab_oracle.c with the host C compiler (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def load_oracle(path: str | None = None):
    """Load the oracle library (the in-tree build, or an explicit .so path)."""
    global _lib
    with _lock:
        if path is not None or _lib is None:
            lib = C.CDLL(path or build_oracle())
            u32p, u8p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint8), C.POINTER(C.c_uint64)
            lib.oracle_create.restype = C.c_void_p
            lib.oracle_create.argtypes = [C.c_uint32, C.c_int, C.c_uint32, C.c_uint32]
            lib.oracle_create_width.restype = C.c_void_p
            lib.oracle_create_width.argtypes = [C.c_uint32, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]
            lib.oracle_destroy.argtypes = [C.c_void_p]
            lib.oracle_hash.restype = C.c_uint32
            lib.oracle_hash.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
            lib.oracle_bucket.restype = C.c_uint32
            lib.oracle_bucket.argtypes = [C.c_void_p, C.c_uint32]
            lib.oracle_insert.argtypes = [C.c_void_p, u32p, u32p, C.c_uint64, u8p, u64p]
            lib.oracle_delete.argtypes = [C.c_void_p, u32p, C.c_uint64, u8p, u64p]
            lib.oracle_search.argtypes = [C.c_void_p, u32p, C.c_uint64, u32p, u8p, u64p]
            lib.oracle_mixed.argtypes = [C.c_void_p, u8p, u32p, u32p, C.c_uint64, u32p, u8p, u64p]
            lib.oracle_stats.argtypes = [C.c_void_p, u32p, u32p, u64p]
            lib.oracle_utilization.restype = C.c_double
            lib.oracle_utilization.argtypes = [C.c_void_p]
            lib.oracle_export.restype = C.c_uint64
            lib.oracle_export.argtypes = [C.c_void_p, u32p, u32p, u32p, C.c_uint64]
            f32p = C.POINTER(C.c_float)
            lib.oracle_learned_bucket.restype = C.c_uint32
            lib.oracle_learned_bucket.argtypes = [f32p, C.c_uint32, C.c_uint32]
            lib.oracle_use_model.restype = C.c_int
            lib.oracle_use_model.argtypes = [C.c_void_p, f32p]
            lib.oracle_fit_points.argtypes = [u32p, u32p, C.c_uint64, f32p]
            lib.oracle_learn_model.restype = C.c_uint64
            lib.oracle_learn_model.argtypes = [u32p, C.c_uint64, C.c_uint32, C.c_uint32, f32p]
            lib.oracle_chain_profile.argtypes = [C.c_void_p, u32p, C.c_uint64, u64p, u32p]
            lib.oracle_set_multiset.restype = C.c_int
            lib.oracle_set_multiset.argtypes = [C.c_void_p, C.c_int]
            lib.oracle_search_all.argtypes = [C.c_void_p, u32p, C.c_uint64, C.c_uint32, u32p, u32p]
            lib.oracle_delete_all.argtypes = [C.c_void_p, u32p, C.c_uint64, u32p]
            lib.oracle_flush.restype = C.c_uint64
            lib.oracle_flush.argtypes = [C.c_void_p]
            lib.oracle_check_alloc.restype = C.c_int
            lib.oracle_check_alloc.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64, C.c_uint32, u64p]
            if path is not None:
                return lib
            _lib = lib
    return _lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


class OracleTable:
    """A slab hash as its plain definition: B insertion-ordered slot arrays."""

    def __init__(self, num_buckets: int, hash_a: int, hash_b: int, key_only: bool = False,
                 lib=None, slab_bytes: int = 128):
        self.lib = lib if lib is not None else load_oracle()
        self.B = int(num_buckets)
        self.key_only = bool(key_only)
        self.slab_bytes = int(slab_bytes)
        if self.slab_bytes == 128:
            self.h = self.lib.oracle_create(self.B, int(self.key_only), int(hash_a), int(hash_b))
        else:
            self.h = self.lib.oracle_create_width(self.B, int(self.key_only), int(hash_a), int(hash_b),
                                                  self.slab_bytes)
        if not self.h:
            raise ValueError("oracle_create rejected its arguments")
        self.lines = 0

    def close(self):
        if self.h:
            self.lib.oracle_destroy(self.h)
            self.h = None

    __del__ = close

    def bucket(self, key: int) -> int:
        return int(self.lib.oracle_bucket(self.h, int(key)))

    def buckets(self, keys) -> np.ndarray:
        return np.array([self.lib.oracle_bucket(self.h, int(k)) for k in np.asarray(keys)],
                        dtype=np.uint32)

    def _count(self):
        return C.c_uint64(0)

    def insert(self, keys, values=None):
        keys = _u32(keys)
        vals = None if values is None else _u32(values)
        found = np.zeros(len(keys), np.uint8)
        ln = self._count()
        self.lib.oracle_insert(self.h, _ptr(keys, C.c_uint32), _ptr(vals, C.c_uint32), len(keys),
                               _ptr(found, C.c_uint8), C.byref(ln))
        self.lines += ln.value
        return found

    def delete(self, keys):
        keys = _u32(keys)
        found = np.zeros(len(keys), np.uint8)
        ln = self._count()
        self.lib.oracle_delete(self.h, _ptr(keys, C.c_uint32), len(keys), _ptr(found, C.c_uint8),
                               C.byref(ln))
        self.lines += ln.value
        return found

    def search(self, keys):
        keys = _u32(keys)
        vals = np.zeros(len(keys), np.uint32)
        found = np.zeros(len(keys), np.uint8)
        ln = self._count()
        self.lib.oracle_search(self.h, _ptr(keys, C.c_uint32), len(keys), _ptr(vals, C.c_uint32),
                               _ptr(found, C.c_uint8), C.byref(ln))
        self.lines += ln.value
        return vals, found

    def mixed(self, ops, keys, values=None):
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = _u32(keys)
        vals = None if values is None else _u32(values)
        res = np.zeros(len(keys), np.uint32)
        found = np.zeros(len(keys), np.uint8)
        ln = self._count()
        self.lib.oracle_mixed(self.h, _ptr(ops, C.c_uint8), _ptr(keys, C.c_uint32),
                              _ptr(vals, C.c_uint32), len(keys), _ptr(res, C.c_uint32),
                              _ptr(found, C.c_uint8), C.byref(ln))
        self.lines += ln.value
        return res, found

    def stats(self):
        """(slots per bucket, slabs per bucket, {live, slots, slabs, reserved})."""
        slots = np.zeros(self.B, np.uint32)
        slabs = np.zeros(self.B, np.uint32)
        tot = np.zeros(4, np.uint64)
        self.lib.oracle_stats(self.h, _ptr(slots, C.c_uint32), _ptr(slabs, C.c_uint32),
                              _ptr(tot, C.c_uint64))
        return slots, slabs, dict(live=int(tot[0]), slots=int(tot[1]), slabs=int(tot[2]),
                                  reserved=int(tot[3]))

    def use_model(self, model):
        """Switch an empty table to a learned bucket function (2 + 2048 float32)."""
        model = np.ascontiguousarray(model, dtype=np.float32)
        if self.lib.oracle_use_model(self.h, _ptr(model, C.c_float)) != 0:
            raise ValueError("the table is not empty")

    def chain_profile(self, keys):
        """(sum, max) of slabs per bucket the keys would form under this table's buckets."""
        keys = _u32(keys)
        sm, mx = C.c_uint64(0), C.c_uint32(0)
        self.lib.oracle_chain_profile(self.h, _ptr(keys, C.c_uint32), len(keys), C.byref(sm), C.byref(mx))
        return int(sm.value), int(mx.value)

    def utilization(self) -> float:
        return float(self.lib.oracle_utilization(self.h))

    def set_multiset(self, on: bool = True):
        """Make the (empty) table a multiset: inserts allow duplicates, deletes empty their slot."""
        if self.lib.oracle_set_multiset(self.h, int(bool(on))) != 0:
            raise ValueError("the table is not empty")

    def search_all(self, keys, cap: int):
        """(counts, values[n, cap]): every live instance of each key in list order."""
        keys = _u32(keys)
        counts = np.zeros(len(keys), np.uint32)
        vals = np.full((len(keys), max(int(cap), 0)), 0xFFFFFFFF, np.uint32)
        self.lib.oracle_search_all(self.h, _ptr(keys, C.c_uint32), len(keys), int(cap),
                                   _ptr(counts, C.c_uint32), _ptr(vals, C.c_uint32) if vals.size else None)
        return counts, vals

    def delete_all(self, keys):
        keys = _u32(keys)
        counts = np.zeros(len(keys), np.uint32)
        self.lib.oracle_delete_all(self.h, _ptr(keys, C.c_uint32), len(keys), _ptr(counts, C.c_uint32))
        return counts

    def flush(self) -> int:
        """Compact every bucket (Sec. 4.3.4); returns the slabs released."""
        return int(self.lib.oracle_flush(self.h))

    def export(self):
        """Live elements as (bucket, key, value) arrays in bucket / list order."""
        n = int(self.lib.oracle_export(self.h, None, None, None, 0))
        b = np.zeros(n, np.uint32)
        k = np.zeros(n, np.uint32)
        v = np.zeros(n, np.uint32)
        self.lib.oracle_export(self.h, _ptr(b, C.c_uint32), _ptr(k, C.c_uint32),
                               _ptr(v, C.c_uint32), n)
        return b, k, v


def hash_of(a: int, b: int, num_buckets: int, key: int, lib=None) -> int:
    """h(k; a, b) = ((a k + b) mod p) mod B for one key, no table needed."""
    lib = lib if lib is not None else load_oracle()
    return int(lib.oracle_hash(int(a), int(b), int(num_buckets), int(key)))


MODEL_FLOATS = 2 + 2 * 1024


def learn_model(keys, stride: int, num_buckets: int, lib=None):
    """Fit the two-level learned bucket model on keys[::stride]; returns (model, m)."""
    lib = lib if lib is not None else load_oracle()
    keys = _u32(keys)
    model = np.zeros(MODEL_FLOATS, np.float32)
    m = lib.oracle_learn_model(_ptr(keys, C.c_uint32), len(keys), int(stride), int(num_buckets),
                               _ptr(model, C.c_float))
    return model, int(m)


def learned_buckets(model, num_buckets: int, keys, lib=None) -> np.ndarray:
    lib = lib if lib is not None else load_oracle()
    model = np.ascontiguousarray(model, dtype=np.float32)
    mp = _ptr(model, C.c_float)
    return np.array([lib.oracle_learned_bucket(mp, int(num_buckets), int(k)) for k in np.asarray(keys)],
                    dtype=np.uint32)


def fit_points(xs, ys, lib=None):
    """(a, b) of the least-squares line through integer points, as the model fits it."""
    lib = lib if lib is not None else load_oracle()
    xs, ys = _u32(xs), _u32(ys)
    ab = np.zeros(2, np.float32)
    lib.oracle_fit_points(_ptr(xs, C.c_uint32), _ptr(ys, C.c_uint32), len(xs), _ptr(ab, C.c_float))
    return ab


def check_alloc(addrs, bitmaps, num_blocks: int, blocks_per_super: int = 1 << 14, lib=None):
    """0 if addresses are valid, distinct and exactly match the bitmaps; see the C doc."""
    lib = lib if lib is not None else load_oracle()
    addrs = _u32(addrs)
    bitmaps = _u32(bitmaps)
    if len(bitmaps) != num_blocks * 32:
        raise ValueError("bitmap array must hold 32 words per memory block")
    where = C.c_uint64(0)
    rc = lib.oracle_check_alloc(_ptr(addrs, C.c_uint32), len(addrs), _ptr(bitmaps, C.c_uint32),
                                int(num_blocks), int(blocks_per_super), C.byref(where))
    return int(rc), int(where.value)
