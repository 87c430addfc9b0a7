"""Python binding of libslabhash.so (include/slabhash.h): argument marshalling only.

Every function keeps the C name and forwards device pointers of torch CUDA
tensors plus the torch stream handle; all work runs in the library's kernels.
There is no CPU path: if the library cannot be loaded, the import of the
binding's entry points raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

SLAB_MODE_KEY_VALUE, SLAB_MODE_KEY_ONLY = 0, 1
SLAB_OP_INSERT, SLAB_OP_DELETE, SLAB_OP_SEARCH = 0, 1, 2
SLAB_OK, SLAB_ERR_INVALID_ARG, SLAB_ERR_RESERVED_KEY = 0, 1, 2
SLAB_ERR_OUT_OF_SLABS, SLAB_ERR_ITER_LIMIT, SLAB_ERR_CUDA, SLAB_ERR_CORRUPT, SLAB_ERR_BUSY = 3, 4, 5, 6, 7
SLAB_FLAG_RESERVED_KEY, SLAB_FLAG_OUT_OF_SLABS, SLAB_FLAG_ITER_LIMIT, SLAB_FLAG_BAD_POINTER = 1, 2, 4, 8
SLAB_EMPTY_KEY = SLAB_NOT_FOUND = 0xFFFFFFFF
SLAB_TOMBSTONE_KEY = 0xFFFFFFFE
SLAB_HASH_PRIME = 4294967291
SLAB_VARIANT_STAGED, SLAB_VARIANT_DIRECT = 0, 1

EXPORTED = [
    "slab_create", "slab_destroy", "slab_reset", "slab_get_info", "slab_get_config", "slab_set_config",
    "slab_insert_batch", "slab_delete_batch", "slab_search_batch", "slab_mixed_batch", "slab_status",
    "slab_stats", "slab_export", "slab_bucket_of", "slab_alloc_batch", "slab_free_batch",
    "slab_copy_bitmaps", "slab_error_string", "slab_probe_random_lines", "slab_probe_random_cas",
    "slab_chain_histogram_noalloc", "slab_learn_buckets", "slab_get_model",
    "slab_group_create", "slab_group_destroy", "slab_group_table", "slab_group_get_config", "slab_group_set_config",
    "slab_group_reset", "slab_group_insert", "slab_group_delete", "slab_group_search", "slab_group_mixed",
    "slab_group_status",
    "slab_server_create", "slab_server_destroy", "slab_server_submit", "slab_server_collect",
    "slab_server_get_stats", "slab_server_run",
    "slab_set_multiset", "slab_search_all_batch", "slab_delete_all_batch", "slab_flush", "slab_grow_pool",
    "slab_hash_params", "slab_create_seeded", "slab_probe_random_or", "slab_probe_random_lines_v4",
    "slab_create_width", "slab_group_create_width", "slab_batch_host",
]
SLAB_SERVER_MAX_SLOTS, SLAB_SERVER_MAX_REQUEST_OPS, SLAB_SERVER_ZERO_COPY, SLAB_SERVER_GROW_POOL = 64, 1 << 24, 1, 2
SLAB_LEARN_AUTO, SLAB_LEARN_ALWAYS, SLAB_LEARN_MEASURE = 0, 1, 2
MODEL_FLOATS = 2 + 2 * 1024


class SlabConfig(C.Structure):
    _fields_ = [("variant", C.c_int32), ("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("iter_limit", C.c_uint32), ("random_probes", C.c_uint32)]


class SlabInfo(C.Structure):
    _fields_ = [("num_buckets", C.c_uint32), ("mode", C.c_int32), ("elements_per_slab", C.c_uint32),
                ("hash_a", C.c_uint32), ("hash_b", C.c_uint32), ("pool_slabs", C.c_uint64),
                ("num_memory_blocks", C.c_uint32), ("blocks_per_super", C.c_uint32),
                ("num_super_blocks", C.c_uint32), ("sm_count", C.c_uint32), ("device_bytes", C.c_uint64),
                ("multiset", C.c_int32), ("slab_bytes", C.c_int32)]


class SlabLearnReport(C.Structure):
    _fields_ = [("sample_size", C.c_uint32), ("use_learned", C.c_uint32), ("max_slabs_learned", C.c_uint32),
                ("max_slabs_universal", C.c_uint32), ("mean_slabs_learned", C.c_double),
                ("mean_slabs_universal", C.c_double)]


class SlabServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("deferred_slot", C.c_uint64),
                ("deferred_memory", C.c_uint64), ("rejected_memory", C.c_uint64), ("pool_grown", C.c_uint64),
                ("pool_slabs", C.c_uint64),
                ("pool_measured", C.c_uint64), ("pool_reserved", C.c_uint64), ("inflight", C.c_uint32),
                ("pad", C.c_uint32)]


class SlabError(RuntimeError):
    def __init__(self, rc: int, what: str = ""):
        self.rc = rc
        super().__init__(f"{what}: {slab_error_string(rc)} (rc={rc})" if what else slab_error_string(rc))


_lib = None
_lock = threading.Lock()


def load_library(build_if_stale: bool = True) -> C.CDLL:
    """Load the in-tree libslabhash.so, building it from source when it is stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_stale and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing; build it with paper_1710_11246_gb300.build.build()")
        lib = C.CDLL(_build.LIB)
        vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        sig = {
            "slab_create": (i32, [u32, i32, u32, u32, u64, C.POINTER(vp)]),
            "slab_destroy": (None, [vp]),
            "slab_reset": (i32, [vp, vp]),
            "slab_get_info": (i32, [vp, C.POINTER(SlabInfo)]),
            "slab_get_config": (i32, [vp, C.POINTER(SlabConfig)]),
            "slab_set_config": (i32, [vp, C.POINTER(SlabConfig)]),
            "slab_insert_batch": (i32, [vp, vp, vp, vp, u32, vp]),
            "slab_delete_batch": (i32, [vp, vp, vp, u32, vp]),
            "slab_search_batch": (i32, [vp, vp, vp, vp, u32, vp]),
            "slab_mixed_batch": (i32, [vp, vp, vp, vp, vp, vp, u32, vp]),
            "slab_status": (i32, [vp, vp, C.POINTER(u32)]),
            "slab_stats": (i32, [vp, vp, vp, C.POINTER(u64), vp]),
            "slab_export": (i32, [vp, vp, vp, vp, u64, C.POINTER(u64), vp]),
            "slab_bucket_of": (i32, [vp, vp, vp, u32, vp]),
            "slab_alloc_batch": (i32, [vp, vp, u32, vp]),
            "slab_free_batch": (i32, [vp, vp, u32, vp]),
            "slab_copy_bitmaps": (i32, [vp, vp, u64, vp]),
            "slab_error_string": (C.c_char_p, [i32]),
            "slab_probe_random_lines": (i32, [vp, u64, u64, u32, i32, i32, vp, vp]),
            "slab_probe_random_lines_v4": (i32, [vp, u64, u64, u32, i32, i32, i32, i32, vp, vp]),
            "slab_create_width": (i32, [u32, i32, u32, u32, u32, u64, C.POINTER(vp)]),
            "slab_batch_host": (i32, [vp, i32, vp, vp, vp, vp, vp, u32, u32, vp, vp]),
            "slab_group_create_width": (i32, [u32, vp, vp, vp, vp, i32, u32, C.POINTER(vp)]),
            "slab_probe_random_cas": (i32, [vp, u64, u64, u32, i32, i32, vp]),
            "slab_chain_histogram_noalloc": (i32, [vp, u32, C.POINTER(u64), C.POINTER(u64), vp]),
            "slab_learn_buckets": (i32, [vp, vp, u32, u32, i32, C.POINTER(SlabLearnReport), vp]),
            "slab_get_model": (i32, [vp, C.POINTER(C.c_float), C.POINTER(u32)]),
            "slab_group_create": (i32, [u32, vp, vp, vp, vp, i32, C.POINTER(vp)]),
            "slab_group_destroy": (None, [vp]),
            "slab_group_table": (i32, [vp, u32, C.POINTER(vp)]),
            "slab_group_get_config": (i32, [vp, C.POINTER(SlabConfig)]),
            "slab_group_set_config": (i32, [vp, C.POINTER(SlabConfig)]),
            "slab_group_reset": (i32, [vp, vp]),
            "slab_group_insert": (i32, [vp, vp, vp, vp, vp, u32, vp]),
            "slab_group_delete": (i32, [vp, vp, vp, vp, u32, vp]),
            "slab_group_search": (i32, [vp, vp, vp, vp, vp, u32, vp]),
            "slab_group_mixed": (i32, [vp, vp, vp, vp, vp, vp, vp, u32, vp]),
            "slab_group_status": (i32, [vp, vp, C.POINTER(u32)]),
            "slab_set_multiset": (i32, [vp, i32]),
            "slab_hash_params": (i32, [u64, C.POINTER(u32), C.POINTER(u32)]),
            "slab_create_seeded": (i32, [u32, i32, u64, u64, C.POINTER(vp)]),
            "slab_probe_random_or": (i32, [vp, u64, u64, u32, i32, i32, vp]),
            "slab_search_all_batch": (i32, [vp, vp, u32, u32, vp, vp, vp]),
            "slab_delete_all_batch": (i32, [vp, vp, vp, u32, vp]),
            "slab_flush": (i32, [vp, C.POINTER(u64), vp]),
            "slab_grow_pool": (i32, [vp, u64]),
            "slab_server_create": (i32, [vp, u32, u32, C.c_double, u32, C.POINTER(vp)]),
            "slab_server_destroy": (None, [vp]),
            "slab_server_submit": (i32, [vp, vp, vp, vp, u32, C.POINTER(u64)]),
            "slab_server_collect": (i32, [vp, u64, vp, vp, i32]),
            "slab_server_get_stats": (i32, [vp, C.POINTER(SlabServerStats)]),
            "slab_server_run": (i32, [vp, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(u64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def slab_error_string(rc: int) -> str:
    return load_library().slab_error_string(int(rc)).decode()


# ------------------------------------------------------------------ marshalling
def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t, itemsize: int, n: int, name: str, nullable: bool = False):
    if t is None:
        if nullable:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous() or t.element_size() != itemsize:
        raise ValueError(f"{name} must be contiguous with {itemsize}-byte elements")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {n}")
    return t.data_ptr() if n or t.numel() else None


def _check(rc: int, what: str):
    if rc != SLAB_OK:
        raise SlabError(rc, what)


# ------------------------------------------------------------------ C-name API
def slab_create_width(num_buckets: int, mode: int, slab_bytes: int, hash_a: int, hash_b: int, pool_slabs: int) -> int:
    h = C.c_void_p()
    _check(load_library().slab_create_width(num_buckets, mode, slab_bytes, hash_a, hash_b, pool_slabs, C.byref(h)),
           "slab_create_width")
    return h.value


SLAB_BATCH_INSERT, SLAB_BATCH_DELETE, SLAB_BATCH_SEARCH, SLAB_BATCH_MIXED = 0, 1, 2, 3


def _host_ptr(a, itemsize: int, n: int, name: str, nullable: bool = False):
    """Host address of a contiguous numpy array or CPU torch tensor with n elements of itemsize bytes."""
    if a is None:
        if nullable:
            return None
        raise ValueError(f"{name} is required")
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous() or a.element_size() != itemsize or a.numel() < n:
            raise ValueError(f"{name}: a contiguous host tensor of {n} x {itemsize}-byte elements is required")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"] or a.itemsize != itemsize or a.size < n:
        raise ValueError(f"{name}: a contiguous host array of {n} x {itemsize}-byte elements is required")
    return a.ctypes.data


def slab_batch_host(t: int, kind: int, keys, values=None, ops=None, results=None, found=None, n: int | None = None,
                    chunk: int = 0, stream=None, done_event=None) -> None:
    """A batch from host memory (slabhash.h slab_batch_host); done_event: a torch.cuda.Event or None."""
    n = (keys.numel() if isinstance(keys, torch.Tensor) else len(keys)) if n is None else n
    ev = None
    if done_event is not None:
        if hasattr(done_event, "cuda_event"):  # a torch.cuda.Event: its CUDA event exists once it is recorded
            if not done_event.cuda_event:
                done_event.record()
            ev = done_event.cuda_event
        else:
            ev = done_event
    _check(load_library().slab_batch_host(
        t, int(kind), _host_ptr(ops, 1, n, "ops", nullable=True), _host_ptr(keys, 4, n, "keys"),
        _host_ptr(values, 4, n, "values", nullable=True), _host_ptr(results, 4, n, "results", nullable=True),
        _host_ptr(found, 1, n, "found", nullable=True), n, int(chunk), _stream(stream), ev), "slab_batch_host")


def slab_create(num_buckets: int, mode: int, hash_a: int, hash_b: int, pool_slabs: int) -> int:
    h = C.c_void_p()
    _check(load_library().slab_create(num_buckets, mode, hash_a, hash_b, pool_slabs, C.byref(h)),
           "slab_create")
    return h.value


def slab_destroy(t: int) -> None:
    load_library().slab_destroy(t)


def slab_reset(t: int, stream=None) -> None:
    _check(load_library().slab_reset(t, _stream(stream)), "slab_reset")


def slab_get_info(t: int) -> SlabInfo:
    info = SlabInfo()
    _check(load_library().slab_get_info(t, C.byref(info)), "slab_get_info")
    return info


def slab_get_config(t: int) -> SlabConfig:
    cfg = SlabConfig()
    _check(load_library().slab_get_config(t, C.byref(cfg)), "slab_get_config")
    return cfg


def slab_set_config(t: int, cfg: SlabConfig) -> None:
    _check(load_library().slab_set_config(t, C.byref(cfg)), "slab_set_config")


def slab_insert_batch(t: int, keys, values, found=None, n: int | None = None, stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_insert_batch(
        t, _dptr(keys, 4, n, "keys"), _dptr(values, 4, n, "values", nullable=True),
        _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)), "slab_insert_batch")


def slab_delete_batch(t: int, keys, found=None, n: int | None = None, stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_delete_batch(
        t, _dptr(keys, 4, n, "keys"), _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
        "slab_delete_batch")


def slab_search_batch(t: int, keys, values_out, found=None, n: int | None = None, stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_search_batch(
        t, _dptr(keys, 4, n, "keys"), _dptr(values_out, 4, n, "values_out"),
        _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)), "slab_search_batch")


def slab_mixed_batch(t: int, ops, keys, values, results, found=None, n: int | None = None,
                     stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_mixed_batch(
        t, _dptr(ops, 1, n, "ops"), _dptr(keys, 4, n, "keys"), _dptr(values, 4, n, "values", nullable=True),
        _dptr(results, 4, n, "results"), _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
        "slab_mixed_batch")


def slab_status(t: int, stream=None) -> tuple[int, int]:
    """(return code, status flags); synchronizes the stream and clears the flags."""
    flags = C.c_uint32(0)
    rc = load_library().slab_status(t, _stream(stream), C.byref(flags))
    if rc == SLAB_ERR_CUDA or rc == SLAB_ERR_INVALID_ARG:
        raise SlabError(rc, "slab_status")
    return rc, flags.value


def slab_stats(t: int, slots=None, slabs=None, stream=None) -> dict:
    info = slab_get_info(t)
    tot = (C.c_uint64 * 6)()
    _check(load_library().slab_stats(
        t, _dptr(slots, 4, info.num_buckets, "slots", nullable=True),
        _dptr(slabs, 4, info.num_buckets, "slabs", nullable=True), tot, _stream(stream)), "slab_stats")
    return dict(live=tot[0], slots=tot[1], slabs=tot[2], pool_allocated=tot[3], prefix_violations=tot[4],
                linked=tot[5])


def slab_export(t: int, buckets, keys, values, capacity: int, stream=None) -> int:
    count = C.c_uint64(0)
    _check(load_library().slab_export(
        t, _dptr(buckets, 4, capacity, "buckets", nullable=True), _dptr(keys, 4, capacity, "keys", nullable=True),
        _dptr(values, 4, capacity, "values", nullable=True), capacity, C.byref(count), _stream(stream)),
        "slab_export")
    return count.value


def slab_bucket_of(t: int, keys, buckets_out, n: int | None = None, stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_bucket_of(t, _dptr(keys, 4, n, "keys"), _dptr(buckets_out, 4, n, "buckets_out"),
                                         n, _stream(stream)), "slab_bucket_of")


def slab_alloc_batch(t: int, addrs_out, n: int | None = None, stream=None) -> None:
    n = addrs_out.numel() if n is None else n
    _check(load_library().slab_alloc_batch(t, _dptr(addrs_out, 4, n, "addrs_out"), n, _stream(stream)),
           "slab_alloc_batch")


def slab_free_batch(t: int, addrs, n: int | None = None, stream=None) -> None:
    n = addrs.numel() if n is None else n
    _check(load_library().slab_free_batch(t, _dptr(addrs, 4, n, "addrs"), n, _stream(stream)),
           "slab_free_batch")


def slab_copy_bitmaps(t: int, dst, stream=None) -> None:
    info = slab_get_info(t)
    n = info.num_memory_blocks * 32
    _check(load_library().slab_copy_bitmaps(t, _dptr(dst, 4, n, "dst"), n, _stream(stream)),
           "slab_copy_bitmaps")


def slab_probe_random_lines(buf, footprint_lines: int, n_reads: int, seed: int, lines_in_flight: int,
                            threads_per_block: int, sink, stream=None) -> None:
    _check(load_library().slab_probe_random_lines(
        _dptr(buf, 4, footprint_lines * 32, "buf"), footprint_lines, n_reads, seed, lines_in_flight,
        threads_per_block, _dptr(sink, 4, 1, "sink"), _stream(stream)), "slab_probe_random_lines")


def slab_probe_random_lines_v4(buf, footprint_lines: int, n_reads: int, seed: int, form: int, lines_in_flight: int,
                               threads_per_block: int, sink, stream=None, line_bytes: int = 128) -> None:
    _check(load_library().slab_probe_random_lines_v4(
        _dptr(buf, 4, footprint_lines * line_bytes // 4, "buf"), footprint_lines, n_reads, seed, form, line_bytes,
        lines_in_flight,
        threads_per_block, _dptr(sink, 4, 1, "sink"), _stream(stream)), "slab_probe_random_lines_v4")


def slab_probe_random_cas(buf, footprint_lines: int, n_ops: int, seed: int, ops_in_flight: int,
                          threads_per_block: int, stream=None) -> None:
    _check(load_library().slab_probe_random_cas(
        _dptr(buf, 8, footprint_lines * 16, "buf"), footprint_lines, n_ops, seed, ops_in_flight,
        threads_per_block, _stream(stream)), "slab_probe_random_cas")


def slab_learn_buckets(t: int, keys, sample_stride: int = 100, policy: int = SLAB_LEARN_AUTO, n: int | None = None,
                       stream=None) -> dict:
    n = keys.numel() if n is None else n
    rep = SlabLearnReport()
    _check(load_library().slab_learn_buckets(t, _dptr(keys, 4, n, "keys"), n, int(sample_stride), int(policy),
                                             C.byref(rep), _stream(stream)), "slab_learn_buckets")
    return {f: getattr(rep, f) for f, _ in rep._fields_}


def slab_get_model(t: int):
    """(model as float32 numpy array of 2 + 2 * 1024, whether the table uses it)."""
    import numpy as np
    model = np.zeros(MODEL_FLOATS, np.float32)
    in_use = C.c_uint32(0)
    _check(load_library().slab_get_model(t, model.ctypes.data_as(C.POINTER(C.c_float)), C.byref(in_use)),
           "slab_get_model")
    return model, bool(in_use.value)


def slab_chain_histogram_noalloc(t: int, n_bins: int, stream=None):
    """(histogram of slabs per list as a uint64 numpy array, slab_stats-style totals).

    The library allocates no device memory for this call; see slabhash.h."""
    import numpy as np
    hist = np.zeros(int(n_bins), dtype=np.uint64)
    tot = (C.c_uint64 * 6)()
    _check(load_library().slab_chain_histogram_noalloc(
        t, int(n_bins), hist.ctypes.data_as(C.POINTER(C.c_uint64)), tot, _stream(stream)),
        "slab_chain_histogram_noalloc")
    return hist, dict(live=tot[0], slots=tot[1], slabs=tot[2], pool_allocated=tot[3], prefix_violations=tot[4],
                      linked=tot[5])


def slab_group_create(num_buckets, hash_a, hash_b, pool_slabs, mode: int = SLAB_MODE_KEY_VALUE,
                      slab_bytes: int = 128) -> int:
    import numpy as np
    nb = np.ascontiguousarray(num_buckets, np.uint32)
    ha = np.ascontiguousarray(hash_a, np.uint32)
    hb = np.ascontiguousarray(hash_b, np.uint32)
    ps = np.ascontiguousarray(pool_slabs, np.uint64)
    if not (len(nb) == len(ha) == len(hb) == len(ps)):
        raise ValueError("per-table arrays differ in length")
    g = C.c_void_p()
    if slab_bytes == 128:
        _check(load_library().slab_group_create(len(nb), nb.ctypes.data, ha.ctypes.data, hb.ctypes.data,
                                                ps.ctypes.data, mode, C.byref(g)), "slab_group_create")
    else:
        _check(load_library().slab_group_create_width(len(nb), nb.ctypes.data, ha.ctypes.data, hb.ctypes.data,
                                                      ps.ctypes.data, mode, slab_bytes, C.byref(g)),
               "slab_group_create_width")
    return g.value


def slab_group_destroy(g: int) -> None:
    load_library().slab_group_destroy(g)


def slab_group_table(g: int, i: int) -> int:
    t = C.c_void_p()
    _check(load_library().slab_group_table(g, int(i), C.byref(t)), "slab_group_table")
    return t.value


def slab_group_get_config(g: int) -> SlabConfig:
    cfg = SlabConfig()
    _check(load_library().slab_group_get_config(g, C.byref(cfg)), "slab_group_get_config")
    return cfg


def slab_group_set_config(g: int, cfg: SlabConfig) -> None:
    _check(load_library().slab_group_set_config(g, C.byref(cfg)), "slab_group_set_config")


def slab_group_reset(g: int, stream=None) -> None:
    _check(load_library().slab_group_reset(g, _stream(stream)), "slab_group_reset")


def _starts(op_start, ntables=None):
    return _dptr(op_start, 4, op_start.numel(), "op_start")


def slab_group_insert(g: int, op_start, keys, values, found=None, stream=None) -> None:
    n = keys.numel()
    _check(load_library().slab_group_insert(g, _starts(op_start), _dptr(keys, 4, n, "keys"),
                                            _dptr(values, 4, n, "values", nullable=True),
                                            _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
           "slab_group_insert")


def slab_group_delete(g: int, op_start, keys, found=None, stream=None) -> None:
    n = keys.numel()
    _check(load_library().slab_group_delete(g, _starts(op_start), _dptr(keys, 4, n, "keys"),
                                            _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
           "slab_group_delete")


def slab_group_search(g: int, op_start, keys, values_out, found=None, stream=None) -> None:
    n = keys.numel()
    _check(load_library().slab_group_search(g, _starts(op_start), _dptr(keys, 4, n, "keys"),
                                            _dptr(values_out, 4, n, "values_out"),
                                            _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
           "slab_group_search")


def slab_group_mixed(g: int, op_start, ops, keys, values, results, found=None, stream=None) -> None:
    n = keys.numel()
    _check(load_library().slab_group_mixed(g, _starts(op_start), _dptr(ops, 1, n, "ops"), _dptr(keys, 4, n, "keys"),
                                           _dptr(values, 4, n, "values", nullable=True),
                                           _dptr(results, 4, n, "results"),
                                           _dptr(found, 1, n, "found", nullable=True), n, _stream(stream)),
           "slab_group_mixed")


def slab_group_status(g: int, stream=None) -> tuple[int, int]:
    flags = C.c_uint32(0)
    rc = load_library().slab_group_status(g, _stream(stream), C.byref(flags))
    if rc == SLAB_ERR_CUDA or rc == SLAB_ERR_INVALID_ARG:
        raise SlabError(rc, "slab_group_status")
    return rc, flags.value


def slab_hash_params(seed: int) -> tuple[int, int]:
    a, b = C.c_uint32(0), C.c_uint32(0)
    _check(load_library().slab_hash_params(int(seed), C.byref(a), C.byref(b)), "slab_hash_params")
    return a.value, b.value


def slab_create_seeded(num_buckets: int, mode: int, seed: int, pool_slabs: int) -> int:
    h = C.c_void_p()
    _check(load_library().slab_create_seeded(num_buckets, mode, int(seed), pool_slabs, C.byref(h)),
           "slab_create_seeded")
    return h.value


def slab_probe_random_or(buf, footprint_words: int, n_ops: int, seed: int, ops_in_flight: int,
                         threads_per_block: int, stream=None) -> None:
    _check(load_library().slab_probe_random_or(_dptr(buf, 4, footprint_words, "buf"), footprint_words, n_ops, seed,
                                               ops_in_flight, threads_per_block, _stream(stream)),
           "slab_probe_random_or")


# ------------------------------------------------------------------ paper variants
def slab_set_multiset(t: int, on: bool = True) -> None:
    _check(load_library().slab_set_multiset(t, int(bool(on))), "slab_set_multiset")


def slab_search_all_batch(t: int, keys, max_per_key: int, counts, values_out=None, n: int | None = None,
                          stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_search_all_batch(
        t, _dptr(keys, 4, n, "keys"), n, max_per_key, _dptr(counts, 4, n, "counts"),
        _dptr(values_out, 4, n * max_per_key, "values_out", nullable=max_per_key == 0), _stream(stream)),
        "slab_search_all_batch")


def slab_delete_all_batch(t: int, keys, counts=None, n: int | None = None, stream=None) -> None:
    n = keys.numel() if n is None else n
    _check(load_library().slab_delete_all_batch(t, _dptr(keys, 4, n, "keys"),
                                                _dptr(counts, 4, n, "counts", nullable=True), n, _stream(stream)),
           "slab_delete_all_batch")


def slab_flush(t: int, stream=None, wait: bool = True):
    """Compact every bucket (Sec. 4.3.4); returns the slabs released when wait is set."""
    r = C.c_uint64(0)
    _check(load_library().slab_flush(t, C.byref(r) if wait else None, _stream(stream)), "slab_flush")
    return r.value if wait else None


def slab_grow_pool(t: int, extra_slabs: int) -> None:
    _check(load_library().slab_grow_pool(t, extra_slabs), "slab_grow_pool")


# ------------------------------------------------------------------ serving
def _hptr(a, dtype, n: int, name: str, nullable: bool = False):
    """Host pointer of a contiguous numpy array of `dtype` with at least n elements."""
    import numpy as np
    if a is None:
        if nullable:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise ValueError(f"{name} must be a contiguous numpy array of {np.dtype(dtype).name}")
    if a.size < n:
        raise ValueError(f"{name} holds {a.size} elements, needs {n}")
    return a.ctypes.data if a.size else None


def slab_server_create(t: int, slots: int, max_request_ops: int, pool_high_water: float = 0.9,
                       flags: int = 0) -> int:
    h = C.c_void_p()
    _check(load_library().slab_server_create(t, slots, max_request_ops, float(pool_high_water), flags,
                                             C.byref(h)), "slab_server_create")
    return h.value


def slab_server_destroy(sv: int) -> None:
    load_library().slab_server_destroy(sv)


def slab_server_submit(sv: int, ops, keys, values) -> tuple[int, int]:
    """(rc, ticket): rc is SLAB_OK, SLAB_ERR_BUSY or SLAB_ERR_OUT_OF_SLABS; other codes raise."""
    import numpy as np
    n = len(keys)
    ticket = C.c_uint64(0)
    rc = load_library().slab_server_submit(sv, _hptr(ops, np.uint8, n, "ops"), _hptr(keys, np.uint32, n, "keys"),
                                           _hptr(values, np.uint32, n, "values", True), n, C.byref(ticket))
    if rc not in (SLAB_OK, SLAB_ERR_BUSY, SLAB_ERR_OUT_OF_SLABS):
        raise SlabError(rc, "slab_server_submit")
    return rc, ticket.value


def slab_server_collect(sv: int, ticket: int, n: int, wait: bool = True):
    """(results uint32[n], found uint8[n]), or None while the request runs (wait=False)."""
    import numpy as np
    res, found = np.empty(n, np.uint32), np.empty(n, np.uint8)
    rc = load_library().slab_server_collect(sv, ticket, _hptr(res, np.uint32, n, "results"),
                                            _hptr(found, np.uint8, n, "found"), int(bool(wait)))
    if rc == SLAB_ERR_BUSY:
        return None
    _check(rc, "slab_server_collect")
    return res, found


def slab_server_get_stats(sv: int) -> dict:
    st = SlabServerStats()
    _check(load_library().slab_server_get_stats(sv, C.byref(st)), "slab_server_get_stats")
    return {f: getattr(st, f) for f, _ in st._fields_ if f != "pad"}


def pinned_empty(n: int, dtype):
    """A numpy array of n elements in page-locked host memory (a pinned torch tensor's storage)."""
    import numpy as np
    tdt = {np.dtype(np.uint8): torch.uint8, np.dtype(np.uint32): torch.int32, np.dtype(np.uint64): torch.int64}
    a = torch.empty(max(int(n), 1), dtype=tdt[np.dtype(dtype)], pin_memory=True).numpy().view(dtype)
    return a[:n]


def pinned_copy(a):
    out = pinned_empty(len(a), a.dtype)
    out[:] = a
    return out


def slab_server_run(sv: int, arrival_ns, op_start, ops, keys, values, pinned_outputs: bool = False) -> dict:
    """Serve a trace (numpy arrays: uint64 arrival_ns[R], uint64 op_start[R + 1], uint8 ops, uint32 keys,
    uint32 values or None). Returns results, found, latency_ns, wait_ns, status and makespan_ns.
    With pinned_outputs the result arrays are page-locked, so the device writes them directly."""
    import numpy as np
    R = len(arrival_ns)
    total = int(op_start[R]) if R else 0
    if pinned_outputs:
        res, found = pinned_empty(total, np.uint32), pinned_empty(total, np.uint8)
    else:
        res, found = np.zeros(total, np.uint32), np.zeros(total, np.uint8)
    out = {"results": res, "found": found, "latency_ns": np.zeros(R, np.uint64), "wait_ns": np.zeros(R, np.uint64),
           "status": np.zeros(R, np.uint8)}
    mk = C.c_uint64(0)
    rc = load_library().slab_server_run(
        sv, R, _hptr(arrival_ns, np.uint64, R, "arrival_ns"), _hptr(op_start, np.uint64, R + 1, "op_start"),
        _hptr(ops, np.uint8, total, "ops"), _hptr(keys, np.uint32, total, "keys"),
        _hptr(values, np.uint32, total, "values", True), res.ctypes.data if total else None,
        found.ctypes.data if total else None, out["latency_ns"].ctypes.data, out["wait_ns"].ctypes.data,
        out["status"].ctypes.data, C.byref(mk))
    _check(rc, "slab_server_run")
    out["makespan_ns"] = mk.value
    return out


# ------------------------------------------------------------------ convenience
def as_device_u32(a, device="cuda") -> torch.Tensor:
    """A uint32 numpy array (or tensor) as a contiguous int32-typed CUDA tensor of the same bits."""
    import numpy as np
    if isinstance(a, torch.Tensor):
        return a.contiguous().to(device)
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)


def to_host_u32(t: torch.Tensor):
    import numpy as np
    return t.cpu().numpy().view(np.uint32)


class SlabHash:
    """Owns one table; methods take and return torch CUDA tensors (int32 storage of uint32 bits)."""

    def __init__(self, num_buckets: int, hash_a: int, hash_b: int, pool_slabs: int,
                 mode: int = SLAB_MODE_KEY_VALUE, slab_bytes: int = 128):
        self.handle = (slab_create(num_buckets, mode, hash_a, hash_b, pool_slabs) if slab_bytes == 128 else
                       slab_create_width(num_buckets, mode, slab_bytes, hash_a, hash_b, pool_slabs))
        self.info = slab_get_info(self.handle)
        self.mode = mode

    def close(self):
        if getattr(self, "handle", None):
            slab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, **kw):
        cfg = slab_get_config(self.handle)
        for k, v in kw.items():
            setattr(cfg, k, v)
        slab_set_config(self.handle, cfg)

    def config(self) -> dict:
        cfg = slab_get_config(self.handle)
        return {f: getattr(cfg, f) for f, _ in cfg._fields_}

    def reset(self, stream=None):
        slab_reset(self.handle, stream)

    def insert(self, keys, values=None, found=None, stream=None):
        slab_insert_batch(self.handle, keys, values, found, stream=stream)

    def delete(self, keys, found=None, stream=None):
        slab_delete_batch(self.handle, keys, found, stream=stream)

    def search(self, keys, values_out=None, found=None, stream=None):
        if values_out is None:
            values_out = torch.empty_like(keys)
        slab_search_batch(self.handle, keys, values_out, found, stream=stream)
        return values_out

    def mixed(self, ops, keys, values, results=None, found=None, stream=None):
        if results is None:
            results = torch.empty_like(keys)
        slab_mixed_batch(self.handle, ops, keys, values, results, found, stream=stream)
        return results

    def status(self, stream=None):
        return slab_status(self.handle, stream)

    def stats(self, per_bucket: bool = False, stream=None):
        if not per_bucket:
            return slab_stats(self.handle, stream=stream)
        dev = torch.device("cuda", torch.cuda.current_device())
        slots = torch.empty(self.info.num_buckets, dtype=torch.int32, device=dev)
        slabs = torch.empty_like(slots)
        tot = slab_stats(self.handle, slots, slabs, stream=stream)
        return slots, slabs, tot

    def export(self, stream=None):
        n = slab_export(self.handle, None, None, None, 0, stream=stream)
        dev = torch.device("cuda", torch.cuda.current_device())
        b = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        k = torch.empty_like(b)
        v = torch.empty_like(b)
        m = slab_export(self.handle, b, k, v, n, stream=stream)
        assert m == n
        return b[:n], k[:n], v[:n]

    def bitmaps(self, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        out = torch.empty(self.info.num_memory_blocks * 32, dtype=torch.int32, device=dev)
        slab_copy_bitmaps(self.handle, out, stream=stream)
        return out

    def buckets_of(self, keys, stream=None):
        out = torch.empty_like(keys)
        slab_bucket_of(self.handle, keys, out, stream=stream)
        return out
