"""ctypes binding of libcht (include/cht.h): argument marshalling only.

Every array argument is a torch tensor (CUDA or CPU) or a numpy array with
8-byte elements for keys and values (int64 or uint64: the same bits) and
uint8 for result codes.  CPU arrays go through the library's host staging.
The stream defaults to torch's current CUDA stream.  There is no fallback:
if libcht.so cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

CHT_OK = 0
CHT_ERR_INVALID_ARG = 1
CHT_ERR_OOM = 2
CHT_ERR_CUDA = 3
CHT_ERR_TABLE_FULL = 4
CHT_ERR_RESERVED_KEY = 5
CHT_ERR_TIMEOUT = 6

OVERWRITE = 0
ADD = 1
STATUS_FULL = 0x1
STATUS_RESERVED = 0x2

CODE_NO, CODE_YES, CODE_FULL, CODE_RESERVED = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class ChtError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib.cht_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})")


class ChtConfig(ctypes.Structure):
    _fields_ = [("group_width", ctypes.c_int), ("lane_cells", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("migrate_tile", ctypes.c_int), ("alpha", ctypes.c_double),
                ("iou_aggregate", ctypes.c_int), ("reuse_tombstones", ctypes.c_int),
                ("full_key_space", ctypes.c_int), ("partition", ctypes.c_int), ("grow_in_kernel", ctypes.c_int),
                ("grow_spin_us", ctypes.c_int), ("grow_fault_inject", ctypes.c_int)]


OP_FIND, OP_INSERT, OP_IOU_ADD, OP_IOU_OVERWRITE, OP_ERASE = 0, 1, 2, 3, 4
OP_UPDATE_ADD, OP_UPDATE_OVERWRITE = 5, 6
PLAN_TIMEOUT = 0x1


class BatchOp(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("op", ctypes.c_int), ("keys", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("n", ctypes.c_uint64), ("vals_out", ctypes.c_void_p),
                ("codes", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_cap_bytes", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                ("max_inflight_steps", ctypes.c_uint32), ("max_step_requests", ctypes.c_uint32),
                ("max_step_ops", ctypes.c_uint64), ("stage_inputs", ctypes.c_int),
                ("hbm_reserve_bytes", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("table", ctypes.c_uint32), ("op", ctypes.c_int), ("keys", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("n", ctypes.c_uint64), ("vals_out", ctypes.c_void_p),
                ("codes", ctypes.c_void_p)]


class ServerProfile(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("parts", ctypes.c_uint64),
                ("chunks", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("migrations", ctypes.c_uint64),
                ("gpu_step_ms", ctypes.c_double), ("engine_ms", ctypes.c_double), ("host_admit_ms", ctypes.c_double)]


class ServerStepRecord(ctypes.Structure):
    _fields_ = [("gpu_ms", ctypes.c_double), ("engine_ms", ctypes.c_double), ("parts", ctypes.c_uint64),
                ("items", ctypes.c_uint64), ("ops", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("migrations", ctypes.c_uint64), ("max_table_log2", ctypes.c_uint32), ("recut", ctypes.c_uint32)]


class PlanConfig(ctypes.Structure):
    _fields_ = [("group_width", ctypes.c_int), ("lane_cells", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("spin_limit_us", ctypes.c_int), ("fault_inject", ctypes.c_int), ("direct_io", ctypes.c_int),
                ("chunk_ops", ctypes.c_int), ("poll_ns", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load libcht.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcht.so not found at {path}")
        lib = ctypes.CDLL(path)
        p, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        sigs = {
            "cht_create": (i32, [u64, i32, p, ctypes.POINTER(p)]),
            "cht_destroy": (i32, [p]),
            "cht_set_config": (i32, [p, ctypes.POINTER(ChtConfig)]),
            "cht_get_config": (i32, [p, ctypes.POINTER(ChtConfig)]),
            "cht_insert": (i32, [p, p, p, u64, p, p]),
            "cht_build": (i32, [p, p, p, u64, p]),
            "cht_merge": (i32, [p, p, p, u64, p]),
            "cht_find": (i32, [p, p, u64, p, p, p]),
            "cht_insert_or_update": (i32, [p, p, p, u64, i32, p, p]),
            "cht_update": (i32, [p, p, p, u64, i32, p, p]),
            "cht_erase": (i32, [p, p, u64, p, p]),
            "cht_migrate": (i32, [p, u64, p]),
            "cht_size": (i32, [p, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64), p]),
            "cht_get_status": (i32, [p, ctypes.POINTER(ctypes.c_uint32), p]),
            "cht_export": (i32, [p, p, p, u64, ctypes.POINTER(u64), p]),
            "cht_copy_cells": (i32, [p, p, u64, ctypes.POINTER(u64), p]),
            "cht_clear": (i32, [p, p]),
            "cht_set_memory_limit": (i32, [u64]),
            "cht_memory_in_use": (u64, []),
            "cht_launch_count": (u64, []),
            "cht_status_string": (ctypes.c_char_p, [i32]),
            "cht_version": (i32, []),
            "cht_plan_create": (i32, [p, u64, ctypes.POINTER(p)]),
            "cht_plan_set_config": (i32, [p, ctypes.POINTER(PlanConfig)]),
            "cht_plan_get_config": (i32, [p, ctypes.POINTER(PlanConfig)]),
            "cht_plan_launch": (i32, [p, p]),
            "cht_plan_status": (i32, [p, ctypes.POINTER(ctypes.c_uint32), p]),
            "cht_plan_autotune": (i32, [p, p, ctypes.POINTER(ctypes.c_double)]),
            "cht_plan_destroy": (i32, [p]),
            "cht_server_create": (i32, [p, ctypes.c_uint32, ctypes.POINTER(ServerConfig), p, ctypes.POINTER(p)]),
            "cht_server_submit": (i32, [p, ctypes.POINTER(Request), ctypes.POINTER(u64)]),
            "cht_server_step": (i32, [p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
            "cht_server_drain": (i32, [p]),
            "cht_server_result": (i32, [p, u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]),
            "cht_server_replay": (i32, [p, p, p, u64, p, ctypes.POINTER(ctypes.c_double)]),
            "cht_server_stats": (i32, [p, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
            "cht_server_get_profile": (i32, [p, ctypes.POINTER(ServerProfile)]),
            "cht_server_get_trace": (i32, [p, ctypes.POINTER(ServerStepRecord), u64, ctypes.POINTER(u64)]),
            "cht_server_destroy": (i32, [p]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != CHT_OK:
        raise ChtError(status, what)


def _ptr(x, elem_size: int, n: int | None = None, what: str = "array"):
    """(pointer, element count, is_cuda) of a tensor / numpy array."""
    if x is None:
        return None, 0, False
    if isinstance(x, np.ndarray):
        if x.dtype.itemsize != elem_size or not x.flags.c_contiguous:
            raise TypeError(f"{what}: need a contiguous array of {elem_size}-byte elements")
        cnt = x.size
        ptr = x.ctypes.data if cnt else None
        cuda = False
    else:
        if x.element_size() != elem_size or not x.is_contiguous():
            raise TypeError(f"{what}: need a contiguous tensor of {elem_size}-byte elements")
        cnt = x.numel()
        ptr = x.data_ptr() if cnt else None
        cuda = x.is_cuda
    if n is not None and cnt < n:
        raise ValueError(f"{what}: holds {cnt} elements, need {n}")
    return ptr, cnt, cuda


def _stream(stream, device=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def memory_in_use() -> int:
    return int(load_library().cht_memory_in_use())


def set_memory_limit(nbytes: int) -> None:
    _check(load_library().cht_set_memory_limit(int(nbytes)), "cht_set_memory_limit")


def launch_count() -> int:
    return int(load_library().cht_launch_count())


def version() -> int:
    return int(load_library().cht_version())


class Table:
    """A libcht table.  Methods mirror the C ABI (cht_insert, cht_find, ...)."""

    def __init__(self, capacity: int, growable: bool = False, stream=None, config: dict | None = None):
        import torch

        self._lib = load_library()
        self.device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        _check(self._lib.cht_create(int(capacity), int(bool(growable)), _stream(stream), ctypes.byref(h)),
               "cht_create")
        self._h = h
        if config:
            self.set_config(**config)

    # -- lifetime ------------------------------------------------------------
    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(self._lib.cht_destroy(self._h), "cht_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    # -- configuration -------------------------------------------------------
    def config(self) -> dict:
        c = ChtConfig()
        _check(self._lib.cht_get_config(self._h, ctypes.byref(c)), "cht_get_config")
        return {f: getattr(c, f) for f, _ in ChtConfig._fields_}

    def set_config(self, **kw):
        cur = self.config()
        cur.update(kw)
        c = ChtConfig(*(float(cur[f]) if t is ctypes.c_double else int(cur[f]) for f, t in ChtConfig._fields_))
        _check(self._lib.cht_set_config(self._h, ctypes.byref(c)), "cht_set_config")

    # -- operations ----------------------------------------------------------
    def insert(self, keys, vals, inserted=None, stream=None):
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        cp, _, _ = _ptr(inserted, 1, n, "inserted")
        _check(self._lib.cht_insert(self._h, kp, vp, n, cp, _stream(stream)), "cht_insert")
        return inserted

    def build(self, keys, vals, stream=None):
        """Sort-based bulk build of this empty table (keeps the last of equal keys)."""
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        _check(self._lib.cht_build(self._h, kp, vp, n, _stream(stream)), "cht_build")

    def merge(self, keys, vals, stream=None):
        """Bulk merge of a batch into this table (Sec. 4.5): batch values replace
        the table's, the last of equal batch keys wins; a new, sorted layout."""
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        _check(self._lib.cht_merge(self._h, kp, vp, n, _stream(stream)), "cht_merge")

    def find(self, keys, vals_out, found=None, stream=None):
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals_out, 8, n, "vals_out")
        cp, _, _ = _ptr(found, 1, n, "found")
        _check(self._lib.cht_find(self._h, kp, n, vp, cp, _stream(stream)), "cht_find")
        return vals_out, found

    def insert_or_update(self, keys, vals, op: int = ADD, inserted=None, stream=None):
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        cp, _, _ = _ptr(inserted, 1, n, "inserted")
        _check(self._lib.cht_insert_or_update(self._h, kp, vp, n, int(op), cp, _stream(stream)),
               "cht_insert_or_update")
        return inserted

    def update(self, keys, vals, op: int = ADD, updated=None, stream=None):
        """cht_update: change the values of present keys (1 = updated, 0 = absent)."""
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        cp, _, _ = _ptr(updated, 1, n, "updated")
        _check(self._lib.cht_update(self._h, kp, vp, n, int(op), cp, _stream(stream)), "cht_update")
        return updated

    def erase(self, keys, erased=None, stream=None):
        kp, n, _ = _ptr(keys, 8, what="keys")
        cp, _, _ = _ptr(erased, 1, n, "erased")
        _check(self._lib.cht_erase(self._h, kp, n, cp, _stream(stream)), "cht_erase")
        return erased

    def migrate(self, new_capacity: int = 0, stream=None):
        _check(self._lib.cht_migrate(self._h, int(new_capacity), _stream(stream)), "cht_migrate")

    def clear(self, stream=None):
        _check(self._lib.cht_clear(self._h, _stream(stream)), "cht_clear")

    # -- state ---------------------------------------------------------------
    def size(self, stream=None, check: bool = False):
        """(live, nonempty, capacity); raises on a set status bit if check."""
        live, ne, cap = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        r = self._lib.cht_size(self._h, ctypes.byref(live), ctypes.byref(ne), ctypes.byref(cap),
                               _stream(stream))
        if r not in (CHT_OK, CHT_ERR_TABLE_FULL, CHT_ERR_RESERVED_KEY) or (check and r != CHT_OK):
            _check(r, "cht_size")
        return int(live.value), int(ne.value), int(cap.value)

    @property
    def capacity(self) -> int:
        return self.size()[2]

    def status(self, stream=None) -> int:
        bits = ctypes.c_uint32()
        _check(self._lib.cht_get_status(self._h, ctypes.byref(bits), _stream(stream)), "cht_get_status")
        return int(bits.value)

    def export(self, stream=None):
        """Live (keys, values) as CUDA int64 tensors, in no particular order."""
        import torch

        live = self.size(stream)[0]
        k = torch.empty(max(live, 1), dtype=torch.int64, device=f"cuda:{self.device}")
        v = torch.empty_like(k)
        n = ctypes.c_uint64()
        _check(self._lib.cht_export(self._h, k.data_ptr(), v.data_ptr(), live, ctypes.byref(n),
                                    _stream(stream)), "cht_export")
        return k[: n.value], v[: n.value]

    def cells(self, stream=None):
        """Raw cells as a (c, 2) CUDA int64 tensor of (key, value)."""
        import torch

        cap = self.size(stream)[2]
        out = torch.empty((cap, 2), dtype=torch.int64, device=f"cuda:{self.device}")
        n = ctypes.c_uint64()
        _check(self._lib.cht_copy_cells(self._h, out.data_ptr(), cap, ctypes.byref(n), _stream(stream)),
               "cht_copy_cells")
        return out


class Plan:
    """cht_plan_*: many batches over many tables, run by one kernel launch.

    `ops` is a list of (table, op, keys, vals, vals_out, codes) tuples with CUDA
    tensors (vals / vals_out / codes may be None where unused).  Batches on the
    same table run in list order; the arrays must stay alive with the plan,
    and no keys / vals array may overlap a vals_out / codes array.
    """

    def __init__(self, ops):
        self._lib = load_library()
        arr = (BatchOp * max(len(ops), 1))()
        self._keep = []
        for i, (table, op, keys, vals, vals_out, codes) in enumerate(ops):
            kp, n, _ = _ptr(keys, 8, what="keys")
            vp, _, _ = _ptr(vals, 8, n, "vals")
            op_, _, _ = _ptr(vals_out, 8, n, "vals_out")
            cp, _, _ = _ptr(codes, 1, n, "codes")
            arr[i] = BatchOp(table._h.value, int(op), kp, vp, n, op_, cp)
            self._keep.append((keys, vals, vals_out, codes))
        h = ctypes.c_void_p()
        _check(self._lib.cht_plan_create(arr, len(ops), ctypes.byref(h)), "cht_plan_create")
        self._h = h

    def config(self) -> dict:
        c = PlanConfig()
        _check(self._lib.cht_plan_get_config(self._h, ctypes.byref(c)), "cht_plan_get_config")
        return {f: getattr(c, f) for f, _ in PlanConfig._fields_}

    def set_config(self, **kw):
        cur = self.config()
        cur.update(kw)
        c = PlanConfig(*(int(cur[f]) for f, _ in PlanConfig._fields_))
        _check(self._lib.cht_plan_set_config(self._h, ctypes.byref(c)), "cht_plan_set_config")

    def launch(self, stream=None):
        _check(self._lib.cht_plan_launch(self._h, _stream(stream)), "cht_plan_launch")

    def status(self, stream=None) -> int:
        bits = ctypes.c_uint32()
        _check(self._lib.cht_plan_status(self._h, ctypes.byref(bits), _stream(stream)), "cht_plan_status")
        return int(bits.value)

    def autotune(self, stream=None) -> float:
        ms = ctypes.c_double()
        _check(self._lib.cht_plan_autotune(self._h, _stream(stream), ctypes.byref(ms)), "cht_plan_autotune")
        return float(ms.value)

    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(self._lib.cht_plan_destroy(self._h), "cht_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """cht_server_*: continuous batching of requests over resident tables.

    Requests are (table index, op, keys, vals, vals_out, codes) with host or
    device arrays that stay alive until the request completes.
    """

    def __init__(self, tables, memory_cap_bytes=0, arena_bytes=0, max_inflight_steps=0, max_step_requests=0,
                 max_step_ops=0, stage_inputs=0, hbm_reserve_bytes=0, stream=None):
        self._lib = load_library()
        arr = (ctypes.c_void_p * len(tables))(*[t._h.value for t in tables])
        cfg = ServerConfig(int(memory_cap_bytes), int(arena_bytes), int(max_inflight_steps),
                           int(max_step_requests), int(max_step_ops), int(stage_inputs), int(hbm_reserve_bytes))
        h = ctypes.c_void_p()
        _check(self._lib.cht_server_create(arr, len(tables), ctypes.byref(cfg), _stream(stream), ctypes.byref(h)),
               "cht_server_create")
        self._h = h
        self._tables = tables
        self._keep = []

    @staticmethod
    def request(table, op, keys, vals=None, vals_out=None, codes=None) -> Request:
        kp, n, _ = _ptr(keys, 8, what="keys")
        vp, _, _ = _ptr(vals, 8, n, "vals")
        op_, _, _ = _ptr(vals_out, 8, n, "vals_out")
        cp, _, _ = _ptr(codes, 1, n, "codes")
        return Request(int(table), int(op), kp, vp, n, op_, cp)

    def submit(self, table, op, keys, vals=None, vals_out=None, codes=None) -> int:
        r = self.request(table, op, keys, vals, vals_out, codes)
        self._keep.append((keys, vals, vals_out, codes))
        rid = ctypes.c_uint64()
        _check(self._lib.cht_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), "cht_server_submit")
        return int(rid.value)

    def step(self):
        a, c = ctypes.c_uint32(), ctypes.c_uint32()
        _check(self._lib.cht_server_step(self._h, ctypes.byref(a), ctypes.byref(c)), "cht_server_step")
        return int(a.value), int(c.value)

    def drain(self):
        _check(self._lib.cht_server_drain(self._h), "cht_server_drain")

    def result(self, rid):
        done, lat, st = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(self._lib.cht_server_result(self._h, int(rid), ctypes.byref(done), ctypes.byref(lat),
                                           ctypes.byref(st)), "cht_server_result")
        return bool(done.value), float(lat.value), int(st.value)

    def replay(self, requests, arrival_s):
        """Submit requests[i] at arrival_s[i] (seconds from now); returns
        (latencies, makespan)."""
        n = len(requests)
        arr = (Request * max(n, 1))(*requests)
        arrivals = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(max(n, 1), dtype=np.float64)
        mk = ctypes.c_double()
        _check(self._lib.cht_server_replay(self._h, arr, arrivals.ctypes.data, n, lat.ctypes.data, ctypes.byref(mk)),
               "cht_server_replay")
        return lat[:n], float(mk.value)

    def stats(self):
        st, done = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.cht_server_stats(self._h, ctypes.byref(st), ctypes.byref(done)), "cht_server_stats")
        return int(st.value), int(done.value)

    def profile(self) -> dict:
        """Where the server's time went (cht_server_get_profile)."""
        pr = ServerProfile()
        _check(self._lib.cht_server_get_profile(self._h, ctypes.byref(pr)), "cht_server_get_profile")
        return {f: getattr(pr, f) for f, _ in ServerProfile._fields_}

    def trace(self) -> np.ndarray:
        """Per-step records (cht_server_get_trace) as a structured array."""
        n = ctypes.c_uint64()
        _check(self._lib.cht_server_get_trace(self._h, None, 0, ctypes.byref(n)), "cht_server_get_trace")
        recs = (ServerStepRecord * max(int(n.value), 1))()
        _check(self._lib.cht_server_get_trace(self._h, recs, n.value, ctypes.byref(n)), "cht_server_get_trace")
        dt = np.dtype([(f, np.float64 if t is ctypes.c_double else np.uint64 if t is ctypes.c_uint64 else np.uint32)
                       for f, t in ServerStepRecord._fields_])
        out = np.zeros(int(n.value), dt)
        for i in range(int(n.value)):
            out[i] = tuple(getattr(recs[i], f) for f, _ in ServerStepRecord._fields_)
        return out

    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(self._lib.cht_server_destroy(self._h), "cht_server_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


NOALLOC_MAX_KEYS = 65536


def find_noalloc(table: Table, keys, vals_out, found=None, stream=None):
    """cht_find_noalloc: find that allocates no device memory.

    For callers that cannot allocate device memory where they look keys up
    (memory owned by another allocator, allocation-free request paths, fixed
    budgets).  Keys and results pass through the library's fixed scratch
    array, so at most NOALLOC_MAX_KEYS keys per call; calls that overlap on
    the GPU share that array and race, so keep them ordered.  Host results are
    valid after the stream is synchronized.
    """
    lib = load_library()
    f = lib.cht_find_noalloc
    if f.argtypes is None:
        p = ctypes.c_void_p
        f.restype = ctypes.c_int
        f.argtypes = [p, p, ctypes.c_uint64, p, p, p]
    kp, n, _ = _ptr(keys, 8, what="keys")
    vp, _, _ = _ptr(vals_out, 8, n, "vals_out")
    cp, _, _ = _ptr(found, 1, n, "found")
    _check(f(table._h, kp, n, vp, cp, _stream(stream)), "cht_find_noalloc")
    return vals_out, found
