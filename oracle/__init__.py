"""CPU oracle for the folklore linear-probing table (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``cht_oracle.c`` -- a plain,
single-threaded C restatement of the paper's table (Sec. 3 Algorithm 1,
Sec. 4.3.1 sequential migration, Sec. 4.4 tombstones) -- through ctypes and
numpy.  It shares no code with the CUDA library and imports nothing from it.

All arrays are numpy ``uint64`` (keys, values, raw cells) or ``uint8``
(per-operation result codes: 0 no, 1 yes, 2 table full, 3 reserved key).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cht_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcht_oracle.so")
_lock = threading.Lock()
_lib = None

OVERWRITE = 0
ADD = 1
EMPTY = 0
TOMBSTONE = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (a second or two)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        sig = {
            "or_hash": (u64, [u64]),
            "or_home": (u64, [p, u64]),
            "or_hash_many": (None, [p, u64, p]),
            "or_home_many": (None, [p, u64, ctypes.c_uint, p]),
            "or_create": (p, [u64, ctypes.c_int, ctypes.c_double]),
            "or_destroy": (None, [p]),
            "or_set_reuse": (None, [p, ctypes.c_int]),
            "or_set_full_keys": (None, [p, ctypes.c_int]),
            "or_capacity": (u64, [p]),
            "or_nonempty": (u64, [p]),
            "or_live": (u64, [p]),
            "or_probes": (u64, [p]),
            "or_migrations": (u64, [p]),
            "or_reset_probes": (None, [p]),
            "or_migrate": (ctypes.c_int, [p, u64]),
            "or_insert": (None, [p, p, p, u64, p]),
            "or_build": (ctypes.c_int, [p, p, p, u64]),
            "or_merge": (ctypes.c_int, [p, p, p, u64]),
            "or_build_sort_bits": (ctypes.c_uint, [ctypes.c_uint]),
            "or_insert_or_update": (None, [p, p, p, u64, ctypes.c_int, p]),
            "or_update": (None, [p, p, p, u64, ctypes.c_int, p]),
            "or_find": (None, [p, p, u64, p, p]),
            "or_erase": (None, [p, p, u64, p]),
            "or_export": (u64, [p, p, p, u64]),
            "or_dump_cells": (None, [p, p]),
            "or_load_cells": (ctypes.c_int, [p, p, u64]),
            "or_check_invariants": (ctypes.c_int, [p, ctypes.c_char_p, ctypes.c_size_t]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _u64(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype == np.int64:
        a = a.view(np.uint64)
    return np.ascontiguousarray(a, dtype=np.uint64)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def hash64(keys) -> np.ndarray:
    """The oracle's 64-bit hash of each key (MurmurHash3 fmix64)."""
    lib = _load()
    k = _u64(keys).ravel()
    out = np.zeros(k.size, dtype=np.uint64)
    lib.or_hash_many(_ptr(k), k.size, _ptr(out))
    return out


def build_sort_bits(log2c: int) -> int:
    """Hash bits the bulk build orders by in a table of 2^log2c cells."""
    return int(_load().or_build_sort_bits(int(log2c)))


def homes(keys, log2c: int) -> np.ndarray:
    """Home cell of each key in a table of 2^log2c cells (top log2c hash bits)."""
    lib = _load()
    k = _u64(keys).ravel()
    out = np.zeros(k.size, dtype=np.uint64)
    lib.or_home_many(_ptr(k), k.size, int(log2c), _ptr(out))
    return out


class OracleTable:
    """Sequential folklore table with phase semantics (one op type per call)."""

    def __init__(self, capacity: int, growable: bool = False, alpha: float = 0.5,
                 reuse_tombstones: bool = False, full_key_space: bool = False):
        self._lib = _load()
        self._t = self._lib.or_create(int(capacity), int(bool(growable)), float(alpha))
        if not self._t:
            raise MemoryError("oracle table allocation failed")
        self._lib.or_set_reuse(self._t, int(bool(reuse_tombstones)))
        self._lib.or_set_full_keys(self._t, int(bool(full_key_space)))

    def close(self):
        if self._t:
            self._lib.or_destroy(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ---------------------------------------------------------------
    @property
    def capacity(self) -> int:
        return int(self._lib.or_capacity(self._t))

    @property
    def nonempty(self) -> int:
        return int(self._lib.or_nonempty(self._t))

    @property
    def live(self) -> int:
        return int(self._lib.or_live(self._t))

    @property
    def probes(self) -> int:
        return int(self._lib.or_probes(self._t))

    @property
    def migrations(self) -> int:
        return int(self._lib.or_migrations(self._t))

    def reset_probes(self):
        self._lib.or_reset_probes(self._t)

    def home(self, key: int) -> int:
        return int(self._lib.or_home(self._t, int(key)))

    def homes(self, keys) -> np.ndarray:
        return homes(keys, self.capacity.bit_length() - 1)

    # -- operations ----------------------------------------------------------
    def insert(self, keys, vals) -> np.ndarray:
        k, v = _u64(keys), _u64(vals)
        assert k.shape == v.shape
        f = np.zeros(k.size, dtype=np.uint8)
        self._lib.or_insert(self._t, _ptr(k), _ptr(v), k.size, _ptr(f))
        return f

    def build(self, keys, vals) -> int:
        """Sort-based bulk build into the empty table (Sec. 3 "Bulk Operations").

        0 = built; 1 = built, reserved keys skipped; -1 = table not empty;
        -2 = the distinct keys would leave no empty cell (table unchanged).
        """
        k, v = _u64(keys), _u64(vals)
        assert k.shape == v.shape
        return int(self._lib.or_build(self._t, _ptr(k), _ptr(v), k.size))

    def merge(self, keys, vals) -> int:
        """Bulk merge of a batch into this (possibly non-empty) table (Sec. 4.5).

        The new table is the sorted placement of the live elements (cell index
        order) followed by the batch, keeping the last of equal keys: batch
        values replace the table's, the last of equal batch keys wins.
        0 = merged; 1 = merged, reserved keys skipped; -2 = no empty cell would
        remain (table unchanged); -1 = out of memory.
        """
        k, v = _u64(keys), _u64(vals)
        assert k.shape == v.shape
        return int(self._lib.or_merge(self._t, _ptr(k), _ptr(v), k.size))

    def insert_or_update(self, keys, vals, op: int = ADD) -> np.ndarray:
        k, v = _u64(keys), _u64(vals)
        assert k.shape == v.shape
        f = np.zeros(k.size, dtype=np.uint8)
        self._lib.or_insert_or_update(self._t, _ptr(k), _ptr(v), k.size, int(op), _ptr(f))
        return f

    def update(self, keys, vals, op: int = ADD) -> np.ndarray:
        """update (Sec. 3): change the value of present keys; 1 = updated, 0 = absent."""
        k, v = _u64(keys), _u64(vals)
        assert k.shape == v.shape
        f = np.zeros(k.size, dtype=np.uint8)
        self._lib.or_update(self._t, _ptr(k), _ptr(v), k.size, int(op), _ptr(f))
        return f

    def find(self, keys):
        k = _u64(keys)
        v = np.zeros(k.size, dtype=np.uint64)
        f = np.zeros(k.size, dtype=np.uint8)
        self._lib.or_find(self._t, _ptr(k), k.size, _ptr(v), _ptr(f))
        return v, f

    def erase(self, keys) -> np.ndarray:
        k = _u64(keys)
        f = np.zeros(k.size, dtype=np.uint8)
        self._lib.or_erase(self._t, _ptr(k), k.size, _ptr(f))
        return f

    def migrate(self, new_capacity: int) -> None:
        if self._lib.or_migrate(self._t, int(new_capacity)) != 0:
            raise ValueError("oracle migration failed (target too small or out of memory)")

    def export(self):
        n = self.live
        k = np.zeros(max(n, 1), dtype=np.uint64)
        v = np.zeros(max(n, 1), dtype=np.uint64)
        m = int(self._lib.or_export(self._t, _ptr(k), _ptr(v), n))
        assert m == n
        return k[:m], v[:m]

    def cells(self) -> np.ndarray:
        """Raw cells as a (c, 2) uint64 array of (key, value)."""
        out = np.zeros((self.capacity, 2), dtype=np.uint64)
        self._lib.or_dump_cells(self._t, _ptr(out))
        return out

    def load_cells(self, cells) -> None:
        c = _u64(cells).reshape(-1, 2)
        if self._lib.or_load_cells(self._t, _ptr(np.ascontiguousarray(c)), c.shape[0]) != 0:
            raise ValueError("snapshot size must be a power of two >= 64")

    def check_invariants(self) -> tuple[int, str]:
        buf = ctypes.create_string_buffer(512)
        r = int(self._lib.or_check_invariants(self._t, buf, 512))
        return r, buf.value.decode()

    def assert_invariants(self) -> None:
        r, msg = self.check_invariants()
        if r != 0:
            raise AssertionError(f"table invariant {r} broken: {msg}")
