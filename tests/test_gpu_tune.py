"""The single-call autotuner (cht_tune) through the C ABI.

It times every probe window on the table as it is and must leave the table
exactly as it found it (cells and counters), for finds and for modifying
operations (restored between trials), and return every window's median time,
fastest first.  The window it reports as fastest must give the same results as
any other (checked against the oracle).
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_same_live_set, codes_buf, to_dev, to_np_u64, to_np_u8, vals_buf

pytestmark = pytest.mark.gpu


class _Res(ctypes.Structure):
    _fields_ = [("group_width", ctypes.c_int), ("lane_cells", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("ms", ctypes.c_double)]


def _tune(lib, t, op, keys, vals, trials=3):
    import torch

    f = lib.cht_tune
    p = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [p, ctypes.c_int, p, p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(_Res), ctypes.c_uint32,
                  ctypes.POINTER(ctypes.c_uint32), p]
    res = (_Res * 64)()
    n = ctypes.c_uint32()
    st = f(t._h, op, keys.data_ptr(), vals.data_ptr() if vals is not None else None, keys.numel(), trials, res, 64,
           ctypes.byref(n), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, [(r.group_width, r.lane_cells, r.ctas_per_sm, r.ms) for r in res[: n.value]]


@pytest.mark.parametrize("op", [0, 1, 4, 5])  # find, insert, erase, update(add)
def test_tune_leaves_table_unchanged(cuda_lib, oracle_mod, op):
    lib = cuda_lib.load_library()
    c = 1 << 16
    wl = W.bounded_workload(16, loads=(0.7,), n_find=20_000)
    m = wl["counts"][0.7]
    t = cuda_lib.Table(c)
    t.insert(to_dev(wl["keys"][:m]), to_dev(wl["vals"][:m]))
    o = oracle_mod.OracleTable(c)
    o.insert(wl["keys"][:m], wl["vals"][:m])
    before = to_np_u64(t.cells())
    size0 = t.size(check=True)
    if op == 1:
        k = W.uniform_keys(5000, start=10**8, seed=70)
    elif op == 0:
        k = np.concatenate([wl["hits"][0.7], wl["misses"][:5000]])
    else:
        k = wl["hits"][0.7]
    st, res = _tune(lib, t, op, to_dev(k), to_dev(W.values_for(k)))
    assert st == cuda_lib.CHT_OK
    assert len(res) == 32  # 16 windows x 2 CTA counts
    assert [r[3] for r in res] == sorted(r[3] for r in res) and res[0][3] > 0
    assert np.array_equal(to_np_u64(t.cells()), before)
    assert t.size(check=True) == size0
    # the fastest window gives the oracle's results
    g, v, ct, _ = res[0]
    t.set_config(group_width=g, lane_cells=v, ctas_per_sm=ct)
    q = np.concatenate([wl["hits"][0.7], wl["misses"]])
    vo, fo = vals_buf(q.size), codes_buf(q.size)
    t.find(to_dev(q), vo, fo)
    ev, ef = o.find(q)
    assert np.array_equal(to_np_u8(fo), ef) and np.array_equal(to_np_u64(vo), ev)
    assert_same_live_set(t, o)


def test_tune_rejects_bad_arguments(cuda_lib):
    lib = cuda_lib.load_library()
    import torch

    t = cuda_lib.Table(1 << 10)
    k = torch.ones(16, dtype=torch.int64, device="cuda")
    assert _tune(lib, t, 9, k, None)[0] == cuda_lib.CHT_ERR_INVALID_ARG  # no such operation
    assert _tune(lib, t, 1, k, None)[0] == cuda_lib.CHT_ERR_INVALID_ARG  # insert without values
    t.set_config(reuse_tombstones=1)
    assert _tune(lib, t, 0, k, None)[0] == cuda_lib.CHT_ERR_INVALID_ARG  # table options are not tuned
