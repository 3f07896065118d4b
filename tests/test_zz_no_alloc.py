"""cht_find_noalloc against cht_find (GPU, through the C ABI).

The allocation-free find stages keys and results through one fixed device
array instead of allocating; it must return exactly what cht_find returns
(bit-exact values and codes, the tolerance of every integer result in this
suite), on consecutive calls that reuse the same scratch, without changing
the library's allocated bytes.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _lib_call(lib, table, keys, vals_out, found, stream):
    f = lib.cht_find_noalloc
    p = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [p, p, ctypes.c_uint64, p, p, p]
    return f(table._h, keys.ctypes.data, keys.size, vals_out.ctypes.data,
             found.ctypes.data if found is not None else None, stream)


def test_find_noalloc_matches_find(cuda_lib):
    import torch

    lib = cuda_lib.load_library()
    c = 1 << 16
    keys = W.uniform_keys(20_000, seed=91)
    vals = W.values_for(keys)
    t = cuda_lib.Table(c)
    t.insert(torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(vals.view(np.int64)).cuda())
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    for call, n in enumerate([cuda_lib.cht.NOALLOC_MAX_KEYS, 12_345]):  # two calls in a row
        q = np.concatenate([keys[rng.integers(0, keys.size, n // 2)],
                            W.uniform_keys(n - n // 2 - 2, start=10**6 * (call + 1), seed=91),
                            np.array([0, (1 << 64) - 1], np.uint64)])
        assert q.size == n
        # existing entry point (device arrays)
        ref_v = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        ref_f = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        t.find(torch.from_numpy(q.view(np.int64)).cuda(), ref_v, ref_f)
        # allocation-free entry point (host arrays, staged through its scratch)
        got_v = np.full(n, 7, np.uint64)
        got_f = np.full(n, 9, np.uint8)
        torch.cuda.synchronize()
        before = cuda_lib.memory_in_use()
        free_before = torch.cuda.mem_get_info()[0]
        assert _lib_call(lib, t, q, got_v, got_f, stream) == cuda_lib.CHT_OK
        torch.cuda.synchronize()
        assert cuda_lib.memory_in_use() == before
        if call > 0:  # after the first call (module and scratch set up): no device bytes taken at all
            assert torch.cuda.mem_get_info()[0] == free_before
        assert np.array_equal(got_v, ref_v.cpu().numpy().view(np.uint64))
        assert np.array_equal(got_f, ref_f.cpu().numpy())
        assert (got_f[: n // 2] == 1).all() and got_f[-1] == 3
    # also through the binding, with device arrays and without codes
    dq = torch.from_numpy(keys[:1000].view(np.int64)).cuda()
    dv = torch.zeros(1000, dtype=torch.int64, device="cuda")
    cuda_lib.cht.find_noalloc(t, dq, dv)
    torch.cuda.synchronize()
    assert np.array_equal(dv.cpu().numpy().view(np.uint64), vals[:1000])
    # batches beyond the scratch are rejected
    big = np.ones(cuda_lib.cht.NOALLOC_MAX_KEYS + 1, np.uint64)
    out_v = np.zeros(big.size, np.uint64)
    assert _lib_call(lib, t, big, out_v, None, stream) == cuda_lib.CHT_ERR_INVALID_ARG
    t.destroy()


def test_find_noalloc_orders_destroy(cuda_lib):
    """A table destroyed right after an allocation-free find issued on another
    stream is released only once that find has finished: cht_destroy waits for
    the stream of the table's last call, and the find counts as one."""
    import torch

    c = 1 << 18
    keys = W.uniform_keys(100_000, seed=92)
    vals = W.values_for(keys)
    t = cuda_lib.Table(c)
    t.insert(torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(vals.view(np.int64)).cuda())
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    n = cuda_lib.cht.NOALLOC_MAX_KEYS
    dq = torch.from_numpy(keys[:n].view(np.int64)).cuda()
    dv = torch.zeros(n, dtype=torch.int64, device="cuda")
    df = torch.zeros(n, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000)  # keep the side stream busy, so the find is still queued
        cuda_lib.cht.find_noalloc(t, dq, dv, df, stream=side)
    t.destroy()
    assert side.query(), "cht_destroy returned before the find on the other stream finished"
    torch.cuda.synchronize()
    assert np.array_equal(dv.cpu().numpy().view(np.uint64), vals[:n])
    assert (df.cpu().numpy() == 1).all()
