"""Helpers shared by the GPU parity tests (conversions and set-valued checks)."""
from collections import defaultdict

import numpy as np

MASK = (1 << 64) - 1


def to_dev(a):
    import torch

    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def to_np_u64(t) -> np.ndarray:
    return np.ascontiguousarray(t.cpu().numpy()).view(np.uint64)


def to_np_u8(t) -> np.ndarray:
    return t.cpu().numpy().astype(np.uint8)


def codes_buf(n):
    import torch

    return torch.full((n,), 255, dtype=torch.uint8, device="cuda")


def vals_buf(n):
    import torch

    return torch.full((n,), -7, dtype=torch.int64, device="cuda")


def ops_by_key(keys, *cols):
    """dict key -> list of (col values...) tuples, in batch order."""
    d = defaultdict(list)
    for row in zip(keys.tolist(), *(c.tolist() for c in cols)):
        d[row[0]].append(row[1:])
    return d


def assert_one_winner(keys, codes, qualifies):
    """For every distinct key: exactly one op reports 1 if qualifies(key), else
    none does; every other op reports 0."""
    for k, rows in ops_by_key(keys, codes).items():
        cs = [r[0] for r in rows]
        assert all(c in (0, 1) for c in cs), (k, cs)
        assert sum(cs) == (1 if qualifies(k) else 0), (k, cs)


def assert_same_live_set(gpu_table, oracle_table):
    gk, gv = gpu_table.export()
    gk, gv = to_np_u64(gk), to_np_u64(gv)
    ok, ov = oracle_table.export()
    o1, o2 = np.argsort(gk), np.argsort(ok)
    assert gk.size == ok.size
    assert np.array_equal(gk[o1], ok[o2])
    assert np.array_equal(gv[o1], ov[o2])
