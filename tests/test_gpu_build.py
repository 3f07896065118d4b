"""GPU parity of the sort-based bulk build (Sec. 3 "Bulk Operations").

The build's layout is deterministic (pairs ordered by hash bits, ties in input
order, the last of equal keys kept, placed as a sequential insertion in that
order), so the GPU's cells must equal the oracle's bit for bit.  Cases cover a
single pair, less than one radix tile, several tiles with a ragged tail, many
placement chunks, heavy duplicates, a tail that wraps past the last cell, a
growable table's sizing, a bounded table that would be full, keys 0 / ~0 with
and without the full key space, host input arrays, and the empty-table rule.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import codes_buf, to_dev, to_np_u64, to_np_u8, vals_buf

pytestmark = pytest.mark.gpu

TOMB = (1 << 64) - 1


def _batch(n, distinct, seed):
    rng = np.random.default_rng(seed)
    base = W.uniform_keys(distinct, start=seed * 1_000_000, seed=41)
    keys = base[rng.permutation(distinct)] if n == distinct else base[rng.integers(0, distinct, n)]
    vals = rng.integers(1, 1 << 62, n).astype(np.uint64)
    return np.ascontiguousarray(keys, dtype=np.uint64), vals


def _both(cuda_lib, oracle_mod, c, keys, vals, **kw):
    t = cuda_lib.Table(c, **kw)
    t.build(to_dev(keys), to_dev(vals))
    o = oracle_mod.OracleTable(c, **kw)
    r = o.build(keys, vals)
    return t, o, r


@pytest.mark.parametrize("log2c,n,distinct", [
    (10, 1, 1),             # a single pair
    (12, 2000, 1500),       # less than one radix tile (2048), duplicates
    (14, 9001, 7000),       # several tiles, ragged tail
    (16, 59000, 58000),     # load 0.885: long runs
    (16, 70000, 3000),      # each key about 23 times
    (18, 200003, 200003),   # load 0.76, no duplicates, many placement chunks
])
def test_build_layout_equals_oracle(cuda_lib, oracle_mod, log2c, n, distinct):
    keys, vals = _batch(n, distinct, seed=log2c + n % 97)
    t, o, r = _both(cuda_lib, oracle_mod, 1 << log2c, keys, vals)
    assert r == 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    live, ne, cap = t.size(check=True)
    assert live == ne == o.live and cap == 1 << log2c
    import torch

    q = to_dev(keys)
    got = torch.empty_like(q)
    t.find(q, got)
    ov, _ = o.find(keys)
    assert np.array_equal(to_np_u64(got), ov)


def test_build_wraps_tail(cuda_lib, oracle_mod):
    # 300 keys homed in the last 64 cells of a 4096-cell table: the sorted
    # insertion runs past the last cell and wraps to the front
    log2c = 12
    cand = W.uniform_keys(200_000, start=0, seed=17)
    h = oracle_mod.homes(cand, log2c)
    tail = cand[h >= (1 << log2c) - 64][:300]
    front = cand[h < 8][:10]
    keys = np.concatenate([tail, front])
    vals = np.arange(1, keys.size + 1, dtype=np.uint64)
    t, o, r = _both(cuda_lib, oracle_mod, 1 << log2c, keys, vals)
    assert r == 0
    cells = o.cells()
    assert cells[0, 0] != 0 and cells[(1 << log2c) - 1, 0] != 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), cells)


def test_build_growable_sizing(cuda_lib, oracle_mod):
    keys, vals = _batch(5000, 4000, seed=8)
    t, o, r = _both(cuda_lib, oracle_mod, 1024, keys, vals, growable=True)
    assert r == 0
    assert t.size()[2] == o.capacity == 16384  # 5000 <= 0.5 * 16384
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())


def test_build_full_then_fits(cuda_lib, oracle_mod):
    import paper_1601_04017_gb300 as cht

    ks = W.uniform_keys(1024, start=0, seed=12)
    t = cht.Table(1024)
    with pytest.raises(cht.ChtError) as ei:
        t.build(to_dev(ks), to_dev(ks))     # 1024 distinct keys leave no empty cell
    assert ei.value.status == cht.CHT_ERR_TABLE_FULL
    assert t.size()[0] == 0 and (to_np_u64(t.cells()) == 0).all()
    t.build(to_dev(ks[:1023]), to_dev(ks[:1023]))
    o = oracle_mod.OracleTable(1024)
    assert o.build(ks[:1023], ks[:1023]) == 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    with pytest.raises(cht.ChtError) as ei:
        t.build(to_dev(ks[:1]), to_dev(ks[:1]))  # not empty any more
    assert ei.value.status == cht.CHT_ERR_INVALID_ARG
    t.clear()
    t.build(to_dev(ks[:10]), to_dev(ks[:10]))    # empty again after clear
    assert t.size()[0] == 10


@pytest.mark.parametrize("full", [False, True])
def test_build_reserved_keys(cuda_lib, oracle_mod, full):
    keys, vals = _batch(3000, 2500, seed=6)
    keys = keys.copy()
    keys[[5, 700, 2999]] = [0, TOMB, 0]
    t = cuda_lib.Table(4096)
    t.set_config(full_key_space=int(full))
    t.build(to_dev(keys), to_dev(vals))
    o = oracle_mod.OracleTable(4096, full_key_space=full)
    assert o.build(keys, vals) == (0 if full else 1)
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    assert t.size()[0] == o.live
    assert bool(t.status() & 2) == (not full)
    if full:
        import torch

        q = to_dev(np.array([0, TOMB], dtype=np.uint64))
        got = torch.empty_like(q)
        t.find(q, got)
        assert to_np_u64(got).tolist() == [int(vals[2999]), int(vals[700])]


def test_build_from_host_arrays_and_empty_batch(cuda_lib, oracle_mod):
    keys, vals = _batch(30000, 20000, seed=3)
    t = cuda_lib.Table(1 << 16)
    t.build(keys[:0], vals[:0])
    assert t.size()[0] == 0
    t.build(keys, vals)                      # numpy: staged through the library
    o = oracle_mod.OracleTable(1 << 16)
    assert o.build(keys, vals) == 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())


def _unfmix64(h):
    """Inverse of the MurmurHash3 fmix64 finalizer (test-side, checked against the oracle's hash)."""
    m = (1 << 64) - 1
    x = h
    x ^= x >> 33
    x = (x * pow(0xc4ceb9fe1a85ec53, -1, 1 << 64)) & m
    x ^= x >> 33
    x = (x * pow(0xff51afd7ed558ccd, -1, 1 << 64)) & m
    x ^= x >> 33
    return x


def test_build_runs_mixing_keys(cuda_lib, oracle_mod):
    # Two keys whose hashes differ only in the lowest bit share every sort
    # bit: their copies form one run, in input order.  A copy of the rare key
    # followed by hundreds of copies of the other defers its survivor test to
    # a CTA-wide scan of the run (both outcomes: a later copy exists / does not).
    base = W.uniform_keys(40_000, start=7_000_000, seed=23)
    hk = int(oracle_mod.hash64(base[:1])[0])
    k_hot = int(base[0])
    k_rare = _unfmix64(hk ^ 1)
    assert int(oracle_mod.hash64(np.array([k_rare], dtype=np.uint64))[0]) == hk ^ 1
    k3 = int(base[1])
    k3_twin = _unfmix64(int(oracle_mod.hash64(base[1:2])[0]) ^ 2)
    run = ([k_rare] + [k_hot] * 300 + [k_rare] + [k_hot] * 200 +   # rare: not the last, then the last
           [k3_twin] + [k3] * 500)                                  # twin: single copy before 500 others
    keys = np.concatenate([base[2:20_000], np.array(run, dtype=np.uint64), base[20_000:]])
    vals = np.arange(1, keys.size + 1, dtype=np.uint64)
    t, o, r = _both(cuda_lib, oracle_mod, 1 << 17, keys, vals)
    assert r == 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    last = {}
    for k, v in zip(keys.tolist(), vals.tolist()):
        last[k] = v
    import torch

    q = np.array([k_hot, k_rare, k3, k3_twin], dtype=np.uint64)
    got = torch.empty(4, dtype=torch.int64, device="cuda")
    t.find(to_dev(q), got)
    assert to_np_u64(got).tolist() == [last[int(k)] for k in q]
    assert t.size()[0] == len(last)


# ---------------------------------------------------------------------------
# bulk merge into a non-empty table (Sec. 4.5): layout bit-exact vs the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log2c,n_ins,n_erase,n,growable,full", [
    (10, 400, 100, 500, False, False),
    (16, 20_000, 5_000, 30_000, True, False),    # grows to 2^17
    (16, 30_000, 3_000, 20_000, False, True),    # full key space, keys 0 / ~0 in the batch
    (18, 100_000, 50_000, 200_000, True, True),  # many tombstones dropped, grows to 2^20
])
def test_merge_layout_equals_oracle(cuda_lib, oracle_mod, log2c, n_ins, n_erase, n, growable, full):
    c = 1 << log2c
    keys = W.uniform_keys(n_ins, start=log2c * 100_000, seed=25)
    t = cuda_lib.Table(c, growable=growable)
    t.set_config(full_key_space=int(full))
    t.insert(to_dev(keys), to_dev(keys ^ np.uint64(77)))
    t.erase(to_dev(keys[:n_erase]))
    o = oracle_mod.OracleTable(c, growable=growable, alpha=0.5, full_key_space=full)
    o.load_cells(to_np_u64(t.cells()).reshape(-1, 2))
    if full:
        z = np.array([0], np.uint64)
        t.insert(to_dev(z), to_dev(np.array([11], np.uint64)))
        o.insert(z, np.array([11], np.uint64))
    rng = np.random.default_rng(log2c)
    pool = np.concatenate([keys, W.uniform_keys(n, start=9 * 10**8, seed=25)])
    bk = pool[rng.integers(0, pool.size, n)]
    bv = rng.integers(1, 1 << 62, n).astype(np.uint64)
    if full:
        bk[::1000] = (1 << 64) - 1
    t.merge(to_dev(bk), to_dev(bv))
    assert o.merge(bk, bv) == 0
    got = to_np_u64(t.cells()).reshape(-1, 2)
    assert got.shape == o.cells().shape
    assert np.array_equal(got, o.cells())
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    if full:
        q = np.array([0, (1 << 64) - 1], np.uint64)
        vo, fo = vals_buf(2), codes_buf(2)
        t.find(to_dev(q), vo, fo)
        ev, ef = o.find(q)
        assert np.array_equal(to_np_u8(fo), ef) and np.array_equal(to_np_u64(vo), ev)


def test_merge_full_bounded_table_unchanged_and_host_arrays(cuda_lib, oracle_mod):
    c = 1 << 10
    keys = W.uniform_keys(900, start=3_000_000, seed=26)
    t = cuda_lib.Table(c)
    t.insert(to_dev(keys), to_dev(keys))
    before = to_np_u64(t.cells())
    more = W.uniform_keys(200, start=4_000_000, seed=26)
    with pytest.raises(cuda_lib.ChtError) as ei:
        t.merge(to_dev(more), to_dev(more))
    assert ei.value.status == cuda_lib.CHT_ERR_TABLE_FULL
    assert np.array_equal(to_np_u64(t.cells()), before) and t.size()[0] == 900
    # host arrays, staged by the library; equals the oracle
    o = oracle_mod.OracleTable(c)
    o.load_cells(before.reshape(-1, 2))
    t.merge(more[:100], more[:100] + np.uint64(1))
    assert o.merge(more[:100], more[:100] + np.uint64(1)) == 0
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    # into an empty table the merge is the build
    k, v = _batch(5000, 3000, seed=8)
    a, b = cuda_lib.Table(1 << 14), cuda_lib.Table(1 << 14)
    a.merge(to_dev(k), to_dev(v))
    b.build(to_dev(k), to_dev(v))
    assert np.array_equal(to_np_u64(a.cells()), to_np_u64(b.cells()))
