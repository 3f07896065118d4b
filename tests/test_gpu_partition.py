"""GPU parity of the hash-partitioned path (Sec. 4.5 "Bulk Operations") against the oracle.

`partition = 1` runs the path on small tables too, so every operation type,
table option and a ragged batch (not a multiple of the 2048-operation tile,
a batch below one tile, one operation) runs through the reorder, the in-order
operation kernel and the gather of the results.  The bar is the direct path's:
bit-exact finds, codes and sums; set-valued where equal keys inside one batch
allow several outcomes.  A final case runs a 2^22-cell table at load 0.9 both
ways.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import (assert_one_winner, assert_same_live_set, codes_buf, to_dev, to_np_u8, to_np_u64,
                         vals_buf)

pytestmark = pytest.mark.gpu

SIZES = [1, 2047, 2048, 2049, 40_001]


def _pair(cht, oracle_mod, c, growable=False, **cfg):
    t = cht.Table(c, growable=growable)
    t.set_config(partition=1, **cfg)
    o = oracle_mod.OracleTable(c, growable=growable, alpha=0.5,
                               reuse_tombstones=bool(cfg.get("reuse_tombstones", 0)),
                               full_key_space=bool(cfg.get("full_key_space", 0)))
    return t, o


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("load", [0.5, 0.9])
def test_partitioned_insert_find_erase(cuda_lib, oracle_mod, n, load):
    log2c = 16
    c = 1 << log2c
    wl = W.bounded_workload(log2c, loads=(load,), n_find=n)
    m = wl["counts"][load]
    keys, vals = wl["keys"][:m], wl["vals"][:m]
    t, o = _pair(cuda_lib, oracle_mod, c)
    codes = codes_buf(m)
    t.insert(to_dev(keys), to_dev(vals), codes)
    assert np.array_equal(to_np_u8(codes), o.insert(keys, vals))
    gcells = to_np_u64(t.cells())
    assert np.array_equal(gcells.reshape(-1, 2)[:, 0] != 0, o.cells()[:, 0] != 0)
    for q in (wl["hits"][load], wl["misses"]):
        vo, fo = vals_buf(q.size), codes_buf(q.size)
        t.find(to_dev(q), vo, fo)
        ev, ef = o.find(q)
        assert np.array_equal(to_np_u8(fo), ef)
        assert np.array_equal(to_np_u64(vo), ev)
        vo2 = vals_buf(q.size)
        t.find(to_dev(q), vo2)  # no codes array: only the values are gathered
        assert np.array_equal(to_np_u64(vo2), ev)
    er = np.concatenate([wl["hits"][load][: n // 2], wl["misses"][: n - n // 2]])
    ec = codes_buf(er.size)
    t.erase(to_dev(er), ec)
    assert np.array_equal(to_np_u8(ec), o.erase(er))
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    assert_same_live_set(t, o)


@pytest.mark.parametrize("s", [0.5, 1.25])
@pytest.mark.parametrize("agg", [0, 1])
@pytest.mark.parametrize("n", [2049, 150_001])
def test_partitioned_insert_or_update_add(cuda_lib, oracle_mod, s, agg, n):
    c = 1 << 17
    keys = W.zipf_keys(n, s, n_ranks=1 << 15, seed=61)
    vals = (np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) | np.uint64(1)
    keys[::997] = 0
    pre = np.unique(keys[keys != 0])[::5]
    t, o = _pair(cuda_lib, oracle_mod, c, iou_aggregate=agg)
    t.insert(to_dev(pre), to_dev(pre))
    o.insert(pre, pre)
    codes = codes_buf(n)
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.ADD, codes)
    o.insert_or_update(keys, vals, oracle_mod.ADD)
    cs = to_np_u8(codes)
    assert (cs[keys == 0] == 3).all()
    pre_set = set(pre.tolist())
    live_ops = keys != 0
    assert_one_winner(keys[live_ops], cs[live_ops], lambda k: k not in pre_set)
    assert_same_live_set(t, o)


@pytest.mark.parametrize("agg", [0, 1])
def test_partitioned_update_and_overwrite(cuda_lib, oracle_mod, agg):
    c = 1 << 15
    keys = W.zipf_keys(30_001, 1.0, n_ranks=1 << 12, seed=62)
    vals = np.arange(1, keys.size + 1, dtype=np.uint64)
    pre = np.unique(keys)[::3]
    t, o = _pair(cuda_lib, oracle_mod, c, iou_aggregate=agg)
    t.insert(to_dev(pre), to_dev(pre))
    o.insert(pre, pre)
    codes = codes_buf(keys.size)
    t.update(to_dev(keys), to_dev(vals), cuda_lib.ADD, codes)
    assert np.array_equal(to_np_u8(codes), o.update(keys, vals, oracle_mod.ADD))
    assert_same_live_set(t, o)
    # overwrite: the stored value is one of the key's operations' values
    codes = codes_buf(keys.size)
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.OVERWRITE, codes)
    o.insert_or_update(keys, vals, oracle_mod.OVERWRITE)
    gk, gv = t.export()
    got = dict(zip(to_np_u64(gk).tolist(), to_np_u64(gv).tolist()))
    ok, _ = o.export()
    assert set(got) == set(ok.tolist())
    allowed = {}
    for k, v in zip(keys.tolist(), vals.tolist()):
        allowed.setdefault(k, set()).add(v)
    assert all(got[k] in allowed[k] for k in allowed)


@pytest.mark.parametrize("opts", [{"reuse_tombstones": 1}, {"full_key_space": 1},
                                  {"reuse_tombstones": 1, "full_key_space": 1}])
def test_partitioned_table_options(cuda_lib, oracle_mod, opts):
    c = 1 << 14
    keys = W.uniform_keys(6000, seed=63)
    keys[::501] = 0
    keys[1::777] = (1 << 64) - 1
    t, o = _pair(cuda_lib, oracle_mod, c, **opts)
    for rnd in range(4):  # erase / re-insert cycles leave and reuse tombstones
        sub = keys[rnd * 500: rnd * 500 + 4000]
        cs = codes_buf(sub.size)
        t.insert(to_dev(sub), to_dev(sub), cs)
        assert np.array_equal(to_np_u8(cs), o.insert(sub, sub))
        er = sub[::2]
        ce = codes_buf(er.size)
        t.erase(to_dev(er), ce)
        assert np.array_equal(to_np_u8(ce), o.erase(er))
        vo, fo = vals_buf(keys.size), codes_buf(keys.size)
        t.find(to_dev(keys), vo, fo)
        ev, ef = o.find(keys)
        assert np.array_equal(to_np_u8(fo), ef) and np.array_equal(to_np_u64(vo), ev)
    assert t.size()[:2] == (o.live, o.nonempty)
    assert_same_live_set(t, o)


def test_partitioned_growable_insert(cuda_lib, oracle_mod):
    keys = W.uniform_keys(300_000, seed=64)
    t, o = _pair(cuda_lib, oracle_mod, 1 << 10, growable=True)
    codes = codes_buf(keys.size)
    t.insert(to_dev(keys), to_dev(keys), codes)
    assert np.array_equal(to_np_u8(codes), o.insert(keys, keys))
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    assert_same_live_set(t, o)


def test_partitioned_2p22_table_load_09(cuda_lib, oracle_mod):
    """2^22 cells, 2^21 operations per find: the partitioned path takes more
    launches than the direct one; both agree with the oracle."""
    log2c = 22
    c = 1 << log2c
    wl = W.bounded_workload(log2c, loads=(0.9,), n_find=1 << 21)
    m = wl["counts"][0.9]
    keys, vals = wl["keys"][:m], wl["vals"][:m]
    t = cuda_lib.Table(c)
    t.set_config(partition=1)
    o = oracle_mod.OracleTable(c)
    l0 = cuda_lib.launch_count()
    codes = codes_buf(m)
    t.insert(to_dev(keys), to_dev(vals), codes)
    assert cuda_lib.launch_count() - l0 >= 5  # histogram, scan (3), scatter, operation, gather
    assert np.array_equal(to_np_u8(codes), o.insert(keys, vals))
    for part in (1, 0):
        t.set_config(partition=part)
        for q in (wl["hits"][0.9], wl["misses"]):
            l0 = cuda_lib.launch_count()
            vo, fo = vals_buf(q.size), codes_buf(q.size)
            t.find(to_dev(q), vo, fo)
            assert (cuda_lib.launch_count() - l0 == 1) == (part == 0)
            ev, ef = o.find(q)
            assert np.array_equal(to_np_u8(fo), ef)
            assert np.array_equal(to_np_u64(vo), ev)
    assert_same_live_set(t, o)


@pytest.mark.parametrize("s", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("n", [1, 4097, 300_001])
def test_hash_sorted_insert_or_update(cuda_lib, oracle_mod, s, n):
    """iou_aggregate = 3: the batch is sorted by the top 16 hash bits (two stable
    passes), aggregated in 4096-operation windows, codes gathered back."""
    c = 1 << 18
    keys = W.zipf_keys(n, s, n_ranks=1 << 16, seed=65)
    vals = (np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) | np.uint64(1)
    keys[::997] = 0
    pre = np.unique(keys[keys != 0])[::5]
    t = cuda_lib.Table(c)
    t.set_config(iou_aggregate=3)
    o = oracle_mod.OracleTable(c)
    t.insert(to_dev(pre), to_dev(pre))
    o.insert(pre, pre)
    codes = codes_buf(n)
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.ADD, codes)
    o.insert_or_update(keys, vals, oracle_mod.ADD)
    cs = to_np_u8(codes)
    assert (cs[keys == 0] == 3).all()
    pre_set = set(pre.tolist())
    live_ops = keys != 0
    assert_one_winner(keys[live_ops], cs[live_ops], lambda k: k not in pre_set)
    assert_same_live_set(t, o)
    # overwrite through the same path: every stored value is one of its key's
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.OVERWRITE)
    gk, gv = t.export()
    got = dict(zip(to_np_u64(gk).tolist(), to_np_u64(gv).tolist()))
    allowed = {}
    for k, v in zip(keys.tolist(), vals.tolist()):
        allowed.setdefault(k, set()).add(v)
    assert all(got[k] in allowed[k] for k in allowed if k != 0)
