"""GPU migration and growth parity (Sec. 4.3.1 Lemma 1; Sec. 4.3.2; Sec. 4.4).

The migration's cell layout is deterministic given the source snapshot: the
GPU's cluster-parallel result must equal, bit for bit, the oracle's
sequential migration of the same snapshot.  Cases cover several tiles and
one tile larger than the table, loads up to 0.99 (long clusters crossing tile
borders), both placement kernels (one lane per cluster below load 0.6, 32-cell
windows above) with each way of writing the target, tombstones (gamma = 1
purge), gamma from 2 to 256, clusters wrapping past the last cell, and a
completely full table (fallback path).
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_same_live_set, codes_buf, to_dev, to_np_u64, to_np_u8, vals_buf

pytestmark = pytest.mark.gpu


def _wrap_keys(oracle_mod, log2c, count, seed):
    cand = W.uniform_keys(1 << 18, start=5 * 10**7, seed=seed)
    h = oracle_mod.homes(cand, log2c)
    return cand[h >= (1 << log2c) - 3][:count]


def _fill(cuda_lib, oracle_mod, log2c, load, erase_frac, seed, wrap=0):
    c = 1 << log2c
    n = int(load * c)
    keys = W.uniform_keys(n, start=seed * 10**6, seed=61)
    if wrap:
        keys = np.concatenate([_wrap_keys(oracle_mod, log2c, wrap, seed), keys])[:n]
    t = cuda_lib.Table(c)
    t.insert(to_dev(keys), to_dev(W.values_for(keys)))
    if erase_frac:
        t.erase(to_dev(keys[: int(erase_frac * n)]))
    return t, keys


@pytest.mark.parametrize("log2c,load,erase,gamma_log2,tile", [
    (12, 0.5, 0.0, 1, 0),
    (16, 0.5, 0.0, 1, 2048),
    (16, 0.9, 0.0, 1, 64),
    (16, 0.95, 0.0, 1, 256),     # long clusters crossing many tiles
    (16, 0.8, 0.4, 0, 512),
    (15, 0.6, 0.2, 2, 128),
    (6, 0.5, 0.0, 1, 2048),      # table smaller than a tile
    (18, 0.7, 0.1, 1, 4096),
    (14, 0.5, 0.0, 4, 1024),     # gamma = 16
    (13, 0.5, 0.0, 8, 256),      # gamma = 256: owned ranges beyond the bitmap (global path)
    (18, 0.9, 0.3, 1, 512),      # many windows whose lanes pick the same target cell
    (16, 0.99, 0.0, 1, 512),     # clusters of thousands of cells: bitmap and global paths
    (16, 0.55, 0.2, 1, 256),     # below load 0.6 (one lane per cluster) with tombstones
    (14, 0.7, 0.0, 4, 1024),     # windows into a 16x larger table (shared bitmap path)
    (13, 0.7, 0.0, 8, 256),      # windows into a 256x larger table (global path)
])
def test_migration_layout_equals_sequential(cuda_lib, oracle_mod, log2c, load, erase, gamma_log2, tile):
    t, _ = _fill(cuda_lib, oracle_mod, log2c, load, erase, seed=log2c + gamma_log2, wrap=5)
    t.set_config(migrate_tile=tile)
    snap = to_np_u64(t.cells())
    live_before = t.size()[0]
    o = oracle_mod.OracleTable(64)
    o.load_cells(snap)
    o.migrate((1 << log2c) << gamma_log2)
    t.migrate((1 << log2c) << gamma_log2)
    got = to_np_u64(t.cells()).reshape(-1, 2)
    assert got.shape == o.cells().shape
    assert np.array_equal(got, o.cells())
    live, ne, cap = t.size(check=True)
    assert live == ne == live_before == o.live
    assert cap == (1 << log2c) << gamma_log2


def test_migration_wraparound_cluster(cuda_lib, oracle_mod):
    log2c = 12
    c = 1 << log2c
    wrap = _wrap_keys(oracle_mod, log2c, 40, 7)
    t = cuda_lib.Table(c)
    t.insert(to_dev(wrap), to_dev(wrap))
    snap = to_np_u64(t.cells()).reshape(-1, 2)
    assert snap[0, 0] != 0 and snap[c - 1, 0] != 0  # the cluster crosses index 0
    o = oracle_mod.OracleTable(64)
    o.load_cells(snap)
    o.migrate(2 * c)
    t.migrate(2 * c)
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())


def test_migration_of_full_table_uses_fallback(cuda_lib, oracle_mod):
    c = 256
    keys = W.uniform_keys(c, seed=62)
    t = cuda_lib.Table(c)
    codes = codes_buf(c)
    t.insert(to_dev(keys), to_dev(keys), codes)
    assert (to_np_u8(codes) == 1).all()
    snap = to_np_u64(t.cells()).reshape(-1, 2)
    assert (snap[:, 0] != 0).all()
    o = oracle_mod.OracleTable(64)
    o.load_cells(snap)
    o.migrate(2 * c)
    t.migrate(2 * c)
    assert np.array_equal(to_np_u64(t.cells()).reshape(-1, 2), o.cells())
    assert t.size()[:2] == (c, c)


def test_migrate_policy_and_bad_capacity(cuda_lib):
    t = cuda_lib.Table(1024)
    keys = W.uniform_keys(400, seed=63)
    t.insert(to_dev(keys), to_dev(keys))
    t.migrate(0)  # 400 live > alpha*c/2 = 256: doubles
    assert t.size() == (400, 400, 2048)
    t.erase(to_dev(keys[:300]))
    t.migrate(0)  # 100 live: same size, tombstones purged
    assert t.size() == (100, 100, 2048)
    with pytest.raises(cuda_lib.ChtError):
        t.migrate(64)  # shrinking below the live count: no empty cell would remain
    assert t.size() == (100, 100, 2048)
    t.migrate(512)  # shrinking (Sec. 4.3.1 "Shrinking")
    assert t.size() == (100, 100, 512)


@pytest.mark.parametrize("log2c,load,erase,shrink_log2", [
    (16, 0.5, 0.6, 1),    # load 0.4 after shrinking by 2
    (16, 0.5, 0.8, 2),
    (18, 0.6, 0.975, 5),  # by 32: most elements spill from short blocks
    (14, 0.9, 0.5, 1),    # long clusters: many spills
    (12, 0.5, 0.97, 5),   # the target (128 cells) is smaller than one block
    (20, 0.3, 0.99, 8),   # by 256
])
def test_shrinking_migration(cuda_lib, oracle_mod, log2c, load, erase, shrink_log2):
    """Shrinking (Sec. 4.3.1): the live set is kept, every key stays reachable
    from its home (the layout's invariants, checked by the oracle on the GPU's
    cells), and the occupied cells equal those of the sequential migration of
    the same snapshot (linear probing's occupancy does not depend on order)."""
    t, _ = _fill(cuda_lib, oracle_mod, log2c, load, erase, seed=log2c + shrink_log2 + 100, wrap=5)
    snap = to_np_u64(t.cells())
    live = t.size()[0]
    o = oracle_mod.OracleTable(64)
    o.load_cells(snap)
    new_c = (1 << log2c) >> shrink_log2
    assert live < new_c
    o.migrate(new_c)
    t.migrate(new_c)
    assert t.size(check=True) == (live, live, new_c)
    got = to_np_u64(t.cells()).reshape(-1, 2)
    assert np.array_equal(got[:, 0] != 0, o.cells()[:, 0] != 0)
    g = oracle_mod.OracleTable(64)
    g.load_cells(got)
    g.assert_invariants()
    assert_same_live_set(t, o)
    # the shrunk table works: finds hit every live key
    gk, gv = t.export()
    vo, fo = vals_buf(live), codes_buf(live)
    t.find(gk, vo, fo)
    assert (to_np_u8(fo) == 1).all() and np.array_equal(to_np_u64(vo), to_np_u64(gv))


def test_migration_oom_leaves_table_unchanged(cuda_lib):
    t = cuda_lib.Table(1 << 16)
    keys = W.uniform_keys(20000, seed=64)
    t.insert(to_dev(keys), to_dev(keys))
    before = to_np_u64(t.cells())
    used = cuda_lib.memory_in_use()
    cuda_lib.set_memory_limit(used + 1024)
    try:
        with pytest.raises(cuda_lib.ChtError) as e:
            t.migrate(1 << 17)
        assert e.value.status == cuda_lib.CHT_ERR_OOM
    finally:
        cuda_lib.set_memory_limit(0)
    assert np.array_equal(to_np_u64(t.cells()), before)
    assert t.size()[2] == 1 << 16
    t.migrate(1 << 17)
    assert t.size()[:2] == (20000, 20000)


@pytest.mark.parametrize("g", [1, 8])
def test_growing_insert_doubles_at_alpha(cuda_lib, oracle_mod, g):
    """Growing table from 2^12 cells, one insert batch of 2^18 keys (scaled config 3a)."""
    n = 1 << 18
    keys = W.uniform_keys(n)
    vals = W.values_for(keys)
    t = cuda_lib.Table(1 << 12, growable=True)
    t.set_config(group_width=g)
    codes = codes_buf(n)
    t.insert(to_dev(keys), to_dev(vals), codes)
    assert (to_np_u8(codes) == 1).all()
    live, ne, cap = t.size(check=True)
    assert (live, ne, cap) == (n, n, 1 << 19)
    o = oracle_mod.OracleTable(1 << 12, growable=True)
    o.insert(keys, vals)
    assert o.capacity == cap
    assert_same_live_set(t, o)
    vo, fo = vals_buf(n), codes_buf(n)
    t.find(to_dev(keys), vo, fo)
    assert (to_np_u8(fo) == 1).all() and np.array_equal(to_np_u64(vo), vals)


def test_growing_aggregation(cuda_lib, oracle_mod):
    keys = W.zipf_keys(300_000, 1.0, n_ranks=1 << 16, seed=65)
    ones = np.ones(keys.size, np.uint64)
    t = cuda_lib.Table(1 << 12, growable=True)
    t.insert_or_update(to_dev(keys), to_dev(ones), cuda_lib.ADD)
    o = oracle_mod.OracleTable(1 << 12, growable=True)
    o.insert_or_update(keys, ones, oracle_mod.ADD)
    assert_same_live_set(t, o)
    assert t.size()[0] == np.unique(keys).size


def test_sliding_window_purges_tombstones(cuda_lib, oracle_mod):
    """Scaled config 3b: a window of live keys slides; migrations purge tombstones."""
    window, batch, rounds = 1 << 14, 1 << 11, 48
    keys = W.uniform_keys(window + batch * rounds, seed=66)
    t = cuda_lib.Table(1 << 12, growable=True)
    o = oracle_mod.OracleTable(1 << 12, growable=True)
    t.insert(to_dev(keys[:window]), to_dev(keys[:window]))
    o.insert(keys[:window], keys[:window])
    caps = set()
    for r in range(rounds):
        ins = keys[window + r * batch: window + (r + 1) * batch]
        dele = keys[r * batch: (r + 1) * batch]
        ci, ce = codes_buf(batch), codes_buf(batch)
        t.insert(to_dev(ins), to_dev(ins), ci)
        t.erase(to_dev(dele), ce)
        o.insert(ins, ins)
        o.erase(dele)
        assert (to_np_u8(ci) == 1).all() and (to_np_u8(ce) == 1).all()
        caps.add(t.size()[2])
    live, ne, cap = t.size(check=True)
    assert live == window == o.live
    assert cap <= 1 << 16  # the table does not keep doubling: tombstones are purged
    assert_same_live_set(t, o)

