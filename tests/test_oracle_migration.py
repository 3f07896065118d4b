"""Pins of the oracle's sequential migration (Sec. 4.3.1, Lemma 1; Sec. 4.4).

Independent facts used:
* gamma = 1 without tombstones is the identity on the layout: re-inserting a
  cluster's elements in index order puts each one back in its own cell.
* Linear probing's occupied-cell set depends only on the multiset of homes,
  not on the insertion order, so the migrated table's occupied cells equal
  those of the same keys inserted in a random order into an empty table.
* Lemma 1 (with the integer-gamma bound derived in its proof): the elements of
  a source cluster a..b land inside gamma*a .. gamma*(b+1)-1 (cyclically).
* A brute-force Python restatement of "visit cells in index order from a
  cluster start and re-insert each live one" on tiny tables.
"""
import numpy as np
import pytest

import workloads as W

TOMB = np.uint64((1 << 64) - 1)


def _filled(oracle_mod, log2c, load, seed, erase_frac=0.0):
    c = 1 << log2c
    n = int(load * c)
    ks = W.uniform_keys(n, start=seed * 100_000, seed=21)
    t = oracle_mod.OracleTable(c)
    t.insert(ks, W.values_for(ks))
    if erase_frac:
        t.erase(ks[: int(erase_frac * n)])
    return t, ks


def _clusters(cells):
    """(start, end) index pairs of every cluster (a..b with a-1, b+1 empty)."""
    c = cells.shape[0]
    ne = cells[:, 0] != 0
    if ne.all() or not ne.any():
        return []
    out = []
    for a in range(c):
        if ne[a] and not ne[(a - 1) % c]:
            b = a
            while ne[(b + 1) % c]:
                b += 1
            out.append((a, b))
    return out


def _bruteforce_migrate(oracle_mod, cells, new_log2c):
    c = cells.shape[0]
    nc = 1 << new_log2c
    dst = np.zeros((nc, 2), dtype=np.uint64)
    ne = cells[:, 0] != 0
    starts = [a for a in range(c) if ne[a] and not ne[(a - 1) % c]]
    s0 = starts[0] if starts else 0
    for j in range(c):
        k, v = cells[(s0 + j) % c]
        if k == 0 or k == TOMB:
            continue
        p = int(oracle_mod.homes(np.array([k], dtype=np.uint64), new_log2c)[0])
        while dst[p, 0] != 0:
            p = (p + 1) % nc
        dst[p] = (k, v)
    return dst


@pytest.mark.parametrize("load", [0.3, 0.5, 0.9])
def test_gamma1_without_tombstones_is_identity(oracle_mod, load):
    t, _ = _filled(oracle_mod, 10, load, 1)
    before = t.cells()
    t.migrate(t.capacity)
    assert np.array_equal(t.cells(), before)
    t.assert_invariants()


@pytest.mark.parametrize("log2c,gamma_log2,load,erase", [(6, 1, 0.5, 0.0), (7, 1, 0.9, 0.3),
                                                         (8, 0, 0.8, 0.5), (8, 2, 0.6, 0.1),
                                                         (9, 1, 0.95, 0.0)])
def test_matches_bruteforce_sequential_migration(oracle_mod, log2c, gamma_log2, load, erase):
    t, _ = _filled(oracle_mod, log2c, load, 2, erase)
    src = t.cells()
    want = _bruteforce_migrate(oracle_mod, src, log2c + gamma_log2)
    t.migrate(t.capacity << gamma_log2)
    assert np.array_equal(t.cells(), want)


@pytest.mark.parametrize("gamma_log2", [0, 1, 2])
@pytest.mark.parametrize("load", [0.5, 0.85])
def test_lemma1_cluster_targets(oracle_mod, gamma_log2, load):
    log2c = 11
    t, _ = _filled(oracle_mod, log2c, load, 3, erase_frac=0.2)
    src = t.cells()
    c, g = src.shape[0], 1 << gamma_log2
    t.migrate(c * g)
    dst = t.cells()
    pos = {int(k): i for i, k in enumerate(dst[:, 0]) if k != 0}
    nc = c * g
    for a, b in _clusters(src):
        lo, hi = g * a, g * (b + 1) - 1  # target window of this cluster
        for i in range(a, b + 1):
            k = int(src[i % c, 0])
            if k in (0, int(TOMB)):
                continue
            off = (pos[k] - lo) % nc
            assert off <= (hi - lo) % nc, (a, b, k)


@pytest.mark.parametrize("gamma_log2", [0, 1, 3])
def test_occupancy_is_order_independent(oracle_mod, gamma_log2):
    log2c = 10
    t, _ = _filled(oracle_mod, log2c, 0.7, 4, erase_frac=0.25)
    live_k, live_v = t.export()
    t.migrate(t.capacity << gamma_log2)
    rng = np.random.default_rng(5)
    order = rng.permutation(live_k.size)
    ref = oracle_mod.OracleTable(t.capacity)
    ref.insert(live_k[order], live_v[order])
    assert np.array_equal(t.cells()[:, 0] != 0, ref.cells()[:, 0] != 0)
    assert t.nonempty == live_k.size and t.live == live_k.size
    t.assert_invariants()


def test_migration_drops_tombstones_keeps_live_set(oracle_mod):
    t, ks = _filled(oracle_mod, 12, 0.6, 5, erase_frac=0.4)
    k0, v0 = t.export()
    t.migrate(t.capacity)
    assert not (t.cells()[:, 0] == TOMB).any()
    k1, v1 = t.export()
    assert sorted(zip(k0.tolist(), v0.tolist())) == sorted(zip(k1.tolist(), v1.tolist()))
    t.assert_invariants()


def test_full_table_migration_starts_at_zero(oracle_mod):
    c = 64
    t = oracle_mod.OracleTable(c)
    ks = W.uniform_keys(c, seed=31)
    t.insert(ks, ks)
    src = t.cells()
    assert (src[:, 0] != 0).all()
    want = _bruteforce_migrate(oracle_mod, src, 7)
    t.migrate(2 * c)
    assert np.array_equal(t.cells(), want)
    t.assert_invariants()


@pytest.mark.parametrize("shrink_log2", [1, 2, 5])
def test_shrinking_migration_matches_bruteforce(oracle_mod, shrink_log2):
    """Shrinking (Sec. 4.3.1): the sequential migration into c / 2^k cells equals
    brute-force re-insertion of the live elements in cluster order, keeps the
    live set and the invariants, and its occupancy equals any insertion order's."""
    log2c = 12
    # leave about 0.45 c' live elements: load 0.45 in the smaller table
    t, _ = _filled(oracle_mod, log2c, 0.5, 6 + shrink_log2, erase_frac=1.0 - 0.9 / (1 << shrink_log2))
    live_k, live_v = t.export()
    assert live_k.size < (1 << (log2c - shrink_log2))
    expect = _bruteforce_migrate(oracle_mod, t.cells(), log2c - shrink_log2)
    t.migrate(t.capacity >> shrink_log2)
    assert t.capacity == 1 << (log2c - shrink_log2)
    assert np.array_equal(t.cells(), expect)
    k1, v1 = t.export()
    assert sorted(zip(live_k.tolist(), live_v.tolist())) == sorted(zip(k1.tolist(), v1.tolist()))
    order = np.random.default_rng(7).permutation(live_k.size)
    ref = oracle_mod.OracleTable(t.capacity)
    ref.insert(live_k[order], live_v[order])
    assert np.array_equal(t.cells()[:, 0] != 0, ref.cells()[:, 0] != 0)
    t.assert_invariants()
