"""Pins of the CPU oracle against plain definitions (no GPU).

Every check here compares the oracle with something other than itself:
a Python dictionary processed op by op (the sequential-dictionary meaning of
Sec. 3's interface), sorted-list reductions, and the table invariants of
linear probing (Sec. 2).  Inputs are tiny and include duplicates, reserved
keys and clusters that wrap around the end of the table.
"""
import numpy as np
import pytest

import workloads as W

MASK = (1 << 64) - 1


class DictModel:
    """A sequential dictionary with the paper's return conventions (Sec. 3)."""

    def __init__(self, full_keys=False):
        self.d = {}
        self.full_keys = full_keys  # keys 0 and ~0 are ordinary keys

    def reserved(self, k):
        return not self.full_keys and (k == 0 or k == MASK)

    def insert(self, k, v):
        if self.reserved(k):
            return 3
        if k in self.d:
            return 0
        self.d[k] = v
        return 1

    def iou(self, k, v, op):
        if self.reserved(k):
            return 3
        if k in self.d:
            self.d[k] = (self.d[k] + v) & MASK if op == 1 else v
            return 0
        self.d[k] = v
        return 1

    def update(self, k, v, op):
        if self.reserved(k):
            return 3
        if k in self.d:
            self.d[k] = (self.d[k] + v) & MASK if op == 1 else v
            return 1
        return 0

    def find(self, k):
        if self.reserved(k):
            return 0, 3
        if k in self.d:
            return self.d[k], 1
        return 0, 0

    def erase(self, k):
        if self.reserved(k):
            return 3
        if k in self.d:
            del self.d[k]
            return 1
        return 0


def _wrap_keys(oracle_mod, log2c, count, rng_seed):
    """Keys whose home is one of the last two cells, forcing wrap-around clusters."""
    cand = W.uniform_keys(1 << 16, start=10_000_000 + rng_seed * (1 << 16), seed=77)
    h = oracle_mod.homes(cand, log2c)
    c = 1 << log2c
    return cand[h >= c - 2][:count]


def _random_batch(rng, pool, n):
    idx = rng.integers(0, len(pool), size=n)
    ks = pool[idx].copy()
    # sprinkle reserved keys
    if n > 4:
        ks[rng.integers(0, n)] = np.uint64(0)
        ks[rng.integers(0, n)] = np.uint64(MASK)
    vs = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    return ks, vs


@pytest.mark.parametrize("log2c", [6, 7, 8, 10])
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("reuse,full_keys", [(False, False), (True, False), (False, True), (True, True)])
def test_oracle_matches_dictionary(oracle_mod, log2c, seed, reuse, full_keys):
    c = 1 << log2c
    rng = np.random.default_rng(1000 * log2c + seed)
    pool = np.concatenate([W.uniform_keys(c // 2, start=seed * 4096, seed=5),
                           _wrap_keys(oracle_mod, log2c, 6, seed)])
    t = oracle_mod.OracleTable(c, reuse_tombstones=reuse, full_key_space=full_keys)
    m = DictModel(full_keys)
    for step in range(40):
        kind = rng.choice(["insert", "iou_add", "iou_ow", "find", "erase", "upd_add", "upd_ow"])
        # keep the number of inserted cells (tombstones count) below c
        if kind in ("insert", "iou_add", "iou_ow") and t.nonempty > c - len(pool):
            kind = "find"
        ks, vs = _random_batch(rng, pool, int(rng.integers(1, 24)))
        if kind == "insert":
            f = t.insert(ks, vs)
            exp = [m.insert(int(k), int(v)) for k, v in zip(ks, vs)]
            assert f.tolist() == exp
        elif kind in ("iou_add", "iou_ow"):
            op = 1 if kind == "iou_add" else 0
            f = t.insert_or_update(ks, vs, op)
            exp = [m.iou(int(k), int(v), op) for k, v in zip(ks, vs)]
            assert f.tolist() == exp
        elif kind in ("upd_add", "upd_ow"):
            op = 1 if kind == "upd_add" else 0
            f = t.update(ks, vs, op)
            exp = [m.update(int(k), int(v), op) for k, v in zip(ks, vs)]
            assert f.tolist() == exp
        elif kind == "find":
            v, f = t.find(ks)
            exp = [m.find(int(k)) for k in ks]
            assert f.tolist() == [e[1] for e in exp]
            assert [int(x) for x in v] == [e[0] for e in exp]
        else:
            f = t.erase(ks)
            exp = [m.erase(int(k)) for k in ks]
            assert f.tolist() == exp
        t.assert_invariants()
        ek, ev = t.export()
        assert dict(zip((int(x) for x in ek), (int(x) for x in ev))) == m.d
        assert t.live == len(m.d)


def test_update_add_equals_sorted_reduction_over_present_keys(oracle_mod):
    """update(add) of a batch with repeats: every present key gains the sum of
    its batch values (sort + run-length sums), absent keys stay absent."""
    c = 1 << 10
    t = oracle_mod.OracleTable(c)
    present = W.uniform_keys(200, seed=21)
    t.insert(present, np.zeros(200, np.uint64))
    rng = np.random.default_rng(22)
    pool = np.concatenate([present, W.uniform_keys(100, start=5000, seed=21)])
    ks = pool[rng.integers(0, pool.size, 3000)]
    vs = rng.integers(0, 1 << 40, ks.size).astype(np.uint64)
    f = t.update(ks, vs, oracle_mod.ADD)
    pset = set(present.tolist())
    assert [int(x) for x in f] == [1 if int(k) in pset else 0 for k in ks]
    order = np.argsort(ks, kind="stable")
    sk, sv = ks[order], vs[order]
    starts = np.flatnonzero(np.r_[True, sk[1:] != sk[:-1]])
    sums = np.add.reduceat(sv, starts)
    got_v, got_f = t.find(sk[starts])
    for k, sm, gv, gf in zip(sk[starts], sums, got_v, got_f):
        if int(k) in pset:
            assert gf == 1 and int(gv) == int(sm)
        else:
            assert gf == 0
    assert t.live == 200 and t.nonempty == 200
    t.assert_invariants()


def test_wraparound_cluster_is_used(oracle_mod):
    """Keys homed at the last cells must spill over index 0 (cyclic probing)."""
    log2c = 8
    ks = _wrap_keys(oracle_mod, log2c, 8, 3)
    assert len(ks) >= 4
    t = oracle_mod.OracleTable(1 << log2c)
    t.insert(ks, ks)
    cells = t.cells()
    occupied = np.nonzero(cells[:, 0])[0]
    assert 0 in occupied  # the cluster wrapped
    v, f = t.find(ks)
    assert (f == 1).all() and (v == ks).all()
    t.assert_invariants()


def test_aggregation_equals_sorted_reduction(oracle_mod):
    """insertOrUpdate(add) sums equal a sort + run-length reduction of the ops."""
    keys = W.zipf_keys(20000, 1.25, n_ranks=4096, seed=9)
    vals = (np.arange(keys.size, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
    t = oracle_mod.OracleTable(1 << 14)
    # pre-existing values for part of the keys
    pre_k = np.unique(keys)[::3]
    pre_v = pre_k ^ np.uint64(0x1234)
    t.insert(pre_k, pre_v)
    f = t.insert_or_update(keys, vals, oracle_mod.ADD)
    order = np.argsort(keys, kind="stable")
    sk, sv = keys[order], vals[order]
    uk, start = np.unique(sk, return_index=True)
    with np.errstate(over="ignore"):
        sums = np.add.reduceat(sv, start)
        pre = dict(zip(pre_k.tolist(), pre_v.tolist()))
        expect = {int(k): (int(s) + pre.get(int(k), 0)) & MASK for k, s in zip(uk, sums)}
    got_v, got_f = t.find(uk)
    assert (got_f == 1).all()
    assert {int(k): int(v) for k, v in zip(uk, got_v)} == expect
    # exactly one insertion per key that was absent before the batch
    inserted = keys[f == 1]
    assert sorted(inserted.tolist()) == sorted(set(uk.tolist()) - set(pre_k.tolist()))


def test_full_bounded_table(oracle_mod):
    """A bounded table filled to 100 % reports 'full' and its probes stop after c cells."""
    c = 64
    t = oracle_mod.OracleTable(c)
    ks = W.uniform_keys(c + 10, seed=11)
    f = t.insert(ks, ks)
    assert (f[:c] == 1).all() and (f[c:] == 2).all()
    v, ff = t.find(W.uniform_keys(5, start=1000, seed=11))
    assert (ff == 0).all() and (v == 0).all()
    v, ff = t.find(ks[:c])
    assert (ff == 1).all()
    t.assert_invariants()


def test_tombstones_are_not_reused(oracle_mod):
    c = 64
    t = oracle_mod.OracleTable(c)
    ks = W.uniform_keys(20, seed=12)
    t.insert(ks, ks)
    assert (t.erase(ks[:10]) == 1).all()
    assert (t.erase(ks[:10]) == 0).all()  # already erased
    assert t.nonempty == 20 and t.live == 10
    # re-inserting an erased key occupies a fresh cell: I grows
    assert (t.insert(ks[:10], ks[:10]) == 1).all()
    assert t.nonempty == 30 and t.live == 20
    t.assert_invariants()


def test_reused_tombstones_keep_counts_and_reachability(oracle_mod):
    """With reuse, re-inserting erased keys takes their tombstones back: the
    non-empty count stays, the tombstone count drops to zero, and every key is
    still found from its home."""
    c = 64
    t = oracle_mod.OracleTable(c, reuse_tombstones=True)
    ks = W.uniform_keys(20, seed=12)
    t.insert(ks, ks)
    assert (t.erase(ks[:10]) == 1).all()
    assert t.nonempty == 20 and t.live == 10
    assert (t.insert(ks[:10], ks[:10] + np.uint64(1)) == 1).all()
    assert t.nonempty == 20 and t.live == 20
    v, f = t.find(ks)
    assert (f == 1).all() and (v[:10] == ks[:10] + np.uint64(1)).all() and (v[10:] == ks[10:]).all()
    t.assert_invariants()


def test_reused_tombstone_fills_a_table_without_empty_cells(oracle_mod):
    """A table with no empty cell but a tombstone still takes a new key."""
    c = 64
    t = oracle_mod.OracleTable(c, reuse_tombstones=True)
    ks = W.uniform_keys(c + 1, seed=13)
    assert (t.insert(ks[:c], ks[:c]) == 1).all()
    assert t.erase(ks[:1])[0] == 1
    assert t.insert(ks[c:], ks[c:])[0] == 1
    assert t.insert(ks[:1], ks[:1])[0] == 2  # now full again
    t.assert_invariants()


@pytest.mark.parametrize("reuse", [False, True])
def test_erase_reinsert_cycles_and_probe_length(oracle_mod, reuse):
    """Erasing and re-inserting the same keys again and again: without reuse
    every cycle leaves a tombstone on the keys' probe paths, so an insert of
    cycle r walks past ~r of them (linear probing, Sec. 2); with reuse each
    key goes back into its own tombstone and the walk stays one cell."""
    c = 1 << 12
    t = oracle_mod.OracleTable(c, reuse_tombstones=reuse)
    ks = W.uniform_keys(4, seed=14)
    t.insert(ks, ks)
    for _ in range(200):
        assert (t.erase(ks) == 1).all()
        t.reset_probes()
        assert (t.insert(ks, ks) == 1).all()
    per_insert = t.probes / ks.size
    if reuse:
        assert per_insert <= 2.0 and t.nonempty == 4
    else:
        assert per_insert >= 150 and t.nonempty == 4 + 4 * 200
    t.assert_invariants()


def test_growable_oracle_doubles_at_alpha(oracle_mod):
    t = oracle_mod.OracleTable(64, growable=True, alpha=0.5)
    ks = W.uniform_keys(1 << 14, seed=1)
    f = t.insert(ks, W.values_for(ks))
    assert (f == 1).all()
    assert t.capacity == 1 << 15  # 2^14 keys at load exactly 0.5
    assert t.migrations == 15 - 6
    v, ff = t.find(ks)
    assert (ff == 1).all() and (v == W.values_for(ks)).all()
    t.assert_invariants()


def test_growable_purges_when_mostly_tombstones(oracle_mod):
    """Sliding window: live stays small, so migrations keep the size (gamma = 1)."""
    t = oracle_mod.OracleTable(256, growable=True, alpha=0.5)
    ks = W.uniform_keys(3000, seed=13)
    window = 40
    t.insert(ks[:window], ks[:window])
    for j in range(window, len(ks)):
        t.insert(ks[j:j + 1], ks[j:j + 1])
        assert t.erase(ks[j - window:j - window + 1])[0] == 1
    assert t.capacity == 256
    assert t.migrations > 0
    assert t.live == window
    t.assert_invariants()


def test_full_key_space_special_slots(oracle_mod):
    """Keys 0 and ~0 in the special slots: dictionary results, kept across
    growth and shrinking migrations, counted as live but never as a cell."""
    t = oracle_mod.OracleTable(64, growable=True, full_key_space=True)
    ks = W.uniform_keys(100, seed=23)
    special = np.array([0, MASK], dtype=np.uint64)
    assert (t.insert(special, np.array([7, 9], dtype=np.uint64)) == 1).all()
    assert (t.insert(special, np.array([1, 1], dtype=np.uint64)) == 0).all()
    t.insert(ks, ks)
    assert t.capacity == 256 and t.nonempty == 100 and t.live == 102
    assert (t.insert_or_update(special, np.array([5, 5], dtype=np.uint64), oracle_mod.ADD) == 0).all()
    v, f = t.find(special)
    assert f.tolist() == [1, 1] and v.tolist() == [12, 14]
    assert t.erase(special[1:]).tolist() == [1] and t.erase(special[1:]).tolist() == [0]
    v, f = t.find(special)
    assert f.tolist() == [1, 0] and v.tolist() == [12, 0]
    assert t.update(special, np.array([3, 3], dtype=np.uint64), oracle_mod.OVERWRITE).tolist() == [1, 0]
    t.migrate(4096)
    t.migrate(256)
    ek, ev = t.export()
    d = dict(zip(ek.tolist(), ev.tolist()))
    assert d[0] == 3 and MASK not in d and len(d) == 101
    assert t.nonempty == 100 and t.live == 101
    t.assert_invariants()
