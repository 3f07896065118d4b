"""Pins of the oracle's sort-based bulk build (Sec. 3 "Bulk Operations").

Independent facts used:
* Dictionary meaning: after building from pairs with repeated keys, every key
  maps to the value of its LAST occurrence (the paper keeps the last of equal
  keys), and the live count is the number of distinct keys -- checked against a
  Python dict.
* A layout is a valid linear-probing table iff no empty cell lies between any
  element's home and its cell (cyclically).
* Characterisation of an insertion in sorted order: reading the table from
  just after an empty cell, the elements appear in sort order (hash bits, then
  input position), and every element sits at its home or right after another
  element.  Together with validity these facts fix every position (the first
  element of a run sits at its home, each next one at max(home, previous + 1)).
* A worked example on 64 cells with keys chosen for their homes, where the
  last home's elements wrap around to the front cells.
"""
import numpy as np
import pytest

import workloads as W

TOMB = (1 << 64) - 1


def _run_keys(cells):
    """Keys in cell order, starting just after the first empty cell."""
    c = cells.shape[0]
    empties = np.nonzero(cells[:, 0] == 0)[0]
    start = (int(empties[0]) + 1) % c
    order = [(start + j) % c for j in range(c)]
    return [(p, int(cells[p, 0])) for p in order if cells[p, 0] != 0]


def _check_valid(cells, log2c, oracle_mod):
    c = cells.shape[0]
    keys = cells[:, 0]
    live = np.nonzero(keys != 0)[0]
    homes = oracle_mod.homes(keys[live], log2c).astype(np.int64)
    for p, h in zip(live, homes):
        q = int(h)
        while q != p:
            assert keys[q] != 0, f"empty cell {q} between home {h} and cell {p}"
            q = (q + 1) % c


def _dup_batch(n, distinct, seed):
    rng = np.random.default_rng(seed)
    base = W.uniform_keys(distinct, start=seed * 1000, seed=31)
    keys = base[rng.integers(0, distinct, n)]
    vals = rng.integers(1, 1 << 62, n).astype(np.uint64)
    return keys, vals


@pytest.mark.parametrize("log2c,n,distinct", [(8, 100, 60), (10, 600, 400), (12, 3500, 1500)])
def test_build_is_the_dictionary_of_last_values(oracle_mod, log2c, n, distinct):
    keys, vals = _dup_batch(n, distinct, seed=log2c)
    t = oracle_mod.OracleTable(1 << log2c)
    assert t.build(keys, vals) == 0
    last = {}
    for k, v in zip(keys.tolist(), vals.tolist()):
        last[k] = v
    assert t.live == t.nonempty == len(last)
    q = np.array(list(last.keys()), dtype=np.uint64)
    got, found = t.find(q)
    assert found.all()
    assert got.tolist() == [last[k] for k in q.tolist()]


@pytest.mark.parametrize("log2c,load", [(8, 0.5), (10, 0.9), (12, 0.97)])
def test_build_layout_is_sorted_insertion(oracle_mod, log2c, load):
    c = 1 << log2c
    keys, vals = _dup_batch(int(load * c * 1.3), int(load * c), seed=log2c + 7)
    t = oracle_mod.OracleTable(c)
    assert t.build(keys, vals) == 0
    cells = t.cells()
    _check_valid(cells, log2c, oracle_mod)
    # sort order: top B hash bits, then the input position of the kept copy
    B = oracle_mod.build_sort_bits(log2c)
    assert B >= log2c
    last_pos = {}
    for i, k in enumerate(keys.tolist()):
        last_pos[k] = i
    run = _run_keys(cells)
    ks = np.array([k for _, k in run], dtype=np.uint64)
    sk = (oracle_mod.hash64(ks) >> np.uint64(64 - B)).tolist()
    order = [(s, last_pos[k]) for s, k in zip(sk, ks.tolist())]
    # cyclic: ascending with at most one descent (where the last homes wrapped)
    descents = sum(1 for a, b in zip(order, order[1:]) if b < a)
    if descents == 1:
        cut = next(i for i, (a, b) in enumerate(zip(order, order[1:])) if b < a) + 1
        order = order[cut:] + order[:cut]
    assert order == sorted(order)
    # compact: each element at its home or right after an occupied cell
    homes = oracle_mod.homes(ks, log2c).tolist()
    for (p, _), h in zip(run, homes):
        assert p == h or cells[(p - 1) % c, 0] != 0


def test_build_worked_example_wraps(oracle_mod):
    # 64 cells; keys picked for their homes: a at home 0, b at home 1 and three
    # keys x, y, z at home 63.  Sorted insertion puts a at 0, b at 1, the first
    # of x, y, z (by hash) at 63 and the other two, wrapping, at 2 and 3.
    cand = W.uniform_keys(20000, start=0, seed=5)
    h = oracle_mod.homes(cand, 6)
    a = cand[h == 0][0]
    b = cand[h == 1][0]
    xyz = cand[h == 63][:3]
    keys = np.array([xyz[0], a, xyz[1], b, xyz[2]], dtype=np.uint64)
    vals = np.arange(1, 6, dtype=np.uint64)
    t = oracle_mod.OracleTable(64)
    assert t.build(keys, vals) == 0
    cells = t.cells()
    B = oracle_mod.build_sort_bits(6)
    s = (oracle_mod.hash64(xyz) >> np.uint64(64 - B)).tolist()
    first, second, third = [xyz[i] for i in sorted(range(3), key=lambda i: (s[i], i))]
    assert cells[0, 0] == a and cells[1, 0] == b
    assert cells[63, 0] == first and cells[2, 0] == second and cells[3, 0] == third
    assert (cells[4:63, 0] == 0).all()
    assert cells[0, 1] == 2 and cells[1, 1] == 4


def test_build_equals_inserting_survivors_in_order(oracle_mod):
    log2c = 11
    keys, vals = _dup_batch(1800, 1500, seed=3)
    t = oracle_mod.OracleTable(1 << log2c)
    assert t.build(keys, vals) == 0
    B = oracle_mod.build_sort_bits(log2c)
    last = {}
    for i, (k, v) in enumerate(zip(keys.tolist(), vals.tolist())):
        last[k] = (i, v)
    ks = np.array(list(last.keys()), dtype=np.uint64)
    s = (oracle_mod.hash64(ks) >> np.uint64(64 - B)).tolist()
    order = sorted(range(len(ks)), key=lambda j: (s[j], last[int(ks[j])][0]))
    u = oracle_mod.OracleTable(1 << log2c)
    sk = ks[order]
    u.insert(sk, np.array([last[int(k)][1] for k in sk], dtype=np.uint64))
    assert np.array_equal(t.cells(), u.cells())


def test_build_full_and_not_empty(oracle_mod):
    ks = W.uniform_keys(64, start=0, seed=9)
    t = oracle_mod.OracleTable(64)
    assert t.build(ks, ks) == -2          # 64 distinct keys leave no empty cell
    assert t.live == 0 and (t.cells() == 0).all()
    assert t.build(ks[:63], ks[:63]) == 0  # 63 do
    assert t.live == 63
    assert t.build(ks[:1], ks[:1]) == -1  # not empty any more
    g = oracle_mod.OracleTable(64, growable=True, alpha=0.5)
    k2 = W.uniform_keys(100, start=500, seed=9)
    assert g.build(k2, k2) == 0
    assert g.capacity == 256 and g.live == 100  # 100 > 0.5 * 128, <= 0.5 * 256


def test_build_reserved_keys(oracle_mod):
    ks = W.uniform_keys(10, start=0, seed=4)
    keys = np.concatenate([ks, np.array([0, TOMB, 0], dtype=np.uint64)])
    vals = np.arange(1, keys.size + 1, dtype=np.uint64)
    t = oracle_mod.OracleTable(64)
    assert t.build(keys, vals) == 1
    assert t.live == 10
    f = oracle_mod.OracleTable(64, full_key_space=True)
    assert f.build(keys, vals) == 0
    assert f.live == 12
    v, found = f.find(np.array([0, TOMB], dtype=np.uint64))
    assert found.all() and v.tolist() == [13, 12]


def test_build_keeps_last_in_runs_mixing_keys(oracle_mod):
    # two keys whose hashes share all B sort bits (a birthday collision found
    # by search over a stream) form one run; interleaved copies must still
    # give the dictionary of last values
    B = oracle_mod.build_sort_bits(10)
    ks = W.uniform_keys(1 << 18, start=0, seed=77)
    top = oracle_mod.hash64(ks) >> np.uint64(64 - B)
    u, first, counts = np.unique(top, return_index=True, return_counts=True)
    j = int(np.nonzero(counts > 1)[0][0])
    a = int(ks[first[j]])
    b = int(ks[np.nonzero(top == u[j])[0][1]])
    assert a != b
    keys = np.array([a, b, b, a, b, a, a, b], dtype=np.uint64)
    vals = np.arange(1, 9, dtype=np.uint64)
    t = oracle_mod.OracleTable(1 << 10)
    assert t.build(keys, vals) == 0
    got, found = t.find(np.array([a, b], dtype=np.uint64))
    assert found.all() and got.tolist() == [7, 8]
    assert t.live == 2


# ---------------------------------------------------------------------------
# bulk merge of a batch into a non-empty table (Sec. 4.5)
# ---------------------------------------------------------------------------
def _filled(oracle_mod, log2c, n_ins, n_erase, seed, growable=False, **kw):
    keys = W.uniform_keys(n_ins, start=seed * 10_000, seed=33)
    t = oracle_mod.OracleTable(1 << log2c, growable=growable, **kw)
    t.insert(keys, keys ^ np.uint64(0xABCDEF))
    t.erase(keys[:n_erase])
    return t, keys


@pytest.mark.parametrize("log2c,n_ins,n_erase,n,distinct", [(8, 90, 30, 60, 40), (10, 400, 100, 500, 300),
                                                            (12, 2000, 900, 1500, 1200)])
def test_merge_is_the_dictionary_update(oracle_mod, log2c, n_ins, n_erase, n, distinct):
    t, keys = _filled(oracle_mod, log2c, n_ins, n_erase, seed=log2c)
    d = dict(zip(*(a.tolist() for a in t.export())))
    # the batch: some keys of the table (live and erased) and new ones, repeated
    rng = np.random.default_rng(log2c)
    pool = np.concatenate([keys, W.uniform_keys(distinct, start=10**7, seed=33)])
    bk = pool[rng.integers(0, pool.size, n)]
    bv = rng.integers(1, 1 << 62, n).astype(np.uint64)
    assert t.merge(bk, bv) == 0
    for k, v in zip(bk.tolist(), bv.tolist()):
        d[k] = v
    gk, gv = t.export()
    assert dict(zip(gk.tolist(), gv.tolist())) == d
    assert t.live == t.nonempty == len(d)  # the new table has no tombstones
    t.assert_invariants()


@pytest.mark.parametrize("log2c,load", [(8, 0.4), (10, 0.85), (12, 0.95)])
def test_merge_layout_is_sorted_insertion(oracle_mod, log2c, load):
    c = 1 << log2c
    t, keys = _filled(oracle_mod, log2c, int(load * c * 0.6), int(load * c * 0.1), seed=log2c + 3)
    before = t.cells()
    table_order = [int(k) for k in before[:, 0] if k != 0 and k != TOMB]  # cell index order
    live = len(table_order)
    bk, bv = _dup_batch(int(load * c) - live + 40, int(load * c) - live, seed=log2c + 11)
    bk[::7] = np.array(table_order[: bk[::7].size], dtype=np.uint64)[: bk[::7].size]  # replace some
    assert t.merge(bk, bv) == 0
    cells = t.cells()
    _check_valid(cells, log2c, oracle_mod)
    # position of the kept copy in the concatenation (table in cell order, batch)
    pos = {k: i for i, k in enumerate(table_order)}
    for j, k in enumerate(bk.tolist()):
        pos[k] = live + j
    B = oracle_mod.build_sort_bits(log2c)
    run = _run_keys(cells)
    ks = np.array([k for _, k in run], dtype=np.uint64)
    sk = (oracle_mod.hash64(ks) >> np.uint64(64 - B)).tolist()
    order = [(s, pos[k]) for s, k in zip(sk, ks.tolist())]
    descents = sum(1 for a, b in zip(order, order[1:]) if b < a)
    assert descents <= 1
    if descents == 1:
        cut = next(i for i, (a, b) in enumerate(zip(order, order[1:])) if b < a) + 1
        order = order[cut:] + order[:cut]
    assert order == sorted(order)
    homes = oracle_mod.homes(ks, log2c).tolist()
    for (p, _), h in zip(run, homes):
        assert p == h or cells[(p - 1) % c, 0] != 0
    assert len(run) == len(pos)


def test_merge_capacity_full_and_empty_table(oracle_mod):
    # growable: the smallest power of two with live + n <= alpha * c'
    t, _ = _filled(oracle_mod, 8, 100, 20, seed=1, growable=True)
    assert t.capacity == 256 and t.live == 80
    bk = W.uniform_keys(300, start=5 * 10**6, seed=33)
    assert t.merge(bk, bk) == 0
    assert t.capacity == 1024 and t.live == 380  # 80 + 300 > 0.5 * 512
    # bounded: c stays; a merge that leaves no empty cell changes nothing
    t2, _ = _filled(oracle_mod, 6, 40, 0, seed=2)
    snap = t2.cells()
    big = W.uniform_keys(24, start=6 * 10**6, seed=33)
    assert t2.merge(big, big) == -2
    assert np.array_equal(t2.cells(), snap) and t2.live == 40
    assert t2.merge(big[:20], big[:20]) == 0 and t2.live == 60 and t2.capacity == 64
    # into an empty table the merge is the build
    k, v = _dup_batch(700, 500, seed=9)
    a = oracle_mod.OracleTable(1 << 10)
    b = oracle_mod.OracleTable(1 << 10)
    assert a.merge(k, v) == 0 and b.build(k, v) == 0
    assert np.array_equal(a.cells(), b.cells())


def test_merge_special_slots(oracle_mod):
    t, _ = _filled(oracle_mod, 8, 50, 0, seed=3, full_key_space=True)
    t.insert(np.array([0], np.uint64), np.array([11], np.uint64))
    bk = np.array([TOMB, 5, TOMB], dtype=np.uint64)
    bv = np.array([1, 2, 3], dtype=np.uint64)
    assert t.merge(bk, bv) == 0
    v, f = t.find(np.array([0, TOMB, 5], dtype=np.uint64))
    assert f.tolist() == [1, 1, 1] and v.tolist() == [11, 3, 2]  # slot 0 kept, slot 1 = last value
    assert t.live == 53
    plain, _ = _filled(oracle_mod, 8, 50, 0, seed=3)
    assert plain.merge(bk, bv) == 1 and plain.live == 51  # reserved keys skipped
