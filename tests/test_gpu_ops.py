"""GPU parity of the batched operations against the CPU oracle (through the C ABI).

Bit-exact where the result is unique (find values and codes, aggregated
sums, final key sets, occupied cells); set-valued where duplicates inside one
batch allow several correct outcomes (which op inserted / erased, which value
an overwrite kept).  Sizes span many CTAs and warps and leave ragged tails.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import (assert_one_winner, assert_same_live_set, codes_buf, ops_by_key, to_dev,
                         to_np_u8, to_np_u64, vals_buf)

pytestmark = pytest.mark.gpu

GROUPS = [0, 1, 2, 4, 8, 16, 32]  # 0 = chosen by load
# (group width, cells per lane): every probe window shape the kernels support
WIDTHS = [(g, 0) for g in GROUPS] + [(2, 2), (4, 2), (8, 2), (16, 2), (1, 4), (2, 4), (4, 4), (8, 4),
                                     (-1, 0), (-1, 2), (-1, 4)]  # -1: one thread per operation


def _table(cht, cap, g=1, growable=False, v=0, **cfg):
    t = cht.Table(cap, growable=growable)
    t.set_config(group_width=g, lane_cells=v, **cfg)
    return t


@pytest.mark.parametrize("g,v", WIDTHS)
@pytest.mark.parametrize("load", [0.5, 0.9])
def test_insert_find_uniform(cuda_lib, oracle_mod, g, v, load):
    log2c = 16
    c = 1 << log2c
    wl = W.bounded_workload(log2c, loads=(load,), n_find=(c // 3) + 17)
    n = wl["counts"][load]
    keys, vals = wl["keys"][:n], wl["vals"][:n]
    t = _table(cuda_lib, c, g, v=v)
    o = oracle_mod.OracleTable(c)
    codes = codes_buf(n)
    t.insert(to_dev(keys), to_dev(vals), codes)
    assert (to_np_u8(codes) == 1).all()
    assert (o.insert(keys, vals) == 1).all()
    live, ne, cap = t.size(check=True)
    assert (live, ne, cap) == (n, n, c)
    # occupied cells depend only on the multiset of homes: equal to the oracle
    gcells = to_np_u64(t.cells())
    assert np.array_equal(gcells.reshape(-1, 2)[:, 0] != 0, o.cells()[:, 0] != 0)
    for q in (wl["hits"][load], wl["misses"]):
        vo, fo = vals_buf(q.size), codes_buf(q.size)
        t.find(to_dev(q), vo, fo)
        ev, ef = o.find(q)
        assert np.array_equal(to_np_u8(fo), ef)
        assert np.array_equal(to_np_u64(vo), ev)
    assert_same_live_set(t, o)


@pytest.mark.parametrize("g,v", [(1, 0), (8, 0), (8, 2), (-1, 2), (-1, 4)])
def test_insert_duplicates_one_winner(cuda_lib, oracle_mod, g, v):
    c = 1 << 14
    base = W.uniform_keys(3000, seed=51)
    rng = np.random.default_rng(1)
    pre = base[:500]
    keys = base[rng.integers(0, base.size, 9001)]
    vals = rng.integers(1, 1 << 62, keys.size).astype(np.uint64)
    t = _table(cuda_lib, c, g, v=v)
    t.insert(to_dev(pre), to_dev(pre))
    codes = codes_buf(keys.size)
    t.insert(to_dev(keys), to_dev(vals), codes)
    cs = to_np_u8(codes)
    pre_set = set(pre.tolist())
    assert_one_winner(keys, cs, lambda k: k not in pre_set)
    # stored value: untouched for pre-existing keys; else one of the key's values
    uk = np.unique(keys)
    vo = vals_buf(uk.size)
    t.find(to_dev(uk), vo)
    got = dict(zip(uk.tolist(), to_np_u64(vo).tolist()))
    by = ops_by_key(keys, vals, cs)
    for k, rows in by.items():
        if k in pre_set:
            assert got[k] == k
        else:
            winner = [v for v, code in rows if code == 1]
            assert got[k] == winner[0]
    live, _, _ = t.size()
    assert live == len(pre_set | set(keys.tolist()))


IOU_PATHS = [(0, 1), (0, 2)] + [(g, 0) for g in GROUPS + [-1]]  # (group width, shared-memory aggregation)


@pytest.mark.parametrize("g,agg", IOU_PATHS)
@pytest.mark.parametrize("s", [0.5, 1.25, 1.5])
def test_insert_or_update_add_exact(cuda_lib, oracle_mod, g, agg, s):
    c = 1 << 17
    keys = W.zipf_keys(150_001, s, n_ranks=1 << 15, seed=52)
    vals = (np.arange(keys.size, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) | np.uint64(1)
    keys[::997] = 0  # reserved keys inside the batch
    pre = np.unique(keys[keys != 0])[::5]
    t = _table(cuda_lib, c, g, iou_aggregate=agg)
    o = oracle_mod.OracleTable(c)
    t.insert(to_dev(pre), to_dev(pre))
    o.insert(pre, pre)
    codes = codes_buf(keys.size)
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.ADD, codes)
    o.insert_or_update(keys, vals, oracle_mod.ADD)
    pre_set = set(pre.tolist())
    cs = to_np_u8(codes)
    assert (cs[keys == 0] == 3).all()
    live_ops = keys != 0
    assert_one_winner(keys[live_ops], cs[live_ops], lambda k: k not in pre_set)
    assert_same_live_set(t, o)  # sums are order-free: bit-exact
    live, ne, _ = t.size()
    assert live == o.live and ne == o.nonempty


@pytest.mark.parametrize("g,agg", [(0, 1), (0, 2), (1, 0), (4, 0)])
def test_insert_or_update_overwrite(cuda_lib, oracle_mod, g, agg):
    c = 1 << 15
    keys = W.zipf_keys(40_000, 1.0, n_ranks=1 << 12, seed=53)
    vals = np.arange(1, keys.size + 1, dtype=np.uint64)
    pre = np.unique(keys)[::3]
    t = _table(cuda_lib, c, g, iou_aggregate=agg)
    t.insert(to_dev(pre), to_dev(pre))
    codes = codes_buf(keys.size)
    t.insert_or_update(to_dev(keys), to_dev(vals), cuda_lib.OVERWRITE, codes)
    pre_set = set(pre.tolist())
    assert_one_winner(keys, to_np_u8(codes), lambda k: k not in pre_set)
    uk = np.unique(keys)
    vo = vals_buf(uk.size)
    t.find(to_dev(uk), vo)
    by = ops_by_key(keys, vals)
    for k, v in zip(uk.tolist(), to_np_u64(vo).tolist()):
        assert v in {r[0] for r in by[k]}


@pytest.mark.parametrize("g,v", [(1, 0), (2, 0), (8, 0), (32, 0), (4, 2), (8, 2), (-1, 2), (-1, 4)])
def test_erase_and_tombstones(cuda_lib, oracle_mod, g, v):
    c = 1 << 15
    keys = W.uniform_keys(20_000, seed=54)
    t = _table(cuda_lib, c, g, v=v)
    o = oracle_mod.OracleTable(c)
    t.insert(to_dev(keys), to_dev(keys))
    o.insert(keys, keys)
    rng = np.random.default_rng(2)
    victims = np.concatenate([keys[rng.integers(0, keys.size, 12_000)],
                              W.uniform_keys(777, start=10**6, seed=54)])  # absent ones too
    codes = codes_buf(victims.size)
    t.erase(to_dev(victims), codes)
    o.erase(victims)
    present = set(keys.tolist())
    assert_one_winner(victims, to_np_u8(codes), lambda k: k in present)
    live, ne, _ = t.size()
    assert live == o.live and ne == o.nonempty == keys.size
    # finds pass over tombstones
    vo, fo = vals_buf(keys.size), codes_buf(keys.size)
    t.find(to_dev(keys), vo, fo)
    ev, ef = o.find(keys)
    assert np.array_equal(to_np_u8(fo), ef) and np.array_equal(to_np_u64(vo), ev)
    # inserting again after erase uses fresh cells (tombstones are not reused)
    again = victims[: 100]
    t.insert(to_dev(again), to_dev(again))
    o.insert(again, again)
    assert_same_live_set(t, o)
    assert t.size()[1] == o.nonempty


@pytest.mark.parametrize("g", [1, -1])
def test_reserved_keys(cuda_lib, g):
    import torch

    t = _table(cuda_lib, 1024, g)
    keys = np.array([5, 0, (1 << 64) - 1, 9], dtype=np.uint64)
    codes = codes_buf(4)
    t.insert(to_dev(keys), to_dev(keys), codes)
    assert to_np_u8(codes).tolist() == [1, 3, 3, 1]
    vo, fo = vals_buf(4), codes_buf(4)
    t.find(to_dev(keys), vo, fo)
    assert to_np_u8(fo).tolist() == [1, 3, 3, 1]
    assert to_np_u64(vo).tolist() == [5, 0, 0, 9]
    with pytest.raises(cuda_lib.ChtError) as e:
        t.size(check=True)
    assert e.value.status == cuda_lib.CHT_ERR_RESERVED_KEY
    assert t.status() & cuda_lib.STATUS_RESERVED
    assert t.status() == 0  # cleared by the previous read
    assert t.size()[:2] == (2, 2)
    torch.cuda.synchronize()


@pytest.mark.parametrize("g,v", [(1, 0), (8, 0), (32, 0), (16, 2), (-1, 2), (-1, 4)])
def test_full_bounded_table(cuda_lib, g, v):
    t = _table(cuda_lib, 64, g, v=v)
    keys = W.uniform_keys(100, seed=55)
    codes = codes_buf(100)
    t.insert(to_dev(keys), to_dev(keys), codes)
    cs = to_np_u8(codes)
    assert (cs == 1).sum() == 64 and (cs == 2).sum() == 36
    assert t.status() & cuda_lib.STATUS_FULL
    vo, fo = vals_buf(100), codes_buf(100)
    t.find(to_dev(keys), vo, fo)
    assert np.array_equal(to_np_u8(fo) == 1, cs == 1)
    miss = W.uniform_keys(10, start=5000, seed=55)
    vo, fo = vals_buf(10), codes_buf(10)
    t.find(to_dev(miss), vo, fo)  # terminates after c cells
    assert (to_np_u8(fo) == 0).all()


def test_empty_batches_and_bad_args(cuda_lib):
    import torch

    t = _table(cuda_lib, 1000)
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    t.insert(e, e)
    t.find(e, e)
    t.erase(e)
    t.insert_or_update(e, e)
    assert t.size() == (0, 0, 1024)
    with pytest.raises(cuda_lib.ChtError):
        t.set_config(group_width=3)
    with pytest.raises(cuda_lib.ChtError):
        t.set_config(group_width=32, lane_cells=2)
    with pytest.raises(cuda_lib.ChtError):
        t.insert_or_update(to_dev(np.array([1], np.uint64)), to_dev(np.array([1], np.uint64)), op=7)


def test_host_arrays_match_device(cuda_lib, oracle_mod):
    c = 1 << 14
    keys = W.uniform_keys(5000, seed=56)
    vals = W.values_for(keys)
    t = _table(cuda_lib, c)
    codes = np.full(keys.size, 255, np.uint8)
    t.insert(keys, vals, codes)  # numpy in, numpy out: staged by the library
    import torch

    torch.cuda.synchronize()
    assert (codes == 1).all()
    q = np.concatenate([keys[::3], W.uniform_keys(100, start=9000, seed=56)])
    vo = np.zeros(q.size, np.uint64)
    fo = np.zeros(q.size, np.uint8)
    t.find(q, vo, fo)
    torch.cuda.synchronize()
    o = oracle_mod.OracleTable(c)
    o.insert(keys, vals)
    ev, ef = o.find(q)
    assert np.array_equal(vo, ev) and np.array_equal(fo, ef)
    # pinned host memory goes through the same staging
    pk = torch.from_numpy(q.view(np.int64)).pin_memory()
    pv = torch.zeros(q.size, dtype=torch.int64).pin_memory()
    pc = torch.zeros(q.size, dtype=torch.uint8).pin_memory()
    t.find(pk, pv, pc)
    torch.cuda.synchronize()
    assert np.array_equal(pv.numpy().view(np.uint64), ev)
    assert np.array_equal(pc.numpy(), ef)


@pytest.mark.parametrize("growable", [False, True])
def test_pinned_host_arrays(cuda_lib, oracle_mod, growable):
    """Pinned host arrays as inputs and outputs of every operation type (the
    growable table also takes its chunked growth path on them)."""
    import torch

    c = 1 << 12 if growable else 1 << 15
    keys = W.uniform_keys(12000, seed=57)
    vals = W.values_for(keys)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()  # noqa: E731
    pk, pv = pin(keys), pin(vals)
    pc = torch.full((keys.size,), 255, dtype=torch.uint8).pin_memory()
    t = cuda_lib.Table(c, growable=growable)
    o = oracle_mod.OracleTable(c, growable=growable)
    t.insert(pk, pv, pc)
    torch.cuda.synchronize()
    assert np.array_equal(pc.numpy(), o.insert(keys, vals))
    z = W.zipf_keys(20000, 1.0, 4000, seed=9)
    pz, pones = pin(z), pin(np.ones(z.size, np.uint64))
    zc = torch.full((z.size,), 255, dtype=torch.uint8).pin_memory()
    t.insert_or_update(pz, pones, cuda_lib.ADD, zc)
    torch.cuda.synchronize()
    oc = ops_by_key(z, o.insert_or_update(z, np.ones(z.size, np.uint64), 1))
    for k, cs in ops_by_key(z, zc.numpy()).items():  # one insertion per new key, as in the oracle
        assert sum(c_[0] for c_ in cs) == sum(x[0] for x in oc[k])
    ec = torch.full((4000,), 255, dtype=torch.uint8).pin_memory()
    t.erase(pin(keys[:4000]), ec)
    torch.cuda.synchronize()
    assert np.array_equal(ec.numpy(), o.erase(keys[:4000]))
    q = np.concatenate([keys, z])
    pq = pin(q)
    qv = torch.zeros(q.size, dtype=torch.int64).pin_memory()
    qc = torch.zeros(q.size, dtype=torch.uint8).pin_memory()
    t.find(pq, qv, qc)
    torch.cuda.synchronize()
    ev, ef = o.find(q)
    assert np.array_equal(qv.numpy().view(np.uint64), ev) and np.array_equal(qc.numpy(), ef)


def _tombstones(t):
    cells = to_np_u64(t.cells()).reshape(-1, 2)
    return int((cells[:, 0] == np.uint64((1 << 64) - 1)).sum())


@pytest.mark.parametrize("g,agg,mode", [(1, 0, "insert"), (4, 0, "insert"), (8, 0, "insert"), (1, 0, "iou_add"),
                                        (4, 0, "iou_ow"), (0, 1, "iou_add"), (0, 2, "iou_ow"), (16, 0, "insert"),
                                        (-1, 0, "insert")])
def test_reuse_tombstones_matches_oracle(cuda_lib, oracle_mod, g, agg, mode):
    """Tombstone reuse: erase, then insert / insertOrUpdate a mix of erased,
    live and fresh keys with duplicates, several rounds; results and contents
    equal the oracle with reuse on, counts are consistent with the cells
    (I = non-empty, D = tombstones), and reused cells keep probes short."""
    c = 1 << 14
    rng = np.random.default_rng(5)
    universe = W.uniform_keys(5000, seed=57)
    t = _table(cuda_lib, c, g, v=2 if g in (4, 8) else 0, iou_aggregate=agg, reuse_tombstones=1)
    o = oracle_mod.OracleTable(c, reuse_tombstones=True)
    t.insert(to_dev(universe[:3000]), to_dev(universe[:3000]))
    o.insert(universe[:3000], universe[:3000])
    for r in range(6):
        victims = universe[rng.integers(0, universe.size, 2000)]
        ec = codes_buf(victims.size)
        t.erase(to_dev(victims), ec)
        oc = o.erase(victims)
        for k in np.unique(victims):
            m = victims == k
            assert int(to_np_u8(ec)[m].sum()) == int(oc[m].sum())
        keys = universe[rng.integers(0, universe.size, 4000)]
        vals = keys ^ np.uint64(0x9E3779B97F4A7C15) if mode == "insert" else \
            rng.integers(1, 1 << 40, keys.size).astype(np.uint64)
        codes = codes_buf(keys.size)
        if mode == "insert":
            t.insert(to_dev(keys), to_dev(vals), codes)
            oc = o.insert(keys, vals)
        else:
            op = cuda_lib.ADD if mode == "iou_add" else cuda_lib.OVERWRITE
            t.insert_or_update(to_dev(keys), to_dev(vals), op, codes)
            oc = o.insert_or_update(keys, vals, oracle_mod.ADD if mode == "iou_add" else oracle_mod.OVERWRITE)
        gc = to_np_u8(codes)
        for k in np.unique(keys):
            m = keys == k
            assert int(gc[m].sum()) == int(oc[m].sum())
        if mode != "iou_ow":
            assert_same_live_set(t, o)  # overwrite keeps one of several values: compared by key below
        gk, _ = t.export()
        ok, _ = o.export()
        assert np.array_equal(np.sort(to_np_u64(gk)), np.sort(ok))
        live, ne, _ = t.size(check=True)
        assert live == o.live
        assert ne - live == _tombstones(t)  # D = tombstones left in the cells
        assert ne == int((to_np_u64(t.cells()).reshape(-1, 2)[:, 0] != 0).sum())
    # reuse keeps the table from filling with tombstones: never more non-empty
    # cells than the keys ever inserted
    assert t.size()[1] <= universe.size


@pytest.mark.parametrize("g,v,agg", [(0, 0, 1), (0, 0, 0), (1, 0, 0), (4, 2, 0), (8, 2, 0), (2, 1, 0), (32, 1, 0),
                                     (-1, 2, 0), (-1, 4, 0)])
@pytest.mark.parametrize("mode", ["add", "overwrite"])
def test_update_matches_oracle(cuda_lib, oracle_mod, g, v, agg, mode):
    """update (Sec. 3): present keys change, absent and erased ones do not; the
    presence code of every operation is exact, add sums are exact, overwrite
    keeps one of the batch's values; nothing is inserted."""
    c = 1 << 15
    rng = np.random.default_rng(9)
    keys = W.uniform_keys(12_000, seed=58)
    t = _table(cuda_lib, c, g, v=v, iou_aggregate=agg)
    o = oracle_mod.OracleTable(c)
    t.insert(to_dev(keys), to_dev(keys))
    o.insert(keys, keys)
    gone = keys[:2000]
    t.erase(to_dev(gone))
    o.erase(gone)
    pool = np.concatenate([keys, W.uniform_keys(3000, start=10**7, seed=58)])
    ks = pool[rng.integers(0, pool.size, 40_001)]
    vs = rng.integers(1, 1 << 40, ks.size).astype(np.uint64)
    op = cuda_lib.ADD if mode == "add" else cuda_lib.OVERWRITE
    codes = codes_buf(ks.size)
    t.update(to_dev(ks), to_dev(vs), op, codes)
    oc = o.update(ks, vs, oracle_mod.ADD if mode == "add" else oracle_mod.OVERWRITE)
    assert np.array_equal(to_np_u8(codes), oc)
    live, ne, _ = t.size(check=True)
    assert (live, ne) == (o.live, o.nonempty)
    if mode == "add":
        assert_same_live_set(t, o)
    else:
        uk = np.unique(ks[oc == 1])
        vo = vals_buf(uk.size)
        t.find(to_dev(uk), vo)
        got = to_np_u64(vo)
        for k, gv in zip(uk, got):
            assert gv in set(vs[ks == k].tolist())


@pytest.mark.parametrize("g,v,agg", [(0, 0, 1), (1, 0, 0), (4, 4, 0), (8, 2, 0), (32, 1, 0), (0, 0, 2), (-1, 4, 0)])
def test_full_key_space_matches_oracle(cuda_lib, oracle_mod, g, v, agg):
    """Keys 0 and ~0 mixed into every operation type (many copies per batch):
    codes, found values and the exported contents equal the oracle's special
    slots; the live count includes them, the cells never hold them."""
    c = 1 << 14
    rng = np.random.default_rng(31)
    t = _table(cuda_lib, c, g, v=v, iou_aggregate=agg, full_key_space=1)
    o = oracle_mod.OracleTable(c, full_key_space=True)
    pool = np.concatenate([W.uniform_keys(3000, seed=59), np.array([0, (1 << 64) - 1], dtype=np.uint64)])
    for r in range(30):
        n = int(rng.integers(1, 3000))
        ks = pool[rng.integers(0, pool.size, n)]
        ks[rng.integers(0, n, max(1, n // 50))] = rng.choice(np.array([0, (1 << 64) - 1], dtype=np.uint64))
        vs = rng.integers(1, 1 << 40, n).astype(np.uint64)
        kind = rng.choice(["insert", "iou_add", "iou_ow", "find", "erase", "upd_add", "upd_ow"])
        codes = codes_buf(n)
        if kind == "find":
            vo = vals_buf(n)
            t.find(to_dev(ks), vo, codes)
            ev, ef = o.find(ks)
            assert np.array_equal(to_np_u8(codes), ef) and np.array_equal(to_np_u64(vo), ev)
            continue
        if kind == "insert":
            vs = ks ^ np.uint64(0x1234567)  # the stored value does not depend on which copy wins
            t.insert(to_dev(ks), to_dev(vs), codes)
            oc = o.insert(ks, vs)
        elif kind in ("iou_add", "iou_ow"):
            op = cuda_lib.ADD if kind == "iou_add" else cuda_lib.OVERWRITE
            vs = vs if kind == "iou_add" else ks ^ np.uint64(0x7654321)
            t.insert_or_update(to_dev(ks), to_dev(vs), op, codes)
            oc = o.insert_or_update(ks, vs, oracle_mod.ADD if kind == "iou_add" else oracle_mod.OVERWRITE)
        elif kind in ("upd_add", "upd_ow"):
            op = cuda_lib.ADD if kind == "upd_add" else cuda_lib.OVERWRITE
            vs = vs if kind == "upd_add" else ks ^ np.uint64(0x55AA)
            t.update(to_dev(ks), to_dev(vs), op, codes)
            oc = o.update(ks, vs, oracle_mod.ADD if kind == "upd_add" else oracle_mod.OVERWRITE)
            assert np.array_equal(to_np_u8(codes), oc)
        else:
            t.erase(to_dev(ks), codes)
            oc = o.erase(ks)
        gc = to_np_u8(codes)
        for k in np.unique(ks):
            m = ks == k
            assert int(gc[m].astype(np.int64).sum()) == int(oc[m].astype(np.int64).sum()), (kind, k)
        live, ne, _ = t.size(check=True)
        assert live == o.live and ne == o.nonempty
        assert_same_live_set(t, o)
    cells = to_np_u64(t.cells()).reshape(-1, 2)
    assert not (cells[:, 0] == 0).all() or o.nonempty == 0
    g_ = oracle_mod.OracleTable(64)
    g_.load_cells(cells)
    g_.assert_invariants()


@pytest.mark.parametrize("mode", ["add", "overwrite"])
@pytest.mark.parametrize("full_keys", [0, 1])
def test_insert_or_update_low_skew_windows(cuda_lib, oracle_mod, mode, full_keys):
    """Enough windows per CTA (2^23 operations) that low-skew stretches run
    without the shared-memory fold and skewed ones with it, in both orders:
    a segment of nearly distinct keys, a Zipf(1.5) segment, nearly distinct
    keys again (with repeats of earlier ones), reserved keys throughout.  Add
    sums bit-exact; overwrite stores a value that depends only on the key, so
    it is exact whichever copy lands last; one insertion code per new key."""
    n_seg = 1 << 21
    rng = np.random.default_rng(61)
    uni = W.uniform_keys(1 << 22, seed=62)
    seg_a = uni[rng.integers(0, uni.size, n_seg)]
    seg_b = W.zipf_keys(n_seg, 1.5, n_ranks=1 << 16, seed=63)
    seg_c = uni[rng.integers(0, uni.size, 2 * n_seg)]
    keys = np.concatenate([seg_a, seg_b, seg_c])
    keys[rng.integers(0, keys.size, 4000)] = 0
    keys[rng.integers(0, keys.size, 4000)] = np.uint64((1 << 64) - 1)
    if mode == "add":
        vals = (np.arange(keys.size, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) | np.uint64(1)
        op, oop = cuda_lib.ADD, oracle_mod.ADD
    else:
        vals = keys ^ np.uint64(0x5DEECE66D)
        op, oop = cuda_lib.OVERWRITE, oracle_mod.OVERWRITE
    pre = uni[::7]
    c = 1 << 24
    t = _table(cuda_lib, c, 0, iou_aggregate=1, full_key_space=full_keys)
    o = oracle_mod.OracleTable(c, full_key_space=bool(full_keys))
    t.insert(to_dev(pre), to_dev(pre))
    o.insert(pre, pre)
    codes = codes_buf(keys.size)
    t.insert_or_update(to_dev(keys), to_dev(vals), op, codes)
    oc = o.insert_or_update(keys, vals, oop)
    cs = to_np_u8(codes)
    reserved = (keys == 0) | (keys == np.uint64((1 << 64) - 1))
    if not full_keys:
        assert (cs[reserved] == 3).all()
    # per key: the number of insertion codes (one for a new key, none for a
    # present one) equals the oracle's
    order = np.argsort(keys, kind="stable")
    ks, gsum, osum = keys[order], cs[order].astype(np.int64), oc[order].astype(np.int64)
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    assert np.array_equal(np.add.reduceat(gsum, starts), np.add.reduceat(osum, starts))
    assert set(np.unique(cs[~reserved]).tolist()) <= {0, 1}
    assert_same_live_set(t, o)
    live, ne, _ = t.size()  # (the sticky status holds the reserved-key bit when full_keys is off)
    assert live == o.live and ne == o.nonempty
