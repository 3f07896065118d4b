"""GPU against the oracle on the benchmark workloads at their full sizes.

Every case runs the CUDA path through the C ABI and the sequential oracle on
identical seeded inputs and compares the results element by element:

* the 2^20-cell bounded table, exact recipe: 2^19 SplitMix64 seed-1 keys with
  value = 3 * key, then 2^19 shuffled hits and 2^19 misses;
* the 2^28-cell bounded table: inserts to load 0.5 and 0.9 with 2^27 hits and
  2^27 misses at each load, and the word count (insertOrUpdate(add 1)) of
  2^28 Zipf(s) operations over 2^26 keys for every s of the workload;
* the growing table: 2^27 inserts into a growable table of 2^12 cells in one
  call (16 doublings), and the layout of its last doubling against the
  oracle's sequential migration of the same snapshot (Sec. 4.3.1, Lemma 1);
* the sliding window: 2^24 live keys, 128 rounds of 2^20 inserts and 2^20
  erases (tombstones purged by the growth policy's migrations).

Bit-exact: find values and codes, insert and erase codes, per-key sums, the
live (key, value) set, sizes and capacities, occupancy and migration layouts.
The oracle runs in worker threads (its C calls release the GIL) while the GPU
side runs, so the whole module takes a few minutes of host time.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import workloads as W
from gpu_helpers import codes_buf, to_dev, to_np_u8, to_np_u64, vals_buf

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _host(t):
    """uint64 numpy copy of a CUDA int64 tensor."""
    return np.ascontiguousarray(t.cpu().numpy()).view(np.uint64)


def _dev64(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _assert_same_pairs(gk, gv, ok, ov):
    """The GPU's exported (key, value) pairs equal the oracle's, as sets
    (compared on the device: both sorted by key)."""
    import torch

    assert gk.numel() == ok.size, (gk.numel(), ok.size)
    if ok.size == 0:
        return
    ok_t, ov_t = _dev64(ok), _dev64(ov)
    gs, gi = torch.sort(gk)
    os_, oi = torch.sort(ok_t)
    assert torch.equal(gs, os_), "live key sets differ"
    assert torch.equal(gv[gi], ov_t[oi]), "values of equal keys differ"


def _assert_same_finds(t, o_result, q_dev):
    import torch

    n = q_dev.numel()
    vo, fo = vals_buf(n), codes_buf(n)
    t.find(q_dev, vo, fo)
    ev, ef = o_result
    assert torch.equal(fo, torch.from_numpy(ef).cuda()), "find codes differ"
    assert torch.equal(vo, _dev64(ev)), "find values differ"


def _assert_same_occupancy(t, o):
    import torch

    g = t.cells()[:, 0] != 0
    oc = torch.from_numpy(o.cells()[:, 0] != 0).cuda()
    assert torch.equal(g, oc), "occupied cells differ"


# ---------------------------------------------------------------------------
# bounded table, 2^20 cells: the exact small recipe
# ---------------------------------------------------------------------------
def test_bounded_2p20_exact_recipe(cuda_lib, oracle_mod):
    log2c = 20
    wl = W.bounded_workload(log2c, loads=(0.5,), n_find=1 << 19)
    n = wl["counts"][0.5]
    assert n == 1 << 19
    keys, vals = wl["keys"][:n], wl["vals"][:n]
    assert np.array_equal(keys, W.uniform_keys(n, 0, W.SEED_UNIFORM))
    assert np.array_equal(vals, keys * np.uint64(3))
    hits, misses = wl["hits"][0.5], wl["misses"]
    assert np.array_equal(np.sort(hits), np.sort(keys)) and hits.size == 1 << 19
    assert np.array_equal(misses, W.uniform_keys(1 << 19, n, W.SEED_UNIFORM))

    t = cuda_lib.Table(1 << log2c)
    o = oracle_mod.OracleTable(1 << log2c)
    codes = codes_buf(n)
    t.insert(to_dev(keys), to_dev(vals), codes)
    oc = o.insert(keys, vals)
    assert (oc == 1).all()
    assert np.array_equal(to_np_u8(codes), oc)
    for q in (hits, misses):
        vo, fo = vals_buf(q.size), codes_buf(q.size)
        t.find(to_dev(q), vo, fo)
        ev, ef = o.find(q)
        assert np.array_equal(to_np_u8(fo), ef)
        assert np.array_equal(to_np_u64(vo), ev)
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    _assert_same_occupancy(t, o)
    gk, gv = t.export()
    ok, ov = o.export()
    _assert_same_pairs(gk, gv, ok, ov)
    t.destroy()
    o.close()


# ---------------------------------------------------------------------------
# bounded table, 2^28 cells: loads 0.5 and 0.9, hits and misses
# ---------------------------------------------------------------------------
def _oracle_bounded(oracle_mod, log2c, keys, vals, n05, n09, h05, h09, miss):
    o = oracle_mod.OracleTable(1 << log2c)
    out = {"ins05": o.insert(keys[:n05], vals[:n05])}
    out["hit05"] = o.find(h05)
    out["miss05"] = o.find(miss)
    out["ins09"] = o.insert(keys[n05:n09], vals[n05:n09])
    out["hit09"] = o.find(h09)
    out["miss09"] = o.find(miss)
    out["size"] = (o.live, o.nonempty, o.capacity)
    out["pairs"] = o.export()
    out["occupied"] = o.cells()[:, 0] != 0
    o.close()
    return out


def test_bounded_2p28_loads_05_09(cuda_lib, oracle_mod):
    import torch

    log2c = 28
    wl = W.bounded_workload(log2c, loads=(0.5, 0.9), n_find=1 << 27, backend="cuda")
    n05, n09 = wl["counts"][0.5], wl["counts"][0.9]
    assert (n05, n09) == (1 << 27, 241_591_910)
    k, v = wl["keys"], wl["vals"]
    h05, h09, miss = wl["hits"][0.5], wl["hits"][0.9], wl["misses"]
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(_oracle_bounded, oracle_mod, log2c, _host(k), _host(v), n05, n09,
                        _host(h05), _host(h09), _host(miss))
        t = cuda_lib.Table(1 << log2c)
        c05 = codes_buf(n05)
        t.insert(k[:n05], v[:n05], c05)
        n = 1 << 27
        vo = {name: vals_buf(n) for name in ("hit05", "miss05", "hit09", "miss09")}
        fo = {name: codes_buf(n) for name in vo}
        t.find(h05, vo["hit05"], fo["hit05"])
        t.find(miss, vo["miss05"], fo["miss05"])
        c09 = codes_buf(n09 - n05)
        t.insert(k[n05:n09], v[n05:n09], c09)
        t.find(h09, vo["hit09"], fo["hit09"])
        t.find(miss, vo["miss09"], fo["miss09"])
        size = t.size(check=True)
        gk, gv = t.export()
        occ = t.cells()[:, 0] != 0
        t.destroy()
        ref = fut.result()
    assert torch.equal(c05, torch.from_numpy(ref["ins05"]).cuda())
    assert torch.equal(c09, torch.from_numpy(ref["ins09"]).cuda())
    assert (ref["ins05"] == 1).all() and (ref["ins09"] == 1).all()
    for name in vo:
        ev, ef = ref[name]
        assert torch.equal(fo[name], torch.from_numpy(ef).cuda()), name
        assert torch.equal(vo[name], _dev64(ev)), name
    assert size == ref["size"]
    assert torch.equal(occ, torch.from_numpy(ref["occupied"]).cuda())
    _assert_same_pairs(gk, gv, *ref["pairs"])


# ---------------------------------------------------------------------------
# word count on the 2^28-cell table: 2^28 Zipf(s) insertOrUpdate(add 1)
# ---------------------------------------------------------------------------
def _oracle_word_count(oracle_mod, log2c, z):
    o = oracle_mod.OracleTable(1 << log2c)
    codes = o.insert_or_update(z, np.ones(z.size, np.uint64), oracle_mod.ADD)
    out = {"codes_sum": int(codes.sum(dtype=np.uint64)), "size": (o.live, o.nonempty, o.capacity),
           "pairs": o.export()}
    o.close()
    return out


@pytest.mark.parametrize("s", [0.5, 1.0, 1.25, 1.5])
def test_word_count_2p28_zipf(cuda_lib, oracle_mod, s):
    import torch

    log2c, nops = 28, 1 << 28
    z = W.zipf_keys(nops, s, 1 << 26, W.SEED_ZIPF, backend="cuda")
    ones = torch.ones(nops, dtype=torch.int64, device="cuda")
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(_oracle_word_count, oracle_mod, log2c, _host(z))
        t = cuda_lib.Table(1 << log2c)
        codes = codes_buf(nops)
        t.insert_or_update(z, ones, cuda_lib.ADD, codes)
        size = t.size(check=True)
        gk, gv = t.export()
        t.destroy()
        # exactly one operation per distinct key reports the insertion (the
        # table was empty): per-key sums of the codes are all 1
        assert int(codes.max()) <= 1
        uk, inv = torch.unique(z, return_inverse=True)
        per_key = torch.zeros(uk.numel(), dtype=torch.int64, device="cuda").index_add_(0, inv, codes.long())
        assert bool((per_key == 1).all())
        del inv, per_key
        ref = fut.result()
    assert size == ref["size"] and size[0] == uk.numel()
    assert int(codes.sum()) == ref["codes_sum"]
    _assert_same_pairs(gk, gv, *ref["pairs"])  # sums are order-free: bit-exact
    # the counts add up to the number of operations
    assert int(gv.sum()) == nops


# ---------------------------------------------------------------------------
# growing table: 2^27 inserts from 2^12 cells; the last doubling's layout
# ---------------------------------------------------------------------------
def _oracle_grow(oracle_mod, keys, vals):
    o = oracle_mod.OracleTable(1 << 12, growable=True, alpha=0.5)
    codes = o.insert(keys, vals)
    out = {"codes_all_1": bool((codes == 1).all()), "size": (o.live, o.nonempty, o.capacity),
           "migrations": o.migrations, "pairs": o.export()}
    o.close()
    return out


def _oracle_migrate(oracle_mod, snap, new_cap):
    o = oracle_mod.OracleTable(64)
    o.load_cells(snap)
    o.migrate(new_cap)
    cells = o.cells()
    o.close()
    return cells


def test_growing_2p27_inserts_from_2p12(cuda_lib, oracle_mod):
    import torch

    n = 1 << 27
    keys = W.uniform_keys(n, backend="cuda")
    vals = W.values_for(keys, backend="cuda")
    with cf.ThreadPoolExecutor(2) as ex:
        fut = ex.submit(_oracle_grow, oracle_mod, _host(keys), _host(vals))
        # one call: 16 doublings by the growth policy
        t = cuda_lib.Table(1 << 12, growable=True)
        codes = codes_buf(n)
        t.insert(keys, vals, codes)
        size = t.size(check=True)
        assert size == (n, n, 1 << 28)
        assert int(codes.min()) == 1 and int(codes.max()) == 1
        gk, gv = t.export()
        t.destroy()
        # the last doubling (2^27 -> 2^28 cells) on its own: fill to the
        # threshold, snapshot, migrate, compare with the sequential migration
        t2 = cuda_lib.Table(1 << 12, growable=True)
        half = n // 2
        t2.insert(keys[:half], vals[:half])
        assert t2.size(check=True) == (half, half, 1 << 27)
        snap = _host(t2.cells())
        fut_m = ex.submit(_oracle_migrate, oracle_mod, snap, 1 << 28)
        t2.migrate(1 << 28)
        got = t2.cells()
        ref_cells = fut_m.result()
        assert got.shape == (1 << 28, 2)
        assert torch.equal(got, _dev64(ref_cells).reshape(got.shape)), \
            "doubling layout differs from the sequential migration"
        del got, ref_cells, snap
        c2 = codes_buf(n - half)
        t2.insert(keys[half:], vals[half:], c2)
        assert int(c2.min()) == 1 and int(c2.max()) == 1
        assert t2.size(check=True) == (n, n, 1 << 28)
        t2.destroy()
        ref = fut.result()
    assert ref["codes_all_1"]
    assert size == ref["size"]
    assert ref["migrations"] == 16
    _assert_same_pairs(gk, gv, *ref["pairs"])


# ---------------------------------------------------------------------------
# sliding window: 2^24 live keys, 2^27 inserts + 2^27 erases
# ---------------------------------------------------------------------------
def _oracle_window(oracle_mod, keys, win, batch, rounds):
    o = oracle_mod.OracleTable(1 << 12, growable=True, alpha=0.5)
    ok = bool((o.insert(keys[:win], keys[:win]) == 1).all())
    caps = []
    for r in range(rounds):
        ins = keys[win + r * batch: win + (r + 1) * batch]
        ok &= bool((o.insert(ins, ins) == 1).all())
        ok &= bool((o.erase(keys[r * batch: (r + 1) * batch]) == 1).all())
        caps.append(o.capacity)
    out = {"codes_all_1": ok, "caps": caps, "size": (o.live, o.nonempty, o.capacity), "pairs": o.export()}
    o.close()
    return out


def test_sliding_window_2p24_live(cuda_lib, oracle_mod):
    import torch

    win, batch, rounds = 1 << 24, 1 << 20, 128
    keys = W.uniform_keys(win + batch * rounds, backend="cuda")
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(_oracle_window, oracle_mod, _host(keys), win, batch, rounds)
        t = cuda_lib.Table(1 << 12, growable=True)
        c0 = codes_buf(win)
        t.insert(keys[:win], keys[:win], c0)
        ci, ce = codes_buf(batch), codes_buf(batch)
        bad = torch.zeros((), dtype=torch.int64, device="cuda")
        caps = []
        for r in range(rounds):
            ins = keys[win + r * batch: win + (r + 1) * batch]
            t.insert(ins, ins, ci)
            t.erase(keys[r * batch: (r + 1) * batch], ce)
            bad += (ci != 1).sum() + (ce != 1).sum()
            caps.append(t.size()[2])
        size = t.size(check=True)
        gk, gv = t.export()
        t.destroy()
        ref = fut.result()
    assert int((c0 != 1).sum()) == 0 and int(bad) == 0
    assert ref["codes_all_1"]
    assert caps == ref["caps"]
    assert size == ref["size"] and size[0] == win
    _assert_same_pairs(gk, gv, *ref["pairs"])


# ---------------------------------------------------------------------------
# batched: 4096 tables (element counts log-uniform 2^8..2^20), every batch in
# one engine launch; every table checked against the oracle
# ---------------------------------------------------------------------------
def _oracle_tables(oracle_mod, wl, tabs, keys, vals, vout, codes):
    """Run the oracle over the batches of `tabs` in order; return the first
    mismatch found (or None) and the final contents per table."""
    bad, contents = None, {}
    for t in tabs:
        o = oracle_mod.OracleTable(int(wl["capacity"][t]))
        for b in wl["by_table"][t]:
            o0, o1 = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
            k = keys[o0:o1]
            op = int(wl["op"][b])
            if op == W.OP_FIND:
                ev, ef = o.find(k)
                if bad is None and not (np.array_equal(ev, vout[o0:o1]) and np.array_equal(ef, codes[o0:o1])):
                    bad = f"table {t} batch {b}: find results differ"
            elif op == W.OP_INSERT:
                oc = o.insert(k, vals[o0:o1])
                if bad is None and not np.array_equal(oc, codes[o0:o1]):
                    bad = f"table {t} batch {b}: insert codes differ"
            else:
                o.insert_or_update(k, vals[o0:o1], oracle_mod.ADD)
        ok, ov = o.export()
        order = np.argsort(ok)
        contents[t] = (ok[order], ov[order])
        o.close()
    return bad, contents


def test_batched_4096_tables_one_launch(cuda_lib, oracle_mod):
    import torch

    wl = W.batched_workload(4096, 8, 20, seed=W.SEED_TABLES)
    nb = len(wl["n"])
    total = int(wl["offsets"][-1])
    keys = torch.empty(total, dtype=torch.int64, device="cuda")
    vals = torch.empty(total, dtype=torch.int64, device="cuda")
    b0 = 0
    while b0 < nb:  # generated in pieces of about 2^27 operations
        b1 = int(np.searchsorted(wl["offsets"], wl["offsets"][b0] + (1 << 27), side="right")) - 1
        b1 = min(max(b1, b0 + 1), nb)
        k, v = W.batched_keys(wl, b0, b1, backend="cuda")
        keys[wl["offsets"][b0]:wl["offsets"][b1]] = k
        vals[wl["offsets"][b0]:wl["offsets"][b1]] = v
        del k, v
        b0 = b1
    vout = torch.zeros(total, dtype=torch.int64, device="cuda")
    codes = torch.full((total,), 255, dtype=torch.uint8, device="cuda")
    tables = [cuda_lib.Table(int(c)) for c in wl["capacity"]]
    segs = []
    for b in range(nb):
        o0, o1 = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
        op = int(wl["op"][b])
        segs.append((tables[int(wl["table"][b])], op, keys[o0:o1], vals[o0:o1] if op != W.OP_FIND else None,
                     vout[o0:o1] if op == W.OP_FIND else None, codes[o0:o1]))
    plan = cuda_lib.Plan(segs)
    l0 = cuda_lib.launch_count()
    plan.launch()
    assert plan.status() == 0
    assert cuda_lib.launch_count() - l0 == 1
    hk, hv = _host(keys), _host(vals)
    hvo, hc = _host(vout), codes.cpu().numpy()
    del keys, vals, vout, codes
    order = np.argsort(wl["table"], kind="stable")
    starts = np.searchsorted(wl["table"][order], np.arange(4097))
    wl["by_table"] = [order[starts[t]:starts[t + 1]] for t in range(4096)]
    groups = [list(range(i, 4096, 16)) for i in range(16)]
    with cf.ThreadPoolExecutor(16) as ex:
        futs = [ex.submit(_oracle_tables, oracle_mod, wl, g, hk, hv, hvo, hc) for g in groups]
        results = [f.result() for f in futs]
    for bad, _ in results:
        assert bad is None, bad
    for _, contents in results:
        for t, (ok, ov) in contents.items():
            gk, gv = tables[t].export()
            gk, gv = _host(gk), _host(gv)
            o = np.argsort(gk)
            assert np.array_equal(gk[o], ok) and np.array_equal(gv[o], ov), f"table {t}: contents differ"
    plan.destroy()
    for t in tables:
        t.destroy()
