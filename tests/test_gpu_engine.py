"""GPU parity of the batched engine (one persistent launch for many tables).

Every table's batches must give exactly what the single calls give, in
order: find values and codes bit-exact against the oracle run table by
table; insertOrUpdate codes set-valued (per distinct key of a batch, the
number of 1 codes equals the oracle's); final contents of every table
bit-exact.  Also: the launch inside a captured CUDA graph, the bounded
dependency wait running out (a count nothing reaches), and the autotuner.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import to_np_u64, to_np_u8

pytestmark = pytest.mark.gpu


def _setup(cht, wl):
    import torch

    keys, vals = W.batched_keys(wl, backend="cuda")
    total = keys.numel()
    vout = torch.full((total,), -1, dtype=torch.int64, device="cuda")
    codes = torch.full((total,), 255, dtype=torch.uint8, device="cuda")
    tables = [cht.Table(int(c)) for c in wl["capacity"]]
    ops = []
    for b in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
        op = int(wl["op"][b])
        t = tables[int(wl["table"][b])]
        ops.append((t, op, keys[lo:hi], vals[lo:hi] if op != W.OP_FIND else None,
                    vout[lo:hi] if op == W.OP_FIND else None, codes[lo:hi]))
    return tables, ops, vout, codes


def _oracle(oracle_mod, wl):
    keys, vals = W.batched_keys(wl)
    tabs = [oracle_mod.OracleTable(int(c)) for c in wl["capacity"]]
    vout = np.zeros(keys.size, np.uint64)
    codes = np.zeros(keys.size, np.uint8)
    for b in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
        t, op = tabs[int(wl["table"][b])], int(wl["op"][b])
        if op == W.OP_FIND:
            vout[lo:hi], codes[lo:hi] = t.find(keys[lo:hi])
        elif op == W.OP_INSERT:
            codes[lo:hi] = t.insert(keys[lo:hi], vals[lo:hi])
        else:
            codes[lo:hi] = t.insert_or_update(keys[lo:hi], vals[lo:hi], oracle_mod.ADD)
    return tabs, keys, vout, codes


def _check(wl, keys, tables, vout, codes, otabs, ovout, ocodes):
    g_v, g_c = to_np_u64(vout), to_np_u8(codes)
    for b in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
        op = int(wl["op"][b])
        if op == W.OP_FIND:
            assert np.array_equal(g_c[lo:hi], ocodes[lo:hi]), b
            assert np.array_equal(g_v[lo:hi], ovout[lo:hi]), b
        elif op == W.OP_INSERT:
            assert np.array_equal(g_c[lo:hi], ocodes[lo:hi]), b
        else:
            seg = keys[lo:hi]
            for k in np.unique(seg):
                m = seg == k
                assert int(g_c[lo:hi][m].astype(np.int64).sum()) == int(ocodes[lo:hi][m].astype(np.int64).sum()), b
    for t, o in zip(tables, otabs):
        gk, gv = t.export()
        gk, gv = to_np_u64(gk), to_np_u64(gv)
        ok, ov = o.export()
        assert gk.size == ok.size
        i, j = np.argsort(gk), np.argsort(ok)
        assert np.array_equal(gk[i], ok[j]) and np.array_equal(gv[i], ov[j])


@pytest.mark.parametrize("g,v,direct,chunk", [(0, 0, 0, 0), (4, 2, 0, 0), (8, 1, 0, 0), (32, 1, 0, 0), (0, 0, 1, 0),
                                               (4, 2, 1, 0), (0, 0, 0, 32), (0, 0, 1, 64), (8, 1, 0, 128)])
def test_engine_matches_oracle(cuda_lib, oracle_mod, g, v, direct, chunk):
    wl = W.batched_workload(48, 6, 11, seed=31)
    tables, ops, vout, codes = _setup(cuda_lib, wl)
    plan = cuda_lib.Plan(ops)
    plan.set_config(group_width=g, lane_cells=v, direct_io=direct, chunk_ops=chunk)
    plan.launch()
    assert plan.status() == 0
    otabs, keys, ovout, ocodes = _oracle(oracle_mod, wl)
    _check(wl, keys, tables, vout, codes, otabs, ovout, ocodes)


def test_engine_in_cuda_graph(cuda_lib, oracle_mod):
    import torch

    wl = W.batched_workload(32, 6, 10, seed=32)
    # warm the engine kernel's launch path outside the capture
    warm_tables, warm_ops, _, _ = _setup(cuda_lib, W.batched_workload(4, 6, 7, seed=33))
    cuda_lib.Plan(warm_ops).launch()
    torch.cuda.synchronize()
    tables, ops, vout, codes = _setup(cuda_lib, wl)
    plan = cuda_lib.Plan(ops)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.launch()
    graph.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    otabs, keys, ovout, ocodes = _oracle(oracle_mod, wl)
    _check(wl, keys, tables, vout, codes, otabs, ovout, ocodes)


def test_engine_dependency_wait_times_out(cuda_lib):
    wl = W.batched_workload(8, 6, 9, seed=34)
    tables, ops, vout, codes = _setup(cuda_lib, wl)
    plan = cuda_lib.Plan(ops)
    plan.set_config(fault_inject=1, spin_limit_us=200)
    plan.launch()
    assert plan.status() & cuda_lib.PLAN_TIMEOUT
    plan.set_config(fault_inject=0, spin_limit_us=0)


def test_engine_autotune_restores_tables(cuda_lib, oracle_mod):
    wl = W.batched_workload(24, 6, 10, seed=35)
    tables, ops, vout, codes = _setup(cuda_lib, wl)
    plan = cuda_lib.Plan(ops)
    ms = plan.autotune()
    assert ms > 0
    for t in tables:
        assert t.size()[:2] == (0, 0)  # contents restored after every trial
    plan.launch()
    assert plan.status() == 0
    otabs, keys, ovout, ocodes = _oracle(oracle_mod, wl)
    _check(wl, keys, tables, vout, codes, otabs, ovout, ocodes)


def test_plan_rejects_host_arrays(cuda_lib):
    import torch

    t = cuda_lib.Table(1024)
    keys = np.arange(1, 9, dtype=np.uint64)
    with pytest.raises(cuda_lib.ChtError):
        cuda_lib.Plan([(t, cuda_lib.OP_INSERT, keys, keys, None, None)])
    torch.cuda.synchronize()


def test_plan_rejects_inputs_overlapping_outputs(cuda_lib):
    import torch

    t = cuda_lib.Table(1024)
    buf = torch.arange(1, 65, dtype=torch.int64, device="cuda")
    vout = torch.zeros(32, dtype=torch.int64, device="cuda")
    # a find whose found values land where a later insert reads its keys
    with pytest.raises(cuda_lib.ChtError):
        cuda_lib.Plan([(t, cuda_lib.OP_FIND, buf[:32], None, buf[16:48], None),
                       (t, cuda_lib.OP_INSERT, buf[40:64], buf[40:64], None, None)])
    # codes inside a key array
    codes = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(cuda_lib.ChtError):
        cuda_lib.Plan([(t, cuda_lib.OP_INSERT, buf[:32], buf[:32], None, buf.view(torch.uint8)[8:40])])
    # disjoint arrays are fine
    cuda_lib.Plan([(t, cuda_lib.OP_FIND, buf[:32], None, vout, codes[:32])]).destroy()
    torch.cuda.synchronize()


@pytest.mark.parametrize("chunk,reuse", [(0, 0), (32, 0), (256, 0), (0, 1), (32, 1)])
def test_engine_chain_of_small_batches(cuda_lib, oracle_mod, chunk, reuse):
    """One table, a long chain of small dependent batches of every kind (the
    engine runs runs of one-item levels in one warp) plus a second table with
    larger batches interleaved; results and final contents vs the oracle."""
    import torch

    rng = np.random.default_rng(77)
    universe = W.uniform_keys(3000, seed=78)
    specs = []
    for i in range(400):
        t = 0 if i % 5 else 1
        n = int(rng.integers(1, 200)) if t == 0 else int(rng.integers(100, 2000))
        op = int(rng.choice([W.OP_FIND, W.OP_INSERT, W.OP_IOU_ADD, W.OP_ERASE, W.OP_UPDATE_ADD],
                            p=[0.35, 0.3, 0.15, 0.1, 0.1]))
        k = universe[rng.integers(0, universe.size, n)]
        if t == 1 and i % 3 == 0:  # the reserved keys, on the table that stores them
            k[: max(1, n // 100)] = np.uint64(0) if i % 2 else np.uint64((1 << 64) - 1)
        # an insert's value is a function of its key: whichever copy of a
        # repeated key wins, the stored value is the same
        v = k ^ np.uint64(0x5DEECE66D) if op == W.OP_INSERT else W.uniform_keys(n, seed=1000 + i)
        specs.append((t, op, k, v))
    total = sum(k.size for _, _, k, _ in specs)
    keys_d = torch.empty(total, dtype=torch.int64, device="cuda")
    vals_d = torch.empty(total, dtype=torch.int64, device="cuda")
    vout = torch.full((total,), -1, dtype=torch.int64, device="cuda")
    codes = torch.full((total,), 255, dtype=torch.uint8, device="cuda")
    # large enough never to fill (which operations fail on a full table depends
    # on their order), small enough to keep long clusters and tombstone runs
    tables = [cuda_lib.Table(1 << 14), cuda_lib.Table(1 << 14)]
    if reuse:
        tables[0].set_config(reuse_tombstones=1)  # one table with reuse, one without, in one launch
    tables[1].set_config(full_key_space=1)  # keys 0 and ~0 in its special slots
    otabs = [oracle_mod.OracleTable(1 << 14, reuse_tombstones=bool(reuse)),
             oracle_mod.OracleTable(1 << 14, full_key_space=True)]
    ops, spans, o = [], [], 0
    for t, op, k, v in specs:
        n = k.size
        keys_d[o:o + n] = torch.from_numpy(k.view(np.int64))
        vals_d[o:o + n] = torch.from_numpy(v.view(np.int64))
        ops.append((tables[t], op, keys_d[o:o + n],
                    vals_d[o:o + n] if op in (W.OP_INSERT, W.OP_IOU_ADD, W.OP_UPDATE_ADD) else None,
                    vout[o:o + n] if op == W.OP_FIND else None, codes[o:o + n]))
        spans.append((o, o + n))
        o += n
    plan = cuda_lib.Plan(ops)
    plan.set_config(chunk_ops=chunk)
    plan.launch()
    assert plan.status() == 0
    g_v, g_c = to_np_u64(vout), to_np_u8(codes)
    assert (g_c != 2).all()  # no table filled up
    for (t, op, k, v), (lo, hi) in zip(specs, spans):
        ot = otabs[t]
        if op == W.OP_FIND:
            ov, oc = ot.find(k)
            assert np.array_equal(g_v[lo:hi], ov) and np.array_equal(g_c[lo:hi], oc)
            continue
        if op == W.OP_INSERT:
            oc = ot.insert(k, v)
        elif op == W.OP_IOU_ADD:
            oc = ot.insert_or_update(k, v, oracle_mod.ADD)
        elif op == W.OP_UPDATE_ADD:
            oc = ot.update(k, v, oracle_mod.ADD)
            assert np.array_equal(g_c[lo:hi], oc)  # presence per operation is unique
            continue
        else:
            oc = ot.erase(k)
        for kk in np.unique(k):  # equal keys in one batch: which one wins is free
            m = k == kk
            assert int(g_c[lo:hi][m].astype(np.int64).sum()) == int(oc[m].astype(np.int64).sum())
    for t, ot in zip(tables, otabs):
        gk, gv = map(to_np_u64, t.export())
        ok, ov = ot.export()
        i, j = np.argsort(gk), np.argsort(ok)
        assert gk.size == ok.size and np.array_equal(gk[i], ok[j]) and np.array_equal(gv[i], ov[j])
