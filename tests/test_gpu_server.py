"""GPU tests of the serving loop: every request's result is the same when it
runs in the mix (continuous batching, concurrent steps) as when it runs alone
(one single call per request, in arrival order), and matches the oracle.

Integer results, so "the same" means bit-exact: find values and codes
exactly; insert / erase / insertOrUpdate codes per distinct key of a request
(which duplicate wins is free); final contents of every table exactly.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import to_np_u64

pytestmark = pytest.mark.gpu


def _host_requests(wl):
    keys, vals = W.serving_keys(wl)
    n = keys.size
    return keys, vals, np.zeros(n, np.uint64), np.full(n, 255, np.uint8)


def _single_calls(cuda_lib, wl, keys, vals, caps):
    import torch

    tables = [cuda_lib.Table(c, growable=True) for c in caps]
    vout = np.zeros(keys.size, np.uint64)
    codes = np.full(keys.size, 255, np.uint8)
    for r in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][r]), int(wl["offsets"][r + 1])
        t, op = tables[int(wl["table"][r])], int(wl["op"][r])
        k = keys[lo:hi]
        if op == W.OP_FIND:
            t.find(k, vout[lo:hi], codes[lo:hi])
        elif op == W.OP_INSERT:
            t.insert(k, vals[lo:hi], codes[lo:hi])
        elif op == W.OP_IOU_ADD:
            t.insert_or_update(k, vals[lo:hi], cuda_lib.ADD, codes[lo:hi])
        else:
            t.erase(k, codes[lo:hi])
        torch.cuda.synchronize()
    return tables, vout, codes


def _compare(wl, keys, a_tabs, a_vout, a_codes, b_tabs, b_vout, b_codes):
    for r in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][r]), int(wl["offsets"][r + 1])
        op = int(wl["op"][r])
        if op == W.OP_FIND:
            assert np.array_equal(a_codes[lo:hi], b_codes[lo:hi]), r
            assert np.array_equal(a_vout[lo:hi], b_vout[lo:hi]), r
        else:
            seg = keys[lo:hi]
            for k in np.unique(seg):
                m = seg == k
                assert int(a_codes[lo:hi][m].astype(int).sum()) == int(b_codes[lo:hi][m].astype(int).sum()), r
    for ta, tb in zip(a_tabs, b_tabs):
        ka, va = ta.export()
        kb, vb = tb.export()
        ka, va, kb, vb = map(to_np_u64, (ka, va, kb, vb))
        i, j = np.argsort(ka), np.argsort(kb)
        assert ka.size == kb.size and np.array_equal(ka[i], kb[j]) and np.array_equal(va[i], vb[j])


@pytest.mark.parametrize("inflight,stage", [(1, 0), (2, 0), (3, 0), (2, 1)])
def test_server_mix_equals_alone(cuda_lib, inflight, stage):
    wl = W.serving_workload(600, n_tables=12, log2_min=7, log2_max=12, size_log2_max=10, seed=41)
    caps = [64] * 12
    keys, vals, vout, codes = _host_requests(wl)
    tables = [cuda_lib.Table(c, growable=True) for c in caps]
    srv = cuda_lib.Server(tables, arena_bytes=1 << 22, max_inflight_steps=inflight, max_step_requests=64,
                          stage_inputs=stage)
    reqs = []
    for r in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][r]), int(wl["offsets"][r + 1])
        op = int(wl["op"][r])
        reqs.append(srv.request(int(wl["table"][r]), op, keys[lo:hi],
                                vals[lo:hi] if op in (W.OP_INSERT, W.OP_IOU_ADD) else None,
                                vout[lo:hi] if op == W.OP_FIND else None, codes[lo:hi]))
    arrivals = W.poisson_arrivals(len(reqs), rate_per_s=200_000.0, seed=3)
    lat, makespan = srv.replay(reqs, arrivals)
    assert (lat > 0).all() and makespan > 0
    steps, done = srv.stats()
    assert done == len(reqs) and steps >= 2
    prof = srv.profile()
    assert prof["steps"] == steps and prof["completed"] == done
    assert prof["parts"] >= len(reqs) and prof["chunks"] >= prof["parts"]
    assert steps <= prof["rounds"] <= prof["parts"]
    assert 0 < prof["engine_ms"] <= prof["gpu_step_ms"] <= makespan * 1e3
    assert prof["migrations"] > 0  # the 64-cell tables had to grow
    tr = srv.trace()
    assert tr.size == steps and int(tr["parts"].sum()) == prof["parts"] and int(tr["items"].sum()) == prof["chunks"]
    assert int(tr["rounds"].sum()) == prof["rounds"] and int(tr["migrations"].sum()) == prof["migrations"]
    assert int(tr["ops"].sum()) == int(wl["offsets"][-1])
    assert abs(float(tr["engine_ms"].sum()) - prof["engine_ms"]) < 1e-6 * max(1.0, prof["engine_ms"]) + 1e-3
    alone_tabs, a_vout, a_codes = _single_calls(cuda_lib, wl, keys, vals, caps)
    _compare(wl, keys, tables, vout, codes, alone_tabs, a_vout, a_codes)
    srv.destroy()


def test_server_matches_oracle(cuda_lib, oracle_mod):
    wl = W.serving_workload(300, n_tables=8, log2_min=7, log2_max=11, size_log2_max=9, seed=42)
    keys, vals, vout, codes = _host_requests(wl)
    tables = [cuda_lib.Table(64, growable=True) for _ in range(8)]
    srv = cuda_lib.Server(tables, arena_bytes=1 << 21)
    for r in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][r]), int(wl["offsets"][r + 1])
        op = int(wl["op"][r])
        srv.submit(int(wl["table"][r]), op, keys[lo:hi], vals[lo:hi] if op in (W.OP_INSERT, W.OP_IOU_ADD) else None,
                   vout[lo:hi] if op == W.OP_FIND else None, codes[lo:hi])
        if r % 7 == 0:
            srv.step()
    srv.drain()
    otabs = [oracle_mod.OracleTable(64, growable=True) for _ in range(8)]
    for r in range(len(wl["n"])):
        lo, hi = int(wl["offsets"][r]), int(wl["offsets"][r + 1])
        t, op, k = otabs[int(wl["table"][r])], int(wl["op"][r]), keys[lo:hi]
        if op == W.OP_FIND:
            ev, ef = t.find(k)
            assert np.array_equal(ev, vout[lo:hi]) and np.array_equal(ef, codes[lo:hi]), r
        elif op == W.OP_INSERT:
            oc = t.insert(k, vals[lo:hi])
        elif op == W.OP_IOU_ADD:
            oc = t.insert_or_update(k, vals[lo:hi], oracle_mod.ADD)
        else:
            oc = t.erase(k)
        if op != W.OP_FIND:
            for kk in np.unique(k):
                m = k == kk
                assert int(codes[lo:hi][m].astype(int).sum()) == int(oc[m].astype(int).sum()), r
    for t, o in zip(tables, otabs):
        gk, gv = map(to_np_u64, t.export())
        ok, ov = o.export()
        i, j = np.argsort(gk), np.argsort(ok)
        assert np.array_equal(gk[i], ok[j]) and np.array_equal(gv[i], ov[j])
    srv.destroy()


def test_server_grows_for_a_large_insert(cuda_lib):
    n = 20_000
    keys = W.uniform_keys(n, seed=43)
    codes = np.zeros(n, np.uint8)
    t = cuda_lib.Table(64, growable=True)
    srv = cuda_lib.Server([t], arena_bytes=1 << 20)
    rid = srv.submit(0, cuda_lib.OP_INSERT, keys, keys, None, codes)
    srv.drain()
    done, lat, st = srv.result(rid)
    assert done and st == cuda_lib.CHT_OK and lat > 0
    assert (codes == 1).all()
    live, ne, cap = t.size(check=True)
    assert live == n and cap == 1 << 16  # pre-sized once for the whole request at load 0.5
    srv.destroy()


def test_server_splits_requests_larger_than_a_step(cuda_lib):
    n = 20_000
    keys = W.uniform_keys(n, seed=45)
    codes = np.zeros(n, np.uint8)
    t = cuda_lib.Table(1 << 16)
    srv = cuda_lib.Server([t], arena_bytes=1 << 20, max_step_ops=4096, stage_inputs=1)
    rid = srv.submit(0, cuda_lib.OP_INSERT, keys, keys, None, codes)
    srv.drain()
    assert srv.result(rid)[0] and (codes == 1).all()
    assert srv.stats()[0] >= 5  # admitted in parts over several steps
    assert t.size()[0] == n
    srv.destroy()


def test_server_rejects_growth_beyond_memory_cap(cuda_lib):
    keys = W.uniform_keys(5000, seed=44)
    codes = np.zeros(5000, np.uint8)
    t = cuda_lib.Table(64, growable=True)
    srv = cuda_lib.Server([t], arena_bytes=1 << 20, memory_cap_bytes=(1 << 20) + 64 * 16 * 8)
    rid = srv.submit(0, cuda_lib.OP_INSERT, keys, keys, None, codes)
    srv.drain()
    done, _, st = srv.result(rid)
    assert done and st == cuda_lib.CHT_ERR_OOM
    srv.destroy()


def test_server_admits_growth_by_free_device_memory(cuda_lib):
    """A growth the device's free memory cannot hold (with the configured
    reserve left free) is not admitted: with nothing in flight the request is
    rejected; with a reserve that fits, the same request grows its table."""
    import torch

    keys = W.uniform_keys(5000, seed=45)
    free_now = torch.cuda.mem_get_info()[0]
    for reserve, want in ((free_now * 2, cuda_lib.CHT_ERR_OOM), (1 << 20, cuda_lib.CHT_OK)):
        codes = np.zeros(5000, np.uint8)
        t = cuda_lib.Table(64, growable=True)
        srv = cuda_lib.Server([t], arena_bytes=1 << 20, hbm_reserve_bytes=reserve)
        rid = srv.submit(0, cuda_lib.OP_INSERT, keys, keys, None, codes)
        srv.drain()
        done, _, st = srv.result(rid)
        assert done and st == want
        if want == cuda_lib.CHT_OK:
            assert (codes == 1).all() and t.size()[0] == 5000
        else:
            assert t.size()[2] == 64  # never grown
        srv.destroy()
        t.destroy()
