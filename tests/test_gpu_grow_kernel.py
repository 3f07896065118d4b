"""In-kernel growth (Sec. 4.3.2: the operating threads migrate the table) against the oracle.

With `grow_in_kernel = 1` an insert or insertOrUpdate batch on a growable
table runs as one cooperative launch that alternates operation rounds and
cluster-wise migrations (Sec. 4.3.1) behind grid barriers.  The results must
be the host-driven policy's: the same capacity and counts as the oracle's
growing table, the same live (key, value) set, insert codes and bit-exact
sums, and the same occupied cells (for inserts without erases the occupancy of
a linear-probing table depends only on the multiset of homes, so it is unique
even though the operations of a round run concurrently).  A barrier whose wait
runs out (a block that never arrives, planted through the testing option)
ends the launch with CHT_ERR_TIMEOUT and leaves a valid table.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_one_winner, assert_same_live_set, codes_buf, to_dev, to_np_u8, to_np_u64

pytestmark = pytest.mark.gpu


def _tables(cht, oracle_mod, c0, **cfg):
    t = cht.Table(c0, growable=True)
    t.set_config(grow_in_kernel=1, **cfg)
    o = oracle_mod.OracleTable(c0, growable=True, alpha=cfg.get("alpha", 0.5))
    return t, o


@pytest.mark.parametrize("n,c0,g", [(1000, 64, 0), (300_000, 1 << 10, 0), (1_000_000, 1 << 12, 4)])
def test_in_kernel_growth_insert(cuda_lib, oracle_mod, n, c0, g):
    keys = W.uniform_keys(n, seed=81)
    vals = W.values_for(keys)
    t, o = _tables(cuda_lib, oracle_mod, c0, group_width=g)
    l0 = cuda_lib.launch_count()
    codes = codes_buf(n)
    t.insert(to_dev(keys), to_dev(vals), codes)
    launches = cuda_lib.launch_count() - l0
    oc = o.insert(keys, vals)
    assert np.array_equal(to_np_u8(codes), oc)
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    assert o.migrations >= 4 and launches == 1  # every migration inside the one launch
    gcells = to_np_u64(t.cells()).reshape(-1, 2)
    assert np.array_equal(gcells[:, 0] != 0, o.cells()[:, 0] != 0)
    assert_same_live_set(t, o)


def test_in_kernel_growth_duplicates_and_tombstones(cuda_lib, oracle_mod):
    # a table with many tombstones: the policy purges (gamma = 1) or doubles by
    # the live count; batches repeat keys and hit present ones
    base = W.uniform_keys(60_000, seed=82)
    t, o = _tables(cuda_lib, oracle_mod, 1 << 12)
    t.insert(to_dev(base[:30_000]), to_dev(base[:30_000]))
    o.insert(base[:30_000], base[:30_000])
    t.erase(to_dev(base[:25_000]))
    o.erase(base[:25_000])
    rng = np.random.default_rng(5)
    batch = base[rng.integers(0, base.size, 200_000)]
    vals = rng.integers(1, 1 << 60, batch.size).astype(np.uint64)
    codes = codes_buf(batch.size)
    live_before = set(o.export()[0].tolist())
    t.insert(to_dev(batch), to_dev(vals), codes)
    o.insert(batch, vals)
    assert_one_winner(batch, to_np_u8(codes), lambda k: k not in live_before)
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    gk, _ = t.export()
    assert set(to_np_u64(gk).tolist()) == set(o.export()[0].tolist())


@pytest.mark.parametrize("s", [0.8, 1.25])
def test_in_kernel_growth_insert_or_update_add(cuda_lib, oracle_mod, s):
    keys = W.zipf_keys(400_000, s, n_ranks=1 << 18, seed=83)
    ones = np.ones(keys.size, np.uint64)
    t, o = _tables(cuda_lib, oracle_mod, 1 << 8)
    codes = codes_buf(keys.size)
    t.insert_or_update(to_dev(keys), to_dev(ones), cuda_lib.ADD, codes)
    o.insert_or_update(keys, ones, oracle_mod.ADD)
    assert_one_winner(keys, to_np_u8(codes), lambda k: True)
    assert t.size(check=True) == (o.live, o.nonempty, o.capacity)
    assert_same_live_set(t, o)  # per-key sums: bit-exact


def test_in_kernel_growth_wait_times_out(cuda_lib, oracle_mod):
    keys = W.uniform_keys(200_000, seed=84)
    t = cuda_lib.Table(1 << 10, growable=True)
    t.set_config(grow_in_kernel=1, grow_spin_us=200, grow_fault_inject=1)
    with pytest.raises(cuda_lib.ChtError) as ei:
        t.insert(to_dev(keys), to_dev(keys))
    assert ei.value.status == cuda_lib.CHT_ERR_TIMEOUT
    # the table is valid and usable: invariants hold, a later call completes
    live, ne, cap = t.size()
    o = oracle_mod.OracleTable(64)
    o.load_cells(to_np_u64(t.cells()).reshape(-1, 2))
    o.assert_invariants()
    assert o.live == live and o.nonempty == ne and cap >= 1 << 10
    t.set_config(grow_fault_inject=0, grow_spin_us=0)
    codes = codes_buf(keys.size)
    t.insert(to_dev(keys), to_dev(keys), codes)
    assert t.size()[0] == keys.size
    assert int((to_np_u8(codes) == 1).sum()) == keys.size - live
