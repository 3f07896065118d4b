"""Host arrays larger than one pipeline piece (2^24 operations): the library
copies piece i+1 in while piece i runs and piece i-1's results go back.  The
results must equal the same call on device arrays: finds, erase and update
codes bit-exact; inserts of distinct keys all 1; insertOrUpdate(add) sums and
the final key set bit-exact (the pieces of a batch are one linearization).
Sizes cover two pieces and more pieces than the three slots (slot reuse).
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_same_live_set, to_dev, to_np_u64, to_np_u8

pytestmark = pytest.mark.gpu

PIECE = 1 << 24


def _pinned(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if a.dtype == np.uint64 else a.dtype)).pin_memory()


@pytest.mark.parametrize("n", [PIECE + 12_345, 3 * PIECE + 7])
@pytest.mark.parametrize("growable", [False, True])
def test_pipelined_host_arrays_match_device_arrays(cuda_lib, oracle_mod, n, growable):
    import torch

    c = 1 << 27
    keys = W.uniform_keys(n, seed=71)
    vals = W.values_for(keys)
    th = cuda_lib.Table(1 << 12 if growable else c, growable=growable)  # host arrays
    td = cuda_lib.Table(1 << 12 if growable else c, growable=growable)  # device arrays
    hk, hv, hc = _pinned(keys), _pinned(vals), torch.full((n,), 9, dtype=torch.uint8).pin_memory()
    th.insert(hk, hv, hc)
    dc = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    td.insert(to_dev(keys), to_dev(vals), dc)
    torch.cuda.synchronize()
    assert (hc.numpy() == 1).all() and (to_np_u8(dc) == 1).all()
    assert th.size(check=True) == td.size(check=True)
    # finds: hits and misses mixed, host results vs device results
    q = np.concatenate([keys[::2], W.uniform_keys(n - keys[::2].size, start=10**9, seed=71)])
    hq, hvo, hfo = _pinned(q), torch.zeros(n, dtype=torch.int64).pin_memory(), torch.zeros(n, dtype=torch.uint8).pin_memory()
    th.find(hq, hvo, hfo)
    dvo, dfo = torch.zeros(n, dtype=torch.int64, device="cuda"), torch.zeros(n, dtype=torch.uint8, device="cuda")
    td.find(to_dev(q), dvo, dfo)
    torch.cuda.synchronize()
    assert np.array_equal(hvo.numpy(), dvo.cpu().numpy()) and np.array_equal(hfo.numpy(), dfo.cpu().numpy())
    # insertOrUpdate(add) with repeated keys: sums are order-free
    z = W.zipf_keys(n, 1.0, n_ranks=1 << 20, seed=72)
    ones = np.ones(n, np.uint64)
    th.insert_or_update(_pinned(z), _pinned(ones), cuda_lib.ADD)
    td.insert_or_update(to_dev(z), to_dev(ones), cuda_lib.ADD)
    # update and erase codes
    hu = torch.zeros(n, dtype=torch.uint8).pin_memory()
    th.update(hq, _pinned(ones), cuda_lib.ADD, hu)
    du = torch.zeros(n, dtype=torch.uint8, device="cuda")
    td.update(to_dev(q), to_dev(ones), cuda_lib.ADD, du)
    he = torch.zeros(n, dtype=torch.uint8).pin_memory()
    th.erase(hq, he)
    de = torch.zeros(n, dtype=torch.uint8, device="cuda")
    td.erase(to_dev(q), de)
    torch.cuda.synchronize()
    assert np.array_equal(hu.numpy(), du.cpu().numpy()) and np.array_equal(he.numpy(), de.cpu().numpy())
    assert th.size(check=True) == td.size(check=True)
    gk, gv = th.export()
    ok, ov = td.export()
    a, b = np.argsort(to_np_u64(gk)), np.argsort(to_np_u64(ok))
    assert np.array_equal(to_np_u64(gk)[a], to_np_u64(ok)[b]) and np.array_equal(to_np_u64(gv)[a], to_np_u64(ov)[b])
    # and the oracle agrees on the whole sequence
    o = oracle_mod.OracleTable(1 << 12 if growable else c, growable=growable, alpha=0.5)
    o.insert(keys, vals)
    o.insert_or_update(z, ones, oracle_mod.ADD)
    assert np.array_equal(o.update(q, ones, oracle_mod.ADD), hu.numpy())
    assert np.array_equal(o.erase(q), he.numpy())
    assert_same_live_set(th, o)
