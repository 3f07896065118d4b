"""The many-tables workload generator (CPU): structure and key streams."""
import numpy as np

import workloads as W


def test_structure_and_rounds():
    wl = W.batched_workload(40, 6, 12, seed=21)
    n_t, cap = wl["n_t"], wl["capacity"]
    assert ((cap & (cap - 1)) == 0).all() and (cap >= 2 * n_t).all() and (cap >= 64).all()
    seen = np.zeros(40, dtype=np.int64)
    ins = np.zeros(40, dtype=np.int64)
    last_round = np.full(40, -1)
    round_idx = 0
    prev_table = -1
    for b in range(len(wl["n"])):
        t, op, n = int(wl["table"][b]), int(wl["op"][b]), int(wl["n"][b])
        if t <= prev_table:
            round_idx += 1
        prev_table = t
        assert seen[t] == round_idx  # the table's k-th batch sits in round k
        seen[t] += 1
        assert 1 <= n <= max(1, n_t[t] // 4)
        if op == W.OP_INSERT:
            assert wl["ins_before"][b] == ins[t]
            ins[t] += n
    assert (ins == n_t).all()


def test_keys_numpy_torch_agree_and_streams_are_sane():
    import torch  # noqa: F401

    wl = W.batched_workload(24, 6, 11, seed=22)
    k, v = W.batched_keys(wl)
    kt, vt = W.batched_keys(wl, backend="cpu")
    assert np.array_equal(k, kt.numpy().view(np.uint64)) and np.array_equal(v, vt.numpy().view(np.uint64))
    inserted = {}
    for b in range(len(wl["n"])):
        t, op = int(wl["table"][b]), int(wl["op"][b])
        seg = k[wl["offsets"][b]:wl["offsets"][b + 1]]
        s = inserted.setdefault(t, set())
        if op == W.OP_INSERT:
            assert not (set(seg.tolist()) & s)  # fresh keys
            s.update(seg.tolist())
    all_ins = [x for s in inserted.values() for x in s]
    assert len(all_ins) == len(set(all_ins)) == int(wl["n_t"].sum())


def test_serving_workload_recipe():
    wl = W.serving_workload(20_000, n_tables=64, log2_min=8, log2_max=12, size_log2_max=12, seed=3)
    assert (wl["n"] >= 1).all() and (wl["n"] <= 1 << 12).all()
    frac = np.bincount(wl["op"], minlength=5) / len(wl["op"])
    assert abs(frac[W.OP_FIND] - 0.5) < 0.02 and abs(frac[W.OP_INSERT] - 0.3) < 0.02
    assert abs(frac[W.OP_IOU_ADD] - 0.15) < 0.02 and abs(frac[W.OP_ERASE] - 0.05) < 0.01
    counts = np.bincount(wl["table"], minlength=64)
    assert counts[0] > counts[1] > counts[3] > counts[15]  # Zipf(1.0) over the tables
    k, _ = W.serving_keys(wl, 0, 500)
    t = np.repeat(wl["table"][:500], wl["n"][:500])
    for tt in np.unique(t)[:5]:
        assert np.unique(k[t == tt]).size <= wl["n_t"][tt]  # drawn from the table's universe
