"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds only input generation -- no part of the hash table's own
arithmetic (no table hash, no home slot, no probing).  Both the CPU oracle and
the CUDA path are fed from here, so the two sides always see identical inputs.

Generators (published methods, written from their definitions):

* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the variant with Stafford's
  "Mix13" finalizer used by Vigna's reference C code): state_i = seed + i*G,
  G = 0x9E3779B97F4A7C15, output_i = mix13(state_i) for i = 1, 2, ...  mix13 is
  a bijection on 64-bit words and the states are distinct for 2^64 steps, so
  the outputs of one stream are pairwise distinct; mix13(0) = 0, so key 0 only
  appears where a state is 0 (never within the prefixes used here), and the
  generator asserts that neither reserved key (0, ~0) occurs.
* Zipf(s) over ranks 1..N by rejection-inversion (Hoermann & Derflinger, ACM
  TOMACS 6(3), 1996), P(k) = k^-s / H_{N,s} (the paper's Sec. 7.3 key
  distribution).  Ranks become keys through the bijection
  key = mix13(rank XOR salt), so distinct ranks give distinct, non-reserved keys.
* A random permutation of 0..n-1 is the stable argsort of the top 63 bits of a
  SplitMix64 stream (uniform because the stream values are distinct w.h.p.).

Every array-returning function takes ``backend``: ``"numpy"`` (default; uint64
arrays, exact modular arithmetic) or a torch device such as ``"cuda"`` (int64
tensors holding the same bit patterns, used to make large benchmark inputs in
HBM quickly).  The two backends agree bit for bit on the integer generators;
the Zipf sampler uses float64 transcendental functions and may differ in rare
samples between backends because library ``log``/``exp`` may round differently.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MIX_M1 = 0xBF58476D1CE4E5B9
MIX_M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1
ZIPF_SALT = 0xA5A5_5A5A_C3C3_3C3C

# Seeds of the benchmark recipe.
SEED_UNIFORM = 1
SEED_ZIPF = 2
SEED_SHUFFLE = 3
SEED_TABLES = 4


def _s64(x: int) -> int:
    """Two's-complement int64 value of a 64-bit pattern."""
    x &= MASK64
    return x - (1 << 64) if x >> 63 else x


# ----------------------------------------------------------------------------
# numpy backend (reference)
# ----------------------------------------------------------------------------
def _mix13_np(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(MIX_M1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(MIX_M2)
    z ^= z >> np.uint64(31)
    return z


def _states_np(seed: int, start: int, count: int) -> np.ndarray:
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return i * np.uint64(GOLDEN_GAMMA) + np.uint64(seed & MASK64)


# ----------------------------------------------------------------------------
# torch backend (int64 tensors with the same bit patterns)
# ----------------------------------------------------------------------------
def _torch():
    import torch

    return torch


def _lsr_t(x, s: int):
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _mix13_t(z):
    torch = _torch()
    z = z ^ _lsr_t(z, 30)
    z = z * torch.tensor(_s64(MIX_M1), dtype=torch.int64, device=z.device)
    z = z ^ _lsr_t(z, 27)
    z = z * torch.tensor(_s64(MIX_M2), dtype=torch.int64, device=z.device)
    z = z ^ _lsr_t(z, 31)
    return z


def _states_t(seed: int, start: int, count: int, device):
    torch = _torch()
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return i * _s64(GOLDEN_GAMMA) + _s64(seed)


# ----------------------------------------------------------------------------
# public generators
# ----------------------------------------------------------------------------
def splitmix64(seed: int, count: int, start: int = 0, backend="numpy"):
    """Outputs start+1 .. start+count of the SplitMix64 stream with this seed."""
    if backend == "numpy":
        return _mix13_np(_states_np(seed, start, count))
    return _mix13_t(_states_t(seed, start, count, backend))


def splitmix64_scalar(seed: int, i: int) -> int:
    """Output i (1-based) of the stream, in plain Python integers."""
    z = (seed + i * GOLDEN_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX_M1) & MASK64
    z = ((z ^ (z >> 27)) * MIX_M2) & MASK64
    return z ^ (z >> 31)


def _check_reserved(keys, backend):
    if backend == "numpy":
        bad = bool(np.any(keys == np.uint64(0)) or np.any(keys == np.uint64(MASK64)))
    else:
        bad = bool(((keys == 0) | (keys == -1)).any().item())
    if bad:
        raise ValueError("reserved key (0 or ~0) in a generated stream; pick another seed or offset")
    return keys


def uniform_keys(count: int, start: int = 0, seed: int = SEED_UNIFORM, backend="numpy"):
    """Distinct uniform non-reserved 64-bit keys: the SplitMix64 stream."""
    return _check_reserved(splitmix64(seed, count, start, backend), backend)


def values_for(keys, backend="numpy"):
    """The benchmark's values: key * 3 mod 2^64."""
    if backend == "numpy":
        with np.errstate(over="ignore"):
            return keys * np.uint64(3)
    return keys * 3


def permutation(n: int, seed: int = SEED_SHUFFLE, backend="numpy"):
    """Uniform random permutation of 0..n-1 (stable argsort of stream >> 1)."""
    if backend == "numpy":
        r = splitmix64(seed, n, 0, "numpy") >> np.uint64(1)
        return np.argsort(r.astype(np.int64), kind="stable")
    torch = _torch()
    r = _lsr_t(splitmix64(seed, n, 0, backend), 1)
    return torch.sort(r, stable=True).indices


def uniform01(count: int, seed: int, start: int = 0, backend="numpy"):
    """Doubles in [0, 1) with 53 random bits: (stream >> 11) * 2^-53."""
    z = splitmix64(seed, count, start, backend)
    if backend == "numpy":
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    torch = _torch()
    return _lsr_t(z, 11).to(torch.float64) * (1.0 / (1 << 53))


def rank_to_key(ranks, salt: int = ZIPF_SALT, backend="numpy"):
    """Bijection rank -> key = mix13(rank XOR salt); ranks < 2^62 never map to 0."""
    if backend == "numpy":
        r = np.asarray(ranks).astype(np.uint64)
        return _check_reserved(_mix13_np(r ^ np.uint64(salt)), backend)
    torch = _torch()
    r = ranks.to(torch.int64)
    return _check_reserved(_mix13_t(r ^ _s64(salt)), backend)


class _ZipfRI:
    """Rejection-inversion for Zipf(s) on 1..N (Hoermann & Derflinger 1996).

    With h(x) = x^-s and its antiderivative H(x) = (x^(1-s) - 1)/(1-s)
    (log x when s = 1), a candidate x = H^-1(u) for u uniform on
    [H(N + 1/2), H(3/2) - 1] is rounded to k = floor(x + 1/2) and accepted if
    k - x <= c0 or u >= H(k + 1/2) - h(k); c0 = 2 - H^-1(H(5/2) - h(2)).  The
    helper forms expm1(t)/t and log1p(t)/t keep s near 1 accurate.
    """

    def __init__(self, s: float, n: int):
        self.s, self.n = float(s), int(n)
        self.hx1 = self._H(1.5) - 1.0
        self.hn = self._H(self.n + 0.5)
        self.c0 = 2.0 - self._Hinv(self._H(2.5) - math.pow(2.0, -self.s))

    def _H(self, x: float) -> float:
        lx = math.log(x)
        t = (1.0 - self.s) * lx
        return (math.expm1(t) / t if abs(t) > 1e-8 else 1.0 + t / 2.0) * lx

    def _Hinv(self, y: float) -> float:
        t = max(-1.0, y * (1.0 - self.s))
        f = math.log1p(t) / t if abs(t) > 1e-8 else 1.0 - t / 2.0
        return math.exp(f * y)

    # vectorised forms (xp = numpy or torch)
    def _H_v(self, x, xp):
        lx = xp.log(x)
        t = (1.0 - self.s) * lx
        small = xp.abs(t) <= 1e-8
        tt = xp.where(small, xp.ones_like(t), t)
        f = xp.where(small, 1.0 + t / 2.0, xp.expm1(tt) / tt)
        return f * lx

    def _Hinv_v(self, y, xp):
        t = y * (1.0 - self.s)
        t = xp.clamp(t, min=-1.0) if xp.__name__ == "torch" else np.maximum(t, -1.0)
        small = xp.abs(t) <= 1e-8
        tt = xp.where(small, xp.ones_like(t), t)
        f = xp.where(small, 1.0 - t / 2.0, xp.log1p(tt) / tt)
        return xp.exp(f * y)

    def sample(self, u, xp):
        """One rejection-inversion round: (ranks, accepted mask) from uniforms u."""
        y = self.hn + u * (self.hx1 - self.hn)
        x = self._Hinv_v(y, xp)
        kf = xp.floor(x + 0.5)
        if xp.__name__ == "torch":
            kf = xp.clamp(kf, 1.0, float(self.n))
        else:
            kf = np.clip(kf, 1.0, float(self.n))
        hk = xp.exp(-self.s * xp.log(kf))
        acc = ((kf - x) <= self.c0) | (y >= self._H_v(kf + 0.5, xp) - hk)
        return kf, acc


def zipf_ranks(count: int, s: float, n_ranks: int, seed: int = SEED_ZIPF, backend="numpy"):
    """count Zipf(s) ranks in 1..n_ranks.

    Uniform j (1-based) of the seed's stream drives sample j; rejected samples
    are redrawn from later parts of the stream, in order, so the result is a
    deterministic function of (count, s, n_ranks, seed, backend).
    """
    z = _ZipfRI(s, n_ranks)
    if backend == "numpy":
        xp = np
        out = np.zeros(count, dtype=np.int64)
    else:
        xp = _torch()
        out = xp.zeros(count, dtype=xp.int64, device=backend)
    todo = xp.arange(count) if backend == "numpy" else xp.arange(count, device=backend)
    offset = 0
    rounds = 0
    while todo.shape[0] > 0:
        m = int(todo.shape[0])
        u = uniform01(m, seed, offset, backend)
        offset += m
        k, acc = z.sample(u, xp)
        if backend == "numpy":
            out[todo[acc]] = k[acc].astype(np.int64)
        else:
            out[todo[acc]] = k[acc].to(xp.int64)
        todo = todo[~acc]
        rounds += 1
        if rounds > 200:
            raise RuntimeError("zipf sampler did not converge")
    return out


def zipf_pmf(s: float, n_ranks: int, ranks) -> np.ndarray:
    """P(k) = k^-s / H_{N,s} for the given ranks (exact normalisation)."""
    ks = np.arange(1, n_ranks + 1, dtype=np.float64)
    hn = float(np.sum(ks ** -s))
    r = np.asarray(ranks, dtype=np.float64)
    return r ** -s / hn


def zipf_keys(count: int, s: float, n_ranks: int = 1 << 26, seed: int = SEED_ZIPF, backend="numpy"):
    """Zipf(s)-distributed keys over n_ranks distinct keys (rank -> key bijection)."""
    return rank_to_key(zipf_ranks(count, s, n_ranks, seed, backend), backend=backend)


# ----------------------------------------------------------------------------
# workload recipes (sizes of the paper's experiments, scaled to this table)
# ----------------------------------------------------------------------------
def load_count(capacity: int, load: float) -> int:
    """Number of keys that fill a table of `capacity` cells to `load`."""
    return int(math.floor(load * capacity))


def bounded_workload(log2_capacity: int, loads=(0.5,), n_find: int | None = None, backend="numpy"):
    """Insert / find-hit / find-miss inputs of one bounded table.

    Inserted keys are the first floor(max(loads) * c) keys of the seed-1 stream
    (values key*3); each load level's find-hit keys are n_find keys drawn from
    the keys inserted up to that level, in a seed-3 random order; the find-miss
    keys are the next n_find stream keys after all inserted ones.
    """
    c = 1 << log2_capacity
    n_max = load_count(c, max(loads))
    if n_find is None:
        n_find = load_count(c, min(loads))
    keys = uniform_keys(n_max, 0, SEED_UNIFORM, backend)
    misses = uniform_keys(n_find, n_max, SEED_UNIFORM, backend)
    hits = {}
    for ld in loads:
        n_ins = load_count(c, ld)
        perm = permutation(n_ins, SEED_SHUFFLE, backend)[:n_find]
        hits[ld] = keys[perm]
    return {
        "capacity": c,
        "keys": keys,
        "vals": values_for(keys, backend),
        "counts": {ld: load_count(c, ld) for ld in loads},
        "hits": hits,
        "misses": misses,
    }


# ----------------------------------------------------------------------------
# many tables with uneven batches (the batched-engine workload)
# ----------------------------------------------------------------------------
OP_FIND, OP_INSERT, OP_IOU_ADD = 0, 1, 2
STREAM_INSERT, STREAM_MISS, STREAM_IOU = 0, 1, 2


def _stream_salt(table, stream, seed):
    """Per (table, stream) seed of an independent SplitMix64 stream (numpy)."""
    t = np.asarray(table, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = t * np.uint64(8) + np.asarray(stream, dtype=np.uint64) + np.uint64(seed) * np.uint64(1 << 40)
    return _mix13_np(x ^ np.uint64(0x6A09E667F3BCC909))


def batched_workload(n_tables: int, log2_min: int, log2_max: int, seed: int = SEED_TABLES,
                     mix=(0.4, 0.5, 0.1)):
    """Structure of the many-tables workload (host side, numpy).

    Table t holds n_t elements, n_t log-uniform on [2^log2_min, 2^log2_max];
    its capacity is the smallest power of two >= 2 n_t (at least 64).  It gets
    a sequence of batches with sizes log-uniform on [1, n_t / 4] and types
    insert / find / insertOrUpdate(add) with probabilities `mix`, until its
    inserts reach n_t.  Inserts take fresh keys of the table's insert stream;
    each find key is, with probability 1/2, an earlier-inserted key (else a
    key of the table's miss stream); each insertOrUpdate key is an earlier key
    or a fresh key of the table's own insertOrUpdate stream, 1/2 each.
    Batches are listed round by round (round r = every table's r-th batch).
    """
    rng = np.random.default_rng(seed)
    n_t = np.floor(np.exp2(rng.uniform(log2_min, log2_max, n_tables))).astype(np.int64)
    cap = np.maximum(64, 1 << np.ceil(np.log2(2 * n_t)).astype(np.int64))
    per_table = []
    for t in range(n_tables):
        nt = int(n_t[t])
        hi = max(1.0, nt / 4.0)
        ins = miss = iou = 0
        rows = []
        while ins < nt:
            size = int(np.floor(np.exp(rng.uniform(0.0, np.log(hi + 1.0)))))
            size = max(1, min(size, int(hi)))
            r = rng.random()
            op = OP_INSERT if r < mix[0] else (OP_FIND if r < mix[0] + mix[1] else OP_IOU_ADD)
            if op == OP_INSERT:
                size = min(size, nt - ins)
            rows.append((t, op, size, ins, miss, iou))
            if op == OP_INSERT:
                ins += size
            elif op == OP_FIND:
                miss += size
            else:
                iou += size
        per_table.append(rows)
    n_rounds = max(len(r) for r in per_table)
    rows = [per_table[t][k] for k in range(n_rounds) for t in range(n_tables) if k < len(per_table[t])]
    arr = np.array(rows, dtype=np.int64).reshape(-1, 6)
    sizes = arr[:, 2]
    offsets = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return {
        "n_tables": n_tables, "n_t": n_t, "capacity": cap, "seed": seed,
        "table": arr[:, 0], "op": arr[:, 1], "n": sizes, "ins_before": arr[:, 3],
        "miss_base": arr[:, 4], "iou_base": arr[:, 5], "offsets": offsets, "rounds": n_rounds,
    }


def batched_keys(wl, first: int = 0, last: int | None = None, backend="numpy"):
    """Keys and values of batches [first, last) as flat arrays (batch b's
    operations at offsets[b] - offsets[first] ...).  Values: key * 3 for
    inserts, 1 for insertOrUpdate(add), 0 for finds.  The torch backend
    computes the same bits on the device."""
    last = len(wl["n"]) if last is None else last
    if backend != "numpy":
        return _batched_keys_t(wl, first, last, backend)
    sizes = wl["n"][first:last]
    total = int(sizes.sum())
    bid = np.repeat(np.arange(first, last, dtype=np.int64), sizes)
    k = np.arange(total, dtype=np.int64) - (wl["offsets"][bid] - wl["offsets"][first])
    table, op = wl["table"][bid], wl["op"][bid]
    ins_before = wl["ins_before"][bid]
    # per-element coin and pick from a counter-based hash of (batch, k)
    h = _mix13_np((bid.astype(np.uint64) << np.uint64(24)) ^ k.astype(np.uint64) ^ np.uint64(wl["seed"] << 56))
    coin = (h & np.uint64(1)) == 1
    pick = (h >> np.uint64(1)) % np.maximum(ins_before, 1).astype(np.uint64)
    stream = np.full(total, STREAM_INSERT, dtype=np.int64)
    j = np.zeros(total, dtype=np.int64)
    is_ins = op == OP_INSERT
    j[is_ins] = ins_before[is_ins] + k[is_ins]
    earlier = (~is_ins) & coin & (ins_before > 0)
    j[earlier] = pick[earlier].astype(np.int64)
    fresh_find = (op == OP_FIND) & ~earlier
    stream[fresh_find] = STREAM_MISS
    j[fresh_find] = wl["miss_base"][bid][fresh_find] + k[fresh_find]
    fresh_iou = (op == OP_IOU_ADD) & ~earlier
    stream[fresh_iou] = STREAM_IOU
    j[fresh_iou] = wl["iou_base"][bid][fresh_iou] + k[fresh_iou]
    salt = _stream_salt(table, stream, wl["seed"])
    with np.errstate(over="ignore"):
        keys = _mix13_np(salt + (j.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN_GAMMA))
    _check_reserved(keys, "numpy")
    vals = np.zeros(total, dtype=np.uint64)
    with np.errstate(over="ignore"):
        vals[is_ins] = keys[is_ins] * np.uint64(3)
    vals[op == OP_IOU_ADD] = 1
    return keys, vals


def _batched_keys_t(wl, first, last, device):
    torch = _torch()

    def col(name):
        return torch.from_numpy(np.ascontiguousarray(wl[name][first:last])).to(device)

    sizes = col("n")
    total = int(wl["offsets"][last] - wl["offsets"][first])
    bidl = torch.repeat_interleave(torch.arange(first, last, dtype=torch.int64, device=device), sizes)
    off = torch.from_numpy(np.ascontiguousarray(wl["offsets"][first:last] - wl["offsets"][first])).to(device)
    off = torch.repeat_interleave(off, sizes)
    k = torch.arange(total, dtype=torch.int64, device=device) - off
    del off

    def per(name):
        return torch.repeat_interleave(col(name), sizes)

    table, op, ins_before = per("table"), per("op"), per("ins_before")
    h = _mix13_t((bidl << 24) ^ k ^ _s64(wl["seed"] << 56))
    del bidl
    coin = (h & 1) == 1
    pick = _lsr_t(h, 1) % torch.clamp(ins_before, min=1)
    stream = torch.full_like(k, STREAM_INSERT)
    is_ins = op == OP_INSERT
    j = torch.where(is_ins, ins_before + k, torch.zeros_like(k))
    earlier = (~is_ins) & coin & (ins_before > 0)
    j = torch.where(earlier, pick, j)
    fresh_find = (op == OP_FIND) & ~earlier
    stream = torch.where(fresh_find, torch.full_like(k, STREAM_MISS), stream)
    j = torch.where(fresh_find, per("miss_base") + k, j)
    fresh_iou = (op == OP_IOU_ADD) & ~earlier
    stream = torch.where(fresh_iou, torch.full_like(k, STREAM_IOU), stream)
    j = torch.where(fresh_iou, per("iou_base") + k, j)
    salt = _mix13_t((table * 8 + stream + _s64(wl["seed"] << 40)) ^ _s64(0x6A09E667F3BCC909))
    keys = _mix13_t(salt + (j + 1) * _s64(GOLDEN_GAMMA))
    _check_reserved(keys, "torch")
    vals = torch.where(is_ins, keys * 3, torch.zeros_like(keys))
    vals = torch.where(op == OP_IOU_ADD, torch.ones_like(keys), vals)
    return keys, vals


# ----------------------------------------------------------------------------
# serving: requests over resident growing tables
# ----------------------------------------------------------------------------
OP_ERASE = 4
OP_UPDATE_ADD, OP_UPDATE_OVERWRITE = 5, 6  # update of present keys only (no insertion)
STREAM_UNIVERSE = 3
SEED_SERVING = 5


def serving_workload(n_requests: int, n_tables: int = 256, log2_min: int = 10, log2_max: int = 24,
                     size_log2_max: int = 16, table_s: float = 1.0, mix=(0.5, 0.3, 0.15, 0.05),
                     seed: int = SEED_SERVING):
    """Structure of the serving workload (host side, numpy).

    Table t has a key universe of n_t keys, n_t log-uniform on
    [2^log2_min, 2^log2_max] (its final size); requests pick their table by
    Zipf(table_s) over the tables (rank r -> table r-1), their size
    log-uniform on [1, 2^size_log2_max] and one operation type: find / insert /
    insertOrUpdate(add) / erase with probabilities `mix`.  Every key is drawn
    uniformly from the request's table universe, so tables never hold more
    than n_t keys and finds hit or miss depending on what is present.
    """
    rng = np.random.default_rng(seed)
    n_t = np.floor(np.exp2(rng.uniform(log2_min, log2_max, n_tables))).astype(np.int64)
    ranks = np.arange(1, n_tables + 1, dtype=np.float64)
    p = ranks ** -table_s
    p /= p.sum()
    table = rng.choice(n_tables, size=n_requests, p=p).astype(np.int64)
    size = np.floor(np.exp(rng.uniform(0.0, size_log2_max * np.log(2.0), n_requests))).astype(np.int64)
    size = np.clip(size, 1, 1 << size_log2_max)
    u = rng.random(n_requests)
    cum = np.cumsum(mix)
    op = np.where(u < cum[0], OP_FIND, np.where(u < cum[1], OP_INSERT, np.where(u < cum[2], OP_IOU_ADD, OP_ERASE)))
    offsets = np.zeros(n_requests + 1, dtype=np.int64)
    np.cumsum(size, out=offsets[1:])
    return {"n_tables": n_tables, "n_t": n_t, "table": table, "n": size, "op": op.astype(np.int64),
            "offsets": offsets, "seed": seed}


def serving_keys(wl, first: int = 0, last: int | None = None, backend="numpy"):
    """Keys and values of requests [first, last): key = universe key
    hash(request, j) mod n_t of the request's table; values: key * 3 for
    inserts, 1 for insertOrUpdate(add)."""
    last = len(wl["n"]) if last is None else last
    if backend == "numpy":
        sizes = wl["n"][first:last]
        total = int(sizes.sum())
        rid = np.repeat(np.arange(first, last, dtype=np.int64), sizes)
        j = np.arange(total, dtype=np.int64) - (wl["offsets"][rid] - wl["offsets"][first])
        t = wl["table"][rid]
        h = _mix13_np((rid.astype(np.uint64) << np.uint64(20)) ^ j.astype(np.uint64) ^ np.uint64(wl["seed"] << 58))
        idx = (h % wl["n_t"][t].astype(np.uint64)).astype(np.int64)
        salt = _stream_salt(t, np.full(total, STREAM_UNIVERSE), wl["seed"])
        with np.errstate(over="ignore"):
            keys = _mix13_np(salt + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN_GAMMA))
        _check_reserved(keys, "numpy")
        op = wl["op"][rid]
        vals = np.zeros(total, dtype=np.uint64)
        with np.errstate(over="ignore"):
            vals[op == OP_INSERT] = keys[op == OP_INSERT] * np.uint64(3)
        vals[op == OP_IOU_ADD] = 1
        return keys, vals
    torch = _torch()

    def col(name):
        return torch.from_numpy(np.ascontiguousarray(wl[name][first:last])).to(backend)

    sizes = col("n")
    total = int(wl["offsets"][last] - wl["offsets"][first])
    rid = torch.repeat_interleave(torch.arange(first, last, dtype=torch.int64, device=backend), sizes)
    off = torch.repeat_interleave(
        torch.from_numpy(np.ascontiguousarray(wl["offsets"][first:last] - wl["offsets"][first])).to(backend), sizes)
    j = torch.arange(total, dtype=torch.int64, device=backend) - off
    del off
    t = torch.repeat_interleave(col("table"), sizes)
    nt = torch.from_numpy(np.ascontiguousarray(wl["n_t"])).to(backend)[t]
    h = _mix13_t((rid << 20) ^ j ^ _s64(wl["seed"] << 58))
    # unsigned h mod n_t with int64 arithmetic: (hi * 2^32 + lo) mod n
    hi = _lsr_t(h, 32)
    lo = h & 0xFFFFFFFF
    idx = ((hi % nt) * (1 << 32) % nt + lo % nt) % nt
    salt = _mix13_t((t * 8 + STREAM_UNIVERSE + _s64(wl["seed"] << 40)) ^ _s64(0x6A09E667F3BCC909))
    keys = _mix13_t(salt + (idx + 1) * _s64(GOLDEN_GAMMA))
    _check_reserved(keys, "torch")
    op = torch.repeat_interleave(col("op"), sizes)
    vals = torch.where(op == OP_INSERT, keys * 3, torch.zeros_like(keys))
    vals = torch.where(op == OP_IOU_ADD, torch.ones_like(keys), vals)
    return keys, vals


def poisson_arrivals(n: int, rate_per_s: float, seed: int = SEED_SERVING + 1) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
