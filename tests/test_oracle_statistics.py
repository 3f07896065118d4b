"""Statistical pins of the oracle's hash and home map, and of the generators.

* Linear probing with a uniform hash has expected probe counts
  (1 + 1/(1-a))/2 per successful and (1 + 1/(1-a)^2)/2 per unsuccessful
  search at load a (Knuth, TAOCP Vol. 3, Sec. 6.4; fixture in tests/golden).
  A hash or home map that clusters (a dropped mixing step, low bits used as
  the home, a wrong shift) moves these means far outside the tolerance.
* The home map's top bits are uniform (chi-square over 256 bins).
* SplitMix64 reproduces the common seed-1234567 test vector.
* The Zipf sampler's top-rank frequencies follow P(k) = k^-s / H_{N,s}
  (Sec. 7.3) within sampling error.
"""
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _read_table("knuth_linear_probing.txt"))
def test_probe_lengths_match_knuth(oracle_mod, row):
    alpha, succ, unsucc = row
    log2c = 18
    c = 1 << log2c
    n = int(alpha * c)
    ks = W.uniform_keys(n, seed=41)
    t = oracle_mod.OracleTable(c)
    t.insert(ks, ks)
    t.reset_probes()
    t.find(ks)
    mean_hit = t.probes / n
    misses = W.uniform_keys(1 << 16, start=n, seed=41)
    t.reset_probes()
    t.find(misses)
    mean_miss = t.probes / misses.size
    # finite-table means differ from the asymptotic forms by well under 5 %;
    # the unsuccessful mean at 0.9 has a heavy tail, hence the wider bound
    assert abs(mean_hit - succ) / succ < 0.05, (mean_hit, succ)
    assert abs(mean_miss - unsucc) / unsucc < (0.12 if alpha >= 0.9 else 0.05), (mean_miss, unsucc)


def test_home_top_bits_uniform(oracle_mod):
    ks = W.uniform_keys(1 << 18, seed=42)
    h = oracle_mod.homes(ks, 8).astype(np.int64)
    counts = np.bincount(h, minlength=256)
    exp = ks.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 255 degrees of freedom: mean 255, sd ~22.6; 400 is > 6 sd
    assert chi2 < 400, chi2


def test_home_of_sequential_keys_uniform(oracle_mod):
    """Consecutive integers (a structured key set) still spread evenly."""
    ks = np.arange(1, (1 << 18) + 1, dtype=np.uint64)
    h = oracle_mod.homes(ks, 8).astype(np.int64)
    counts = np.bincount(h, minlength=256)
    exp = ks.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 400, chi2


def test_hash_is_injective_on_sample(oracle_mod):
    ks = np.arange(1, (1 << 20) + 1, dtype=np.uint64)
    h = oracle_mod.hash64(ks)
    assert np.unique(h).size == ks.size


def test_splitmix64_vector():
    want = [int(r[0]) for r in _read_table_int("splitmix64_seed1234567.txt")]
    got = [int(x) for x in W.splitmix64(1234567, 5)]
    assert got == want
    assert [W.splitmix64_scalar(1234567, i) for i in range(1, 6)] == want


def _read_table_int(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(x) for x in line.split()])
    return rows


def test_uniform_keys_distinct_and_nonreserved():
    ks = W.uniform_keys(1 << 20)
    assert np.unique(ks).size == ks.size
    assert not (ks == 0).any() and not (ks == np.uint64((1 << 64) - 1)).any()


def test_permutation_is_permutation():
    p = W.permutation(100_000)
    assert np.array_equal(np.sort(p), np.arange(100_000))


@pytest.mark.parametrize("s", [0.5, 1.0, 1.25, 1.5])
def test_zipf_top_ranks(s):
    n_ranks = 1 << 20
    count = 1 << 19
    r = W.zipf_ranks(count, s, n_ranks, seed=7)
    assert r.min() >= 1 and r.max() <= n_ranks
    top = 20
    obs = np.bincount(np.minimum(r, top + 1), minlength=top + 2)[1:]
    p = W.zipf_pmf(s, n_ranks, np.arange(1, top + 1))
    exp = np.concatenate([p, [1.0 - p.sum()]]) * count
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    # 20 degrees of freedom: 60 is beyond the 1e-5 tail
    assert chi2 < 60, (s, chi2)


def test_zipf_rank_to_key_is_injective():
    ranks = np.arange(1, (1 << 20) + 1)
    ks = W.rank_to_key(ranks)
    assert np.unique(ks).size == ks.size


def test_hash_full_avalanche(oracle_mod):
    """The MurmurHash3 finalizer was designed for full avalanche: flipping any
    input bit flips every output bit with probability close to 1/2.  A dropped
    multiply or xor-shift leaves some (input, output) bit pairs far from it."""
    n = 4096
    ks = W.uniform_keys(n, seed=43)
    base = oracle_mod.hash64(ks)
    worst = 0.0
    for i in range(64):
        flipped = oracle_mod.hash64(ks ^ np.uint64(1 << i))
        diff = base ^ flipped
        bits = (diff[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)
        p = bits.mean(axis=0)
        worst = max(worst, float(np.abs(p - 0.5).max()))
    # binomial sd at n = 4096 is 0.0078; 0.05 is > 6 sd
    assert worst < 0.05, worst


# MurmurHash3's fmix64 multipliers and their published inverses modulo 2^64
# (the pair used to invert the finalizer).  The test below runs the inverse
# written with the INVERSE constants, so it does not restate the oracle's
# forward formula: a changed multiplier or shift in the oracle's hash makes
# hash(unfmix(h)) differ from h.
_FMIX_M1, _FMIX_M2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
_FMIX_INV1, _FMIX_INV2 = 0x4F74430C22A54005, 0x9CB4B2F8129337DB


def _unfmix64(h: int) -> int:
    m = (1 << 64) - 1
    x = h
    x ^= x >> 33
    x = (x * _FMIX_INV2) & m
    x ^= x >> 33
    x = (x * _FMIX_INV1) & m
    x ^= x >> 33
    return x


def test_hash_is_murmur3_fmix64_fixed_vectors(oracle_mod):
    assert (_FMIX_M1 * _FMIX_INV1) % (1 << 64) == 1
    assert (_FMIX_M2 * _FMIX_INV2) % (1 << 64) == 1
    outs = [0, 1, 2, 3, 0x8000000000000000, 0x0123456789ABCDEF, 0xFEDCBA9876543210,
            0xFFFFFFFFFFFFFFFF, 0xDEADBEEFCAFEBABE, 1 << 32, (1 << 32) - 1, 0x5555555555555555]
    ins = np.array([_unfmix64(h) for h in outs], dtype=np.uint64)
    got = oracle_mod.hash64(ins)
    assert [int(x) for x in got] == outs
    assert int(ins[0]) == 0  # the finalizer fixes 0
