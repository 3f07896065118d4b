"""Generate the automatic probe-window rule of libcht by measurement.

Runs the single-call autotuner (cht_tune: every probe window -- group width G,
cells per lane V, resident CTAs per SM -- timed with at least three trials,
median kept) on tables of 2^20, 2^24, 2^26 and 2^28 cells at loads 0.25, 0.5, 0.7
and 0.9, for find (a batch of hits and a batch of misses of c/2 operations each, at
most 2^26, ranked by the sum of the two), insert (two batches that end at the load: the fresh keys that fill
the table from the previous load level to this one, and the keys up to this
load into an empty table; ranked by the sum of the two), erase and update
(present keys), and writes

  csrc/cht_tuned.inc   the rule the runtime's automatic window choice reads:
                       per operation, table size range and load band, the
                       fastest window;
  a Markdown summary   (--summary PATH) with the best and runner-up times.

Run it on the GPU the library is tuned for, then rebuild:
    python -m paper_1601_04017_gb300.tune --summary profiles/autotune_windows.md
"""
from __future__ import annotations

import argparse
import ctypes
import os
import sys
import time


HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The library's built-in window (used where no rule applies): below load 0.6
# finds 2 lanes x 4 cells, the others 1 x 2; above it finds and inserts 4 x 4,
# the others 4 x 2 (all at the occupancy maximum).  A measured winner replaces
# it only if it is faster by more than MARGIN (timing noise of single-digit
# microsecond calls would otherwise pick windows at random).
MARGIN = 0.03


def builtin_window(op: int, load: float):
    if load < 0.6:
        return (2, 4, 0) if op == 0 else (1, 2, 0)
    return (4, 4, 0) if op in (0, 1) else (4, 2, 0)


# tuned sizes (log2 of the capacity) and the sizes each one stands for: 2^20
# cells fit the 129 MB L2, 2^24 cells (256 MB) half fit, 2^26 and 2^28 are
# HBM-resident
SIZES = (20, 24, 26, 28)
SIZE_RANGES = {20: (0, 22), 24: (23, 24), 26: (25, 26), 28: (27, 40)}
LOADS = (0.25, 0.5, 0.7, 0.9)       # tuned loads
BANDS = {0.25: (0.0, 0.375), 0.5: (0.375, 0.6), 0.7: (0.6, 0.8), 0.9: (0.8, 1.01)}
MODE_NAMES = {0: "cht::kFind", 1: "cht::kInsert", 4: "cht::kErase", 5: "cht::kUpdAdd"}


def rank_by_sum(a: dict, b: dict) -> list:
    """Windows ranked by the sum of their times on two batches (a, b: window
    (G, V, CTAs/SM) -> ms), fastest first, as (G, V, CTAs/SM, ms) rows."""
    return sorted(((w[0], w[1], w[2], a[w] + b[w]) for w in a if w in b), key=lambda r: r[3])


def choose(res: list, builtin: tuple, margin: float = MARGIN) -> tuple:
    """The rule's window: the fastest measured one if it beats the built-in
    window by more than `margin`, else the built-in one (timing noise of short
    calls would otherwise pick windows at random).  res: ranked rows."""
    best = res[0]
    base = next(r for r in res if (r[0], r[1], r[2]) == builtin)
    return best if best[3] < (1.0 - margin) * base[3] else base


def rule_line(mode_name: str, lo: int, hi: int, blo: float, bhi: float, g: int, v: int, ct: int,
              ms: float, nops: int) -> str:
    """One entry of cht_tuned.inc."""
    return f"{{{mode_name}, {lo}, {hi}, {blo:.3f}f, {bhi:.3f}f, {g}, {v}, {ct}}},  // {ms:.4f} ms for {nops} ops\n"


class TuneResult(ctypes.Structure):
    _fields_ = [("group_width", ctypes.c_int), ("lane_cells", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("ms", ctypes.c_double)]


def tune_one(lib, table, op, keys, vals, trials):
    import torch

    res = (TuneResult * 64)()
    nres = ctypes.c_uint32()
    f = lib.cht_tune
    f.restype = ctypes.c_int
    p = ctypes.c_void_p
    f.argtypes = [p, ctypes.c_int, p, p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(TuneResult), ctypes.c_uint32,
                  ctypes.POINTER(ctypes.c_uint32), p]
    st = f(table._h, op, keys.data_ptr(), vals.data_ptr() if vals is not None else None, keys.numel(), trials, res,
           64, ctypes.byref(nres), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError(f"cht_tune failed with status {st}")
    return [(r.group_width, r.lane_cells, r.ctas_per_sm, r.ms) for r in res[: nres.value]]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trials", type=int, default=3)
    ap.add_argument("--sizes", type=int, nargs="*", default=list(SIZES))
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "cht_tuned.inc"))
    ap.add_argument("--summary", default="")
    args = ap.parse_args()

    import torch

    import paper_1601_04017_gb300 as cht
    import workloads as W

    lib = cht.load_library()
    rows, summary = [], []
    t_start = time.time()
    for log2c in args.sizes:
        c = 1 << log2c
        n_max = W.load_count(c, max(LOADS))
        keys = W.uniform_keys(n_max + c // 2, backend="cuda")
        vals = W.values_for(keys, backend="cuda")
        t = cht.Table(c)
        t_empty = cht.Table(c)  # stays empty: the tuner restores it after every trial
        filled = 0
        for ld in LOADS:
            n_ld = W.load_count(c, ld)
            # the insert batches end at load `ld`: one fills the table from the
            # previous level (tuned before it is applied), one fills an empty
            # table; each window is ranked by the sum of its two times
            ins_k, ins_v = keys[filled:n_ld], vals[filled:n_ld]
            ra = {r[:3]: r[3] for r in tune_one(lib, t, 1, ins_k, ins_v, args.trials)}
            rb = {r[:3]: r[3] for r in tune_one(lib, t_empty, 1, keys[:n_ld], vals[:n_ld], args.trials)}
            res_ins = rank_by_sum(ra, rb)
            t.insert(ins_k, ins_v)
            filled = n_ld
            # find / erase / update batches of c/2 operations (at most 2^26):
            # present keys (as many as the table holds, up to that) and as
            # many absent ones -- the batch sizes the workloads use
            nq = min(c // 2, 1 << 26)
            present = keys[:filled][torch.randperm(filled, device="cuda")[:nq]]
            fresh = keys[n_max: n_max + nq]
            batches = {
                0: (torch.cat([present, fresh]), None),
                1: (ins_k, ins_v),
                4: (present, None),
                5: (present, vals[: present.numel()]),
            }
            for op, (k, v) in batches.items():
                if op == 0:
                    # finds: a batch of hits and a batch of misses, each window
                    # ranked by the sum of its two times
                    rh = {r[:3]: r[3] for r in tune_one(lib, t, 0, present, None, args.trials)}
                    rm = {r[:3]: r[3] for r in tune_one(lib, t, 0, fresh, None, args.trials)}
                    res = rank_by_sum(rh, rm)
                else:
                    res = res_ins if op == 1 else tune_one(lib, t, op, k, v, args.trials)
                base = next(r for r in res if (r[0], r[1], r[2]) == builtin_window(op, ld))
                g, vv, ct, ms = choose(res, builtin_window(op, ld))
                lo, hi = SIZE_RANGES[log2c]
                blo, bhi = BANDS[ld]
                nops = k.numel() if op != 1 else ins_k.numel() + n_ld  # (the ranked times cover both batches)
                rows.append((MODE_NAMES[op], lo, hi, blo, bhi, g, vv, ct, ms, nops))
                second = res[1] if len(res) > 1 else None
                summary.append((log2c, ld, MODE_NAMES[op], nops, res[0], second, base, (g, vv, ct)))
                torch.cuda.synchronize()
        t.destroy()
        t_empty.destroy()
        del keys, vals
        torch.cuda.empty_cache()
    with open(args.out, "w") as f:
        f.write("// Generated by paper_1601_04017_gb300/tune.py on the GPU the library was tuned for\n"
                "// (median of >= 3 trials per window).  Per operation, table size range (log2 of\n"
                "// the capacity) and load band: the fastest window (G lanes, V cells per lane,\n"
                "// resident CTAs per SM, 0 = occupancy maximum) and its time for the tuning batch.\n")
        for row in rows:
            f.write(rule_line(*row))
    if args.summary:
        with open(args.summary, "w") as f:
            f.write("# Probe-window autotuning (cht_tune) on this GPU\n\n")
            f.write("Command: `python -m paper_1601_04017_gb300.tune --summary "
                    f"{os.path.relpath(args.summary, ROOT)}` ({time.time() - t_start:.0f} s).\n"
                    "Every window: median of >= 3 trials; the table is restored between trials of a "
                    "modifying operation.  The rule it writes is `csrc/cht_tuned.inc`.\n\n")
            f.write(f"A measured window replaces the built-in one only if it is more than {MARGIN:.0%} faster.\n\n")
            f.write("| log2 c | load | op | ops | best (G, V, CTAs/SM): ms | runner-up | built-in window | rule |\n"
                    "|---|---|---|---|---|---|---|---|\n")
            for (l2, ld, m, nops, b, s2, base, pick) in summary:
                fmt = lambda r: f"({r[0]}, {r[1]}, {r[2]}): {r[3]:.4f}" if r else "-"  # noqa: E731
                f.write(f"| {l2} | {ld} | {m.split('::')[1]} | {nops} | {fmt(b)} | {fmt(s2)} | {fmt(base)} | "
                        f"{pick} |\n")
    print(f"wrote {args.out} ({len(rows)} rules)")


if __name__ == "__main__":
    main()
