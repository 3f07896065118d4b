"""Benchmark of the batched hash-table hot path on one GB300 (or N replicas).

One step is one pass of the whole path over the 2^28-cell workload
(4 GiB table, 16-byte cells):
  create the table (zeroed) | insert 2^27 uniform keys (load 0.5) |
  find 2^27 hits + 2^27 misses | insert up to load 0.9 (241,591,910 keys) |
  find 2^27 hits + 2^27 misses | for s in {0.5, 1.0, 1.25, 1.5}: a fresh
  2^28-cell table and 2^28 insertOrUpdate(add 1) ops drawn Zipf(s) over 2^26
  keys (word count) | erase 2^27 keys | migrate the load-0.9 table to 2^29
  cells (gamma = 2) | destroy | a growable table of 2^12 cells takes the
  2^27 load-0.5 keys in one insert call, doubling 15 times at load 0.5
  (growth policy and migrations).
value = operations (inserts + finds + insertOrUpdates + erases) per second of
the whole step, migration and table creation included.  Inputs are resident
in HBM before the timed region; every input is far larger than the 129 MB L2.
`e2e` repeats the same steps through the same C ABI with pinned HOST arrays
(the library stages them to the device and copies the results back).

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload: the same recipe at 2^23 cells.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

LOG2C = 28
GROW_LOG2C0 = 12
ZIPF_S = (0.5, 1.0, 1.25, 1.5)
ZIPF_RANKS = 1 << 26
METRIC = "Mops/s for insert/find/insertOrUpdate at 1 GB300 vs random-access roofline; p50/p99"
UNIT = "Mops/s"


# ----------------------------------------------------------------------------
# roofline arithmetic (algorithmic bytes per operation)
# ----------------------------------------------------------------------------
def sectors(cells: float) -> float:
    """Expected 32-byte sectors a probe of `cells` cells from a random home touches."""
    return 1.0 + (cells - 1.0) / 2.0


def knuth_hit(a: float) -> float:
    return 0.5 * (1.0 + 1.0 / (1.0 - a))


def knuth_miss(a: float) -> float:
    return 0.5 * (1.0 + 1.0 / (1.0 - a) ** 2)


def insert_probe_cells(a0: float, a1: float) -> float:
    """Mean probe length of inserts that fill the table from load a0 to a1:
    the unsuccessful-search length averaged over the fill (Knuth)."""
    if a0 == 0.0:
        return knuth_hit(a1)
    return 0.5 * (1.0 + (1.0 / (1.0 - a1) - 1.0 / (1.0 - a0)) / (a1 - a0))


def algorithmic_bytes(kind: str, **kw) -> float:
    """Bytes one operation must move to or from HBM (32-byte sectors):
    its input/output streams plus the 32-byte sectors its probe touches
    (plus one dirty sector written back for an insert)."""
    if kind == "find_hit":
        return 8 + 8 + 1 + 32 * sectors(knuth_hit(kw["load"]))
    if kind == "find_miss":
        return 8 + 8 + 1 + 32 * sectors(knuth_miss(kw["load"]))
    if kind == "insert":
        return 16 + 1 + 32 * sectors(insert_probe_cells(kw["a0"], kw["a1"])) + 32
    if kind == "iou":
        # streams + each distinct key's cell read and written once, amortised
        return 16 + 1 + 64.0 * kw["distinct"] / kw["ops"]
    if kind == "erase":
        return 8 + 1 + 32 * sectors(knuth_hit(kw["load"])) + 32
    if kind == "migrate":
        return 16 + 16 * kw["gamma"]  # per source cell
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# clocks sampling during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = sorted(sm)[len(sm) // 2:]  # upper half: samples under load
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
def make_inputs(device: str):
    """All step inputs, generated on the device (same recipe as the tests)."""
    import torch

    c = 1 << LOG2C
    wl = W.bounded_workload(LOG2C, loads=(0.5, 0.9), n_find=1 << 27, backend=device)
    zipf = {s: W.zipf_keys(1 << 28, s, ZIPF_RANKS, W.SEED_ZIPF, backend=device) for s in ZIPF_S}
    distinct = {s: int(torch.unique(z).numel()) for s, z in zipf.items()}
    ones = torch.ones(1 << 28, dtype=torch.int64, device=device)
    torch.cuda.synchronize()
    return {"c": c, "wl": wl, "zipf": zipf, "distinct": distinct, "ones": ones}


class StepRunner:
    """Runs one step; records per-call CUDA events when asked."""

    def __init__(self, cht, inp, host: bool = False, partition: int = 0, grow_in_kernel: int = 0):
        import torch

        self.cht, self.inp, self.host = cht, inp, host
        self.tcfg = {"partition": partition}
        self.gcfg = dict(self.tcfg, grow_in_kernel=grow_in_kernel)
        self.torch = torch
        wl = inp["wl"]
        n05, n09 = wl["counts"][0.5], wl["counts"][0.9]
        self.n05, self.n09 = n05, n09
        nf = 1 << 27
        self.calls = []  # (name, fn, ops)
        dev = "cuda"
        if host:
            pin = lambda t: t.cpu().pin_memory()  # noqa: E731
            self.keys = pin(wl["keys"])
            self.vals = pin(wl["vals"])
            self.h05, self.h09, self.miss = pin(wl["hits"][0.5]), pin(wl["hits"][0.9]), pin(wl["misses"])
            self.zipf = {s: pin(z) for s, z in inp["zipf"].items()}
            self.ones = pin(inp["ones"])
            mk = lambda n, dt: torch.empty(n, dtype=dt).pin_memory()  # noqa: E731
        else:
            self.keys, self.vals = wl["keys"], wl["vals"]
            self.h05, self.h09, self.miss = wl["hits"][0.5], wl["hits"][0.9], wl["misses"]
            self.zipf, self.ones = inp["zipf"], inp["ones"]
            mk = lambda n, dt: torch.empty(n, dtype=dt, device=dev)  # noqa: E731
        self.codes = mk(1 << 28, torch.uint8)
        self.vout = mk(nf, torch.int64)
        self.ops_per_step = n09 + 4 * nf + 4 * (1 << 28) + nf + n05
        self.h2d = 8 * (2 * n09 + 4 * nf + 4 * 2 * (1 << 28) + nf + 2 * n05) if host else 0
        self.d2h = (n09 + 4 * (9 * nf) + 4 * (1 << 28) + nf + n05) if host else 0

    def step(self, events: dict | None = None):
        cht, torch = self.cht, self.torch
        s = torch.cuda.current_stream()
        n05, n09, nf = self.n05, self.n09, 1 << 27

        def timed(name, fn):
            if events is None:
                fn()
                return
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0 = time.perf_counter()
            a.record(s)
            fn()
            b.record(s)
            events.setdefault(name, []).append((a, b))
            events.setdefault("_host_ms", {}).setdefault(name, []).append((time.perf_counter() - h0) * 1e3)

        t = cht.Table(1 << LOG2C, config=self.tcfg)
        timed("insert_0.5", lambda: t.insert(self.keys[:n05], self.vals[:n05], self.codes[:n05]))
        timed("find_hit_0.5", lambda: t.find(self.h05, self.vout, self.codes[:nf]))
        timed("find_miss_0.5", lambda: t.find(self.miss, self.vout, self.codes[:nf]))
        timed("insert_0.9", lambda: t.insert(self.keys[n05:n09], self.vals[n05:n09], self.codes[: n09 - n05]))
        timed("find_hit_0.9", lambda: t.find(self.h09, self.vout, self.codes[:nf]))
        timed("find_miss_0.9", lambda: t.find(self.miss, self.vout, self.codes[:nf]))
        for sv in ZIPF_S:
            t2 = cht.Table(1 << LOG2C, config=self.tcfg)
            timed(f"iou_add_s{sv}", lambda: t2.insert_or_update(self.zipf[sv], self.ones, cht.ADD, self.codes))
            t2.destroy()
        timed("erase", lambda: t.erase(self.keys[:nf], self.codes[:nf]))
        timed("migrate_x2", lambda: t.migrate(2 << LOG2C))
        t.destroy()
        tg = cht.Table(1 << GROW_LOG2C0, growable=True, config=self.gcfg)
        timed("grow_insert", lambda: tg.insert(self.keys[:n05], self.vals[:n05], self.codes[:n05]))
        tg.destroy()


def per_op_bytes(inp):
    b = {
        "insert_0.5": algorithmic_bytes("insert", a0=0.0, a1=0.5),
        "insert_0.9": algorithmic_bytes("insert", a0=0.5, a1=0.9),
        "find_hit_0.5": algorithmic_bytes("find_hit", load=0.5),
        "find_miss_0.5": algorithmic_bytes("find_miss", load=0.5),
        "find_hit_0.9": algorithmic_bytes("find_hit", load=0.9),
        "find_miss_0.9": algorithmic_bytes("find_miss", load=0.9),
        "erase": algorithmic_bytes("erase", load=0.9),
    }
    for sv in ZIPF_S:
        b[f"iou_add_s{sv}"] = algorithmic_bytes("iou", distinct=inp["distinct"][sv], ops=1 << 28)
    # growth: the inserts (at loads 0.25..0.5) plus every doubling's migration
    # traffic (48 B per source cell, 2^12 + ... + 2^27 source cells), per insert
    n05 = inp["wl"]["counts"][0.5]
    src_cells = sum(1 << k for k in range(GROW_LOG2C0, LOG2C))
    b["grow_insert"] = algorithmic_bytes("insert", a0=0.25, a1=0.5) + 48.0 * src_cells / n05
    return b


def op_counts(inp):
    wl = inp["wl"]
    n05, n09 = wl["counts"][0.5], wl["counts"][0.9]
    nf = 1 << 27
    d = {"insert_0.5": n05, "insert_0.9": n09 - n05, "find_hit_0.5": nf, "find_miss_0.5": nf,
         "find_hit_0.9": nf, "find_miss_0.9": nf, "erase": nf, "migrate_x2": 1 << LOG2C,
         "grow_insert": n05}
    for sv in ZIPF_S:
        d[f"iou_add_s{sv}"] = 1 << 28
    return d


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_mops(ops_per_step: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput of N replicas: all ranks' operations over the
    slowest rank's time (weak scaling: every rank runs the full step)."""
    return ops_per_step * steps * world / (ms_max * 1e-3) / 1e6


def latency_percentiles(cht, inp, reps: int):
    """p50/p99 of single calls at the small (2^20-cell) workload, 2^19 ops each."""
    import torch

    wl = W.bounded_workload(20, loads=(0.5,), n_find=1 << 19, backend="cuda")
    n = wl["counts"][0.5]
    codes = torch.empty(n, dtype=torch.uint8, device="cuda")
    vout = torch.empty(n, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    out = {}
    t = cht.Table(1 << 20)
    samples = {"insert": [], "find_hit": [], "find_miss": []}
    for _ in range(reps):
        t.clear()
        for name, fn in (("insert", lambda: t.insert(wl["keys"], wl["vals"], codes)),
                         ("find_hit", lambda: t.find(wl["hits"][0.5], vout, codes)),
                         ("find_miss", lambda: t.find(wl["misses"], vout, codes))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            samples[name].append(a.elapsed_time(b))
    t.destroy()
    for k, v in samples.items():
        v = sorted(v)
        p50 = v[len(v) // 2]
        p99 = v[min(len(v) - 1, int(math.ceil(0.99 * len(v))) - 1)]
        out[k] = {"p50_ms": round(p50, 5), "p99_ms": round(p99, 5), "mean_ms": round(statistics.mean(v), 5),
                  "reps": len(v), "mops_at_p50": round(n / (p50 * 1e-3) / 1e6, 1)}
    # The same calls back to back (the host enqueues ahead of the GPU, so the
    # host-side cost of a call is hidden) and replayed from a CUDA graph (no
    # host work at all: the device time of a call).  As in the single calls,
    # the finds read one table, which stays in L2 (16 MiB); each insert fills
    # a table just cleared (the clear's memset is timed alone and subtracted).
    # frac_of_roofline: algorithmic bytes at load 0.5 over the measured copy
    # bandwidth.
    R = 32
    peak = load_peaks()[0]
    t1 = cht.Table(1 << 20)
    t1.insert(wl["keys"], wl["vals"], codes)
    t2 = cht.Table(1 << 20)
    torch.cuda.synchronize()

    def timed_calls(calls, graph):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if not graph:
            torch.cuda.synchronize()
            a.record(s)
            for fn in calls:
                fn()
            b.record(s)
            b.synchronize()
            return a.elapsed_time(b) / len(calls)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for fn in calls:
                fn()
        g.replay()
        torch.cuda.synchronize()
        a.record(s)
        g.replay()
        b.record(s)
        b.synchronize()
        del g
        return a.elapsed_time(b) / len(calls)

    def ins():
        t2.clear()
        t2.insert(wl["keys"], wl["vals"], codes)

    for name, bpo, call, base in (("insert", 89.0, ins, t2.clear),
                                  ("find_hit", 57.0, lambda: t1.find(wl["hits"][0.5], vout, codes), None),
                                  ("find_miss", 73.0, lambda: t1.find(wl["misses"], vout, codes), None)):
        for kind, graph in (("back_to_back", False), ("graph", True)):
            per_ms = timed_calls([call] * R, graph)
            if base is not None:
                per_ms -= timed_calls([base] * R, graph)
            mops = n / (per_ms * 1e-3) / 1e6
            out[f"{name}_{kind}"] = {"ms_per_call": round(per_ms, 5), "mops": round(mops, 1),
                                     "frac_of_roofline": round(mops * 1e6 * bpo / (peak * 1e9), 4)}
    t1.destroy()
    t2.destroy()
    return out


# Which kernel runs each timed call of the step (the automatic probe windows:
# op_kernel<G lanes, V cells per lane, mode>).  The growing insert mixes
# inserts and migrations and is left out of the per-kernel figures.
CALL_KERNEL = {
    "insert_0.5": "op_kernel<1,2,insert>",
    "find_hit_0.5": "op_kernel<2,4,find>", "find_miss_0.5": "op_kernel<2,4,find>",
    "insert_0.9": "op_kernel<4,4,insert>",
    "find_hit_0.9": "op_kernel<4,4,find>", "find_miss_0.9": "op_kernel<4,4,find>",
    "erase": "op_kernel<4,2,erase>",
    "migrate_x2": "migrate_window_kernel",
    **{f"iou_add_s{sv}": "iou_agg_kernel<insertOrUpdate add>" for sv in ZIPF_S},
}


def kernel_rooflines(breakdown, counts, bpo, peak, peak_kind):
    """Per kernel: algorithmic bytes of all its calls in a step over their
    summed CUDA-event time (= bytes per launch / mean launch time).  The
    dominant kernel is the one with the largest summed time; the others are
    listed after it."""
    fam = {}
    for name, row in breakdown.items():
        k = CALL_KERNEL.get(name)
        if k is None:
            continue
        if name == "migrate_x2":
            b = algorithmic_bytes("migrate", gamma=2) * counts[name]
        else:
            b = bpo[name] * counts[name]
        f = fam.setdefault(k, {"ms": 0.0, "bytes": 0.0, "calls": []})
        f["ms"] += row["ms"]
        f["bytes"] += b
        f["calls"].append(name)
    rows = []
    for k, f in fam.items():
        gbs = f["bytes"] / (f["ms"] * 1e-3) / 1e9
        rows.append({"bound": "hbm", "kernel": k, "calls": f["calls"], "launches_per_step": len(f["calls"]),
                     "ms_per_step": round(f["ms"], 4), "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "peak_source": peak_kind,
                     "bytes_per_launch": round(f["bytes"] / len(f["calls"]))})
    rows.sort(key=lambda r: -r["ms_per_step"])
    dom = dict(rows[0])
    # DRAM bytes per launch from ncu captures of the current kernel
    # (profiles/traffic.json, how they were taken is recorded beside them)
    dom["traffic"] = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f).get(dom["kernel"])
        if tr:
            dom["traffic"] = tr["traffic_bytes_per_launch"]
            dom["traffic_over_algorithmic"] = round(tr["traffic_bytes_per_launch"] / dom["bytes_per_launch"], 2)
    except (OSError, ValueError, KeyError):
        pass
    return dom, rows[1:]


# The ceiling of random modifications of 16-byte cells on this GPU (a random
# line read and a dirty sector written back per operation), measured by
# `python bench.py --probe-random-access --probe-out profiles/ceilings.json`:
# the modifying calls whose operations nearly all reach the table, against it.
MODIFY_CEILING = {"insert_0.5": "random_cas16_g_per_s", "erase": "random_fetch_add_g_per_s",
                  "iou_add_s0.5": "random_fetch_add_g_per_s"}


def random_modify_context(breakdown, counts):
    try:
        with open(os.path.join(ROOT, "profiles", "ceilings.json")) as f:
            ceil = json.load(f)
    except (OSError, ValueError):
        return None
    out = {"source": "profiles/ceilings.json (" + ceil.get("how", "") + ")"}
    for name, key in MODIFY_CEILING.items():
        row = breakdown.get(name)
        c = ceil.get(key)
        if not row or not c:
            continue
        g = counts[name] / (row["ms"] * 1e-3) / 1e9
        out[name] = {"g_ops_per_s": round(g, 2), "ceiling_g_per_s": c, "ceiling": key, "frac": round(g / c, 3)}
    return out


def load_half_fractions(breakdown, peak):
    """The load-0.5 figures the project aims at (>= 0.5 of the random-access
    roofline for find and insert): the 2^28-cell step's calls and, when
    measured, the 2^20-cell calls replayed from a CUDA graph."""
    out = {"goal_frac": 0.5, "peak": peak, "unit": "GB/s"}
    for name in ("insert_0.5", "find_hit_0.5", "find_miss_0.5"):
        row = breakdown.get(name)
        if row and "gbs" in row:
            out[f"2p28_{name}"] = round(row["gbs"] / peak, 4)
    return out


def pinned_copy_gbs(nbytes: int = 1 << 32) -> dict:
    """Plain cudaMemcpyAsync bandwidth between pinned host memory and the
    device on this machine (one 4 GiB copy each way, after one warm-up)."""
    import torch

    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    out = {}
    for name, dst, src in (("h2d", d, h), ("d2h", h, d)):
        dst.copy_(src, non_blocking=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        dst.copy_(src, non_blocking=True)
        b.record(s)
        b.synchronize()
        out[name] = round(nbytes / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    # both directions at once (half of the buffers each way, two streams): the
    # link's shared ceiling, which the pipelined calls' copies run against
    half = nbytes // 2
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    s_in.wait_event(a)
    s_out.wait_event(a)
    with torch.cuda.stream(s_in):
        d[:half].copy_(h[:half], non_blocking=True)
    with torch.cuda.stream(s_out):
        h[half:].copy_(d[half:], non_blocking=True)
    s.wait_stream(s_in)
    s.wait_stream(s_out)
    b.record(s)
    b.synchronize()
    out["both_total"] = round(nbytes / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    del h, d
    return out


def side_workloads(args) -> dict:
    """Small runs of the batched and serving workloads beside the step, so one
    bench line carries their evidence: 256 tables in one engine launch against
    one launch per batch (sampled tables checked against the oracle), and 10^4
    served requests with p50 / p99 at Poisson arrivals of half the capacity,
    against the same requests as single calls (results compared).  Outside
    the timed region; the full-size runs are `--workload batched|serving`."""
    import copy

    out = {}
    b = copy.copy(args)
    b.batched_tables, b.batched_log2_min, b.batched_log2_max = 256, 8, 20
    b.steps, b.warmup, b.batched_verify = 2, 1, 4
    b.batched_engine_only, b.no_graph_baseline = False, True
    r = run_batched(b)
    out["batched_256_tables"] = {
        "tables": r["tables"], "batches": r["batches"], "ops": r["ops"],
        "engine_ms": r["engine"]["ms"], "engine_mops": r["engine"]["mops"],
        "per_call_ms": r["per_call"]["ms"], "per_call_mops": r["per_call"]["mops"],
        "engine_over_per_call": round(r["per_call"]["ms"] / r["engine"]["ms"], 1),
        "verified_tables": r["verified_tables"]}
    v = copy.copy(args)
    v.serving_requests, v.serving_arrays, v.serving_loads, v.serving_baseline_loads = 10_000, "device", [0.5], [0.5]
    v.no_serving_baseline, v.serving_trace = False, ""
    r = run_serving(v)
    sc = r["single_calls"]
    out["serving_1e4_requests"] = {
        "requests": r["requests"], "ops": r["ops"],
        "served": {"capacity_mops": r["capacity"]["mops"], "capacity_requests_per_s": r["capacity"]["requests_per_s"],
                   "p50_ms_at_0.5": r["load_0.5"]["p50_ms"], "p99_ms_at_0.5": r["load_0.5"]["p99_ms"]},
        "single_calls": {"capacity_mops": sc["capacity"]["mops"],
                         "capacity_requests_per_s": sc["capacity"]["requests_per_s"],
                         "p50_ms_at_0.5": sc["load_0.5"]["p50_ms"], "p99_ms_at_0.5": sc["load_0.5"]["p99_ms"]},
        "results_equal": sc["results_equal_served"]}
    return out


def run_gpu(args):
    import torch

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_1601_04017_gb300 as cht

    cht.load_library()
    inp = make_inputs("cuda")
    pmode = {"off": 0, "on": 1}[args.partition]
    gk = {"off": 0, "on": 1}[args.grow_in_kernel]
    runner = StepRunner(cht, inp, partition=pmode, grow_in_kernel=gk)
    for _ in range(args.warmup):
        runner.step()
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = cht.launch_count()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    events: dict = {}
    e0.record(s)
    for _ in range(args.steps):
        runner.step(events)
    e1.record(s)
    torch.cuda.synchronize()
    launches = cht.launch_count() - l0
    barrier(pg)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(pg, ms, device="cuda")
    ms_step = ms_max / args.steps
    value = aggregate_mops(runner.ops_per_step, args.steps, world, ms_max)

    # per-call breakdown and the dominant kernel's roofline
    counts = op_counts(inp)
    bpo = per_op_bytes(inp)
    peak, peak_kind = load_peaks()
    events.pop("_host_ms", None)
    breakdown = {}
    for name, evs in events.items():
        t_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        row = {"ms": round(t_ms, 4), "mops": round(counts[name] / (t_ms * 1e-3) / 1e6, 1)}
        if name in bpo:
            gbs = bpo[name] * counts[name] / (t_ms * 1e-3) / 1e9
            row.update({"bytes_per_op": round(bpo[name], 2), "gbs": round(gbs, 1),
                        "frac_of_" + peak_kind: round(gbs / peak, 4)})
        elif name == "migrate_x2":
            gbs = algorithmic_bytes("migrate", gamma=2) * counts[name] / (t_ms * 1e-3) / 1e9
            row.update({"bytes_per_src_cell": 48, "gbs": round(gbs, 1),
                        "frac_of_" + peak_kind: round(gbs / peak, 4)})
        breakdown[name] = row
    roofline, roofline_others = kernel_rooflines(breakdown, counts, bpo, peak, peak_kind)
    modify_ctx = random_modify_context(breakdown, counts)
    if modify_ctx and "iou_add_s0.5" in modify_ctx and roofline["kernel"].startswith("iou_agg"):
        # the dominant kernel's low-skew call against the random-modify ceiling
        roofline["random_modify"] = dict(modify_ctx["iou_add_s0.5"], call="iou_add_s0.5")
    target = load_half_fractions(breakdown, peak)

    # end-to-end through the same API with pinned host arrays
    e2e = None
    if not args.no_e2e:
        hrunner = StepRunner(cht, inp, host=True, partition=pmode, grow_in_kernel=gk)
        hrunner.step()
        torch.cuda.synchronize()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(max(1, args.e2e_steps)):
            hrunner.step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        # one more step with CUDA events around each call (not part of the timing)
        hev: dict = {}
        hrunner.step(hev)
        torch.cuda.synchronize()
        host_ms = hev.pop("_host_ms", {})
        e2e_calls = {k: round(statistics.mean(a.elapsed_time(b) for a, b in v), 3) for k, v in hev.items()}
        e2e_host = {k: round(statistics.mean(v), 3) for k, v in host_ms.items()}
        el = max_over_ranks(pg, el, device="cuda")
        e2e = {"value": round(hrunner.ops_per_step * max(1, args.e2e_steps) * world / el / 1e6, 1),
               "unit": UNIT, "h2d_bytes_per_step": hrunner.h2d, "d2h_bytes_per_step": hrunner.d2h,
               "steps": max(1, args.e2e_steps), "pinned_copy_gbs": pinned_copy_gbs(), "calls_ms": e2e_calls,
               "calls_host_ms": e2e_host}
        del hrunner

    lat = latency_percentiles(cht, inp, args.latency_reps) if args.latency_reps > 0 else None
    if lat:
        for name in ("insert", "find_hit", "find_miss"):
            g = lat.get(f"{name}_graph")
            if g:
                target[f"2p20_{name}_graph"] = g["frac_of_roofline"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_once()
    side = None
    ops_step = runner.ops_per_step
    if rank == 0 and world == 1 and not args.no_side_workloads:
        del runner, inp
        torch.cuda.empty_cache()
        side = side_workloads(args)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (SplitMix64 uniform keys, Zipf rejection-inversion; generated on device)",
            "config": {"workload": "bounded table 2^28 cells: insert to load 0.5/0.9, find 2^27 hits + "
                                   "2^27 misses at each load, insertOrUpdate(add 1) 2^28 Zipf ops over "
                                   "2^26 keys for s in {0.5,1.0,1.25,1.5}, erase 2^27, migrate x2; "
                                   "growable table 2^12 cells taking 2^27 inserts (15 doublings)",
                       "capacity_cells": 1 << LOG2C, "ops_per_step": ops_step,
                       "partition": args.partition, "grow_in_kernel": args.grow_in_kernel,
                       "l2": "inputs and table far larger than L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "probe_window": "auto (the autotuned rule): at 2^28 cells finds 2 lanes x 64 B at "
                                       "load 0.5 and 4 x 64 B at 0.9, inserts 1 x 32 B below 0.6 and "
                                       "4 x 64 B at 0.9"},
            "roofline": roofline, "roofline_other_kernels": roofline_others, "target": target,
            "random_modify_ceiling": modify_ctx,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "breakdown": breakdown, "latency_config1": lat, "side_workloads": side,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


# ----------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ----------------------------------------------------------------------------
CPU_LOG2C = 23
CPU_BASELINE_MIN_S = 10.0  # the cpu_baseline leg repeats the sample step for at least this long


def cpu_sample_step(oracle, inp) -> tuple[int, float]:
    """The bench step's recipe on a 2^23-cell oracle table; (ops, seconds)."""
    wl = inp["wl"]
    n05, n09 = wl["counts"][0.5], wl["counts"][0.9]
    ops = 0
    t0 = time.perf_counter()
    t = oracle.OracleTable(1 << CPU_LOG2C)
    t.insert(wl["keys"][:n05], wl["vals"][:n05])
    t.find(wl["hits"][0.5])
    t.find(wl["misses"])
    t.insert(wl["keys"][n05:n09], wl["vals"][n05:n09])
    t.find(wl["hits"][0.9])
    t.find(wl["misses"])
    nf = wl["misses"].size
    ops += n09 + 4 * nf
    for sv in ZIPF_S:
        t2 = oracle.OracleTable(1 << CPU_LOG2C)
        z = inp["zipf"][sv]
        t2.insert_or_update(z, np.ones(z.size, np.uint64), oracle.ADD)
        ops += z.size
        t2.close()
    t.erase(wl["keys"][:nf])
    ops += nf
    t.migrate(2 << CPU_LOG2C)
    t.close()
    tg = oracle.OracleTable(1 << 12, growable=True, alpha=0.5)
    tg.insert(wl["keys"][:n05], wl["vals"][:n05])
    ops += n05
    tg.close()
    return ops, time.perf_counter() - t0


def cpu_inputs():
    wl = W.bounded_workload(CPU_LOG2C, loads=(0.5, 0.9), n_find=1 << (CPU_LOG2C - 1))
    zipf = {s: W.zipf_keys(1 << CPU_LOG2C, s, ZIPF_RANKS >> 6, W.SEED_ZIPF) for s in ZIPF_S}
    return {"wl": wl, "zipf": zipf}


SAMPLE_DESC = ("the same step recipe at 2^23 cells: insert to load 0.5/0.9, 2^22 find hits + misses at "
               "each load, 2^23 Zipf insertOrUpdate(add) per s over 2^20 keys, erase 2^22, migrate x2, "
               "growable 2^12-cell table taking 2^22 inserts")


def host_cpu() -> dict:
    """CPU model and logical core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


class PinnedToOneCore:
    """Run the enclosed block with this process pinned to one core (the lowest
    it may use), like `taskset -c <core>`; the oracle is single-threaded and
    runs in this process.  The previous affinity is restored afterwards."""

    def __enter__(self):
        self.prev = None
        self.core = None
        if hasattr(os, "sched_getaffinity"):
            try:
                self.prev = os.sched_getaffinity(0)
                self.core = min(self.prev)
                os.sched_setaffinity(0, {self.core})
            except OSError:
                self.prev = None
        return self

    def __exit__(self, *exc):
        if self.prev is not None:
            os.sched_setaffinity(0, self.prev)


def cpu_baseline_once():
    import oracle

    oracle.build()
    inp = cpu_inputs()
    ops, sec, reps = 0, 0.0, 0
    with PinnedToOneCore() as pin:
        while sec < CPU_BASELINE_MIN_S and reps < 20:
            o, t = cpu_sample_step(oracle, inp)
            ops, sec, reps = ops + o, sec + t, reps + 1
    return {"value": round(ops / sec / 1e6, 2), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} x " + SAMPLE_DESC, "seconds": round(sec, 2), "pinned_core": pin.core,
            "compiler": "gcc -O3", **host_cpu()}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    inp = cpu_inputs()
    tot_ops, tot_s, per = 0, 0.0, []
    with PinnedToOneCore() as pin:
        for _ in range(args.warmup):
            cpu_sample_step(oracle, inp)
        for _ in range(args.steps):
            ops, sec = cpu_sample_step(oracle, inp)
            tot_ops += ops
            tot_s += sec
            per.append(sec)
    value = tot_ops / tot_s / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_s / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": SAMPLE_DESC, "capacity_cells": 1 << CPU_LOG2C},
        "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": SAMPLE_DESC, "pinned_core": pin.core, "compiler": "gcc -O3", **host_cpu()},
        "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# many tables, uneven batches: one persistent launch vs one launch per batch
# ----------------------------------------------------------------------------
def run_batched(args):
    """4096 tables (n_t log-uniform 2^8..2^20, capacity pow2 >= 2 n_t), each
    with a sequence of batches (sizes log-uniform 1..n_t/4; insert / find /
    insertOrUpdate(add) 40/50/10, uniform keys) until its inserts reach n_t:
    the whole workload as one engine plan (one kernel launch, autotuned) vs
    the same batches as one single call (one launch) each, eager and
    captured in a CUDA graph.  Sampled tables are checked against the oracle."""
    import torch

    import paper_1601_04017_gb300 as cht

    cht.load_library()
    n_tables, lo, hi = args.batched_tables, args.batched_log2_min, args.batched_log2_max
    wl = W.batched_workload(n_tables, lo, hi, seed=W.SEED_TABLES)
    total = int(wl["offsets"][-1])
    keys = torch.empty(total, dtype=torch.int64, device="cuda")
    vals = torch.empty(total, dtype=torch.int64, device="cuda")
    b0 = 0
    nb = len(wl["n"])
    while b0 < nb:  # generate in pieces of about 2^27 operations
        b1 = int(np.searchsorted(wl["offsets"], wl["offsets"][b0] + (1 << 27), side="right")) - 1
        b1 = min(max(b1, b0 + 1), nb)
        k, v = W.batched_keys(wl, b0, b1, backend="cuda")
        keys[wl["offsets"][b0]:wl["offsets"][b1]] = k
        vals[wl["offsets"][b0]:wl["offsets"][b1]] = v
        del k, v
        b0 = b1
    vout = torch.zeros(total, dtype=torch.int64, device="cuda")
    codes = torch.zeros(total, dtype=torch.uint8, device="cuda")
    tables = [cht.Table(int(c)) for c in wl["capacity"]]
    segs = []
    for b in range(nb):
        o0, o1 = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
        op = int(wl["op"][b])
        segs.append((tables[int(wl["table"][b])], op, keys[o0:o1], vals[o0:o1] if op != W.OP_FIND else None,
                     vout[o0:o1] if op == W.OP_FIND else None, codes[o0:o1]))
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()

    def clear_all():
        for t in tables:
            t.clear()
        torch.cuda.synchronize()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b)

    def per_call():
        for (t, op, k, v, vo, c) in segs:
            if op == W.OP_FIND:
                t.find(k, vo, c)
            elif op == W.OP_INSERT:
                t.insert(k, v, c)
            else:
                t.insert_or_update(k, v, cht.ADD, c)

    t0 = time.perf_counter()
    plan = cht.Plan(segs)
    plan_build_s = time.perf_counter() - t0
    tuned_ms = plan.autotune()
    cfg = plan.config()
    eng = []
    for _ in range(args.warmup + args.steps):
        clear_all()
        eng.append(timed(plan.launch))
        assert plan.status() == 0, "engine dependency wait ran out"
    eng = eng[args.warmup:]
    # sampled tables against the oracle (the whole plan's results)
    verified = verify_batched_sample(wl, tables, keys, vout, codes, args.batched_verify)
    percall = []
    for _ in range(0 if args.batched_engine_only else max(1, min(args.steps, 2))):
        clear_all()
        percall.append(timed(per_call))
    graph_ms = None
    if not args.no_graph_baseline and not args.batched_engine_only:
        try:
            clear_all()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                per_call()
            clear_all()
            graph_ms = timed(g.replay)
            del g
        except Exception as exc:  # the capture may not fit; report why
            graph_ms = f"not measured: {type(exc).__name__}"
    ms = statistics.median(eng)
    line = {
        "workload": f"batched: {n_tables} tables, n_t log-uniform 2^{lo}..2^{hi}, capacity pow2 >= 2 n_t, "
                    "batches log-uniform 1..n_t/4, insert/find/insertOrUpdate(add) 40/50/10, uniform keys",
        "tables": n_tables, "batches": nb, "ops": total, "rounds": int(wl["rounds"]),
        "table_bytes": int(wl["capacity"].sum()) * 16,
        "engine": {"ms": round(ms, 3), "mops": round(total / (ms * 1e-3) / 1e6, 1), "launches_per_run": 1,
                   "autotuned": cfg, "autotune_best_ms": round(tuned_ms, 3), "plan_build_s": round(plan_build_s, 2)},
        "per_call": None if not percall else
                    {"ms": round(statistics.median(percall), 3),
                     "mops": round(total / (statistics.median(percall) * 1e-3) / 1e6, 1), "launches_per_run": nb},
        "per_call_graph": (graph_ms if not isinstance(graph_ms, float) else
                           {"ms": round(graph_ms, 3), "mops": round(total / (graph_ms * 1e-3) / 1e6, 1)}),
        "verified_tables": verified, "steps": args.steps, "warmup": args.warmup,
    }
    return line


def verify_batched_sample(wl, tables, keys, vout, codes, n_sample):
    """Run the oracle on a sample of tables (every batch of each, in order) and
    compare find results and final contents with the engine's run."""
    import oracle

    oracle.build()
    if n_sample <= 0:
        return 0
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(wl["n_tables"], size=min(n_sample, wl["n_tables"]), replace=False).tolist())
    g_codes = codes.cpu().numpy()
    checked = 0
    for t in pick:
        bs = np.nonzero(wl["table"] == t)[0]
        ot = oracle.OracleTable(int(wl["capacity"][t]))
        for b in bs:
            o0, o1 = int(wl["offsets"][b]), int(wl["offsets"][b + 1])
            k = keys[o0:o1].cpu().numpy().view(np.uint64)
            op = int(wl["op"][b])
            if op == W.OP_FIND:
                ev, ef = ot.find(k)
                gv = vout[o0:o1].cpu().numpy().view(np.uint64)
                if not (np.array_equal(ev, gv) and np.array_equal(ef, g_codes[o0:o1])):
                    raise AssertionError(f"table {t} batch {b}: find results differ from the oracle")
            elif op == W.OP_INSERT:
                v = k * np.uint64(3)
                if not np.array_equal(ot.insert(k, v), g_codes[o0:o1]):
                    raise AssertionError(f"table {t} batch {b}: insert codes differ from the oracle")
            else:
                ot.insert_or_update(k, np.ones(k.size, np.uint64), oracle.ADD)
        gk, gv = tables[t].export()
        gk, gv = gk.cpu().numpy().view(np.uint64), gv.cpu().numpy().view(np.uint64)
        ok, ov = ot.export()
        i, j = np.argsort(gk), np.argsort(ok)
        if not (np.array_equal(gk[i], ok[j]) and np.array_equal(gv[i], ov[j])):
            raise AssertionError(f"table {t}: final contents differ from the oracle")
        ot.close()
        checked += 1
    return checked


# ----------------------------------------------------------------------------
# serving: Poisson requests over resident growing tables
# ----------------------------------------------------------------------------
def run_serving(args):
    """256 growable tables (start 1024 cells; key universes log-uniform
    2^10..2^24), requests of 1..65536 ops (log-uniform), table ~ Zipf(1.0),
    find / insert / insertOrUpdate(add) / erase 50/30/15/5, request arrays in
    pinned host memory, device memory cap 64 GiB.  First the capacity (all
    requests at time 0), then Poisson arrivals at 0.5 / 0.7 / 0.9 of it:
    p50 / p99 request latency (arrival to completion) and throughput."""
    import torch

    import paper_1601_04017_gb300 as cht

    cht.load_library()
    nreq = args.serving_requests
    wl = W.serving_workload(nreq, n_tables=256, log2_min=10, log2_max=24, size_log2_max=16, table_s=1.0,
                            mix=tuple(args.serving_mix))
    total = int(wl["offsets"][-1])
    on_dev = args.serving_arrays == "device"

    def buf(dtype):
        return torch.zeros(total, dtype=dtype, device="cuda") if on_dev else \
            torch.zeros(total, dtype=dtype).pin_memory()

    keys_h, vals_h, vout_h, codes_h = buf(torch.int64), buf(torch.int64), buf(torch.int64), buf(torch.uint8)
    r0 = 0
    while r0 < nreq:
        r1 = int(np.searchsorted(wl["offsets"], wl["offsets"][r0] + (1 << 27), side="right")) - 1
        r1 = min(max(r1, r0 + 1), nreq)
        k, v = W.serving_keys(wl, r0, r1, backend="cuda")
        keys_h[wl["offsets"][r0]:wl["offsets"][r1]].copy_(k)
        vals_h[wl["offsets"][r0]:wl["offsets"][r1]].copy_(v)
        del k, v
        r0 = r1
    torch.cuda.synchronize()
    kp, vp, op_, cp = keys_h.data_ptr(), vals_h.data_ptr(), vout_h.data_ptr(), codes_h.data_ptr()
    reqs = []
    for r in range(nreq):
        o, n, op = int(wl["offsets"][r]), int(wl["n"][r]), int(wl["op"][r])
        reqs.append(cht.cht.Request(int(wl["table"][r]), op, kp + 8 * o,
                                    vp + 8 * o if op in (W.OP_INSERT, W.OP_IOU_ADD) else None, n,
                                    op_ + 8 * o if op == W.OP_FIND else None, cp + o))

    def fresh_tables():
        tables = [cht.Table(1024, growable=True) for _ in range(256)]
        for t in tables:
            t.set_config(reuse_tombstones=args.serving_reuse_tombstones)
        return tables

    def contents(tables):
        out = []
        for t in tables:
            k, v = t.export()
            k, v = k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint64)
            o = np.argsort(k)
            out.append((k[o], v[o]))
        return out

    def run(arrivals, keep=False):
        tables = fresh_tables()
        srv = cht.Server(tables, memory_cap_bytes=64 << 30, arena_bytes=1 << 30, max_inflight_steps=2,
                         stage_inputs=args.serving_stage_inputs)
        lat, mk = srv.replay(reqs, arrivals)
        steps, done = srv.stats()
        prof = srv.profile()
        prof["trace"] = srv.trace()
        grown = sum(t.size()[2] for t in tables) * 16
        srv.destroy()
        if keep:
            prof["contents"] = contents(tables)
        for t in tables:
            t.destroy()
        torch.cuda.synchronize()
        return lat, mk, steps, done, grown, prof

    # The baseline: the same requests as single calls (one cht_* call per
    # request, in arrival order, each waiting for its arrival time), results in
    # their own arrays.  Latency = completion (a CUDA event after the call)
    # minus arrival.
    base_vout, base_codes = buf(torch.int64), buf(torch.uint8)
    s_cur = torch.cuda.current_stream()

    def single_calls(arrivals):
        tables = fresh_tables()
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nreq)]
        ev0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(s_cur)
        for r in range(nreq):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[r]:
                    pass
            o, n, op = int(wl["offsets"][r]), int(wl["n"][r]), int(wl["op"][r])
            t = tables[int(wl["table"][r])]
            k = keys_h[o:o + n]
            if op == W.OP_FIND:
                t.find(k, base_vout[o:o + n], base_codes[o:o + n])
            elif op == W.OP_INSERT:
                t.insert(k, vals_h[o:o + n], base_codes[o:o + n])
            elif op == W.OP_IOU_ADD:
                t.insert_or_update(k, vals_h[o:o + n], cht.ADD, base_codes[o:o + n])
            else:
                t.erase(k, base_codes[o:o + n])
            ends[r].record(s_cur)
        torch.cuda.synchronize()
        mk = time.perf_counter() - t0
        done_s = np.array([ev0.elapsed_time(e) * 1e-3 for e in ends])
        lat = done_s - (arrivals if arrivals is not None else 0.0)
        res = {"contents": contents(tables)}
        for t in tables:
            t.destroy()
        return lat, mk, res

    def same_results(served_vout, served_codes, served_contents, base_contents):
        """Finds bit-exact per operation; insert / insertOrUpdate / erase codes
        summed per (request, key) (which of equal keys in a request reports
        the change is free); every final table equal.  Compared in pieces of
        about 2^26 operations (host memory)."""
        r0 = 0
        while r0 < nreq:
            r1 = int(np.searchsorted(wl["offsets"], wl["offsets"][r0] + (1 << 26), side="right")) - 1
            r1 = min(max(r1, r0 + 1), nreq)
            o0, o1 = int(wl["offsets"][r0]), int(wl["offsets"][r1])
            rid = np.repeat(np.arange(r0, r1), wl["n"][r0:r1])
            is_find = wl["op"][rid] == W.OP_FIND
            sv, sc = served_vout[o0:o1].cpu().numpy(), served_codes[o0:o1].cpu().numpy()
            bv, bc = base_vout[o0:o1].cpu().numpy(), base_codes[o0:o1].cpu().numpy()
            if not (np.array_equal(sv[is_find], bv[is_find]) and np.array_equal(sc[is_find], bc[is_find])):
                return False
            m = ~is_find
            kk = keys_h[o0:o1].cpu().numpy().view(np.uint64)[m]
            rr = rid[m]
            if kk.size:
                order = np.lexsort((kk, rr))
                kk, rr = kk[order], rr[order]
                starts = np.concatenate([[0], np.nonzero((kk[1:] != kk[:-1]) | (rr[1:] != rr[:-1]))[0] + 1])
                if not np.array_equal(np.add.reduceat(sc[m][order].astype(np.int64), starts),
                                      np.add.reduceat(bc[m][order].astype(np.int64), starts)):
                    return False
            r0 = r1
        return all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
                   for a, b in zip(served_contents, base_contents))

    def breakdown(prof, mk, name):
        tr = prof["trace"]
        if args.serving_trace:
            np.save(f"{args.serving_trace}_{name}.npy", tr)
        per_round = tr["engine_ms"] * 1e3 / np.maximum(tr["rounds"], 1)
        return {"gpu_busy_s": round(prof["gpu_step_ms"] / 1e3, 4), "engine_s": round(prof["engine_ms"] / 1e3, 4),
                "host_admit_s": round(prof["host_admit_ms"] / 1e3, 4), "makespan_s": round(mk, 4),
                "dependent_rounds": prof["rounds"], "parts": prof["parts"], "work_items": prof["chunks"],
                "migrations": prof["migrations"],
                "engine_us_per_round_p50_p90": [round(float(np.percentile(per_round, q)), 2) for q in (50, 90)],
                "recut_steps": int(tr["recut"].sum()), "largest_table_log2": int(tr["max_table_log2"].max())}

    lat0, mk0, steps0, done0, grown, prof0 = run(np.zeros(nreq), keep=True)
    assert done0 == nreq
    cap_rps = nreq / mk0
    cap_vout, cap_codes = vout_h.clone(), codes_h.clone()
    out = {"workload": "serving: 256 growable tables (key universes log-uniform 2^10..2^24), requests of 1..65536 "
                       "ops (log-uniform), table ~ Zipf(1.0), find/insert/insertOrUpdate(add)/erase "
                       f"{'/'.join(str(round(100 * x)) for x in args.serving_mix)}, "
                       f"request arrays in {'device' if on_dev else 'pinned host'} memory, memory cap 64 GiB",
           "request_arrays": "copied through the device arena" if args.serving_stage_inputs else
                             "read and written in place (zero-copy)",
           "table_config": {"growable": True, "alpha": 0.5, "reuse_tombstones": args.serving_reuse_tombstones},
           "requests": nreq, "ops": total, "final_table_bytes": grown,
           "capacity": {"makespan_s": round(mk0, 4), "requests_per_s": round(cap_rps, 1),
                        "mops": round(total / mk0 / 1e6, 1), "steps": steps0,
                        "p50_ms": round(float(np.percentile(lat0, 50)) * 1e3, 3),
                        "p99_ms": round(float(np.percentile(lat0, 99)) * 1e3, 3),
                        "time": breakdown(prof0, mk0, "capacity")}}
    for frac in args.serving_loads:
        arr = W.poisson_arrivals(nreq, frac * cap_rps)
        lat, mk, steps, done, _, prof = run(arr)
        out[f"load_{frac}"] = {"offered_requests_per_s": round(frac * cap_rps, 1), "makespan_s": round(mk, 4),
                               "mops": round(total / mk / 1e6, 1), "steps": steps,
                               "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                               "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                               "max_ms": round(float(lat.max()) * 1e3, 3),
                               "time": breakdown(prof, mk, f"load_{frac}")}
    if not args.no_serving_baseline:
        blat, bmk, bres = single_calls(None)
        same = same_results(cap_vout, cap_codes, prof0["contents"], bres["contents"])
        out["single_calls"] = {"what": "the same requests, one cht_* call each in arrival order (no server)",
                               "capacity": {"makespan_s": round(bmk, 4), "mops": round(total / bmk / 1e6, 1),
                                            "requests_per_s": round(nreq / bmk, 1),
                                            "p50_ms": round(float(np.percentile(blat, 50)) * 1e3, 3),
                                            "p99_ms": round(float(np.percentile(blat, 99)) * 1e3, 3)},
                               "results_equal_served": bool(same)}
        for frac in (args.serving_loads if args.serving_baseline_loads is None else args.serving_baseline_loads):
            arr = W.poisson_arrivals(nreq, frac * cap_rps)
            blat, bmk, _ = single_calls(arr)
            out["single_calls"][f"load_{frac}"] = {
                "offered_requests_per_s": round(frac * cap_rps, 1), "makespan_s": round(bmk, 4),
                "mops": round(total / bmk / 1e6, 1), "p50_ms": round(float(np.percentile(blat, 50)) * 1e3, 3),
                "p99_ms": round(float(np.percentile(blat, 99)) * 1e3, 3)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--grow-in-kernel", default="off", choices=["off", "on"],
                    help="table option of the growable table: migrations inside one cooperative launch")
    ap.add_argument("--partition", default="off", choices=["off", "on"],
                    help="table option for every table of the step: hash-partitioned execution of the batches")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side-workloads", action="store_true",
                    help="skip the small batched and serving runs reported beside the step")
    ap.add_argument("--latency-reps", type=int, default=100)
    ap.add_argument("--window-rounds", type=int, default=128,
                    help="sliding-window case: rounds of 2^20 inserts + 2^20 erases (128 = 2^27 of each)")
    ap.add_argument("--case", choices=["find", "insert", "migrate", "shrink", "iou", "grow", "contention", "window", "build",
                                       "smallcalls"],
                    help="run one small single-operation case (for profiling) instead of the benchmark")
    ap.add_argument("--case-log2c", type=int, default=26)
    ap.add_argument("--case-load", type=float, default=0.9)
    ap.add_argument("--case-s", type=float, default=1.0)
    ap.add_argument("--case-agg", type=int, default=1, choices=[0, 1, 2, 3],
                    help="insertOrUpdate aggregation of the case's tables (table option iou_aggregate)")
    ap.add_argument("--case-group-width", type=int, default=0, choices=[-1, 0, 1, 2, 4, 8, 16, 32],
                    help="--case: probe window group width (0 = the automatic rule, -1 = one thread per operation)")
    ap.add_argument("--probe-random-access", action="store_true",
                    help="measure the HBM random-read and random-modify ceilings instead of the benchmark")
    ap.add_argument("--probe-out", default="",
                    help="--probe-random-access: also write the 4 GiB ceilings as JSON to this path")
    ap.add_argument("--workload", default="bounded", choices=["bounded", "batched", "serving"],
                    help="bounded: the 2^28-cell table step (the bench line); batched: many tables, "
                         "one engine launch vs one launch per batch")
    ap.add_argument("--batched-tables", type=int, default=4096)
    ap.add_argument("--batched-log2-min", type=int, default=8)
    ap.add_argument("--batched-log2-max", type=int, default=20)
    ap.add_argument("--batched-verify", type=int, default=16)
    ap.add_argument("--no-graph-baseline", action="store_true")
    ap.add_argument("--batched-engine-only", action="store_true",
                    help="time the engine only (no per-batch launch baselines), e.g. for profiling")
    ap.add_argument("--serving-requests", type=int, default=100_000)
    ap.add_argument("--serving-loads", type=float, nargs="*", default=[0.5, 0.7, 0.9])
    ap.add_argument("--serving-reuse-tombstones", type=int, default=1, choices=[0, 1],
                    help="table option: inserts take the first tombstone on their path")
    ap.add_argument("--serving-mix", type=float, nargs=4, default=[0.5, 0.3, 0.15, 0.05],
                    help="find / insert / insertOrUpdate(add) / erase fractions of the requests")
    ap.add_argument("--no-serving-baseline", action="store_true",
                    help="skip the single-call baseline of the serving workload")
    ap.add_argument("--serving-baseline-loads", type=float, nargs="*", default=None,
                    help="Poisson loads for the single-call baseline (default: the served loads)")
    ap.add_argument("--serving-trace", default="",
                    help="save each run's per-step server trace to <prefix>_<run>.npy")
    ap.add_argument("--serving-arrays", default="pinned", choices=["pinned", "device"],
                    help="where the request arrays live: pinned host memory or device memory")
    ap.add_argument("--serving-stage-inputs", type=int, default=0, choices=[0, 1],
                    help="1: copy every request through the device arena instead of reading it in place")
    args = ap.parse_args()
    if args.workload == "batched":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.case:
        import bench_cases

        bench_cases.run_case(args)
        return
    if args.probe_random_access:
        import bench_cases

        bench_cases.probe_random_access(args.probe_out)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
