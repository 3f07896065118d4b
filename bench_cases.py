"""Single-operation cases and the HBM random-read probe of `bench.py`.

`python bench.py --case find|insert|iou|grow|window|shrink|contention|build|migrate`
runs one small case of one operation (each timed with CUDA events after one
untimed run of the case) and prints one JSON line: the inputs the ncu captures
are taken on.  `python bench.py --probe-random-access` measures the random-read
ceiling of the HBM with a plain gather kernel (no hash table), built at run
time from the source below.  Neither is part of the benchmark's timed step.
"""
from __future__ import annotations

import json
import os
import subprocess

import workloads as W

from bench import GROW_LOG2C0, ZIPF_RANKS, ZIPF_S

def run_case(args):
    """One small case of one operation, timed with CUDA events; prints JSON."""
    import torch

    import paper_1601_04017_gb300 as cht

    cht.load_library()
    log2c, load = args.case_log2c, args.case_load
    c = 1 << log2c
    tcfg = {"partition": {"off": 0, "on": 1}[args.partition], "iou_aggregate": args.case_agg,
            "group_width": args.case_group_width}
    s = torch.cuda.current_stream()

    def tm(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        return round(a.elapsed_time(b), 4)

    out = {"case": args.case, "log2c": log2c, "load": load, "partition": args.partition, "agg": args.case_agg,
           "group_width": args.case_group_width,
           "s": args.case_s}
    if args.case == "shrink":
        # the same shrink once untimed, so the timed one does not include the
        # memory pool's first growth to these sizes
        wl = W.bounded_workload(log2c, loads=(load,), n_find=c // 2, backend="cuda")
        n = wl["counts"][load]
        t = cht.Table(c, config=tcfg)
        t.insert(wl["keys"][:n], wl["vals"][:n])
        t.erase(wl["keys"][: n - n // 8])
        t.migrate(c // 4)
        t.destroy()
        torch.cuda.synchronize()
    if args.case in ("find", "insert", "migrate", "shrink"):
        wl = W.bounded_workload(log2c, loads=(load,), n_find=c // 2, backend="cuda")
        n = wl["counts"][load]
        codes = torch.empty(n, dtype=torch.uint8, device="cuda")
        vout = torch.empty(c // 2, dtype=torch.int64, device="cuda")
        # the whole case twice, the first untimed: kernels loaded, memory pool grown
        for rep in range(2):
            t = cht.Table(c, config=tcfg)
            out["insert_ms"] = tm(lambda: t.insert(wl["keys"][:n], wl["vals"][:n], codes))
            if args.case == "find":
                out["find_hit_ms"] = tm(lambda: t.find(wl["hits"][load], vout, codes[: c // 2]))
                out["find_miss_ms"] = tm(lambda: t.find(wl["misses"], vout, codes[: c // 2]))
            if args.case == "migrate":
                out["migrate_x2_ms"] = tm(lambda: t.migrate(2 * c))
            if args.case == "shrink":
                # erase all but 1/8 of the keys, then shrink by 4 (load 0.5 x 1/8 x 4)
                t.erase(wl["keys"][: n - n // 8])
                live = t.size()[0]
                out["live"] = live
                out["shrink_x4_ms"] = tm(lambda: t.migrate(c // 4))
                out["shrink_src_cells_per_s"] = round(c / (out["shrink_x4_ms"] * 1e-3), 1)
            t.destroy()
    elif args.case == "build":
        # Sort-based bulk build (Sec. 3 "Bulk Operations") of the bench table's
        # keys at the given load, against inserting the same keys one call
        # (each into a cleared table; one untimed round first)
        wl = W.bounded_workload(log2c, loads=(load,), n_find=1 << 20, backend="cuda")
        n = wl["counts"][load]
        k, v = wl["keys"][:n], wl["vals"][:n]
        t = cht.Table(c, config=tcfg)
        for timed in (False, True):
            t.clear()
            ms_b = tm(lambda: t.build(k, v))
            t.clear()
            ms_i = tm(lambda: t.insert(k, v))
            if timed:
                out["build_ms"], out["insert_ms"] = ms_b, ms_i
        t.clear()
        t.build(k, v)
        got = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
        fc = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        t.find(wl["hits"][load], got, fc)
        out["n"] = n
        out["build_mops"] = round(n / (out["build_ms"] * 1e-3) / 1e6, 1)
        out["sampled_finds_ok"] = bool((fc == 1).all().item()) and bool(
            torch.equal(got, W.values_for(wl["hits"][load], backend="cuda")))
        out["live"] = t.size()[0]
        # batches with repeated keys (Zipf(s) over n/2 ranks): the build keeps
        # the last value per key without contention; insertOrUpdate(overwrite)
        # of the same batch is the per-operation way to the same key set
        for s_ in (0.5, 1.0, 1.5):
            z = W.zipf_keys(n, s_, n // 2, W.SEED_ZIPF, backend="cuda")
            zv = torch.arange(1, n + 1, dtype=torch.int64, device="cuda")
            for timed in (False, True):
                t.clear()
                mb = tm(lambda: t.build(z, zv))
                t.clear()
                mi = tm(lambda: t.insert_or_update(z, zv, cht.OVERWRITE))
            out[f"zipf{s_}_build_ms"], out[f"zipf{s_}_iou_overwrite_ms"] = mb, mi
        t.destroy()
    elif args.case == "contention":
        # Contended operations on a filled table (the paper's E4 overwrite and
        # E5 find under skew): N = c/4 rank keys are present (load 0.25);
        # c/2 operations per run draw keys Zipf(s) over those N ranks.
        nr = c // 4
        present = W.rank_to_key(torch.arange(1, nr + 1, dtype=torch.int64, device="cuda"), backend="cuda")
        t = cht.Table(c, config=tcfg)
        t.insert(present, present)
        vout = torch.empty(c // 2, dtype=torch.int64, device="cuda")
        codes = torch.empty(c // 2, dtype=torch.uint8, device="cuda")
        vals = torch.ones(c // 2, dtype=torch.int64, device="cuda")
        for s_ in ZIPF_S:
            z = W.zipf_keys(c // 2, s_, nr, W.SEED_ZIPF, backend="cuda")
            out[f"find_s{s_}_ms"] = tm(lambda: t.find(z, vout, codes))
            out[f"update_add_s{s_}_ms"] = tm(lambda: t.update(z, vals, cht.ADD, codes))
            out[f"update_overwrite_s{s_}_ms"] = tm(lambda: t.update(z, vals, cht.OVERWRITE, codes))
            out[f"iou_overwrite_s{s_}_ms"] = tm(lambda: t.insert_or_update(z, vals, cht.OVERWRITE, codes))
            out[f"iou_add_s{s_}_ms"] = tm(lambda: t.insert_or_update(z, vals, cht.ADD, codes))
        out["ops_per_run"] = c // 2
        t.destroy()
    elif args.case == "iou":
        z = W.zipf_keys(c, args.case_s, min(ZIPF_RANKS, c // 4), W.SEED_ZIPF, backend="cuda")
        ones = torch.ones(c, dtype=torch.int64, device="cuda")
        codes = torch.empty(c, dtype=torch.uint8, device="cuda")
        for rep in range(2):  # the first untimed: kernels loaded, memory pool grown
            t = cht.Table(c, config=tcfg)
            out["iou_ms"] = tm(lambda: t.insert_or_update(z, ones, cht.ADD, codes))
            t.destroy()
    elif args.case == "window":
        # Sliding window on a growable table (the paper's E7): 2^24 live keys;
        # 2^27 / 2^20 rounds, each inserting the next 2^20 keys of the stream
        # and erasing the 2^20 inserted 2^24 keys earlier.  Migrations purge
        # the tombstones (gamma = 1) or grow the table (gamma = 2) as the
        # policy decides.  Reported: operations/s and insert+erase pairs/s.
        win, batch = 1 << 24, 1 << 20
        rounds = args.window_rounds
        keys = W.uniform_keys(win + batch * rounds, backend="cuda")
        t = cht.Table(1 << GROW_LOG2C0, growable=True)
        codes = torch.empty(batch, dtype=torch.uint8, device="cuda")
        t.insert(keys[:win], keys[:win])
        torch.cuda.synchronize()
        mig0 = t.size()[2]

        def run():
            for r in range(rounds):
                ins = keys[win + r * batch: win + (r + 1) * batch]
                t.insert(ins, ins, codes)
                t.erase(keys[r * batch: (r + 1) * batch], codes)

        ms = tm(run)
        live, ne, cap = t.size(check=True)
        assert live == win
        out.update({"rounds": rounds, "window": win, "batch": batch, "ms": ms,
                    "mops": round(2 * batch * rounds / (ms * 1e-3) / 1e6, 1),
                    "pairs_per_s_M": round(batch * rounds / (ms * 1e-3) / 1e6, 1),
                    "capacity_before": mig0, "capacity_after": cap, "nonempty_after": ne})
        t.destroy()
    elif args.case == "smallcalls":
        # Per-call cost of calls of 2^10 .. 2^20 operations on a 2^20-cell table
        # at load 0.5 (L2-resident), device time per call from 32 calls replayed
        # in one CUDA graph: finds of present keys, and inserts of fresh keys
        # into a table just cleared (the clear's own replay time subtracted).
        # A least-squares line over the sizes gives the fixed cost per call and
        # the time per operation.
        import numpy as np

        c = 1 << 20
        wl = W.bounded_workload(20, loads=(0.5,), n_find=c // 2, backend="cuda")
        n05 = wl["counts"][0.5]
        t1 = cht.Table(c)
        t1.insert(wl["keys"][:n05], wl["vals"][:n05])
        t2 = cht.Table(c)
        vout = torch.empty(c, dtype=torch.int64, device="cuda")
        codes = torch.empty(c, dtype=torch.uint8, device="cuda")
        fresh = W.uniform_keys(c, start=1 << 40, backend="cuda")
        R = 32

        def graph_ms(fn):
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                for _ in range(R):
                    fn()
            g.replay()
            ms = tm(g.replay) / R
            del g
            return ms

        sizes = [1 << k for k in range(10, 21)]
        rows = []
        clear_ms = graph_ms(t2.clear)
        for n in sizes:
            q = wl["hits"][0.5][:n] if n <= n05 else torch.cat([wl["hits"][0.5], wl["hits"][0.5]])[:n]
            f_ms = graph_ms(lambda: t1.find(q, vout[:n], codes[:n]))

            def ins():
                t2.clear()
                t2.insert(fresh[:n], fresh[:n], codes[:n])

            i_ms = graph_ms(ins) - clear_ms if n <= n05 else None
            rows.append({"n": n, "find_us": round(f_ms * 1e3, 3), "insert_us": None if i_ms is None else
                         round(i_ms * 1e3, 3)})
        ns = np.array([r["n"] for r in rows], dtype=np.float64)
        fu = np.array([r["find_us"] for r in rows])
        slope, icpt = np.polyfit(ns, fu, 1)
        ok = [r for r in rows if r["insert_us"] is not None]
        islope, iicpt = np.polyfit(np.array([r["n"] for r in ok], np.float64), np.array([r["insert_us"] for r in ok]), 1)
        out.update({"log2c": 20, "load": 0.5, "rows": rows, "clear_us": round(clear_ms * 1e3, 3),
                    "find_fit": {"fixed_us": round(float(icpt), 3), "ns_per_op": round(float(slope) * 1e3, 4)},
                    "insert_fit": {"fixed_us": round(float(iicpt), 3), "ns_per_op": round(float(islope) * 1e3, 4)}})
        t1.destroy()
        t2.destroy()
    elif args.case == "grow":
        keys = W.uniform_keys(c // 2, backend="cuda")
        vals = W.values_for(keys, backend="cuda")
        t = cht.Table(1 << GROW_LOG2C0, growable=True,
                      config=dict(tcfg, grow_in_kernel={"off": 0, "on": 1}[args.grow_in_kernel]))
        out["grow_insert_ms"] = tm(lambda: t.insert(keys, vals))
        out["capacity"] = t.size()[2]
        t.destroy()
    print(json.dumps(out), flush=True)


RANDOM_READ_CU = r"""
#include <cuda_runtime.h>
typedef unsigned long long u64;
__device__ __forceinline__ u64 mix(u64 x) { x ^= x >> 31; x *= 0x7fb5d329728ea185ull; x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull; x ^= x >> 33; return x; }
template <int W> __global__ void rr(const unsigned char* buf, u64 mask, u64 n, u64* out) {
  u64 acc = 0; const u64 stride = u64(gridDim.x) * blockDim.x;
  for (u64 i = u64(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned char* p = buf + (mix(i + 1) & mask) * W;
    if (W == 16) { u64 a, b; asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p)); acc ^= a ^ b; }
    else for (int k = 0; k < W / 32; ++k) { u64 a, b, c, d;
      asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 32 * k));
      acc ^= a ^ b ^ c ^ d; }
  }
  out[u64(blockIdx.x) * blockDim.x + threadIdx.x] = acc;
}
// Random modifications of 16-byte cells (the table's cell layout) at random
// cell indices: K = 0 a fetch-and-add on the cell's second word whose result is
// unused (a reduction); K = 1 a load of the cell, then that add (an update of a
// present key: the add follows the load); K = 2 the 16-byte CAS of an empty
// cell to a filled one (an insert's claim; the buffer starts zeroed).
struct alignas(16) Cell16 { u64 k, v; };
template <int K> __global__ void rm(Cell16* buf, u64 mask, u64 n, u64* out) {
  u64 acc = 0; const u64 stride = u64(gridDim.x) * blockDim.x;
  for (u64 i = u64(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    Cell16* p = buf + (mix(i + 1) & mask);
    if (K == 0) atomicAdd(&p->v, 1ull);
    if (K == 1) { u64 a, b; asm volatile("ld.global.cg.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
      atomicAdd(&p->v, (a & 1ull) | 1ull); acc ^= b; }
    if (K == 2) { Cell16 e{0, 0}, d{i + 1, i}; Cell16 o = atomicCAS(p, e, d); acc ^= o.k; }
  }
  out[u64(blockIdx.x) * blockDim.x + threadIdx.x] = acc;
}
extern "C" float run_rm(void* buf, u64 bytes, u64 n, int kind, u64* out, int grid) {
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  const u64 mask = bytes / 16 - 1; cudaEventRecord(a);
  if (kind == 0) rm<0><<<grid, 256>>>((Cell16*)buf, mask, n, out);
  if (kind == 1) rm<1><<<grid, 256>>>((Cell16*)buf, mask, n, out);
  if (kind == 2) rm<2><<<grid, 256>>>((Cell16*)buf, mask, n, out);
  cudaEventRecord(b); cudaEventSynchronize(b); float ms = 0; cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a); cudaEventDestroy(b);
  return cudaGetLastError() == cudaSuccess ? ms : -1.0f;
}
extern "C" float run_rr(const void* buf, u64 bytes, u64 n, int width, u64* out, int grid) {
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  const u64 mask = bytes / width - 1; cudaEventRecord(a);
  if (width == 16) rr<16><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  if (width == 32) rr<32><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  if (width == 64) rr<64><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  if (width == 128) rr<128><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  if (width == 256) rr<256><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  if (width == 512) rr<512><<<grid, 256>>>((const unsigned char*)buf, mask, n, out);
  cudaEventRecord(b); cudaEventSynchronize(b); float ms = 0; cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a); cudaEventDestroy(b);
  return cudaGetLastError() == cudaSuccess ? ms : -1.0f;
}
"""


def probe_random_access(out_path: str = ""):
    """Random-read bandwidth of the HBM: n reads of W bytes at uniformly random
    W-aligned offsets of a 4 GiB buffer (and of a 16 MiB, L2-resident one).
    This is the practical ceiling of a probe that touches one sector per step.
    Then the rate of random modifications of 16-byte cells (an atomic add, a
    load followed by the add, a 16-byte CAS claim): the ceiling of the
    modifying operations, which dirty a random line each."""
    import ctypes
    import tempfile

    import torch

    from paper_1601_04017_gb300 import _build

    d = tempfile.mkdtemp(prefix="cht_probe_")
    src, so = os.path.join(d, "rr.cu"), os.path.join(d, "rr.so")
    with open(src, "w") as f:
        f.write(RANDOM_READ_CU)
    subprocess.check_call([_build.nvcc_path(), *_build.ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC",
                           "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.run_rr.restype = ctypes.c_float
    lib.run_rr.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                           ctypes.c_int]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid = sms * 32
    out = torch.empty(grid * 256, dtype=torch.int64, device="cuda")
    res = []
    for log2b in (24, 32):
        nbytes = 1 << log2b
        buf = torch.randint(0, 1 << 62, (nbytes // 8,), dtype=torch.int64, device="cuda")
        for width in (16, 32, 64, 128, 256, 512):
            n = (1 << 32) // width
            lib.run_rr(buf.data_ptr(), nbytes, n, width, out.data_ptr(), grid)
            ms = lib.run_rr(buf.data_ptr(), nbytes, n, width, out.data_ptr(), grid)
            res.append({"buffer_bytes": nbytes, "width_bytes": width, "ms": round(ms, 4),
                        "gbs": round(n * width / ms / 1e6, 1), "greads_per_s": round(n / ms / 1e6, 2)})
        del buf
    # random modifications of 16-byte cells: 2^27 per run, on a 4 GiB buffer
    # (HBM) and a 16 MiB one (L2); the CAS runs on a zeroed buffer each time
    lib.run_rm.restype = ctypes.c_float
    lib.run_rm.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                           ctypes.c_int]
    mod = []
    names = {0: "fetch_add", 1: "load_then_add", 2: "cas16_claim"}
    for log2b in (24, 32):
        nbytes = 1 << log2b
        buf = torch.zeros(nbytes // 8, dtype=torch.int64, device="cuda")
        n = 1 << 27
        for kind in (0, 1, 2):
            times = []
            for _ in range(2):  # warm, then timed
                if kind == 2:
                    buf.zero_()
                times.append(lib.run_rm(buf.data_ptr(), nbytes, n, kind, out.data_ptr(), grid))
            ms = times[-1]
            mod.append({"buffer_bytes": nbytes, "kind": names[kind], "ms": round(ms, 4),
                        "gops_per_s": round(n / ms / 1e6, 2)})
        del buf
    line = {"probe": "random_read", "results": res, "random_modify": mod}
    print(json.dumps(line), flush=True)
    if out_path:
        # the ceilings the benchmark quotes beside its byte roofline
        hbm = {m["kind"]: m["gops_per_s"] for m in mod if m["buffer_bytes"] == 1 << 32}
        rd = {r["width_bytes"]: r["greads_per_s"] for r in res if r["buffer_bytes"] == 1 << 32}
        with open(out_path, "w") as f:
            json.dump({"how": "python bench.py --probe-random-access --probe-out " + out_path +
                       " (4 GiB buffer, uniformly random 16-byte cells / W-byte reads, CUDA events)",
                       "random_read_32B_g_per_s": rd.get(32), "random_fetch_add_g_per_s": hbm.get("fetch_add"),
                       "random_load_then_add_g_per_s": hbm.get("load_then_add"),
                       "random_cas16_g_per_s": hbm.get("cas16_claim")}, f, indent=1)
