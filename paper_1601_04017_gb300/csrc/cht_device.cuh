// Device-side building blocks of libcht: the cell type, the hash and home
// map, window loads and the per-table device state.  Header-only; included
// by the kernel translation units of the CUDA library (never by the oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cht {

typedef unsigned long long u64;
typedef unsigned int u32;

// One table cell: <key, value>, 16-byte aligned so a 2-word CAS covers it
// (Sec. 3: cells aligned to 16 bytes, one double-word CAS on key and value).
struct __align__(16) Cell {
    u64 key;
    u64 val;
};

constexpr u64 kEmpty = 0ull;       // empty_key
constexpr u64 kTomb = ~0ull;       // del_key (tombstone, Sec. 4.4)
constexpr u32 kFull = 1u;          // sticky status bits, as in cht.h
constexpr u32 kReserved = 2u;

// Per-operation result codes.
constexpr unsigned char kNo = 0, kYes = 1, kCodeFull = 2, kCodeReserved = 3;

// Per-table counters and status, resident in device memory.
//   I: non-empty cells (tombstones included), D: tombstones (Sec. 4.2/4.4).
//   status: sticky kFull / kReserved bits.
//   mig_fail: set by a migration CTA that could not bound its cluster range.
//   export_pos: output cursor of the export compaction.
struct DevState {
    u64 I;
    u64 D;
    u32 status;
    u32 mig_fail;
    u64 export_pos;
    // full key space: keys 0 and ~0 live here, beside the cells
    // (slot 0: key 0, slot 1: key ~0); untouched by migrations
    u64 sp_val[2];
    u32 sp_present[2];
};

// fmix64, the 64-bit finalizer of MurmurHash3 (Appleby, public domain).
__device__ __forceinline__ u64 fmix64(u64 x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Scaling map h_c(x) = floor(h(x) * c / 2^64) for c = 2^log2c (Sec. 4.3.1):
// the top log2c bits.  `shift` is 64 - log2c.
__device__ __forceinline__ u64 home_of(u64 key, u32 shift) { return fmix64(key) >> shift; }

__device__ __forceinline__ bool is_reserved(u64 k) { return k == kEmpty || k == kTomb; }

// ---------------------------------------------------------------------------
// Window loads.  A lane loads either one cell (16 B) or an aligned pair of
// cells (32 B = one DRAM sector) with a single 256-bit load (sm_100+).
// `.nc` goes through the read-only path (finds: nothing writes the table);
// `.cg` caches in L2 only, the coherence point for concurrent modifiers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld_cell_nc(const Cell* p, u64& k, u64& v) {
    asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(k), "=l"(v) : "l"(p));
}
__device__ __forceinline__ void ld_cell_cg(const Cell* p, u64& k, u64& v) {
    asm volatile("ld.global.cg.v2.u64 {%0,%1}, [%2];" : "=l"(k), "=l"(v) : "l"(p));
}
__device__ __forceinline__ void ld_pair_nc(const Cell* p, u64& k0, u64& v0, u64& k1, u64& v1) {
    asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(k0), "=l"(v0), "=l"(k1), "=l"(v1)
                 : "l"(p));
}
__device__ __forceinline__ void ld_pair_cg(const Cell* p, u64& k0, u64& v0, u64& k1, u64& v1) {
    asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(k0), "=l"(v0), "=l"(k1), "=l"(v1)
                 : "l"(p));
}

// Streaming (evict-first) loads of the operation inputs and stores of results.
__device__ __forceinline__ u64 ld_stream(const u64* p) {
    u64 x;
    asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(x) : "l"(p));
    return x;
}

// 2-word CAS on a whole cell; returns the cell's previous content.
__device__ __forceinline__ Cell cas_cell(Cell* p, Cell expect, Cell desired) {
    return atomicCAS(p, expect, desired);
}

}  // namespace cht
