// Sort-based bulk build (Sec. 3 "Bulk Operations"): the table is built from a
// batch by sorting the batch by hash, dropping all but the last of equal keys,
// and placing the survivors as an insertion in that order would: element i
// (in sorted order) lands at P_i = max(home_i, P_{i-1} + 1), the paper's
// "start looking at max(h(x), i)" rule.  Positions past the last cell wrap to
// the first empty cells from cell 0 on.
//
// GB300 mapping.
//   1. LSD radix sort of the (key, value) cells by the top B bits of the hash
//      (B = 32 for tables of up to 2^32 cells), 8 bits per pass: a histogram
//      kernel (one CTA per tile of 2048 cells), an exclusive scan of the
//      digit-major histogram, and a stable scatter (warp ranks from ballots
//      of the digit bits, warp offsets in shared memory).  The first pass reads
//      the caller's key and value arrays and notes keys 0 / ~0 (for the special
//      slots or the reserved status bit, both set only once the build is sure).
//   2. Placement as a scan: with r_i the number of survivors before i,
//      P_i = r_i + max over survivors j <= i of (home_j - r_j), so a scan of
//      (count, max) pairs under (C1, M1) + (C2, M2) = (C1 + C2,
//      max(M1, M2 - C1)) gives every position at once.  One pass reduces
//      chunks of 2048 cells (8 consecutive ones per thread), one CTA scans the
//      chunk totals, one pass writes the cells (positions rise with i: a
//      chunk's survivors are staged by rank and stored by consecutive threads).
//   3. One thread places the survivors whose position passed the last cell
//      (the tail of the sorted order) at the first empty cells from 0, in
//      order, and sets the counters and special slots.
#include "cht_internal.h"

namespace cht {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr u32 kSortTile = kSortThreads * kSortItems;  // cells per radix tile
constexpr int kScanThreads = 256;
constexpr u32 kScanChunk = kScanThreads * 16;          // u32 per scan chunk
constexpr int kPlaceItems = 8;
constexpr u32 kPlaceChunk = 256 * kPlaceItems;         // cells per placement chunk
constexpr long long kNegInf = -(1ll << 62);

struct SortSrc {
    const Cell* cells;  // null: read keys / vals (the first pass)
    const u64* keys;
    const u64* vals;
};

__device__ __forceinline__ void load_src(const SortSrc& s, u64 i, u64& k, u64& v) {
    if (s.cells) {
        ld_cell_nc(s.cells + i, k, v);
    } else {
        k = s.keys[i];
        v = s.vals[i];
    }
}

// top B bits of the hash
__device__ __forceinline__ u64 sort_key(u64 k, u32 B) { return fmix64(k) >> (64u - B); }

// Inclusive sum over a 256-thread block; `total` gets the block sum.  sh:
// 8 words of shared scratch.
__device__ __forceinline__ u32 block_incl_u32(u32 x, u32& total, u32* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    u32 pre = 0, tot = 0;
    for (int j = 0; j < kScanThreads / 32; ++j) {
        if (j < w) pre += sh[j];
        tot += sh[j];
    }
    __syncthreads();
    total = tot;
    return pre + x;
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(SortSrc src, u64 n, u32 B, u32 shift, u32* hist,
                                                                  u64 ntiles, BuildExtra* ex, int full_keys) {
    __shared__ u32 bins[256];
    bins[threadIdx.x] = 0;
    __syncthreads();
    const u64 base = u64(blockIdx.x) * kSortTile;
    for (int q = 0; q < kSortItems; ++q) {
        const u64 i = base + u64(q) * kSortThreads + threadIdx.x;
        if (i >= n) break;
        u64 k, v;
        load_src(src, i, k, v);
        atomicAdd(&bins[u32(sort_key(k, B) >> shift) & 255u], 1u);
        if (!src.cells && is_reserved(k)) {
            // first pass: keys 0 / ~0 take the special slots (the last copy's
            // value) or set the reserved status bit; they never enter the table
            if (full_keys)
                atomicMax(&ex->sp_last[k == kEmpty ? 0 : 1], i + 1);
            else
                atomicOr(&ex->reserved, 1ull);
        }
    }
    __syncthreads();
    hist[u64(threadIdx.x) * ntiles + blockIdx.x] = bins[threadIdx.x];
}

// Stable scatter of one tile: warp w ranks its 256 cells (8 steps of 32
// consecutive ones): eight ballots give each lane the lanes with its digit,
// a per-warp counter in shared memory the count of earlier steps.  The warps'
// per-digit counts and the tile's digit counts are then scanned, the tile is
// reordered by digit in shared memory (stable), and written out from there:
// consecutive threads write consecutive cells of a digit's run, so the
// stores coalesce.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(SortSrc src, Cell* dst, u64 n, u32 B,
                                                                     u32 shift, const u32* offs, u64 ntiles) {
    constexpr int kW = kSortThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    Cell* const stage = reinterpret_cast<Cell*>(smem);                        // kSortTile cells
    u32(*const wcnt)[257] = reinterpret_cast<u32(*)[257]>(stage + kSortTile);  // [kW][257]
    u32* const goff = &wcnt[kW][0];                                          // 256
    u32* const tstart = goff + 256;                                          // 256
    unsigned char* const sdig = reinterpret_cast<unsigned char*>(tstart + 256);  // kSortTile
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 below = (1u << lane) - 1u;
    for (int j = threadIdx.x; j < kW * 257; j += kSortThreads) (&wcnt[0][0])[j] = 0;
    goff[threadIdx.x] = offs[u64(threadIdx.x) * ntiles + blockIdx.x];
    __syncthreads();

    const u64 tbase = u64(blockIdx.x) * kSortTile;
    const u64 base = tbase + u64(w) * (32 * kSortItems);
    u64 ks[kSortItems], vs[kSortItems];
    u32 dg[kSortItems], rk[kSortItems];
    // all loads first (in flight together), then the ranking votes
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const u64 i = base + u64(q) * 32 + lane;
        ks[q] = 0;
        vs[q] = 0;
        if (i < n) load_src(src, i, ks[q], vs[q]);
    }
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const u64 i = base + u64(q) * 32 + lane;
        const bool valid = i < n;
        const u32 d = valid ? u32(sort_key(ks[q], B) >> shift) & 255u : 0u;
        // lanes with the same digit: eight ballots, one per digit bit
        u32 peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const u32 m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        dg[q] = valid ? d : 256u;  // past the end: a bin never stored
        const u32 b = wcnt[w][dg[q]];
        rk[q] = b + __popc(peers & below);
        __syncwarp();
        if (valid && (peers & below) == 0u) wcnt[w][d] = b + __popc(peers);  // the group's lowest lane
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: exclusive scan over the warps, then over the digits
        const int d = threadIdx.x;
        u32 run = 0;
        for (int x = 0; x < kW; ++x) {
            const u32 t = wcnt[x][d];
            wcnt[x][d] = run;
            run += t;
        }
        u32 tot;
        const u32 incl = block_incl_u32(run, tot, tstart);  // uses tstart[0..7] as scratch
        tstart[d] = incl - run;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        if (dg[q] < 256u) {
            const u32 j = tstart[dg[q]] + wcnt[w][dg[q]] + rk[q];
            Cell cl;
            cl.key = ks[q];
            cl.val = vs[q];
            stage[j] = cl;
            sdig[j] = (unsigned char)dg[q];
        }
    }
    __syncthreads();
    const u32 cnt = n - tbase < kSortTile ? u32(n - tbase) : kSortTile;
    for (u32 j = threadIdx.x; j < cnt; j += kSortThreads) {
        const u32 d = sdig[j];
        dst[u64(goff[d]) + (j - tstart[d])] = stage[j];
    }
}

u64 scatter_smem_bytes() {
    return size_t(kSortTile) * sizeof(Cell) + size_t(kSortThreads / 32) * 257 * 4 + 512 * 4 + kSortTile;
}

// ---------------------------------------------------------------------------
// exclusive scan of u32 (the digit-major histogram), in place
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const u32* in, u64 m, u32* part) {
    __shared__ u32 sh[kScanThreads / 32];
    const u64 base = u64(blockIdx.x) * kScanChunk;
    u32 s = 0;
    for (int q = 0; q < 16; ++q) {
        const u64 i = base + u64(q) * kScanThreads + threadIdx.x;
        if (i < m) s += in[i];
    }
    u32 total;
    block_incl_u32(s, total, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(u32* part, u64 np) {
    __shared__ u32 sh[kScanThreads / 32];
    u32 carry = 0;
    for (u64 b = 0; b < np; b += kScanThreads) {
        const u64 i = b + threadIdx.x;
        const u32 x = i < np ? part[i] : 0u;
        u32 total;
        const u32 incl = block_incl_u32(x, total, sh);
        if (i < np) part[i] = carry + incl - x;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(u32* data, u64 m, const u32* part) {
    __shared__ u32 sh[kScanThreads / 32];
    const u64 base = u64(blockIdx.x) * kScanChunk;
    u32 carry = part[blockIdx.x];
    for (int q = 0; q < 16; ++q) {
        const u64 i = base + u64(q) * kScanThreads + threadIdx.x;
        const u32 x = i < m ? data[i] : 0u;
        u32 total;
        const u32 incl = block_incl_u32(x, total, sh);
        if (i < m) data[i] = carry + incl - x;
        carry += total;
    }
}

cudaError_t scan_exclusive(u32* data, u64 m, u32* part, cudaStream_t s) {
    const u64 nb = (m + kScanChunk - 1) / kScanChunk;
    scan_reduce_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(data, m, part);
    scan_partials_kernel<<<1, kScanThreads, 0, s>>>(part, nb);
    scan_apply_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(data, m, part);
    count_launch();
    count_launch();
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// placement: scan of (count, max) pairs
// ---------------------------------------------------------------------------
struct Agg {
    u32 c;        // survivors
    long long m;  // max over survivors j of (home_j - rank_j), ranks local to the segment
};

__device__ __forceinline__ Agg agg_join(Agg a, Agg b) {
    Agg r;
    r.c = a.c + b.c;
    const long long bm = b.m - (long long)a.c;
    r.m = a.m > bm ? a.m : bm;
    return r;
}

// Inclusive scan of one Agg per thread over a 256-thread block; `total` gets
// the block's join.
__device__ __forceinline__ Agg block_incl_agg(Agg x, Agg& total, u32* shc, long long* shm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        Agg y;
        y.c = __shfl_up_sync(0xffffffffu, x.c, o);
        y.m = __shfl_up_sync(0xffffffffu, x.m, o);
        if (lane >= o) x = agg_join(y, x);
    }
    if (lane == 31) {
        shc[w] = x.c;
        shm[w] = x.m;
    }
    __syncthreads();
    Agg pre = {0u, kNegInf}, tot = {0u, kNegInf};
    for (int j = 0; j < 8; ++j) {
        Agg t;
        t.c = shc[j];
        t.m = shm[j];
        if (j < w) pre = agg_join(pre, t);
        tot = agg_join(tot, t);
    }
    __syncthreads();
    total = tot;
    return agg_join(pre, x);
}

struct PlaceArgs {
    const Cell* srt;       // sorted cells
    u64 n;
    u32 B, log2c;
    Agg* parts;            // per chunk: its join (count passes), then its exclusive prefix
    unsigned char* flags;  // per sorted cell: 1 survivor, 0 not, 2 deferred
    u32* deferred;         // cells whose survivor test was deferred (count in ex->n_deferred)
    unsigned char* dirty;  // per chunk: a deferred cell of it turned out to survive
    Cell* cells;           // the table
    Cell* ov;              // survivors past the last cell, by rank
    BuildExtra* ex;
};

__device__ __forceinline__ u64 ld_key(const Cell* p) {
    u64 k;
    asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(k) : "l"(p));
    return k;
}

constexpr int kRunScan = 32;  // cells a survivor test looks ahead before deferring

// Survivor test, first try.  A cell survives if its key is not reserved and
// no later cell of the same sort key (equal keys have equal hashes, so their
// copies share that run) holds the same key.  Nearly always the next cell
// decides; when a different key with the same top B hash bits sits between
// (a run mixing keys), up to kRunScan cells are looked at, after which the
// test is deferred (2) to a CTA of its own (build_resolve_kernel), so that a
// rare key inside a long run of copies of another key costs no long scan by
// one thread.
__device__ __forceinline__ unsigned char survivor_first(const PlaceArgs& a, u64 i, u64 k, u64 kn) {
    if (is_reserved(k)) return 0;
    if (i + 1 >= a.n) return 1;
    const u64 s = sort_key(k, a.B);
    if (sort_key(kn, a.B) != s) return 1;
    if (kn == k) return 0;
    for (u64 j = i + 2; j < a.n && j < i + 2 + kRunScan; ++j) {
        const u64 kj = ld_key(a.srt + j);
        if (sort_key(kj, a.B) != s) return 1;
        if (kj == k) return 0;
    }
    return i + 2 + kRunScan >= a.n ? 1 : 2;
}

// Count passes (MODE 0: decide survivors and write the flags; MODE 1: only
// for chunks where a deferred cell survived, recount from the flags) and the
// write pass
// (MODE 2).  Each thread takes kPlaceItems consecutive sorted cells.  The
// count passes store each chunk's join; the write pass turns the chunk's
// exclusive prefix plus the thread's into ranks and positions.
template <int MODE>
__global__ void __launch_bounds__(256) build_place_kernel(PlaceArgs a) {
    __shared__ u32 shc[8];
    __shared__ long long shm[8];
    __shared__ u32 ic[256];
    __shared__ long long im[256];
    if (MODE == 1 && a.dirty[blockIdx.x] == 0) return;
    const u64 c = 1ull << a.log2c;
    const u32 hshift = a.B - a.log2c;
    const u64 i0 = u64(blockIdx.x) * kPlaceChunk + u64(threadIdx.x) * kPlaceItems;
    u64 ks[kPlaceItems], vs[kPlaceItems];
#pragma unroll
    for (int q = 0; q < kPlaceItems; q += 2) {
        ks[q] = ks[q + 1] = kEmpty;
        vs[q] = vs[q + 1] = 0;
        if (i0 + q + 1 < a.n)
            ld_pair_nc(a.srt + i0 + q, ks[q], vs[q], ks[q + 1], vs[q + 1]);  // i0 is even: 32-byte aligned
        else if (i0 + q < a.n)
            ld_cell_nc(a.srt + i0 + q, ks[q], vs[q]);
    }
    u32 sv = 0;
    if (MODE == 0) {
        const u64 knext = i0 + kPlaceItems < a.n ? ld_key(a.srt + i0 + kPlaceItems) : kEmpty;
#pragma unroll
        for (int q = 0; q < kPlaceItems; ++q) {
            if (i0 + q >= a.n) continue;
            const unsigned char f = survivor_first(a, i0 + q, ks[q], q + 1 < kPlaceItems ? ks[q + 1] : knext);
            a.flags[i0 + q] = f;
            if (f == 1) sv |= 1u << q;
            if (f == 2) a.deferred[atomicAdd(&a.ex->n_deferred, 1u)] = u32(i0 + q);
        }
    } else {
#pragma unroll
        for (int q = 0; q < kPlaceItems; ++q)
            if (i0 + q < a.n && a.flags[i0 + q] == 1) sv |= 1u << q;
    }
    Agg loc = {0u, kNegInf};
#pragma unroll
    for (int q = 0; q < kPlaceItems; ++q) {
        if (!((sv >> q) & 1u)) continue;
        const Agg x = {1u, (long long)(sort_key(ks[q], a.B) >> hshift)};
        loc = agg_join(loc, x);
    }
    Agg tot;
    const Agg incl = block_incl_agg(loc, tot, shc, shm);
    if (MODE != 2) {
        if (threadIdx.x == 0) a.parts[blockIdx.x] = tot;
        return;
    }
    ic[threadIdx.x] = incl.c;
    im[threadIdx.x] = incl.m;
    __syncthreads();
    const Agg first = a.parts[blockIdx.x];
    Agg carry = first;
    if (threadIdx.x > 0) {
        const Agg left = {ic[threadIdx.x - 1], im[threadIdx.x - 1]};
        carry = agg_join(carry, left);
    }
    // the chunk's survivors, by rank, with their positions: staged so that
    // consecutive threads then store consecutive survivors (rising positions)
    extern __shared__ __align__(16) unsigned char psm[];
    Cell* const stage = reinterpret_cast<Cell*>(psm);
    u64* const spos = reinterpret_cast<u64*>(stage + kPlaceChunk);
#pragma unroll
    for (int q = 0; q < kPlaceItems; ++q) {
        if (!((sv >> q) & 1u)) continue;
        const u64 home = sort_key(ks[q], a.B) >> hshift;
        const u64 rank = carry.c;
        const long long hm = (long long)home - (long long)rank;
        const long long m = carry.m > hm ? carry.m : hm;
        const u32 j = carry.c - first.c;
        spos[j] = rank + u64(m);
        stage[j].key = ks[q];
        stage[j].val = vs[q];
        const Agg x = {1u, (long long)home};
        carry = agg_join(carry, x);
    }
    __syncthreads();
    for (u32 j = threadIdx.x; j < tot.c; j += 256) {
        const u64 p = spos[j];
        if (p < c) {
            a.cells[p] = stage[j];
        } else {
            const u64 rank = u64(first.c) + j;
            a.ov[rank] = stage[j];
            atomicMin(&a.ex->first_ov, rank);
        }
    }
}

u64 place_smem_bytes() { return size_t(kPlaceChunk) * (sizeof(Cell) + sizeof(u64)); }

// ---------------------------------------------------------------------------
// Deferred survivor tests: one CTA per deferred cell scans the rest of its run
// 2048 cells at a time (coalesced) for another copy of its key; a survivor
// marks its chunk for the recount.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) build_resolve_kernel(PlaceArgs a) {
    __shared__ u64 sh_found[8], sh_end[8];
    const u32 nd = a.ex->n_deferred;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (u32 d = blockIdx.x; d < nd; d += gridDim.x) {
        const u64 i = a.deferred[d];
        const u64 k = ld_key(a.srt + i);
        const u64 s = sort_key(k, a.B);
        unsigned char f = 1;
        for (u64 j0 = i + 2; j0 < a.n; j0 += kPlaceChunk) {
            u64 found = ~0ull, end = ~0ull;
            for (int q = 0; q < kPlaceItems; ++q) {
                const u64 j = j0 + u64(q) * 256 + threadIdx.x;
                if (j >= a.n) {
                    end = end < a.n ? end : a.n;
                    continue;
                }
                const u64 kj = ld_key(a.srt + j);
                if (sort_key(kj, a.B) != s) end = end < j ? end : j;
                else if (kj == k) found = found < j ? found : j;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const u64 f2 = __shfl_xor_sync(0xffffffffu, found, o);
                const u64 e2 = __shfl_xor_sync(0xffffffffu, end, o);
                found = f2 < found ? f2 : found;
                end = e2 < end ? e2 : end;
            }
            if (lane == 0) {
                sh_found[w] = found;
                sh_end[w] = end;
            }
            __syncthreads();
            found = sh_found[0];
            end = sh_end[0];
            for (int v = 1; v < 8; ++v) {
                found = sh_found[v] < found ? sh_found[v] : found;
                end = sh_end[v] < end ? sh_end[v] : end;
            }
            __syncthreads();
            if (found < end) {  // a later copy inside the run
                f = 0;
                break;
            }
            if (end != ~0ull) break;  // the run ended first
        }
        if (threadIdx.x == 0) {
            a.flags[i] = f;
            if (f) a.dirty[i / kPlaceChunk] = 1;
        }
    }
}

// One CTA: exclusive prefixes of the chunk joins, the survivor count S.
__global__ void __launch_bounds__(256) build_place_scan_kernel(Agg* parts, u64 np, BuildExtra* ex) {
    __shared__ u32 shc[8];
    __shared__ long long shm[8];
    __shared__ u32 ic[256];
    __shared__ long long im[256];
    Agg carry = {0u, kNegInf};
    for (u64 b = 0; b < np; b += 256) {
        const u64 i = b + threadIdx.x;
        Agg x = {0u, kNegInf};
        if (i < np) x = parts[i];
        Agg tot;
        const Agg incl = block_incl_agg(x, tot, shc, shm);
        ic[threadIdx.x] = incl.c;
        im[threadIdx.x] = incl.m;
        __syncthreads();
        if (i < np) {
            // the join has no inverse (max), so the exclusive prefix is the
            // carry joined with the previous thread's inclusive one
            Agg left = {0u, kNegInf};
            if (threadIdx.x > 0) {
                left.c = ic[threadIdx.x - 1];
                left.m = im[threadIdx.x - 1];
            }
            parts[i] = agg_join(carry, left);
        }
        __syncthreads();
        carry = agg_join(carry, tot);
    }
    if (threadIdx.x == 0) {
        ex->S = carry.c;
        ex->first_ov = ~0ull;
    }
}

// One thread: survivors whose position passed the last cell take the first
// empty cells from cell 0 on, in sorted order (a sequential insertion wraps
// the same way; the cells before them are final); then the counters and the
// special slots (the last copy's value).
__global__ void build_finish_kernel(Cell* cells, u32 log2c, const Cell* ov, BuildExtra* ex, DevState* st,
                                    const u64* vals) {
    if (threadIdx.x != 0) return;
    const u64 c = 1ull << log2c;
    const u64 S = ex->S;
    u64 cursor = 0;
    for (u64 r = ex->first_ov; r < S; ++r) {
        while (cursor < c && cells[cursor].key != kEmpty) ++cursor;
        if (cursor >= c) {  // cannot happen while S < c
            st->status |= kFull;
            break;
        }
        cells[cursor] = ov[r];
        ++cursor;
    }
    st->I = S;
    st->D = 0;
    if (ex->reserved) st->status |= kReserved;
    for (int sl = 0; sl < 2; ++sl) {
        const u64 last = ex->sp_last[sl];
        if (last) {
            st->sp_present[sl] = 1u;
            st->sp_val[sl] = vals[last - 1];
        }
    }
}

}  // namespace

u32 build_sort_bits(u32 log2c) { return log2c <= 32 ? 32u : 8u * ((log2c + 7u) / 8u); }

namespace {
// Scratch layout: two sort buffers, the digit histogram and its scan
// partials, the chunk joins, the survivor flags, the deferred list, the
// chunks' recount marks, the counters.
struct Layout {
    u64 ntiles, hist_n, nparts, nchunks;
    u64 off_buf1, off_hist, off_part, off_parts, off_flags, off_def, off_dirty, off_ex, total;
    explicit Layout(u64 n) {
        auto al = [](u64 x) { return (x + 255) & ~255ull; };
        ntiles = (n + kSortTile - 1) / kSortTile;
        hist_n = 256 * ntiles;
        nparts = (hist_n + kScanChunk - 1) / kScanChunk;
        nchunks = (n + kPlaceChunk - 1) / kPlaceChunk;
        off_buf1 = al(n * sizeof(Cell));
        off_hist = off_buf1 + al(n * sizeof(Cell));
        off_part = off_hist + al(hist_n * 4);
        off_parts = off_part + al(nparts * 4);
        off_flags = off_parts + al(nchunks * sizeof(Agg));
        off_def = off_flags + al(n);
        off_dirty = off_def + al(n * 4);
        off_ex = off_dirty + al(nchunks);
        total = off_ex + al(sizeof(BuildExtra));
    }
};

PlaceArgs place_args(const Cell* sorted, u64 n, u32 log2c, void* scratch, BuildExtra* ex) {
    const Layout L(n);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    PlaceArgs a;
    a.srt = sorted;
    a.n = n;
    a.B = build_sort_bits(log2c);
    a.log2c = log2c;
    a.parts = reinterpret_cast<Agg*>(base + L.off_parts);
    a.flags = base + L.off_flags;
    a.deferred = reinterpret_cast<u32*>(base + L.off_def);
    a.dirty = base + L.off_dirty;
    a.cells = nullptr;
    // the survivors past the last cell go to whichever sort buffer does not
    // hold the sorted cells
    Cell* b0 = reinterpret_cast<Cell*>(base);
    a.ov = sorted == b0 ? reinterpret_cast<Cell*>(base + L.off_buf1) : b0;
    a.ex = ex;
    return a;
}
}  // namespace

u64 build_scratch_bytes(u64 n) { return Layout(n).total; }

u64 scan_partials(u64 m) { return (m + kScanChunk - 1) / kScanChunk; }
cudaError_t scan_exclusive_u32(u32* data, u64 m, u32* part, cudaStream_t s) { return scan_exclusive(data, m, part, s); }

cudaError_t launch_build_sort(const u64* keys, const u64* vals, u64 n, u32 log2c, int full_keys, void* scratch,
                              const Cell** sorted, BuildExtra** ex_out, cudaStream_t s) {
    const u32 B = build_sort_bits(log2c);
    const Layout L(n);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    Cell* buf[2] = {reinterpret_cast<Cell*>(base), reinterpret_cast<Cell*>(base + L.off_buf1)};
    u32* hist = reinterpret_cast<u32*>(base + L.off_hist);
    u32* part = reinterpret_cast<u32*>(base + L.off_part);
    BuildExtra* ex = reinterpret_cast<BuildExtra*>(base + L.off_ex);
    cudaError_t e = cudaMemsetAsync(ex, 0, sizeof(BuildExtra), s);
    if (e != cudaSuccess) return e;
    SortSrc src;
    src.cells = nullptr;
    src.keys = keys;
    src.vals = vals;
    e = cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(scatter_smem_bytes()));
    if (e != cudaSuccess) return e;
    int cur = 0;
    for (u32 shift = 0; shift < B; shift += 8) {
        radix_hist_kernel<<<unsigned(L.ntiles), kSortThreads, 0, s>>>(src, n, B, shift, hist, L.ntiles, ex,
                                                                    full_keys);
        count_launch();
        e = scan_exclusive(hist, L.hist_n, part, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<unsigned(L.ntiles), kSortThreads, scatter_smem_bytes(), s>>>(src, buf[cur], n, B,
                                                                                          shift, hist, L.ntiles);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        src.cells = buf[cur];
        cur ^= 1;
    }
    *sorted = src.cells;
    *ex_out = ex;
    return cudaSuccess;
}

cudaError_t launch_build_count(const Cell* sorted, u64 n, u32 log2c, void* scratch, BuildExtra* ex,
                               cudaStream_t s) {
    const Layout L(n);
    const PlaceArgs a = place_args(sorted, n, log2c, scratch, ex);
    cudaError_t e = cudaMemsetAsync(a.dirty, 0, L.nchunks, s);
    if (e != cudaSuccess) return e;
    build_place_kernel<0><<<unsigned(L.nchunks), 256, 0, s>>>(a);
    // deferred survivor tests (both kernels return at once when there are none)
    build_resolve_kernel<<<unsigned(sm_count() * 4), 256, 0, s>>>(a);
    build_place_kernel<1><<<unsigned(L.nchunks), 256, 0, s>>>(a);
    build_place_scan_kernel<<<1, 256, 0, s>>>(a.parts, L.nchunks, ex);
    for (int i = 0; i < 4; ++i) count_launch();
    return cudaGetLastError();
}

cudaError_t launch_build_place(const Cell* sorted, u64 n, Cell* cells, u32 log2c, void* scratch, BuildExtra* ex,
                               DevState* st, const u64* vals, cudaStream_t s) {
    const Layout L(n);
    PlaceArgs a = place_args(sorted, n, log2c, scratch, ex);
    a.cells = cells;
    cudaError_t e = cudaFuncSetAttribute(build_place_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(place_smem_bytes()));
    if (e != cudaSuccess) return e;
    build_place_kernel<2><<<unsigned(L.nchunks), 256, place_smem_bytes(), s>>>(a);
    build_finish_kernel<<<1, 32, 0, s>>>(cells, log2c, a.ov, ex, st, vals);
    count_launch();
    count_launch();
    return cudaGetLastError();
}

}  // namespace cht
