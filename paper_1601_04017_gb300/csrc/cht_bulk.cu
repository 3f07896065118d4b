// Hash-partitioned execution of large batches (Sec. 4.5 "Bulk Operations":
// a batch of size m = Omega(n) is integer-sorted by hash and co-partitioned
// with the table, so that the pieces are processed with locality).
//
// GB300 mapping.  A batch that touches most of a table larger than L2 makes
// every operation fetch a random DRAM line; long probes at high load fetch
// several, and the same lines again for other operations.  Here the batch is
// first reordered by the top 8 bits of the hash -- the top bits of every home
// slot, so partition d holds exactly the operations whose probes start in the
// d-th 1/256 of the table -- and the operation kernel then walks the
// reordered batch in order (warps take consecutive pieces, grid-stride), so
// the operations in flight at any moment touch one or two table slices,
// which stay in L2 while the DRAM streams each slice about once.  Stages:
//   1. part_hist_kernel: per tile of 2048 operations, counts per partition,
//      stored partition-major (hist[d * ntiles + tile]).
//   2. exclusive scan of the histogram (plus one sentinel = n): the start of
//      each (partition, tile) run in the reordered batch.
//   3. part_scatter_kernel: a stable scatter of the keys (and values) into
//      the reordered arrays, with each operation's offset in its tile (u16).
//      Ranking as in the bulk build's radix scatter: eight ballots give the
//      lanes of a warp step with the same digit, per-warp counters in shared
//      memory the earlier steps; the tile is staged by digit and stored in
//      digit runs.
//   4. the operation kernel on the reordered arrays (results reordered too).
//   5. part_gather_kernel: per tile, the tile's 256 runs of results are read
//      back (consecutive threads, consecutive elements of a run), placed by
//      their stored offsets in shared memory and written out in the caller's
//      order with coalesced stores.
// Every per-operation result is the same as the direct kernel's: under phase
// semantics the order of the operations of one batch is not observable,
// except which of several equal-key operations wins, which is set-valued.
#include "cht_internal.h"

namespace cht {
namespace {

constexpr int kPThreads = 256;
constexpr int kPItems = 8;
constexpr u32 kPTile = kPThreads * kPItems;  // operations per tile (< 2^16: offsets fit u16)
constexpr u32 kPBins = 256;
constexpr int kPWarps = kPThreads / 32;

__device__ __forceinline__ u32 part_of(u64 key, u32 shift) { return u32(fmix64(key) >> shift) & (kPBins - 1u); }

__device__ __forceinline__ u64 ld_cs(const u64* p) {
    u64 x;
    asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(x) : "l"(p));
    return x;
}

__global__ void __launch_bounds__(kPThreads) part_hist_kernel(const u64* keys, u64 n, u32 shift, u32* hist,
                                                              u64 ntiles) {
    __shared__ u32 bins[kPBins];
    bins[threadIdx.x] = 0;
    __syncthreads();
    const u64 base = u64(blockIdx.x) * kPTile;
    u64 k[kPItems];
#pragma unroll
    for (int q = 0; q < kPItems; ++q) {
        const u64 i = base + u64(q) * kPThreads + threadIdx.x;
        k[q] = i < n ? ld_cs(keys + i) : 0;
    }
#pragma unroll
    for (int q = 0; q < kPItems; ++q) {
        const u64 i = base + u64(q) * kPThreads + threadIdx.x;
        if (i < n) atomicAdd(&bins[part_of(k[q], shift)], 1u);
    }
    __syncthreads();
    hist[u64(threadIdx.x) * ntiles + blockIdx.x] = bins[threadIdx.x];
}

// Shared memory of the scatter: staged keys (and values), offsets in the
// tile, digits, per-warp digit counters, the tile's digit starts and the
// runs' global starts.
template <bool kVals>
constexpr size_t scatter_smem() {
    return size_t(kPTile) * 8 * (kVals ? 2 : 1) + size_t(kPTile) * 2 + kPTile + size_t(kPWarps) * 257 * 4 +
           2 * kPBins * 4;
}

template <bool kVals>
__global__ void __launch_bounds__(kPThreads) part_scatter_kernel(const u64* keys, const u64* vals, u64 n,
                                                                 u32 shift, const u32* offs, u64 ntiles,
                                                                 u64* pkeys, u64* pvals, unsigned short* ppos) {
    extern __shared__ __align__(16) unsigned char smem[];
    u64* const skey = reinterpret_cast<u64*>(smem);
    u64* const sval = skey + kPTile;  // used only with values
    unsigned short* const spos = reinterpret_cast<unsigned short*>(skey + (kVals ? 2 : 1) * kPTile);
    unsigned char* const sdig = reinterpret_cast<unsigned char*>(spos + kPTile);
    u32(*const wcnt)[257] = reinterpret_cast<u32(*)[257]>(sdig + kPTile);
    u32* const tstart = &wcnt[kPWarps][0];  // tile start of each digit's run (also scan scratch)
    u32* const goff = tstart + kPBins;      // global start of each digit's run of this tile
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 below = (1u << lane) - 1u;
    for (int j = threadIdx.x; j < kPWarps * 257; j += kPThreads) (&wcnt[0][0])[j] = 0;
    goff[threadIdx.x] = offs[u64(threadIdx.x) * ntiles + blockIdx.x];
    __syncthreads();

    const u64 tbase = u64(blockIdx.x) * kPTile;
    const u32 wbase = u32(w) * (32 * kPItems);  // this warp's first offset in the tile
    u64 ks[kPItems], vs[kPItems];
    u32 dg[kPItems], rk[kPItems];
#pragma unroll
    for (int q = 0; q < kPItems; ++q) {
        const u64 i = tbase + wbase + u64(q) * 32 + lane;
        ks[q] = i < n ? ld_cs(keys + i) : 0;
        vs[q] = (kVals && i < n) ? ld_cs(vals + i) : 0;
    }
#pragma unroll
    for (int q = 0; q < kPItems; ++q) {
        const u64 i = tbase + wbase + u64(q) * 32 + lane;
        const bool valid = i < n;
        const u32 d = valid ? part_of(ks[q], shift) : 0u;
        u32 peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const u32 m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        dg[q] = valid ? d : kPBins;  // past the end: never stored
        const u32 b = wcnt[w][dg[q]];
        rk[q] = b + __popc(peers & below);
        __syncwarp();
        if (valid && (peers & below) == 0u) wcnt[w][d] = b + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: exclusive over the warps, then the tile's digit starts
        const int d = threadIdx.x;
        u32 run = 0;
        for (int x = 0; x < kPWarps; ++x) {
            const u32 t = wcnt[x][d];
            wcnt[x][d] = run;
            run += t;
        }
        // inclusive block scan of `run` over the 256 digits (warp shuffles,
        // then the warps' totals)
        u32 x = run;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ u32 wtot[kPWarps];
        if (lane == 31) wtot[w] = x;
        __syncthreads();
        u32 pre = 0;
        for (int j = 0; j < w; ++j) pre += wtot[j];
        tstart[d] = pre + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPItems; ++q) {
        if (dg[q] < kPBins) {
            const u32 j = tstart[dg[q]] + wcnt[w][dg[q]] + rk[q];
            skey[j] = ks[q];
            if (kVals) sval[j] = vs[q];
            spos[j] = (unsigned short)(wbase + u32(q) * 32 + u32(lane));
            sdig[j] = (unsigned char)dg[q];
        }
    }
    __syncthreads();
    const u32 cnt = n - tbase < kPTile ? u32(n - tbase) : kPTile;
    for (u32 j = threadIdx.x; j < cnt; j += kPThreads) {
        const u32 d = sdig[j];
        const u64 dst = u64(goff[d]) + (j - tstart[d]);
        pkeys[dst] = skey[j];
        if (kVals) pvals[dst] = sval[j];
        ppos[dst] = spos[j];
    }
}

// Results back into the caller's order, one tile per CTA.
template <bool kVout, bool kCodes>
__global__ void __launch_bounds__(kPThreads) part_gather_kernel(const unsigned short* ppos, const u64* pvout,
                                                                const unsigned char* pcodes, const u32* offs,
                                                                u64 ntiles, u64 n, u64* vals_out,
                                                                unsigned char* codes) {
    __shared__ u32 rstart[kPBins];    // global start of each digit's run of this tile
    __shared__ u32 tpre[kPBins + 1];  // exclusive prefix of the run lengths within the tile
    __shared__ u32 wtot[kPWarps];
    __shared__ __align__(16) u64 sv[kVout ? kPTile : 1];
    __shared__ __align__(16) unsigned char sc[kCodes ? kPTile : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d = threadIdx.x;
    const u64 idx = u64(d) * ntiles + blockIdx.x;
    const u32 s0 = offs[idx], len = offs[idx + 1] - s0;  // offs has a sentinel: offs[256 * ntiles] = n
    rstart[d] = s0;
    u32 x = len;
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    u32 pre = 0, tot = 0;
    for (int j = 0; j < kPWarps; ++j) {
        if (j < w) pre += wtot[j];
        tot += wtot[j];
    }
    tpre[d] = pre + x - len;
    if (d == 0) tpre[kPBins] = tot;
    __syncthreads();
    const u32 cnt = tot;  // = operations in this tile
    for (u32 j = threadIdx.x; j < cnt; j += kPThreads) {
        // the digit whose run holds element j: the last d with tpre[d] <= j
        u32 lo = 0, hi = kPBins;  // tpre[lo] <= j < tpre[hi]
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (tpre[mid] <= j) lo = mid;
            else hi = mid;
        }
        const u64 src = u64(rstart[lo]) + (j - tpre[lo]);
        const u32 p = ppos[src];
        if (kVout) sv[p] = pvout[src];
        if (kCodes) sc[p] = pcodes[src];
    }
    __syncthreads();
    const u64 tbase = u64(blockIdx.x) * kPTile;
    for (u32 j = threadIdx.x; j < cnt; j += kPThreads) {
        if (kVout) vals_out[tbase + j] = sv[j];
        if (kCodes) codes[tbase + j] = sc[j];
    }
}

// ---------------------------------------------------------------------------
// Live cells in cell index order (the table side of a bulk merge): per chunk
// of kCompactChunk cells a count, an exclusive scan of the counts, then each
// chunk's live cells written in order from its offset.
// ---------------------------------------------------------------------------
constexpr u32 kCompactChunk = 4096;
constexpr u32 kCompactPerWarp = kCompactChunk / kPWarps;  // 512 cells, 16 windows of 32

__device__ __forceinline__ bool live_key(u64 k) { return k != kEmpty && k != kTomb; }

__global__ void __launch_bounds__(kPThreads) live_count_kernel(const Cell* cells, u64 c, u32* counts) {
    __shared__ u32 wsum[kPWarps];
    const u64 base = u64(blockIdx.x) * kCompactChunk;
    u32 cnt = 0;
    for (u32 j = threadIdx.x; j < kCompactChunk; j += kPThreads) {
        const u64 i = base + j;
        if (i < c && live_key(cells[i].key)) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int w = 0; w < kPWarps; ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kPThreads) live_write_kernel(const Cell* cells, u64 c, const u32* offs,
                                                               u64* keys_out, u64* vals_out) {
    __shared__ u32 wcount[kPWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 below = (1u << lane) - 1u;
    const u64 base = u64(blockIdx.x) * kCompactChunk + u64(w) * kCompactPerWarp;
    u32 cnt = 0;
    for (u32 j = 0; j < kCompactPerWarp; j += 32) {
        const u64 i = base + j + lane;
        cnt += __popc(__ballot_sync(0xffffffffu, i < c && live_key(cells[i].key)));
    }
    if (lane == 0) wcount[w] = cnt;
    __syncthreads();
    u64 out = offs[blockIdx.x];
    for (int x = 0; x < w; ++x) out += wcount[x];
    for (u32 j = 0; j < kCompactPerWarp; j += 32) {
        const u64 i = base + j + lane;
        u64 k = 0, v = 0;
        if (i < c) ld_cell_nc(cells + i, k, v);
        const bool lv = i < c && live_key(k);
        const u32 m = __ballot_sync(0xffffffffu, lv);
        if (lv) {
            const u64 o = out + __popc(m & below);
            keys_out[o] = k;
            vals_out[o] = v;
        }
        out += __popc(m);
    }
}

u64 align256(u64 x) { return (x + 255) & ~u64(255); }

// Scratch layout of one partitioned call.
struct PLayout {
    u64 ntiles, hist_n, parts;
    u64 o_hist, o_part, o_keys, o_vals, o_vout, o_codes, o_pos, o_ticket, total;
    PLayout(u64 n, PartitionIO io) {
        ntiles = (n + kPTile - 1) / kPTile;
        hist_n = u64(kPBins) * ntiles + 1;  // + the sentinel
        parts = scan_partials(hist_n);
        u64 o = 0;
        o_hist = o;
        o = align256(o + hist_n * 4);
        o_part = o;
        o = align256(o + parts * 4);
        o_keys = o;
        o = align256(o + n * 8);
        o_vals = o;
        if (io.vals) o = align256(o + n * 8);
        o_vout = o;
        if (io.vals_out) o = align256(o + n * 8);
        o_codes = o;
        if (io.codes) o = align256(o + n);
        o_pos = o;
        o = align256(o + n * 2);
        o_ticket = o;
        o = align256(o + 8);
        total = o;
    }
};

}  // namespace

u64 partition_scratch_bytes(u64 n, PartitionIO io) { return PLayout(n, io).total; }

namespace {

// Scratch of a two-pass (16-bit) sort of the batch.
struct SLayout {
    u64 ntiles, hist_n, parts;
    u64 o_ha, o_hb, o_pa, o_pb, o_ka, o_va, o_posa, o_kb, o_vb, o_posb, o_ca, o_cb, total;
    SLayout(u64 n, bool codes) {
        ntiles = (n + kPTile - 1) / kPTile;
        hist_n = u64(kPBins) * ntiles + 1;
        parts = scan_partials(hist_n);
        u64 o = 0;
        auto take = [&](u64 bytes) {
            const u64 at = o;
            o = align256(o + bytes);
            return at;
        };
        o_ha = take(hist_n * 4);
        o_hb = take(hist_n * 4);
        o_pa = take(parts * 4);
        o_pb = take(parts * 4);
        o_ka = take(n * 8);
        o_va = take(n * 8);
        o_posa = take(n * 2);
        o_kb = take(n * 8);
        o_vb = take(n * 8);
        o_posb = take(n * 2);
        o_ca = codes ? take(n) : 0;
        o_cb = codes ? take(n) : 0;
        total = o;
    }
};

// One stable 8-bit pass: histogram, scan, scatter of keys and values.
cudaError_t sort_pass(const u64* keys, const u64* vals, u64 n, u32 shift, u32* hist, u64 hist_n, u32* part,
                      u64 ntiles, u64* okeys, u64* ovals, unsigned short* opos, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist + hist_n - 1, 0, sizeof(u32), s);
    if (e != cudaSuccess) return e;
    part_hist_kernel<<<unsigned(ntiles), kPThreads, 0, s>>>(keys, n, shift, hist, ntiles);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive_u32(hist, hist_n, part, s)) != cudaSuccess) return e;
    constexpr size_t sm = scatter_smem<true>();
    static bool attr = false;
    if (!attr) {
        if ((e = cudaFuncSetAttribute(part_scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(sm))) != cudaSuccess)
            return e;
        attr = true;
    }
    part_scatter_kernel<true><<<unsigned(ntiles), kPThreads, sm, s>>>(keys, vals, n, shift, hist, ntiles, okeys,
                                                                      ovals, opos);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

u64 sorted16_scratch_bytes(u64 n, bool codes) { return SLayout(n, codes).total; }

cudaError_t launch_sorted16(const OpArgs& a, void* scratch, PartitionRun run, void* ctx, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const bool codes = a.codes != nullptr;
    const SLayout L(a.n, codes);
    unsigned char* b = static_cast<unsigned char*>(scratch);
    u32* ha = reinterpret_cast<u32*>(b + L.o_ha);
    u32* hb = reinterpret_cast<u32*>(b + L.o_hb);
    u64* ka = reinterpret_cast<u64*>(b + L.o_ka);
    u64* va = reinterpret_cast<u64*>(b + L.o_va);
    unsigned short* pa = reinterpret_cast<unsigned short*>(b + L.o_posa);
    u64* kb = reinterpret_cast<u64*>(b + L.o_kb);
    u64* vb = reinterpret_cast<u64*>(b + L.o_vb);
    unsigned short* pb = reinterpret_cast<unsigned short*>(b + L.o_posb);
    unsigned char* ca = codes ? b + L.o_ca : nullptr;
    unsigned char* cb = codes ? b + L.o_cb : nullptr;
    // LSD order: the lower byte of the top 16 hash bits first, then the top byte
    cudaError_t e = sort_pass(a.keys, a.vals, a.n, 48, ha, L.hist_n, reinterpret_cast<u32*>(b + L.o_pa), L.ntiles,
                              ka, va, pa, s);
    if (e == cudaSuccess)
        e = sort_pass(ka, va, a.n, 56, hb, L.hist_n, reinterpret_cast<u32*>(b + L.o_pb), L.ntiles, kb, vb, pb, s);
    if (e != cudaSuccess) return e;
    OpArgs o = a;
    o.keys = kb;
    o.vals = vb;
    o.codes = cb;
    if ((e = run(o, ctx, s)) != cudaSuccess) return e;
    if (codes) {
        const unsigned grid = unsigned(L.ntiles);
        part_gather_kernel<false, true><<<grid, kPThreads, 0, s>>>(pb, nullptr, cb, hb, L.ntiles, a.n, nullptr, ca);
        part_gather_kernel<false, true><<<grid, kPThreads, 0, s>>>(pa, nullptr, ca, ha, L.ntiles, a.n, nullptr,
                                                                   a.codes);
        count_launch();
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

u64 compact_scratch_bytes(u32 log2c) {
    const u64 nchunks = ((1ull << log2c) + kCompactChunk - 1) / kCompactChunk;
    return align256((nchunks + 1) * 4) + align256(scan_partials(nchunks + 1) * 4);
}

cudaError_t launch_compact_live(const Cell* cells, u32 log2c, u64* keys_out, u64* vals_out, void* scratch,
                                cudaStream_t s) {
    const u64 c = 1ull << log2c;
    const u64 nchunks = (c + kCompactChunk - 1) / kCompactChunk;
    u32* counts = static_cast<u32*>(scratch);
    u32* part = reinterpret_cast<u32*>(static_cast<unsigned char*>(scratch) + align256((nchunks + 1) * 4));
    live_count_kernel<<<unsigned(nchunks), kPThreads, 0, s>>>(cells, c, counts);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = scan_exclusive_u32(counts, nchunks, part, s)) != cudaSuccess) return e;
    live_write_kernel<<<unsigned(nchunks), kPThreads, 0, s>>>(cells, c, counts, keys_out, vals_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_partitioned(const OpArgs& a, PartitionIO io, void* scratch, PartitionRun run, void* ctx,
                               cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.log2c < 8) return cudaErrorInvalidValue;
    const PLayout L(a.n, io);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    u32* hist = reinterpret_cast<u32*>(base + L.o_hist);
    u32* part = reinterpret_cast<u32*>(base + L.o_part);
    u64* pkeys = reinterpret_cast<u64*>(base + L.o_keys);
    u64* pvals = io.vals ? reinterpret_cast<u64*>(base + L.o_vals) : nullptr;
    u64* pvout = io.vals_out ? reinterpret_cast<u64*>(base + L.o_vout) : nullptr;
    unsigned char* pcodes = io.codes ? base + L.o_codes : nullptr;
    unsigned short* ppos = reinterpret_cast<unsigned short*>(base + L.o_pos);
    const u32 shift = 64u - 8u;  // top 8 hash bits = top 8 bits of the home slot
    const unsigned grid = unsigned(L.ntiles);

    cudaError_t e = cudaMemsetAsync(hist + L.hist_n - 1, 0, sizeof(u32), s);  // the sentinel
    if (e != cudaSuccess) return e;
    part_hist_kernel<<<grid, kPThreads, 0, s>>>(a.keys, a.n, shift, hist, L.ntiles);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive_u32(hist, L.hist_n, part, s)) != cudaSuccess) return e;
    if (io.vals) {
        constexpr size_t sm = scatter_smem<true>();
        static bool attr = false;
        if (!attr) {
            if ((e = cudaFuncSetAttribute(part_scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(sm))) != cudaSuccess)
                return e;
            attr = true;
        }
        part_scatter_kernel<true><<<grid, kPThreads, sm, s>>>(a.keys, a.vals, a.n, shift, hist, L.ntiles, pkeys,
                                                              pvals, ppos);
    } else {
        constexpr size_t sm = scatter_smem<false>();
        static bool attr = false;
        if (!attr) {
            if ((e = cudaFuncSetAttribute(part_scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(sm))) != cudaSuccess)
                return e;
            attr = true;
        }
        part_scatter_kernel<false><<<grid, kPThreads, sm, s>>>(a.keys, nullptr, a.n, shift, hist, L.ntiles, pkeys,
                                                               nullptr, ppos);
    }
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    OpArgs b = a;
    b.keys = pkeys;
    b.vals = pvals;
    b.vals_out = pvout;
    b.codes = pcodes;
    b.ticket = reinterpret_cast<unsigned long long*>(base + L.o_ticket);
    if ((e = cudaMemsetAsync(b.ticket, 0, 8, s)) != cudaSuccess) return e;
    if ((e = run(b, ctx, s)) != cudaSuccess) return e;

    if (io.vals_out || io.codes) {
        if (io.vals_out && io.codes)
            part_gather_kernel<true, true><<<grid, kPThreads, 0, s>>>(ppos, pvout, pcodes, hist, L.ntiles, a.n,
                                                                      a.vals_out, a.codes);
        else if (io.vals_out)
            part_gather_kernel<true, false><<<grid, kPThreads, 0, s>>>(ppos, pvout, nullptr, hist, L.ntiles, a.n,
                                                                       a.vals_out, nullptr);
        else
            part_gather_kernel<false, true><<<grid, kPThreads, 0, s>>>(ppos, nullptr, pcodes, hist, L.ntiles, a.n,
                                                                       nullptr, a.codes);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cht
