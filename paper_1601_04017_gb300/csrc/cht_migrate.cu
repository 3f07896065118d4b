// Cluster-wise parallel migration (Sec. 4.3.1, Lemma 1; tombstone purge,
// Sec. 4.4) and the forall/export compaction (Sec. 3 "Bulk Operations").
//
// Migration into a table gamma = 2^g times larger (g >= 0).  The source is
// cut into tiles of T cells.  Tile [d, d+T) moves its borders to just after
// the next empty cell: m(d) = d if cell d-1 is empty, else (first empty cell
// >= d) + 1.  It migrates the source range [m(d), m(d+T)), which consists of
// whole clusters, and owns the target range [gamma*m(d), gamma*m(d+T)).  By
// Lemma 1 a cluster a..b lands inside gamma*a .. gamma*(b+1)-1 (the
// integer-gamma form of the lemma's bound), so the owned target ranges of
// different tiles are disjoint and together cover the target table: no
// atomics on the table and no separate initialisation -- each tile writes
// every cell of its range, empties included (Sec. 4.3.1: the target is
// initialised by the same threads that fill it, region by region).  A tile's
// live cells are re-inserted in source index order, so the layout equals the
// sequential migration (Lemma 1).
//
// GB300 mapping.  A border kernel computes m(d) for every tile once (a short
// forward scan per tile).  In the migration kernel every warp then works on
// its own tiles with no block-wide barrier, so a long cluster only delays
// its own warp.  The warp reads its source range coalesced, 32 cells per
// window with the next 64 in flight, and re-inserts the window's live cells
// in source order: all lanes look up the first free target cell at or after
// their new home at once, and rounds of warp votes settle lanes that picked
// the same cell (place_window), so the layout is the sequential one.  The
// occupancy of the warp's owned target range is a bitmap in shared memory.
// For owned ranges of up to 2048 cells (nearly all at loads up to 0.9 with
// tiles of 512) the warp records which source cell went to each target
// cell and then writes the whole range in one coalesced pass -- every
// 32-byte sector once and whole; longer ranges store elements directly and
// zero-fill the rest.
// A border scan that finds no empty cell within kMaxScan cells (a full
// table, or a cluster longer than that) sets mig_fail; a single-CTA fallback
// kernel, always launched after the tile kernel, then redoes the whole
// migration sequentially.
#include "cht_migrate.cuh"

namespace cht {
namespace {

// The kernels of a host-driven migration: one thread per tile for the
// borders, then one warp per tile (in turn) for the placement.
__global__ void __launch_bounds__(256) migrate_border_kernel(MigArgs a) {
    migrate_borders(a, u64(blockIdx.x) * blockDim.x + threadIdx.x, u64(gridDim.x) * blockDim.x);
}

__global__ void __launch_bounds__(kMigBlock, 5) migrate_window_kernel(MigArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    migrate_window_tiles(a, smem, u64(blockIdx.x) * kMigWarps + (threadIdx.x >> 5), u64(gridDim.x) * kMigWarps);
}

__global__ void __launch_bounds__(kMigBlock, 5) migrate_walk_kernel(MigArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    migrate_walk_tiles(a, smem, u64(blockIdx.x) * kMigWarps + (threadIdx.x >> 5), u64(gridDim.x) * kMigWarps);
}

// Sequential migration of the whole table by one thread (after a block-wide
// zero fill), used only when a tile CTA reported mig_fail.  Visits the source
// in index order from the first cluster start (index 0 if there is none).
__global__ void __launch_bounds__(kMigBlock) migrate_fallback_kernel(MigArgs a) {
    if (a.st->mig_fail == 0) return;
    const u64 c = 1ull << a.slog2, cmask = c - 1;
    const u64 nc = 1ull << a.dlog2, nmask = nc - 1;
    const u32 dshift = 64u - a.dlog2;
    for (u64 i = threadIdx.x; i < nc; i += blockDim.x) {
        Cell z;
        z.key = 0;
        z.val = 0;
        a.dst[i] = z;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    u64 start = 0;
    for (u64 i = 0; i < c; ++i) {
        if (a.src[i].key != kEmpty && a.src[(i - 1) & cmask].key == kEmpty) {
            start = i;
            break;
        }
    }
    u64 moved = 0;
    for (u64 j = 0; j < c; ++j) {
        const Cell cl = a.src[(start + j) & cmask];
        if (cl.key == kEmpty || cl.key == kTomb) continue;
        u64 p = home_of(cl.key, dshift);
        u64 steps = 0;
        while (a.dst[p].key != kEmpty && steps < nc) {
            p = (p + 1) & nmask;
            ++steps;
        }
        if (steps >= nc) {
            a.st->mig_fail = 4u;  // target too small: cannot happen for gamma >= 1
            return;
        }
        a.dst[p] = cl;
        ++moved;
    }
    a.st->I = moved;
    a.st->mig_fail = 8u;  // fallback ran and completed
}

__global__ void __launch_bounds__(256) export_kernel(const Cell* __restrict__ cells, u64 c,
                                                     u64* __restrict__ keys_out,
                                                     u64* __restrict__ vals_out, u64 max_n,
                                                     DevState* st) {
    const int lane = threadIdx.x & 31;
    const u64 stride = u64(gridDim.x) * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x < 2 && st->sp_present[threadIdx.x]) {
        // full key space: the special slots' keys (0, ~0) are live elements too
        const u64 p = atomicAdd(&st->export_pos, 1ull);
        if (p < max_n) {
            keys_out[p] = threadIdx.x ? kTomb : kEmpty;
            if (vals_out) vals_out[p] = st->sp_val[threadIdx.x];
        }
    }
    for (u64 base = u64(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); base < c;
         base += stride) {
        const u64 i = base + lane;
        u64 k = 0, v = 0;
        if (i < c) ld_cell_nc(cells + i, k, v);
        const bool live = i < c && !is_reserved(k);
        const u32 b = __ballot_sync(0xffffffffu, live);
        if (!b) continue;
        u64 pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(&st->export_pos, u64(__popc(b)));
        pos0 = __shfl_sync(0xffffffffu, pos0, 0);
        if (live) {
            const u64 p = pos0 + __popc(b & ((1u << lane) - 1u));
            if (p < max_n) {
                keys_out[p] = k;
                if (vals_out) vals_out[p] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Shrinking (Sec. 4.3.1 "Shrinking"): Lemma 1 does not hold for gamma < 1, so
// the paper cuts the source into blocks, maps each block a..b to a disjoint
// target block a'..b' with the scaling function, and migrates in two phases:
// first every element whose new home lies in its block's target block and
// whose probe stays inside it is placed there (no other thread touches that
// target block), then, after a barrier (here: the kernel boundary), the
// elements that did not fit are inserted concurrently with atomic operations.
//
// Here a warp owns one target block of kShrinkBlock cells, staged in shared
// memory, and the 2^k * kShrinkBlock source cells that map onto it (the new
// home is the top bits of the hash, so it is the old home >> k).  Lanes read
// the source coalesced and place their elements into the shared block by
// linear probing with shared-memory CAS; an element whose new home lies in
// another block (a cluster that began in the previous source block, or
// wrapped around), or whose probe would run past the block's end, goes to a
// spill list.  The block is then written whole, empties included.  Every
// placement is one a sequential insertion could make (it only looked at cells
// of its own block), so the occupied cells equal those of the sequential
// migration of the same elements (linear probing's occupancy does not depend
// on the insertion order); which key sits where may differ.
constexpr u32 kShrinkBlock = 256;

struct ShrinkArgs {
    const Cell* src;
    u32 slog2;
    Cell* dst;
    u32 dlog2;
    DevState* st;
    Cell* spill;                // capacity: 2^dlog2 cells (more than the live count)
    unsigned long long* nspill; // zero before the launch
    u32 block;                  // target cells per warp (kShrinkBlock, or c' if smaller)
};

__global__ void __launch_bounds__(kMigBlock) shrink_kernel(ShrinkArgs a) {
    extern __shared__ __align__(16) unsigned char shrink_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(shrink_smem) + size_t(wib) * 2 * a.block;
    u64* sval = reinterpret_cast<u64*>(skey + a.block);
    const u32 k = a.slog2 - a.dlog2;
    const u64 nblocks = (1ull << a.dlog2) / a.block;
    const u64 span = u64(a.block) << k;  // source cells per block
    const u32 dshift = 64u - a.dlog2;
    u64 moved = 0;
    for (u64 blk = (u64(blockIdx.x) * kMigWarps + wib); blk < nblocks; blk += u64(gridDim.x) * kMigWarps) {
        const u64 t0 = blk * a.block;  // first target cell of the block
        for (u32 j = lane; j < a.block; j += 32) {
            skey[j] = kEmpty;
            sval[j] = 0;
        }
        __syncwarp();
        const u64 s0 = blk * span;
        for (u64 i = lane; i < span; i += 32) {
            u64 key, val;
            ld_cell_nc(a.src + s0 + i, key, val);
            const bool live = key != kEmpty && key != kTomb;
            bool spill = false;
            if (live) {
                const u64 h = home_of(key, dshift);
                spill = true;
                if (h >= t0 && h < t0 + a.block) {
                    for (u32 q = u32(h - t0); q < a.block; ++q) {
                        if (atomicCAS(&skey[q], kEmpty, key) == kEmpty) {
                            sval[q] = val;
                            spill = false;
                            ++moved;
                            break;
                        }
                    }
                }
            }
            // warp-aggregated append to the spill list
            const u32 m = __ballot_sync(0xffffffffu, spill);
            if (m) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.nspill, u64(__popc(m)));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (spill) {
                    Cell c;
                    c.key = key;
                    c.val = val;
                    a.spill[base + __popc(m & ((1u << lane) - 1u))] = c;
                }
            }
        }
        __syncwarp();
        for (u32 j = lane; j < a.block; j += 32) {
            Cell c;
            c.key = skey[j];
            c.val = sval[j];
            a.dst[t0 + j] = c;
        }
        __syncwarp();  // the next block reuses the shared area
    }
    for (int o = 16; o > 0; o >>= 1) moved += __shfl_xor_sync(0xffffffffu, moved, o);
    if (lane == 0 && moved) atomicAdd(&a.st->I, moved);
}

// Second phase: insert the spilled elements concurrently (16-byte CAS into
// an empty cell, linear probing from the new home).  Keys are distinct, so a
// failed CAS only means another element took the cell.  The target holds
// fewer elements than cells, so every probe ends; it is still bounded by c'.
__global__ void __launch_bounds__(256) shrink_spill_kernel(ShrinkArgs a) {
    const u64 n = *a.nspill;
    const u64 cap = 1ull << a.dlog2, mask = cap - 1;
    const u32 dshift = 64u - a.dlog2;
    u64 moved = 0;
    for (u64 i = u64(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += u64(gridDim.x) * blockDim.x) {
        const Cell e = a.spill[i];
        u64 pos = home_of(e.key, dshift);
        for (u64 probed = 0; probed < cap; ++probed, pos = (pos + 1) & mask) {
            u64 ck, cv;
            ld_cell_cg(a.dst + pos, ck, cv);
            if (ck != kEmpty) continue;
            Cell expect;
            expect.key = kEmpty;
            expect.val = 0;
            const Cell old = cas_cell(a.dst + pos, expect, e);
            if (old.key == kEmpty && old.val == 0) {
                ++moved;
                break;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) moved += __shfl_xor_sync(0xffffffffu, moved, o);
    if ((threadIdx.x & 31) == 0 && moved) atomicAdd(&a.st->I, moved);
}

}  // namespace

cudaError_t launch_shrink(const Cell* src, u32 src_log2, Cell* dst, u32 dst_log2, DevState* st, Cell* spill,
                          unsigned long long* nspill, cudaStream_t s) {
    if (dst_log2 >= src_log2) return cudaErrorInvalidValue;
    ShrinkArgs a;
    a.src = src;
    a.slog2 = src_log2;
    a.dst = dst;
    a.dlog2 = dst_log2;
    a.st = st;
    a.spill = spill;
    a.nspill = nspill;
    const u64 cnew = 1ull << dst_log2;
    a.block = cnew < kShrinkBlock ? u32(cnew) : kShrinkBlock;
    const size_t smem = size_t(kMigWarps) * 2 * a.block * sizeof(u64);
    const u64 nblocks = cnew / a.block;
    u64 grid = (nblocks + kMigWarps - 1) / kMigWarps;
    const u64 gcap = u64(sm_count()) * 8;
    if (grid > gcap) grid = gcap;
    shrink_kernel<<<unsigned(grid), kMigBlock, smem, s>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    shrink_spill_kernel<<<unsigned(sm_count() * 4), 256, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

u64 migrate_border_count(u32 src_log2, int tile) {
    const u64 c = 1ull << src_log2;
    u64 T = tile > 0 ? u64(tile) : 256u;
    if (T > c) T = c;
    return c / T;
}

cudaError_t launch_migrate(const Cell* src, u32 src_log2, Cell* dst, u32 dst_log2, DevState* st,
                           int tile, bool windows, u64* border, cudaStream_t s) {
    const u64 c = 1ull << src_log2;
    u32 T = tile > 0 ? u32(tile) : 256u;
    if (T > c) T = u32(c);
    MigArgs a;
    a.src = src;
    a.slog2 = src_log2;
    a.dst = dst;
    a.dlog2 = dst_log2;
    a.st = st;
    a.border = border;
    a.tile = T;
    a.start_cap = migrate_start_cap(T, windows);
    const u64 ntiles = c / T;
    u64 bgrid = (ntiles + 255) / 256;
    const u64 bcap = u64(sm_count()) * 8;
    if (bgrid > bcap) bgrid = bcap;
    migrate_border_kernel<<<unsigned(bgrid), 256, 0, s>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = migrate_smem_bytes(a.start_cap);
    const void* fn = windows ? reinterpret_cast<const void*>(migrate_window_kernel)
                             : reinterpret_cast<const void*>(migrate_walk_kernel);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMigBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    u64 grid = u64(sm_count()) * per_sm;
    const u64 need = (ntiles + kMigWarps - 1) / kMigWarps;
    if (grid > need) grid = need;
    if (windows)
        migrate_window_kernel<<<unsigned(grid), kMigBlock, smem, s>>>(a);
    else
        migrate_walk_kernel<<<unsigned(grid), kMigBlock, smem, s>>>(a);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    migrate_fallback_kernel<<<1, kMigBlock, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_export(const Cell* cells, u32 log2c, u64* keys_out, u64* vals_out, u64 max_n,
                          DevState* st, cudaStream_t s) {
    const u64 c = 1ull << log2c;
    u64 grid = (c + 255) / 256;
    const u64 cap = u64(sm_count()) * 8;
    if (grid > cap) grid = cap;
    export_kernel<<<unsigned(grid), 256, 0, s>>>(cells, c, keys_out, vals_out, max_n, st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cht
