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
// atomics and no separate initialisation -- each tile writes every cell of
// its range, empties included (the paper's "each thread is responsible for
// initializing all cells in its region").  Each cluster is re-inserted by one
// thread in source index order, so the layout equals the sequential
// migration (Lemma 1).
//
// GB300 mapping.  Persistent CTAs walk the tiles.  The copy engine (TMA,
// untiled bulk copies) brings the window [d-1, d+T+H) -- the tile, its
// predecessor cell and a halo of H cells -- into one of two shared buffers
// while the CTA works on the previous tile (mbarrier completion, bounded
// waits).  Cluster starts are compacted into a list so every thread inserts.
// The owned target range is staged in shared memory (the part beyond the
// staging capacity goes straight to global memory) and written back by a
// bulk store.  A border scan that finds no empty cell within kMaxScan cells,
// or a bulk-copy wait that runs out, sets mig_fail; a single-CTA fallback
// kernel, always launched after the tile kernel, then redoes the whole
// migration sequentially (only for pathological tables: full, or with a
// cluster longer than kMaxScan cells).
#include "cht_internal.h"
#include "cht_tma.cuh"

namespace cht {
namespace {

constexpr int kMigBlock = 256;
constexpr u32 kMaxScan = 1u << 16;  // longest cluster overhang a tile CTA handles
constexpr u32 kMigTimeoutBit = 16u;
constexpr long long kDrainLimit = 4000000000ll;  // cycles to wait for copies in flight

struct MigArgs {
    const Cell* src;
    u32 slog2;
    Cell* dst;
    u32 dlog2;
    DevState* st;
    u32 tile;        // T, power of two, <= c/2
    u32 halo;        // H cells after the tile brought in with it
    u32 lw_pad;      // cells per window buffer (T + H + 1 rounded up to 8)
    u32 tgt_cap;     // cells of shared-memory target staging
    long long wait_limit;  // bound of one bulk-copy wait, in clock cycles
    int inject_stall;      // testing: wait once on a barrier nothing arrives on
};

__device__ __forceinline__ u64 warp_sum(u64 x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kMigBlock) migrate_kernel(MigArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    Cell* const buf0 = reinterpret_cast<Cell*>(smem);
    Cell* const buf1 = buf0 + a.lw_pad;
    Cell* const tgt = buf1 + a.lw_pad;
    u32* const starts = reinterpret_cast<u32*>(tgt + a.tgt_cap);
    __shared__ unsigned long long bars[3];
    __shared__ u64 s_m0, s_m1;
    __shared__ u32 s_first_tile, s_first_halo, s_nstarts;
    __shared__ int s_fail, s_timeout;

    const u64 c = 1ull << a.slog2, cmask = c - 1;
    const u64 nc = 1ull << a.dlog2, nmask = nc - 1;
    const u32 g = a.dlog2 - a.slog2;
    const u32 dshift = 64u - a.dlog2;
    const u32 T = a.tile, H = a.halo, Lw = T + H + 1;
    const u64 ntiles = c / T;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    u64 moved = 0;
    int bad = 0;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // thread 0: bring the window [d-1, d+T+H) of tile `t` into buffer `b`
    auto issue = [&](u64 t, int b) {
        Cell* dstb = b ? buf1 : buf0;
        const u64 s0 = (t * T - 1) & cmask;
        u64 first = c - s0;
        if (first > Lw) first = Lw;
        mbar_arrive_expect_tx(&bars[b], Lw * 16u);
        bulk_g2s(dstb, a.src + s0, u32(first * 16), &bars[b]);
        if (first < Lw) bulk_g2s(dstb + first, a.src, u32((Lw - first) * 16), &bars[b]);
    };

    u32 parity = 0;  // bit b: parity of the next completion of bars[b]
    u64 tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) issue(tile, 0);
    int b = 0;
    for (; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const u64 d = tile * T;
        const u64 nt = tile + gridDim.x;
        if (tid == 0) {
            s_first_tile = 0xffffffffu;
            s_first_halo = 0xffffffffu;
            s_nstarts = 0;
            s_fail = 0;
            s_timeout = 0;
            if (nt < ntiles) {
                fence_proxy_async_smem();
                issue(nt, b ^ 1);
            }
        }
        __syncthreads();
        bool ok = true;
        if (a.inject_stall && tile == blockIdx.x) ok = mbar_wait_bounded(&bars[2], 0, a.wait_limit);
        if (ok) ok = mbar_wait_bounded(&bars[b], (parity >> b) & 1u, a.wait_limit);
        parity ^= 1u << b;
        if (!ok) s_timeout = 1;
        __syncthreads();
        if (s_timeout) {
            // give up: let the copies in flight land, then leave it to the fallback
            if (tid == 0) {
                atomicOr(&a.st->mig_fail, kMigTimeoutBit);
                atomicOr(&a.st->status, 4u);
                mbar_wait_bounded(&bars[b], ((parity >> b) & 1u) ^ 1u, kDrainLimit);
                if (nt < ntiles) mbar_wait_bounded(&bars[b ^ 1], (parity >> (b ^ 1)) & 1u, kDrainLimit);
                bulk_wait_all();
            }
            __syncthreads();
            return;
        }
        const Cell* w = b ? buf1 : buf0;  // w[k] = cell d - 1 + k
        auto key_at = [&](u64 i) -> u64 {  // unwrapped index i >= d - 1
            const u64 k = i - (d - 1);
            return k < Lw ? w[k].key : a.src[i & cmask].key;
        };
        auto cell_at = [&](u64 i) -> Cell {
            const u64 k = i - (d - 1);
            return k < Lw ? w[k] : a.src[i & cmask];
        };
        for (u32 k = 1 + tid; k < Lw; k += kMigBlock) {
            if (w[k].key == kEmpty) {
                if (k <= T) atomicMin(&s_first_tile, k - 1);
                else atomicMin(&s_first_halo, k - 1 - T);
            }
        }
        __syncthreads();

        // ---- moved borders m(d) and m(d+T) (warp 0)
        if (wid == 0) {
            u64 m0 = 0, m1 = 0;
            bool own = true;
            int fail = 0;
            if (w[0].key == kEmpty) m0 = d;
            else if (s_first_tile != 0xffffffffu) m0 = d + s_first_tile + 1;
            else own = false;  // the whole tile lies inside a cluster begun earlier
            if (!own) {
                // The owner of that cluster is an earlier tile, whose forward
                // border scan fails if the cluster outruns it.  If no empty
                // cell precedes the tile within the bound, no tile owns the
                // cluster (a full table): report it.
                bool found = false;
                for (u32 off = 0; off < kMaxScan && off < c; off += 32) {
                    const bool e = a.src[(d - 1 - off - lane) & cmask].key == kEmpty;
                    if (__ballot_sync(0xffffffffu, e)) {
                        found = true;
                        break;
                    }
                }
                if (!found) fail = 1;
            } else if (w[T].key == kEmpty) {
                m1 = d + T;
            } else if (s_first_halo != 0xffffffffu) {
                m1 = d + T + s_first_halo + 1;
            } else {
                bool found = false;
                for (u32 off = 0; off < kMaxScan && off < c; off += 32) {
                    const u64 i = d + T + H + off + lane;
                    const u32 bb = __ballot_sync(0xffffffffu, a.src[i & cmask].key == kEmpty);
                    if (bb) {
                        m1 = d + T + H + off + (__ffs(bb) - 1) + 1;
                        found = true;
                        break;
                    }
                }
                if (!found) fail = 1;
            }
            if (lane == 0) {
                s_m0 = own ? m0 : 0;
                s_m1 = own ? m1 : 0;
                s_fail = fail;
            }
        }
        // the previous tile's bulk store must have read the staging area
        if (tid == 0) bulk_wait_read_all();
        __syncthreads();
        if (s_fail) {
            if (tid == 0) atomicOr(&a.st->mig_fail, 1u);
            __syncthreads();  // everyone has read s_fail before thread 0 resets it
            continue;
        }
        const u64 m0 = s_m0, m1 = s_m1;
        const u64 L = m1 - m0;      // source cells of this tile's clusters
        const u64 tl = L << g;      // owned target cells
        const u64 tbase = m0 << g;  // first owned target cell (unwrapped)
        const u64 staged = tl < a.tgt_cap ? tl : a.tgt_cap;
        if (L > 0) {
            for (u64 k = tid; k < staged; k += kMigBlock) {
                tgt[k].key = 0;
                tgt[k].val = 0;
            }
            for (u64 k = staged + tid; k < tl; k += kMigBlock) {
                Cell z;
                z.key = 0;
                z.val = 0;
                a.dst[(tbase + k) & nmask] = z;
            }
            // cluster starts in [m0, min(m1, d+T)): non-empty after an empty
            const u64 sl = (m1 < d + T ? m1 : d + T) - m0;
            for (u64 j0 = u64(wid) * 32; j0 < sl; j0 += kMigBlock) {
                const u64 j = j0 + lane;
                const bool is_start = j < sl && key_at(m0 + j) != kEmpty && key_at(m0 + j - 1) == kEmpty;
                const u32 bb = __ballot_sync(0xffffffffu, is_start);
                u32 base = 0;
                if (lane == 0 && bb) base = atomicAdd(&s_nstarts, u32(__popc(bb)));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (is_start) starts[base + __popc(bb & ((1u << lane) - 1u))] = u32(j);
            }
            __syncthreads();
            // one thread per cluster: re-insert its live cells in index order
            const u32 ns = s_nstarts;
            for (u32 q = tid; q < ns && !bad; q += kMigBlock) {
                for (u64 i = m0 + starts[q];; ++i) {
                    const Cell cl = cell_at(i);
                    if (cl.key == kEmpty) break;
                    if (cl.key == kTomb) continue;
                    u64 loc = (home_of(cl.key, dshift) - tbase) & nmask;
                    for (;; ++loc) {
                        if (loc >= tl) {
                            bad = 1;
                            break;
                        }
                        if (loc < staged) {
                            if (tgt[loc].key == kEmpty) {
                                tgt[loc] = cl;
                                break;
                            }
                        } else {
                            Cell* gp = a.dst + ((tbase + loc) & nmask);
                            if (gp->key == kEmpty) {
                                *gp = cl;
                                break;
                            }
                        }
                    }
                    if (bad) break;
                    ++moved;
                }
            }
        }
        // write the staged target range back with a bulk store
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && staged > 0) {
            const u64 s0 = tbase & nmask;
            u64 first = nc - s0;
            if (first > staged) first = staged;
            bulk_s2g(a.dst + s0, tgt, u32(first * 16));
            if (first < staged) bulk_s2g(a.dst, tgt + first, u32((staged - first) * 16));
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
    if (bad) atomicOr(&a.st->mig_fail, 2u);
    moved = warp_sum(moved);
    if (lane == 0 && moved) atomicAdd(&a.st->I, moved);
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

}  // namespace

cudaError_t launch_migrate(const Cell* src, u32 src_log2, Cell* dst, u32 dst_log2, DevState* st,
                           int tile, long long wait_limit, int inject_stall, cudaStream_t s) {
    const u64 c = 1ull << src_log2;
    u32 T = tile > 0 ? u32(tile) : 1024u;
    if (T > 4096) T = 4096;  // two window buffers must fit in shared memory
    if (T > c / 2) T = u32(c / 2);
    u32 H = T / 4 < 64 ? 64 : T / 4;
    if (H > 256) H = 256;
    if (H > c / 4) H = u32(c / 4);
    const u32 g = dst_log2 - src_log2;
    const u32 lw_pad = (T + H + 1 + 7) & ~7u;
    const u32 start_cap = T / 2 + 32;
    // shared memory: two window buffers, the start list, the target staging
    const size_t fixed = 2 * size_t(lw_pad) * sizeof(Cell) + size_t(start_cap) * 4;
    const size_t budget = 100 * 1024;
    u64 want = g <= 4 ? (u64(T + H) << g) : 0;
    const u64 room = fixed < budget ? (budget - fixed) / sizeof(Cell) : 0;
    if (want > room) want = room;
    MigArgs a;
    a.src = src;
    a.slog2 = src_log2;
    a.dst = dst;
    a.dlog2 = dst_log2;
    a.st = st;
    a.tile = T;
    a.halo = H;
    a.lw_pad = lw_pad;
    a.tgt_cap = u32(want);
    a.wait_limit = wait_limit > 0 ? wait_limit : 2000000000ll;
    a.inject_stall = inject_stall;
    const size_t smem = fixed + size_t(a.tgt_cap) * sizeof(Cell);
    cudaError_t e = cudaFuncSetAttribute(migrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, migrate_kernel, kMigBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const u64 ntiles = c / T;
    u64 grid = u64(sm_count()) * per_sm;
    if (grid > ntiles) grid = ntiles;
    migrate_kernel<<<unsigned(grid), kMigBlock, smem, s>>>(a);
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
