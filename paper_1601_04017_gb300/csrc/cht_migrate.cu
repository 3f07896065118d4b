// Cluster-wise parallel migration (Sec. 4.3.1, Lemma 1; tombstone purge,
// Sec. 4.4) and the forall/export compaction (Sec. 3 "Bulk Operations").
//
// Migration into a table gamma = 2^g times larger (g >= 0).  The source is
// cut into tiles of T cells, one CTA per tile (grid-stride).  Tile [d, d+T)
// moves its borders to just after the next empty cell: m(d) = d if cell d-1
// is empty, else (first empty cell >= d) + 1.  The CTA migrates the source
// range [m(d), m(d+T)), which consists of whole clusters, and owns the target
// range [gamma*m(d), gamma*m(d+T)).  By Lemma 1 a cluster a..b lands inside
// gamma*a .. gamma*(b+1)-1 (the integer-gamma form of the lemma's bound), so
// the owned target ranges of different tiles are disjoint and together cover
// the target table: no atomics and no separate initialisation are needed --
// each CTA writes every cell of its range, empties included (the paper's
// "each thread is responsible for initializing all cells in its region").
// Inside the CTA each cluster is re-inserted by one thread in source index
// order, so the layout equals the sequential migration (Lemma 1).
//
// The target range is staged in shared memory when it fits (the common case:
// about gamma*T cells) and written out with coalesced stores; otherwise the
// CTA zero-fills it in global memory and inserts there directly.  A border
// scan that finds no empty cell within kMaxScan cells sets mig_fail; a
// single-CTA fallback kernel, always launched after the tile kernel, then
// redoes the whole migration sequentially (only for pathological tables:
// full, or with a cluster longer than kMaxScan cells).
#include "cht_internal.h"

namespace cht {
namespace {

constexpr int kMigBlock = 256;
constexpr u32 kMaxScan = 1u << 16;  // longest cluster overhang a tile CTA handles

struct MigArgs {
    const Cell* src;
    u32 slog2;
    Cell* dst;
    u32 dlog2;
    DevState* st;
    u32 tile;       // T, power of two, <= source capacity
    u32 tgt_cap;    // cells of shared-memory target staging (0 = global only)
    u32 bm_words;   // 32-bit words of the cluster-start bitmask
};

__device__ __forceinline__ u64 warp_sum(u64 x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kMigBlock) migrate_kernel(MigArgs a) {
    extern __shared__ uint4 smem[];
    Cell* s_src = reinterpret_cast<Cell*>(smem);
    Cell* s_tgt = s_src + a.tile;
    u32* s_bm = reinterpret_cast<u32*>(s_tgt + a.tgt_cap);
    __shared__ u64 s_m0, s_m1;
    __shared__ u32 s_first_empty;
    __shared__ int s_fail;
    __shared__ u64 s_part[kMigBlock / 32];

    const u64 c = 1ull << a.slog2, cmask = c - 1;
    const u64 nc = 1ull << a.dlog2, nmask = nc - 1;
    const u32 g = a.dlog2 - a.slog2;
    const u32 dshift = 64u - a.dlog2;
    const u32 T = a.tile;
    const u64 ntiles = c / T;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const u64 d = tile * T;
        if (tid == 0) {
            s_first_empty = 0xffffffffu;
            s_fail = 0;
        }
        // ---- stage the source tile (two cells per 256-bit load)
        for (u32 i = tid; i < T / 2; i += kMigBlock) {
            u64 k0, v0, k1, v1;
            ld_pair_nc(a.src + d + 2 * i, k0, v0, k1, v1);
            s_src[2 * i].key = k0;
            s_src[2 * i].val = v0;
            s_src[2 * i + 1].key = k1;
            s_src[2 * i + 1].val = v1;
        }
        __syncthreads();
        for (u32 i = tid; i < T; i += kMigBlock)
            if (s_src[i].key == kEmpty) atomicMin(&s_first_empty, i);
        __syncthreads();

        // ---- moved borders m(d) and m(d+T)
        if (wid == 0) {
            const bool prev_empty = a.src[(d - 1) & cmask].key == kEmpty;
            u64 m0, m1 = 0;
            bool own = true;
            if (prev_empty) {
                m0 = d;
            } else if (s_first_empty != 0xffffffffu) {
                m0 = d + s_first_empty + 1;
            } else {
                own = false;  // the whole tile lies inside a cluster begun earlier
                m0 = 0;
            }
            int fail = 0;
            if (!own) {
                // The tile lies inside a cluster that starts before it; the
                // owner of that cluster is an earlier tile, whose forward
                // border scan fails if the cluster outruns it.  If no empty
                // cell precedes the tile within the scan bound, no tile may
                // own the cluster (a full table): report it.
                bool found = false;
                for (u32 off = 0; off < kMaxScan && off < c; off += 32) {
                    const u64 i = d - 1 - off - lane;
                    const bool e = a.src[i & cmask].key == kEmpty;
                    if (__ballot_sync(0xffffffffu, e)) {
                        found = true;
                        break;
                    }
                }
                if (!found) fail = 1;
            }
            if (own) {
                if (s_src[T - 1].key == kEmpty) {
                    m1 = d + T;
                } else {
                    bool found = false;
                    for (u32 off = 0; off < kMaxScan && off < c; off += 32) {
                        const u64 i = d + T + off + lane;
                        const bool e = a.src[i & cmask].key == kEmpty;
                        const u32 b = __ballot_sync(0xffffffffu, e);
                        if (b) {
                            m1 = d + T + off + (__ffs(b) - 1) + 1;
                            found = true;
                            break;
                        }
                    }
                    if (!found) fail = 1;
                }
                if (!fail && m1 < m0) m1 = m0;
            }
            if (lane == 0) {
                s_m0 = own ? m0 : 0;
                s_m1 = own ? m1 : 0;
                s_fail = fail;
            }
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) atomicOr(&a.st->mig_fail, 1u);
            __syncthreads();
            continue;
        }
        const u64 m0 = s_m0, m1 = s_m1;
        const u64 L = m1 - m0;          // source cells of this CTA's clusters
        const u64 tl = L << g;          // owned target cells
        const u64 tbase = m0 << g;      // first owned target cell (unwrapped)
        u64 moved = 0;
        if (L > 0) {
            const bool staged = tl <= a.tgt_cap;
            // source cell i (unwrapped index >= d - 1)
            auto src_key = [&](u64 i) -> u64 {
                return (i >= d && i < d + T) ? s_src[i - d].key : a.src[i & cmask].key;
            };
            auto src_cell = [&](u64 i) -> Cell {
                return (i >= d && i < d + T) ? s_src[i - d] : a.src[i & cmask];
            };
            int bad = 0;
            if (staged) {
                // zero the staged target range and the cluster-start bitmask
                const u32 words = u32((L + 31) / 32);
                for (u32 w = tid; w < words; w += kMigBlock) s_bm[w] = 0;
                for (u64 i = tid; i < tl; i += kMigBlock) {
                    s_tgt[i].key = 0;
                    s_tgt[i].val = 0;
                }
                __syncthreads();
                // cluster starts: a non-empty cell whose predecessor is empty
                for (u64 j = tid; j < L; j += kMigBlock) {
                    const u64 i = m0 + j;
                    if (src_key(i) != kEmpty && src_key(i - 1) == kEmpty)
                        atomicOr(&s_bm[j >> 5], 1u << (j & 31));
                }
                __syncthreads();
                // each thread takes 32-cell words of the bitmask and re-inserts
                // the clusters that start there, in source index order
                for (u32 w = tid; w < words; w += kMigBlock) {
                    u32 bits = s_bm[w];
                    while (bits) {
                        const u32 b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        for (u64 j = u64(w) * 32 + b; j < L; ++j) {
                            const Cell cl = src_cell(m0 + j);
                            if (cl.key == kEmpty) break;
                            if (cl.key == kTomb) continue;
                            u64 loc = (home_of(cl.key, dshift) - tbase) & nmask;
                            while (loc < tl && s_tgt[loc].key != kEmpty) ++loc;
                            if (loc >= tl) {
                                bad = 1;
                                break;
                            }
                            s_tgt[loc] = cl;
                            ++moved;
                        }
                    }
                }
                __syncthreads();
                for (u64 i = tid; i < tl; i += kMigBlock) a.dst[(tbase + i) & nmask] = s_tgt[i];
            } else {
                // long range or large gamma: zero-fill the owned target range
                // in global memory, then each thread re-inserts the clusters
                // that start in its own contiguous chunk of the source range
                for (u64 i = tid; i < tl; i += kMigBlock) {
                    Cell z;
                    z.key = 0;
                    z.val = 0;
                    a.dst[(tbase + i) & nmask] = z;
                }
                __syncthreads();
                const u64 ch = (L + kMigBlock - 1) / kMigBlock;
                const u64 lo = u64(tid) * ch;
                const u64 hi = lo + ch < L ? lo + ch : L;
                for (u64 s0 = lo; s0 < hi; ++s0) {
                    if (!(src_key(m0 + s0) != kEmpty && src_key(m0 + s0 - 1) == kEmpty)) continue;
                    for (u64 j = s0; j < L; ++j) {
                        const Cell cl = src_cell(m0 + j);
                        if (cl.key == kEmpty) break;
                        if (cl.key == kTomb) continue;
                        u64 loc = (home_of(cl.key, dshift) - tbase) & nmask;
                        while (loc < tl && a.dst[(tbase + loc) & nmask].key != kEmpty) ++loc;
                        if (loc >= tl) {
                            bad = 1;
                            break;
                        }
                        a.dst[(tbase + loc) & nmask] = cl;
                        ++moved;
                    }
                }
            }
            if (bad) atomicOr(&a.st->mig_fail, 2u);
        }
        // ---- moved-element count -> new I
        moved = warp_sum(moved);
        if (lane == 0) s_part[wid] = moved;
        __syncthreads();
        if (tid == 0) {
            u64 tot = 0;
            for (int w = 0; w < kMigBlock / 32; ++w) tot += s_part[w];
            if (tot) atomicAdd(&a.st->I, tot);
        }
        __syncthreads();
    }
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
                           int tile, cudaStream_t s) {
    const u64 c = 1ull << src_log2;
    u32 T = tile > 0 ? u32(tile) : 2048u;
    if (T > c) T = u32(c);
    if (T < 64) T = 64;
    const u32 g = dst_log2 - src_log2;
    // shared memory: source tile + target staging + start bitmask
    // staged target: the tile plus a margin for clusters running past its
    // end, times gamma; the bitmask covers the staged source range
    const u32 span = T + T / 8 + 64;
    const u32 bm_words = span / 32 + 1;
    const size_t fixed = size_t(T) * sizeof(Cell) + size_t(bm_words) * 4;
    const size_t budget = 200 * 1024;
    u64 want = (g <= 3) ? (u64(span) << g) : 0;
    if (fixed + want * sizeof(Cell) > budget) want = 0;
    MigArgs a;
    a.src = src;
    a.slog2 = src_log2;
    a.dst = dst;
    a.dlog2 = dst_log2;
    a.st = st;
    a.tile = T;
    a.tgt_cap = u32(want);
    a.bm_words = bm_words;
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
