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
#include "cht_internal.h"

namespace cht {
namespace {

constexpr int kMigBlock = 256;
constexpr int kMigWarps = kMigBlock / 32;
constexpr u32 kMaxScan = 1u << 16;      // longest overhang of a tile's last cluster
constexpr u32 kMapCells = 2048;        // per warp: owned ranges written through the map
constexpr u32 kRegionWords = 1024;     // per warp: map (2048 x u16) or a 32768-cell bitmap
constexpr u32 kSmallBitWords = kMapCells / 32;
constexpr u64 kNoBorder = ~0ull;

struct MigArgs {
    const Cell* src;
    u32 slog2;
    Cell* dst;
    u32 dlog2;
    DevState* st;
    u64* border;     // m(d) of every tile (scratch, ntiles entries)
    u32 tile;        // T, power of two, <= c
    u32 start_cap;   // per-warp capacity of the cluster-start list (walk kernel)
};

__device__ __forceinline__ u64 ld_key_nc(const Cell* p) {
    u64 k;
    asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(k) : "l"(p));
    return k;
}

// m(d) for every tile: d itself if cell d-1 is empty, else one past the
// first empty cell >= d (unwrapped: may exceed c for the last tiles).
__global__ void __launch_bounds__(256) migrate_border_kernel(MigArgs a) {
    const u64 c = 1ull << a.slog2, cmask = c - 1;
    const u64 ntiles = c / a.tile;
    for (u64 t = u64(blockIdx.x) * blockDim.x + threadIdx.x; t < ntiles; t += u64(gridDim.x) * blockDim.x) {
        const u64 d = t * a.tile;
        u64 m = kNoBorder;
        if (ld_key_nc(a.src + ((d - 1) & cmask)) == kEmpty) {
            m = d;
        } else {
            const u64 lim = c < kMaxScan ? c : kMaxScan;
            for (u64 i = d; i < d + lim; i += 2) {
                u64 k0, v0, k1, v1;
                ld_pair_nc(a.src + (i & cmask), k0, v0, k1, v1);  // d is even: pairs stay aligned
                if (k0 == kEmpty) { m = i + 1; break; }
                if (k1 == kEmpty) { m = i + 2; break; }
            }
        }
        if (m == kNoBorder) atomicOr(&a.st->mig_fail, 1u);
        a.border[t] = m;
    }
}

__device__ __forceinline__ u64 warp_sum(u64 x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Re-insertion of one window of 32 consecutive source cells (lane i holds
// source offset off - lane + i) in source order, exactly as a sequential
// migration would.  A live lane's candidate is the first free cell >= its new
// home; lanes with the same candidate form a group, and the group's m-th lane
// (in lane order) proposes the m-th free cell from the candidate on.  Taken in
// lane order, a proposal is the sequential placement if no earlier lane
// proposes the same cell: the cells from the lane's home to its candidate were
// taken before the window, the first m free ones after it go to the group's
// earlier lanes, and every earlier lane takes its own, different, proposal.
// So each round commits every pending lane below the first lane whose
// proposal repeats an earlier one (at least the lowest pending lane); the
// others look again from their candidate.  Sets `fail` if an element found no
// free cell in the owned range, which Lemma 1 rules out for a consistent
// table (the caller then leaves the migration to the fallback).
//
// Owned ranges of up to 32768 cells: the range's occupancy bitmap `bm` is in
// shared memory and offsets are 32-bit; MODE 0 records the source offset of
// each placed cell in `map`, MODE 1 stores the cell directly.
template <int MODE>
__device__ __forceinline__ void place_window_smem(u32* bm, unsigned short* map, Cell* dst, u64 tbase, u64 nmask,
                                                  u32 tl, u32 dshift, u64 k, u64 v, bool valid, u32 off, int lane,
                                                  u32& moved, bool& fail) {
    const bool live = valid && !is_reserved(k);
    u32 loc = 0;
    if (live) {
        const u64 o = (home_of(k, dshift) - tbase) & nmask;
        if (o < tl) loc = u32(o);
        else fail = true;  // outside the owned range: inconsistent source
    }
    u32 pending = __ballot_sync(0xffffffffu, live && !fail);
    const u32 below = (1u << lane) - 1u;
    const u32 wend = (tl + 31) >> 5;
    const volatile u32* vbm = bm;
    while (pending) {
        const bool mine = (pending >> lane) & 1u;
        // candidate: the first free cell >= loc (loc < tl for every lane)
        u32 w = loc >> 5;
        u32 bits = ~vbm[w] & (~0u << (loc & 31));
        if (mine)
            while (bits == 0 && ++w < wend) bits = ~vbm[w];
        const u32 c = bits ? (w << 5) + u32(__ffs(bits) - 1) : tl;
        // sentinels (bit 31 set) never match a real cell offset (< 2^15)
        const u32 cand = mine ? c : (0x80000000u | u32(lane));
        const u32 m = __popc(__match_any_sync(0xffffffffu, cand) & below);
        u32 prop = cand;
        // no shared candidate: every pending lane's candidate is its placement
        const bool grouped = __any_sync(0xffffffffu, mine && m != 0u);
        if (mine && m != 0u && c < tl) {
            // the m-th free cell after c: drop c, then skip m - 1 free cells
            u32 r = m;
            bits &= bits - 1u;
            for (;;) {
                const u32 cnt = __popc(bits);
                if (r <= cnt) {
                    for (; r > 1u; --r) bits &= bits - 1u;
                    prop = (w << 5) + u32(__ffs(bits) - 1);
                    break;
                }
                r -= cnt;
                if (++w >= wend) {
                    prop = tl;
                    break;
                }
                bits = ~vbm[w];
            }
        }
        // (every lane takes part in both votes: neither sits behind a lane
        // branch; `grouped` is the same for the whole warp)
        u32 commit = pending;
        if (grouped) {
            const u32 psame = __match_any_sync(0xffffffffu, prop);
            const u32 dups = __ballot_sync(0xffffffffu, mine && (psame & below) != 0u);
            commit = pending & ((dups & (0u - dups)) - 1u);  // all pending lanes if dups == 0
        }
        if ((commit >> lane) & 1u) {
            if (prop < tl) {
                atomicOr(&bm[prop >> 5], 1u << (prop & 31));
                if (MODE == 0) {
                    map[prop] = (unsigned short)off;
                } else {
                    Cell cl;
                    cl.key = k;
                    cl.val = v;
                    dst[(tbase + prop) & nmask] = cl;
                }
                ++moved;
            } else {
                fail = true;
            }
        }
        if (mine && c < tl) loc = c;
        pending &= ~commit;
        __syncwarp();
    }
}

// The same for owned ranges beyond the shared bitmap (a table grown by a
// large factor, or clusters of tens of thousands of cells): the target cells
// themselves, read from L2, are the occupancy, and offsets are 64-bit.
__device__ __forceinline__ void place_window_global(Cell* dst, u64 tbase, u64 nmask, u64 tl, u32 dshift, u64 k,
                                                    u64 v, bool valid, int lane, u64& moved, bool& fail) {
    const bool live = valid && !is_reserved(k);
    u64 loc = live ? ((home_of(k, dshift) - tbase) & nmask) : 0;
    if (live && loc >= tl) fail = true;
    u32 pending = __ballot_sync(0xffffffffu, live && !fail);
    const u32 below = (1u << lane) - 1u;
    while (pending) {
        const bool mine = (pending >> lane) & 1u;
        u64 cand = ~0ull - u64(lane);  // never a real candidate: those are < tl
        if (mine) {
            for (; loc < tl; ++loc) {
                u64 tk, tv;
                ld_cell_cg(dst + ((tbase + loc) & nmask), tk, tv);
                if (tk == kEmpty) break;
            }
            cand = loc;
        }
        const u32 same = __match_any_sync(0xffffffffu, cand);
        const u32 dups = __ballot_sync(0xffffffffu, mine && (same & below) != 0u);
        const u32 commit = pending & ((dups & (0u - dups)) - 1u);
        if ((commit >> lane) & 1u) {
            if (cand < tl) {
                Cell cl;
                cl.key = k;
                cl.val = v;
                dst[(tbase + cand) & nmask] = cl;
                ++moved;
            } else {
                fail = true;
            }
        }
        pending &= ~commit;
        __syncwarp();
    }
}

// The placement pass of one tile: source cells [m0, m0 + L) in order, 64 per
// step (two windows), the next 64 loading while these are placed.  MODE 0
// needs only the keys here (the write pass gathers whole cells).
template <int MODE>
__device__ __forceinline__ bool place_range(const MigArgs& a, u32* bm, unsigned short* map, u64 m0, u64 L,
                                            u64 tbase, u64 tl, int lane, u64& moved) {
    const u64 cmask = (1ull << a.slog2) - 1, nmask = (1ull << a.dlog2) - 1;
    const u32 dshift = 64u - a.dlog2;
    bool fail = false;
    u64 k0 = 0, v0 = 0, k1 = 0, v1 = 0;
    auto load = [&](u64 j, u64& k, u64& v) {
        if (j < L) {
            if (MODE == 0) k = ld_key_nc(a.src + ((m0 + j) & cmask));
            else ld_cell_nc(a.src + ((m0 + j) & cmask), k, v);
        }
    };
    load(lane, k0, v0);
    load(32 + lane, k1, v1);
    for (u64 j = 0; j < L; j += 64) {
        u64 n0 = 0, w0 = 0, n1 = 0, w1 = 0;
        load(j + 64 + lane, n0, w0);
        load(j + 96 + lane, n1, w1);
        if (MODE < 2) {
            u32 mv = 0;
            place_window_smem<MODE>(bm, map, a.dst, tbase, nmask, u32(tl), dshift, k0, v0, j + lane < L,
                                    u32(j + lane), lane, mv, fail);
            place_window_smem<MODE>(bm, map, a.dst, tbase, nmask, u32(tl), dshift, k1, v1, j + 32 + lane < L,
                                    u32(j + 32 + lane), lane, mv, fail);
            moved += mv;
        } else {
            place_window_global(a.dst, tbase, nmask, tl, dshift, k0, v0, j + lane < L, lane, moved, fail);
            place_window_global(a.dst, tbase, nmask, tl, dshift, k1, v1, j + 32 + lane < L, lane, moved, fail);
        }
        if (__any_sync(0xffffffffu, fail)) return true;
        k0 = n0;
        v0 = w0;
        k1 = n1;
        v1 = w1;
    }
    return false;
}

// The part of a tile that every migration kernel shares: its source range
// [m0, m0 + L) of whole clusters, its owned target range [tbase, tbase + tl)
// and how that range is written (0: source-offset map, 1: shared bitmap and
// direct stores, 2: global probing).  False if the tile owns nothing.
struct Tile {
    u64 m0, L, tl, tbase, sl;  // sl: cells of [m0, d + T) where clusters can start
    int mode;
};

__device__ __forceinline__ bool tile_of(const MigArgs& a, u64 t, u64 ntiles, Tile& x) {
    const u64 c = 1ull << a.slog2;
    const u64 m0 = a.border[t];
    const u64 b1 = t + 1 < ntiles ? a.border[t + 1] : a.border[0];
    if (m0 == kNoBorder || b1 == kNoBorder) return false;  // fallback redoes everything
    const u64 m1 = t + 1 < ntiles ? b1 : b1 + c;
    if (m1 <= m0) return false;  // the tile lies inside a cluster owned by an earlier tile
    const u32 g = a.dlog2 - a.slog2;
    const u64 dT = (t + 1) * u64(a.tile);
    x.m0 = m0;
    x.L = m1 - m0;
    x.tl = x.L << g;
    x.tbase = m0 << g;
    x.sl = (m1 < dT ? m1 : dT) - m0;
    x.mode = x.tl <= kMapCells ? 0 : (x.tl <= u64(kRegionWords) * 32 ? 1 : 2);
    return true;
}

// Clears the owned range's bitmap (modes 0, 1) or zero-fills its target
// cells (mode 2) before placement.
__device__ __forceinline__ void clear_owned(const MigArgs& a, const Tile& x, u32* bm, int lane) {
    const u64 nmask = (1ull << a.dlog2) - 1;
    if (x.mode < 2) {
        const u32 words = u32((x.tl + 31) / 32);
        for (u32 w = lane; w < words; w += 32) bm[w] = 0;
    } else {
        const Cell zero = {0ull, 0ull};
        for (u64 k = lane; k < x.tl; k += 32) a.dst[(x.tbase + k) & nmask] = zero;
    }
    __syncwarp();
}

// Writes the owned target range after placement: mode 0 every cell once
// (placed cells gathered from the source through the map, four gathers in
// flight per lane, the rest zero), mode 1 the zero cells.
__device__ __forceinline__ void write_owned(const MigArgs& a, const Tile& x, const u32* bm,
                                            const unsigned short* map, int lane) {
    const u64 cmask = (1ull << a.slog2) - 1, nmask = (1ull << a.dlog2) - 1;
    const Cell zero = {0ull, 0ull};
    __syncwarp();
    if (x.mode == 0) {
        const u32 tl = u32(x.tl);
        for (u32 k0 = 0; k0 < tl; k0 += 128) {
            Cell cl[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const u32 k = k0 + u * 32 + lane;
                cl[u] = zero;
                if (k < tl && ((bm[k >> 5] >> (k & 31)) & 1u))
                    ld_cell_nc(a.src + ((x.m0 + map[k]) & cmask), cl[u].key, cl[u].val);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const u32 k = k0 + u * 32 + lane;
                if (k < tl) a.dst[(x.tbase + k) & nmask] = cl[u];
            }
        }
    } else if (x.mode == 1) {
        for (u64 k = lane; k < x.tl; k += 32)
            if (!((bm[k >> 5] >> (k & 31)) & 1u)) a.dst[(x.tbase + k) & nmask] = zero;
    }
    __syncwarp();
}

// Migration by windows (tables at load >= 0.6, where clusters are long): the
// warp places the tile's cells 32 at a time in source order (place_range).
__global__ void __launch_bounds__(kMigBlock, 5) migrate_window_kernel(MigArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // per warp: a region of kRegionWords words (the source-offset map of a
    // short owned range, or the occupancy bitmap of a long one) and the
    // small bitmap of the map mode
    u32* const region = reinterpret_cast<u32*>(smem) + wib * (kRegionWords + kSmallBitWords);
    unsigned short* const map = reinterpret_cast<unsigned short*>(region);
    u32* const small_bm = region + kRegionWords;
    const u64 ntiles = (1ull << a.slog2) / a.tile;
    const u64 nwarps = u64(gridDim.x) * kMigWarps;
    u64 moved = 0;
    bool bad = false;
    for (u64 t = u64(blockIdx.x) * kMigWarps + wib; t < ntiles && !bad; t += nwarps) {
        Tile x;
        if (!tile_of(a, t, ntiles, x)) continue;
        u32* const bm = x.mode == 0 ? small_bm : region;
        clear_owned(a, x, bm, lane);
        if (x.mode == 0)
            bad = place_range<0>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        else if (x.mode == 1)
            bad = place_range<1>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        else
            bad = place_range<2>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        if (bad) break;
        write_owned(a, x, bm, map, lane);
    }
    if (bad && lane == 0) atomicOr(&a.st->mig_fail, 2u);
    moved = warp_sum(moved);
    if (lane == 0 && moved) atomicAdd(&a.st->I, moved);
}

// Migration by clusters (tables below load 0.6, where clusters are short and
// many): each lane re-inserts whole clusters of the tile in source order.
// The tile's keys are read with all loads in flight (eight 32-cell chunks at
// a time) and the cluster starts -- a live cell after an empty one -- come
// from ballots of the empties; the walks then read cells the scan has just
// brought into L1.  Lanes own disjoint target ranges by Lemma 1, so a lane
// only ever claims its own cells.
__global__ void __launch_bounds__(kMigBlock, 5) migrate_walk_kernel(MigArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    u32* const region = reinterpret_cast<u32*>(smem) + wib * (kRegionWords + kSmallBitWords);
    unsigned short* const map = reinterpret_cast<unsigned short*>(region);
    u32* const small_bm = region + kRegionWords;
    unsigned short* const starts =
        reinterpret_cast<unsigned short*>(reinterpret_cast<u32*>(smem) + kMigWarps * (kRegionWords + kSmallBitWords)) +
        wib * a.start_cap;

    const u64 cmask = (1ull << a.slog2) - 1;
    const u64 nmask = (1ull << a.dlog2) - 1;
    const u32 dshift = 64u - a.dlog2;
    const u32 below = (1u << lane) - 1u;
    const u64 ntiles = (1ull << a.slog2) / a.tile;
    const u64 nwarps = u64(gridDim.x) * kMigWarps;
    u64 moved = 0;
    int bad = 0;

    for (u64 t = u64(blockIdx.x) * kMigWarps + wib; t < ntiles; t += nwarps) {
        Tile x;
        if (!tile_of(a, t, ntiles, x)) continue;
        u32* const bm = x.mode == 0 ? small_bm : region;
        clear_owned(a, x, bm, lane);

        // ---- cluster starts in [m0, m0 + sl); cell m0 - 1 is empty
        u32 ns = 0, carry = 1u;
        for (u64 j0 = 0; j0 < x.sl; j0 += 256) {
            u64 key[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const u64 j = j0 + q * 32 + lane;
                key[q] = j < x.sl ? ld_key_nc(a.src + ((x.m0 + j) & cmask)) : kEmpty;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (j0 + q * 32 >= x.sl) break;
                const u32 e = __ballot_sync(0xffffffffu, key[q] == kEmpty);  // past sl counts as empty
                const u32 st = ~e & ((e << 1) | carry);
                carry = e >> 31;
                if ((st >> lane) & 1u) starts[ns + __popc(st & below)] = (unsigned short)(j0 + q * 32 + lane);
                ns += __popc(st);
            }
        }
        __syncwarp();

        // ---- one lane per cluster: re-insert its live cells in index order
        const u64 tl = x.tl, tbase = x.tbase;
        for (u32 q = lane; q < ns && !bad; q += 32) {
            for (u64 i = x.m0 + starts[q];; ++i) {
                u64 k, v;
                ld_cell_nc(a.src + (i & cmask), k, v);
                if (k == kEmpty) break;
                if (k == kTomb) continue;
                u64 loc = (home_of(k, dshift) - tbase) & nmask;
                if (loc >= tl) {
                    bad = 1;
                    break;
                }
                if (x.mode < 2) {
                    // first free bit >= loc (bits of other lanes' ranges are
                    // never in this cluster's window, so a plain read is safe)
                    u32 w = u32(loc >> 5);
                    u32 free = ~reinterpret_cast<volatile u32*>(bm)[w] & (~0u << (loc & 31));
                    while (free == 0 && u64(w + 1) * 32 < tl) {
                        ++w;
                        free = ~reinterpret_cast<volatile u32*>(bm)[w];
                    }
                    loc = u64(w) * 32 + (free ? u32(__ffs(free) - 1) : 32u);
                    if (free == 0 || loc >= tl) {
                        bad = 1;
                        break;
                    }
                    atomicOr(&bm[w], 1u << (loc & 31));
                    if (x.mode == 0) {
                        map[loc] = (unsigned short)(i - x.m0);
                    } else {
                        Cell cl;
                        cl.key = k;
                        cl.val = v;
                        a.dst[(tbase + loc) & nmask] = cl;
                    }
                } else {
                    for (;; ++loc) {
                        if (loc >= tl) {
                            bad = 1;
                            break;
                        }
                        u64 tk, tv;
                        ld_cell_cg(a.dst + ((tbase + loc) & nmask), tk, tv);
                        if (tk == kEmpty) break;
                    }
                    if (bad) break;
                    Cell cl;
                    cl.key = k;
                    cl.val = v;
                    a.dst[(tbase + loc) & nmask] = cl;
                }
                ++moved;
            }
        }
        if (__any_sync(0xffffffffu, bad)) {
            bad = 1;
            break;
        }
        write_owned(a, x, bm, map, lane);
    }
    if (bad && lane == 0) atomicOr(&a.st->mig_fail, 2u);
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
    a.start_cap = windows ? 0u : (T / 2 + 8 + 7) & ~7u;
    const u64 ntiles = c / T;
    u64 bgrid = (ntiles + 255) / 256;
    const u64 bcap = u64(sm_count()) * 8;
    if (bgrid > bcap) bgrid = bcap;
    migrate_border_kernel<<<unsigned(bgrid), 256, 0, s>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = size_t(kMigWarps) * ((kRegionWords + kSmallBitWords) * 4 + size_t(a.start_cap) * 2);
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
