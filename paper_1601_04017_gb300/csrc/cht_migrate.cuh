// Device-side pieces of the cluster-wise migration (Sec. 4.3.1, Lemma 1),
// shared by the migration kernels (cht_migrate.cu) and the persistent growing
// kernel (cht_grow.cu), which runs them between its operation rounds.  See
// cht_migrate.cu for the design.
#pragma once

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

// Source loads: the read-only path when the source was written before the
// launch (the migration kernels), L2 only (kCg) when it was written earlier
// in the same launch (the persistent growing kernel, whose SMs may hold stale
// lines of a buffer from an earlier round in their L1).
template <bool kCg>
__device__ __forceinline__ u64 src_key(const Cell* p) {
    if (kCg) {
        u64 k;
        asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(k) : "l"(p));
        return k;
    }
    return ld_key_nc(p);
}
template <bool kCg>
__device__ __forceinline__ void src_cell(const Cell* p, u64& k, u64& v) {
    if (kCg) ld_cell_cg(p, k, v);
    else ld_cell_nc(p, k, v);
}
template <bool kCg>
__device__ __forceinline__ void src_pair(const Cell* p, u64& k0, u64& v0, u64& k1, u64& v1) {
    if (kCg) ld_pair_cg(p, k0, v0, k1, v1);
    else ld_pair_nc(p, k0, v0, k1, v1);
}

// m(d) for every tile: d itself if cell d-1 is empty, else one past the
// first empty cell >= d (unwrapped: may exceed c for the last tiles).
// Threads first, first + stride, ... each take tiles in turn.
template <bool kCg = false>
__device__ __forceinline__ void migrate_borders(const MigArgs& a, u64 first, u64 stride) {
    const u64 c = 1ull << a.slog2, cmask = c - 1;
    const u64 ntiles = c / a.tile;
    for (u64 t = first; t < ntiles; t += stride) {
        const u64 d = t * a.tile;
        u64 m = kNoBorder;
        if (src_key<kCg>(a.src + ((d - 1) & cmask)) == kEmpty) {
            m = d;
        } else {
            const u64 lim = c < kMaxScan ? c : kMaxScan;
            for (u64 i = d; i < d + lim; i += 2) {
                u64 k0, v0, k1, v1;
                src_pair<kCg>(a.src + (i & cmask), k0, v0, k1, v1);  // d is even: pairs stay aligned
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
template <int MODE, bool kCg = false>
__device__ __forceinline__ bool place_range(const MigArgs& a, u32* bm, unsigned short* map, u64 m0, u64 L,
                                            u64 tbase, u64 tl, int lane, u64& moved) {
    const u64 cmask = (1ull << a.slog2) - 1, nmask = (1ull << a.dlog2) - 1;
    const u32 dshift = 64u - a.dlog2;
    bool fail = false;
    u64 k0 = 0, v0 = 0, k1 = 0, v1 = 0;
    auto load = [&](u64 j, u64& k, u64& v) {
        if (j < L) {
            if (MODE == 0) k = src_key<kCg>(a.src + ((m0 + j) & cmask));
            else src_cell<kCg>(a.src + ((m0 + j) & cmask), k, v);
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
template <bool kCg = false>
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
                    src_cell<kCg>(a.src + ((x.m0 + map[k]) & cmask), cl[u].key, cl[u].val);
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
// Warp `warp` of `nwarps` (wib: its index in the block, which picks its part
// of the block's shared memory `smem`) takes tiles warp, warp + nwarps, ...
template <bool kCg = false>
__device__ __forceinline__ void migrate_window_tiles(const MigArgs& a, unsigned char* smem, u64 warp, u64 nwarps) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // per warp: a region of kRegionWords words (the source-offset map of a
    // short owned range, or the occupancy bitmap of a long one) and the
    // small bitmap of the map mode
    u32* const region = reinterpret_cast<u32*>(smem) + wib * (kRegionWords + kSmallBitWords);
    unsigned short* const map = reinterpret_cast<unsigned short*>(region);
    u32* const small_bm = region + kRegionWords;
    const u64 ntiles = (1ull << a.slog2) / a.tile;
    u64 moved = 0;
    bool bad = false;
    for (u64 t = warp; t < ntiles && !bad; t += nwarps) {
        Tile x;
        if (!tile_of(a, t, ntiles, x)) continue;
        u32* const bm = x.mode == 0 ? small_bm : region;
        clear_owned(a, x, bm, lane);
        if (x.mode == 0)
            bad = place_range<0, kCg>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        else if (x.mode == 1)
            bad = place_range<1, kCg>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        else
            bad = place_range<2, kCg>(a, bm, map, x.m0, x.L, x.tbase, x.tl, lane, moved);
        if (bad) break;
        write_owned<kCg>(a, x, bm, map, lane);
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
template <bool kCg = false>
__device__ __forceinline__ void migrate_walk_tiles(const MigArgs& a, unsigned char* smem, u64 warp, u64 nwarps) {
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
    u64 moved = 0;
    int bad = 0;

    for (u64 t = warp; t < ntiles; t += nwarps) {
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
                key[q] = j < x.sl ? src_key<kCg>(a.src + ((x.m0 + j) & cmask)) : kEmpty;
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
                src_cell<kCg>(a.src + (i & cmask), k, v);
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
        write_owned<kCg>(a, x, bm, map, lane);
    }
    if (bad && lane == 0) atomicOr(&a.st->mig_fail, 2u);
    moved = warp_sum(moved);
    if (lane == 0 && moved) atomicAdd(&a.st->I, moved);
}

// Shared memory of the tile loops for one 256-thread block.
inline size_t migrate_smem_bytes(u32 start_cap) {
    return size_t(kMigWarps) * ((kRegionWords + kSmallBitWords) * 4 + size_t(start_cap) * 2);
}

__host__ __device__ inline u32 migrate_start_cap(u32 tile, bool windows) { return windows ? 0u : (tile / 2 + 8 + 7) & ~7u; }

}  // namespace
}  // namespace cht
