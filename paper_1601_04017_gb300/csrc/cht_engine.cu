// Batched engine: many tables and many uneven operation batches in one
// persistent kernel launch.
//
// The host turns a list of batches (each: one table, one operation type, n
// keys) into chunks of at most kChunkOps operations, ordered round by round
// (round r holds the r-th batch of every table that has one).  Warps of a
// persistent grid take chunks from a device work queue (one atomic counter).
// Per table, batches must keep the phase semantics of single calls: every
// operation of batch k happens before any of batch k+1.  A chunk therefore
// carries `need`, the number of chunks of its table's earlier batches, and
// waits until the table's completion counter reaches it.  Chunks leave the
// queue in plan order, so every chunk a waiter depends on is already held by
// a running warp: the wait always ends.  It is still bounded (clock cycles):
// a wait that runs out sets a timeout bit and an abort bit that makes every
// warp stop taking chunks, so the launch ends either way and the host reads
// the status.  Different tables are independent, so their batches overlap on
// the device -- small tables do not leave the GPU idle the way one launch per
// batch does.
//
// Coherence: a later chunk of a table may run on another SM right after an
// earlier one modified the table, so every table read in the engine goes
// through L2 (finds included); writers fence before they count a chunk done
// and a waiter fences after it has seen the count it needs.
//
// Staged I/O (the default): a warp copies its chunk's keys and values into
// its own shared-memory area with one coalesced pass, runs the probe loop
// from there and writes the found values and result codes back with one
// coalesced pass.  The probe loop itself touches the request arrays one
// scattered element at a time; when those arrays are in host memory (a
// serving loop reading requests in place across NVLink-C2C) every such
// access is a separate round trip, and staging turns them into a few
// full-width transfers.  The copy-in happens before the dependency wait
// (inputs are never written by the plan), so on a chain of dependent
// batches -- one hot table's requests in arrival order -- its latency is off
// the critical path.
//
// Waiting: many warps can wait on the same table's counter (they take items
// far ahead of the level in progress).  Each polls with a plain relaxed load
// and sleeps in between for 16 ns per item it still waits for (at least
// 128 ns, at most max_backoff_ns): warps whose turn is near poll often, the
// many far behind them rarely, so the counter's L2 line is not flooded
// while the warps it waits for are updating it.
//
// Groups: a chain of small dependent batches (levels of one item each) is
// run by one warp in order -- no hand-off through the counter between them,
// which costs a few microseconds per level.
#include <atomic>

#include "cht_ops.cuh"

namespace cht {
namespace {

constexpr u32 kEngineTimeout = 1u;
constexpr u32 kEngineAbort = 2u;

__device__ __forceinline__ u64 ld_relaxed_u64(const unsigned long long* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void red_release_add(unsigned long long* p, u64 v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Shared memory one warp uses to stage a chunk: keys, values (find results
// reuse this array: finds read no values) and one result byte per operation.
constexpr u32 kStageWarpBytes = kChunkOps * (8 + 8 + 1);
static_assert(kStageWarpBytes % 8 == 0, "warp areas stay 8-byte aligned");

template <int G, int V, int MODE, bool kStaged, int F>
__device__ __forceinline__ void engine_window(const OpArgs& a, u64 first, u64 end, u64& n_ins, u64& n_del,
                                              u32& sbits, const WarpStage& sg) {
    warp_ops<G, V, MODE, true, kStaged, F>(a, first, end, n_ins, n_del, sbits, sg);
}

// kEF: the flag variants (tombstone reuse, full key space) some table of the
// launch needs; each item takes the variant of its own table.
template <int G, int V, int MODE, bool kStaged, int kEF>
__device__ __forceinline__ void engine_mode(const OpArgs& a, u64 first, u64 end, u64& n_ins, u64& n_del,
                                            u32& sbits, const WarpStage& sg) {
    if constexpr (kEF == 0) {
        engine_window<G, V, MODE, kStaged, 0>(a, first, end, n_ins, n_del, sbits, sg);
    } else {
        constexpr bool fills = mode_fills(MODE);
        const int f = ((kEF & kFlagReuse) && fills && a.reuse ? kFlagReuse : 0) |
                      ((kEF & kFlagFullKeys) && a.full_keys ? kFlagFullKeys : 0);
        if (f == 0) {
            engine_window<G, V, MODE, kStaged, 0>(a, first, end, n_ins, n_del, sbits, sg);
        } else if (f == kFlagReuse) {
            if constexpr ((kEF & kFlagReuse) && fills)
                engine_window<G, V, MODE, kStaged, kFlagReuse>(a, first, end, n_ins, n_del, sbits, sg);
        } else if (f == kFlagFullKeys) {
            if constexpr ((kEF & kFlagFullKeys) != 0)
                engine_window<G, V, MODE, kStaged, kFlagFullKeys>(a, first, end, n_ins, n_del, sbits, sg);
        } else {
            if constexpr ((kEF & kFlagReuse) && (kEF & kFlagFullKeys) && fills)
                engine_window<G, V, MODE, kStaged, kFlagReuse | kFlagFullKeys>(a, first, end, n_ins, n_del, sbits,
                                                                              sg);
        }
    }
}

template <int G, int V, bool kStaged, int kEF>
__device__ __forceinline__ void engine_run(int mode, const OpArgs& a, u64 first, u64 end, u64& n_ins,
                                           u64& n_del, u32& sbits, const WarpStage& sg) {
    switch (mode) {
        case kFind: engine_mode<G, V, kFind, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg); break;
        case kInsert: engine_mode<G, V, kInsert, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg); break;
        case kIouAdd: engine_mode<G, V, kIouAdd, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg); break;
        case kIouOverwrite:
            engine_mode<G, V, kIouOverwrite, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg);
            break;
        case kUpdAdd: engine_mode<G, V, kUpdAdd, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg); break;
        case kUpdOverwrite:
            engine_mode<G, V, kUpdOverwrite, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg);
            break;
        default: engine_mode<G, V, kErase, kStaged, kEF>(a, first, end, n_ins, n_del, sbits, sg); break;
    }
}

// Copy one item's keys (and values) into the warp's staging area.
__device__ __forceinline__ void stage_in(const EngineChunk& ch, const EngineBatch& b, const WarpStage& sg, int lane) {
    const bool has_vals = mode_has_vals(int(b.mode));
    for (u32 j = lane; j < ch.count; j += 32) {
        sg.keys[j] = ld_stream(b.keys + ch.start + j);
        if (has_vals) sg.vals[j] = ld_stream(b.vals + ch.start + j);
    }
}

// Run one item whose dependencies are met and write its results.  With
// `count` > 0 the item then counts itself and the `count` - 1 items before
// it in its group done for its table; with 0 (an item inside a group) the
// next item of the group, run by this same warp, only needs this warp's
// lanes to agree on memory order, which __syncwarp gives.
template <int G, int V, bool kStaged, int kEF>
__device__ __forceinline__ void run_item(const EngineArgs& e, const EngineChunk& ch, const EngineBatch& b,
                                         const EngineTable& t, WarpStage& sg, int lane, u32 count) {
    OpArgs a;
    a.cells = t.cells;
    a.log2c = t.log2c;
    a.reuse = t.flags & kTabReuse;
    a.full_keys = t.flags & kTabFullKeys;
    a.keys = b.keys;
    a.vals = b.vals;
    a.vals_out = b.vals_out;
    a.codes = b.codes;
    a.n = b.n;
    a.st = t.st;
    const u64 end = ch.start + ch.count;
    u64 n_ins = 0, n_del = 0;
    u32 sbits = 0;
    if (kStaged) {
        sg.base = ch.start;
        engine_run<G, V, true, kEF>(b.mode, a, ch.start, end, n_ins, n_del, sbits, sg);
    } else {
        engine_run<G, V, false, kEF>(b.mode, a, ch.start, end, n_ins, n_del, sbits, sg);
    }
    // Count the items done as soon as the table writes are ordered: the
    // results (found values, codes -- possibly in host memory) and the
    // table's counters are read only after the launch, so they are written
    // after the release and stay out of the fence's wait.
    if (count) fence_acq_rel_gpu();  // this lane's table writes before the items are counted
    __syncwarp();
    if (count && lane == 0) red_release_add(e.done + b.table, u64(count));
    if (kStaged) {
        for (u32 j = lane; j < ch.count; j += 32) {
            if (b.mode == kFind) b.vals_out[ch.start + j] = sg.vout[j];
            if (b.codes) b.codes[ch.start + j] = sg.codes[j];
        }
    }
    warp_flush_counters(t.st, n_ins, n_del, sbits);
    __syncwarp();  // the next item overwrites this one's staging area
}

template <int G, int V, bool kStaged, int kEF>
__global__ void __launch_bounds__(kOpBlock) engine_kernel(EngineArgs e) {
    constexpr u32 FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char engine_smem[];
    const int lane = threadIdx.x & 31;
    WarpStage sg{};
    if (kStaged) {
        unsigned char* w = engine_smem + (threadIdx.x >> 5) * kStageWarpBytes;
        sg.keys = reinterpret_cast<u64*>(w);
        sg.vals = sg.keys + kChunkOps;
        sg.vout = sg.vals;
        sg.codes = reinterpret_cast<unsigned char*>(sg.vals + kChunkOps);
    }
    for (;;) {
        u64 c = 0;
        if (lane == 0) c = atomicAdd(e.next, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if (c >= e.n_chunks) break;
        if (*reinterpret_cast<volatile u32*>(e.status) & kEngineAbort) break;
        const EngineChunk ch = e.chunks[c];
        const EngineBatch b = e.batches[ch.batch];
        const EngineTable t = e.tables[b.table];
        if (kStaged) stage_in(ch, b, sg, lane);
        // wait for every item of this table's earlier levels; the sleep
        // between polls grows with the number of items still missing
        int ok = 1;
        if (lane == 0) {
            u64 need = ch.need;
            if (e.inject_stall && c == 0) need = ~0ull;  // testing: a count nothing reaches
            u64 seen = ld_relaxed_u64(e.done + b.table);
            if (seen < need) {
                const long long t0 = clock64();
                for (;;) {
                    const u64 gap = need - seen;
                    const u64 ns = gap > e.max_backoff_ns / 16 ? e.max_backoff_ns : gap * 16 < 128 ? 128 : gap * 16;
                    __nanosleep(unsigned(ns));
                    seen = ld_relaxed_u64(e.done + b.table);
                    if (seen >= need) break;
                    if (clock64() - t0 > e.spin_limit ||
                        (*reinterpret_cast<volatile u32*>(e.status) & kEngineAbort)) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) {
            if (lane == 0) atomicOr(e.status, kEngineTimeout | kEngineAbort);
            break;
        }
        fence_acq_rel_gpu();  // lane 0: table reads after the count it saw ...
        __syncwarp();         // ... and the other lanes' reads after lane 0's fence
        run_item<G, V, kStaged, kEF>(e, ch, b, t, sg, lane, ch.nfollow ? 0u : 1u);
        // the group this item leads: later levels of the same table, in
        // order; the whole group is counted done by its last item
        for (u32 f = 0; f < ch.nfollow; ++f) {
            const EngineChunk fc = e.chunks[ch.follow_first + f];
            const EngineBatch fb = e.batches[fc.batch];
            if (kStaged) {
                stage_in(fc, fb, sg, lane);
                __syncwarp();
            }
            run_item<G, V, kStaged, kEF>(e, fc, fb, t, sg, lane, f + 1 == ch.nfollow ? ch.nfollow + 1u : 0u);
        }
    }
    if (e.n_snap) {
        // the last warp to finish reads the counts every other warp flushed
        // (their fence orders the flush before their count here) and writes
        // the snapshot, possibly straight into pinned host memory
        u64 prior = 0;
        if (lane == 0) {
            __threadfence();
            prior = atomicAdd(e.warps_done, 1ull);
        }
        prior = __shfl_sync(FULL, prior, 0);
        const u64 nwarps = u64(gridDim.x) * (blockDim.x / 32);
        if (prior + 1 == nwarps) {
            __threadfence();
            for (u32 i = lane; i < e.n_snap; i += 32) {
                const DevState* st = e.tables[e.snap_tables[i]].st;
                e.snap_out[2 * i] = *reinterpret_cast<const volatile unsigned long long*>(&st->I);
                e.snap_out[2 * i + 1] = *reinterpret_cast<const volatile unsigned long long*>(&st->D);
            }
        }
    }
}

template <int G, int V, bool kStaged, int kEF = 0>
cudaError_t launch_engine_gvs(const EngineArgs& e, int ctas_per_sm, cudaStream_t s) {
    const u32 smem = kStaged ? (kOpBlock / 32) * kStageWarpBytes : 0;
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t err =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel<G, V, kStaged, kEF>, kOpBlock, smem);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
        occ.store(per_sm, std::memory_order_relaxed);
    }
    // persistent grid: never more CTAs than can be resident at once
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    u64 grid = u64(sm_count()) * u64(per_sm);
    const u64 need = (e.n_chunks + kOpBlock / 32 - 1) / (kOpBlock / 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    engine_kernel<G, V, kStaged, kEF><<<unsigned(grid), kOpBlock, smem, s>>>(e);
    count_launch();
    return cudaGetLastError();
}

template <int G, int V>
cudaError_t launch_engine_gv(const EngineArgs& e, bool staged, int ctas_per_sm, cudaStream_t s) {
    return staged ? launch_engine_gvs<G, V, true>(e, ctas_per_sm, s)
                  : launch_engine_gvs<G, V, false>(e, ctas_per_sm, s);
}

}  // namespace

cudaError_t launch_engine(const EngineArgs& e, int group_width, int lane_cells, int ctas_per_sm, bool staged,
                          cudaStream_t s) {
    if (e.n_chunks == 0) return cudaSuccess;
    const int ef = (e.any_reuse ? kFlagReuse : 0) | (e.any_full ? kFlagFullKeys : 0);
    if (ef) {
        // tables with tombstone reuse or the full key space: staged I/O and
        // 1 or 4 lanes of one sector, the nearest to the configured window
        const bool wide = group_width >= 4;
        switch (ef) {
            case kFlagReuse:
                return wide ? launch_engine_gvs<4, 2, true, kFlagReuse>(e, ctas_per_sm, s)
                            : launch_engine_gvs<1, 2, true, kFlagReuse>(e, ctas_per_sm, s);
            case kFlagFullKeys:
                return wide ? launch_engine_gvs<4, 2, true, kFlagFullKeys>(e, ctas_per_sm, s)
                            : launch_engine_gvs<1, 2, true, kFlagFullKeys>(e, ctas_per_sm, s);
            default:
                return wide ? launch_engine_gvs<4, 2, true, kFlagReuse | kFlagFullKeys>(e, ctas_per_sm, s)
                            : launch_engine_gvs<1, 2, true, kFlagReuse | kFlagFullKeys>(e, ctas_per_sm, s);
        }
    }
    if (lane_cells == 2) {
        switch (group_width) {
            case 1: return launch_engine_gv<1, 2>(e, staged, ctas_per_sm, s);
            case 4: return launch_engine_gv<4, 2>(e, staged, ctas_per_sm, s);
            case 8: return launch_engine_gv<8, 2>(e, staged, ctas_per_sm, s);
            case 16: return launch_engine_gv<16, 2>(e, staged, ctas_per_sm, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (group_width) {
        case 1: return launch_engine_gv<1, 2>(e, staged, ctas_per_sm, s);
        case 4: return launch_engine_gv<4, 1>(e, staged, ctas_per_sm, s);
        case 8: return launch_engine_gv<8, 1>(e, staged, ctas_per_sm, s);
        case 16: return launch_engine_gv<16, 1>(e, staged, ctas_per_sm, s);
        case 32: return launch_engine_gv<32, 1>(e, staged, ctas_per_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cht
