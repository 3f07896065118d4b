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
// and waiters load the counter with acquire semantics.
#include <atomic>

#include "cht_ops.cuh"

namespace cht {
namespace {

constexpr u32 kEngineTimeout = 1u;
constexpr u32 kEngineAbort = 2u;

__device__ __forceinline__ u64 ld_acquire_u64(const unsigned long long* p) {
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, u64 v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int G, int V>
__global__ void __launch_bounds__(kOpBlock) engine_kernel(EngineArgs e) {
    constexpr u32 FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        u64 c = 0;
        if (lane == 0) c = atomicAdd(e.next, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if (c >= e.n_chunks) break;
        if (*reinterpret_cast<volatile u32*>(e.status) & kEngineAbort) break;
        const EngineChunk ch = e.chunks[c];
        const EngineBatch b = e.batches[ch.batch];
        const EngineTable t = e.tables[b.table];
        // wait for every chunk of this table's earlier batches
        int ok = 1;
        if (lane == 0) {
            u64 need = ch.need;
            if (e.inject_stall && c == 0) need = ~0ull;  // testing: a count nothing reaches
            if (ld_acquire_u64(e.done + b.table) < need) {
                const long long t0 = clock64();
                while (ld_acquire_u64(e.done + b.table) < need) {
                    if (clock64() - t0 > e.spin_limit) {
                        ok = 0;
                        break;
                    }
                    if (*reinterpret_cast<volatile u32*>(e.status) & kEngineAbort) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) {
            if (lane == 0) atomicOr(e.status, kEngineTimeout | kEngineAbort);
            break;
        }
        __threadfence();  // order this warp's table reads after the acquire
        OpArgs a;
        a.cells = t.cells;
        a.log2c = t.log2c;
        a.keys = b.keys;
        a.vals = b.vals;
        a.vals_out = b.vals_out;
        a.codes = b.codes;
        a.n = b.n;
        a.st = t.st;
        const u64 end = ch.start + ch.count;
        u64 n_ins = 0, n_del = 0;
        u32 sbits = 0;
        switch (b.mode) {
            case kFind: warp_ops<G, V, kFind, true>(a, ch.start, end, n_ins, n_del, sbits); break;
            case kInsert: warp_ops<G, V, kInsert, true>(a, ch.start, end, n_ins, n_del, sbits); break;
            case kIouAdd: warp_ops<G, V, kIouAdd, true>(a, ch.start, end, n_ins, n_del, sbits); break;
            case kIouOverwrite: warp_ops<G, V, kIouOverwrite, true>(a, ch.start, end, n_ins, n_del, sbits); break;
            default: warp_ops<G, V, kErase, true>(a, ch.start, end, n_ins, n_del, sbits); break;
        }
        warp_flush_counters(t.st, n_ins, n_del, sbits);
        __threadfence();  // this lane's table writes before the chunk is counted
        __syncwarp();
        if (lane == 0) red_release_add(e.done + b.table, 1ull);
    }
}

template <int G, int V>
cudaError_t launch_engine_gv(const EngineArgs& e, int ctas_per_sm, cudaStream_t s) {
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel<G, V>, kOpBlock, 0);
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
    engine_kernel<G, V><<<unsigned(grid), kOpBlock, 0, s>>>(e);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_engine(const EngineArgs& e, int group_width, int lane_cells, int ctas_per_sm, cudaStream_t s) {
    if (e.n_chunks == 0) return cudaSuccess;
    if (lane_cells == 2) {
        switch (group_width) {
            case 1: return launch_engine_gv<1, 2>(e, ctas_per_sm, s);
            case 4: return launch_engine_gv<4, 2>(e, ctas_per_sm, s);
            case 8: return launch_engine_gv<8, 2>(e, ctas_per_sm, s);
            case 16: return launch_engine_gv<16, 2>(e, ctas_per_sm, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (group_width) {
        case 1: return launch_engine_gv<1, 2>(e, ctas_per_sm, s);
        case 4: return launch_engine_gv<4, 1>(e, ctas_per_sm, s);
        case 8: return launch_engine_gv<8, 1>(e, ctas_per_sm, s);
        case 16: return launch_engine_gv<16, 1>(e, ctas_per_sm, s);
        case 32: return launch_engine_gv<32, 1>(e, ctas_per_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cht
