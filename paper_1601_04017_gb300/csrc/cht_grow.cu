// In-kernel growth (Sec. 4.3.2: the threads that run the operations are
// recruited for the migration, "uaGrow"/"usGrow"; Sec. 4.3.1 cluster-wise
// migration; Sec. 4.4 gamma from the live count).
//
// One persistent, cooperative launch runs a whole insert or insertOrUpdate
// batch on a growable table.  It proceeds in rounds separated by grid-wide
// barriers.  At the start of a round one thread (block 0, thread 0) reads the
// exact counters and decides: if the non-empty cells I have reached
// floor(alpha * c), the round is a migration -- to 2c if more than
// alpha * c / 2 elements are live, else to c (a tombstone purge) -- otherwise
// an operation round of min(floor(alpha * c) - I, rest) operations, so I never
// passes the threshold (the same chunks the host-driven policy makes).  Every
// warp of the grid then works on the round: operation pieces from a ticket
// counter with the group probe loop, or the migration's tile borders, a
// barrier, and the tile placement (the same device code as the migration
// kernels).  The barriers replace the host's counter read-back and the
// launches between rounds.
//
// Memory.  The host allocates two target tables of the largest capacity the
// batch can need (every operation a new key) and the border scratch; the table
// moves initial cells -> target 1 -> target 2 -> target 1 ... and the host
// frees what is not the final table after the launch.
//
// Bounded waits.  A barrier wait gives up after `spin_limit` clock cycles: the
// waiter sets the timeout bit and every block leaves at its next barrier.  The
// table stays valid (every cell is written whole, the migration target only
// replaces the source once its placement has finished), the batch is partly
// applied, and the host reports CHT_ERR_TIMEOUT.
#include "cht_migrate.cuh"
#include "cht_ops.cuh"

namespace cht {
namespace {

constexpr int kGrowBlock = 256;
constexpr u32 kGrowPiece = 256;  // operations per warp piece
constexpr u32 kGrowTile = 512;   // migration tile (load below 0.6)

enum : int { kActOps = 0, kActMigrate = 1, kActDone = 2 };

struct GrowArgs {
    OpArgs op;        // the batch; op.cells / op.log2c: the initial table
    Cell* tab[3];     // [0] the initial cells, [1], [2] the targets
    u32 max_log2;     // capacity of the targets
    double alpha;
    GrowCtl* ctl;
    u64* border;      // tile borders of the largest source
    long long spin_limit;
    int stall_block;  // testing: this block never arrives at a barrier (-1: none)
};

// Grid barrier with a bounded wait.  Returns false if some wait ran out (now
// or before): the caller leaves the kernel.
__device__ __forceinline__ bool grid_sync(const GrowArgs& g, u32& gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        GrowCtl* c = g.ctl;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&c->arrived, 1u) + 1u == gridDim.x) {
            atomicExch(&c->arrived, 0u);
            __threadfence();
            atomicExch(&c->gen, gen + 1u);
        } else {
            const long long t0 = clock64();
            while (*reinterpret_cast<volatile unsigned int*>(&c->gen) == gen) {
                if (*reinterpret_cast<volatile unsigned int*>(&c->error)) break;
                if (clock64() - t0 > g.spin_limit) {
                    atomicOr(&c->error, kGrowTimeout);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile unsigned int*>(&c->error) & kGrowTimeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    ++gen;
    return s_ok != 0;
}

template <int G, int V, int MODE>
__global__ void __launch_bounds__(kGrowBlock) grow_kernel(GrowArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    GrowCtl* const c = g.ctl;
    DevState* const st = g.op.st;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    const u64 warp = (u64(blockIdx.x) * kGrowBlock + threadIdx.x) >> 5;
    const u64 nwarps = (u64(gridDim.x) * kGrowBlock) >> 5;
    u32 gen = 0;
    if (int(blockIdx.x) == g.stall_block) return;  // testing: a block that never arrives
    for (;;) {
        if (leader) {  // decide the round (everyone else waits at the barrier)
            // (counters and control words are read through L2: other SMs wrote them)
            const u32 l2 = *reinterpret_cast<volatile unsigned int*>(&c->log2c);
            const u64 cap = 1ull << l2;
            const u64 limit = u64(floor(g.alpha * double(cap)));
            const u64 I = *reinterpret_cast<volatile unsigned long long*>(&st->I);
            const u64 D = *reinterpret_cast<volatile unsigned long long*>(&st->D);
            const u64 rest = g.op.n - *reinterpret_cast<volatile unsigned long long*>(&c->done);
            if (rest == 0) {
                c->action = kActDone;
            } else if (I >= limit) {
                const u64 half = u64(floor(g.alpha * double(cap) / 2.0));
                const u32 nl = l2 + (I - D > half ? 1u : 0u);
                if (nl > g.max_log2) {
                    atomicOr(&c->error, kGrowTooSmall);
                    c->action = kActDone;
                } else {
                    c->action = kActMigrate;
                    c->next_log2 = nl;
                    c->windows = double(I) >= 0.6 * double(cap) ? 1u : 0u;
                }
            } else {
                c->action = kActOps;
                c->chunk = limit - I < rest ? limit - I : rest;
                c->ticket = 0;
            }
        }
        if (!grid_sync(g, gen)) return;
        const int act = *reinterpret_cast<volatile int*>(&c->action);
        if (act == kActDone) return;
        const u32 cur = *reinterpret_cast<volatile unsigned int*>(&c->cur);
        const u32 log2c = *reinterpret_cast<volatile unsigned int*>(&c->log2c);
        if (act == kActOps) {
            const u64 done = *reinterpret_cast<volatile unsigned long long*>(&c->done);
            const u64 chunk = *reinterpret_cast<volatile unsigned long long*>(&c->chunk);
            OpArgs b = g.op;
            b.cells = g.tab[cur];
            b.log2c = log2c;
            b.keys = g.op.keys + done;
            b.vals = g.op.vals + done;
            b.codes = g.op.codes ? g.op.codes + done : nullptr;
            b.n = chunk;
            u64 n_ins = 0, n_del = 0;
            u32 sbits = 0;
            for (;;) {
                u64 piece = 0;
                if ((threadIdx.x & 31) == 0) piece = atomicAdd(&c->ticket, 1ull);
                piece = __shfl_sync(0xffffffffu, piece, 0);
                const u64 begin = piece * kGrowPiece;
                if (begin >= chunk) break;
                const u64 end = begin + kGrowPiece < chunk ? begin + kGrowPiece : chunk;
                warp_ops<G, V, MODE, false, false, 0>(b, begin, end, n_ins, n_del, sbits);
            }
            warp_flush_counters(st, n_ins, n_del, sbits);
            if (!grid_sync(g, gen)) return;
            if (leader) c->done = done + chunk;
            continue;
        }
        // migration round: borders, then placement (Sec. 4.3.1)
        const u32 tgt = cur == 1u ? 2u : 1u;
        MigArgs m;
        m.src = g.tab[cur];
        m.slog2 = log2c;
        m.dst = g.tab[tgt];
        m.dlog2 = *reinterpret_cast<volatile unsigned int*>(&c->next_log2);
        m.st = st;
        m.border = g.border;
        m.tile = (1ull << log2c) < kGrowTile ? u32(1ull << log2c) : kGrowTile;
        const bool windows = *reinterpret_cast<volatile unsigned int*>(&c->windows) != 0;
        m.start_cap = migrate_start_cap(m.tile, windows);
        migrate_borders<true>(m, u64(blockIdx.x) * kGrowBlock + threadIdx.x, u64(gridDim.x) * kGrowBlock);
        if (leader) {  // the kernels below accumulate the moved elements into I
            st->I = 0;
            st->D = 0;
            st->mig_fail = 0;
        }
        if (!grid_sync(g, gen)) return;
        if (windows) migrate_window_tiles<true>(m, smem, warp, nwarps);
        else migrate_walk_tiles<true>(m, smem, warp, nwarps);
        if (!grid_sync(g, gen)) return;
        if (leader) {
            if (*reinterpret_cast<volatile unsigned int*>(&st->mig_fail)) {
                // a tile could not bound its cluster range: the host redoes
                // this migration with its fallback and finishes the batch
                atomicOr(&c->error, kGrowMigFail);
                c->fail_tgt = tgt;
                c->action = kActDone;
            } else {
                c->cur = tgt;
                c->log2c = m.dlog2;
                ++c->migrations;
            }
        }
        if (!grid_sync(g, gen)) return;
        if (*reinterpret_cast<volatile unsigned int*>(&c->error)) return;
    }
}

template <int MODE>
cudaError_t launch_mode(const GrowArgs& g, int group_width, int lane_cells, cudaStream_t s) {
    // the windows of the automatic rule below load 0.6 (the growth threshold
    // keeps the load at or below alpha)
    auto pick = [&](auto kernel) -> cudaError_t {
        const size_t smem = migrate_smem_bytes(migrate_start_cap(kGrowTile, false));
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGrowBlock, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        GrowArgs a = g;
        void* params[] = {&a};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(unsigned(sm_count() * per_sm)),
                                        dim3(kGrowBlock), params, smem, s);
        count_launch();
        return e;
    };
    if (group_width == 4) return pick(grow_kernel<4, 2, MODE>);
    (void)lane_cells;
    return pick(grow_kernel<1, 2, MODE>);
}

}  // namespace

// a purge (gamma = 1) at the largest capacity migrates a source of max_log2
u64 grow_border_count(u32 max_log2) { return migrate_border_count(max_log2, kGrowTile); }

cudaError_t launch_grow(const OpArgs& op, Mode mode, Cell* t1, Cell* t2, u32 max_log2, double alpha, GrowCtl* ctl,
                        u64* border, long long spin_limit, int stall_block, int group_width, cudaStream_t s) {
    GrowArgs g;
    g.op = op;
    g.tab[0] = op.cells;
    g.tab[1] = t1;
    g.tab[2] = t2;
    g.max_log2 = max_log2;
    g.alpha = alpha;
    g.ctl = ctl;
    g.border = border;
    g.spin_limit = spin_limit;
    g.stall_block = stall_block;
    switch (mode) {
        case kInsert: return launch_mode<kInsert>(g, group_width, 2, s);
        case kIouAdd: return launch_mode<kIouAdd>(g, group_width, 2, s);
        case kIouOverwrite: return launch_mode<kIouOverwrite>(g, group_width, 2, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cht
