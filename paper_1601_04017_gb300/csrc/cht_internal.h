// Internal host-side interface between the C-ABI runtime (cht_runtime.cu)
// and the kernel translation units (cht_ops.cu, cht_migrate.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cht_device.cuh"

namespace cht {

enum Mode : int { kFind = 0, kInsert = 1, kIouAdd = 2, kIouOverwrite = 3, kErase = 4, kUpdAdd = 5, kUpdOverwrite = 6 };

// Modes that read a value per operation / that may fill an empty cell.
__host__ __device__ constexpr bool mode_has_vals(int m) {
    return m == kInsert || m == kIouAdd || m == kIouOverwrite || m == kUpdAdd || m == kUpdOverwrite;
}
__host__ __device__ constexpr bool mode_fills(int m) { return m == kInsert || m == kIouAdd || m == kIouOverwrite; }

// One batched operation over a table of 2^log2c cells.
struct OpArgs {
    Cell* cells;
    u32 log2c;
    u32 reuse;            // inserts may take the first tombstone on their path
    u32 full_keys;        // keys 0 and ~0 go to the special slots in st
    const u64* keys;
    const u64* vals;      // insert / insert_or_update input values (else NULL)
    u64* vals_out;        // find output values (else NULL)
    unsigned char* codes; // per-op result codes (nullable)
    u64 n;
    DevState* st;
    // 0: each warp takes one contiguous slice of the batch; else warps take
    // consecutive pieces of `chunk` operations in batch order from a ticket
    // counter (`ticket`, zero before the launch; the aggregation kernel takes
    // its windows from it too), so the operations in flight at any moment
    // are a narrow range of the batch -- the hash-partitioned path relies on
    // it.  A static grid-stride order would let warps drift apart over the
    // hundreds of pieces each runs.
    u32 chunk = 0;
    unsigned long long* ticket = nullptr;
};

// Launch one batched operation. group_width in {1,2,4,8,16,32}; lane_cells
// 1 or 2 (G = 1 always uses 2; G = 32 only 1); ctas_per_sm 0 = occupancy
// maximum.  Returns the launch error (cudaSuccess if none).
cudaError_t launch_op(Mode mode, const OpArgs& a, int group_width, int lane_cells, int ctas_per_sm,
                      cudaStream_t s);

// insertOrUpdate (mode kIouAdd or kIouOverwrite) with CTA-level
// aggregation of equal keys in shared memory before the table is touched.
// warp_dedup: first combine equal keys of each warp step (extreme skew).
cudaError_t launch_iou_aggregated(Mode mode, const OpArgs& a, bool warp_dedup, int ctas_per_sm, cudaStream_t s);
// The same with 1024-thread CTAs and windows of 4096 operations (8192
// shared-memory slots): for batches sorted by hash, where a window holds the
// whole groups of a key's operations.  insertOrUpdate modes only.
cudaError_t launch_iou_aggregated_wide(Mode mode, const OpArgs& a, bool warp_dedup, cudaStream_t s);

// Cluster-wise migration of `src` (2^src_log2 cells) into `dst`
// (2^dst_log2 cells, dst_log2 >= src_log2).  dst needs no initialisation:
// every target cell is written.  `st` receives the new I (it must be zero
// on entry) and mig_fail.  tile: source cells per warp task (power of two,
// 0 = default); windows: place cells 32 at a time per warp (long clusters)
// instead of one cluster per lane; border: device scratch of
// migrate_border_count() u64.
u64 migrate_border_count(u32 src_log2, int tile);
cudaError_t launch_migrate(const Cell* src, u32 src_log2, Cell* dst, u32 dst_log2, DevState* st,
                           int tile, bool windows, u64* border, cudaStream_t s);

// Shrinking migration (Sec. 4.3.1 "Shrinking") of `src` into `dst` (2^dst_log2
// cells, dst_log2 < src_log2, more cells than live elements; no
// initialisation needed).  `st` receives the new I (zero on entry).  spill:
// scratch of 2^dst_log2 cells; nspill: one counter, zero on entry.
cudaError_t launch_shrink(const Cell* src, u32 src_log2, Cell* dst, u32 dst_log2, DevState* st, Cell* spill,
                          unsigned long long* nspill, cudaStream_t s);

// Sort-based bulk build (Sec. 3 "Bulk Operations") into an empty table, in
// three stream-ordered steps over one scratch block of build_scratch_bytes(n):
// launch_build_sort sorts the batch's cells by the top build_sort_bits(log2c)
// hash bits (stable) and routes keys 0 / ~0; launch_build_count counts the
// survivors (the last copy of each key) into ex->S; launch_build_place writes
// them into the zeroed cells, wraps the tail and sets I, D and the special
// slots.  n < 2^32.
struct BuildExtra {
    u64 sp_last[2];  // 1 + input position of the last key 0 / ~0 (0: none)
    u64 S;           // survivors
    u64 first_ov;    // lowest rank placed past the last cell (~0: none)
    u64 reserved;    // nonzero: a key 0 / ~0 was skipped (full key space off)
    u32 n_deferred;  // cells whose survivor test was deferred to a CTA scan
    u32 pad;
};
u32 build_sort_bits(u32 log2c);
u64 build_scratch_bytes(u64 n);
cudaError_t launch_build_sort(const u64* keys, const u64* vals, u64 n, u32 log2c, int full_keys, void* scratch,
                              const Cell** sorted, BuildExtra** ex, cudaStream_t s);
cudaError_t launch_build_count(const Cell* sorted, u64 n, u32 log2c, void* scratch, BuildExtra* ex,
                               cudaStream_t s);
cudaError_t launch_build_place(const Cell* sorted, u64 n, Cell* cells, u32 log2c, void* scratch, BuildExtra* ex,
                               DevState* st, const u64* vals, cudaStream_t s);

// Exclusive scan of m u32 in place (three kernels); `part` holds
// scan_partials(m) u32.
u64 scan_partials(u64 m);
cudaError_t scan_exclusive_u32(u32* data, u64 m, u32* part, cudaStream_t s);

// Hash-partitioned execution of one large batch (cht_bulk.cu, Sec. 4.5): the
// operations are reordered by the top 8 bits of their hash (the home slot's
// top bits, i.e. which 1/256 of the table they touch), the operation kernel
// runs over them in that order, and the per-operation results are put back
// into the caller's order.  `run` launches the operation kernel on the
// reordered arguments it is given.  Scratch: partition_scratch_bytes(n, ...)
// bytes, 256-byte aligned.
struct PartitionIO {
    bool vals;       // the operation reads a value per key
    bool vals_out;   // it writes a found value per key (find)
    bool codes;      // it writes a result code per key
};
u64 partition_scratch_bytes(u64 n, PartitionIO io);
typedef cudaError_t (*PartitionRun)(const OpArgs& a, void* ctx, cudaStream_t s);
cudaError_t launch_partitioned(const OpArgs& a, PartitionIO io, void* scratch, PartitionRun run, void* ctx,
                               cudaStream_t s);

// A batch sorted by the top 16 bits of its keys' hash (two stable 8-bit
// passes, cht_bulk.cu) before `run` executes the operation on the sorted keys
// and values; the result codes are put back into the caller's order (two
// gathers).  All operations of one key then lie in one contiguous run of the
// sorted batch (the run of their 1/65536 of the hash range), so a window of
// 4096 consecutive operations holds whole runs of ~4096 / (n / 65536) keys'
// operations.  Scratch:
// sorted16_scratch_bytes(n, codes != nullptr), about 38 bytes per operation.
u64 sorted16_scratch_bytes(u64 n, bool codes);
cudaError_t launch_sorted16(const OpArgs& a, void* scratch, PartitionRun run, void* ctx, cudaStream_t s);

// The live cells (neither empty nor tombstone) in cell index order into
// keys_out / vals_out (deterministic; the bulk merge's table side).  Scratch:
// compact_scratch_bytes(log2c).
u64 compact_scratch_bytes(u32 log2c);
cudaError_t launch_compact_live(const Cell* cells, u32 log2c, u64* keys_out, u64* vals_out, void* scratch,
                                cudaStream_t s);

// In-kernel growth (cht_grow.cu, Sec. 4.3.2): one cooperative launch runs an
// insert / insertOrUpdate batch on a growable table, migrating between
// operation rounds.  Control words in device memory, zeroed by the host
// except cur = 0, log2c = the table's, done = 0.
constexpr unsigned kGrowTimeout = 1u;   // a barrier wait ran out
constexpr unsigned kGrowMigFail = 2u;   // a migration tile failed: the host redoes that migration
constexpr unsigned kGrowTooSmall = 4u;  // the targets cannot hold the next capacity
struct GrowCtl {
    unsigned int arrived;  // barrier
    unsigned int gen;
    unsigned int error;
    unsigned int cur;      // table buffer: 0 the initial cells, 1 / 2 the targets
    unsigned int log2c;
    unsigned int next_log2;
    unsigned int windows;
    unsigned int migrations;
    unsigned int fail_tgt;
    int action;
    unsigned long long done;    // operations applied in finished rounds
    unsigned long long chunk;   // operations of the current round
    unsigned long long ticket;  // pieces taken in the current round
};
u64 grow_border_count(u32 max_log2);
// group_width 1 (one lane per key, one sector per lane) or 4 (four lanes x one sector).
cudaError_t launch_grow(const OpArgs& op, Mode mode, Cell* t1, Cell* t2, u32 max_log2, double alpha, GrowCtl* ctl,
                        u64* border, long long spin_limit, int stall_block, int group_width, cudaStream_t s);

// Compact the live cells into keys_out / vals_out (max_n entries); the count
// lands in st->export_pos, which must be zero on entry.
cudaError_t launch_export(const Cell* cells, u32 log2c, u64* keys_out, u64* vals_out, u64 max_n,
                          DevState* st, cudaStream_t s);

// ---- batched engine (cht_engine.cu) ----------------------------------------
constexpr u32 kChunkOps = 256;  // operations per engine work item

// EngineTable::flags
constexpr u32 kTabReuse = 1u;     // tombstone reuse by inserts
constexpr u32 kTabFullKeys = 2u;  // keys 0 and ~0 in the special slots

struct EngineTable {
    Cell* cells;
    u32 log2c;
    u32 flags;  // table configuration, kTab* bits
    DevState* st;
};

struct EngineBatch {
    const u64* keys;
    const u64* vals;
    u64* vals_out;
    unsigned char* codes;
    u64 n;
    u32 table;  // index into the plan's table array
    u32 mode;   // Mode
};

// One work item: operations [start, start + count) of one batch.  A queue
// item may lead a group: the warp that runs it then runs `nfollow` more
// items of the same table, chunks[follow_first ..], in order and without
// waiting (each is a later dependency level of that table, so program order
// is the ordering it needs).  Followers sit after the queue in the array.
struct EngineChunk {
    u64 start;  // first operation of the batch in this chunk
    u64 need;   // items of the table's earlier levels that must be done first
    u32 batch;
    uint16_t count;
    uint16_t nfollow;
    u32 follow_first;
    u32 pad;
};
static_assert(sizeof(EngineChunk) == 32, "work items are 32 bytes");

struct EngineArgs {
    const EngineTable* tables;
    const EngineBatch* batches;
    const EngineChunk* chunks;
    u64 n_chunks;  // queue items (followers come after them)
    unsigned long long* next;  // work-queue cursor (zero before a launch)
    unsigned long long* done;  // per table: completed chunks (zero before a launch)
    u32* status;               // engine status bits (zero before a launch)
    long long spin_limit;      // bound of one dependency wait, in clock cycles
    unsigned max_backoff_ns;   // longest sleep between two polls of a dependency counter
    int any_reuse;             // some table of the launch reuses tombstones
    int any_full;              // some table of the launch has the full key space
    // optional snapshot at the end of the launch: the last warp to finish
    // writes I, D of tables[snap_tables[i]] to snap_out[2i], snap_out[2i + 1]
    // (n_snap = 0: none); warps_done: a counter, zero before the launch
    const u32* snap_tables;
    u32 n_snap;
    unsigned long long* snap_out;
    unsigned long long* warps_done;
    int inject_stall;          // testing: the first chunk waits for a count nothing reaches
};

// staged: copy each work item's keys / values through shared memory (else
// the probe loops access the batch arrays in place).
cudaError_t launch_engine(const EngineArgs& e, int group_width, int lane_cells, int ctas_per_sm, bool staged,
                          cudaStream_t s);


}  // namespace cht

#include <vector>

#include "../../include/cht.h"

namespace cht {

// Order batches into engine work items round by round (round r = every
// table's r-th batch).  `need` of an item = its table's items in earlier
// dependency levels (a run of consecutive finds on a table is one level).
// Consecutive levels of one table that are one item each are grouped: the
// first is a queue item that leads the rest.  chunk_ops: operations per
// item (32..256, a power of two), 0 = sized per table from the length of
// its chain of levels.  Returns the number of queue items; `chunks` holds
// them followed by the followers.
u64 plan_order(const std::vector<EngineBatch>& batches, size_t n_tables, int chunk_ops,
               std::vector<EngineChunk>& chunks);

// Runtime services for translation units outside the runtime.
struct TableInfo {
    Cell* cells;
    u32 log2c;
    DevState* st;
    int device;
    int growable;
    double alpha;
    u64 bound;  // upper bound on the number of non-empty cells
    int reuse;      // tombstone reuse by inserts
    int full_keys;  // keys 0 and ~0 in the special slots
};
TableInfo table_info(const cht_table* h);
void table_set_bound(cht_table* h, u64 bound, bool exact);
// Synchronize s and read the table's exact counters (also refreshes its bound).
cht_status table_read_counts(cht_table* h, u64* I, u64* D, cudaStream_t s);
// Migrate into 2^new_log2 cells; live = exact live count (or ~0 if unknown).
cht_status table_migrate_to(cht_table* h, u32 new_log2, u64 live, cudaStream_t s);
cht_status runtime_alloc(void** p, u64 bytes, cudaStream_t s);
void runtime_free(void* p, u64 bytes, cudaStream_t s);

// Device memory available to new allocations of this library on `device`:
// the driver's free bytes plus what the stream-ordered pool holds unused.
u64 device_free_bytes(int device);

// Kernel launches issued so far (process-wide).
void count_launch();

// SM count of the current device (cached).
int sm_count();

}  // namespace cht

struct cht_table;

namespace cht {

// Read-only view of a table's device state and tunables (for entry points
// that live outside the runtime translation unit); group_width is the
// effective width a find would use now.
void table_view(const cht_table* h, Cell** cells, u32* log2c, DevState** st, int* device,
                int* group_width, int* lane_cells, int* ctas_per_sm, int* full_keys);

// Record the stream of a call's work on the table, as every entry point does:
// cht_destroy and later migrations order the release of the cells after it.
void table_note_stream(cht_table* h, cudaStream_t s);

}  // namespace cht
