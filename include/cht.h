/*
 * libcht -- a GB300 (sm_103a) concurrent hash table: the folklore
 * linear-probing table of Maier, Sanders & Dementiev, "Concurrent Hash
 * Tables: Fast and General(?)!" (arXiv 1601.04017), with batched operations
 * and cluster-wise migration for growth.
 *
 * Data model
 *   A table is an array of c cells of 16 bytes, <key u64, value u64>, c a
 *   power of two >= 64 (Sec. 6 "Bounded Hash Tables").  Key 0 marks an empty
 *   cell and key ~0 a tombstone (Sec. 3 "Deletions", Sec. 4.4); neither can be
 *   stored.  The home cell of key x is the top log2(c) bits of fmix64(x)
 *   (MurmurHash3's 64-bit finalizer), i.e. the scaling map
 *   h_c(x) = floor(h(x) * c / 2^64) of Sec. 4.3.1, so doubling c keeps the
 *   order of clusters and lets migration run cluster by cluster (Lemma 1).
 *
 * Calls, streams and phase semantics
 *   Every operation call is one batch of ONE operation type.  Calls are
 *   asynchronous and ordered on the CUDA stream passed in; a batch behaves as
 *   if its operations ran in some sequential order (linearizability, Sec. 3),
 *   and consecutive calls on one stream see each other's effects.  Calls on
 *   one table must be issued on one stream, or ordered by the caller; calls
 *   that overlap on the device on the same table are not supported.
 *
 * Pointers
 *   Every array argument may be device memory or host memory.  Host arrays
 *   (pageable or pinned) are staged through library-owned device buffers:
 *   inputs are copied in on the stream before the kernel, outputs are copied
 *   back on the stream after it; results in a host output array are valid
 *   once the stream has been synchronized.  Batches of more than 2^24
 *   operations with host arrays run in pieces of 2^24 through three device
 *   slots kept by the library (about 420 MB each, allocated on a device's
 *   first such call), so the copies of one piece overlap the kernel of
 *   another; the pieces run in order, one linearization of the batch.  The caller owns every array and
 *   keeps it alive until the work on the stream has completed.  The library
 *   owns the table memory.  `stream` may be NULL (the legacy default stream).
 *
 * Per-operation result codes (optional uint8 output arrays; NULL = not wanted)
 *   0  no   (key already present / not found / not erased)
 *   1  yes  (inserted / found / erased)
 *   2  table full: every cell was probed without success (bounded table)
 *   3  reserved key (0 or ~0); the operation did not touch the table
 *   Codes 2 and 3 also set bits in the table's sticky device status, which
 *   cht_size() and cht_get_status() report.
 *
 * Errors
 *   Argument errors return at once with no side effect.  Device-side
 *   conditions (full table, reserved keys) are reported per operation and in
 *   the sticky status.  CUDA errors return CHT_ERR_CUDA.
 */
#ifndef CHT_H
#define CHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-compatible with cudaStream_t; no CUDA header is needed to include this. */
struct CUstream_st;
typedef struct CUstream_st *cht_stream_t;

typedef struct cht_table *cht_handle;

typedef enum {
    CHT_OK = 0,
    CHT_ERR_INVALID_ARG = 1,  /* NULL handle/pointer, bad size, bad op */
    CHT_ERR_OOM = 2,          /* device allocation failed; table unchanged */
    CHT_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
    CHT_ERR_TABLE_FULL = 4,   /* some operation found no free cell */
    CHT_ERR_RESERVED_KEY = 5, /* some operation used key 0 or ~0 */
    CHT_ERR_TIMEOUT = 6       /* reserved: a bounded device wait gave up */
} cht_status;

typedef enum {
    CHT_OVERWRITE = 0, /* value <- d (Sec. 3, single-word store specialisation) */
    CHT_ADD = 1        /* value <- value + d mod 2^64 (fetch-and-add specialisation) */
} cht_update_op;

/* Sticky device status bits (cht_get_status). */
#define CHT_STATUS_FULL 0x1u
#define CHT_STATUS_RESERVED 0x2u

/* Tunables.  group_width G: lanes that probe one key together, each loading
 * lane_cells cells per probe step (G in {1,2,4,8,16,32}; a warp refills a
 * group with its next operation when the group's key is decided); -1: one
 * thread per operation, the paper's own form (each thread runs its operations
 * one at a time from a grid-stride sequence, V = 2 or 4 cells per step;
 * tables with reuse_tombstones or full_key_space run it as G = 1).  0
 * (default) picks the window per batch from the table's size and load (for
 * insert: the load after the batch) by the measured rule the library was
 * built with (the single-call autotuner's output; where it has no entry:
 * below load 0.6, finds 2 lanes x 4 cells and the others 1 lane x 2 cells;
 * above it, finds and inserts 4 lanes x 4 cells and the others 4 lanes x 2
 * cells).  lane_cells V: 1 (16 bytes), 2 (one 32-byte sector) or 4 (two
 * sectors, loaded together); 0 = default (2 for G = 1, 4 for G = -1, else 1);
 * G = 32 allows only 1, G = 16 at most 2, G = -1 not 1.  ctas_per_sm: resident CTAs per
 * SM for the operation kernels (0 = occupancy maximum).  migrate_tile:
 * source cells per migration warp task (power of two, 64..8192; 0 = by load:
 * 512 below load 0.6, else 1024).  alpha: growth threshold in (0, 1) (Sec. 4.3.2; default 0.5).
 * iou_aggregate: 1 (default) folds equal keys of each window of 1024
 * insertOrUpdate or update operations in shared memory first (one table
 * operation per distinct key and window), and for insertOrUpdate also combines
 * equal keys within each warp step in a window that follows a window with
 * fewer distinct keys than a fifth of its operations; 2 always combines them
 * (insertOrUpdate); 3 first sorts an insertOrUpdate batch by the top 16 bits
 * of the hash (two stable 8-bit passes, Sec. 4.5 integer sorting) so that the
 * windows -- 4096 operations per 1024-thread CTA -- hold every operation of
 * the keys they see, and puts the result codes back into the caller's order
 * (about 38 bytes of scratch per operation; measured slower than 1 on GB300 at
 * every skew: the sort passes cost more than the aggregation saves); 0 probes
 * every operation with the group kernel.  reuse_tombstones: 0 (default) = the paper's rule,
 * an erased cell is never used again until a migration drops it (Sec. 3
 * "Deletions"); 1 = an insert / insert-or-update that finds its key absent
 * puts it into the first tombstone on its probe path (safe under phase
 * semantics: no erase runs during an insert batch).  Results are the same
 * either way; reuse keeps probes short when keys are erased and inserted
 * again and again, where without it every cycle leaves a tombstone on the
 * key's probe path.  full_key_space: 0 (default) = keys 0 and ~0 are the
 * empty and deleted markers and operations on them return code 3 with the
 * CHT_STATUS_RESERVED bit; 1 = the two keys are stored in two special slots
 * beside the table and behave like any other key (every operation, export,
 * and the live count of cht_size include them; they never occupy a cell and
 * migrations leave them alone).  partition: 1 = run a batch hash-partitioned
 * (Sec. 4.5 "Bulk Operations": sort the batch by hash and co-partition it
 * with the table; tables of at least 256 cells, batches below 2^32
 * operations): the batch is first reordered by the top 8 bits of the hash
 * (which 1/256 of the table each probe starts in), the operation runs over
 * the reordered batch in order so the table lines in use stay in L2, and the
 * results are put back into the caller's order; about 19 bytes of
 * stream-ordered device scratch per operation for the call.  0 (default) =
 * the direct kernel.  Results are the same either way.  Measured on GB300
 * (2^26 cells, 2^25 operations): the reorder and the gather cost about 16 ns
 * per operation, more than the L2 locality saves except for misses at load
 * 0.9 (4.46 vs 4.97 ms), so it is off by default.  grow_in_kernel: 1 = an
 * insert / insert_or_update on a growable table without table options runs as
 * one cooperative kernel launch that migrates between its operation rounds
 * (Sec. 4.3.2, the operating threads are recruited for the migration; grid
 * barriers with bounded waits instead of the host reading the counters back
 * between chunks); it allocates two tables of the largest capacity the batch
 * can need for the call and reads the final state back once (one
 * synchronization of the stream).  A barrier wait longer than grow_spin_us
 * microseconds (0 = one second) ends the launch with CHT_ERR_TIMEOUT, the
 * table valid and the batch partly applied.  0 (default) = host-driven chunks.
 * grow_fault_inject: testing only; 1 = one block of the growth launch never
 * reaches a barrier, so the others' waits run out. */
typedef struct {
    int group_width;
    int lane_cells;
    int ctas_per_sm;
    int migrate_tile;
    double alpha;
    int iou_aggregate;
    int reuse_tombstones;
    int full_key_space;
    int partition;
    int grow_in_kernel;
    int grow_spin_us;
    int grow_fault_inject;
} cht_config;

/* Create a table of at least `capacity` cells (rounded up to a power of two,
 * minimum 64, maximum 2^40), all empty (Sec. 3 "Initialization").  growable
 * != 0: insert and insert_or_update migrate the table to a larger (gamma = 2)
 * or same-size (gamma = 1, tombstone purge) one before the number of
 * non-empty cells could exceed alpha * c (Sec. 4.3.2, Sec. 4.4).  The table
 * memory is zeroed on `stream`.  CHT_ERR_OOM if the memory is not there. */
cht_status cht_create(uint64_t capacity, int growable, cht_stream_t stream, cht_handle *out);

/* Free the table (stream-ordered on its last stream) and the handle. */
cht_status cht_destroy(cht_handle h);

/* Replace the tunables (NULL restores defaults).  Takes effect on the next call. */
cht_status cht_set_config(cht_handle h, const cht_config *cfg);
cht_status cht_get_config(cht_handle h, cht_config *cfg);

/* insert (Sec. 3, Algorithm 1 with the insert return rule): for each i <
 * n, store <keys[i], vals[i]> unless the key is present.  If several
 * operations of the batch carry the same absent key, exactly one of them
 * inserts (code 1; the stored value is that operation's) and the others
 * report 0.  keys/vals: n u64 each; inserted: n u8 result codes or NULL. */
cht_status cht_insert(cht_handle h, const uint64_t *keys, const uint64_t *vals, uint64_t n,
                      uint8_t *inserted, cht_stream_t stream);

/* Sort-based bulk build (Sec. 3 "Bulk Operations") of an EMPTY table (no
 * insert since creation or the last cht_clear; else CHT_ERR_INVALID_ARG) from
 * n < 2^32 pairs.  Of equal keys the last (in input order) is kept.  The
 * pairs are ordered by the top B bits of the 64-bit hash (B = 32 for tables
 * of up to 2^32 cells, else log2(c) rounded up to a multiple of 8), ties in
 * input order, and placed as inserting them one by one in that order would
 * place them; the layout is therefore deterministic.  A growable table first
 * takes the smallest capacity >= c with n <= alpha * c'.  Keys 0 / ~0 go to
 * the special slots with the full key space on, else they are skipped and
 * set the RESERVED status bit.  CHT_ERR_TABLE_FULL, table unchanged, if the
 * distinct keys would leave no empty cell (only possible for n >= c; the call
 * then synchronizes `stream` once).  keys / vals: n u64 each, host or device;
 * the scratch (about 32 B per pair) is freed stream-ordered. */
cht_status cht_build(cht_handle h, const uint64_t *keys, const uint64_t *vals, uint64_t n,
                     cht_stream_t stream);

/* Bulk merge of a batch into a table that may hold elements (Sec. 4.5: sort
 * the batch by hash, keep the last of equal keys, and merge batch and table
 * into a new table).  The new table is the sorted placement of the table's
 * live elements, in cell index order, followed by the batch in input order:
 * ordered by the top B hash bits as in cht_build (ties in that order), all
 * but the last of equal keys dropped -- so a batch element replaces the
 * table's element of the same key and the last of equal batch keys wins --
 * and placed as inserting them one by one in that order would; tombstones are
 * dropped.  The layout is deterministic given the table's cells.  A growable
 * table takes the smallest capacity >= c with live + n <= alpha * c'; a
 * bounded one keeps c and returns CHT_ERR_TABLE_FULL, table unchanged, if no
 * empty cell would remain.  Keys 0 / ~0 of the batch: the special slots (last
 * value) with the full key space on, else skipped with the RESERVED status
 * bit; slots the batch does not name keep their content.  live + n < 2^32.
 * The call reads the live count back (one synchronization of `stream`);
 * scratch of about 48 B per element of the concatenation plus the new cells
 * are allocated stream-ordered, the old cells freed stream-ordered.  keys /
 * vals: n u64 each, host or device. */
cht_status cht_merge(cht_handle h, const uint64_t *keys, const uint64_t *vals, uint64_t n,
                     cht_stream_t stream);

/* find (Sec. 3 "Lookup", copy semantics): vals_out[i] = the value stored
 * with keys[i], or 0 if absent; found[i] = 1 / 0 (3 for a reserved key).
 * Writes nothing to the table.  vals_out: n u64 (required); found: n u8 or NULL. */
cht_status cht_find(cht_handle h, const uint64_t *keys, uint64_t n, uint64_t *vals_out,
                    uint8_t *found, cht_stream_t stream);

/* insertOrUpdate (Sec. 3, Algorithm 1): insert <k, d> if k is absent, else
 * update its value by `op` (CHT_ADD: fetch-and-add; CHT_OVERWRITE: store).
 * Code 1 iff this operation inserted: for an absent key exactly one of the
 * batch's operations on it reports 1.  With CHT_ADD the final value is the
 * previous value (0 if absent) plus the sum of the batch's d for that key,
 * mod 2^64, independent of order; with CHT_OVERWRITE it is one of those d. */
cht_status cht_insert_or_update(cht_handle h, const uint64_t *keys, const uint64_t *vals,
                                uint64_t n, cht_update_op op, uint8_t *inserted,
                                cht_stream_t stream);

/* update (Sec. 3, update(x, d, up)): if keys[i] is present, change its value
 * by `op` (CHT_ADD: fetch-and-add d; CHT_OVERWRITE: store d) and report 1;
 * if absent, report 0 and change nothing (3 for a reserved key).  Never fills
 * a cell, so it never grows the table.  Every operation on a present key
 * reports 1; with CHT_ADD the final value is the previous one plus the sum
 * of the batch's d for that key, mod 2^64; with CHT_OVERWRITE it is one of
 * those d.  keys/vals: n u64 each; updated: n u8 result codes or NULL. */
cht_status cht_update(cht_handle h, const uint64_t *keys, const uint64_t *vals, uint64_t n,
                      cht_update_op op, uint8_t *updated, cht_stream_t stream);

/* erase (Sec. 4.4): replace the key of the cell holding keys[i] by the
 * tombstone (value kept).  For a present key exactly one of the batch's
 * operations on it reports 1.  Tombstones keep occupying their cells until
 * the next migration purges them. */
cht_status cht_erase(cht_handle h, const uint64_t *keys, uint64_t n, uint8_t *erased,
                     cht_stream_t stream);

/* Migrate into a new table of new_capacity cells (rounded up to a power of
 * two, minimum 64), dropping tombstones (Sec. 4.3.1, Sec. 4.4).
 * new_capacity = 0 applies the growth policy: double if more than alpha*c/2
 * elements are live, else keep the size.  Growing or keeping the size
 * (gamma >= 1): the cell layout equals the sequential migration that visits
 * the old cells in index order from a cluster start (Lemma 1).  Shrinking
 * (Sec. 4.3.1 "Shrinking"; the live elements must be fewer than the new
 * capacity, else CHT_ERR_INVALID_ARG and no change): each block of the target
 * takes the elements that land in it, the rest are inserted concurrently;
 * the occupied cells equal those of the sequential migration, which key sits
 * where may differ.  The new table is allocated before the old one is
 * released: on CHT_ERR_OOM the table is unchanged.  Reads the live count
 * back from the device when the policy or a shrink needs it (synchronizes
 * `stream`). */
cht_status cht_migrate(cht_handle h, uint64_t new_capacity, cht_stream_t stream);

/* Synchronize `stream` and report: live elements (I - D, plus the keys in
 * the special slots under full_key_space), non-empty cells I (tombstones
 * included), capacity c.  Any out-pointer may be NULL.
 * Returns CHT_ERR_TABLE_FULL / CHT_ERR_RESERVED_KEY if the sticky status has
 * that bit set (the status is not cleared), else CHT_OK. */
cht_status cht_size(cht_handle h, uint64_t *live, uint64_t *nonempty, uint64_t *capacity,
                    cht_stream_t stream);

/* Synchronize `stream`, return the sticky status bits in *bits and clear them. */
cht_status cht_get_status(cht_handle h, uint32_t *bits, cht_stream_t stream);

/* forall (Sec. 3 "Bulk Operations"): write the live elements to keys_out /
 * vals_out (max_n entries each, in no particular order) and their number to
 * *n_out; fails with CHT_ERR_INVALID_ARG, writing the number to *n_out, if it
 * exceeds max_n.  vals_out may be NULL.  Synchronizes `stream`. */
cht_status cht_export(cht_handle h, uint64_t *keys_out, uint64_t *vals_out, uint64_t max_n,
                      uint64_t *n_out, cht_stream_t stream);

/* Copy the raw cell array (2*c u64: key, value, key, value, ...) to
 * cells_out, which holds max_cells cells; *n_cells receives c.  Used to check
 * layouts.  Asynchronous for device memory. */
cht_status cht_copy_cells(cht_handle h, uint64_t *cells_out, uint64_t max_cells,
                          uint64_t *n_cells, cht_stream_t stream);

/* Make every cell empty again and reset the counters (capacity unchanged). */
cht_status cht_clear(cht_handle h, cht_stream_t stream);

/* ---- Batched engine: many tables, many batches, one persistent launch -------
 * A plan holds a list of batches over any number of tables (all on one
 * device).  Each batch is one operation type on one table, exactly as a
 * single call of cht_find / cht_insert / cht_insert_or_update / cht_erase
 * would run it; batches on the same table run in list order with phase
 * semantics (every operation of an earlier batch before any of a later one),
 * batches on different tables are independent and overlap on the device.
 * cht_plan_launch runs the whole plan in ONE kernel launch: the batches are
 * cut into work items of 256 operations that warps of a persistent grid take
 * from a device work queue; an item waits (bounded) until its table's earlier
 * items are done.  Arrays must be device memory and stay valid while the plan
 * exists; the plan applies no growth policy (a full table reports code 2).
 * The launch is stream-ordered and can be captured in a CUDA graph. */
typedef enum {
    CHT_OP_FIND = 0,
    CHT_OP_INSERT = 1,
    CHT_OP_IOU_ADD = 2,
    CHT_OP_IOU_OVERWRITE = 3,
    CHT_OP_ERASE = 4,
    CHT_OP_UPDATE_ADD = 5,
    CHT_OP_UPDATE_OVERWRITE = 6
} cht_op_kind;

typedef struct {
    cht_handle table;
    int op;                 /* cht_op_kind */
    const uint64_t *keys;   /* n keys */
    const uint64_t *vals;   /* n values (insert, insert-or-update), else NULL */
    uint64_t n;
    uint64_t *vals_out;     /* n found values (find), else NULL */
    uint8_t *codes;         /* n result codes as for the single calls, or NULL */
} cht_batch_op;

typedef struct cht_plan *cht_plan_handle;

/* group_width / lane_cells: probe window as in cht_config (0 = 1 lane x one
 * sector); ctas_per_sm: 0 = occupancy maximum; spin_limit_us: bound of one
 * dependency wait (0 = about one second) -- a wait that runs out stops the
 * launch with CHT_PLAN_TIMEOUT in the plan status; fault_inject: testing
 * only, bit 0 makes the first work item wait for a count nothing reaches;
 * direct_io: 0 = each warp copies its work item's keys and values into
 * shared memory with one coalesced pass and writes results back with one
 * (the default), 1 = the probe loops read and write the batch arrays in
 * place; chunk_ops: operations per work item, 32 / 64 / 128 / 256, or 0 =
 * per table: 256 unless the table's chain of dependent batches would
 * outlast the plan's other work, then smaller (more warps per batch);
 * poll_ns: longest sleep of a waiting work item between two polls of its
 * table's completion counter (0 = 8192 ns; the sleep is 16 ns per item still
 * awaited, at least 128 ns; longer = less traffic on that counter, later
 * wake-up). */
typedef struct {
    int group_width;
    int lane_cells;
    int ctas_per_sm;
    int spin_limit_us;
    int fault_inject;
    int direct_io;
    int chunk_ops;
    int poll_ns;
} cht_plan_config;

#define CHT_PLAN_TIMEOUT 0x1u

/* Build a plan from n_ops batch descriptors (copied; the arrays they point to
 * are not).  Validates every descriptor (host arrays are rejected with
 * CHT_ERR_INVALID_ARG).  The engine reads a work item's keys and values
 * before the work it depends on has finished, so no batch's keys / vals may
 * overlap any batch's vals_out / codes (CHT_ERR_INVALID_ARG otherwise).
 * Allocates the plan's device buffers. */
cht_status cht_plan_create(const cht_batch_op *ops, uint64_t n_ops, cht_plan_handle *out);
cht_status cht_plan_set_config(cht_plan_handle p, const cht_plan_config *cfg);
cht_status cht_plan_get_config(cht_plan_handle p, cht_plan_config *cfg);
/* Run the plan: reset its counters and launch the engine on `stream`. */
cht_status cht_plan_launch(cht_plan_handle p, cht_stream_t stream);
/* Synchronize `stream` and return the status bits of the last launch. */
cht_status cht_plan_status(cht_plan_handle p, uint32_t *bits, cht_stream_t stream);
/* Try the engine's probe windows and CTAs/SM on this plan and keep the
 * fastest by the median of three runs each: every run works on the plan's
 * tables, which are restored from a copy afterwards (their contents are
 * unchanged on return; the plan's output arrays hold the results of the last
 * run).  *best_ms (nullable) receives the best median.  Needs device memory
 * for one copy of every table. */
cht_status cht_plan_autotune(cht_plan_handle p, cht_stream_t stream, double *best_ms);
cht_status cht_plan_destroy(cht_plan_handle p);

/* ---- Serving loop: continuous batching over resident tables ----------------
 * A server owns a queue of requests over a fixed set of tables (each request:
 * one operation type on one table, host or device arrays).  Every scheduling
 * step admits queued requests as device memory in its request arena frees up,
 * copies their inputs in, runs all of them in ONE engine launch (requests on
 * the same table in arrival order, phase semantics as for single calls; other
 * tables overlap), copies the results back and records when each request
 * completes.  The next step is prepared and launched while the previous one
 * still runs (up to max_inflight_steps), so requests that arrive meanwhile
 * join the next step: continuous batching.  Growable tables keep the load
 * bound: before an insert / insert-or-update request whose operations could
 * push a table's non-empty cells (known exactly from counters snapshotted
 * after each step, plus what is in flight) past alpha * c, the table is
 * migrated, stream-ordered, to the smallest capacity that holds them all.  A
 * request larger than a step (max_step_ops) or than the free arena is
 * admitted in parts; later requests on its table wait for the rest.
 * Admission keeps the tables plus the arena within memory_cap_bytes and every
 * growth within the device's free memory: before a step grows a table it asks
 * the device for its free bytes (cudaMemGetInfo, plus what the stream-ordered
 * pool holds unused) and admits the growth only if hbm_reserve_bytes remain
 * free afterwards; otherwise the table's requests wait for steps in flight to
 * finish.  A request whose table can never fit is rejected (CHT_ERR_OOM). */
typedef struct cht_server *cht_server_handle;

typedef struct {
    uint64_t memory_cap_bytes;   /* tables + request arena (0 = no cap) */
    uint64_t arena_bytes;        /* device ring for staged request data (0 = 1 GiB) */
    uint32_t max_inflight_steps; /* 0 = 2 */
    uint32_t max_step_requests;  /* 0 = 8192 */
    uint64_t max_step_ops;       /* 0 = 2^26 */
    int stage_inputs;            /* 0: the engine reads and writes request arrays the
                                    GPU can address (device memory, pinned host memory,
                                    pageable host memory where the device reports
                                    pageable-memory access -- NVLink-C2C on Grace) in
                                    place and stages only the others through the
                                    arena; 1: stage every request through the arena */
    uint64_t hbm_reserve_bytes;  /* device memory to leave free when admitting a
                                    growth (0 = 1 GiB) */
} cht_server_config;

/* A request's arrays must stay alive and unchanged until it completes, and
 * its keys / vals must not overlap the vals_out / codes of any request in
 * flight (the engine reads inputs ahead of the work they wait for). */
typedef struct {
    uint32_t table;          /* index into the server's table list */
    int op;                  /* cht_op_kind */
    const uint64_t *keys;
    const uint64_t *vals;    /* insert / insert-or-update */
    uint64_t n;              /* 0 < n */
    uint64_t *vals_out;      /* find */
    uint8_t *codes;          /* nullable */
} cht_request;

/* tables: n_tables handles on one device; the server does not own them. */
cht_status cht_server_create(const cht_handle *tables, uint32_t n_tables, const cht_server_config *cfg,
                             cht_stream_t stream, cht_server_handle *out);
/* Queue a request; its arrival time is now.  *id (nullable) receives its id
 * (0, 1, 2, ... in submission order).  The arrays must stay valid until the
 * request completes. */
cht_status cht_server_submit(cht_server_handle s, const cht_request *req, uint64_t *id);
/* One scheduling iteration without blocking: note completed steps, admit
 * queued requests and launch a step if there is room.  Counts are nullable. */
cht_status cht_server_step(cht_server_handle s, uint32_t *admitted, uint32_t *completed);
/* Run scheduling iterations until every submitted request has completed. */
cht_status cht_server_drain(cht_server_handle s);
/* State of request id: *done = 1 when completed (its outputs are in place),
 * *latency_s = completion - arrival, *req_status = CHT_OK or the reason it
 * was rejected (a request larger than the arena: CHT_ERR_OOM). */
cht_status cht_server_result(cht_server_handle s, uint64_t id, int *done, double *latency_s,
                             cht_status *req_status);
/* Replay: submit request i when arrival_s[i] seconds have passed since the
 * call started (arrival_s non-decreasing), schedule continuously until all
 * have completed; latency_s[i] (nullable) = completion - scheduled arrival;
 * *makespan_s (nullable) = last completion - start. */
cht_status cht_server_replay(cht_server_handle s, const cht_request *reqs, const double *arrival_s,
                             uint64_t n, double *latency_s, double *makespan_s);
/* Steps launched so far and requests completed so far. */
cht_status cht_server_stats(cht_server_handle s, uint64_t *steps, uint64_t *completed);

/* Where a server's time went, summed over the steps that have completed
 * (times from CUDA events on the server's stream; host time from the wall
 * clock).  gpu_step_ms: device time from a step's first migration or copy to
 * its last copy back (steps run one after another on the stream, so the
 * makespan minus this is time the stream had no step to run); engine_ms: the
 * engine launches (with the step's metadata upload when no migration or copy
 * precedes the launch); host_admit_ms: host time spent admitting requests
 * and preparing launches (steps that launched); rounds: sum over steps of
 * the longest chain of dependent batches (one table's requests in arrival
 * order); parts: request parts launched; chunks: engine work items;
 * migrations: growth migrations started. */
typedef struct {
    uint64_t steps;
    uint64_t completed;
    uint64_t parts;
    uint64_t chunks;
    uint64_t rounds;
    uint64_t migrations;
    double gpu_step_ms;
    double engine_ms;
    double host_admit_ms;
} cht_server_profile;
cht_status cht_server_get_profile(cht_server_handle s, cht_server_profile *out);

/* One record per completed step, in completion order.  gpu_ms / engine_ms
 * as in cht_server_profile; ops: operations launched; rounds: longest chain
 * of dependent batches; max_table_log2: log2 cells of the largest table of
 * the server at launch; recut: 1 if the step's work items were cut at 256
 * operations because the per-table sizing needed more metadata than a step
 * may use. */
typedef struct {
    double gpu_ms;
    double engine_ms;
    uint64_t parts;
    uint64_t items;
    uint64_t ops;
    uint64_t rounds;
    uint64_t migrations;
    uint32_t max_table_log2;
    uint32_t recut;
} cht_server_step_record;
/* Copy up to max records (from the first step) into out; *n = records kept. */
cht_status cht_server_get_trace(cht_server_handle s, cht_server_step_record *out, uint64_t max, uint64_t *n);
cht_status cht_server_destroy(cht_server_handle s);

/* Cap, in bytes, on the device memory this library allocates at any time for
 * tables and staging (0 = no cap).  An allocation that would exceed it fails
 * with CHT_ERR_OOM exactly like a failed cudaMalloc. */
cht_status cht_set_memory_limit(uint64_t bytes);
uint64_t cht_memory_in_use(void);

/* Number of kernel launches this library has issued (process-wide). */
uint64_t cht_launch_count(void);

/* find without any device allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc where they look keys up -- a process
 * whose device memory another allocator already owns (a framework's caching
 * pool, a serving system's fixed arena), a latency-critical path that must not
 * block or synchronize on an allocation, or an embedding with a fixed memory
 * budget.  Same arguments and results as cht_find; keys, vals_out and found
 * may be host or device arrays.  Keys and results pass through one fixed
 * scratch array in device memory that the library holds on every GPU that
 * loads it until the process exits (CHT_NOALLOC_MAX_KEYS * 17 bytes, about
 * 1.1 MiB); batches larger than CHT_NOALLOC_MAX_KEYS return
 * CHT_ERR_INVALID_ARG.  The first call on a device looks up the scratch's
 * device address there; make that first call before any stream capture.
 * Every call shares the one scratch array: calls whose work overlaps on the
 * GPU (different streams or threads, not ordered) race and may return each
 * other's results, so order them.  Results in host arrays are valid once the
 * stream has been synchronized.  Allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine). */
#define CHT_NOALLOC_MAX_KEYS 65536u
cht_status cht_find_noalloc(cht_handle h, const uint64_t *keys, uint64_t n, uint64_t *vals_out,
                            uint8_t *found, cht_stream_t stream);

/* Single-call autotuner.  Times one batch of operation `op` (CHT_OP_FIND,
 * _INSERT, _ERASE, _UPDATE_ADD / _OVERWRITE, _IOU_ADD / _OVERWRITE through the
 * probe kernel) on this table with every probe window -- group width G in
 * {-1 (one thread per operation), 1, 2, 4, 8, 16, 32}, cells per lane V in
 * {1, 2, 4} where the kernels exist,
 * resident CTAs per SM in {occupancy maximum, 4} -- `trials` times each (at
 * least 3; a find trial is the mean of 8 launches back to back), restoring the
 * table's cells and counters before every trial of a modifying operation and
 * once more at the end, so the table is unchanged.
 * results[0 .. *n_results) receive every candidate with the median of its
 * trials, fastest first (max_results bounds the count).  keys / vals: device
 * arrays of n entries (vals for operations with values).  Tables with tombstone
 * reuse or the full key space are not tuned (CHT_ERR_INVALID_ARG).  Scratch of
 * the table's size is allocated for the call.  The library's automatic window
 * rule comes from running this over table sizes and loads (the generator is
 * paper_1601_04017_gb300/tune.py). */
typedef struct {
    int group_width;
    int lane_cells;
    int ctas_per_sm;  /* 0 = occupancy maximum */
    double ms;        /* median over the trials */
} cht_tune_result;
cht_status cht_tune(cht_handle h, int op, const uint64_t *keys, const uint64_t *vals, uint64_t n, int trials,
                    cht_tune_result *results, uint32_t max_results, uint32_t *n_results, cht_stream_t stream);

/* Static string for a status code. */
const char *cht_status_string(cht_status s);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int cht_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CHT_H */
