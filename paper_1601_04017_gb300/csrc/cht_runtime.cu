// Host runtime and C ABI of libcht (declared in include/cht.h).
//
// The runtime owns the table memory, validates arguments, stages host
// arrays through device buffers, and applies the growth policy of growable
// tables: before a batch that could push the number of non-empty cells I
// past alpha*c it reads I back, inserts a chunk that fits, and migrates the
// table -- doubling it when more than alpha*c/2 elements are live, otherwise
// migrating at the same size to purge tombstones (Sec. 4.3.2 trigger and
// growth factor; Sec. 4.4 size choice by the live count I - D).  Migration
// and operations are ordered on the caller's stream, which gives the
// "synchronized" growing protocol of Sec. 4.3.2: no operation runs while a
// migration does, so fetch-and-add updates stay legal.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/cht.h"
#include "cht_internal.h"

using cht::Cell;
using cht::DevState;
using cht::u32;
using cht::u64;

namespace {

constexpr u64 kMinCap = 64;
constexpr u32 kMaxLog2 = 40;

std::atomic<u64> g_launches{0};
std::atomic<u64> g_mem_in_use{0};
std::atomic<u64> g_mem_limit{0};
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Keep freed stream-ordered memory in the pool so repeated staging and
// migrations do not go back to the driver.
void prepare_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64 || g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        u64 thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready[dev] = true;
}

// Stream-ordered allocation with the library-wide memory cap.
cht_status lib_alloc(void** p, u64 bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    const u64 lim = g_mem_limit.load();
    const u64 now = g_mem_in_use.fetch_add(bytes) + bytes;
    if (lim != 0 && now > lim) {
        g_mem_in_use.fetch_sub(bytes);
        return CHT_ERR_OOM;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_mem_in_use.fetch_sub(bytes);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? CHT_ERR_OOM : CHT_ERR_CUDA;
    }
    if ((reinterpret_cast<uintptr_t>(*p) & 255u) != 0) {  // cells need 32-byte alignment
        cudaFreeAsync(*p, s);
        g_mem_in_use.fetch_sub(bytes);
        *p = nullptr;
        return CHT_ERR_CUDA;
    }
    return CHT_OK;
}

void lib_free(void* p, u64 bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    cudaFreeAsync(p, s);
    g_mem_in_use.fetch_sub(bytes);
}

bool is_host_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Stages host arrays of one call through device buffers on the stream.
class Staging {
  public:
    explicit Staging(cudaStream_t s) : s_(s) {}
    ~Staging() { release(); }

    // Device view of an input array (copied in when it lives on the host).
    cht_status in(const void* p, u64 bytes, const void** out) {
        *out = p;
        if (!p || bytes == 0 || !is_host_pointer(p)) return CHT_OK;
        void* d = nullptr;
        cht_status st = lib_alloc(&d, bytes, s_);
        if (st != CHT_OK) return st;
        bufs_.push_back({d, bytes});
        if (cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s_) != cudaSuccess) return CHT_ERR_CUDA;
        *out = d;
        return CHT_OK;
    }

    // Device view of an output array (copied back by finish()).
    cht_status out(void* p, u64 bytes, void** out) {
        *out = p;
        if (!p || bytes == 0 || !is_host_pointer(p)) return CHT_OK;
        void* d = nullptr;
        cht_status st = lib_alloc(&d, bytes, s_);
        if (st != CHT_OK) return st;
        bufs_.push_back({d, bytes});
        backs_.push_back({p, d, bytes});
        *out = d;
        return CHT_OK;
    }

    cht_status finish() {
        cht_status r = CHT_OK;
        for (const Back& b : backs_)
            if (cudaMemcpyAsync(b.host, b.dev, b.bytes, cudaMemcpyDeviceToHost, s_) != cudaSuccess)
                r = CHT_ERR_CUDA;
        backs_.clear();
        release();
        return r;
    }

  private:
    struct Buf {
        void* p;
        u64 bytes;
    };
    struct Back {
        void* host;
        void* dev;
        u64 bytes;
    };
    void release() {
        for (const Buf& b : bufs_) lib_free(b.p, b.bytes, s_);
        bufs_.clear();
    }
    cudaStream_t s_;
    std::vector<Buf> bufs_;
    std::vector<Back> backs_;
};

cht_config default_config() {
    cht_config c;
    c.group_width = 0;
    c.lane_cells = 0;
    c.ctas_per_sm = 0;
    c.migrate_tile = 0;
    c.alpha = 0.5;
    c.iou_aggregate = 1;
    c.reuse_tombstones = 0;
    c.full_key_space = 0;
    c.partition = 0;
    c.grow_in_kernel = 0;
    c.grow_spin_us = 0;
    c.grow_fault_inject = 0;
    return c;
}

bool valid_config(const cht_config& c) {
    const int g = c.group_width;
    if (!(g == -1 || g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32)) return false;
    if (!(c.lane_cells == 0 || c.lane_cells == 1 || c.lane_cells == 2 || c.lane_cells == 4)) return false;
    if (g == -1 && c.lane_cells == 1) return false;
    if ((g == 32 && c.lane_cells >= 2) || (g == 16 && c.lane_cells == 4)) return false;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 64) return false;
    const int t = c.migrate_tile;
    if (t != 0 && (t < 64 || t > 8192 || (t & (t - 1)) != 0)) return false;
    if (!(c.alpha > 0.0 && c.alpha < 1.0)) return false;
    if (c.iou_aggregate < 0 || c.iou_aggregate > 3) return false;
    if (c.reuse_tombstones < 0 || c.reuse_tombstones > 1) return false;
    if (c.full_key_space < 0 || c.full_key_space > 1) return false;
    if (c.partition < 0 || c.partition > 1) return false;
    if (c.grow_in_kernel < 0 || c.grow_in_kernel > 1 || c.grow_spin_us < 0 || c.grow_fault_inject < 0 ||
        c.grow_fault_inject > 1)
        return false;
    return true;
}

u32 log2_ceil_cap(u64 capacity) {
    u32 l = 6;
    while (l < kMaxLog2 && (1ull << l) < capacity) ++l;
    return l;
}

}  // namespace

struct cht_table {
    Cell* cells = nullptr;
    u64 cells_bytes = 0;  // size of the cells' allocation (at least cap() cells)
    u32 log2c = 0;
    DevState* st = nullptr;
    int growable = 0;
    int device = 0;
    cht_config cfg = default_config();
    u64 i_bound = 0;      // upper bound on the device's I
    bool i_exact = true;  // i_bound equals the device's I
    cudaStream_t last = nullptr;

    u64 cap() const { return 1ull << log2c; }
};

namespace {

cht_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CHT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CHT_ERR_OOM : CHT_ERR_CUDA;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

cht_status read_state(cht_table* h, DevState* out, cudaStream_t s) {
    if (cudaMemcpyAsync(out, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CHT_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

// Migrate h into 2^new_log2 cells (new_log2 >= log2c).  `live` is the exact
// live count if known (else ~0).  Allocates first: on failure h is unchanged.
cht_status do_migrate(cht_table* h, u32 new_log2, u64 live, cudaStream_t s) {
    // everything is allocated before the table's counters are touched: on
    // CHT_ERR_OOM the table is unchanged
    const bool shrink = new_log2 < h->log2c;
    if (shrink && live == ~0ull) return CHT_ERR_INVALID_ARG;  // shrinking needs the exact live count
    Cell* dst = nullptr;
    const u64 bytes = (1ull << new_log2) * sizeof(Cell);
    cht_status r = lib_alloc(reinterpret_cast<void**>(&dst), bytes, s);
    if (r != CHT_OK) return r;
    // below load 0.6 (short clusters) one lane re-inserts each cluster; above
    // it (long clusters) the warp places 32 cells at a time.  Tiles of 512 and
    // 1024 cells were the fastest of 256..2048 for each (2^28 cells, GB300).
    const bool windows = double(h->i_bound) >= 0.6 * double(h->cap());
    int tile = h->cfg.migrate_tile;
    if (tile == 0) tile = windows ? 1024 : 512;
    // scratch: the moved border of every migration tile (growing), or the
    // spill list of c' cells plus its counter (shrinking)
    const u64 sbytes = shrink ? bytes + 256 : cht::migrate_border_count(h->log2c, tile) * sizeof(u64);
    unsigned char* scratch = nullptr;
    r = lib_alloc(reinterpret_cast<void**>(&scratch), sbytes, s);
    if (r != CHT_OK) {
        lib_free(dst, bytes, s);
        return r;
    }
    // I and D restart (the kernels accumulate the moved count into I)
    cudaError_t e = cudaMemsetAsync(&h->st->I, 0, 2 * sizeof(u64), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->st->mig_fail, 0, sizeof(u32), s);
    if (shrink) {
        unsigned long long* nspill = reinterpret_cast<unsigned long long*>(scratch + bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(nspill, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess)
            e = cht::launch_shrink(h->cells, h->log2c, dst, new_log2, h->st, reinterpret_cast<Cell*>(scratch),
                                   nspill, s);
    } else if (e == cudaSuccess) {
        e = cht::launch_migrate(h->cells, h->log2c, dst, new_log2, h->st, tile, windows,
                                reinterpret_cast<u64*>(scratch), s);
    }
    lib_free(scratch, sbytes, s);
    if (e != cudaSuccess) {
        lib_free(dst, bytes, s);
        return cuda_status(e);
    }
    lib_free(h->cells, h->cells_bytes, s);
    h->cells = dst;
    h->cells_bytes = bytes;
    h->log2c = new_log2;
    if (live != ~0ull) {
        h->i_bound = live;
        h->i_exact = true;
    } else {
        h->i_exact = false;  // new I <= old I, so i_bound stays an upper bound
    }
    return CHT_OK;
}

// Probe width for a batch: the configured one, or (auto) by the load the
// probes will see -- short probes want one sector per lane (G = 1), long
// probes at high load want wider windows so fewer dependent steps are needed.
struct Width {
    int g, v;
    int ctas = 0;  // resident CTAs per SM from the measured rule (0 = the configured / maximum)
};

// The measured rule (cht_tuned.inc, written by tune.py): per operation kind,
// range of log2 c and load band, the fastest window of the tuning sweep.
struct TunedWindow {
    int mode;
    u32 log2_lo, log2_hi;
    float load_lo, load_hi;
    int g, v, ctas;
};
const TunedWindow kTuned[] = {
#include "cht_tuned.inc"
    {-1, 0, 0, 0.f, 0.f, 0, 0, 0}};

bool tuned_window(cht::Mode mode, u32 log2c, double load, Width* w) {
    // insertOrUpdate tunes like insert, update (overwrite) like update (add)
    const int m = (mode == cht::kIouAdd || mode == cht::kIouOverwrite) ? int(cht::kInsert)
                  : mode == cht::kUpdOverwrite                          ? int(cht::kUpdAdd)
                                                                        : int(mode);
    for (const TunedWindow& t : kTuned) {
        if (t.mode != m || log2c < t.log2_lo || log2c > t.log2_hi || load < t.load_lo || load >= t.load_hi) continue;
        w->g = t.g;
        w->v = t.v;
        w->ctas = t.ctas;
        return true;
    }
    return false;
}

Width pick_width(const cht_table* h, cht::Mode mode, u64 n) {
    Width w{h->cfg.group_width, h->cfg.lane_cells};
    if (w.g == 0) {
        // Only a plain insert batch is assumed to add n new cells; insertOrUpdate
        // batches are mostly updates of few hot keys, which want G = 1.  Measured
        // on GB300 (2^28 cells, 2^27 operations per call): a random access moves
        // a whole 128-byte DRAM line, so below load 0.6 finds read one line per
        // step (2 lanes x 2 sectors) and modifications one sector per lane;
        // above it finds and inserts use 4 lanes x 2 sectors (256-byte windows,
        // two lines, each lane's two loads in flight together) and the others
        // 4 lanes x 1 sector.
        u64 filled = h->i_bound;
        if (mode == cht::kInsert) filled += n;
        if (filled > h->cap()) filled = h->cap();
        const double load = double(filled) / double(h->cap());
        if (h->cfg.lane_cells == 0 && tuned_window(mode, h->log2c, load, &w)) return w;
        if (load < 0.6) {
            w.g = mode == cht::kFind ? 2 : 1;
            if (w.v == 0) w.v = mode == cht::kFind ? 4 : 2;
        } else {
            w.g = 4;
            if (w.v == 0) w.v = (mode == cht::kFind || mode == cht::kInsert) ? 4 : 2;
        }
    }
    if (w.g == -1) w.v = w.v == 2 ? 2 : 4;
    else if (w.g == 1 && w.v != 4) w.v = 2;
    else if (w.v == 0 || w.g == 32) w.v = 1;
    return w;
}

// Operations per in-order piece of a warp on a partitioned batch: the grid
// then has about (resident warps x kOrderedChunk) operations in flight, a
// narrow range of the reordered batch and so of the table.
constexpr u32 kOrderedChunk = 128;

bool aggregated(const cht_table* h, cht::Mode mode) {
    return (mode == cht::kIouAdd || mode == cht::kIouOverwrite || mode == cht::kUpdAdd ||
            mode == cht::kUpdOverwrite) &&
           h->cfg.iou_aggregate != 0;
}

// The hash-partitioned path (Sec. 4.5), a table option (partition = 1).
bool use_partition(const cht_table* h, u64 n) {
    return h->cfg.partition == 1 && n < (1ull << 32) && h->log2c >= 8;
}

// insertOrUpdate on a hash-sorted batch (iou_aggregate = 3): the batch is
// sorted by the top 16 hash bits first, so one aggregation window holds all
// operations of the keys it sees.
bool use_sorted_agg(const cht_table* h, cht::Mode mode, u64 n) {
    return (mode == cht::kIouAdd || mode == cht::kIouOverwrite) && h->cfg.iou_aggregate == 3 && n < (1ull << 32);
}

struct KernelCtx {
    const cht_table* h;
    cht::Mode mode;
    u64 n;  // batch size for the width choice
};

cudaError_t run_kernel(const cht::OpArgs& a, void* ctx, cudaStream_t s) {
    const KernelCtx* k = static_cast<const KernelCtx*>(ctx);
    if (aggregated(k->h, k->mode))
        return cht::launch_iou_aggregated(k->mode, a, k->h->cfg.iou_aggregate == 2, k->h->cfg.ctas_per_sm, s);
    const Width w = pick_width(k->h, k->mode, k->n);
    return cht::launch_op(k->mode, a, w.g, w.v, k->h->cfg.ctas_per_sm ? k->h->cfg.ctas_per_sm : w.ctas, s);
}

// insertOrUpdate on a batch sorted by hash: 1024-thread CTAs, 4096-operation
// windows
cudaError_t run_sorted_agg(const cht::OpArgs& a, void* ctx, cudaStream_t s) {
    const KernelCtx* k = static_cast<const KernelCtx*>(ctx);
    return cht::launch_iou_aggregated_wide(k->mode, a, false, s);
}

cudaError_t run_kernel_ordered(const cht::OpArgs& a, void* ctx, cudaStream_t s) {
    cht::OpArgs b = a;
    b.chunk = kOrderedChunk;  // (the aggregation kernel walks its windows in order anyway)
    return run_kernel(b, ctx, s);
}

cht_status launch(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, u64* vals_out,
                  unsigned char* codes, u64 n, cudaStream_t s) {
    cht::OpArgs a;
    a.cells = h->cells;
    a.log2c = h->log2c;
    a.reuse = u32(h->cfg.reuse_tombstones);
    a.full_keys = u32(h->cfg.full_key_space);
    a.keys = keys;
    a.vals = vals;
    a.vals_out = vals_out;
    a.codes = codes;
    a.n = n;
    a.st = h->st;
    KernelCtx ctx{h, mode, n};
    if (n == 0) return CHT_OK;
    if (!use_partition(h, n) && use_sorted_agg(h, mode, n)) {
        const u64 bytes = cht::sorted16_scratch_bytes(n, codes != nullptr);
        void* scratch = nullptr;
        cht_status r = lib_alloc(&scratch, bytes, s);
        if (r != CHT_OK) return r;
        const cudaError_t e = cht::launch_sorted16(a, scratch, run_sorted_agg, &ctx, s);
        lib_free(scratch, bytes, s);
        return cuda_status(e);
    }
    if (!use_partition(h, n)) return cuda_status(run_kernel(a, &ctx, s));
    cht::PartitionIO io;
    io.vals = cht::mode_has_vals(mode);
    io.vals_out = vals_out != nullptr;
    io.codes = codes != nullptr;
    const u64 bytes = cht::partition_scratch_bytes(n, io);
    void* scratch = nullptr;
    cht_status r = lib_alloc(&scratch, bytes, s);
    if (r != CHT_OK) return r;
    const cudaError_t e = cht::launch_partitioned(a, io, scratch, run_kernel_ordered, &ctx, s);
    lib_free(scratch, bytes, s);
    return cuda_status(e);
}

cht_status run_modify_host(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals,
                           unsigned char* codes, u64 n, cudaStream_t s);

// In-kernel growth (cht_grow.cu): the whole batch in one cooperative launch
// that migrates between operation rounds.  The targets take the largest
// capacity the batch can need (every operation a new key); after the launch
// the host adopts the final table and frees the rest (one read-back).
// *handled = false if the batch cannot need a migration (then nothing ran).
cht_status grow_in_kernel(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, unsigned char* codes,
                          u64 n, cudaStream_t s, bool* handled) {
    *handled = false;
    const double alpha = h->cfg.alpha;
    const u64 bound = h->i_bound + n;
    if (bound <= u64(std::floor(alpha * double(h->cap())))) return CHT_OK;
    u32 ml = h->log2c;
    while (ml < kMaxLog2 && u64(std::floor(alpha * double(1ull << ml))) < bound) ++ml;
    const u64 tbytes = (1ull << ml) * sizeof(Cell);
    const u64 bbytes = cht::grow_border_count(ml) * sizeof(u64);
    Cell *t1 = nullptr, *t2 = nullptr;
    u64* border = nullptr;
    cht::GrowCtl* ctl = nullptr;
    cht_status r = lib_alloc(reinterpret_cast<void**>(&t1), tbytes, s);
    if (r == CHT_OK) r = lib_alloc(reinterpret_cast<void**>(&t2), tbytes, s);
    if (r == CHT_OK) r = lib_alloc(reinterpret_cast<void**>(&border), bbytes, s);
    if (r == CHT_OK) r = lib_alloc(reinterpret_cast<void**>(&ctl), sizeof(cht::GrowCtl), s);
    auto release = [&]() {
        lib_free(t1, tbytes, s);
        lib_free(t2, tbytes, s);
        lib_free(border, bbytes, s);
        lib_free(ctl, sizeof(cht::GrowCtl), s);
    };
    if (r != CHT_OK) {
        release();
        return r;
    }
    *handled = true;
    cht::GrowCtl init;
    std::memset(&init, 0, sizeof(init));
    init.log2c = h->log2c;
    cht::OpArgs a;
    a.cells = h->cells;
    a.log2c = h->log2c;
    a.reuse = 0;
    a.full_keys = 0;
    a.keys = keys;
    a.vals = vals;
    a.vals_out = nullptr;
    a.codes = codes;
    a.n = n;
    a.st = h->st;
    const Width w = pick_width(h, mode, 0);
    const long long spin = (h->cfg.grow_spin_us > 0 ? (long long)h->cfg.grow_spin_us : 1000000ll) * 2100;  // ~2.1 GHz
    cudaError_t e = cudaMemcpyAsync(ctl, &init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cht::launch_grow(a, mode, t1, t2, ml, alpha, ctl, border, spin, h->cfg.grow_fault_inject ? 1 : -1,
                             w.g == 1 ? 1 : 4, s);
    cht::GrowCtl fin;
    DevState ds;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fin, ctl, sizeof(fin), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ds, h->st, sizeof(ds), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release();  // the launch did not run (or its results are unknown): the table is as before
        return cuda_status(e);
    }
    // adopt the table the kernel left (a failed migration's target is dropped)
    Cell* tabs[3] = {h->cells, t1, t2};
    const u32 cur = fin.cur > 2 ? 0 : fin.cur;
    if (cur != 0) {
        lib_free(h->cells, h->cells_bytes, s);
        h->cells = tabs[cur];
        h->cells_bytes = tbytes;
        h->log2c = fin.log2c;
        if (cur == 1) t1 = nullptr;
        else t2 = nullptr;
    }
    release();
    h->i_bound = ds.I;
    h->i_exact = true;
    if (fin.error & cht::kGrowTimeout) return CHT_ERR_TIMEOUT;
    if (fin.error) {
        // a migration tile could not bound its cluster (or the targets were too
        // small): the host-driven policy, whose migration has a fallback,
        // finishes the batch
        const u64 done = fin.done;
        return run_modify_host(h, mode, keys + done, vals + done, codes ? codes + done : nullptr, n - done, s);
    }
    return CHT_OK;
}

// insert / insert_or_update with the growth policy of growable tables,
// driven from the host: read the counters, insert a chunk that fits below
// the threshold, migrate, repeat.
cht_status run_modify_host(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals,
                           unsigned char* codes, u64 n, cudaStream_t s) {
    if (!h->growable) {
        const cht_status r = launch(h, mode, keys, vals, nullptr, codes, n, s);
        h->i_bound += n;  // after the launch: the width choice projects n itself
        h->i_exact = false;
        return r;
    }
    u64 done = 0;
    while (done < n) {
        const u64 limit = u64(std::floor(h->cfg.alpha * double(h->cap())));
        const u64 rest = n - done;
        if (h->i_bound + rest <= limit) {
            cht_status r = launch(h, mode, keys + done, vals + done, nullptr, codes ? codes + done : nullptr,
                                  rest, s);
            if (r != CHT_OK) return r;
            h->i_bound += rest;
            h->i_exact = false;
            break;
        }
        u64 I = h->i_bound, D = 0;
        bool have_d = false;
        if (!h->i_exact) {
            DevState ds;
            cht_status r = read_state(h, &ds, s);
            if (r != CHT_OK) return r;
            I = ds.I;
            D = ds.D;
            have_d = true;
            h->i_bound = I;
            h->i_exact = true;
        }
        if (I >= limit) {
            if (!have_d) {
                DevState ds;
                cht_status r = read_state(h, &ds, s);
                if (r != CHT_OK) return r;
                D = ds.D;
            }
            const u64 live = I - D;
            const u64 half = u64(std::floor(h->cfg.alpha * double(h->cap()) / 2.0));
            u32 nl = h->log2c + (live > half ? 1u : 0u);
            if (nl > kMaxLog2) return CHT_ERR_OOM;
            cht_status r = do_migrate(h, nl, live, s);
            if (r != CHT_OK) return r;
            continue;
        }
        const u64 chunk = (limit - I) < rest ? (limit - I) : rest;
        cht_status r = launch(h, mode, keys + done, vals + done, nullptr, codes ? codes + done : nullptr,
                              chunk, s);
        if (r != CHT_OK) return r;
        h->i_bound += chunk;
        h->i_exact = false;
        done += chunk;
    }
    return CHT_OK;
}

// insert / insert_or_update on a table: in-kernel growth where configured and
// possible (a growable table without table options), else host-driven.
cht_status run_modify(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, unsigned char* codes, u64 n,
                      cudaStream_t s) {
    if (h->growable && h->cfg.grow_in_kernel && !h->cfg.reuse_tombstones && !h->cfg.full_key_space &&
        cht::mode_fills(mode) && n > 0) {
        bool handled = false;
        const cht_status r = grow_in_kernel(h, mode, keys, vals, codes, n, s, &handled);
        if (handled) return r;
    }
    return run_modify_host(h, mode, keys, vals, codes, n, s);
}

}  // namespace

namespace cht {

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

u64 device_free_bytes(int device) {
    DeviceGuard g(device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    u64 pooled = 0;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        unsigned long long reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            pooled = reserved - used;
    }
    cudaGetLastError();
    return u64(free_b) + pooled;
}

int sm_count() {
    static std::atomic<int> cached[64];
    const int dev = current_device();
    if (dev < 0 || dev >= 64) return 1;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v < 1) v = 1;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

namespace {

// Latency model of the engine used to size work items (chunk_ops = 0):
// a chain of dependent batches (one table's batches in order) costs per
// batch about kRoundUs (hand-off between warps, fences, the wait's
// back-off) plus kLaneOpUs per operation a lane handles in sequence
// (ceil(chunk / 32) with one lane per key); independent work runs at about
// kOpsPerUs.  A table whose chain at 256-operation items would outlast the
// whole plan's work gets smaller items (more warps per batch, fewer
// operations in sequence per lane) -- as small as needed, at least 32.
constexpr double kRoundUs = 4.0;
constexpr double kLaneOpUs = 0.8;
constexpr double kOpsPerUs = 30000.0;
// Longest run of one-item levels one warp runs in sequence.
constexpr u32 kMaxGroup = 4096;


}  // namespace

u64 plan_order(const std::vector<EngineBatch>& batches, size_t n_tables, int chunk_ops,
               std::vector<EngineChunk>& chunks) {
    const size_t nb = batches.size();
    constexpr u32 kNone = ~0u;
    // Dependency levels.  A find right after a find of the same table does
    // not wait for it (finds do not modify the table, so both see the state
    // after the last modifying batch): it joins the level of the run of finds
    // it belongs to.  Levels get global ids in batch order; per level: its
    // table, first batch, number of batches, largest batch, and the next
    // level of the same table.
    std::vector<u32> round_of(nb), level_of(nb), rounds(n_tables, 0), cur_level(n_tables, kNone);
    std::vector<char> last_find(n_tables, 0);
    std::vector<u32> lv_table, lv_first, lv_count, lv_next;
    std::vector<u64> lv_ops;
    lv_table.reserve(nb);
    lv_first.reserve(nb);
    lv_count.reserve(nb);
    lv_next.reserve(nb);
    lv_ops.reserve(nb);
    for (size_t b = 0; b < nb; ++b) {
        const u32 t = batches[b].table;
        round_of[b] = rounds[t]++;
        const bool find = batches[b].mode == kFind;
        if (!(find && last_find[t])) {
            const u32 L = u32(lv_table.size());
            if (cur_level[t] != kNone) lv_next[cur_level[t]] = L;
            lv_table.push_back(t);
            lv_first.push_back(u32(b));
            lv_count.push_back(0);
            lv_next.push_back(kNone);
            lv_ops.push_back(0);
            cur_level[t] = L;
        }
        const u32 L = cur_level[t];
        level_of[b] = L;
        ++lv_count[L];
        lv_ops[L] = std::max(lv_ops[L], batches[b].n);
        last_find[t] = find;
    }
    const size_t nl = lv_table.size();
    // work-item size per table
    std::vector<u32> chunk_of(n_tables, kChunkOps);
    if (chunk_ops > 0) {
        std::fill(chunk_of.begin(), chunk_of.end(), u32(chunk_ops));
    } else {
        u64 total = 0;
        for (const EngineBatch& eb : batches) total += eb.n;
        const double work_us = double(total) / kOpsPerUs;
        // chain length per table at items of 256 / 128 / 64 / 32 operations
        std::vector<double> chain(4 * n_tables, 0.0);
        for (size_t L = 0; L < nl; ++L)
            for (int j = 0; j < 4; ++j) {
                const u64 c = u64(kChunkOps) >> j;
                chain[4 * lv_table[L] + j] += kRoundUs + kLaneOpUs * double((std::min<u64>(lv_ops[L], c) + 31) / 32);
            }
        for (size_t t = 0; t < n_tables; ++t) {
            int j = 0;
            while (j < 3 && chain[4 * t + j] > work_us) ++j;
            chunk_of[t] = kChunkOps >> j;
        }
    }
    // Groups: runs of consecutive one-item levels of a table (one batch of at
    // most one item).  group_len[L] = levels in the group led by L, 0 for the
    // other levels of a group, 1 for a level on its own.
    std::vector<u32> group_len(nl, 1), open(n_tables, kNone);
    for (size_t L = 0; L < nl; ++L) {
        const u32 t = lv_table[L];
        const bool single = lv_count[L] == 1 && lv_ops[L] <= chunk_of[t];
        if (!single) {
            open[t] = kNone;
        } else if (open[t] != kNone && group_len[open[t]] < kMaxGroup) {
            ++group_len[open[t]];
            group_len[L] = 0;
        } else {
            open[t] = u32(L);
        }
    }
    // batches in round order (stable counting sort)
    const u32 n_rounds = n_tables ? *std::max_element(rounds.begin(), rounds.end()) : 0;
    std::vector<u32> start(size_t(n_rounds) + 1, 0), order(nb);
    for (size_t b = 0; b < nb; ++b) ++start[round_of[b] + 1];
    for (u32 r = 0; r < n_rounds; ++r) start[r + 1] += start[r];
    for (size_t b = 0; b < nb; ++b) order[start[round_of[b]]++] = u32(b);
    // Emit.  Items of each table are counted as they are emitted (followers
    // when their leader is); the items before a level are what it needs.
    std::vector<u64> items_so_far(n_tables, 0), level_need(n_tables, 0);
    std::vector<u32> emit_level(n_tables, kNone);
    std::vector<EngineChunk> followers;
    chunks.clear();
    chunks.reserve(nb);
    auto item = [](u64 first, u64 need, u32 b, u64 count) {
        EngineChunk ch;
        ch.start = first;
        ch.need = need;
        ch.batch = b;
        ch.count = uint16_t(count);
        ch.nfollow = 0;
        ch.follow_first = 0;
        ch.pad = 0;
        return ch;
    };
    for (const u32 b : order) {
        const EngineBatch& eb = batches[b];
        const u32 t = eb.table;
        const u32 L = level_of[b];
        const u32 glen = group_len[L];
        if (glen == 0) continue;  // runs as a follower of its group's leader
        if (L != emit_level[t]) {  // a new level: wait for all earlier items
            emit_level[t] = L;
            level_need[t] = items_so_far[t];
        }
        if (glen > 1) {
            EngineChunk lead = item(0, level_need[t], b, eb.n);
            lead.nfollow = uint16_t(glen - 1);
            lead.follow_first = u32(followers.size());  // made absolute below
            chunks.push_back(lead);
            ++items_so_far[t];
            u32 f = L;
            for (u32 k = 1; k < glen; ++k) {
                f = lv_next[f];
                const u32 fb = lv_first[f];
                followers.push_back(item(0, 0, fb, batches[fb].n));
                ++items_so_far[t];
            }
            continue;
        }
        const u32 c = chunk_of[t];
        for (u64 s0 = 0; s0 < eb.n; s0 += c) chunks.push_back(item(s0, level_need[t], b, eb.n - s0 < c ? eb.n - s0 : c));
        items_so_far[t] += (eb.n + c - 1) / c;
    }
    const u64 n_queue = chunks.size();
    for (EngineChunk& ch : chunks)
        if (ch.nfollow) ch.follow_first += u32(n_queue);
    chunks.insert(chunks.end(), followers.begin(), followers.end());
    return n_queue;
}

TableInfo table_info(const cht_table* h) {
    TableInfo i;
    i.cells = h->cells;
    i.log2c = h->log2c;
    i.st = h->st;
    i.device = h->device;
    i.growable = h->growable;
    i.alpha = h->cfg.alpha;
    i.bound = h->i_bound;
    i.reuse = h->cfg.reuse_tombstones;
    i.full_keys = h->cfg.full_key_space;
    return i;
}

void table_set_bound(cht_table* h, u64 bound, bool exact) {
    h->i_bound = bound;
    h->i_exact = exact;
}

cht_status table_read_counts(cht_table* h, u64* I, u64* D, cudaStream_t s) {
    DevState ds;
    cht_status r = read_state(h, &ds, s);
    if (r != CHT_OK) return r;
    *I = ds.I;
    *D = ds.D;
    h->i_bound = ds.I;
    h->i_exact = true;
    return CHT_OK;
}

cht_status table_migrate_to(cht_table* h, u32 new_log2, u64 live, cudaStream_t s) {
    return do_migrate(h, new_log2, live, s);
}

cht_status runtime_alloc(void** p, u64 bytes, cudaStream_t s) { return lib_alloc(p, bytes, s); }
void runtime_free(void* p, u64 bytes, cudaStream_t s) { lib_free(p, bytes, s); }

void table_view(const cht_table* h, Cell** cells, u32* log2c, DevState** st, int* device, int* group_width,
                int* lane_cells, int* ctas_per_sm, int* full_keys) {
    *cells = h->cells;
    *log2c = h->log2c;
    *st = h->st;
    *device = h->device;
    const Width w = pick_width(h, kFind, 0);  // the width a find would use now
    *group_width = w.g;
    *lane_cells = w.v;
    *ctas_per_sm = h->cfg.ctas_per_sm;
    *full_keys = h->cfg.full_key_space;
}

void table_note_stream(cht_table* h, cudaStream_t s) { h->last = s; }

}  // namespace cht

extern "C" {

cht_status cht_create(uint64_t capacity, int growable, cht_stream_t stream, cht_handle* out) {
    if (!out) return CHT_ERR_INVALID_ARG;
    *out = nullptr;
    if (capacity > (1ull << kMaxLog2)) return CHT_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cht_table* h = new (std::nothrow) cht_table();
    if (!h) return CHT_ERR_OOM;
    h->device = current_device();
    prepare_pool(h->device);
    h->log2c = log2_ceil_cap(capacity < kMinCap ? kMinCap : capacity);
    h->growable = growable ? 1 : 0;
    h->cells_bytes = h->cap() * sizeof(Cell);
    cht_status r = lib_alloc(reinterpret_cast<void**>(&h->cells), h->cells_bytes, s);
    if (r != CHT_OK) {
        delete h;
        return r;
    }
    r = lib_alloc(reinterpret_cast<void**>(&h->st), sizeof(DevState), s);
    if (r != CHT_OK) {
        lib_free(h->cells, h->cells_bytes, s);
        delete h;
        return r;
    }
    if (cudaMemsetAsync(h->cells, 0, h->cap() * sizeof(Cell), s) != cudaSuccess ||
        cudaMemsetAsync(h->st, 0, sizeof(DevState), s) != cudaSuccess) {
        lib_free(h->cells, h->cells_bytes, s);
        lib_free(h->st, sizeof(DevState), s);
        delete h;
        return CHT_ERR_CUDA;
    }
    h->last = s;
    *out = h;
    return CHT_OK;
}

cht_status cht_destroy(cht_handle h) {
    if (!h) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    lib_free(h->cells, h->cells_bytes, h->last);
    lib_free(h->st, sizeof(DevState), h->last);
    cudaError_t e = cudaStreamSynchronize(h->last);
    delete h;
    return cuda_status(e);
}

cht_status cht_set_config(cht_handle h, const cht_config* cfg) {
    if (!h) return CHT_ERR_INVALID_ARG;
    cht_config c = cfg ? *cfg : default_config();
    if (!valid_config(c)) return CHT_ERR_INVALID_ARG;
    h->cfg = c;
    return CHT_OK;
}

cht_status cht_get_config(cht_handle h, cht_config* cfg) {
    if (!h || !cfg) return CHT_ERR_INVALID_ARG;
    *cfg = h->cfg;
    return CHT_OK;
}

// ---------------------------------------------------------------------------
// Pipelined staging of host arrays.  A call with host arrays larger than one
// piece is cut into pieces of kPipeChunk operations that cycle through
// kPipeSlots device slots: piece i+1 is copied in on a copy stream while piece
// i runs on the caller's stream and piece i-1's results are copied out on a
// second copy stream.  Pieces of one batch run one after another on the
// caller's stream, which is one linearization of the batch (phase semantics
// hold per piece and across them).  Device arrays are used in place.  The
// slots (about 420 MB per slot) are allocated on a device's first pipelined
// call and kept until the process exits; calls on one device take the slots
// one after another (a host lock around the enqueueing, events on the GPU).
// ---------------------------------------------------------------------------
constexpr u64 kPipeChunk = 1ull << 24;
constexpr int kPipeSlots = 3;

struct PipeSlot {
    u64* keys = nullptr;
    u64* vals = nullptr;
    u64* vout = nullptr;
    unsigned char* codes = nullptr;
    cudaEvent_t loaded = nullptr;    // its inputs are on the device
    cudaEvent_t consumed = nullptr;  // the kernel that read them is done
    cudaEvent_t drained = nullptr;   // its results are back in host memory
};

struct DevPipe {
    std::mutex mu;
    bool tried = false, ok = false;
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t start = nullptr;  // the work on the caller's stream before a call
    PipeSlot slot[kPipeSlots];
    int next = 0;
};
DevPipe g_pipe[64];

bool pipe_ready(int dev) {
    DevPipe& P = g_pipe[dev];
    if (P.tried) return P.ok;
    P.tried = true;
    const u64 per = kPipeChunk * (8 + 8 + 8 + 1);
    if (cudaStreamCreateWithFlags(&P.cin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&P.cout, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    unsigned char* mem = nullptr;
    if (cudaMalloc(&mem, per * kPipeSlots) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g_mem_in_use.fetch_add(per * kPipeSlots);
    for (int i = 0; i < kPipeSlots; ++i) {
        PipeSlot& q = P.slot[i];
        unsigned char* b = mem + i * per;
        q.keys = reinterpret_cast<u64*>(b);
        q.vals = q.keys + kPipeChunk;
        q.vout = q.vals + kPipeChunk;
        q.codes = reinterpret_cast<unsigned char*>(q.vout + kPipeChunk);
        if (cudaEventCreateWithFlags(&q.loaded, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&q.consumed, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&q.drained, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    P.ok = true;
    return true;
}

// One piece's work: the batch's operations [lo, lo + m) with device arrays.
typedef cht_status (*PieceFn)(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, u64* vout,
                              unsigned char* codes, u64 m, cudaStream_t s);

cht_status piece_modify(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, u64*, unsigned char* codes,
                        u64 m, cudaStream_t s) {
    return run_modify(h, mode, keys, vals, codes, m, s);
}

cht_status piece_launch(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, u64* vout,
                        unsigned char* codes, u64 m, cudaStream_t s) {
    return launch(h, mode, keys, vals, vout, codes, m, s);
}

// Runs the call through the pipeline if some array is in host memory and the
// batch is larger than one piece; *handled = false otherwise (the caller
// then stages the plain way).
cht_status pipelined(cht_table* h, cht::Mode mode, const u64* keys, const u64* vals, u64* vout,
                     unsigned char* codes, u64 n, cudaStream_t s, PieceFn fn, bool* handled) {
    *handled = false;
    const bool hk = is_host_pointer(keys), hv = vals && is_host_pointer(vals);
    const bool ho = vout && is_host_pointer(vout), hc = codes && is_host_pointer(codes);
    if (n <= kPipeChunk || !(hk || hv || ho || hc) || h->device < 0 || h->device >= 64) return CHT_OK;
    DevPipe& P = g_pipe[h->device];
    std::lock_guard<std::mutex> lk(P.mu);
    if (!pipe_ready(h->device)) return CHT_OK;
    *handled = true;
    // the copies in wait for the work already on s (it may write the inputs)
    if (cudaEventRecord(P.start, s) != cudaSuccess || cudaStreamWaitEvent(P.cin, P.start, 0) != cudaSuccess)
        return CHT_ERR_CUDA;
    bool used[kPipeSlots] = {};
    cht_status r = CHT_OK;
    for (u64 lo = 0; lo < n && r == CHT_OK; lo += kPipeChunk) {
        const u64 m = n - lo < kPipeChunk ? n - lo : kPipeChunk;
        PipeSlot& q = P.slot[P.next];
        used[P.next] = true;
        P.next = (P.next + 1) % kPipeSlots;
        // inputs: wait until the slot's previous kernel has read its inputs
        if (cudaStreamWaitEvent(P.cin, q.consumed, 0) != cudaSuccess) return CHT_ERR_CUDA;
        const u64* dk = keys + lo;
        const u64* dv = vals ? vals + lo : nullptr;
        if (hk) {
            if (cudaMemcpyAsync(q.keys, keys + lo, m * 8, cudaMemcpyHostToDevice, P.cin) != cudaSuccess)
                return CHT_ERR_CUDA;
            dk = q.keys;
        }
        if (hv) {
            if (cudaMemcpyAsync(q.vals, vals + lo, m * 8, cudaMemcpyHostToDevice, P.cin) != cudaSuccess)
                return CHT_ERR_CUDA;
            dv = q.vals;
        }
        if (cudaEventRecord(q.loaded, P.cin) != cudaSuccess) return CHT_ERR_CUDA;
        // the kernel: after its inputs, and after the slot's previous results left
        if (cudaStreamWaitEvent(s, q.loaded, 0) != cudaSuccess || cudaStreamWaitEvent(s, q.drained, 0) != cudaSuccess)
            return CHT_ERR_CUDA;
        u64* dvo = vout ? (ho ? q.vout : vout + lo) : nullptr;
        unsigned char* dc = codes ? (hc ? q.codes : codes + lo) : nullptr;
        r = fn(h, mode, dk, dv, dvo, dc, m, s);
        if (cudaEventRecord(q.consumed, s) != cudaSuccess) return CHT_ERR_CUDA;
        // results back once the kernel is done
        if (ho || hc) {
            if (cudaStreamWaitEvent(P.cout, q.consumed, 0) != cudaSuccess) return CHT_ERR_CUDA;
            if (ho && cudaMemcpyAsync(vout + lo, q.vout, m * 8, cudaMemcpyDeviceToHost, P.cout) != cudaSuccess)
                return CHT_ERR_CUDA;
            if (hc && cudaMemcpyAsync(codes + lo, q.codes, m, cudaMemcpyDeviceToHost, P.cout) != cudaSuccess)
                return CHT_ERR_CUDA;
            if (cudaEventRecord(q.drained, P.cout) != cudaSuccess) return CHT_ERR_CUDA;
        }
    }
    // the call completes on s when every result is back
    for (int i = 0; i < kPipeSlots; ++i)
        if (used[i] && cudaStreamWaitEvent(s, P.slot[i].drained, 0) != cudaSuccess) return CHT_ERR_CUDA;
    return r;
}

static cht_status modify_call(cht_handle h, cht::Mode mode, const uint64_t* keys, const uint64_t* vals,
                              uint64_t n, uint8_t* codes, cht_stream_t stream) {
    if (!h || (n > 0 && (!keys || !vals))) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    bool piped = false;
    cht_status r = pipelined(h, mode, reinterpret_cast<const u64*>(keys), reinterpret_cast<const u64*>(vals), nullptr, codes, n,
                                 s, piece_modify, &piped);
    if (piped) return r;
    Staging stg(s);
    const void *dk, *dv;
    void* dc;
    r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.in(vals, n * 8, &dv);
    if (r == CHT_OK) r = stg.out(codes, n, &dc);
    if (r != CHT_OK) return r;
    r = run_modify(h, mode, static_cast<const u64*>(dk), static_cast<const u64*>(dv),
                   static_cast<unsigned char*>(dc), n, s);
    cht_status f = stg.finish();
    return r != CHT_OK ? r : f;
}

cht_status cht_insert(cht_handle h, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                      uint8_t* inserted, cht_stream_t stream) {
    return modify_call(h, cht::kInsert, keys, vals, n, inserted, stream);
}

cht_status cht_insert_or_update(cht_handle h, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                                cht_update_op op, uint8_t* inserted, cht_stream_t stream) {
    if (op != CHT_ADD && op != CHT_OVERWRITE) return CHT_ERR_INVALID_ARG;
    return modify_call(h, op == CHT_ADD ? cht::kIouAdd : cht::kIouOverwrite, keys, vals, n, inserted,
                       stream);
}

cht_status cht_update(cht_handle h, const uint64_t* keys, const uint64_t* vals, uint64_t n, cht_update_op op,
                      uint8_t* updated, cht_stream_t stream) {
    if (op != CHT_ADD && op != CHT_OVERWRITE) return CHT_ERR_INVALID_ARG;
    if (!h || (n > 0 && (!keys || !vals))) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    const cht::Mode um = op == CHT_ADD ? cht::kUpdAdd : cht::kUpdOverwrite;
    bool piped = false;
    cht_status r = pipelined(h, um, reinterpret_cast<const u64*>(keys), reinterpret_cast<const u64*>(vals), nullptr, updated,
                                 n, s, piece_launch, &piped);
    if (piped) return r;
    Staging stg(s);
    const void *dk, *dv;
    void* dc;
    r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.in(vals, n * 8, &dv);
    if (r == CHT_OK) r = stg.out(updated, n, &dc);
    if (r != CHT_OK) return r;
    // no cell is filled: neither growth nor the bound on I is involved
    r = launch(h, op == CHT_ADD ? cht::kUpdAdd : cht::kUpdOverwrite, static_cast<const u64*>(dk),
               static_cast<const u64*>(dv), nullptr, static_cast<unsigned char*>(dc), n, s);
    cht_status f = stg.finish();
    return r != CHT_OK ? r : f;
}

cht_status cht_build(cht_handle h, const uint64_t* keys, const uint64_t* vals, uint64_t n, cht_stream_t stream) {
    if (!h || (n > 0 && (!keys || !vals)) || n >= (1ull << 32)) return CHT_ERR_INVALID_ARG;
    if (h->i_bound != 0) return CHT_ERR_INVALID_ARG;  // not empty since creation or the last clear
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    Staging stg(s);
    const void *dk, *dv;
    cht_status r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.in(vals, n * 8, &dv);
    if (r != CHT_OK) return r;
    // a growable table takes, empty, the capacity that holds n elements at
    // alpha (n bounds the distinct keys); nothing to migrate
    if (h->growable) {
        u32 nl = h->log2c;
        while (double(n) > h->cfg.alpha * double(1ull << nl)) ++nl;
        if (nl != h->log2c) {
            Cell* cells = nullptr;
            const u64 bytes = (1ull << nl) * sizeof(Cell);
            r = lib_alloc(reinterpret_cast<void**>(&cells), bytes, s);
            if (r != CHT_OK) return r;
            if (cudaMemsetAsync(cells, 0, bytes, s) != cudaSuccess) {
                lib_free(cells, bytes, s);
                return CHT_ERR_CUDA;
            }
            lib_free(h->cells, h->cells_bytes, s);
            h->cells = cells;
            h->cells_bytes = bytes;
            h->log2c = nl;
        }
    }
    const u64 sbytes = cht::build_scratch_bytes(n);
    void* scratch = nullptr;
    r = lib_alloc(&scratch, sbytes, s);
    if (r != CHT_OK) return r;
    const Cell* sorted = nullptr;
    cht::BuildExtra* ex = nullptr;
    cudaError_t e = cht::launch_build_sort(static_cast<const u64*>(dk), static_cast<const u64*>(dv), n, h->log2c,
                                           h->cfg.full_key_space, scratch, &sorted, &ex, s);
    if (e == cudaSuccess) e = cht::launch_build_count(sorted, n, h->log2c, scratch, ex, s);
    if (e == cudaSuccess && n >= h->cap()) {
        // only a batch of >= c elements can leave no empty cell: read the
        // survivor count before touching the table
        u64 S = 0;
        e = cudaMemcpyAsync(&S, &ex->S, sizeof(u64), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && S >= h->cap()) {
            lib_free(scratch, sbytes, s);
            stg.finish();
            return CHT_ERR_TABLE_FULL;
        }
    }
    if (e == cudaSuccess)
        e = cht::launch_build_place(sorted, n, h->cells, h->log2c, scratch, ex, h->st, static_cast<const u64*>(dv), s);
    lib_free(scratch, sbytes, s);
    if (e != cudaSuccess) return cuda_status(e);
    h->i_bound = n;
    h->i_exact = false;
    return stg.finish();
}

cht_status cht_merge(cht_handle h, const uint64_t* keys, const uint64_t* vals, uint64_t n, cht_stream_t stream) {
    if (!h || (n > 0 && (!keys || !vals))) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    // the live count sizes the table side of the concatenation (one read)
    DevState ds;
    cht_status r = read_state(h, &ds, s);
    if (r != CHT_OK) return r;
    const u64 live = ds.I - ds.D, tot = live + n;
    if (tot >= (1ull << 32)) return CHT_ERR_INVALID_ARG;
    Staging stg(s);
    const void *dk, *dv;
    r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.in(vals, n * 8, &dv);
    if (r != CHT_OK) return r;
    // a growable table takes the capacity that holds live + n at alpha
    u32 nl = h->log2c;
    if (h->growable)
        while (double(tot) > h->cfg.alpha * double(1ull << nl) && nl < kMaxLog2) ++nl;
    const u64 ncap = 1ull << nl, cbytes = ncap * sizeof(Cell);
    // scratch: the concatenation (keys, values), the compaction's counts, the build's buffers
    const u64 cat_bytes = (tot * 8 + 255) & ~255ull;
    const u64 cmp_bytes = cht::compact_scratch_bytes(h->log2c);
    const u64 bld_bytes = cht::build_scratch_bytes(tot);
    const u64 sbytes = 2 * cat_bytes + cmp_bytes + bld_bytes;
    unsigned char* scratch = nullptr;
    Cell* cells = nullptr;
    r = lib_alloc(reinterpret_cast<void**>(&scratch), sbytes, s);
    if (r != CHT_OK) return r;
    r = lib_alloc(reinterpret_cast<void**>(&cells), cbytes, s);
    if (r != CHT_OK) {
        lib_free(scratch, sbytes, s);
        return r;
    }
    u64* ck = reinterpret_cast<u64*>(scratch);
    u64* cv = reinterpret_cast<u64*>(scratch + cat_bytes);
    void* cmp = scratch + 2 * cat_bytes;
    void* bld = scratch + 2 * cat_bytes + cmp_bytes;
    // the table's live elements in cell index order, then the batch
    cudaError_t e = cht::launch_compact_live(h->cells, h->log2c, ck, cv, cmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck + live, dk, n * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cv + live, dv, n * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cells, 0, cbytes, s);
    const Cell* sorted = nullptr;
    cht::BuildExtra* ex = nullptr;
    if (e == cudaSuccess)
        e = cht::launch_build_sort(ck, cv, tot, nl, h->cfg.full_key_space, bld, &sorted, &ex, s);
    if (e == cudaSuccess) e = cht::launch_build_count(sorted, tot, nl, bld, ex, s);
    if (e == cudaSuccess && tot >= ncap) {
        // only tot >= c' can leave no empty cell: check before touching the table
        u64 S = 0;
        e = cudaMemcpyAsync(&S, &ex->S, sizeof(u64), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && S >= ncap) {
            lib_free(cells, cbytes, s);
            lib_free(scratch, sbytes, s);
            stg.finish();
            return CHT_ERR_TABLE_FULL;
        }
    }
    // the finish kernel sets I = survivors, D = 0 and the special slots the batch names
    if (e == cudaSuccess) e = cht::launch_build_place(sorted, tot, cells, nl, bld, ex, h->st, cv, s);
    lib_free(scratch, sbytes, s);
    if (e != cudaSuccess) {
        lib_free(cells, cbytes, s);
        return cuda_status(e);
    }
    lib_free(h->cells, h->cells_bytes, s);
    h->cells = cells;
    h->cells_bytes = cbytes;
    h->log2c = nl;
    h->i_bound = tot;
    h->i_exact = false;
    return stg.finish();
}

cht_status cht_find(cht_handle h, const uint64_t* keys, uint64_t n, uint64_t* vals_out, uint8_t* found,
                    cht_stream_t stream) {
    if (!h || (n > 0 && (!keys || !vals_out))) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    bool piped = false;
    cht_status r = pipelined(h, cht::kFind, reinterpret_cast<const u64*>(keys), nullptr,
                                 reinterpret_cast<u64*>(vals_out), found, n, s, piece_launch, &piped);
    if (piped) return r;
    Staging stg(s);
    const void* dk;
    void *dv, *dc;
    r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.out(vals_out, n * 8, &dv);
    if (r == CHT_OK) r = stg.out(found, n, &dc);
    if (r != CHT_OK) return r;
    r = launch(h, cht::kFind, static_cast<const u64*>(dk), nullptr, static_cast<u64*>(dv),
               static_cast<unsigned char*>(dc), n, s);
    cht_status f = stg.finish();
    return r != CHT_OK ? r : f;
}

cht_status cht_erase(cht_handle h, const uint64_t* keys, uint64_t n, uint8_t* erased, cht_stream_t stream) {
    if (!h || (n > 0 && !keys)) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    bool piped = false;
    cht_status r = pipelined(h, cht::kErase, reinterpret_cast<const u64*>(keys), nullptr, nullptr, erased, n, s,
                                 piece_launch, &piped);
    if (piped) return r;
    Staging stg(s);
    const void* dk;
    void* dc;
    r = stg.in(keys, n * 8, &dk);
    if (r == CHT_OK) r = stg.out(erased, n, &dc);
    if (r != CHT_OK) return r;
    r = launch(h, cht::kErase, static_cast<const u64*>(dk), nullptr, nullptr, static_cast<unsigned char*>(dc),
               n, s);
    cht_status f = stg.finish();
    return r != CHT_OK ? r : f;
}

cht_status cht_migrate(cht_handle h, uint64_t new_capacity, cht_stream_t stream) {
    if (!h) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    u32 nl;
    u64 live = ~0ull;
    if (new_capacity == 0) {
        DevState ds;
        cht_status r = read_state(h, &ds, s);
        if (r != CHT_OK) return r;
        live = ds.I - ds.D;
        const u64 half = u64(std::floor(h->cfg.alpha * double(h->cap()) / 2.0));
        nl = h->log2c + (live > half ? 1u : 0u);
    } else {
        if (new_capacity > (1ull << kMaxLog2)) return CHT_ERR_INVALID_ARG;
        nl = log2_ceil_cap(new_capacity);
    }
    if (nl > kMaxLog2) return CHT_ERR_INVALID_ARG;
    if (nl < h->log2c) {  // shrinking: the live elements must leave an empty cell
        if (live == ~0ull) {
            DevState ds;
            cht_status r = read_state(h, &ds, s);
            if (r != CHT_OK) return r;
            live = ds.I - ds.D;
        }
        if (live >= (1ull << nl)) return CHT_ERR_INVALID_ARG;
    }
    return do_migrate(h, nl, live, s);
}

cht_status cht_size(cht_handle h, uint64_t* live, uint64_t* nonempty, uint64_t* capacity,
                    cht_stream_t stream) {
    if (!h) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevState ds;
    cht_status r = read_state(h, &ds, s);
    if (r != CHT_OK) return r;
    h->i_bound = ds.I;
    h->i_exact = true;
    if (live) *live = ds.I - ds.D + ds.sp_present[0] + ds.sp_present[1];
    if (nonempty) *nonempty = ds.I;
    if (capacity) *capacity = h->cap();
    if (ds.status & CHT_STATUS_FULL) return CHT_ERR_TABLE_FULL;
    if (ds.status & CHT_STATUS_RESERVED) return CHT_ERR_RESERVED_KEY;
    return CHT_OK;
}

cht_status cht_get_status(cht_handle h, uint32_t* bits, cht_stream_t stream) {
    if (!h || !bits) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevState ds;
    cht_status r = read_state(h, &ds, s);
    if (r != CHT_OK) return r;
    *bits = ds.status;
    if (cudaMemsetAsync(&h->st->status, 0, sizeof(u32), s) != cudaSuccess) return CHT_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

cht_status cht_export(cht_handle h, uint64_t* keys_out, uint64_t* vals_out, uint64_t max_n, uint64_t* n_out,
                      cht_stream_t stream) {
    if (!h || !n_out || (max_n > 0 && !keys_out)) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    Staging stg(s);
    void *dk = nullptr, *dv = nullptr;
    cht_status r = stg.out(keys_out, max_n * 8, &dk);
    if (r == CHT_OK && vals_out) r = stg.out(vals_out, max_n * 8, &dv);
    if (r != CHT_OK) return r;
    if (cudaMemsetAsync(&h->st->export_pos, 0, sizeof(u64), s) != cudaSuccess) return CHT_ERR_CUDA;
    r = cuda_status(cht::launch_export(h->cells, h->log2c, static_cast<u64*>(dk), static_cast<u64*>(dv), max_n,
                                       h->st, s));
    cht_status f = stg.finish();
    if (r != CHT_OK) return r;
    if (f != CHT_OK) return f;
    DevState ds;
    r = read_state(h, &ds, s);
    if (r != CHT_OK) return r;
    *n_out = ds.export_pos;
    return ds.export_pos > max_n ? CHT_ERR_INVALID_ARG : CHT_OK;
}

cht_status cht_copy_cells(cht_handle h, uint64_t* cells_out, uint64_t max_cells, uint64_t* n_cells,
                          cht_stream_t stream) {
    if (!h || !cells_out) return CHT_ERR_INVALID_ARG;
    if (n_cells) *n_cells = h->cap();
    if (max_cells < h->cap()) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return cuda_status(cudaMemcpyAsync(cells_out, h->cells, h->cap() * sizeof(Cell), cudaMemcpyDefault, s));
}

cht_status cht_clear(cht_handle h, cht_stream_t stream) {
    if (!h) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    if (cudaMemsetAsync(h->cells, 0, h->cap() * sizeof(Cell), s) != cudaSuccess) return CHT_ERR_CUDA;
    if (cudaMemsetAsync(h->st, 0, sizeof(DevState), s) != cudaSuccess) return CHT_ERR_CUDA;
    h->i_bound = 0;
    h->i_exact = true;
    return CHT_OK;
}

cht_status cht_tune(cht_handle h, int op, const uint64_t* keys, const uint64_t* vals, uint64_t n, int trials,
                    cht_tune_result* results, uint32_t max_results, uint32_t* n_results, cht_stream_t stream) {
    if (!h || !keys || n == 0 || !results || !n_results || op < CHT_OP_FIND || op > CHT_OP_UPDATE_OVERWRITE)
        return CHT_ERR_INVALID_ARG;
    const cht::Mode mode = cht::Mode(op);
    if (cht::mode_has_vals(mode) && !vals) return CHT_ERR_INVALID_ARG;
    if (h->cfg.reuse_tombstones || h->cfg.full_key_space) return CHT_ERR_INVALID_ARG;
    if (is_host_pointer(keys) || (vals && is_host_pointer(vals))) return CHT_ERR_INVALID_ARG;
    if (trials < 3) trials = 3;
    *n_results = 0;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last = s;
    const bool modify = mode != cht::kFind;
    const u64 tbytes = h->cap() * sizeof(Cell);
    // scratch: the outputs, and a copy of the table for the restores
    const u64 obytes = ((n * 8 + 255) & ~255ull) + ((n + 255) & ~255ull);
    const u64 sbytes = obytes + (modify ? tbytes + 256 : 0);
    unsigned char* scratch = nullptr;
    cht_status r = lib_alloc(reinterpret_cast<void**>(&scratch), sbytes, s);
    if (r != CHT_OK) return r;
    u64* vout = reinterpret_cast<u64*>(scratch);
    unsigned char* codes = scratch + ((n * 8 + 255) & ~255ull);
    Cell* save_cells = modify ? reinterpret_cast<Cell*>(scratch + obytes) : nullptr;
    DevState* save_st = modify ? reinterpret_cast<DevState*>(scratch + obytes + tbytes) : nullptr;
    auto restore = [&](bool save) -> cudaError_t {
        if (!modify) return cudaSuccess;
        cudaError_t e = cudaMemcpyAsync(save ? static_cast<void*>(save_cells) : static_cast<void*>(h->cells),
                                        save ? static_cast<void*>(h->cells) : static_cast<void*>(save_cells), tbytes,
                                        cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(save ? static_cast<void*>(save_st) : static_cast<void*>(h->st),
                                save ? static_cast<void*>(h->st) : static_cast<void*>(save_st), sizeof(DevState),
                                cudaMemcpyDeviceToDevice, s);
        return e;
    };
    struct Cand {
        int g, v;
    };
    static const Cand cands[] = {{-1, 2}, {-1, 4}, {1, 2},  {1, 4},  {2, 1},  {2, 2}, {2, 4}, {4, 1},
                                 {4, 2},  {4, 4},  {8, 1},  {8, 2},  {8, 4},  {16, 1}, {16, 2}, {32, 1}};
    static const int ctas[] = {0, 4};
    cht::OpArgs a;
    a.cells = h->cells;
    a.log2c = h->log2c;
    a.reuse = 0;
    a.full_keys = 0;
    a.keys = reinterpret_cast<const u64*>(keys);
    a.vals = cht::mode_has_vals(mode) ? reinterpret_cast<const u64*>(vals) : nullptr;
    a.vals_out = mode == cht::kFind ? vout : nullptr;
    a.codes = codes;
    a.n = n;
    a.st = h->st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = restore(true);
    std::vector<cht_tune_result> all;
    // finds leave the table as it is: a trial times kFindReps launches back to
    // back (as calls are issued) and keeps their mean, which also averages out
    // the launch-to-launch noise of short calls
    constexpr int kFindReps = 8;
    const int reps = mode == cht::kFind ? kFindReps : 1;
    for (const Cand& c : cands) {
        for (int ct : ctas) {
            std::vector<double> t;
            for (int k = 0; k < trials && e == cudaSuccess; ++k) {
                if (k > 0 || !all.empty()) e = restore(false);
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cht::launch_op(mode, a, c.g, c.v, ct, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                t.push_back(ms / reps);
            }
            if (e != cudaSuccess) break;
            std::sort(t.begin(), t.end());
            cht_tune_result res;
            res.group_width = c.g;
            res.lane_cells = c.v;
            res.ctas_per_sm = ct;
            res.ms = t[t.size() / 2];
            all.push_back(res);
        }
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = restore(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lib_free(scratch, sbytes, s);
    if (e != cudaSuccess) return cuda_status(e);
    std::stable_sort(all.begin(), all.end(),
                     [](const cht_tune_result& x, const cht_tune_result& y) { return x.ms < y.ms; });
    const u32 m = u32(std::min<size_t>(all.size(), max_results));
    for (u32 i = 0; i < m; ++i) results[i] = all[i];
    *n_results = m;
    return CHT_OK;
}

cht_status cht_set_memory_limit(uint64_t bytes) {
    g_mem_limit.store(bytes);
    return CHT_OK;
}

uint64_t cht_memory_in_use(void) { return g_mem_in_use.load(); }

uint64_t cht_launch_count(void) { return g_launches.load(); }

const char* cht_status_string(cht_status s) {
    switch (s) {
        case CHT_OK: return "ok";
        case CHT_ERR_INVALID_ARG: return "invalid argument";
        case CHT_ERR_OOM: return "out of device memory";
        case CHT_ERR_CUDA: return "CUDA error";
        case CHT_ERR_TABLE_FULL: return "table full";
        case CHT_ERR_RESERVED_KEY: return "reserved key (0 or ~0)";
        case CHT_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int cht_version(void) { return 100; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched engine plans (declared in cht.h).  The host orders the work items
// round by round -- the r-th batch of every table forms round r -- and gives
// every item the number of its table's items in earlier rounds, which the
// engine kernel waits for.
// ---------------------------------------------------------------------------
struct cht_plan {
    int device = 0;
    std::vector<cht_table*> tables;
    std::vector<u64> new_cells;  // per table: upper bound of cells its batches can fill
    cht::EngineTable* d_tables = nullptr;
    cht::EngineBatch* d_batches = nullptr;
    cht::EngineChunk* d_chunks = nullptr;
    unsigned long long* d_counters = nullptr;  // [0] queue cursor, [1 + t] table t's done items
    u32* d_status = nullptr;
    u64 n_batches = 0, n_chunks = 0;
    u64 bytes_tables = 0, bytes_batches = 0, bytes_chunks = 0, bytes_counters = 0;
    std::vector<cht::EngineBatch> batches;  // host copy: work items are rebuilt when chunk_ops changes
    cht_plan_config cfg{0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

cht_status upload(void** dst, u64* bytes_out, const void* src, u64 bytes) {
    *bytes_out = bytes;
    cht_status r = lib_alloc(dst, bytes, nullptr);
    if (r != CHT_OK) return r;
    if (bytes && cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, nullptr) != cudaSuccess) return CHT_ERR_CUDA;
    return CHT_OK;
}

void plan_free(cht_plan* p) {
    lib_free(p->d_tables, p->bytes_tables, nullptr);
    lib_free(p->d_batches, p->bytes_batches, nullptr);
    lib_free(p->d_chunks, p->bytes_chunks, nullptr);
    lib_free(p->d_counters, p->bytes_counters, nullptr);
    cudaStreamSynchronize(nullptr);
}

cht::EngineArgs plan_args(const cht_plan* p) {
    cht::EngineArgs e;
    e.tables = p->d_tables;
    e.batches = p->d_batches;
    e.chunks = p->d_chunks;
    e.n_chunks = p->n_chunks;
    e.next = p->d_counters;
    e.done = p->d_counters + 1;
    e.status = p->d_status;
    e.spin_limit = (p->cfg.spin_limit_us > 0 ? (long long)p->cfg.spin_limit_us : 1000000ll) * 2000;  // ~2 GHz
    e.inject_stall = p->cfg.fault_inject & 1;
    e.max_backoff_ns = p->cfg.poll_ns > 0 ? unsigned(p->cfg.poll_ns) : 8192u;
    e.any_reuse = 0;
    e.any_full = 0;
    for (const cht_table* h : p->tables) {
        e.any_reuse |= h->cfg.reuse_tombstones;
        e.any_full |= h->cfg.full_key_space;
    }
    e.snap_tables = nullptr;
    e.n_snap = 0;
    e.snap_out = nullptr;
    e.warps_done = nullptr;
    return e;
}

cht_status plan_run(cht_plan* p, cudaStream_t s) {
    if (cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, s) != cudaSuccess) return CHT_ERR_CUDA;
    const int g = p->cfg.group_width > 0 ? p->cfg.group_width : 1;
    const int v = g == 1 ? 2 : (p->cfg.lane_cells > 0 ? p->cfg.lane_cells : 1);
    return cuda_status(cht::launch_engine(plan_args(p), g, v, p->cfg.ctas_per_sm, p->cfg.direct_io == 0, s));
}

}  // namespace

extern "C" {

// True if no batch's keys / vals range overlaps any batch's vals_out /
// codes range (byte intervals; sort the outputs, binary-search each input).
static bool inputs_disjoint_from_outputs(const std::vector<cht::EngineBatch>& batches) {
    std::vector<std::pair<uintptr_t, uintptr_t>> outs;
    for (const cht::EngineBatch& b : batches) {
        if (b.vals_out) outs.emplace_back(uintptr_t(b.vals_out), uintptr_t(b.vals_out) + b.n * 8);
        if (b.codes) outs.emplace_back(uintptr_t(b.codes), uintptr_t(b.codes) + b.n);
    }
    if (outs.empty()) return true;
    std::sort(outs.begin(), outs.end());
    // prefix maximum of the ends, so one search answers "any output overlaps"
    std::vector<uintptr_t> max_end(outs.size());
    uintptr_t m = 0;
    for (size_t i = 0; i < outs.size(); ++i) max_end[i] = m = std::max(m, outs[i].second);
    auto overlaps = [&](uintptr_t lo, uintptr_t hi) {
        // outputs starting before hi; the one with the largest end decides
        const size_t k = size_t(std::lower_bound(outs.begin(), outs.end(), std::make_pair(hi, uintptr_t(0))) -
                                outs.begin());
        return k > 0 && max_end[k - 1] > lo;
    };
    for (const cht::EngineBatch& b : batches) {
        if (overlaps(uintptr_t(b.keys), uintptr_t(b.keys) + b.n * 8)) return false;
        if (b.vals && overlaps(uintptr_t(b.vals), uintptr_t(b.vals) + b.n * 8)) return false;
    }
    return true;
}

cht_status cht_plan_create(const cht_batch_op* ops, uint64_t n_ops, cht_plan_handle* out) {
    if (!out || (n_ops > 0 && !ops)) return CHT_ERR_INVALID_ARG;
    *out = nullptr;
    cht_plan* p = new (std::nothrow) cht_plan();
    if (!p) return CHT_ERR_OOM;
    std::unordered_map<cht_table*, u32> index;
    std::vector<cht::EngineBatch> batches;
    batches.reserve(n_ops);
    for (u64 i = 0; i < n_ops; ++i) {
        const cht_batch_op& o = ops[i];
        const bool has_vals = cht::mode_has_vals(o.op);
        bool ok = o.table && o.op >= CHT_OP_FIND && o.op <= CHT_OP_UPDATE_OVERWRITE;
        if (ok && o.n > 0) {
            ok = o.keys && !is_host_pointer(o.keys) && (!has_vals || (o.vals && !is_host_pointer(o.vals))) &&
                 (o.op != CHT_OP_FIND || (o.vals_out && !is_host_pointer(o.vals_out))) &&
                 (!o.codes || !is_host_pointer(o.codes));
        }
        if (ok && !p->tables.empty() && o.table->device != p->device) ok = false;
        if (!ok) {
            delete p;
            return CHT_ERR_INVALID_ARG;
        }
        if (o.n == 0) continue;
        auto it = index.find(o.table);
        u32 t;
        if (it == index.end()) {
            t = u32(p->tables.size());
            index.emplace(o.table, t);
            if (p->tables.empty()) p->device = o.table->device;
            p->tables.push_back(o.table);
            p->new_cells.push_back(0);
        } else {
            t = it->second;
        }
        cht::EngineBatch b;
        b.keys = reinterpret_cast<const u64*>(o.keys);
        b.vals = has_vals ? reinterpret_cast<const u64*>(o.vals) : nullptr;
        b.vals_out = o.op == CHT_OP_FIND ? reinterpret_cast<u64*>(o.vals_out) : nullptr;
        b.codes = o.codes;
        b.n = o.n;
        b.table = t;
        b.mode = u32(o.op);
        batches.push_back(b);
        if (cht::mode_fills(o.op)) p->new_cells[t] += o.n;
    }
    // The engine may read a work item's inputs before the items it depends
    // on have run, so no input array may overlap any output array.
    if (!inputs_disjoint_from_outputs(batches)) {
        delete p;
        return CHT_ERR_INVALID_ARG;
    }
    // work items, round by round; need = the table's items in earlier levels
    std::vector<cht::EngineChunk> chunks;
    const u64 n_queue = cht::plan_order(batches, p->tables.size(), 0, chunks);
    std::vector<cht::EngineTable> tabs(p->tables.size());
    for (size_t t = 0; t < p->tables.size(); ++t) {
        tabs[t].cells = p->tables[t]->cells;
        tabs[t].log2c = p->tables[t]->log2c;
        tabs[t].flags = (p->tables[t]->cfg.reuse_tombstones ? cht::kTabReuse : 0u) |
                        (p->tables[t]->cfg.full_key_space ? cht::kTabFullKeys : 0u);
        tabs[t].st = p->tables[t]->st;
    }
    DeviceGuard g(p->tables.empty() ? current_device() : p->device);
    p->n_batches = batches.size();
    p->n_chunks = n_queue;
    cht_status r = upload(reinterpret_cast<void**>(&p->d_tables), &p->bytes_tables, tabs.data(),
                          tabs.size() * sizeof(cht::EngineTable));
    if (r == CHT_OK)
        r = upload(reinterpret_cast<void**>(&p->d_batches), &p->bytes_batches, batches.data(),
                   batches.size() * sizeof(cht::EngineBatch));
    if (r == CHT_OK)
        r = upload(reinterpret_cast<void**>(&p->d_chunks), &p->bytes_chunks, chunks.data(),
                   chunks.size() * sizeof(cht::EngineChunk));
    if (r == CHT_OK) {
        // counters and the status word share one allocation
        p->bytes_counters = (1 + p->tables.size()) * sizeof(unsigned long long) + sizeof(unsigned long long);
        r = lib_alloc(reinterpret_cast<void**>(&p->d_counters), p->bytes_counters, nullptr);
        if (r == CHT_OK) p->d_status = reinterpret_cast<u32*>(p->d_counters + 1 + p->tables.size());
    }
    if (r == CHT_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) r = CHT_ERR_CUDA;
    if (r != CHT_OK) {
        plan_free(p);
        delete p;
        return r;
    }
    p->batches = std::move(batches);
    *out = p;
    return CHT_OK;
}

cht_status cht_plan_set_config(cht_plan_handle p, const cht_plan_config* cfg) {
    if (!p) return CHT_ERR_INVALID_ARG;
    cht_plan_config c = cfg ? *cfg : cht_plan_config{0, 0, 0, 0, 0, 0, 0, 0};
    const int g = c.group_width;
    if (!(g == 0 || g == 1 || g == 4 || g == 8 || g == 16 || g == 32)) return CHT_ERR_INVALID_ARG;
    if (c.lane_cells < 0 || c.lane_cells > 2 || (g == 32 && c.lane_cells == 2)) return CHT_ERR_INVALID_ARG;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 64 || c.spin_limit_us < 0 || c.fault_inject < 0 || c.fault_inject > 1 ||
        c.direct_io < 0 || c.direct_io > 1)
        return CHT_ERR_INVALID_ARG;
    if (c.poll_ns < 0 || c.poll_ns > 1000000) return CHT_ERR_INVALID_ARG;
    if (!(c.chunk_ops == 0 || c.chunk_ops == 32 || c.chunk_ops == 64 || c.chunk_ops == 128 || c.chunk_ops == 256))
        return CHT_ERR_INVALID_ARG;
    if (c.chunk_ops != p->cfg.chunk_ops && p->n_chunks > 0) {  // rebuild the work items
        std::vector<cht::EngineChunk> chunks;
        const u64 n_queue = cht::plan_order(p->batches, p->tables.size(), c.chunk_ops, chunks);
        DeviceGuard g(p->device);
        cht::EngineChunk* d = nullptr;
        u64 bytes = 0;
        cht_status r = upload(reinterpret_cast<void**>(&d), &bytes, chunks.data(), chunks.size() * sizeof(cht::EngineChunk));
        if (r == CHT_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) r = CHT_ERR_CUDA;
        if (r != CHT_OK) {
            lib_free(d, bytes, nullptr);
            return r;
        }
        lib_free(p->d_chunks, p->bytes_chunks, nullptr);
        p->d_chunks = d;
        p->bytes_chunks = bytes;
        p->n_chunks = n_queue;
    }
    p->cfg = c;
    return CHT_OK;
}

cht_status cht_plan_get_config(cht_plan_handle p, cht_plan_config* cfg) {
    if (!p || !cfg) return CHT_ERR_INVALID_ARG;
    *cfg = p->cfg;
    return CHT_OK;
}

cht_status cht_plan_launch(cht_plan_handle p, cht_stream_t stream) {
    if (!p) return CHT_ERR_INVALID_ARG;
    if (p->n_chunks == 0) return CHT_OK;
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cht_status r = plan_run(p, s);
    if (r != CHT_OK) return r;
    for (size_t t = 0; t < p->tables.size(); ++t) {
        cht_table* h = p->tables[t];
        h->i_bound += p->new_cells[t];
        if (h->i_bound > h->cap()) h->i_bound = h->cap();
        h->i_exact = false;
        h->last = s;
    }
    return CHT_OK;
}

cht_status cht_plan_status(cht_plan_handle p, uint32_t* bits, cht_stream_t stream) {
    if (!p || !bits) return CHT_ERR_INVALID_ARG;
    *bits = 0;
    if (p->n_chunks == 0) return CHT_OK;
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    u32 st = 0;
    if (cudaMemcpyAsync(&st, p->d_status, sizeof(u32), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CHT_ERR_CUDA;
    cht_status r = cuda_status(cudaStreamSynchronize(s));
    *bits = st & CHT_PLAN_TIMEOUT;
    return r;
}

cht_status cht_plan_autotune(cht_plan_handle p, cht_stream_t stream, double* best_ms) {
    if (!p) return CHT_ERR_INVALID_ARG;
    if (p->n_chunks == 0) return CHT_OK;
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // one copy of every table (cells + device state) to restore between trials
    u64 total = 0;
    for (cht_table* h : p->tables) total += h->cap() * sizeof(Cell) + sizeof(DevState);
    unsigned char* backup = nullptr;
    cht_status r = lib_alloc(reinterpret_cast<void**>(&backup), total, s);
    if (r != CHT_OK) return r;
    auto copy_tables = [&](bool save) -> cht_status {
        u64 off = 0;
        for (cht_table* h : p->tables) {
            const u64 nb = h->cap() * sizeof(Cell);
            void* a = backup + off;
            if (cudaMemcpyAsync(save ? a : h->cells, save ? static_cast<void*>(h->cells) : a, nb,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return CHT_ERR_CUDA;
            off += nb;
            void* b = backup + off;
            if (cudaMemcpyAsync(save ? b : h->st, save ? static_cast<void*>(h->st) : b, sizeof(DevState),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return CHT_ERR_CUDA;
            off += sizeof(DevState);
        }
        return CHT_OK;
    };
    const cht_plan_config keep = p->cfg;
    struct Cand {
        int g, v, ctas, direct;
    };
    const Cand cands[] = {{1, 2, 0, 0}, {4, 2, 0, 0}, {8, 2, 0, 0},  {4, 1, 0, 0},  {8, 1, 0, 0},
                          {16, 1, 0, 0}, {32, 1, 0, 0}, {1, 2, 2, 0}, {1, 2, 0, 1}, {4, 2, 0, 1}};
    double best = 1e30;
    cht_plan_config best_cfg = keep;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = CHT_ERR_CUDA;
    if (r == CHT_OK) r = copy_tables(true);
    constexpr int kTrials = 3;  // the median of three runs per candidate
    for (const Cand& c : cands) {
        if (r != CHT_OK) break;
        p->cfg.group_width = c.g;
        p->cfg.lane_cells = c.v;
        p->cfg.ctas_per_sm = c.ctas;
        p->cfg.direct_io = c.direct;
        float t[kTrials] = {};
        bool ok = true;
        for (int k = 0; k < kTrials && r == CHT_OK; ++k) {
            if (cudaEventRecord(e0, s) != cudaSuccess) r = CHT_ERR_CUDA;
            if (r == CHT_OK) r = plan_run(p, s);
            if (r == CHT_OK && cudaEventRecord(e1, s) != cudaSuccess) r = CHT_ERR_CUDA;
            if (r == CHT_OK && cudaEventSynchronize(e1) != cudaSuccess) r = CHT_ERR_CUDA;
            if (r == CHT_OK && cudaEventElapsedTime(&t[k], e0, e1) != cudaSuccess) r = CHT_ERR_CUDA;
            u32 st = 0;
            if (r == CHT_OK && cudaMemcpy(&st, p->d_status, sizeof(u32), cudaMemcpyDeviceToHost) != cudaSuccess)
                r = CHT_ERR_CUDA;
            if (st != 0) ok = false;
            if (r == CHT_OK) r = copy_tables(false);
        }
        if (r != CHT_OK) break;
        std::sort(t, t + kTrials);
        const double ms = t[kTrials / 2];
        if (ok && ms < best) {
            best = ms;
            best_cfg = p->cfg;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lib_free(backup, total, s);
    cudaStreamSynchronize(s);
    p->cfg = best < 1e30 ? best_cfg : keep;
    p->cfg.spin_limit_us = keep.spin_limit_us;
    p->cfg.fault_inject = keep.fault_inject;
    if (best_ms) *best_ms = best < 1e30 ? best : 0.0;
    return r;
}

cht_status cht_plan_destroy(cht_plan_handle p) {
    if (!p) return CHT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    plan_free(p);
    delete p;
    return CHT_OK;
}

}  // extern "C"
