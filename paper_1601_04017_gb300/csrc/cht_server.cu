// Serving loop of libcht (declared in include/cht.h): continuous batching of
// requests over resident tables, built on the batched engine.
//
// Scheduling step: note completed steps (event queries; no blocking), then
// admit queued requests in arrival order -- skipping a table whose earlier
// request is not fully admitted, so every table sees its requests in arrival
// order -- while the step's limits and the request arena allow; run all
// admitted requests in one engine launch, snapshot the touched tables'
// counters and record an event.  Request arrays the GPU can address (device
// memory, pinned host memory, pageable host memory on systems such as Grace
// with NVLink-C2C) are read and written by the kernel in place -- no copy
// calls per request; the others are staged through a device ring (the
// arena): inputs copied in before the launch, results copied back after it.
// Up to max_inflight_steps steps are in flight; the host prepares the next
// step while the device runs the current one.
//
// Growth (growable tables, Sec. 4.3.2 trigger): the host knows each table's
// non-empty cells exactly as of its last completed step (the snapshots) plus
// an upper bound of what its in-flight steps add.  When an insert /
// insert-or-update request would push that bound past alpha * c, the table is
// first migrated to the smallest power-of-two capacity that holds the bound
// plus the whole request (bulk pre-sizing, Sec. 4.5; tombstones are dropped,
// Sec. 4.4).  The migration is ordered on the stream after the steps in
// flight, so admission never waits for counts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <initializer_list>
#include <list>
#include <new>
#include <vector>

#include "cht_internal.h"

using cht::u32;
using cht::u64;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// FIFO ring allocator over [0, cap) with monotone logical offsets; an
// allocation never wraps (it skips the ring's tail end instead).
struct Ring {
    u64 cap = 0, head = 0, tail = 0;
    bool alloc(u64 bytes, u64* off) {
        bytes = (bytes + 255) & ~255ull;
        if (bytes == 0 || bytes > cap) return false;
        u64 h = head;
        if ((h % cap) + bytes > cap) h += cap - (h % cap);
        if (h + bytes - tail > cap) return false;
        *off = h % cap;
        head = h + bytes;
        return true;
    }
    // bytes a new allocation could get right now without wrapping
    u64 contiguous_free() const {
        const u64 used = head - tail;
        const u64 to_end = cap - (head % cap);
        const u64 free_total = cap - used;
        if (to_end >= free_total) return free_total;
        // skipping to the start wastes to_end bytes
        return to_end > free_total - to_end ? to_end : free_total - to_end;
    }
};

struct Part {
    u64 req;
    u64 off;  // first operation of the request in this part
    u64 n;
    bool direct;  // arrays addressed in place (no staging copies)
    u64* d_keys;
    u64* d_vals;
    u64* d_vout;
    unsigned char* d_codes;
};

struct Step {
    std::vector<Part> parts;
    cudaEvent_t ev = nullptr;
    // timing: start of the step's device work (migrations, copies), engine
    // launch start / end; the step ends at `ev`
    cudaEvent_t t_begin = nullptr, t_eng0 = nullptr, t_eng1 = nullptr;
    bool eng_from_begin = false;  // no migration or copy ran before the engine: t_eng0 not recorded
    cudaEvent_t up = nullptr;     // the step's metadata upload (on the upload stream) is done
    u64 arena_end = 0, meta_end = 0, dmeta_end = 0;
    std::vector<u32> touched;
    std::vector<u64> new_cells;          // per touched table
    unsigned long long* snap = nullptr;  // pinned: (I, D) per touched table
    cht_server_step_record rec{};        // completed by poll() with the times
};

struct Req {
    cht_request r;
    bool direct = false;  // the engine addresses the request's arrays in place
    double t_arrival = 0, t_done = 0;
    u64 admitted = 0;
    u32 parts_inflight = 0;
    int state = 0;  // 0 queued, 1 fully admitted, 2 done, 3 rejected
    cht_status status = CHT_OK;
};

bool has_vals(int op) { return cht::mode_has_vals(op); }
bool fills(int op) { return cht::mode_fills(op); }

u64 per_op_bytes(const cht_request& r) {
    return 8 + (has_vals(r.op) ? 8 : 0) + (r.op == CHT_OP_FIND ? 8 : 0) + (r.codes ? 1 : 0);
}

}  // namespace

struct cht_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t ustream = nullptr;  // uploads of step metadata, overlapping the running step
    std::vector<cht_table*> tables;
    cht_server_config cfg{};
    unsigned char* arena = nullptr;  // device: request data
    Ring aring;
    unsigned char* meta = nullptr;  // pinned host: step metadata before upload
    Ring mring;
    unsigned char* dmeta = nullptr;  // device: step metadata
    Ring dring;
    u64 meta_bytes = 0;
    u64 max_step_items = 0;  // engine work items one step may use
    std::vector<Req> reqs;
    std::list<u64> queue;
    std::deque<Step> inflight;
    std::vector<u64> known_I, known_D, pending_new;
    std::vector<u32> parts_inflight;
    std::vector<cudaEvent_t> spare_events;
    std::vector<cudaEvent_t> spare_timers;
    std::vector<cudaEvent_t> spare_sync;  // upload-done events (no timing)
    u64 steps = 0, completed = 0;
    cht_server_profile prof{};
    std::vector<cht_server_step_record> trace;  // one record per completed step
    bool pageable_ok = false;  // device can address pageable host memory
};

namespace {

u64 tables_bytes(const cht_server* s) {
    u64 b = 0;
    for (cht_table* h : s->tables) b += (1ull << cht::table_info(h).log2c) * sizeof(cht::Cell);
    return b;
}

cht_status poll(cht_server* s, u32* completed_now) {
    u32 done = 0;
    while (!s->inflight.empty()) {
        Step& st = s->inflight.front();
        const cudaError_t q = cudaEventQuery(st.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
            cudaGetLastError();
            return CHT_ERR_CUDA;
        }
        const double t = now_s();
        for (const Part& p : st.parts) {
            Req& rq = s->reqs[p.req];
            --rq.parts_inflight;
            --s->parts_inflight[rq.r.table];
            if (rq.state == 1 && rq.parts_inflight == 0) {
                rq.state = 2;
                rq.t_done = t;
                ++s->completed;
                ++done;
            }
        }
        for (size_t k = 0; k < st.touched.size(); ++k) {
            const u32 t_ = st.touched[k];
            s->known_I[t_] = st.snap[2 * k];
            s->known_D[t_] = st.snap[2 * k + 1];
            s->pending_new[t_] -= st.new_cells[k];
            cht::table_set_bound(s->tables[t_], s->known_I[t_] + s->pending_new[t_], s->pending_new[t_] == 0);
        }
        float ms_step = 0, ms_eng = 0;
        if (cudaEventElapsedTime(&ms_step, st.t_begin, st.ev) == cudaSuccess) s->prof.gpu_step_ms += ms_step;
        if (cudaEventElapsedTime(&ms_eng, st.eng_from_begin ? st.t_begin : st.t_eng0, st.t_eng1) == cudaSuccess)
            s->prof.engine_ms += ms_eng;
        cudaGetLastError();
        st.rec.gpu_ms = ms_step;
        st.rec.engine_ms = ms_eng;
        s->trace.push_back(st.rec);
        s->aring.tail = st.arena_end;
        s->mring.tail = st.meta_end;
        s->dring.tail = st.dmeta_end;
        s->spare_events.push_back(st.ev);
        s->spare_timers.push_back(st.t_begin);
        s->spare_timers.push_back(st.t_eng0);
        s->spare_timers.push_back(st.t_eng1);
        if (st.up) s->spare_sync.push_back(st.up);
        s->inflight.pop_front();
    }
    if (completed_now) *completed_now = done;
    return CHT_OK;
}

// Admit what fits and launch one step.  *admitted = requests (or parts) in it.
cudaEvent_t take_timer(cht_server* s) {
    cudaEvent_t e = nullptr;
    if (!s->spare_timers.empty()) {
        e = s->spare_timers.back();
        s->spare_timers.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

cht_status admit_and_launch(cht_server* s, u32* admitted) {
    *admitted = 0;
    if (s->inflight.size() >= s->cfg.max_inflight_steps || s->queue.empty()) return CHT_OK;
    const size_t nt = s->tables.size();
    Step st;
    st.t_begin = take_timer(s);
    st.t_eng0 = take_timer(s);
    st.t_eng1 = take_timer(s);
    if (!st.t_begin || !st.t_eng0 || !st.t_eng1) {
        for (cudaEvent_t e : {st.t_begin, st.t_eng0, st.t_eng1})
            if (e) s->spare_timers.push_back(e);
        return CHT_ERR_CUDA;
    }
    // the timers go back to the spare list unless a step takes them
    struct TimerGuard {
        cht_server* s;
        Step* st;
        ~TimerGuard() {
            if (st && st->t_begin) {
                s->spare_timers.push_back(st->t_begin);
                s->spare_timers.push_back(st->t_eng0);
                s->spare_timers.push_back(st->t_eng1);
            }
        }
    } guard{s, &st};
    if (cudaEventRecord(st.t_begin, s->stream) != cudaSuccess) return CHT_ERR_CUDA;
    // device memory a growth may still take in this step: asked once per
    // step that grows a table, then decreased by each growth admitted
    long long hbm_left = 0;
    bool hbm_known = false;
    bool enqueued_before_engine = false;  // a migration or staging copy precedes the engine
    std::vector<char> blocked(nt, 0);
    std::vector<u64> step_new(nt, 0);
    std::vector<Part> parts;
    u64 ops = 0;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        if (parts.size() >= s->cfg.max_step_requests || ops >= s->cfg.max_step_ops) break;
        Req& rq = s->reqs[*it];
        const u32 t = rq.r.table;
        if (blocked[t]) {
            ++it;
            continue;
        }
        cht_table* h = s->tables[t];
        u64 m = rq.r.n - rq.admitted;
        if (m > s->cfg.max_step_ops - ops) m = s->cfg.max_step_ops - ops;
        const cht::TableInfo ti = cht::table_info(h);
        if (fills(rq.r.op) && ti.growable) {
            // Room check with an upper bound of the non-empty cells (every
            // admitted insert counted as new).  If the part does not fit, grow
            // now to the smallest capacity whose alpha-limit holds the bound
            // plus the whole part (the bulk pre-sizing of Sec. 4.5); the
            // migration is stream-ordered after the steps in flight, so it
            // needs neither a wait nor the exact count (it also drops
            // tombstones, which only lowers the count).
            const u64 used = s->known_I[t] + s->pending_new[t] + step_new[t];
            const u64 limit = u64(std::floor(ti.alpha * double(1ull << ti.log2c)));
            if (used + m > limit) {
                u32 nl = ti.log2c;
                while (nl < 40 && u64(std::floor(ti.alpha * double(1ull << nl))) < used + m) ++nl;
                const u64 need = (1ull << nl) * sizeof(cht::Cell);
                if (!hbm_known) {
                    hbm_left = (long long)cht::device_free_bytes(s->device) - (long long)s->cfg.hbm_reserve_bytes;
                    hbm_known = true;
                }
                const bool over_cap =
                    s->cfg.memory_cap_bytes && tables_bytes(s) + need + s->cfg.arena_bytes > s->cfg.memory_cap_bytes;
                if (over_cap || (long long)need > hbm_left) {
                    if (s->inflight.empty() && parts.empty()) {  // can never fit: reject
                        rq.state = 3;
                        rq.status = CHT_ERR_OOM;
                        rq.t_done = now_s();
                        ++s->completed;
                        it = s->queue.erase(it);
                        continue;
                    }
                    blocked[t] = 1;
                    ++it;
                    continue;
                }
                cht_status r = cht::table_migrate_to(h, nl, ~0ull, s->stream);
                if (r != CHT_OK) return r;
                hbm_left -= (long long)need;
                enqueued_before_engine = true;
                ++s->prof.migrations;
                ++st.rec.migrations;
            }
        }
        if (rq.direct) {  // the engine reads / writes the request's arrays in place
            Part p;
            p.req = *it;
            p.off = rq.admitted;
            p.n = m;
            p.d_keys = const_cast<u64*>(reinterpret_cast<const u64*>(rq.r.keys)) + rq.admitted;
            p.d_vals = has_vals(rq.r.op) ? const_cast<u64*>(reinterpret_cast<const u64*>(rq.r.vals)) + rq.admitted : nullptr;
            p.d_vout = rq.r.op == CHT_OP_FIND ? reinterpret_cast<u64*>(rq.r.vals_out) + rq.admitted : nullptr;
            p.d_codes = rq.r.codes ? rq.r.codes + rq.admitted : nullptr;
            p.direct = true;
            parts.push_back(p);
        } else {
        // arena space for this part
        const u64 pb = per_op_bytes(rq.r);
        const u64 fit = s->aring.contiguous_free() / pb;
        if (fit == 0) break;
        if (m > fit) m = fit;
        // up to four regions (keys, values or found values, codes), 256-byte aligned
        auto part_bytes = [&](u64 mm) {
            const u64 kb = (mm * 8 + 255) & ~255ull;
            return kb * (1 + (has_vals(rq.r.op) || rq.r.op == CHT_OP_FIND ? 1 : 0)) +
                   (rq.r.codes ? ((mm + 255) & ~255ull) : 0);
        };
        u64 off = 0;
        while (m > 0 && !s->aring.alloc(part_bytes(m), &off)) m /= 2;  // padding or ring end: smaller part
        if (m == 0) break;
        const u64 kb2 = (m * 8 + 255) & ~255ull;
        Part p;
        p.req = *it;
        p.off = rq.admitted;
        p.n = m;
        unsigned char* base = s->arena + off;
        p.d_keys = reinterpret_cast<u64*>(base);
        p.d_vals = has_vals(rq.r.op) ? reinterpret_cast<u64*>(base + kb2) : nullptr;
        p.d_vout = rq.r.op == CHT_OP_FIND ? reinterpret_cast<u64*>(base + kb2) : nullptr;
        p.d_codes = rq.r.codes ? base + kb2 * (has_vals(rq.r.op) || rq.r.op == CHT_OP_FIND ? 2 : 1) : nullptr;
        if (cudaMemcpyAsync(p.d_keys, rq.r.keys + rq.admitted, m * 8, cudaMemcpyDefault, s->stream) != cudaSuccess)
            return CHT_ERR_CUDA;
        enqueued_before_engine = true;
        if (p.d_vals &&
            cudaMemcpyAsync(p.d_vals, rq.r.vals + rq.admitted, m * 8, cudaMemcpyDefault, s->stream) != cudaSuccess)
            return CHT_ERR_CUDA;
        p.direct = false;
        parts.push_back(p);
        }
        rq.admitted += m;
        ++rq.parts_inflight;
        ++s->parts_inflight[t];
        if (fills(rq.r.op)) step_new[t] += m;
        ops += m;
        if (rq.admitted == rq.r.n) {
            rq.state = 1;
            it = s->queue.erase(it);
        } else {
            blocked[t] = 1;  // later requests of this table wait for the rest
            ++it;
        }
    }
    if (parts.empty()) return CHT_OK;

    // ---- step metadata: tables, batches (one per part, arrival order), items
    std::vector<cht::EngineTable> tabs(nt);
    for (size_t t = 0; t < nt; ++t) {
        const cht::TableInfo ti = cht::table_info(s->tables[t]);
        tabs[t].cells = ti.cells;
        tabs[t].log2c = ti.log2c;
        tabs[t].flags = (ti.reuse ? cht::kTabReuse : 0u) | (ti.full_keys ? cht::kTabFullKeys : 0u);
        tabs[t].st = ti.st;
    }
    std::vector<cht::EngineBatch> batches(parts.size());
    for (size_t i = 0; i < parts.size(); ++i) {
        const Req& rq = s->reqs[parts[i].req];
        batches[i].keys = parts[i].d_keys;
        batches[i].vals = parts[i].d_vals;
        batches[i].vals_out = parts[i].d_vout;
        batches[i].codes = parts[i].d_codes;
        batches[i].n = parts[i].n;
        batches[i].table = rq.r.table;
        batches[i].mode = u32(rq.r.op);
    }
    // work items sized per table from its chain of dependent requests; if
    // that needs more metadata than a step may use, take 64-operation items
    std::vector<cht::EngineChunk> chunks;
    u64 n_queue = cht::plan_order(batches, nt, 0, chunks);
    if (chunks.size() > s->max_step_items) {
        n_queue = cht::plan_order(batches, nt, 64, chunks);
        st.rec.recut = 1;
    }
    std::vector<u32> touched;
    std::vector<u64> tnew;
    {
        std::vector<char> seen(nt, 0);
        for (const cht::EngineBatch& b : batches)
            if (!seen[b.table]) {
                seen[b.table] = 1;
                touched.push_back(b.table);
                tnew.push_back(step_new[b.table]);
            }
    }
    // One upload holds the step's metadata: tables, batches, work items, the
    // engine's counters (zero), the touched tables' indices; the snapshot of
    // their counts is gathered on the device after the engine and read back
    // with one copy.
    const u64 b_tabs = nt * sizeof(cht::EngineTable), b_bat = batches.size() * sizeof(cht::EngineBatch);
    const u64 b_chk = chunks.size() * sizeof(cht::EngineChunk), b_cnt = (3 + nt) * sizeof(unsigned long long);
    const u64 b_tch = touched.size() * sizeof(u32), b_snap = touched.size() * 16;
    const u64 o_bat = (b_tabs + 255) & ~255ull, o_chk = o_bat + ((b_bat + 255) & ~255ull);
    const u64 o_cnt = o_chk + ((b_chk + 255) & ~255ull), o_tch = o_cnt + ((b_cnt + 255) & ~255ull);
    const u64 o_snap = o_tch + ((b_tch + 255) & ~255ull);
    const u64 total_meta = o_snap + b_snap;
    u64 hoff = 0, doff = 0;
    if (!s->mring.alloc(total_meta, &hoff) || !s->dring.alloc(total_meta, &doff)) return CHT_ERR_OOM;
    unsigned char* hm = s->meta + hoff;
    unsigned char* dm = s->dmeta + doff;
    memcpy(hm, tabs.data(), b_tabs);
    memcpy(hm + o_bat, batches.data(), b_bat);
    memcpy(hm + o_chk, chunks.data(), b_chk);
    memset(hm + o_cnt, 0, b_cnt);
    memcpy(hm + o_tch, touched.data(), b_tch);
    // the upload runs on its own stream, so it overlaps the step still running
    // on the main stream; the engine launch waits for it
    if (!s->spare_sync.empty()) {
        st.up = s->spare_sync.back();
        s->spare_sync.pop_back();
    } else if (cudaEventCreateWithFlags(&st.up, cudaEventDisableTiming) != cudaSuccess) {
        st.up = nullptr;
        return CHT_ERR_CUDA;
    }
    if (cudaMemcpyAsync(dm, hm, o_tch + b_tch, cudaMemcpyHostToDevice, s->ustream) != cudaSuccess ||
        cudaEventRecord(st.up, s->ustream) != cudaSuccess || cudaStreamWaitEvent(s->stream, st.up, 0) != cudaSuccess) {
        s->spare_sync.push_back(st.up);
        st.up = nullptr;
        return CHT_ERR_CUDA;
    }
    cht::EngineArgs e;
    e.tables = reinterpret_cast<const cht::EngineTable*>(dm);
    e.batches = reinterpret_cast<const cht::EngineBatch*>(dm + o_bat);
    e.chunks = reinterpret_cast<const cht::EngineChunk*>(dm + o_chk);
    e.n_chunks = n_queue;
    e.next = reinterpret_cast<unsigned long long*>(dm + o_cnt);
    e.done = e.next + 1;
    e.status = reinterpret_cast<u32*>(e.done + nt);
    e.spin_limit = 2000000000ll;
    e.max_backoff_ns = 8192;
    e.any_reuse = 0;
    e.any_full = 0;
    for (const cht::EngineTable& et : tabs) {
        e.any_reuse |= int(et.flags & cht::kTabReuse);
        e.any_full |= int((et.flags & cht::kTabFullKeys) != 0);
    }
    e.inject_stall = 0;
    // the engine's last warp writes the touched tables' counts straight into
    // the step's pinned snapshot (no separate kernel or copy)
    st.snap = reinterpret_cast<unsigned long long*>(hm + o_snap);
    e.snap_tables = reinterpret_cast<const u32*>(dm + o_tch);
    e.n_snap = u32(touched.size());
    e.snap_out = st.snap;
    e.warps_done = e.done + nt + 1;
    // nothing before the engine in this step: its start is the step's start
    st.eng_from_begin = !enqueued_before_engine;
    if (!st.eng_from_begin && cudaEventRecord(st.t_eng0, s->stream) != cudaSuccess) return CHT_ERR_CUDA;
    if (cht::launch_engine(e, 1, 2, 0, true, s->stream) != cudaSuccess) {
        cudaGetLastError();
        return CHT_ERR_CUDA;
    }
    if (cudaEventRecord(st.t_eng1, s->stream) != cudaSuccess) return CHT_ERR_CUDA;
    {
        // longest chain of dependent batches in this step (= its rounds)
        std::vector<u32> per_table(nt, 0);
        u32 rounds = 0;
        for (const cht::EngineBatch& b : batches) rounds = std::max(rounds, ++per_table[b.table]);
        s->prof.rounds += rounds;
        s->prof.chunks += chunks.size();
        s->prof.parts += batches.size();
        st.rec.rounds = rounds;
        st.rec.items = chunks.size();
        st.rec.parts = batches.size();
        for (const cht::EngineBatch& b : batches) st.rec.ops += b.n;
        for (const cht::EngineTable& et : tabs) st.rec.max_table_log2 = std::max(st.rec.max_table_log2, et.log2c);
    }
    // staged results back to the caller's arrays
    for (const Part& p : parts) {
        if (p.direct) continue;
        const Req& rq = s->reqs[p.req];
        if (p.d_vout && cudaMemcpyAsync(rq.r.vals_out + p.off, p.d_vout, p.n * 8, cudaMemcpyDefault, s->stream) !=
                            cudaSuccess)
            return CHT_ERR_CUDA;
        if (p.d_codes &&
            cudaMemcpyAsync(rq.r.codes + p.off, p.d_codes, p.n, cudaMemcpyDefault, s->stream) != cudaSuccess)
            return CHT_ERR_CUDA;
    }
    if (!s->spare_events.empty()) {
        st.ev = s->spare_events.back();
        s->spare_events.pop_back();
    } else if (cudaEventCreate(&st.ev) != cudaSuccess) {
        return CHT_ERR_CUDA;
    }
    if (cudaEventRecord(st.ev, s->stream) != cudaSuccess) return CHT_ERR_CUDA;
    st.arena_end = s->aring.head;
    st.meta_end = s->mring.head;
    st.dmeta_end = s->dring.head;
    for (size_t k = 0; k < touched.size(); ++k) s->pending_new[touched[k]] += tnew[k];
    st.touched = std::move(touched);
    st.new_cells = std::move(tnew);
    *admitted = u32(parts.size());
    st.parts = std::move(parts);
    s->inflight.push_back(std::move(st));
    guard.st = nullptr;  // the step in flight owns its timers now
    ++s->steps;
    return CHT_OK;
}

}  // namespace

// Can kernels on the server's device read and write p in place?
bool addressable(const cht_server* s, const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return at.device == s->device;
    if (at.type == cudaMemoryTypeHost) return true;  // pinned: mapped into the device's address space
    return s->pageable_ok;
}

extern "C" {

cht_status cht_server_create(const cht_handle* tables, uint32_t n_tables, const cht_server_config* cfg,
                             cht_stream_t stream, cht_server_handle* out) {
    if (!out || !tables || n_tables == 0) return CHT_ERR_INVALID_ARG;
    *out = nullptr;
    cht_server* s = new (std::nothrow) cht_server();
    if (!s) return CHT_ERR_OOM;
    s->cfg = cfg ? *cfg : cht_server_config{0, 0, 0, 0, 0, 0, 0};
    if (s->cfg.arena_bytes == 0) s->cfg.arena_bytes = 1ull << 30;
    if (s->cfg.hbm_reserve_bytes == 0) s->cfg.hbm_reserve_bytes = 1ull << 30;
    if (s->cfg.max_inflight_steps == 0) s->cfg.max_inflight_steps = 2;
    if (s->cfg.max_step_requests == 0) s->cfg.max_step_requests = 8192;
    if (s->cfg.max_step_ops == 0) s->cfg.max_step_ops = 1ull << 26;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    for (uint32_t i = 0; i < n_tables; ++i) {
        if (!tables[i]) {
            delete s;
            return CHT_ERR_INVALID_ARG;
        }
        const cht::TableInfo ti = cht::table_info(tables[i]);
        if (i == 0) s->device = ti.device;
        if (ti.device != s->device) {
            delete s;
            return CHT_ERR_INVALID_ARG;
        }
        s->tables.push_back(tables[i]);
    }
    const size_t nt = s->tables.size();
    s->known_I.assign(nt, 0);
    s->known_D.assign(nt, 0);
    s->pending_new.assign(nt, 0);
    s->parts_inflight.assign(nt, 0);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    if (cudaStreamCreateWithFlags(&s->ustream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s->ustream = nullptr;
        if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
        delete s;
        return CHT_ERR_CUDA;
    }
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, s->device) != cudaSuccess) {
        cudaGetLastError();
        pageable = 0;
    }
    s->pageable_ok = pageable != 0;
    // exact starting counts of every table
    cht_status r = CHT_OK;
    for (size_t t = 0; t < nt && r == CHT_OK; ++t) r = cht::table_read_counts(s->tables[t], &s->known_I[t], &s->known_D[t], s->stream);
    // metadata rings: room for several steps of the largest size (twice
    // over, so a step also fits when the free space is split at the ring end)
    // work items: room for items of 64 operations on average (the per-table
    // sizing cuts long chains finer than 256)
    s->max_step_items = s->cfg.max_step_ops / 64 + s->cfg.max_step_requests;
    s->meta_bytes = (s->max_step_items + s->cfg.max_step_requests + 1) * 48 +
                    nt * (sizeof(cht::EngineTable) + 40) + (1u << 20);
    s->meta_bytes *= 2 * (s->cfg.max_inflight_steps + 1);
    s->aring.cap = s->cfg.arena_bytes;
    s->mring.cap = s->meta_bytes;
    s->dring.cap = s->meta_bytes;
    if (r == CHT_OK) r = cht::runtime_alloc(reinterpret_cast<void**>(&s->arena), s->cfg.arena_bytes, s->stream);
    if (r == CHT_OK) r = cht::runtime_alloc(reinterpret_cast<void**>(&s->dmeta), s->meta_bytes, s->stream);
    if (r == CHT_OK && cudaHostAlloc(reinterpret_cast<void**>(&s->meta), s->meta_bytes, cudaHostAllocDefault) != cudaSuccess)
        r = CHT_ERR_OOM;
    if (r == CHT_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) r = CHT_ERR_CUDA;
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (r != CHT_OK) {
        cht_server_destroy(s);
        return r;
    }
    *out = s;
    return CHT_OK;
}

cht_status cht_server_submit(cht_server_handle s, const cht_request* req, uint64_t* id) {
    if (!s || !req || req->table >= s->tables.size() || req->op < CHT_OP_FIND || req->op > CHT_OP_UPDATE_OVERWRITE ||
        req->n == 0 || !req->keys || (has_vals(req->op) && !req->vals) || (req->op == CHT_OP_FIND && !req->vals_out))
        return CHT_ERR_INVALID_ARG;
    Req rq;
    rq.r = *req;
    rq.direct = !s->cfg.stage_inputs && addressable(s, req->keys) && (!has_vals(req->op) || addressable(s, req->vals)) &&
                (req->op != CHT_OP_FIND || addressable(s, req->vals_out)) && (!req->codes || addressable(s, req->codes));
    rq.t_arrival = now_s();
    const u64 i = s->reqs.size();
    s->reqs.push_back(rq);
    s->queue.push_back(i);
    if (id) *id = i;
    return CHT_OK;
}

cht_status cht_server_step(cht_server_handle s, uint32_t* admitted, uint32_t* completed) {
    if (!s) return CHT_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    u32 c = 0, a = 0;
    cht_status r = poll(s, &c);
    const double h0 = now_s();
    if (r == CHT_OK) r = admit_and_launch(s, &a);
    if (a) s->prof.host_admit_ms += (now_s() - h0) * 1e3;
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (admitted) *admitted = a;
    if (completed) *completed = c;
    return r;
}

cht_status cht_server_drain(cht_server_handle s) {
    if (!s) return CHT_ERR_INVALID_ARG;
    while (s->completed < s->reqs.size()) {
        cht_status r = cht_server_step(s, nullptr, nullptr);
        if (r != CHT_OK) return r;
        if (!s->inflight.empty() && s->inflight.size() >= s->cfg.max_inflight_steps) cudaEventSynchronize(s->inflight.front().ev);
        else if (s->queue.empty() && !s->inflight.empty()) cudaEventSynchronize(s->inflight.front().ev);
    }
    return CHT_OK;
}

cht_status cht_server_result(cht_server_handle s, uint64_t id, int* done, double* latency_s, cht_status* req_status) {
    if (!s || id >= s->reqs.size()) return CHT_ERR_INVALID_ARG;
    const Req& rq = s->reqs[id];
    if (done) *done = rq.state >= 2;
    if (latency_s) *latency_s = rq.state >= 2 ? rq.t_done - rq.t_arrival : 0.0;
    if (req_status) *req_status = rq.status;
    return CHT_OK;
}

cht_status cht_server_replay(cht_server_handle s, const cht_request* reqs, const double* arrival_s, uint64_t n,
                             double* latency_s, double* makespan_s) {
    if (!s || (n > 0 && (!reqs || !arrival_s))) return CHT_ERR_INVALID_ARG;
    const u64 first = s->reqs.size();
    const double t0 = now_s();
    u64 next = 0;
    while (next < n || s->completed < s->reqs.size()) {
        const double t = now_s() - t0;
        while (next < n && arrival_s[next] <= t) {
            uint64_t id;
            cht_status r = cht_server_submit(s, &reqs[next], &id);
            if (r != CHT_OK) return r;
            s->reqs[id].t_arrival = t0 + arrival_s[next];  // scheduled arrival
            ++next;
        }
        cht_status r = cht_server_step(s, nullptr, nullptr);
        if (r != CHT_OK) return r;
    }
    double last = t0;
    for (u64 i = 0; i < n; ++i) {
        const Req& rq = s->reqs[first + i];
        if (latency_s) latency_s[i] = rq.t_done - rq.t_arrival;
        if (rq.t_done > last) last = rq.t_done;
    }
    if (makespan_s) *makespan_s = last - t0;
    return CHT_OK;
}

cht_status cht_server_stats(cht_server_handle s, uint64_t* steps, uint64_t* completed) {
    if (!s) return CHT_ERR_INVALID_ARG;
    if (steps) *steps = s->steps;
    if (completed) *completed = s->completed;
    return CHT_OK;
}

cht_status cht_server_get_profile(cht_server_handle s, cht_server_profile* out) {
    if (!s || !out) return CHT_ERR_INVALID_ARG;
    *out = s->prof;
    out->steps = s->steps;
    out->completed = s->completed;
    return CHT_OK;
}

cht_status cht_server_get_trace(cht_server_handle s, cht_server_step_record* out, uint64_t max, uint64_t* n) {
    if (!s || !n || (max > 0 && !out)) return CHT_ERR_INVALID_ARG;
    const u64 k = std::min<u64>(max, s->trace.size());
    for (u64 i = 0; i < k; ++i) out[i] = s->trace[i];
    *n = s->trace.size();
    return CHT_OK;
}

cht_status cht_server_destroy(cht_server_handle s) {
    if (!s) return CHT_ERR_INVALID_ARG;
    if (s->stream || !s->inflight.empty()) cudaStreamSynchronize(s->stream);
    if (s->ustream) cudaStreamSynchronize(s->ustream);
    for (Step& st : s->inflight)
        for (cudaEvent_t e : {st.ev, st.t_begin, st.t_eng0, st.t_eng1, st.up})
            if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    for (cudaEvent_t e : s->spare_timers) cudaEventDestroy(e);
    for (cudaEvent_t e : s->spare_sync) cudaEventDestroy(e);
    if (s->ustream) cudaStreamDestroy(s->ustream);
    if (s->arena) cht::runtime_free(s->arena, s->cfg.arena_bytes, s->stream);
    if (s->dmeta) cht::runtime_free(s->dmeta, s->meta_bytes, s->stream);
    if (s->meta) cudaFreeHost(s->meta);
    cudaStreamSynchronize(s->stream);
    delete s;
    return CHT_OK;
}

}  // extern "C"
