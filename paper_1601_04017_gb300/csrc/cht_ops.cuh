// Batched probe kernels of libcht: find, insert, insertOrUpdate (add /
// overwrite) and erase over the folklore linear-probing table (Sec. 3,
// Algorithm 1; tombstone erase, Sec. 4.4).
//
// Work layout.  Each warp owns a contiguous slice of the operation batch.
// Its lanes form 32/G groups of G lanes; a group probes one key at a time
// over an aligned window of W = G*V cells, each lane fetching V cells (V = 2:
// one 256-bit load = one 32-byte DRAM sector; V = 1: one 16-byte load).
// A group that finishes its key immediately takes the next key of the warp's
// slice ("refill"), so every probe step of the warp issues loads for all of
// its groups instead of idling while the slowest probe of a fixed set of 32
// keys finishes.  Keys loaded in the same refill step are pre-reduced with
// __match_any_sync: one leader per distinct key performs the table operation
// (with the summed value for insertOrUpdate(add)); the others resolve at once
// as "not inserted / updated / not erased", which is a valid linearization
// (they are ordered right after the leader).
//
// Probe step (Algorithm 1).  The first cell in probe order that holds the key
// or is empty decides: find reads it; erase CASes its key to the tombstone;
// insert / insertOrUpdate CAS <0,0> -> <k,d> into an empty cell and, if the
// CAS reveals the same key, apply the update (fetch-and-add or store, the
// specialised atomicUpdate of Sec. 3); a CAS that reveals another key moves
// on to the next cell (Algorithm 1 re-reads the cell; the CAS already
// returned its content).  Keys only ever change empty -> key -> tombstone,
// so a stale window can only show "empty" too early, which the CAS corrects.
// Every probe is bounded by c cells; an insert that sees all c cells reports
// "table full".
#pragma once

#include "cht_internal.h"

namespace cht {

constexpr int kOpBlock = 256;

template <int G>
struct GroupConsts {
    static constexpr u32 leaders = G == 1 ? 0xffffffffu
                                 : G == 2 ? 0x55555555u
                                 : G == 4 ? 0x11111111u
                                 : G == 8 ? 0x01010101u
                                 : G == 16 ? 0x00010001u
                                           : 0x00000001u;
};

// Outcome of a leader's atomic step.  kStepRestart: a tombstone the probe
// meant to reuse was taken by another key first -- probe again from the cell
// after it; kStepDoneReused: inserted into a reused tombstone.
enum : int { kStepDoneNo = 0, kStepDoneYes = 1, kStepContinue = 2, kStepRestart = 3, kStepDoneReused = 4 };

constexpr u64 kNoPos = ~0ull;

template <int MODE>
__device__ __forceinline__ int modify_at(Cell* cp, bool is_key, u64 key, u64 d) {
    if (MODE == kUpdAdd || MODE == kUpdOverwrite) {  // update: present keys only
        if (!is_key) return kStepDoneNo;
        if (MODE == kUpdAdd) atomicAdd(&cp->val, d);
        else atomicExch(&cp->val, d);
        return kStepDoneYes;
    }
    if (is_key) {
        if (MODE == kInsert) return kStepDoneNo;
        if (MODE == kIouAdd) { atomicAdd(&cp->val, d); return kStepDoneNo; }
        if (MODE == kIouOverwrite) { atomicExch(&cp->val, d); return kStepDoneNo; }
        // kErase: 1-word CAS of the key to the tombstone, value untouched.
        const u64 old = atomicCAS(&cp->key, key, kTomb);
        return old == key ? kStepDoneYes : kStepDoneNo;
    }
    // empty cell
    if (MODE == kErase) return kStepDoneNo;
    Cell expect;
    expect.key = kEmpty;
    expect.val = 0;
    Cell desired;
    desired.key = key;
    desired.val = d;
    const Cell old = cas_cell(cp, expect, desired);
    if (old.key == kEmpty && old.val == 0) return kStepDoneYes;
    if (old.key == key) {
        if (MODE == kIouAdd) atomicAdd(&cp->val, d);
        if (MODE == kIouOverwrite) atomicExch(&cp->val, d);
        return kStepDoneNo;
    }
    return kStepContinue;
}

// Full key space: an operation on key 0 or ~0 works on the table's special
// slot for it (slot 0 / 1 in DevState) with the dictionary meaning; under
// phase semantics one batch holds one operation type, so presence flips only
// one way per batch.  The value of an absent key is 0, so insertOrUpdate(add)
// can add unconditionally.  Returns the operation's result code.
template <int MODE>
__device__ __forceinline__ unsigned char special_op(DevState* st, u64 key, u64 d, u64* vout) {
    const int s = key == kTomb ? 1 : 0;
    unsigned int* pres = &st->sp_present[s];
    unsigned long long* val = reinterpret_cast<unsigned long long*>(&st->sp_val[s]);
    if (MODE == kFind) {
        const u32 p = *reinterpret_cast<volatile unsigned int*>(pres);
        *vout = p ? *reinterpret_cast<volatile unsigned long long*>(val) : 0;
        return p ? kYes : kNo;
    }
    if (MODE == kUpdAdd || MODE == kUpdOverwrite) {
        if (*reinterpret_cast<volatile unsigned int*>(pres) == 0) return kNo;
        if (MODE == kUpdAdd) atomicAdd(val, d);
        else atomicExch(val, d);
        return kYes;
    }
    if (MODE == kErase) {
        if (atomicCAS(pres, 1u, 0u) != 1u) return kNo;
        atomicExch(val, 0ull);
        return kYes;
    }
    const bool ins = atomicCAS(pres, 0u, 1u) == 0u;
    if (MODE == kIouAdd) atomicAdd(val, d);
    else if (MODE == kIouOverwrite || ins) atomicExch(val, d);
    return ins ? kYes : kNo;
}

// Tombstone reuse (insert modes, reuse on): the probe has shown `key`
// absent (it reached an empty cell or saw every cell) after passing the
// tombstone at cp.  Claim it with a 16-byte CAS on the content read now.
// Under phase semantics tombstones only change by such claims, so a cell that
// is no longer a tombstone, or a failed CAS, means another key took the cell
// (start again after it) or the same key did (then it is present: update it).
template <int MODE>
__device__ __forceinline__ int claim_tomb(Cell* cp, u64 key, u64 d) {
    u64 ck, cv;
    ld_cell_cg(cp, ck, cv);
    if (ck != kTomb) {
        if (ck != key) return kStepRestart;
        if (MODE == kIouAdd) atomicAdd(&cp->val, d);
        if (MODE == kIouOverwrite) atomicExch(&cp->val, d);
        return kStepDoneNo;
    }
    Cell expect;
    expect.key = kTomb;
    expect.val = cv;
    Cell desired;
    desired.key = key;
    desired.val = d;
    const Cell old = cas_cell(cp, expect, desired);
    if (old.key == kTomb && old.val == cv) return kStepDoneReused;
    if (old.key == key) {
        if (MODE == kIouAdd) atomicAdd(&cp->val, d);
        if (MODE == kIouOverwrite) atomicExch(&cp->val, d);
        return kStepDoneNo;
    }
    return kStepRestart;
}

// One warp runs the operations [next, end) of the batch with the group
// refill loop; counters and status bits accumulate into the caller's
// registers (every lane of the warp must call it).  kCoherent: finds read the
// table through L2 like the modifying modes (required when the same kernel
// launch also modifies the table); otherwise finds use the read-only path.
// Where a warp takes its keys / values and puts its results: the batch's
// arrays in global memory, or (kStaged) a per-warp area in shared memory that
// holds operations [base, base + count) -- the engine fills it with one
// coalesced pass and writes the results back with one, which matters when
// the arrays live in host memory across NVLink-C2C.
struct WarpStage {
    u64* keys;
    u64* vals;
    u64* vout;
    unsigned char* codes;
    u64 base;
};

template <bool kStaged>
__device__ __forceinline__ u64 op_key(const OpArgs& a, const WarpStage& sg, u64 idx) {
    return kStaged ? sg.keys[idx - sg.base] : ld_stream(a.keys + idx);
}
template <bool kStaged>
__device__ __forceinline__ u64 op_val(const OpArgs& a, const WarpStage& sg, u64 idx) {
    return kStaged ? sg.vals[idx - sg.base] : ld_stream(a.vals + idx);
}
template <bool kStaged>
__device__ __forceinline__ void op_code(const OpArgs& a, const WarpStage& sg, u64 idx, unsigned char c) {
    if (kStaged) sg.codes[idx - sg.base] = c;
    else if (a.codes) a.codes[idx] = c;
}
template <bool kStaged>
__device__ __forceinline__ void op_vout(const OpArgs& a, const WarpStage& sg, u64 idx, u64 v) {
    if (kStaged) sg.vout[idx - sg.base] = v;
    else a.vals_out[idx] = v;
}

// kFlags: bit 0 = tombstone reuse (insert modes), bit 1 = full key space;
// compile-time, so a table without them runs the plain probe loop.
constexpr int kFlagReuse = 1;
constexpr int kFlagFullKeys = 2;

template <int G, int V, int MODE, bool kCoherent = false, bool kStaged = false, int kFlags = 0>
__device__ __forceinline__ void warp_ops(const OpArgs& a, u64 next, const u64 end, u64& n_ins, u64& n_del,
                                         u32& sbits, const WarpStage& sg = WarpStage{}) {
    constexpr u32 W = G * V;
    constexpr u32 FULL = 0xffffffffu;
    constexpr bool kModify = MODE != kFind;
    constexpr bool kHasVals = mode_has_vals(MODE);
    constexpr bool kInsLike = mode_fills(MODE);  // modes that may fill a cell
    constexpr bool kUpdate = MODE == kUpdAdd || MODE == kUpdOverwrite;
    // (not in the engine, kCoherent: over its many small, mostly L2-resident
    // tables the CAS-first step made the 4096-table workload 45 % slower)
    constexpr bool kCasFirst = MODE == kInsert && G == 1 && kFlags == 0 && !kCoherent;
    // Finds whose window spans more than one 128-byte line skip the sectors
    // that lie wholly before `first` (cells before it are never examined): on
    // the first step this saves the line in front of the home cell's.
    // (Inserts keep whole windows: with the extra predicates the 5-CTA bound
    // spilled more registers and the load-0.9 inserts took 10.2 -> 14.4 ms;
    // one-line windows gain nothing, the line is fetched whole anyway.)
    constexpr bool kSkipBeforeFirst = MODE == kFind && W * sizeof(Cell) > 128;

    const u64 cap = 1ull << a.log2c;
    const u64 cmask = cap - 1;
    const u32 shift = 64u - a.log2c;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int g0 = lane & ~(G - 1);
    const u32 group_lanes = (G == 32) ? FULL : (((1u << G) - 1u) << g0);
    const u32 below_group = (1u << g0) - 1u;

    bool active = false;
    u64 idx = 0, key = 0, d = 0, pos = 0, probed = 0;
    // tombstone reuse: tdist = 1 + the distance from the current key's home
    // to the first tombstone on its path (0: none yet)
    constexpr bool reuse = kInsLike && (kFlags & kFlagReuse) != 0;
    constexpr bool kFullKeys = (kFlags & kFlagFullKeys) != 0;  // (kFull is the status bit)
    u64 tdist = 0;

    // Unstaged: the warp's next 64 keys (and values) are held in registers,
    // two windows of 32 -- lane j holds operation wbase + j of `cur` and
    // wbase + 32 + j of `nxt` -- loaded with coalesced 256-byte reads one
    // window ahead, so a refill takes its key by shuffle instead of a
    // dependent load from memory.  Invariant: next - wbase < 32 between
    // refills (a refill takes at most 32 operations).
    u64 wbase = next, k_cur = 0, v_cur = 0, k_nxt = 0, v_nxt = 0;
    if (!kStaged) {
        if (wbase + lane < end) {
            k_cur = ld_stream(a.keys + wbase + lane);
            if (kHasVals) v_cur = ld_stream(a.vals + wbase + lane);
        }
        if (wbase + 32 + lane < end) {
            k_nxt = ld_stream(a.keys + wbase + 32 + lane);
            if (kHasVals) v_nxt = ld_stream(a.vals + wbase + 32 + lane);
        }
    }

    for (;;) {
        // ---- refill idle groups from this warp's slice
        bool fresh = false;
        const u32 idle = __ballot_sync(FULL, !active) & GroupConsts<G>::leaders;
        if (idle != 0 && next < end) {
            const u64 my = next + __popc(idle & below_group);
            u64 wk = 0, wv = 0;
            if (!kStaged) {  // every lane shuffles; only idle groups use the result
                const u32 o = u32(my - wbase);
                const u64 xk = __shfl_sync(FULL, k_cur, o & 31), yk = __shfl_sync(FULL, k_nxt, o & 31);
                wk = o < 32 ? xk : yk;
                if (kHasVals) {
                    const u64 xv = __shfl_sync(FULL, v_cur, o & 31), yv = __shfl_sync(FULL, v_nxt, o & 31);
                    wv = o < 32 ? xv : yv;
                }
            }
            if (!active) {
                if (my < end) {
                    idx = my;
                    key = kStaged ? op_key<kStaged>(a, sg, idx) : wk;
                    if (kHasVals) d = kStaged ? op_val<kStaged>(a, sg, idx) : wv;
                    if (is_reserved(key)) {
                        if (gl == 0) {
                            if (kFullKeys) {
                                u64 v = 0;
                                op_code<kStaged>(a, sg, idx, special_op<MODE>(a.st, key, d, &v));
                                if (MODE == kFind) op_vout<kStaged>(a, sg, idx, v);
                            } else {
                                op_code<kStaged>(a, sg, idx, kCodeReserved);
                                if (MODE == kFind) op_vout<kStaged>(a, sg, idx, 0);
                            }
                        }
                        if (!kFullKeys) sbits |= kReserved;
                    } else {
                        fresh = true;
                        active = true;
                        pos = home_of(key, shift);
                        probed = 0;
                        tdist = 0;
                    }
                }
            }
            next += __popc(idle);
            if (!kStaged && next - wbase >= 32) {  // slide: nxt becomes cur, load the one after
                wbase += 32;
                k_cur = k_nxt;
                v_cur = v_nxt;
                if (wbase + 32 + lane < end) {
                    k_nxt = ld_stream(a.keys + wbase + 32 + lane);
                    if (kHasVals) v_nxt = ld_stream(a.vals + wbase + 32 + lane);
                }
            }
        }

        // ---- pre-reduce equal keys loaded in this step (modifying modes; an
        // update reports presence per operation, so each one probes itself)
        if (kModify && !kUpdate) {
            const u32 fm = __ballot_sync(FULL, fresh && gl == 0);
            if (fm & (fm - 1u)) {
                bool dup = false;
                if (fresh && gl == 0) {
                    const u32 same = __match_any_sync(fm, key);
                    const int lead = __ffs(same) - 1;
                    if (MODE == kIouAdd) {
                        u32 rem = same;
                        u64 total = 0;
                        while (__any_sync(fm, rem != 0)) {
                            const int src = rem ? __ffs(rem) - 1 : lane;
                            const u64 x = __shfl_sync(fm, d, src);
                            if (rem) {
                                total += x;
                                rem &= rem - 1u;
                            }
                        }
                        d = total;
                    }
                    dup = lane != lead;
                }
                if (G > 1) {
                    dup = __shfl_sync(FULL, dup, g0);
                    if (MODE == kIouAdd) d = __shfl_sync(FULL, d, g0);
                }
                if (dup) {
                    if (gl == 0) op_code<kStaged>(a, sg, idx, kNo);
                    active = false;
                }
            }
        }

        // ---- insert, one lane per key (the window of short probes at low
        // load), single calls: the home cell's 16-byte CAS is a fresh key's
        // first probe step.  It claims an empty home at once, and a taken home comes back
        // as the CAS's result, so most keys need one round trip instead of a
        // load followed by the CAS.  (Tombstone reuse needs the first
        // tombstone of the path, so tables with table options keep the plain
        // loop.)
        if (kCasFirst && fresh && active) {
            Cell expect;
            expect.key = kEmpty;
            expect.val = 0;
            Cell desired;
            desired.key = key;
            desired.val = d;
            const Cell old = cas_cell(a.cells + pos, expect, desired);
            if (old.key == kEmpty && old.val == 0) {
                op_code<kStaged>(a, sg, idx, kYes);
                ++n_ins;
                active = false;
            } else if (old.key == key) {
                op_code<kStaged>(a, sg, idx, kNo);
                active = false;
            } else {
                probed = 1;
                pos = (pos + 1) & cmask;
            }
        }

        if (!__any_sync(FULL, active)) {
            if (next >= end) break;
            continue;
        }

        // ---- one probe step: load the window holding `pos`
        const u64 base = pos & ~u64(W - 1);
        const u32 first = u32(pos - base);
        // each lane holds V consecutive cells of the window (V = 2: one
        // 32-byte sector; V = 4: two sectors, issued back to back)
        u64 kk[V], vv[V];
#pragma unroll
        for (int j = 0; j < V; ++j) kk[j] = vv[j] = 0;
        int hit = -1;
        bool match = false;
        u64 hv = 0;
        if (active) {
            const Cell* p = a.cells + base + u32(gl) * V;
            const u32 o0 = u32(gl) * V;
            if (V == 1) {
                if (!kSkipBeforeFirst || o0 >= first) {
                    if (kModify || kCoherent) ld_cell_cg(p, kk[0], vv[0]);
                    else ld_cell_nc(p, kk[0], vv[0]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < V; j += 2) {
                    if (!kSkipBeforeFirst || o0 + j + 1 >= first) {
                        if (kModify || kCoherent) ld_pair_cg(p + j, kk[j], vv[j], kk[j + 1], vv[j + 1]);
                        else ld_pair_nc(p + j, kk[j], vv[j], kk[j + 1], vv[j + 1]);
                    }
                }
            }
#pragma unroll
            for (int j = V - 1; j >= 0; --j) {  // the lowest qualifying cell wins
                if (o0 + j >= first && (kk[j] == key || kk[j] == kEmpty)) {
                    hit = int(o0 + j);
                    match = kk[j] == key;
                    hv = vv[j];
                }
            }
        }
        int ghit = hit;
        bool gmatch = match;
        u64 gval = hv;
        if (G > 1) {
            const u32 b = __ballot_sync(FULL, hit >= 0) & group_lanes;
            const int src = b ? __ffs(b) - 1 : lane;
            ghit = __shfl_sync(FULL, hit, src);
            gmatch = __shfl_sync(FULL, int(match), src) != 0;
            if (MODE == kFind) gval = __shfl_sync(FULL, hv, src);
        }
        if (kInsLike && reuse) {
            // first tombstone of the window at or after `first` (lanes hold
            // the window's cells in order, so the lowest lane has it)
            int toff = -1;
            if (active) {
                const u32 o0 = u32(gl) * V;
#pragma unroll
                for (int j = V - 1; j >= 0; --j)
                    if (o0 + j >= first && kk[j] == kTomb) toff = int(o0 + j);
            }
            if (G > 1) {
                const u32 b = __ballot_sync(FULL, toff >= 0) & group_lanes;
                const int src = b ? __ffs(b) - 1 : lane;
                const int t2 = __shfl_sync(FULL, toff, src);
                toff = b ? t2 : -1;
            }
            // only a tombstone before the deciding cell is on the path
            if (active && tdist == 0 && toff >= 0 && (ghit < 0 || toff < ghit))
                tdist = probed + u32(toff) - first + 1;
        }

        int outcome = kStepContinue;
        if (active && ghit >= 0) {
            if (MODE == kFind) {
                if (gl == 0) {
                    op_vout<kStaged>(a, sg, idx, gmatch ? gval : 0);
                    op_code<kStaged>(a, sg, idx, gmatch ? kYes : kNo);
                }
                active = false;
            } else if (gl == 0) {
                if (kInsLike && !gmatch && tdist != 0)
                    outcome = claim_tomb<MODE>(a.cells + ((home_of(key, shift) + tdist - 1) & cmask), key, d);
                else
                    outcome = modify_at<MODE>(a.cells + base + u32(ghit), gmatch, key, d);
            }
        }
        if (kModify && G > 1) outcome = __shfl_sync(FULL, outcome, g0);

        if (active) {
            if (ghit < 0) {
                probed += W - first;
                pos = (base + W) & cmask;
            } else if (kModify) {
                if (outcome == kStepContinue) {
                    probed += u32(ghit) - first + 1;
                    pos = (base + u32(ghit) + 1) & cmask;
                } else if (kInsLike && outcome == kStepRestart) {
                    pos = (home_of(key, shift) + tdist) & cmask;
                    probed = tdist;
                    tdist = 0;
                } else {
                    if (gl == 0) {
                        op_code<kStaged>(a, sg, idx, outcome == kStepDoneReused ? kYes : (unsigned char)outcome);
                        if (outcome == kStepDoneYes) {
                            if (MODE == kErase) ++n_del;
                            else if (kInsLike) ++n_ins;
                        }
                        if (kInsLike && outcome == kStepDoneReused) --n_del;  // one tombstone fewer (mod 2^64)
                    }
                    active = false;
                }
            }
            if (kInsLike && reuse && active && probed >= cap && tdist != 0) {
                // every cell seen, no empty one and no key: take the tombstone
                // (group-uniform branch: shuffle within the group only)
                int fo = kStepContinue;
                if (gl == 0) fo = claim_tomb<MODE>(a.cells + ((home_of(key, shift) + tdist - 1) & cmask), key, d);
                if (G > 1) fo = __shfl_sync(group_lanes, fo, g0);
                if (fo == kStepRestart) {
                    pos = (home_of(key, shift) + tdist) & cmask;
                    probed = tdist;
                    tdist = 0;
                } else {
                    if (gl == 0) {
                        op_code<kStaged>(a, sg, idx, fo == kStepDoneReused ? kYes : (unsigned char)fo);
                        if (fo == kStepDoneReused) --n_del;
                    }
                    active = false;
                }
            }
            if (active && probed >= cap) {
                // every cell was examined without a decision
                if (gl == 0) {
                    if (MODE == kFind) {
                        op_vout<kStaged>(a, sg, idx, 0);
                        op_code<kStaged>(a, sg, idx, kNo);
                    } else if (MODE == kErase || kUpdate) {
                        op_code<kStaged>(a, sg, idx, kNo);
                    } else {
                        op_code<kStaged>(a, sg, idx, kCodeFull);
                    }
                }
                if (kInsLike) sbits |= kFull;
                active = false;
            }
        }
    }

}

// Sum the CTA's counters and status bits into the table's device state with
// one atomic per counter and CTA (a warp each would put thousands of atomics
// on the same two words at the end of a launch).  Every thread of the CTA
// calls it once, at the end of the kernel.
__device__ __forceinline__ void block_flush_counters(DevState* st, u64 n_ins, u64 n_del, u32 sbits) {
    constexpr u32 FULL = 0xffffffffu;
    __shared__ unsigned long long s_ins, s_del;
    __shared__ u32 s_bits;
    if (threadIdx.x == 0) {
        s_ins = 0;
        s_del = 0;
        s_bits = 0;
    }
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        n_ins += __shfl_xor_sync(FULL, n_ins, o);
        n_del += __shfl_xor_sync(FULL, n_del, o);
    }
    const u32 any_status = __reduce_or_sync(FULL, sbits);
    if ((threadIdx.x & 31) == 0) {
        if (n_ins) atomicAdd(&s_ins, n_ins);
        if (n_del) atomicAdd(&s_del, n_del);
        if (any_status) atomicOr(&s_bits, any_status);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_ins) atomicAdd(&st->I, s_ins);
        if (s_del) atomicAdd(&st->D, s_del);
        if (s_bits) atomicOr(&st->status, s_bits);
    }
}

// Sum the warp's counters and status bits into the table's device state.
__device__ __forceinline__ void warp_flush_counters(DevState* st, u64 n_ins, u64 n_del, u32 sbits) {
    constexpr u32 FULL = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
        n_ins += __shfl_xor_sync(FULL, n_ins, o);
        n_del += __shfl_xor_sync(FULL, n_del, o);
    }
    const u32 any_status = __reduce_or_sync(FULL, sbits);
    if ((threadIdx.x & 31) == 0) {
        if (n_ins) atomicAdd(&st->I, n_ins);
        if (n_del) atomicAdd(&st->D, n_del);
        if (any_status) atomicOr(&st->status, any_status);
    }
}

// Two sectors per lane (V = 4) need more registers; for the wide windows
// (G >= 4, the long probes at high load) asking for 5 resident CTAs per SM
// (48 registers) keeps 40 warps' loads in flight instead of 32 (measured:
// find misses at load 0.9 3 % faster, inserts to 0.9 7 %).  The 2-lane
// window of short probes is faster with its natural register count.
template <int G, int V>
constexpr int op_min_blocks() {
    return (V == 4 && G >= 4) ? 5 : 1;
}

// Programmatic dependent launch: the operation kernels are launched so that
// the next one on the stream may be scheduled while this one drains; each
// lets its dependents start at once and then waits until the grids before it
// have completed and their memory is visible (a no-op when it was launched
// the ordinary way).  Stream order of every memory effect is unchanged; the
// launch latency of back-to-back calls overlaps the previous call's tail.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int G, int V, int MODE, int kFlags>
__global__ void __launch_bounds__(kOpBlock, op_min_blocks<G, V>()) op_kernel(OpArgs a) {
    pdl_enter();
    // each warp owns a contiguous slice of the batch, or (a.chunk != 0) takes
    // pieces of a.chunk operations in batch order from the ticket counter, so
    // that the whole grid moves through the batch together
    u64 n_ins = 0, n_del = 0;
    u32 sbits = 0;
    if (a.chunk == 0) {
        const u64 warp = (u64(blockIdx.x) * kOpBlock + threadIdx.x) >> 5;
        const u64 nwarps = (u64(gridDim.x) * kOpBlock) >> 5;
        const u64 per = (a.n + nwarps - 1) / nwarps;
        const u64 begin = warp * per;
        const u64 end = begin + per < a.n ? begin + per : a.n;
        warp_ops<G, V, MODE, false, false, kFlags>(a, begin, end, n_ins, n_del, sbits);
    } else {
        for (;;) {
            u64 piece = 0;
            if ((threadIdx.x & 31) == 0) piece = atomicAdd(a.ticket, 1ull);
            piece = __shfl_sync(0xffffffffu, piece, 0);
            const u64 begin = piece * a.chunk;
            if (begin >= a.n) break;
            const u64 end = begin + a.chunk < a.n ? begin + a.chunk : a.n;
            warp_ops<G, V, MODE, false, false, kFlags>(a, begin, end, n_ins, n_del, sbits);
        }
    }
    // (one atomic per warp: the CTA-level flush costs the 5-CTA window kernels
    // register spills, and these kernels serve the large batches)
    warp_flush_counters(a.st, n_ins, n_del, sbits);
}

// ---------------------------------------------------------------------------
// Per-thread operations (group_width = -1): the paper's own form, one thread
// per operation (Algorithm 1 and the find / erase / update probes of Sec. 3):
// each thread runs one operation at a time over a grid-stride sequence of the
// batch and probes V cells (one or two 32-byte sectors, aligned) per step;
// inserts claim the home cell with the 16-byte CAS first.  No group shuffles
// and no refill bookkeeping, so few instructions and registers per operation
// and more resident warps per SM -- for short probes (low load), where the
// lanes of a warp finish in about the same number of steps.  Tables without
// table options only (reuse_tombstones and full_key_space take the group
// loop); the next operation's key and value are loaded before the current
// one probes, and results are stored after the warp reconverges (coalesced).
// ---------------------------------------------------------------------------
constexpr int kThreadBlock = 256;

// One operation; returns its code and (find) the value found.
template <int V, int MODE>
__device__ __forceinline__ unsigned char thread_op(const OpArgs& a, u64 key, u64 d, u64 cap, u32 shift,
                                                   u64& n_ins, u64& n_del, u32& sbits, u64& vout) {
    constexpr bool kInsLike = mode_fills(MODE);
    constexpr bool kUpdate = MODE == kUpdAdd || MODE == kUpdOverwrite;
    const u64 cmask = cap - 1;
    vout = 0;
    if (is_reserved(key)) {
        sbits |= kReserved;
        return kCodeReserved;
    }
    u64 pos = home_of(key, shift);
    u64 probed = 0;
    if (MODE == kInsert) {
        Cell expect;
        expect.key = kEmpty;
        expect.val = 0;
        Cell desired;
        desired.key = key;
        desired.val = d;
        const Cell old = cas_cell(a.cells + pos, expect, desired);
        if (old.key == kEmpty && old.val == 0) {
            ++n_ins;
            return kYes;
        }
        if (old.key == key) return kNo;
        probed = 1;
        pos = (pos + 1) & cmask;
    }
    while (probed < cap) {
        const u64 base = pos & ~u64(V - 1);
        const u32 first = u32(pos - base);
        u64 kk[V], vv[V];
        const Cell* p = a.cells + base;
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            if (MODE == kFind) ld_pair_nc(p + j, kk[j], vv[j], kk[j + 1], vv[j + 1]);
            else ld_pair_cg(p + j, kk[j], vv[j], kk[j + 1], vv[j + 1]);
        }
        int hit = -1;
        bool match = false;
        u64 hv = 0;
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {  // the lowest qualifying cell wins
            if (u32(j) >= first && (kk[j] == key || kk[j] == kEmpty)) {
                hit = j;
                match = kk[j] == key;
                hv = vv[j];
            }
        }
        if (hit < 0) {
            probed += V - first;
            pos = (base + V) & cmask;
            continue;
        }
        if (MODE == kFind) {
            vout = match ? hv : 0;
            return match ? kYes : kNo;
        }
        const int out = modify_at<MODE>(a.cells + base + u32(hit), match, key, d);
        if (out != kStepContinue) {
            if (out == kStepDoneYes) {
                if (MODE == kErase) ++n_del;
                else if (kInsLike) ++n_ins;
            }
            return (unsigned char)out;
        }
        probed += u32(hit) - first + 1;
        pos = (base + u32(hit) + 1) & cmask;
    }
    // every cell was examined without a decision
    if (MODE == kFind || MODE == kErase || kUpdate) return kNo;
    sbits |= kFull;
    return kCodeFull;
}

template <int V, int MODE>
__global__ void __launch_bounds__(kThreadBlock) thread_kernel(OpArgs a) {
    constexpr bool kHasVals = mode_has_vals(MODE);
    pdl_enter();
    const u64 cap = 1ull << a.log2c;
    const u32 shift = 64u - a.log2c;
    u64 n_ins = 0, n_del = 0;
    u32 sbits = 0;
    const u64 stride = u64(gridDim.x) * kThreadBlock;
    u64 i = u64(blockIdx.x) * kThreadBlock + threadIdx.x;
    u64 key = 0, d = 0;
    if (i < a.n) {
        key = ld_stream(a.keys + i);
        if (kHasVals) d = ld_stream(a.vals + i);
    }
    // the lanes of a warp hold consecutive operations and step together (a
    // warp-uniform loop), so they meet at the stores
    for (;; i += stride) {
        const bool live = i < a.n;
        if (!__any_sync(0xffffffffu, live)) break;
        const u64 j = i + stride;
        u64 nk = 0, nd = 0;
        if (j < a.n) {
            nk = ld_stream(a.keys + j);
            if (kHasVals) nd = ld_stream(a.vals + j);
        }
        u64 v = 0;
        unsigned char c = 0;
        if (live) c = thread_op<V, MODE>(a, key, d, cap, shift, n_ins, n_del, sbits, v);
        __syncwarp();
        if (live) {
            if (MODE == kFind) a.vals_out[i] = v;
            if (a.codes) a.codes[i] = c;
        }
        key = nk;
        d = nd;
    }
    block_flush_counters(a.st, n_ins, n_del, sbits);
}

}  // namespace cht

namespace cht {

// ---------------------------------------------------------------------------
// insertOrUpdate with CTA-level aggregation in shared memory.
//
// A CTA takes windows of kAggWindow consecutive operations.  Equal keys of the
// window are folded into one slot of a shared-memory table (open addressing,
// kAggSlots >= 2 * kAggWindow slots, so every key finds a slot): the add
// operator sums the values (fetch-and-add on the slot), overwrite keeps the
// value of the slot's first operation.  The window is then flushed: one
// global insertOrUpdate per distinct key (Algorithm 1 with the specialised
// atomicUpdate), whose result -- inserted or updated -- goes to the slot's
// first operation; every other operation of the key reports "updated"
// (linearized right after it).  Under skewed keys this turns millions of
// atomics on one hot cell into one per window.  A warp may first combine the
// equal keys of its load step with __match_any_sync, which pays off only
// under extreme skew (many lanes on one shared-memory slot): DEDUP 2 always
// does, DEDUP 1 (insertOrUpdate's default) does it for a window when the
// CTA's previous window had fewer distinct keys than a fifth of its
// operations, DEDUP 0 (update) never.
// ---------------------------------------------------------------------------
constexpr int kAggBlock = 256;
constexpr int kAggWindow = 1024;
constexpr int kAggSlots = 2048;

// One operation on the global table by one thread (sector-wise probe).
template <int MODE, bool kReuse>
__device__ __forceinline__ unsigned char global_modify(const OpArgs& a, u64 key, u64 d, u64 cap, u32 shift,
                                                       u64& n_ins, u64& n_reused, u32& sbits,
                                                       u64 pos = kNoPos, u64 probed = 0) {
    const u64 cmask = cap - 1;
    if (pos == kNoPos) pos = home_of(key, shift);
    u64 tpos = kNoPos, tprobed = 0;  // tombstone reuse (a.reuse): first one on the path
    for (;;) {
        while (probed < cap) {
            const u64 base = pos & ~1ull;
            const u32 first = u32(pos - base);
            u64 k0, v0, k1, v1;
            ld_pair_cg(a.cells + base, k0, v0, k1, v1);
            int hit = -1;
            bool match = false;
            if (first == 0 && (k0 == key || k0 == kEmpty)) {
                hit = 0;
                match = k0 == key;
            } else if (k1 == key || k1 == kEmpty) {
                hit = 1;
                match = k1 == key;
            }
            if (kReuse && tpos == kNoPos) {  // first tombstone before the deciding cell
                if (first == 0 && k0 == kTomb) {
                    tpos = base & cmask;
                    tprobed = probed + 1;
                } else if (k1 == kTomb && hit < 0) {
                    tpos = (base + 1) & cmask;
                    tprobed = probed + 2 - first;
                }
            }
            if (hit < 0) {
                probed += 2 - first;
                pos = (base + 2) & cmask;
                continue;
            }
            const int out = (!match && tpos != kNoPos) ? claim_tomb<MODE>(a.cells + tpos, key, d)
                                                       : modify_at<MODE>(a.cells + base + hit, match, key, d);
            if (out == kStepContinue) {
                probed += u32(hit) - first + 1;
                pos = (base + u32(hit) + 1) & cmask;
                continue;
            }
            if (out == kStepRestart) {
                pos = (tpos + 1) & cmask;
                probed = tprobed;
                tpos = kNoPos;
                continue;
            }
            if (out == kStepDoneYes && mode_fills(MODE)) ++n_ins;
            if (out == kStepDoneReused) {
                ++n_reused;
                return kYes;
            }
            return (unsigned char)out;
        }
        if (tpos == kNoPos) break;
        // every cell seen, no empty one and no key: take the tombstone (only
        // insert modes record one)
        const int out = claim_tomb<MODE>(a.cells + tpos, key, d);
        if (out == kStepRestart) {
            pos = (tpos + 1) & cmask;
            probed = tprobed;
            tpos = kNoPos;
            continue;
        }
        if (out == kStepDoneReused) {
            ++n_reused;
            return kYes;
        }
        return (unsigned char)out;
    }
    if (!mode_fills(MODE)) return kNo;  // update: every cell seen, the key is absent
    sbits |= kFull;
    return kCodeFull;
}

// Shared memory of the aggregation kernel: slot keys, values and first ops;
// for update modes also each operation's slot and each slot's result (every
// operation on a key reports whether the key was present).
// BLOCK threads per CTA, windows of 4 * BLOCK operations, 8 * BLOCK slots:
// 256 (the default) or 1024 (hash-sorted batches, whose key groups span whole
// buckets of the sort).
template <int MODE, int BLOCK = kAggBlock>
constexpr size_t agg_smem_bytes() {
    return size_t(8 * BLOCK) * (8 + 8 + 2) + size_t(4 * BLOCK) * 2 +
           ((MODE == kUpdAdd || MODE == kUpdOverwrite) ? size_t(4 * BLOCK) * 2 + 8 * BLOCK : 0);
}

// The flush of one window's distinct keys, kAggWindow / kAggBlock at most per
// thread, with the memory accesses of all of a thread's keys in flight at
// once: first every key's home sector is loaded, then every key whose sector
// decides it issues its atomic (the CAS into the empty cell, or the update of
// its cell), and only the few keys that need more -- a sector without a
// deciding cell, a CAS lost to another key -- continue one by one with the
// sector-wise probe from where they stopped.  Same results as probing each key
// on its own (Algorithm 1 per key; the keys are distinct).
template <int MODE>
__device__ __forceinline__ void flush_keys(const OpArgs& a, const u64* fk, const u64* fd, const bool* fv,
                                           unsigned char* res, u64 cap, u32 shift, u64& n_ins, u64& n_reused,
                                           u32& sbits) {
    constexpr int R = kAggWindow / kAggBlock;
    constexpr bool kUpdate = MODE == kUpdAdd || MODE == kUpdOverwrite;
    const u64 cmask = cap - 1;
    u64 pos[R], k0[R], v0[R], k1[R], v1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        k0[r] = v0[r] = k1[r] = v1[r] = 0;
        pos[r] = 0;
        if (fv[r]) {
            pos[r] = home_of(fk[r], shift);
            ld_pair_cg(a.cells + (pos[r] & ~1ull), k0[r], v0[r], k1[r], v1[r]);
        }
    }
    // 0 done, 1 CAS issued, 2 probe on from pos[r]
    int st[R];
    Cell old[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        st[r] = 0;
        old[r].key = old[r].val = 0;
        if (!fv[r]) continue;
        const u64 key = fk[r];
        const u64 base = pos[r] & ~1ull;
        int hit = -1;
        bool match = false;
        if ((pos[r] & 1ull) == 0 && (k0[r] == key || k0[r] == kEmpty)) {
            hit = 0;
            match = k0[r] == key;
        } else if (k1[r] == key || k1[r] == kEmpty) {
            hit = 1;
            match = k1[r] == key;
        }
        if (hit < 0) {
            st[r] = 2;
            pos[r] = (base + 2) & cmask;
            continue;
        }
        Cell* cp = a.cells + base + hit;
        if (match) {
            if (MODE == kIouAdd || MODE == kUpdAdd) atomicAdd(&cp->val, fd[r]);
            else atomicExch(&cp->val, fd[r]);
            res[r] = kUpdate ? kYes : kNo;
        } else if (kUpdate) {
            res[r] = kNo;  // an empty cell before the key: absent
        } else {
            Cell expect;
            expect.key = kEmpty;
            expect.val = 0;
            Cell desired;
            desired.key = key;
            desired.val = fd[r];
            old[r] = cas_cell(cp, expect, desired);
            st[r] = 1;
            pos[r] = base + hit;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (st[r] != 1) continue;
        if (old[r].key == kEmpty && old[r].val == 0) {
            ++n_ins;
            res[r] = kYes;
            st[r] = 0;
        } else if (old[r].key == fk[r]) {  // another copy of the key won the cell: update it
            Cell* cp = a.cells + pos[r];
            if (MODE == kIouAdd) atomicAdd(&cp->val, fd[r]);
            else atomicExch(&cp->val, fd[r]);
            res[r] = kNo;
            st[r] = 0;
        } else {
            st[r] = 2;
            pos[r] = (pos[r] + 1) & cmask;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (st[r] != 2) continue;
        const u64 probed = (pos[r] - home_of(fk[r], shift)) & cmask;
        res[r] = global_modify<MODE, false>(a, fk[r], fd[r], cap, shift, n_ins, n_reused, sbits, pos[r],
                                            probed == 0 ? cap : probed);
    }
}

template <int MODE, int DEDUP, bool kReuse, int BLOCK = kAggBlock>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) iou_agg_kernel(OpArgs a) {
    constexpr int kB = BLOCK, kW = 4 * BLOCK, kS = 8 * BLOCK;
    pdl_enter();
    constexpr bool kUpdate = MODE == kUpdAdd || MODE == kUpdOverwrite;
    constexpr bool kAdd = MODE == kIouAdd || MODE == kUpdAdd;
    extern __shared__ __align__(16) unsigned char agg_smem[];
    u64* const skey = reinterpret_cast<u64*>(agg_smem);
    u64* const sval = skey + kS;
    // window offset of the slot's first op (< kW: 16 bits)
    unsigned short* const slead = reinterpret_cast<unsigned short*>(sval + kS);
    unsigned short* const slist = slead + kS;  // the window's claimed slots
    unsigned short* const sslot = slist + kW;                                   // update: op -> slot
    unsigned char* const sres = reinterpret_cast<unsigned char*>(sslot + kW);   // update: slot result
    const u64 cap = 1ull << a.log2c;
    const u32 shift = 64u - a.log2c;
    const int tid = threadIdx.x;
    u64 n_ins = 0, n_reused = 0;
    u32 sbits = 0;
    __shared__ u32 s_distinct[2];  // distinct keys (claimed slots) of this CTA's window, by window parity
    __shared__ unsigned long long s_wsum[kB];  // warp pre-reduction: per lane, its group's sum
    s_wsum[tid] = 0;
    for (int s = tid; s < kS; s += kB) {
        skey[s] = kEmpty;
        sval[s] = 0;
    }
    if (tid < 2) s_distinct[tid] = 0;
    __syncthreads();
    bool dedup = DEDUP == 2;
    const u64 nwin = (a.n + kW - 1) / kW;
    // windows: blockIdx.x, + gridDim.x, ... or, with a ticket counter, the
    // next window in batch order (every window already ends in a barrier,
    // which publishes the next ticket to the block)
    __shared__ u64 s_next[2];
    u64 w = blockIdx.x;
    if (a.ticket) {
        if (tid == 0) s_next[0] = atomicAdd(a.ticket, 1ull);
        __syncthreads();
        w = s_next[0];
    }
    for (u32 round = 0; w < nwin; ++round) {
        const u64 w0 = w * kW;
        const int par = int(round & 1);
        if (a.ticket && tid == 0) s_next[(round + 1) & 1] = atomicAdd(a.ticket, 1ull);
        // this thread's operations of the window, all loads issued before any
        // is used (the loads are volatile asm, which the compiler keeps in
        // program order: interleaved with the folding below they would cost one
        // memory round trip each)
        constexpr int kPer = kW / kB;
        u64 wk[kPer], wv[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const u64 idx = w0 + u32(j * kB + tid);
            wk[j] = idx < a.n ? ld_stream(a.keys + idx) : 0;
            wv[j] = idx < a.n ? ld_stream(a.vals + idx) : 0;
        }
        // fold the window's operations into the slots
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const u32 off = u32(j * kB + tid);
            const u64 idx = w0 + off;
            bool valid = idx < a.n;
            u64 key = 0, d = 0;
            if (kUpdate) sslot[off] = 0xffffu;
            if (valid) {
                key = wk[j];
                d = wv[j];
                if (is_reserved(key)) {
                    if (a.full_keys) {
                        const unsigned char r = special_op<MODE>(a.st, key, d, nullptr);
                        if (a.codes) a.codes[idx] = r;
                    } else {
                        if (a.codes) a.codes[idx] = kCodeReserved;
                        sbits |= kReserved;
                    }
                    valid = false;
                }
            }
            // optionally, equal keys within the warp first: one lane per key goes
            // on (dedup is the same for the whole block)
            const u32 vm = dedup ? __ballot_sync(0xffffffffu, valid) : 0u;
            if (dedup && valid) {
                const u32 same = __match_any_sync(vm, key);
                const int lane = tid & 31;
                if (kAdd) {
                    // the group's sum: every lane adds its value into its
                    // leader's word of a warp-private scratch (a few cycles of
                    // shared-memory atomics instead of a shuffle round per
                    // member), the leader takes it and clears the word
                    const int lead = __ffs(same) - 1;
                    unsigned long long* const ws = s_wsum + (tid & ~31);
                    atomicAdd(ws + lead, d);
                    __syncwarp(vm);
                    if (lane == lead) {
                        d = ws[lead];
                        ws[lead] = 0;
                    }
                    __syncwarp(vm);
                }
                if (lane != __ffs(same) - 1) {
                    if (a.codes) a.codes[idx] = kNo;
                    valid = false;
                }
            }
            if (!valid) continue;
            u32 s = u32(fmix64(key)) & (kS - 1);
            for (;;) {
                const u64 k0 = *reinterpret_cast<volatile u64*>(skey + s);
                bool mine = false, same = k0 == key;
                if (k0 == kEmpty) {
                    const u64 old = atomicCAS(reinterpret_cast<unsigned long long*>(skey + s), kEmpty, key);
                    mine = old == kEmpty;
                    same = old == key;
                }
                if (mine) {
                    if (kAdd) atomicAdd(reinterpret_cast<unsigned long long*>(sval + s), d);
                    else sval[s] = d;
                    slead[s] = (unsigned short)off;
                    if (kUpdate) sslot[off] = (unsigned short)s;
                    slist[atomicAdd(&s_distinct[par], 1u)] = (unsigned short)s;
                    break;
                }
                if (same) {
                    if (kAdd) atomicAdd(reinterpret_cast<unsigned long long*>(sval + s), d);
                    if (kUpdate) sslot[off] = (unsigned short)s;
                    else if (a.codes) a.codes[idx] = kNo;
                    break;
                }
                s = (s + 1) & (kS - 1);
            }
        }
        __syncthreads();
        if (DEDUP == 1) {
            // the next window of this CTA combines within warps if this one had
            // few distinct keys
            const u64 ops = a.n - w0 < u64(kW) ? a.n - w0 : u64(kW);
            dedup = u64(s_distinct[par]) * 2 < ops;
        }
        if (tid == 0) s_distinct[par ^ 1] = 0;  // the next window's counter (read by all before it)
        // flush: one global operation per distinct key of the window (the
        // dense list of claimed slots; at most kW / kB per thread)
        const u32 nd = s_distinct[par];
        if (kReuse) {  // tombstone reuse tracks the first tombstone of each path: one key at a time
            for (u32 j = tid; j < nd; j += kB) {
                const u32 sl = slist[j];
                const unsigned char r =
                    global_modify<MODE, kReuse>(a, skey[sl], sval[sl], cap, shift, n_ins, n_reused, sbits);
                if (kUpdate) sres[sl] = r;
                else if (a.codes) a.codes[w0 + slead[sl]] = r;
                skey[sl] = kEmpty;
                sval[sl] = 0;
            }
        } else {
            constexpr int R = kW / kB;
            u64 fk[R], fd[R];
            bool fv[R];
            u32 fs[R];
            unsigned char res[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const u32 j = u32(tid + r * kB);
                fv[r] = j < nd;
                fs[r] = fv[r] ? slist[j] : 0u;
                fk[r] = fv[r] ? skey[fs[r]] : 0;
                fd[r] = fv[r] ? sval[fs[r]] : 0;
                res[r] = kNo;
            }
            flush_keys<MODE>(a, fk, fd, fv, res, cap, shift, n_ins, n_reused, sbits);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!fv[r]) continue;
                if (kUpdate) sres[fs[r]] = res[r];
                else if (a.codes) a.codes[w0 + slead[fs[r]]] = res[r];
                skey[fs[r]] = kEmpty;
                sval[fs[r]] = 0;
            }
        }
        __syncthreads();
        if (kUpdate && a.codes) {  // every operation takes its key's result
            for (int off = tid; off < kW; off += kB) {
                const unsigned short sl = sslot[off];
                if (sl != 0xffffu) a.codes[w0 + off] = sres[sl];
            }
            __syncthreads();
        }
        w = a.ticket ? s_next[(round + 1) & 1] : w + gridDim.x;
    }
    constexpr u32 FULL = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
        n_ins += __shfl_xor_sync(FULL, n_ins, o);
        n_reused += __shfl_xor_sync(FULL, n_reused, o);
    }
    const u32 any_status = __reduce_or_sync(FULL, sbits);
    if ((tid & 31) == 0) {
        if (n_ins) atomicAdd(&a.st->I, n_ins);
        if (n_reused) atomicAdd(&a.st->D, 0ull - n_reused);  // reused tombstones: D falls
        if (any_status) atomicOr(&a.st->status, any_status);
    }
}

}  // namespace cht
