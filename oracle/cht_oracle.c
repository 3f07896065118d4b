/*
 * Oracle for the folklore linear-probing hash table of Maier, Sanders and
 * Dementiev, "Concurrent Hash Tables: Fast and General(?)!" (arXiv 1601.04017).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
 * restatement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library, and it never reads a
 * value produced by the CUDA library except through an explicit snapshot that
 * a test hands it (or_load_cells) in order to migrate that snapshot itself.
 *
 * Semantics ("phase semantics"): every call processes a batch of ONE operation
 * type, strictly in input order, one operation at a time.  That sequential
 * order is one valid linearization of a concurrent batch (Sec. 3,
 * linearizability); where a concurrent batch may legitimately end differently
 * (duplicate keys inside one insert / overwrite / erase batch) the tests
 * compare set-valued, not against this particular order.
 *
 * Cell layout: <key, value>, both 64-bit; key 0 marks an empty cell, key ~0 a
 * tombstone (Sec. 3 "Deletions", Sec. 4.4).  Capacity is a power of two
 * (Sec. 6 "Bounded Hash Tables"); the home cell of key x is the top log2(c)
 * bits of the 64-bit hash, i.e. floor(h(x) * c / 2^64) (Sec. 4.3.1, scaling
 * map h_c).
 *
 * Per-operation result codes: 0 = no (already present / absent / not erased),
 * 1 = yes (inserted / found / erased), 2 = table full (probed every cell),
 * 3 = reserved key (0 or ~0; the table is not touched).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define OR_EMPTY 0ull
#define OR_TOMB (~0ull)
#define OR_MIN_CAP 64ull

enum { OR_NO = 0, OR_YES = 1, OR_FULL = 2, OR_RESERVED = 3 };
enum { OR_OVERWRITE = 0, OR_ADD = 1 };

typedef struct {
    uint64_t key;
    uint64_t val;
} or_cell;

typedef struct {
    uint64_t cap;      /* c, a power of two */
    unsigned log2c;
    or_cell *cells;
    uint64_t I;        /* non-empty cells, tombstones included (Sec. 4.4) */
    uint64_t D;        /* tombstones (Sec. 4.2 deletion counter) */
    int growable;      /* migrate automatically when I would exceed alpha*c */
    double alpha;      /* fill threshold for growth (Sec. 4.3.2) */
    uint64_t probes;   /* cells inspected by all operations so far (statistics) */
    uint64_t migrations;
    int reuse_tombstones; /* inserts may take the first tombstone on their path */
    int full_keys;        /* keys 0 and ~0 live in two special slots (Sec. 5) */
    int sp_present[2];    /* special slot 0: key 0, slot 1: key ~0 */
    uint64_t sp_val[2];
} or_table;

/* 64-bit finalizer of MurmurHash3 (Appleby, public domain): the paper hashes
 * with two CRC32C instructions (Sec. 7.3); any good 64-bit mixer serves, and
 * results do not depend on the choice. */
uint64_t or_hash(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

/* Scaling map h_c(x) = floor(h(x) * c / U) with U = 2^64 and c = 2^log2c
 * (Sec. 4.3.1): a right shift keeps the top log2c bits. */
static uint64_t home_of(uint64_t key, unsigned log2c)
{
    return or_hash(key) >> (64 - log2c);
}

uint64_t or_home(const or_table *t, uint64_t key) { return home_of(key, t->log2c); }

/* Batch forms of the hash and of the home map for an arbitrary log2(c). */
void or_hash_many(const uint64_t *keys, uint64_t n, uint64_t *out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = or_hash(keys[j]);
}

void or_home_many(const uint64_t *keys, uint64_t n, unsigned log2c, uint64_t *out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = home_of(keys[j], log2c);
}

/* Smallest power of two >= max(x, 64) (Sec. 6 restricts c to powers of two). */
static uint64_t round_cap(uint64_t x, unsigned *log2c)
{
    uint64_t c = OR_MIN_CAP;
    unsigned l = 6;
    while (c < x) {
        c <<= 1;
        ++l;
    }
    *log2c = l;
    return c;
}

or_table *or_create(uint64_t capacity, int growable, double alpha)
{
    or_table *t = (or_table *)calloc(1, sizeof(or_table));
    if (!t) return NULL;
    if (capacity > (1ull << 40)) { free(t); return NULL; }
    t->cap = round_cap(capacity, &t->log2c);
    /* Initialization: every key starts as the empty key (Sec. 3). */
    t->cells = (or_cell *)calloc(t->cap, sizeof(or_cell));
    if (!t->cells) { free(t); return NULL; }
    t->growable = growable;
    t->alpha = alpha;
    return t;
}

void or_destroy(or_table *t)
{
    if (!t) return;
    free(t->cells);
    free(t);
}

/* Tombstone reuse (off by default, which is the paper's rule: a deleted cell
 * is never used again, Sec. 3 "Deletions").  Under phase semantics no erase
 * runs while an insert batch does, so an insert that finds its key absent may
 * put it into the first tombstone on its probe path instead of the first
 * empty cell: the cell stays non-empty (I unchanged, D - 1), every key stays
 * reachable from its home, and every result is the same as without reuse. */
void or_set_reuse(or_table *t, int on) { t->reuse_tombstones = on; }

/* Full key space (off by default: keys 0 and ~0 are reserved and rejected
 * with code 3).  The paper keeps the empty and deleted markers out of the
 * key space and notes they could be stored separately; on, the two keys
 * live in two slots beside the table, outside every probe, and behave like
 * any other key: insert / insertOrUpdate / update / find / erase apply the
 * dictionary meaning to the slot; migrations leave the slots alone. */
void or_set_full_keys(or_table *t, int on) { t->full_keys = on; }

enum { SP_FIND = 0, SP_INSERT = 1, SP_IOU = 2, SP_ERASE = 3, SP_UPDATE = 4 };

static int special_op(or_table *t, uint64_t k, uint64_t d, int kind, int op, uint64_t *vout)
{
    const int s = k == OR_TOMB;
    const int was = t->sp_present[s];
    switch (kind) {
    case SP_FIND:
        if (vout) *vout = was ? t->sp_val[s] : 0;
        return was ? OR_YES : OR_NO;
    case SP_INSERT:
        if (was) return OR_NO;
        t->sp_present[s] = 1;
        t->sp_val[s] = d;
        return OR_YES;
    case SP_IOU:
        if (!was) {
            t->sp_present[s] = 1;
            t->sp_val[s] = d;
            return OR_YES;
        }
        t->sp_val[s] = (op == OR_ADD) ? t->sp_val[s] + d : d;
        return OR_NO;
    case SP_UPDATE:
        if (!was) return OR_NO;
        t->sp_val[s] = (op == OR_ADD) ? t->sp_val[s] + d : d;
        return OR_YES;
    default: /* SP_ERASE */
        if (!was) return OR_NO;
        t->sp_present[s] = 0;
        t->sp_val[s] = 0;
        return OR_YES;
    }
}

uint64_t or_capacity(const or_table *t) { return t->cap; }
uint64_t or_nonempty(const or_table *t) { return t->I; }
uint64_t or_live(const or_table *t) { return t->I - t->D + t->sp_present[0] + t->sp_present[1]; }
uint64_t or_probes(const or_table *t) { return t->probes; }
uint64_t or_migrations(const or_table *t) { return t->migrations; }
void or_reset_probes(or_table *t) { t->probes = 0; }

static int is_reserved(uint64_t k) { return k == OR_EMPTY || k == OR_TOMB; }

/* A cluster start is a non-empty cell whose predecessor (cyclically) is empty
 * (Lemma 1's definition of a cluster a..b with a-1 and b+1 empty). Returns c
 * if the table has no empty cell or no non-empty cell. */
static uint64_t first_cluster_start(const or_table *t)
{
    uint64_t mask = t->cap - 1;
    for (uint64_t i = 0; i < t->cap; ++i) {
        if (t->cells[i].key != OR_EMPTY && t->cells[(i - 1) & mask].key == OR_EMPTY)
            return i;
    }
    return t->cap;
}

/* Sequential migration into a new table of new_cap cells (Sec. 4.3.1): visit
 * the old cells in index order, beginning at a cluster start, and insert every
 * live element (tombstones are dropped, Sec. 4.4) by plain linear probing
 * into the initially empty target.  Lemma 1 says the parallel cluster-wise
 * migration ends in exactly this layout when new_cap = gamma * c, gamma >= 1.
 * If the old table has no empty cell at all there is no cluster start and the
 * walk begins at index 0.  Returns 0 on success, -1 if new_cap cannot hold the
 * live elements or memory runs out. */
int or_migrate(or_table *t, uint64_t new_cap)
{
    unsigned nl;
    uint64_t nc = round_cap(new_cap, &nl);
    uint64_t live = t->I - t->D;
    if (nc < live) return -1;
    or_cell *dst = (or_cell *)calloc(nc, sizeof(or_cell));
    if (!dst) return -1;
    uint64_t omask = t->cap - 1, nmask = nc - 1;
    uint64_t start = first_cluster_start(t);
    if (start == t->cap) start = 0;
    uint64_t moved = 0;
    for (uint64_t j = 0; j < t->cap; ++j) {
        const or_cell *s = &t->cells[(start + j) & omask];
        if (s->key == OR_EMPTY || s->key == OR_TOMB) continue;
        uint64_t p = home_of(s->key, nl);
        while (dst[p].key != OR_EMPTY) p = (p + 1) & nmask;
        dst[p] = *s;
        ++moved;
    }
    free(t->cells);
    t->cells = dst;
    t->cap = nc;
    t->log2c = nl;
    t->I = moved;  /* the migration re-seeds I; D restarts at 0 (Sec. 4.2) */
    t->D = 0;
    t->migrations++;
    return 0;
}

/* Growth trigger (Sec. 4.3.2, Sec. 4.4): before an operation that may occupy
 * a new cell, if I + 1 would exceed floor(alpha * c), migrate first.  The
 * live count I - D chooses the target size: double (gamma = 2) when more than
 * alpha*c/2 elements are live, otherwise the same size (gamma = 1), which
 * only purges tombstones. */
static void grow_if_needed(or_table *t)
{
    if (!t->growable) return;
    uint64_t limit = (uint64_t)(t->alpha * (double)t->cap);
    if (t->I + 1 <= limit) return;
    uint64_t live = t->I - t->D;
    uint64_t half = (uint64_t)(t->alpha * (double)t->cap / 2.0);
    uint64_t nc = live > half ? 2 * t->cap : t->cap;
    or_migrate(t, nc);
}

/* insertOrUpdate (Algorithm 1), sequential: probe from the home cell; at the
 * first empty cell store <k, d> and report an insertion; at a cell holding k
 * apply the update and report an update.  Tombstones are passed over like any
 * other non-empty cell and never reused (Sec. 3 "Deletions") -- unless reuse
 * is on: then the key goes into the first tombstone the probe passed, once
 * the probe has shown the key absent (an empty cell, or all c cells seen).
 * Mode 0 is the plain insert of Sec. 3 (a present key is left untouched). */
static int or_modify1(or_table *t, uint64_t k, uint64_t d, int mode, int op)
{
    if (is_reserved(k)) return t->full_keys ? special_op(t, k, d, mode == 1 ? SP_IOU : SP_INSERT, op, NULL) : OR_RESERVED;
    grow_if_needed(t);
    uint64_t mask = t->cap - 1;
    uint64_t i = home_of(k, t->log2c);
    or_cell *tomb = NULL;
    for (uint64_t step = 0; step < t->cap; ++step, i = (i + 1) & mask) {
        or_cell *c = &t->cells[i];
        t->probes++;
        if (c->key == OR_EMPTY) {
            if (tomb) {
                tomb->key = k;
                tomb->val = d;
                t->D--;
                return OR_YES;
            }
            c->key = k;
            c->val = d;
            t->I++;
            return OR_YES;
        }
        if (c->key == k) {
            if (mode == 1) c->val = (op == OR_ADD) ? c->val + d : d;
            return OR_NO;
        }
        if (c->key == OR_TOMB && t->reuse_tombstones && !tomb) tomb = c;
    }
    if (tomb) {  /* no empty cell anywhere, the key is absent */
        tomb->key = k;
        tomb->val = d;
        t->D--;
        return OR_YES;
    }
    return OR_FULL;
}

void or_insert(or_table *t, const uint64_t *keys, const uint64_t *vals, uint64_t n, uint8_t *flags)
{
    for (uint64_t j = 0; j < n; ++j) {
        int r = or_modify1(t, keys[j], vals[j], 0, 0);
        if (flags) flags[j] = (uint8_t)r;
    }
}

void or_insert_or_update(or_table *t, const uint64_t *keys, const uint64_t *vals, uint64_t n,
                         int op, uint8_t *flags)
{
    for (uint64_t j = 0; j < n; ++j) {
        int r = or_modify1(t, keys[j], vals[j], 1, op);
        if (flags) flags[j] = (uint8_t)r;
    }
}

/* Sort-based bulk build (Sec. 3 "Bulk Operations"): building a table from a
 * batch of n elements by sorting them by hash.  Reading taken here (the
 * paper's text stops mid-sentence):
 *   - the table must be empty (returns -1 otherwise); a growable table first
 *     grows, empty, to the smallest power of two c' >= c with n <= floor(alpha
 *     c'), since n bounds the number of distinct keys (Sec. 3: grow to an
 *     upper bound of the new size first);
 *   - the elements are ordered by the top B bits of their hash, B = 32 for
 *     tables of up to 2^32 cells (else log2(c) rounded up to a multiple of 8),
 *     ties in input order; B >= log2(c), so the order is also by home cell;
 *   - among equal keys all but the last (in input order) are dropped (Sec. 3:
 *     keep the last);
 *   - the survivors are inserted one by one in that order, each at the first
 *     empty cell from its home on (wrapping past the last cell); a sorted
 *     insertion's free cell search can start at max(home, previous position),
 *     which is what the paper's merge does;
 *   - keys 0 and ~0 go to the special slots (last value wins) with the full
 *     key space on, else they are skipped and the result is 1;
 *   - if the survivors would leave no empty cell (a bounded table), nothing
 *     is changed and the result is -2.
 * Returns 0 on success, 1 on success with reserved keys skipped. */
typedef struct {
    uint64_t s;   /* top B hash bits */
    uint64_t idx; /* input position */
} or_sortkey;

static int cmp_sortkey(const void *a, const void *b)
{
    const or_sortkey *x = (const or_sortkey *)a, *y = (const or_sortkey *)b;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

unsigned or_build_sort_bits(unsigned log2c) { return log2c <= 32 ? 32u : 8u * ((log2c + 7u) / 8u); }

int or_build(or_table *t, const uint64_t *keys, const uint64_t *vals, uint64_t n)
{
    if (t->I != 0 || t->sp_present[0] || t->sp_present[1]) return -1;
    if (t->growable) {
        uint64_t nc = t->cap;
        while (n > (uint64_t)(t->alpha * (double)nc)) nc <<= 1;
        if (nc != t->cap) {
            or_cell *cells = (or_cell *)calloc(nc, sizeof(or_cell));
            if (!cells) return -1;
            free(t->cells);
            t->cells = cells;
            t->cap = round_cap(nc, &t->log2c);
        }
    }
    const unsigned B = or_build_sort_bits(t->log2c);
    or_sortkey *v = (or_sortkey *)malloc((n ? n : 1) * sizeof(or_sortkey));
    if (!v) return -1;
    uint64_t m = 0;
    int reserved = 0, sp_set[2] = {0, 0};
    uint64_t sp_v[2] = {0, 0};
    for (uint64_t i = 0; i < n; ++i) {
        if (is_reserved(keys[i])) {
            const int sl = keys[i] == OR_TOMB;
            if (t->full_keys) {
                sp_set[sl] = 1;
                sp_v[sl] = vals[i];
            } else {
                reserved = 1;
            }
            continue;
        }
        v[m].s = or_hash(keys[i]) >> (64 - B);
        v[m].idx = i;
        ++m;
    }
    qsort(v, m, sizeof(or_sortkey), cmp_sortkey);
    /* keep the last of equal keys: equal keys have equal hashes, so a later
     * copy of v[a]'s key lies in v[a]'s run of equal sort keys */
    uint64_t S = 0;
    for (uint64_t a = 0; a < m; ++a) {
        int later = 0;
        for (uint64_t b = a + 1; b < m && v[b].s == v[a].s && !later; ++b)
            later = keys[v[b].idx] == keys[v[a].idx];
        if (!later) v[S++] = v[a];
    }
    if (S >= t->cap) {
        free(v);
        return -2;
    }
    const uint64_t mask = t->cap - 1;
    for (uint64_t j = 0; j < S; ++j) {
        const uint64_t k = keys[v[j].idx];
        uint64_t p = home_of(k, t->log2c);
        while (t->cells[p].key != OR_EMPTY) {
            t->probes++;
            p = (p + 1) & mask;
        }
        t->cells[p].key = k;
        t->cells[p].val = vals[v[j].idx];
    }
    t->I = S;
    t->D = 0;
    for (int sl = 0; sl < 2; ++sl)
        if (sp_set[sl]) {
            t->sp_present[sl] = 1;
            t->sp_val[sl] = sp_v[sl];
        }
    free(v);
    return reserved;
}

/* update (Sec. 3 interface: update(x, d, up)): probe from home like find; at
 * the cell holding k set value <- up(value, d) (overwrite: d; add: value + d
 * mod 2^64) and report 1; reaching an empty cell (or seeing every cell)
 * means k is absent: report 0 and change nothing.  Never fills a cell. */
void or_update(or_table *t, const uint64_t *keys, const uint64_t *vals, uint64_t n, int op, uint8_t *flags)
{
    uint64_t mask = t->cap - 1;
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t k = keys[j];
        int r = OR_NO;
        if (is_reserved(k)) {
            r = t->full_keys ? special_op(t, k, vals[j], SP_UPDATE, op, NULL) : OR_RESERVED;
        } else {
            uint64_t i = home_of(k, t->log2c);
            for (uint64_t step = 0; step < t->cap; ++step, i = (i + 1) & mask) {
                or_cell *c = &t->cells[i];
                t->probes++;
                if (c->key == OR_EMPTY) break;
                if (c->key == k) {
                    c->val = (op == OR_ADD) ? c->val + vals[j] : vals[j];
                    r = OR_YES;
                    break;
                }
            }
        }
        if (flags) flags[j] = (uint8_t)r;
    }
}

/* find (Sec. 3 "Lookup"): probe from home until the key (hit, copy of the
 * value) or an empty cell (miss; value 0).  Writes nothing to the table. */
void or_find(or_table *t, const uint64_t *keys, uint64_t n, uint64_t *vals_out, uint8_t *flags)
{
    uint64_t mask = t->cap - 1;
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t k = keys[j];
        int r = OR_NO;
        uint64_t v = 0;
        if (is_reserved(k)) {
            r = t->full_keys ? special_op(t, k, 0, SP_FIND, 0, &v) : OR_RESERVED;
        } else {
            uint64_t i = home_of(k, t->log2c);
            for (uint64_t step = 0; step < t->cap; ++step, i = (i + 1) & mask) {
                const or_cell *c = &t->cells[i];
                t->probes++;
                if (c->key == k) { r = OR_YES; v = c->val; break; }
                if (c->key == OR_EMPTY) break;
            }
        }
        if (vals_out) vals_out[j] = v;
        if (flags) flags[j] = (uint8_t)r;
    }
}

/* erase (Sec. 4.4): replace the key of the cell holding k by the tombstone
 * key, value untouched.  I is unchanged (the cell stays non-empty); D grows. */
void or_erase(or_table *t, const uint64_t *keys, uint64_t n, uint8_t *flags)
{
    uint64_t mask = t->cap - 1;
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t k = keys[j];
        int r = OR_NO;
        if (is_reserved(k)) {
            r = t->full_keys ? special_op(t, k, 0, SP_ERASE, 0, NULL) : OR_RESERVED;
        } else {
            uint64_t i = home_of(k, t->log2c);
            for (uint64_t step = 0; step < t->cap; ++step, i = (i + 1) & mask) {
                or_cell *c = &t->cells[i];
                t->probes++;
                if (c->key == k) { c->key = OR_TOMB; t->D++; r = OR_YES; break; }
                if (c->key == OR_EMPTY) break;
            }
        }
        if (flags) flags[j] = (uint8_t)r;
    }
}

/* forall (Sec. 3 "Bulk Operations"): the live elements in cell order. Returns
 * how many were written (at most max_n). */
static uint64_t export_cells(const or_table *t, uint64_t *keys, uint64_t *vals, uint64_t max_n)
{
    uint64_t m = 0;
    for (uint64_t i = 0; i < t->cap; ++i) {
        const or_cell *c = &t->cells[i];
        if (c->key == OR_EMPTY || c->key == OR_TOMB) continue;
        if (m < max_n) {
            if (keys) keys[m] = c->key;
            if (vals) vals[m] = c->val;
        }
        ++m;
    }
    return m;
}

/* forall (Sec. 3): every live element, the table's cells first, then the
 * special slots' keys (0, then ~0) when present. */
uint64_t or_export(const or_table *t, uint64_t *keys, uint64_t *vals, uint64_t max_n)
{
    uint64_t m = export_cells(t, keys, vals, max_n);
    for (int s = 0; s < 2; ++s) {
        if (!t->sp_present[s]) continue;
        if (m < max_n) {
            if (keys) keys[m] = s ? OR_TOMB : OR_EMPTY;
            if (vals) vals[m] = t->sp_val[s];
        }
        ++m;
    }
    return m;
}

/* Raw cell array as 2*c words (key, value, key, value, ...). */
void or_dump_cells(const or_table *t, uint64_t *out)
{
    memcpy(out, t->cells, t->cap * sizeof(or_cell));
}

/* Replace the contents by a snapshot of c cells (c must be a power of two
 * >= 64).  I and D are recomputed from the cells.  Returns 0 or -1. */
int or_load_cells(or_table *t, const uint64_t *cells, uint64_t c)
{
    unsigned l;
    if (c != round_cap(c, &l)) return -1;
    or_cell *nc = (or_cell *)malloc(c * sizeof(or_cell));
    if (!nc) return -1;
    memcpy(nc, cells, c * sizeof(or_cell));
    free(t->cells);
    t->cells = nc;
    t->cap = c;
    t->log2c = l;
    t->I = t->D = 0;
    for (uint64_t i = 0; i < c; ++i) {
        if (nc[i].key != OR_EMPTY) t->I++;
        if (nc[i].key == OR_TOMB) t->D++;
    }
    return 0;
}

/* Bulk merge of a batch into a non-empty table (Sec. 4.5: integer-sort the
 * batch by hash, keep the last of equal keys, and merge batch and table into
 * a new table, each element placed from max(home, previous position) on).
 * Reading taken here (the paper's text stops mid-sentence): the new table is
 * the sorted placement of the table's live elements followed by the batch --
 * the table's elements in cell index order, then the batch in input order,
 * ordered by the top B hash bits with ties in that order, all but the last of
 * equal keys dropped (so a batch element replaces the table's element of the
 * same key, and the last of equal batch elements wins), placed as or_build
 * places them.  Tombstones are dropped (a new table).  Capacity: a growable
 * table takes the smallest power of two c' >= c with live + n <= floor(alpha
 * c'); a bounded table keeps c.  Keys 0 / ~0 of the batch: the special slots
 * (last value) with the full key space on, else skipped (result 1); slots the
 * batch does not touch keep their content.  -2: no empty cell would remain
 * (table unchanged); -1: out of memory (unchanged). */
int or_merge(or_table *t, const uint64_t *keys, const uint64_t *vals, uint64_t n)
{
    const uint64_t live = t->I - t->D, tot = live + n;
    uint64_t *k = (uint64_t *)malloc((tot ? tot : 1) * sizeof(uint64_t));
    uint64_t *v = (uint64_t *)malloc((tot ? tot : 1) * sizeof(uint64_t));
    or_table *nt = or_create(t->cap, t->growable, t->alpha);
    if (!k || !v || !nt) {
        free(k);
        free(v);
        or_destroy(nt);
        return -1;
    }
    nt->full_keys = t->full_keys;
    nt->reuse_tombstones = t->reuse_tombstones;
    uint64_t m = 0;
    for (uint64_t i = 0; i < t->cap; ++i) {
        const uint64_t key = t->cells[i].key;
        if (key == OR_EMPTY || key == OR_TOMB) continue;
        k[m] = key;
        v[m] = t->cells[i].val;
        ++m;
    }
    for (uint64_t j = 0; j < n; ++j, ++m) {
        k[m] = keys[j];
        v[m] = vals[j];
    }
    const int r = or_build(nt, k, v, m);
    free(k);
    free(v);
    if (r < 0) {
        or_destroy(nt);
        return r;
    }
    free(t->cells);
    t->cells = nt->cells;
    t->cap = nt->cap;
    t->log2c = nt->log2c;
    t->I = nt->I;
    t->D = 0;
    t->probes += nt->probes;
    for (int sl = 0; sl < 2; ++sl)
        if (nt->sp_present[sl]) {
            t->sp_present[sl] = 1;
            t->sp_val[sl] = nt->sp_val[sl];
        }
    free(nt);
    return r;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Table invariants (Sec. 2 "Linear Probing"; proof of Lemma 1):
 *  1. every live key sits at or after its home with no empty cell between the
 *     home and its position (cyclically);
 *  2. every live key occurs exactly once;
 *  3. I equals the number of non-empty cells and I - D the number of live ones.
 * Returns 0 if all hold, else the number of the first broken invariant, with
 * a short description in msg. */
int or_check_invariants(const or_table *t, char *msg, size_t msglen)
{
    uint64_t mask = t->cap - 1, nonempty = 0, tomb = 0, live = 0;
    for (uint64_t i = 0; i < t->cap; ++i) {
        uint64_t k = t->cells[i].key;
        if (k == OR_EMPTY) continue;
        ++nonempty;
        if (k == OR_TOMB) { ++tomb; continue; }
        ++live;
        uint64_t h = home_of(k, t->log2c);
        for (uint64_t p = h; p != i; p = (p + 1) & mask) {
            if (t->cells[p].key == OR_EMPTY) {
                if (msg) snprintf(msg, msglen, "key %llu at %llu: empty cell %llu between home %llu and slot",
                                  (unsigned long long)k, (unsigned long long)i,
                                  (unsigned long long)p, (unsigned long long)h);
                return 1;
            }
        }
    }
    uint64_t *ks = (uint64_t *)malloc((live ? live : 1) * sizeof(uint64_t));
    if (!ks) return -1;
    uint64_t m = export_cells(t, ks, NULL, live);
    qsort(ks, m, sizeof(uint64_t), cmp_u64);
    for (uint64_t j = 1; j < m; ++j) {
        if (ks[j] == ks[j - 1]) {
            if (msg) snprintf(msg, msglen, "key %llu stored twice", (unsigned long long)ks[j]);
            free(ks);
            return 2;
        }
    }
    free(ks);
    if (t->I != nonempty || t->I - t->D != live || t->D != tomb) {
        if (msg) snprintf(msg, msglen, "counts: I=%llu D=%llu but nonempty=%llu tombstones=%llu live=%llu",
                          (unsigned long long)t->I, (unsigned long long)t->D,
                          (unsigned long long)nonempty, (unsigned long long)tomb,
                          (unsigned long long)live);
        return 3;
    }
    if (msg && msglen) msg[0] = 0;
    return 0;
}
