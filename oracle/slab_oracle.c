/*
 * Plain CPU oracle for the slab hash (Ashkiani, Farach-Colton, Owens,
 * "A Dynamic Hash Table for the GPU", arXiv 1710.11246).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path calls, links or loads
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header or constant table with the CUDA library.
 *
 * What it computes is the plain definition of the data structure, not the
 * GPU algorithm:
 *   - B buckets (Sec. 3.3). Each bucket is an array of slot positions in list
 *     order (key, value, state). In a set table (the default) a slot is
 *     "used" once written and stays used: deletion turns it into a tombstone
 *     (Sec. 3.2 "Deletion") that is never written again, so keys stay unique.
 *     In a multiset table (duplicates allowed, Sec. 3.2 INSERT) deletion
 *     empties the slot, and a later insert takes the first empty slot in list
 *     order before appending.
 *   - FLUSH (Sec. 4.3.4) compacts a bucket: its live elements keep their list
 *     order and move to the front; tombstones and holes disappear.
 *   - h(k) = ((a k + b) mod p) mod B with plain 64-bit `%` (Sec. 3.3).
 *   - replace / delete / search with the set semantics of Sec. 3.2
 *     (replace = insert with uniqueness; delete and search act on the only
 *     live instance of k, since keys are unique).
 *   - Slab bookkeeping that follows from the slab layout of Sec. 4.2: M data
 *     elements per slab, so a bucket with `len` used slots occupies
 *     max(1, ceil(len / M)) slabs, and the slot at position s lies in slab
 *     floor(s / M). A slab of W 4-byte words keeps its last two words for the
 *     auxiliary word and the next pointer, so M = (W - 2) / 2 pairs or W - 2
 *     keys: 15 or 30 for the paper's 128-byte slab (W = 32), 7 or 14 for a
 *     64-byte slab (W = 16).
 *   - "Lines touched" per operation: how many slabs a lookup must read in
 *     list order before it stops (Sec. 3.2 search / replace / delete walks).
 *
 * Pins for every function live in tests/test_oracle_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NOT_FOUND 0xFFFFFFFFu /* value reported for a search miss */
#define OR_KEY_LIMIT 0xFFFFFFFEu /* keys >= this are the two reserved sentinels (Sec. 3.2 footnote) */
#define OR_PRIME 4294967291ull   /* 2^32 - 5 */

enum { OR_OP_INSERT = 0, OR_OP_DELETE = 1, OR_OP_SEARCH = 2 };

enum { OR_TOMB = 0, OR_LIVE = 1, OR_HOLE = 2 }; /* slot states */

typedef struct {
    uint32_t key;
    uint32_t value;
    uint8_t live; /* OR_LIVE, OR_TOMB (set tables) or OR_HOLE (emptied, multiset tables) */
} or_slot;

typedef struct {
    or_slot *s;
    uint32_t len;
    uint32_t cap;
} or_bucket;

typedef struct {
    uint32_t B;        /* number of buckets (base slabs) */
    int learned;       /* buckets from the learned model instead of the universal hash */
    float model[2 + 2 * 1024];
    uint32_t M;        /* data elements per slab: 15 / 30 (128-byte slabs) or 7 / 14 (64-byte) */
    int key_only;
    int multiset;      /* duplicates allowed: INSERT instead of REPLACE, deletes empty their slot */
    uint64_t a, b, p;  /* universal hash parameters */
    or_bucket *bk;
    uint64_t live;     /* number of live elements */
    uint64_t reserved; /* ops skipped because their key was a sentinel */
} or_table;

/* Sec. 4.2: a slab of W words holds data in words 0..W-3, the auxiliary word in
 * W-2 and the next pointer in W-1, so M = (W - 2) / 2 pairs in key-value mode and
 * W - 2 keys in key-only mode. slab_bytes = 4 W is 128 (the paper's slab: M = 15
 * or 30) or 64 (M = 7 or 14). */
or_table *oracle_create_width(uint32_t num_buckets, int key_only, uint32_t a, uint32_t b, uint32_t slab_bytes)
{
    if (num_buckets == 0 || (slab_bytes != 64u && slab_bytes != 128u)) return NULL;
    or_table *t = (or_table *)calloc(1, sizeof(or_table));
    if (!t) return NULL;
    const uint32_t W = slab_bytes / 4u;
    t->B = num_buckets;
    t->key_only = key_only ? 1 : 0;
    t->M = key_only ? W - 2u : (W - 2u) / 2u;
    t->a = a;
    t->b = b;
    t->p = OR_PRIME;
    t->bk = (or_bucket *)calloc(num_buckets, sizeof(or_bucket));
    if (!t->bk) { free(t); return NULL; }
    return t;
}

or_table *oracle_create(uint32_t num_buckets, int key_only, uint32_t a, uint32_t b)
{
    return oracle_create_width(num_buckets, key_only, a, b, 128u);
}

void oracle_destroy(or_table *t)
{
    if (!t) return;
    for (uint32_t i = 0; i < t->B; i++) free(t->bk[i].s);
    free(t->bk);
    free(t);
}

/* Sec. 3.3: h(k; a, b) = ((a k + b) mod p) mod B. a, b < p < 2^32, so a k + b < 2^64. */
uint32_t oracle_hash(uint32_t a, uint32_t b, uint32_t num_buckets, uint32_t key)
{
    uint64_t x = (uint64_t)a * (uint64_t)key + (uint64_t)b;
    return (uint32_t)((x % OR_PRIME) % num_buckets);
}

/*
 * Learned bucket function (a library extension, not in the paper). A model is
 * 2 + 2 * 1024 floats: a root line (a, b) picks one of 1024 leaves, the leaf's
 * line (a, b) gives the bucket. Each line is evaluated in float as a * x, rounded,
 * plus b, rounded (this file is compiled with -ffp-contract=off so the two
 * roundings stay separate), with x the key rounded to float; the result is floored
 * and clamped to [0, limit), NaN and negatives giving 0.
 */
static uint32_t linear_piece(float a, float b, float x, uint32_t limit)
{
    float p = a * x;
    p = p + b;
    if (!(p >= 0.0f)) return 0;
    if (p >= (float)limit) return limit - 1;
    return (uint32_t)p;
}

uint32_t oracle_learned_bucket(const float *model, uint32_t num_buckets, uint32_t key)
{
    float x = (float)key;
    uint32_t leaf = linear_piece(model[0], model[1], x, 1024);
    return linear_piece(model[2 + 2 * leaf], model[3 + 2 * leaf], x, num_buckets);
}

uint32_t oracle_bucket(const or_table *t, uint32_t key)
{
    if (t->learned) return oracle_learned_bucket(t->model, t->B, key);
    return oracle_hash((uint32_t)t->a, (uint32_t)t->b, t->B, key);
}

/* Replace the table's bucket function by a learned model (the table must be empty). */
int oracle_use_model(or_table *t, const float *model)
{
    if (t->live != 0) return -1;
    for (uint32_t i = 0; i < t->B; i++)
        if (t->bk[i].len) return -1;
    memcpy(t->model, model, sizeof(t->model));
    t->learned = 1;
    return 0;
}

typedef unsigned __int128 or_u128;
typedef __int128 or_s128;

static double u128_to_double(or_u128 v)
{
    double hi = (double)(uint64_t)(v >> 64);
    double lo = (double)(uint64_t)v;
    hi = hi * 18446744073709551616.0; /* 2^64: exact */
    return hi + lo;
}

static double s128_to_double(or_s128 v)
{
    if (v < 0) return -u128_to_double((or_u128)(-v));
    return u128_to_double((or_u128)v);
}

/* Least squares line y = (a' x + b') / q through n >= 1 points (x, q y) with exact
 * integer moments of x and of the scaled targets q y: a' = (n Sxy - Sx Sy) /
 * (n Sxx - Sx^2), b' = (Sy - a' Sx) / n, a = a' / q, b = b' / q, each operation in
 * correctly rounded double, then rounded to float; a' = 0, b' = Sy / n when the
 * points share one x. */
static void fit_line(uint64_t n, or_u128 sx, or_u128 sy, or_u128 sxx, or_u128 sxy, uint64_t q, float *a, float *b)
{
    or_s128 N = (or_s128)n;
    or_s128 den = N * (or_s128)sxx - (or_s128)sx * (or_s128)sx;
    or_s128 num = N * (or_s128)sxy - (or_s128)sx * (or_s128)sy;
    double dn = (double)n, dq = (double)q;
    double a1 = 0.0, b1;
    if (den > 0) {
        a1 = s128_to_double(num) / s128_to_double(den);
        double t = a1 * u128_to_double(sx);
        double u = u128_to_double(sy) - t;
        b1 = u / dn;
    } else {
        b1 = u128_to_double(sy) / dn;
    }
    double a64 = a1 / dq;
    double b64 = b1 / dq;
    *a = (float)a64;
    *b = (float)b64;
}

static void add_point(or_u128 *sx, or_u128 *sy, or_u128 *sxx, or_u128 *sxy, uint32_t x, uint64_t y)
{
    *sx += x;
    *sy += y;
    *sxx += (or_u128)((uint64_t)x * x);
    *sxy += (or_u128)x * (or_u128)y;
}

/* The least-squares line through the integer points (xs[i], ys[i]), i < n (n >= 1). */
void oracle_fit_points(const uint32_t *xs, const uint32_t *ys, uint64_t n, float *ab)
{
    or_u128 sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (uint64_t i = 0; i < n; i++) add_point(&sx, &sy, &sxx, &sxy, xs[i], ys[i]);
    fit_line(n, sx, sy, sxx, sxy, 1, &ab[0], &ab[1]);
}

static int cmp_u32(const void *p, const void *q)
{
    uint32_t x = *(const uint32_t *)p, y = *(const uint32_t *)q;
    return (x > y) - (x < y);
}

/*
 * Fit the two-level model on the sample keys[0], keys[stride], keys[2 stride], ...:
 * sort the m sample keys; the root fits leaf position i * 1024 / m against the i-th
 * smallest key; each leaf fits bucket position i * B / m over the sample keys the
 * root sends to it; a leaf with no sample key is flat at c * B / m, c the number of
 * sample keys the root sends to lower leaves. Returns m, or 0 if n or stride is 0.
 */
uint64_t oracle_learn_model(const uint32_t *keys, uint64_t n, uint32_t stride, uint32_t num_buckets, float *model)
{
    if (n == 0 || stride == 0) return 0;
    uint64_t m = (n + stride - 1) / stride;
    uint32_t *x = (uint32_t *)malloc(m * sizeof(uint32_t));
    uint32_t *leaf = (uint32_t *)malloc(m * sizeof(uint32_t));
    if (!x || !leaf) abort();
    for (uint64_t i = 0; i < m; i++) x[i] = keys[i * stride];
    qsort(x, m, sizeof(uint32_t), cmp_u32);

    or_u128 sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (uint64_t i = 0; i < m; i++) add_point(&sx, &sy, &sxx, &sxy, x[i], i * 1024);
    fit_line(m, sx, sy, sxx, sxy, m, &model[0], &model[1]);
    for (uint64_t i = 0; i < m; i++) leaf[i] = linear_piece(model[0], model[1], (float)x[i], 1024);

    uint64_t below = 0; /* sample keys sent to leaves < j */
    for (uint32_t j = 0; j < 1024; j++) {
        or_u128 lx = 0, ly = 0, lxx = 0, lxy = 0;
        uint64_t cnt = 0;
        for (uint64_t i = 0; i < m; i++) {
            if (leaf[i] != j) continue;
            add_point(&lx, &ly, &lxx, &lxy, x[i], i * (uint64_t)num_buckets);
            cnt++;
        }
        if (cnt) {
            fit_line(cnt, lx, ly, lxx, lxy, m, &model[2 + 2 * j], &model[3 + 2 * j]);
        } else {
            double start = (double)(below * (uint64_t)num_buckets) / (double)m;
            model[2 + 2 * j] = 0.0f;
            model[3 + 2 * j] = (float)start;
        }
        below += cnt;
    }
    free(x);
    free(leaf);
    return m;
}

/* Slabs per bucket that `n` keys would form under the table's bucket function:
 * *sum and *max of max(1, ceil(load / M)) over the buckets. */
void oracle_chain_profile(const or_table *t, const uint32_t *keys, uint64_t n, uint64_t *sum, uint32_t *max)
{
    uint32_t *load = (uint32_t *)calloc(t->B, sizeof(uint32_t));
    if (!load) abort();
    for (uint64_t i = 0; i < n; i++)
        if (keys[i] < OR_KEY_LIMIT) load[oracle_bucket(t, keys[i])]++;
    uint64_t s = 0;
    uint32_t mx = 0;
    for (uint32_t b = 0; b < t->B; b++) {
        uint32_t k = load[b] == 0 ? 1 : (load[b] + t->M - 1) / t->M;
        s += k;
        if (k > mx) mx = k;
    }
    free(load);
    *sum = s;
    *max = mx;
}

/* Position of the first live slot (in list order) holding `key`, or -1. */
static int64_t find_live(const or_bucket *bk, uint32_t key)
{
    for (uint32_t s = 0; s < bk->len; s++)
        if (bk->s[s].live == OR_LIVE && bk->s[s].key == key) return (int64_t)s;
    return -1;
}

static uint64_t slabs_of(const or_table *t, uint32_t len)
{
    return len == 0 ? 1 : (len + t->M - 1) / t->M;
}

static void append(or_bucket *bk, uint32_t key, uint32_t value)
{
    if (bk->len == bk->cap) {
        uint32_t nc = bk->cap ? bk->cap * 2 : 4;
        or_slot *ns = (or_slot *)realloc(bk->s, (size_t)nc * sizeof(or_slot));
        if (!ns) abort();
        bk->s = ns;
        bk->cap = nc;
    }
    bk->s[bk->len].key = key;
    bk->s[bk->len].value = value;
    bk->s[bk->len].live = OR_LIVE;
    bk->len++;
}

/* Sec. 3.2 INSERT (multiset tables): S <- S U {<k,v>} with no uniqueness check; the
 * pair goes into the first empty slot in list order (a hole left by a delete),
 * else at the tail. Lines: the slabs read up to that slot. */
static void op_insert_dup(or_table *t, uint32_t key, uint32_t value, uint64_t *lines)
{
    or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    if (t->key_only) value = 0;
    uint32_t s = 0;
    while (s < bk->len && bk->s[s].live != OR_HOLE) s++;
    if (lines) *lines += (uint64_t)s / t->M + 1;
    if (s < bk->len) {
        bk->s[s].key = key;
        bk->s[s].value = value;
        bk->s[s].live = OR_LIVE;
    } else {
        append(bk, key, value);
    }
    t->live++;
}

/* Remove the element at position s: a tombstone in a set table, a hole (an empty
 * slot later inserts may fill) in a multiset table (Sec. 3.2 "Deletion"). */
static void kill(or_table *t, or_bucket *bk, uint32_t s)
{
    bk->s[s].live = t->multiset ? OR_HOLE : OR_TOMB;
    t->live--;
}

/* Sec. 3.2 REPLACE: S <- (S - {<k,*>}) U {<k,v>}. If k is live, overwrite its value
 * in place; otherwise write a new slot at the tail of the list (first empty slot;
 * tombstones are not reused). Returns 1 if k was already present.
 * Lines: a hit at slot s reads slabs 0..s/M; a new key lands in slot len and reads
 * slabs 0..len/M (the last one freshly allocated when len is a multiple of M). */
static int op_replace(or_table *t, uint32_t key, uint32_t value, uint64_t *lines)
{
    or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    if (t->key_only) value = 0;
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        bk->s[s].value = value;
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    if (lines) *lines += (uint64_t)bk->len / t->M + 1;
    append(bk, key, value);
    t->live++;
    return 0;
}

/* Sec. 3.2 DELETE: remove the first live <k,v> in list order (the only one in a
 * set table). Returns 1 if k was present. A miss reads every slab of the list. */
static int op_delete(or_table *t, uint32_t key, uint64_t *lines)
{
    or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        kill(t, bk, (uint32_t)s);
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    if (lines) *lines += slabs_of(t, bk->len);
    return 0;
}

/* Sec. 3.2 SEARCH: return the first live <k,v> in list order, or "not found". */
static int op_search(const or_table *t, uint32_t key, uint32_t *value, uint64_t *lines)
{
    const or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        *value = t->key_only ? 0 : bk->s[s].value;
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    *value = OR_NOT_FOUND;
    if (lines) *lines += slabs_of(t, bk->len);
    return 0;
}

/* Batches apply their ops one after another in index order. Under the batch
 * contract (each key in at most one op per batch) every order gives the same
 * results. found[i] = 1 iff the key was live just before op i. */
void oracle_insert(or_table *t, const uint32_t *keys, const uint32_t *values, uint64_t n,
                   uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else if (t->multiset) op_insert_dup(t, keys[i], values ? values[i] : 0u, lines);
        else f = op_replace(t, keys[i], values ? values[i] : 0u, lines);
        if (found) found[i] = (uint8_t)f;
    }
}

void oracle_delete(or_table *t, const uint32_t *keys, uint64_t n, uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else f = op_delete(t, keys[i], lines);
        if (found) found[i] = (uint8_t)f;
    }
}

void oracle_search(or_table *t, const uint32_t *keys, uint64_t n, uint32_t *values,
                   uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t v = OR_NOT_FOUND;
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else f = op_search(t, keys[i], &v, lines);
        if (values) values[i] = v;
        if (found) found[i] = (uint8_t)f;
    }
}

/* Sec. 6.3 concurrent batch: one op per element. results[i]:
 *   search -> stored value, or OR_NOT_FOUND on a miss;
 *   insert -> 1 if the key was new, 0 if an existing value was replaced;
 *   delete -> 1 if the key was deleted, 0 if it was absent.
 * Unknown op codes are skipped (result 0, found 0). */
void oracle_mixed(or_table *t, const uint8_t *ops, const uint32_t *keys, const uint32_t *values,
                  uint64_t n, uint32_t *results, uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t r = 0;
        int f = 0;
        if (ops[i] == OR_OP_SEARCH) r = OR_NOT_FOUND;
        if (ops[i] > OR_OP_SEARCH) {
            /* not an op */
        } else if (keys[i] >= OR_KEY_LIMIT) {
            t->reserved++;
        } else if (ops[i] == OR_OP_INSERT) {
            if (t->multiset) op_insert_dup(t, keys[i], values ? values[i] : 0u, lines);
            else f = op_replace(t, keys[i], values ? values[i] : 0u, lines);
            r = f ? 0u : 1u;
        } else if (ops[i] == OR_OP_DELETE) {
            f = op_delete(t, keys[i], lines);
            r = (uint32_t)f;
        } else {
            f = op_search(t, keys[i], &r, lines);
        }
        if (results) results[i] = r;
        if (found) found[i] = (uint8_t)f;
    }
}

/* Per-bucket used slots (live + tombstoned; holes are empty) and slab counts
 * (the list spans every position ever written), plus totals
 * {live, used slots, slabs, reserved-key ops}. */
void oracle_stats(const or_table *t, uint32_t *slots, uint32_t *slabs, uint64_t *totals)
{
    uint64_t used = 0, nslabs = 0;
    for (uint32_t i = 0; i < t->B; i++) {
        const or_bucket *bk = &t->bk[i];
        uint32_t u = 0;
        for (uint32_t s = 0; s < bk->len; s++) u += bk->s[s].live != OR_HOLE;
        uint64_t k = slabs_of(t, bk->len);
        if (slots) slots[i] = u;
        if (slabs) slabs[i] = (uint32_t)k;
        used += u;
        nslabs += k;
    }
    if (totals) {
        totals[0] = t->live;
        totals[1] = used;
        totals[2] = nslabs;
        totals[3] = t->reserved;
    }
}

/* Sec. 3.3 memory utilization: (x / (M x + y)) * n / sum_i k_i, with x the bytes
 * of one element (8 for a pair, 4 for a key), y = 8 bytes of the auxiliary word
 * and the next pointer, and k_i the number of slabs of bucket i. */
double oracle_utilization(const or_table *t)
{
    uint64_t tot[4];
    oracle_stats(t, NULL, NULL, tot);
    double x = t->key_only ? 4.0 : 8.0;
    double y = 8.0;
    return (x / (t->M * x + y)) * (double)tot[0] / (double)tot[2];
}

/* All live elements as (bucket, key, value), buckets in order, slots in list order. */
uint64_t oracle_export(const or_table *t, uint32_t *buckets, uint32_t *keys, uint32_t *values,
                       uint64_t cap)
{
    uint64_t c = 0;
    for (uint32_t i = 0; i < t->B; i++) {
        const or_bucket *bk = &t->bk[i];
        for (uint32_t s = 0; s < bk->len; s++) {
            if (bk->s[s].live != OR_LIVE) continue;
            if (c < cap) {
                if (buckets) buckets[c] = i;
                if (keys) keys[c] = bk->s[s].key;
                if (values) values[c] = t->key_only ? 0u : bk->s[s].value;
            }
            c++;
        }
    }
    return c;
}

/* Make an empty table a multiset (duplicates allowed). Returns 0, or -1 if the
 * table already holds elements. */
int oracle_set_multiset(or_table *t, int on)
{
    for (uint32_t i = 0; i < t->B; i++)
        if (t->bk[i].len) return -1;
    t->multiset = on ? 1 : 0;
    return 0;
}

/* Sec. 3.2 SEARCHALL: every live <k,*> in list order. counts[i] = the number of
 * instances of keys[i]; their values (0 in key-only mode) go to
 * values[i * cap + j] for j < min(counts[i], cap), the rest of the row untouched. */
void oracle_search_all(const or_table *t, const uint32_t *keys, uint64_t n, uint32_t cap, uint32_t *counts,
                       uint32_t *values)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t c = 0;
        if (keys[i] < OR_KEY_LIMIT) {
            const or_bucket *bk = &t->bk[oracle_bucket(t, keys[i])];
            for (uint32_t s = 0; s < bk->len; s++) {
                if (bk->s[s].live != OR_LIVE || bk->s[s].key != keys[i]) continue;
                if (c < cap && values) values[i * cap + c] = t->key_only ? 0u : bk->s[s].value;
                c++;
            }
        }
        if (counts) counts[i] = c;
    }
}

/* Sec. 3.2 DELETEALL: remove every live <k,*>; counts[i] = how many. */
void oracle_delete_all(or_table *t, const uint32_t *keys, uint64_t n, uint32_t *counts)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t c = 0;
        if (keys[i] >= OR_KEY_LIMIT) {
            t->reserved++;
        } else {
            or_bucket *bk = &t->bk[oracle_bucket(t, keys[i])];
            for (uint32_t s = 0; s < bk->len; s++)
                if (bk->s[s].live == OR_LIVE && bk->s[s].key == keys[i]) {
                    kill(t, bk, s);
                    c++;
                }
        }
        if (counts) counts[i] = c;
    }
}

/* Sec. 4.3.4 FLUSH of every bucket: the live elements keep their list order and
 * move to the front of the list, tombstones and holes disappear, and the list
 * keeps max(1, ceil(live / M)) slabs. Returns the number of slabs released. */
uint64_t oracle_flush(or_table *t)
{
    uint64_t released = 0;
    for (uint32_t i = 0; i < t->B; i++) {
        or_bucket *bk = &t->bk[i];
        uint64_t before = slabs_of(t, bk->len);
        uint32_t w = 0;
        for (uint32_t s = 0; s < bk->len; s++)
            if (bk->s[s].live == OR_LIVE) bk->s[w++] = bk->s[s];
        bk->len = w;
        released += before - slabs_of(t, w);
    }
    return released;
}

/*
 * SlabAlloc state check (Sec. 5 "SlabAlloc" and "Memory structure").
 *
 * A 32-bit slab address has the unit index within its memory block in bits
 * [0,10), the memory block within its super block in bits [10,24) and the
 * super block in bits [24,32). A memory block holds 1024 units and one 32-bit
 * bitmap word per 32 units: word w of a block covers units 32w .. 32w+31, bit
 * (unit mod 32) of it set iff that unit is allocated. Blocks are numbered
 * super block by super block, `blocks_per_super` to a super block.
 *
 * Given the addresses a set of allocations returned and the bitmap words the
 * allocator holds afterwards, checks that every address decodes to an existing
 * unit, that no address appears twice, and that the bitmaps mark exactly those
 * units. Returns 0 if all hold; 1 bad address, 2 duplicate, 3 bitmap mismatch.
 * *where receives the offending address index (1, 2) or bitmap word (3).
 */
int oracle_check_alloc(const uint32_t *addrs, uint64_t n, const uint32_t *bitmaps,
                       uint64_t num_blocks, uint32_t blocks_per_super, uint64_t *where)
{
    uint64_t words = num_blocks * 32;
    uint32_t *expect = (uint32_t *)calloc(words ? words : 1, sizeof(uint32_t));
    if (!expect) abort();
    int rc = 0;
    for (uint64_t i = 0; i < n && rc == 0; i++) {
        uint32_t a = addrs[i];
        uint32_t unit = a & 1023u;
        uint32_t blk = (a >> 10) & 0x3FFFu;
        uint32_t sb = a >> 24;
        uint64_t block = (uint64_t)sb * blocks_per_super + blk;
        if (blk >= blocks_per_super || block >= num_blocks) { rc = 1; *where = i; break; }
        uint64_t w = block * 32 + unit / 32;
        uint32_t bit = 1u << (unit % 32);
        if (expect[w] & bit) { rc = 2; *where = i; break; }
        expect[w] |= bit;
    }
    for (uint64_t w = 0; w < words && rc == 0; w++)
        if (expect[w] != bitmaps[w]) { rc = 3; *where = w; }
    free(expect);
    return rc;
}
