/*
 * bsort_oracle.c -- TEST INFRASTRUCTURE, not part of the library.
 *
 * A plain, slow CPU statement of GPU Bucket Sort
 * (Dehne & Zaboli, "Deterministic Sample Sort for GPUs", Section 4,
 * Algorithm 1, Steps 1-9), written from the paper's step definitions so that
 * a reader can check every step against the text by eye.  Only the tests,
 * the package's smoke check and the benchmark's CPU-baseline leg may load
 * this file; the CUDA library never does, and the two share no code.
 *
 * Everything is integer work (comparisons, counts, copies); no floating
 * point is involved except the order-preserving key transform for float32
 * keys, which is a pure bit manipulation.
 *
 * Readings of points where the paper is silent (kept identical in the CUDA
 * path, which is written separately):
 *   - Elements are compared in "composite order": (key, position), so every
 *     element is distinct.  Inside Steps 3-8 the position of an element of
 *     sublist i at sorted rank r is p = i*t + r; because each sublist is
 *     sorted stably and sublists are contiguous index ranges, this order is
 *     the same as (key, original index).
 *   - Step 3 takes, from each sorted sublist of t items, the samples at
 *     ranks (k+1)*w - 1, k = 0..s-1, with w = t/s (the last item of each of
 *     s equal chunks).
 *   - Step 5 takes the global samples (splitters) g_j = S[(j+1)*m - 1],
 *     j = 0..s-1, from the sorted sample list S; g_{s-1} is the global
 *     maximum, so the s splitters define exactly s buckets.  As an extension
 *     the number of buckets b may differ from s: then g_j = S[r_j] with
 *     r_j = floor((j+1)*m*s/b) - 1, j = 0..b-1 (equidistant in the sample
 *     list; b = s gives the paper's choice).
 *   - Bucket j of sublist i holds the items x with g_{j-1} < x <= g_j in
 *     composite order (g_{-1} = minus infinity).
 *   - n need not be a multiple of t: the input is padded virtually to
 *     n' = ceil(n/t)*t with sentinels (key = the largest key of the type,
 *     position >= n) that are larger than every real item in composite order;
 *     they end in the tail of the output and are dropped.
 *   - Parity is pinned by the tests (brute force on tiny inputs, an
 *     independent textbook merge sort, closed-form bucket sizes and the
 *     bucket-size bound), not by this file itself.
 *
 * oracle_paper_sort runs on one thread.  oracle_paper_sort_mt runs the same
 * code with the independent iterations of Steps 2, 6 and 8 (one per
 * sublist) and Step 9 (one per bucket) spread over POSIX threads in
 * contiguous ranges; nothing else changes, so both give identical results.
 * It exists only to time the oracle on all host cores.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t key;
    uint64_t val;
    uint64_t pos; /* original index (pads: >= n) */
} oelem_t;

/* Composite order used by Steps 2-9: (key, pos). */
static int elem_less(const oelem_t *a, const oelem_t *b)
{
    if (a->key != b->key) return a->key < b->key;
    return a->pos < b->pos;
}

/* Sample record of Step 3: (key, p) with p = i*t + r. */
typedef struct {
    uint64_t key;
    uint64_t p;
} orec_t;

static int rec_less(const orec_t *a, const orec_t *b)
{
    if (a->key != b->key) return a->key < b->key;
    return a->p < b->p;
}

/* ---- top-down merge sort (used for Steps 2, 4 and 9) ------------------- */

static void msort_elems_rec(oelem_t *a, oelem_t *tmp, uint64_t lo, uint64_t hi)
{
    if (hi - lo < 2) return;
    uint64_t mid = lo + (hi - lo) / 2;
    msort_elems_rec(a, tmp, lo, mid);
    msort_elems_rec(a, tmp, mid, hi);
    uint64_t x = lo, y = mid, o = lo;
    while (x < mid && y < hi) {
        /* take from the left run unless the right item is strictly smaller */
        if (elem_less(&a[y], &a[x])) tmp[o++] = a[y++];
        else tmp[o++] = a[x++];
    }
    while (x < mid) tmp[o++] = a[x++];
    while (y < hi) tmp[o++] = a[y++];
    memcpy(a + lo, tmp + lo, (hi - lo) * sizeof(oelem_t));
}

static int msort_elems(oelem_t *a, uint64_t n)
{
    if (n < 2) return 0;
    oelem_t *tmp = (oelem_t *)malloc(n * sizeof(oelem_t));
    if (!tmp) return -1;
    msort_elems_rec(a, tmp, 0, n);
    free(tmp);
    return 0;
}

static void msort_recs_rec(orec_t *a, orec_t *tmp, uint64_t lo, uint64_t hi)
{
    if (hi - lo < 2) return;
    uint64_t mid = lo + (hi - lo) / 2;
    msort_recs_rec(a, tmp, lo, mid);
    msort_recs_rec(a, tmp, mid, hi);
    uint64_t x = lo, y = mid, o = lo;
    while (x < mid && y < hi) {
        if (rec_less(&a[y], &a[x])) tmp[o++] = a[y++];
        else tmp[o++] = a[x++];
    }
    while (x < mid) tmp[o++] = a[x++];
    while (y < hi) tmp[o++] = a[y++];
    memcpy(a + lo, tmp + lo, (hi - lo) * sizeof(orec_t));
}

static int msort_recs(orec_t *a, uint64_t n)
{
    if (n < 2) return 0;
    orec_t *tmp = (orec_t *)malloc(n * sizeof(orec_t));
    if (!tmp) return -1;
    msort_recs_rec(a, tmp, 0, n);
    free(tmp);
    return 0;
}

/* ---- float32 key transform (reading of the paper's silence on key types) */

/* Order-preserving map of IEEE-754 binary32 bits to uint32: negative values
 * (sign set) are bit-inverted, non-negative values get the sign bit set.  The
 * resulting unsigned order is -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN. */
uint32_t oracle_f32_to_key(uint32_t bits)
{
    if (bits & 0x80000000u) return ~bits;
    return bits | 0x80000000u;
}

uint32_t oracle_key_to_f32(uint32_t key)
{
    if (key & 0x80000000u) return key & 0x7FFFFFFFu;
    return ~key;
}

void oracle_f32_to_key_array(const uint32_t *bits, uint32_t *keys, uint64_t n)
{
    for (uint64_t x = 0; x < n; ++x) keys[x] = oracle_f32_to_key(bits[x]);
}

void oracle_key_to_f32_array(const uint32_t *keys, uint32_t *bits, uint64_t n)
{
    for (uint64_t x = 0; x < n; ++x) bits[x] = oracle_key_to_f32(keys[x]);
}

/* ---- Algorithm 1 --------------------------------------------------------- */

/* Plan quantities of Step 1. */
uint64_t oracle_num_sublists(uint64_t n, uint64_t t)
{
    return t ? (n + t - 1) / t : 0;
}

/* ---- running independent loop iterations on several threads ------------ */

/* fn(ctx, lo, hi) runs iterations [lo, hi) of a loop whose iterations touch
 * disjoint data; it returns nonzero on failure. */
typedef int (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);

typedef struct {
    range_fn fn;
    void *ctx;
    uint64_t lo, hi;
    int rc;
} range_job;

static void *range_thread(void *arg)
{
    range_job *j = (range_job *)arg;
    j->rc = j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

/* Iterations [0, count) in `threads` contiguous ranges (threads <= 1: on the
 * calling thread; a range whose thread cannot be started runs on the calling
 * thread).  Returns nonzero if any range failed. */
static int run_ranges(int threads, uint64_t count, range_fn fn, void *ctx)
{
    if (threads <= 1 || count < 2) return fn(ctx, 0, count);
    if ((uint64_t)threads > count) threads = (int)count;
    pthread_t *tid = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
    range_job *job = (range_job *)malloc((size_t)threads * sizeof(range_job));
    char *live = (char *)calloc((size_t)threads, 1);
    if (!tid || !job || !live) {
        free(tid);
        free(job);
        free(live);
        return fn(ctx, 0, count);
    }
    int rc = 0;
    for (int k = 0; k < threads; ++k) {
        job[k].fn = fn;
        job[k].ctx = ctx;
        job[k].lo = count * (uint64_t)k / (uint64_t)threads;
        job[k].hi = count * (uint64_t)(k + 1) / (uint64_t)threads;
        job[k].rc = 0;
        live[k] = pthread_create(&tid[k], NULL, range_thread, &job[k]) == 0;
        if (!live[k]) job[k].rc = fn(ctx, job[k].lo, job[k].hi);
    }
    for (int k = 0; k < threads; ++k) {
        if (live[k]) pthread_join(tid[k], NULL);
        rc |= job[k].rc;
    }
    free(tid);
    free(job);
    free(live);
    return rc;
}

/* The arrays of one oracle_paper_sort call, shared by its loop bodies. */
typedef struct {
    oelem_t *A, *B;
    orec_t *G;
    uint64_t *c, *a, *l;
    uint64_t m, t, b, np;
} sort_state;

/* Step 2: local sort of sublists [lo, hi) (stable: composite order). */
static int step2_sublists(void *ctx, uint64_t lo, uint64_t hi)
{
    sort_state *st = (sort_state *)ctx;
    oelem_t *A = st->A;
    const uint64_t t = st->t;
    for (uint64_t i = lo; i < hi; ++i)
        if (msort_elems(A + i * t, t)) return -1;
    return 0;
}

/* Step 6: sample indexing for sublists [lo, hi).  c[i][j+1] = number of
 * items of sorted sublist i that are <= g_j in composite order, where the
 * item at rank r of sublist i is (key, i*t + r); found by binary search
 * because the sublist is sorted in that order.  c[i][0] = 0.  Bucket A_ij is
 * ranks [c[i][j], c[i][j+1]) and a_ij is its size. */
static int step6_sublists(void *ctx, uint64_t i0, uint64_t i1)
{
    sort_state *st = (sort_state *)ctx;
    const oelem_t *A = st->A;
    const orec_t *G = st->G;
    uint64_t *c = st->c, *a = st->a;
    const uint64_t t = st->t, b = st->b, m = st->m;
    for (uint64_t i = i0; i < i1; ++i) {
        c[i * (b + 1) + 0] = 0;
        for (uint64_t j = 0; j < b; ++j) {
            uint64_t lo = 0, hi = t; /* first rank whose item is > g_j */
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                orec_t item;
                item.key = A[i * t + mid].key;
                item.p = i * t + mid;
                if (rec_less(&G[j], &item)) hi = mid;
                else lo = mid + 1;
            }
            c[i * (b + 1) + j + 1] = lo;
        }
        for (uint64_t j = 0; j < b; ++j)
            a[j * m + i] = c[i * (b + 1) + j + 1] - c[i * (b + 1) + j];
    }
    return 0;
}

/* Step 8 for sublists [lo, hi): move every bucket A_ij to l_ij. */
static int step8_sublists(void *ctx, uint64_t i0, uint64_t i1)
{
    sort_state *st = (sort_state *)ctx;
    const oelem_t *A = st->A;
    oelem_t *B = st->B;
    const uint64_t *c = st->c, *a = st->a, *l = st->l;
    const uint64_t t = st->t, b = st->b, m = st->m;
    for (uint64_t i = i0; i < i1; ++i)
        for (uint64_t j = 0; j < b; ++j) {
            uint64_t src = i * t + c[i * (b + 1) + j];
            uint64_t len = a[j * m + i];
            for (uint64_t q = 0; q < len; ++q) B[l[j * m + i] + q] = A[src + q];
        }
    return 0;
}

/* Step 9 for buckets [j0, j1): sort every sublist B_j. */
static int step9_buckets(void *ctx, uint64_t j0, uint64_t j1)
{
    sort_state *st = (sort_state *)ctx;
    oelem_t *B = st->B;
    const uint64_t *l = st->l;
    const uint64_t b = st->b, m = st->m, np = st->np;
    for (uint64_t j = j0; j < j1; ++j) {
        uint64_t lo = l[j * m + 0];
        uint64_t hi = (j + 1 < b) ? l[(j + 1) * m + 0] : np;
        if (msort_elems(B + lo, hi - lo)) return -1;
    }
    return 0;
}

/*
 * GPU Bucket Sort, Algorithm 1 Steps 1-9, with every intermediate exposed.
 *
 *   keys, vals : n input items (vals may be NULL: keys only)
 *   t          : sublist size n/m of Step 1 (a multiple of s)
 *   s          : samples per sublist (Step 3)
 *   b          : global samples = buckets (Step 5); 0 means b = s (paper)
 *   key_max    : the largest key of the key type (pad sentinel key)
 *   out_keys, out_vals : n sorted items (out_vals may be NULL)
 *   threads    : (oracle_paper_sort_mt) threads for Steps 2, 6, 8 and 9
 *
 * Optional intermediates (NULL to skip), with m = ceil(n/t), n' = m*t:
 *   tile_keys, tile_pos   [n']   Step 2: sorted sublists, sublist-major
 *   samp_keys, samp_p     [m*s]  Step 3: samples, sublist-major, p = i*t + r
 *   spl_keys, spl_p       [b]    Step 5: global samples g_0..g_{b-1}
 *   counts                [m*b]  Step 6: a_ij stored bucket-major a[j*m + i]
 *   offsets               [m*b]  Step 7: l_ij stored bucket-major l[j*m + i]
 *   reloc_keys, reloc_pos [n']   Step 8: relocated array B_1 ... B_b
 *   bucket_start          [b+1]  start of B_j in the relocated array; [b] = n'
 *
 * Returns 0, or -1 on bad parameters / allocation failure.
 */
int oracle_paper_sort_mt(const uint64_t *keys, const uint64_t *vals, uint64_t n,
                         uint64_t t, uint64_t s, uint64_t b, uint64_t key_max,
                         uint64_t *out_keys, uint64_t *out_vals,
                         uint64_t *tile_keys, uint64_t *tile_pos,
                         uint64_t *samp_keys, uint64_t *samp_p,
                         uint64_t *spl_keys, uint64_t *spl_p,
                         uint64_t *counts, uint64_t *offsets,
                         uint64_t *reloc_keys, uint64_t *reloc_pos,
                         uint64_t *bucket_start, int threads)
{
    if (n == 0) return 0;
    if (t == 0 || s == 0 || s > t || (t % s) != 0) return -1;

    /* Step 1: split A into m sublists of t = n/m items (virtual padding). */
    const uint64_t m = (n + t - 1) / t;
    const uint64_t np = m * t;
    const uint64_t w = t / s;
    if (b == 0) b = s;
    if (b > m * s) return -1;

    oelem_t *A = (oelem_t *)malloc(np * sizeof(oelem_t));
    orec_t *S = (orec_t *)malloc(m * s * sizeof(orec_t));
    orec_t *G = (orec_t *)malloc(b * sizeof(orec_t));
    uint64_t *c = (uint64_t *)malloc(m * (b + 1) * sizeof(uint64_t));
    uint64_t *a = (uint64_t *)malloc(m * b * sizeof(uint64_t));
    uint64_t *l = (uint64_t *)malloc(m * b * sizeof(uint64_t));
    oelem_t *B = (oelem_t *)malloc(np * sizeof(oelem_t));
    sort_state st;
    st.A = A; st.B = B; st.G = G; st.c = c; st.a = a; st.l = l;
    st.m = m; st.t = t; st.b = b; st.np = np;
    if (!A || !S || !G || !c || !a || !l || !B) goto fail;

    for (uint64_t x = 0; x < np; ++x) {
        if (x < n) {
            A[x].key = keys[x];
            A[x].val = vals ? vals[x] : 0;
        } else {
            A[x].key = key_max;
            A[x].val = 0;
        }
        A[x].pos = x;
    }

    /* Step 2: local sort of every sublist A_i (stable: composite order). */
    if (run_ranges(threads, m, step2_sublists, &st)) goto fail;
    if (tile_keys)
        for (uint64_t x = 0; x < np; ++x) tile_keys[x] = A[x].key;
    if (tile_pos)
        for (uint64_t x = 0; x < np; ++x) tile_pos[x] = A[x].pos;

    /* Step 3: s equidistant samples per sorted sublist, ranks (k+1)w - 1. */
    for (uint64_t i = 0; i < m; ++i)
        for (uint64_t k = 0; k < s; ++k) {
            uint64_t r = (k + 1) * w - 1;
            S[i * s + k].key = A[i * t + r].key;
            S[i * s + k].p = i * t + r;
        }
    if (samp_keys)
        for (uint64_t x = 0; x < m * s; ++x) samp_keys[x] = S[x].key;
    if (samp_p)
        for (uint64_t x = 0; x < m * s; ++x) samp_p[x] = S[x].p;

    /* Step 4: sort all s*m samples. */
    if (msort_recs(S, m * s)) goto fail;

    /* Step 5: b equidistant global samples g_j = S[r_j],
     * r_j = floor((j+1)*m*s/b) - 1 (= (j+1)m - 1 when b = s). */
    for (uint64_t j = 0; j < b; ++j) G[j] = S[(j + 1) * m * s / b - 1];
    if (spl_keys)
        for (uint64_t j = 0; j < b; ++j) spl_keys[j] = G[j].key;
    if (spl_p)
        for (uint64_t j = 0; j < b; ++j) spl_p[j] = G[j].p;

    /* Step 6: sample indexing, every sublist (step6_sublists). */
    if (run_ranges(threads, m, step6_sublists, &st)) goto fail;
    if (counts) memcpy(counts, a, m * b * sizeof(uint64_t));

    /* Step 7: prefix sum over a_11..a_m1, a_12..a_m2, ..., a_1s..a_ms
     * (bucket-major), exclusive: l_ij = start of A_ij in the final order. */
    {
        uint64_t run = 0;
        for (uint64_t x = 0; x < m * b; ++x) {
            l[x] = run;
            run += a[x];
        }
    }
    if (offsets) memcpy(offsets, l, m * b * sizeof(uint64_t));

    /* Step 8: move every bucket A_ij to l_ij; B_j = A_1j u ... u A_mj. */
    if (run_ranges(threads, m, step8_sublists, &st)) goto fail;
    if (reloc_keys)
        for (uint64_t x = 0; x < np; ++x) reloc_keys[x] = B[x].key;
    if (reloc_pos)
        for (uint64_t x = 0; x < np; ++x) reloc_pos[x] = B[x].pos;
    if (bucket_start) {
        for (uint64_t j = 0; j < b; ++j) bucket_start[j] = l[j * m + 0];
        bucket_start[b] = np;
    }

    /* Step 9: sort every sublist B_j. */
    if (run_ranges(threads, b, step9_buckets, &st)) goto fail;

    /* Output: the first n items (pads are the largest items, so they are
     * exactly the last n' - n). */
    for (uint64_t x = 0; x < n; ++x) {
        out_keys[x] = B[x].key;
        if (out_vals) out_vals[x] = B[x].val;
    }

    free(A); free(S); free(G); free(c); free(a); free(l); free(B);
    return 0;
fail:
    free(A); free(S); free(G); free(c); free(a); free(l); free(B);
    return -1;
}

/* The single-threaded form (the statement the tests pin). */
int oracle_paper_sort(const uint64_t *keys, const uint64_t *vals, uint64_t n,
                      uint64_t t, uint64_t s, uint64_t b, uint64_t key_max,
                      uint64_t *out_keys, uint64_t *out_vals,
                      uint64_t *tile_keys, uint64_t *tile_pos,
                      uint64_t *samp_keys, uint64_t *samp_p,
                      uint64_t *spl_keys, uint64_t *spl_p,
                      uint64_t *counts, uint64_t *offsets,
                      uint64_t *reloc_keys, uint64_t *reloc_pos,
                      uint64_t *bucket_start)
{
    return oracle_paper_sort_mt(keys, vals, n, t, s, b, key_max, out_keys, out_vals,
                                tile_keys, tile_pos, samp_keys, samp_p, spl_keys, spl_p,
                                counts, offsets, reloc_keys, reloc_pos, bucket_start, 1);
}

/* ---- O2: independent textbook bottom-up merge sort ----------------------- */

/*
 * Stable sort of (key, val) pairs by key: bottom-up merging of runs of width
 * 1, 2, 4, ... between two buffers.  Written separately from the code above
 * (no shared helpers) so that it can serve as an independent check of the
 * final output of oracle_paper_sort.
 */
int oracle_textbook_sort(const uint64_t *keys, const uint64_t *vals, uint64_t n,
                         uint64_t *out_keys, uint64_t *out_vals)
{
    if (n == 0) return 0;
    uint64_t *k0 = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *k1 = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *v0 = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *v1 = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!k0 || !k1 || !v0 || !v1) {
        free(k0); free(k1); free(v0); free(v1);
        return -1;
    }
    for (uint64_t x = 0; x < n; ++x) {
        k0[x] = keys[x];
        v0[x] = vals ? vals[x] : 0;
    }
    for (uint64_t width = 1; width < n; width *= 2) {
        for (uint64_t lo = 0; lo < n; lo += 2 * width) {
            uint64_t mid = lo + width < n ? lo + width : n;
            uint64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            uint64_t x = lo, y = mid, o = lo;
            while (o < hi) {
                /* stable: the right run wins only on a strictly smaller key */
                int take_right = (x >= mid) || (y < hi && k0[y] < k0[x]);
                if (take_right) { k1[o] = k0[y]; v1[o] = v0[y]; ++y; }
                else            { k1[o] = k0[x]; v1[o] = v0[x]; ++x; }
                ++o;
            }
        }
        uint64_t *tk = k0; k0 = k1; k1 = tk;
        uint64_t *tv = v0; v0 = v1; v1 = tv;
    }
    for (uint64_t x = 0; x < n; ++x) {
        out_keys[x] = k0[x];
        if (out_vals) out_vals[x] = v0[x];
    }
    free(k0); free(k1); free(v0); free(v1);
    return 0;
}
