// bsort_api.cu -- host runtime behind include/bsort.h: the planner (Step 1
// parameters and the Step-9 unit), the workspace layout, the launch sequence
// of Algorithm 1 (Dehne & Zaboli, Section 4) and the error word.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <new>
#include <utility>
#include <vector>

#include <cuda.h>

#include "../../include/bsort.h"
#include "bsort_internal.h"

namespace {

using namespace bsort;

constexpr uint64_t kAlign = 256;
constexpr uint64_t kMaxN = (1ull << 32) - (1ull << 16);
// Keys-only sorts of 32-bit keys above kTwoLevelAbove keys (or wherever no
// one-level plan exists) take two levels: a top level of Algorithm 1 with
// buckets of about kTopBucket keys, each bucket then sorted by a plan of
// its own (Step 9 may use any exact sort).  (At 2^30 keys the best one-level
// plan sorts at 24 Gkeys/s, four 2^28-key buckets at about 40.)
constexpr uint64_t kTwoLevelAbove = 1ull << 30;
constexpr uint64_t kMaxTwoLevelN = 1ull << 34;
constexpr uint64_t kTopBucket = 1ull << 28;
constexpr uint64_t kMaxSamples = 8192;  // s per sublist (Step 6 keeps 12*s bytes in SMEM)
constexpr int kMaxTimed = 40;   // launches recorded per call
constexpr int kPipe = 16;       // host entry: key chunks in, position slices out
// Batches: segments up to kBatchDirectMax keys (default) are sorted whole by
// one unit; up to kBatchSampledMax by segment-aware sampling with sublists
// of kSegTile keys and s = kBatchSamples (m*s <= kRecordChunk); larger ones
// by one plain sort each.
constexpr uint32_t kBatchDirectMax = 131072;
constexpr uint32_t kBatchSampledMax = (uint32_t)kRecordChunk / 1024 * (uint32_t)kSegTile;
constexpr uint32_t kBatchSamples = 1024;
constexpr uint32_t kBatchUnit = 32768;  // Step-9 unit of sampled segments
// 64-bit keys: sublists of kSegTileU64 keys, s = 256 samples per sublist up
// to 32 sublists and 128 above (m*s <= kSegRecordsU64), Step-9 units of
// kSegTileU64 keys, so up to 64 sublists.
constexpr uint32_t kBatchSampledMaxU64 = kSegRecordsU64 / 128 * (uint32_t)kSegTileU64;
constexpr uint32_t kBatchUnitU64 = (uint32_t)kSegTileU64;
constexpr int kRing = 64;       // calls kept for bsort_kernel_times

uint64_t align_up(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Full plan of one job, including the workspace layout.
struct Plan {
    bsort_plan_info info;
    bool pairs;
    bool wide;       // 64-bit keys
    int kb;          // key bytes (4 or 8)
    int vb;          // value bytes (0 keys only)
    int tile_chunk;  // items per CTA in Step 2 (t = tile_ctas * tile_chunk)
    int unit_chunk;  // items per CTA in Step 9 (capacity = unit_ctas * unit_chunk)
    int small_chunk;  // two-tier Step 9: one-CTA units of this many items (0: one tier)
    uint32_t n_rec;      // m*s sample records
    uint32_t n_runs;     // m*b runs A_ij (counts, offsets)
    uint32_t n_rec_pad;  // rounded up to kRecordChunk
    uint32_t scan_chunks;
    // workspace offsets (bytes)
    uint64_t off_hdr, off_tiles_k, off_tiles_v, off_reloc_k, off_reloc_v, off_samples,
        off_rec_a, off_rec_b, off_spl, off_counts, off_offsets, off_status,
        off_units, off_units2, off_srcb, off_blk, off_cum, off_jr, off_rs, total;
    bool rec_radix;  // Steps 4-5 by the radix sort of the records (else chunks + merges)
    bool relocate;  // materialise Step 8 (else fused into Step 9's load)
    bool radix;     // 32768-key chunks of 32-bit keys sorted by digits
    // two-level plans (n' >= 2^32): 64-bit bucket offsets, bucket starts,
    // and the workspace of the bucket sorts
    uint64_t off_off64, off_csum, off_cpre, off_starts, off_child, child_bytes;
};

}  // namespace

struct bsort_server;  // the request loop of bsort_submit (below)

struct bsort_ctx {
    int device = 0;
    uint32_t flags = 0;
    uint32_t force_t = 0, force_s = 0, force_b = 0;
    bool auto_b = false;  // BSORT_BUCKETS_AUTO: the planner's b even when s is given
    void *ws = nullptr;
    uint64_t ws_bytes = 0;
    bool ws_owned = false;
    bool ws_fixed = false;  // caller workspace or fixed budget: never grow
    bool kernels_ready = false;
    Plan last{};
    bool have_last = false;
    char err[512] = {0};
    // timing ring: call c uses ev[c % kRing][0 .. n_ev[c % kRing]]
    cudaEvent_t ev[kRing][kMaxTimed + 1] = {};
    const char *ev_name[kMaxTimed] = {};
    int n_ev[kRing] = {};
    uint32_t direct_max = kBatchDirectMax;  // batches: largest segment sorted whole
    bool direct_max_set = false;            // direct_max given by the caller
    void *stage = nullptr;           // pinned staging of batch descriptors
    uint64_t stage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;  // last copy out of stage
    bool stage_pending = false;
    uint64_t calls_recorded = 0;  // calls since the last bsort_kernel_times
    uint64_t call_seq = 0;
    bool events_made = false;
    uint64_t serve_budget = 0;        // bytes for served requests (0: 4 GiB)
    bsort_server *server = nullptr;   // started by the first bsort_submit
    // BSORT_FLAG_GRAPHS: replayable launch sequences of plain sorts
    struct Graph {
        int kt = 0;
        uint32_t vb = 0;
        uint64_t n = 0;
        const void *kin = nullptr, *vin = nullptr;
        void *kout = nullptr, *vout = nullptr, *ws = nullptr;
        cudaStream_t st = nullptr;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<Graph> graphs;
    // BSORT_FLAG_GRAPHS for bsort_sort_batch: the launch sequence of one
    // segment table, replayed when the same table comes again; the graph
    // owns a pinned copy of the batch descriptors its first node uploads
    struct BatchGraph {
        int kt = 0;
        const void *kin = nullptr;
        void *kout = nullptr, *ws = nullptr;
        cudaStream_t st = nullptr;
        uint64_t hash = 0;
        std::vector<uint64_t> table;  // begin, n of every segment
        void *desc = nullptr;         // pinned descriptors
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<BatchGraph> batch_graphs;
    uint64_t graph_clock = 0;
    bool capturing = false;  // no timing events while a sort is captured
    // bsort_sort_keys_host: copy stream and its events (made on first use)
    cudaStream_t xfer = nullptr;
    cudaEvent_t xev[2 * kPipe + 2] = {};
    int num_sms = 0;
};

namespace {

bsort_status fail(bsort_t h, bsort_status st, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

bsort_status cuda_fail(bsort_t h, cudaError_t e, const char *what)
{
    return fail(h, BSORT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Largest bucket with b splitters taken from the m*s samples: a bucket
// spans at most ceil(m*s/b) sample ranks, w items each, plus w-1 items of
// every other sublist (for b = s: n'/s + (m-1)(w-1), Lemma 1).
uint64_t bound_for(uint64_t n_pad, uint64_t m, uint64_t s, uint64_t b)
{
    const uint64_t t = n_pad / m;
    const uint64_t w = t / s;
    return (m * s + b - 1) / b * w + (m - 1) * (w - 1);
}

// Bucket count for a plan whose units hold Q items: at least the smallest b
// whose bound fits Q, else about (k + 0.1) buckets per unit for the smallest
// whole k that allows it, so that greedy packing fills units to ~k/(k+0.1)
// instead of leaving a unit with one bucket when two nearly fit.  Returns 0
// when no b <= bmax keeps every bucket within Q.
uint64_t choose_buckets(uint64_t np, uint64_t m, uint64_t s, uint64_t Q, uint64_t bmax)
{
    if (bound_for(np, m, s, bmax) > Q) return 0;
    uint64_t lo = 1, hi = bmax;  // smallest b with bound <= Q (bound falls with b)
    while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (bound_for(np, m, s, mid) <= Q) hi = mid;
        else lo = mid + 1;
    }
    for (uint64_t k = 1;; ++k) {
        const uint64_t b = ((10 * k + 1) * np + 10 * Q - 1) / (10 * Q);
        if (b >= bmax) return bmax;
        if (b >= lo) return b;
    }
}

// Spread of bucket sizes on random keys: each of the m sublists adds a
// uniform error in [0, w) at both ends of a bucket, so its size varies by
// about sigma = w * sqrt(m / 6).
double bucket_sigma(uint64_t m, uint64_t w) { return (double)w * __builtin_sqrt((double)m / 6.0); }

// Average bucket a two-tier Step 9 aims at: four sigmas below one CTA's Q1
// items, so that hardly any bucket spills into the cluster tier.
uint64_t two_tier_target(uint64_t m, uint64_t w, uint64_t Q1)
{
    const double a = (double)Q1 - 4.0 * bucket_sigma(m, w);
    return a > 0 ? (uint64_t)a : 0;
}

// Bucket count for a two-tier Step 9 (one-CTA units of Q1 items, cluster
// units of Q2 >= bound for the rest): at least the smallest b whose bound
// fits Q2, else the b whose average bucket is two_tier_target, so that
// nearly every bucket fills a one-CTA unit alone.  Returns 0 when no
// b <= bmax fits Q2.
uint64_t choose_buckets_two_tier(uint64_t np, uint64_t m, uint64_t s, uint64_t Q1, uint64_t Q2,
                                 uint64_t bmax)
{
    if (bound_for(np, m, s, bmax) > Q2) return 0;
    uint64_t lo = 1, hi = bmax;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (bound_for(np, m, s, mid) <= Q2) hi = mid;
        else lo = mid + 1;
    }
    const uint64_t avg = two_tier_target(m, np / m / s, Q1);
    const uint64_t b = avg ? (np + avg - 1) / avg : bmax;
    return b > bmax ? bmax : (b < lo ? lo : b);
}

// Whether bucket sizes are regular enough for a two-tier Step 9: the
// average bucket four sigmas below Q1 must still fill at least 90% of it
// (89% for 64-bit keys, whose alternative is a tier of 8-CTA merge units:
// measured at 2^28 keys, t = 65536 with one-CTA units of 89% fill sorts in
// 20.2 ms, t = 131072 with w = 16 in 23.1 ms).
bool tiers_regular(uint64_t m, uint64_t w, uint64_t Q1, bool wide)
{
    return 4.0 * bucket_sigma(m, w) <= (wide ? 0.11 : 0.10) * (double)Q1;
}

// Sort-unit shapes (items per CTA) and cluster sizes the kernels provide.
const int kChunks[] = {2048, 4096, 8192, 16384, 32768};
const int kClusters[] = {1, 2, 4, 8};

int max_chunk(bool pairs) { return pairs ? kMaxCapPairs : kMaxCapKeys; }

// Smallest unit (chunk, ctas) holding `items`: one CTA with the smallest
// chunk that fits, else a cluster of the largest chunk.  Returns false if
// even the largest cluster is too small.
bool unit_for(uint64_t items, bool pairs, int *chunk, int *ctas)
{
    const int cm = max_chunk(pairs);
    for (int c : kChunks) {
        if (c > cm) break;
        if ((uint64_t)c >= items) {
            *chunk = c;
            *ctas = 1;
            return true;
        }
    }
    for (int k : kClusters) {
        if ((uint64_t)k * cm >= items) {
            *chunk = cm;
            *ctas = k;
            return true;
        }
    }
    return false;
}

// Sublist size t -> (chunk, ctas): t <= max chunk is one CTA, larger t a
// cluster of max-chunk CTAs.
bool tile_shape(uint64_t t, bool pairs, int *chunk, int *ctas)
{
    const int cm = max_chunk(pairs);
    for (int c : kChunks)
        if (c <= cm && (uint64_t)c == t) {
            *chunk = c;
            *ctas = 1;
            return true;
        }
    for (int k : kClusters)
        if (k > 1 && (uint64_t)k * cm == t) {
            *chunk = cm;
            *ctas = k;
            return true;
        }
    return false;
}

double log2d(double x) { return x > 1 ? __builtin_log2(x) : 0.0; }

// Modelled cost of a plan, in units of about 8.1 ps (one unit per key is
// one single-CTA sort pass over 32K-key chunks).  The factors are measured
// on GB300 at n = 2^28 uint32 keys: a Step-2 sublist sorted by one CTA or
// a cluster of 2 / 4 / 8 CTAs costs 1.04 / 1.29 / 1.75 / 2.6 passes
// (distributed-shared-memory merge rounds; 8-CTA clusters also leave SMs
// idle); Step 9 costs 1.1 passes with one-CTA units (one tier of one CTA,
// or two tiers) and 1.65 / 2.1 / 3.1 with cluster units (rounds plus unit
// fill).  Step 4 costs 6.8 units per sample; Steps 6-8 0.325 per key plus
// 1.85 per run A_ij (m*b of them), and 4 more per run when a 1024-position
// block of the relocation meets more runs than it stages (more than ~200
// on average).  64-bit keys keep the sample-window Step 6 (3.9 per run).
double plan_cost(uint64_t np, uint64_t s, uint64_t runs, int tchunk, int tctas, int uchunk,
                 int uctas, bool wide)
{
    const double n = (double)np;
    auto f1 = [](int c) { return c == 1 ? 1.04 : c == 2 ? 1.29 : c == 4 ? 1.75 : 2.6; };
    auto f9 = [](int c) { return c == 1 ? 1.1 : c == 2 ? 1.65 : c == 4 ? 2.1 : 3.1; };
    const double chunk_levels = log2d(tchunk) / 15.0;  // smaller chunks sort faster
    const double unit_levels = log2d(uchunk) / 15.0;
    const double t = (double)tchunk * tctas;
    const double w = t / (double)s;
    const double samples = n / w;
    const double r = (double)runs;
    if (wide)
        return n * (f1(tctas) * chunk_levels + f9(uctas) * unit_levels + (w >= 32 ? 0.3 : 0.35)) +
               7.0 * samples + 3.9 * r;
    const double per_run = 1.85 + (1024.0 * r > 200.0 * n ? 4.0 : 0.0);
    return n * (f1(tctas) * chunk_levels + f9(uctas) * unit_levels + 0.325) + 6.8 * samples +
           per_run * r;
}

// Measured plans for keys-only sorts of 32-bit keys whose Step-9 units
// (and sublists of t = 32768) are radix-sorting CTAs: (t, s) per size
// class of n, the fastest of a sweep of t in {32768, 65536, 131072} and s in
// {512, ..., 8192} on GB300 (uniform keys; b chosen by the planner for each
// pair, as below).  Sizes outside the table use the cost model.
struct TunedPlan {
    int log2n_max;  // n <= 2^log2n_max
    uint32_t t, s;
};
const TunedPlan kTuned[] = {
#include "bsort_tuned.inc"
};

bool tuned_plan(uint64_t n, uint64_t *t, uint64_t *s)
{
    for (const TunedPlan &e : kTuned) {
        if (n <= (1ull << e.log2n_max)) {
            *t = e.t;
            *s = e.s;
            return true;
        }
    }
    return false;
}

bsort_status make_plan_with(bsort_t h, bsort_key_type kt, uint32_t vb, uint64_t n, Plan *P,
                            bool use_table);

// Plan of n >= kMaxN 32-bit keys (keys only): the top level sorts sublists of
// t = 32768 (one CTA each), takes b buckets of about kTopBucket keys, and the
// largest sample distance w whose share of the bucket bound, (m-1)(w-1),
// stays within a quarter of the average bucket; Step 9 sorts each bucket by
// a plan of its own in a slice of the workspace sized for the bound.
bsort_status make_plan(bsort_t h, bsort_key_type kt, uint32_t vb, uint64_t n, Plan *P);

bsort_status make_plan_two_level(bsort_t h, bsort_key_type kt, uint64_t n, Plan *P)
{
    P->pairs = false;
    P->wide = false;
    P->kb = 4;
    P->vb = 0;
    P->relocate = true;
    P->radix = !(h && (h->flags & BSORT_FLAG_MERGE_SORT));
    bsort_plan_info &I = P->info;
    const uint64_t t = 32768;
    const uint64_t m = (n + t - 1) / t;
    const uint64_t np = m * t;
    // (BSORT_FLAG_TEST_TWO_LEVEL: buckets of about 2^16 keys, so that small
    // inputs take many of them)
    const uint64_t top = h && (h->flags & BSORT_FLAG_TEST_TWO_LEVEL) ? (1ull << 16) : kTopBucket;
    uint64_t b = (np + top - 1) / top;
    if (b < 2) b = 2;
    uint64_t w = 1;
    while (w * 2 <= t && (m - 1) * (w * 2 - 1) <= np / (4 * b)) w *= 2;
    const uint64_t s = t / w;
    if (m * s >= (1ull << 32) || m * b >= (1ull << 32))
        return fail(h, BSORT_EUNSUPPORTED, "n = %llu: too many samples", (unsigned long long)n);
    I.n = n;
    I.n_padded = np;
    I.t = (uint32_t)t;
    I.s = (uint32_t)s;
    I.m = (uint32_t)m;
    I.w = (uint32_t)w;
    I.b = (uint32_t)b;
    I.bucket_bound = bound_for(np, m, s, b);
    if (I.bucket_bound >= kMaxN)
        return fail(h, BSORT_EUNSUPPORTED, "n = %llu: bucket bound %llu too large",
                    (unsigned long long)n, (unsigned long long)I.bucket_bound);
    I.tile_ctas = 1;
    I.levels = 2;
    P->tile_chunk = (int)t;
    // the bucket sorts: a plan for the bound, with a quarter more room
    bsort_ctx child;
    child.device = h ? h->device : 0;
    child.flags = h ? (h->flags & (BSORT_FLAG_MERGE_SORT | BSORT_FLAG_PLAN_MODEL)) : 0;
    Plan C;
    bsort_status rs = make_plan(&child, BSORT_U32, 0, I.bucket_bound, &C);
    if (rs != BSORT_OK)
        return fail(h, rs, "n = %llu: no plan for a bucket of %llu keys", (unsigned long long)n,
                    (unsigned long long)I.bucket_bound);
    P->child_bytes = align_up(C.total + C.total / 4 + (1u << 20));
    I.unit_ctas = C.info.single_tile ? C.info.unit_ctas : 0;
    I.unit_capacity = I.bucket_bound;
    P->n_rec = (uint32_t)(m * s);
    P->n_runs = (uint32_t)(m * b);
    P->n_rec_pad = (uint32_t)((P->n_rec + kRecordChunk - 1) / kRecordChunk * kRecordChunk);
    uint32_t merges = 0;
    for (uint32_t L = kRecordChunk; L < P->n_rec_pad; L <<= 1) ++merges;
    I.num_kernels = 1 + 1 + merges + (merges ? 1 : 0) + 2 /*S6*/ + 3 /*S7*/ + 2 /*S8*/ +
                    (uint32_t)b * C.info.num_kernels;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const uint32_t chunks = (P->n_runs + kScanChunk - 1) / kScanChunk;
    P->off_hdr = take(kAlign);
    P->off_tiles_k = take(np * 4);
    P->off_reloc_k = take(np * 4);
    P->off_samples = take((uint64_t)P->n_rec * 8);
    P->off_rec_a = take((uint64_t)P->n_rec_pad * 8);
    P->off_rec_b = take(P->n_rec_pad > (uint32_t)kRecordChunk ? (uint64_t)P->n_rec_pad * 8 : 0);
    P->off_spl = take(b * 8);
    P->off_cum = take((uint64_t)P->n_runs * 4);
    P->off_jr = take(sample_index_scratch_words(I.t, I.m) * 4);
    P->off_off64 = take(((uint64_t)P->n_runs + 1) * 8);
    P->off_csum = take((uint64_t)chunks * 4);
    P->off_cpre = take((uint64_t)chunks * 8);
    P->off_starts = take((b + 1) * 8);
    P->off_child = take(P->child_bytes);
    P->total = o;
    I.workspace_bytes = o;
    return BSORT_OK;
}

// The plan of one job: the tabled (t, s) for n's size class when there is
// one and it admits a plan, else the cost model's choice; keys-only sorts
// of 32-bit keys that no one-level plan fits take two levels.
bsort_status make_plan(bsort_t h, bsort_key_type kt, uint32_t vb, uint64_t n, Plan *P)
{
    bsort_status st = make_plan_with(h, kt, vb, n, P, true);
    if (st == BSORT_EUNSUPPORTED) st = make_plan_with(h, kt, vb, n, P, false);
    const bool forced = h && (h->force_t || h->force_s || h->force_b);
    if (st == BSORT_EUNSUPPORTED && vb == 0 && kt != BSORT_U64 && n > (1ull << 28) && !forced &&
        n <= kMaxTwoLevelN) {
        memset(P, 0, sizeof(*P));
        st = make_plan_two_level(h, kt, n, P);
    }
    return st;
}

bsort_status make_plan_with(bsort_t h, bsort_key_type kt, uint32_t vb, uint64_t n, Plan *P,
                            bool use_table)
{
    memset(P, 0, sizeof(*P));
    P->info.levels = 1;
    if (kt != BSORT_U32 && kt != BSORT_F32 && kt != BSORT_U64)
        return fail(h, BSORT_EINVAL, "unknown key type %d", (int)kt);
    if (vb != 0 && vb != 4 && vb != 8) return fail(h, BSORT_EINVAL, "val_bytes must be 0, 4 or 8");
    if (kt == BSORT_U64 && vb != 0)
        return fail(h, BSORT_EUNSUPPORTED, "64-bit keys are sorted keys-only (no values)");
    const bool force_two = h && (h->flags & BSORT_FLAG_TEST_TWO_LEVEL) && vb == 0 &&
                           kt != BSORT_U64 && n > 2 * 32768;
    const bool big_keys = vb == 0 && kt != BSORT_U64 && n > kTwoLevelAbove &&
                          !(h && (h->force_t || h->force_s || h->force_b));
    if (force_two || (big_keys && n <= kMaxTwoLevelN)) return make_plan_two_level(h, kt, n, P);
    if (n >= kMaxN) {
        if (vb != 0 || kt == BSORT_U64)
            return fail(h, BSORT_EUNSUPPORTED,
                        "n = %llu: from 2^32 - 2^16 keys on, only keys-only sorts of 32-bit keys",
                        (unsigned long long)n);
        if (n > kMaxTwoLevelN)
            return fail(h, BSORT_EUNSUPPORTED, "n = %llu exceeds 2^34", (unsigned long long)n);
        return make_plan_two_level(h, kt, n, P);
    }
    // 64-bit keys and pairs sort 64-bit words: the smaller chunk shapes
    const bool pairs = vb != 0 || kt == BSORT_U64;
    const int cm = max_chunk(pairs);
    P->pairs = vb != 0;
    P->wide = kt == BSORT_U64;
    P->kb = P->wide ? 8 : 4;
    P->vb = (int)vb;
    bsort_plan_info &I = P->info;
    I.n = n;
    uint64_t forced_t = h ? h->force_t : 0;
    uint64_t forced_s = h ? h->force_s : 0;
    const uint64_t forced_b = h ? h->force_b : 0;
    bool auto_b = h ? h->auto_b : false;  // b chosen below even if s is forced
    if (forced_b > (uint64_t)kMaxBuckets)
        return fail(h, BSORT_EUNSUPPORTED, "b = %llu exceeds %d buckets",
                    (unsigned long long)forced_b, kMaxBuckets);
    int uchunk = 0, uctas = 0;

    if (forced_t == 0 && forced_s == 0 && forced_b == 0 && unit_for(n, pairs, &uchunk, &uctas) ||
        (forced_t && n <= forced_t && unit_for(n, pairs, &uchunk, &uctas))) {
        // c7: n fits one Step-9 unit; the sort needs no sampling.
        I.single_tile = 1;
        I.n_padded = n;
        I.t = (uint32_t)n;
        I.s = 1;
        I.b = 1;
        I.m = n ? 1 : 0;
        I.w = (uint32_t)n;
        I.bucket_bound = n;
        I.tile_ctas = 0;
        I.unit_ctas = n ? (uint32_t)uctas : 0;
        P->unit_chunk = uchunk;
        I.unit_capacity = (uint64_t)uchunk * uctas;
        I.num_kernels = n > 1 ? 1 : 0;
    } else {
        // keys-only 32-bit sorts with radix units take (t, s) from the table
        // measured for n's size class; the bucket count is then chosen below
        // as for any plan
        const bool radix_ok = vb == 0 && kt != BSORT_U64 &&
                              !(h && (h->flags & (BSORT_FLAG_MERGE_SORT | BSORT_FLAG_PLAN_MODEL)));
        uint64_t tt = 0, ts = 0;
        if (use_table && radix_ok && !forced_t && !forced_s && !forced_b &&
            tuned_plan(n, &tt, &ts)) {
            forced_t = tt;
            forced_s = ts;
            auto_b = true;
        }
        // candidates: forced t or every sublist shape; forced s or every
        // power of two with w = t/s >= 16 and s <= kMaxSamples.  The unit is
        // sized for b = s (or the forced b); the bucket count is chosen after.
        const bool wide = kt == BSORT_U64;
        double best = -1.0;
        uint64_t bt = 0, bs = 0;
        int btc = 0, btk = 0, buc = 0, buk = 0;
        const uint64_t tlist[] = {2048, 4096, 8192, 16384, 32768, 65536, 131072, 262144};
        for (uint64_t t : tlist) {
            if (forced_t && t != forced_t) continue;
            int tc, tk;
            if (!tile_shape(t, pairs, &tc, &tk)) continue;
            if (!forced_t && t < (uint64_t)cm) continue;  // smaller sublists only on request
            const uint64_t m = (n + t - 1) / t;
            const uint64_t np = m * t;
            if (np >= kMaxN) continue;
            for (uint64_t sv = 1; sv <= t; sv <<= 1) {
                if (forced_s ? sv != forced_s : (sv > kMaxSamples || t / sv < 16)) continue;
                const uint64_t bv = forced_b ? forced_b : sv;
                if (bv > m * sv) continue;
                const uint64_t bound = bound_for(np, m, sv, bv);
                int uc, uk;
                if (!unit_for(bound, pairs, &uc, &uk)) continue;
                // Step 9 as planned below: two tiers (one-CTA units) when the
                // bound needs a cluster and b can reach ~1.05 buckets per
                // one-CTA unit; the bucket count estimated the same way
                // (two tiers: a unit per bucket, up to kMaxBucketsTiers buckets)
                const uint64_t bmx = m * sv < (uint64_t)kMaxBucketsTiers ? m * sv
                                                                         : (uint64_t)kMaxBucketsTiers;
                const uint64_t tgt = two_tier_target(m, t / sv, (uint64_t)cm);
                const uint64_t b2 = tgt ? (np + tgt - 1) / tgt : bmx + 1;
                const bool tiers = uk > 1 && !forced_b && (!forced_s || auto_b) && b2 <= bmx &&
                                   bound_for(np, m, sv, b2) <= (uint64_t)uc * uk &&
                                   tiers_regular(m, t / sv, (uint64_t)cm, wide);
                const uint64_t b_est = forced_b ? forced_b : (forced_s && !auto_b) ? sv
                                       : tiers ? b2 : (21 * np + 10ull * uc * uk - 1) / (10ull * uc * uk);
                // (the cluster tier's launch costs ~40 us even when nearly empty)
                const double c = tiers ? plan_cost(np, sv, m * b_est, tc, tk, cm, 1, wide) + 5e6
                                       : plan_cost(np, sv, m * b_est, tc, tk, uc, uk, wide);
                if (best < 0 || c < best) {
                    best = c;
                    bt = t; bs = sv; btc = tc; btk = tk; buc = uc; buk = uk;
                }
            }
            if (forced_s && !bs) {
                if (forced_s > t || t % forced_s != 0)
                    return fail(h, BSORT_EINVAL, "s = %llu must divide t = %llu",
                                (unsigned long long)forced_s, (unsigned long long)t);
            }
        }
        if (forced_t && !bt && !forced_s) {
            int tc, tk;
            if (!tile_shape(forced_t, pairs, &tc, &tk))
                return fail(h, BSORT_EUNSUPPORTED, "sublist size t = %llu not supported",
                            (unsigned long long)forced_t);
        }
        if (!bt) {
            if (forced_t && forced_s) {
                const uint64_t m = (n + forced_t - 1) / forced_t;
                const uint64_t bv = forced_b ? forced_b : forced_s;
                if (bv > m * forced_s)
                    return fail(h, BSORT_EINVAL, "b = %llu exceeds the m*s = %llu samples",
                                (unsigned long long)bv, (unsigned long long)(m * forced_s));
                return fail(h, BSORT_EUNSUPPORTED,
                            "bucket bound %llu exceeds the largest Step-9 unit (%d items)",
                            (unsigned long long)bound_for(m * forced_t, m, forced_s, bv), 8 * cm);
            }
            return fail(h, BSORT_EUNSUPPORTED, "no plan keeps every bucket within a Step-9 unit");
        }
        const uint64_t m = (n + bt - 1) / bt;
        I.single_tile = 0;
        I.n_padded = m * bt;
        I.t = (uint32_t)bt;
        I.s = (uint32_t)bs;
        I.m = (uint32_t)m;
        I.w = (uint32_t)(bt / bs);
        I.tile_ctas = (uint32_t)btk;
        I.unit_ctas = (uint32_t)buk;
        P->tile_chunk = btc;
        P->unit_chunk = buc;
        I.unit_capacity = (uint64_t)buc * buk;
        // Step 9 in two tiers when the bound needs a cluster and the
        // average bucket is at most 1/1.05 of the largest one-CTA unit:
        // one-CTA units for the buckets that fit it (nearly all), cluster
        // units only for the others.  A free b is chosen for that when it can
        // be (at most bmax buckets).
        // (one tier packs buckets greedily in one CTA: at most kMaxBuckets;
        // two tiers make every bucket a unit: at most kMaxBucketsTiers)
        const uint64_t bmax = m * bs < (uint64_t)kMaxBuckets ? m * bs : (uint64_t)kMaxBuckets;
        const uint64_t bmax2 = m * bs < (uint64_t)kMaxBucketsTiers ? m * bs
                                                                   : (uint64_t)kMaxBucketsTiers;
        const uint64_t tgt = two_tier_target(m, bt / bs, (uint64_t)cm);
        const bool tiers_wanted = buk > 1 && tgt && (I.n_padded + tgt - 1) / tgt <= bmax2 &&
                                  tiers_regular(m, bt / bs, (uint64_t)cm, wide);
        uint64_t b = bs;  // the paper's rule, kept when s is given
        if (forced_b) {
            b = forced_b;
        } else if (!forced_s || auto_b) {
            const uint64_t bc =
                tiers_wanted ? choose_buckets_two_tier(I.n_padded, m, bs, (uint64_t)cm,
                                                       I.unit_capacity, bmax2)
                             : choose_buckets(I.n_padded, m, bs, I.unit_capacity, bmax);
            if (bc) b = bc;
        }
        if (buk > 1 && 105 * I.n_padded <= 100 * (uint64_t)cm * b &&
            tiers_regular(m, bt / bs, (uint64_t)cm, wide)) {  // average at most Q1/1.05
            P->small_chunk = cm;
            I.unit_small = (uint32_t)cm;
        } else if (b > (uint64_t)kMaxBuckets) {
            // one tier after all: the greedy packing's bucket limit holds
            const uint64_t bc = choose_buckets(I.n_padded, m, bs, I.unit_capacity, bmax);
            b = bc ? bc : bs;
        }
        I.b = (uint32_t)b;
        I.bucket_bound = bound_for(I.n_padded, m, bs, b);
        P->n_rec = (uint32_t)(m * bs);
        P->n_runs = (uint32_t)(m * b);
        P->n_rec_pad = (uint32_t)((P->n_rec + kRecordChunk - 1) / kRecordChunk * kRecordChunk);
        P->scan_chunks = (P->n_runs + kScanChunk - 1) / kScanChunk;
        const bool reloc = P->wide || !(h && (h->flags & BSORT_FLAG_LOW_MEMORY));
        const uint32_t s9 = P->small_chunk ? 2 : 1;  // Step-9 launches
        if (P->wide) {
            // records (16 bytes) merged from runs of s: ceil(log2 m) passes
            P->n_rec_pad = P->n_rec;
            uint32_t merges = 0;
            for (uint64_t L = bs; L < P->n_rec; L <<= 1) ++merges;
            I.num_kernels = 1 /*S2-3*/ + merges + 1 /*S5*/ + 2 /*S6*/ + 1 /*S7*/ +
                            1 /*run index*/ + 1 /*S8*/ + 1 /*units*/ + s9;
        } else {
            uint32_t merges = 0;
            for (uint32_t L = kRecordChunk; L < P->n_rec_pad; L <<= 1) ++merges;
            P->rec_radix = P->n_rec_pad > (uint32_t)kRecordChunk &&
                           records_radix_fits(P->n_rec, I.b);
            const uint32_t s45 = P->rec_radix
                                     ? 5u  /*histogram, four digit passes*/
                                     : 1u + merges + (merges ? 1u : 0u);  /*chunks, merges, S5*/
            const uint32_t s78 = reloc && bucket_relocate_fits(I.m)
                                     ? 1u                              /*S7-8 fused*/
                                     : 1u + 1u + (reloc ? 1u : 0u);    /*S7, run index, S8*/
            I.num_kernels = 1 /*S2-3*/ + s45 + 2 /*S6*/ + s78 + 1 /*units*/ + s9;
        }
    }

    // workspace layout
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P->relocate = P->wide || !(h && (h->flags & BSORT_FLAG_LOW_MEMORY));
    P->radix = !P->pairs && !P->wide && !(h && (h->flags & BSORT_FLAG_MERGE_SORT));
    P->off_hdr = take(kAlign);  // error word (int) + scan ticket (uint32)
    if (!I.single_tile) {
        const uint64_t np = I.n_padded;
        const uint64_t kb = (uint64_t)P->kb;
        const uint64_t rb = P->wide ? 16 : 8;  // sample record bytes
        P->off_tiles_k = take(np * kb);
        P->off_tiles_v = take(np * (uint64_t)vb);
        P->off_reloc_k = take(P->relocate ? np * kb : 0);
        P->off_reloc_v = take(P->relocate ? np * (uint64_t)vb : 0);
        P->off_samples = take((uint64_t)P->n_rec * rb);
        P->off_rec_a = take((uint64_t)P->n_rec_pad * rb);
        P->off_rec_b = take(P->wide || P->n_rec_pad > (uint32_t)kRecordChunk
                                ? (uint64_t)P->n_rec_pad * rb : 0);
        P->off_spl = take((uint64_t)I.b * rb);
        P->off_counts = take(0);  // a_ij are read back as offset differences
        P->off_offsets = take(((uint64_t)P->n_runs + 1) * 4);
        P->off_status = take((uint64_t)P->scan_chunks * 8);
        P->off_units = take((1 + 2 * (uint64_t)I.b) * 4);
        P->off_units2 = take(P->small_chunk ? (1 + 2 * (uint64_t)I.b) * 4 : 0);
        P->off_srcb = take((uint64_t)P->n_runs * 4);
        P->off_blk = take((np + kBlockItems - 1) / kBlockItems * 4);
        // Step 6: cumulative counts and segment ranges
        P->off_cum = take((uint64_t)P->n_runs * 4);
        P->off_jr = take(sample_index_scratch_words(I.t, I.m, P->wide ? 4096u : 1024u) * 4);
        P->off_rs = take(P->rec_radix ? records_radix_scratch_bytes(P->n_rec) : 0);
    }
    P->total = o;
    I.workspace_bytes = o;
    return BSORT_OK;
}

// Grid (in units) of the cluster tier of a two-tier Step 9: units above q1
// items are at most n_pad / (q1 + 1) and at most one per bucket.
// (The launch covers at most 256 units at a time; its clusters then loop.)
uint32_t large_units_max(uint64_t n_pad, uint32_t q1, uint32_t b)
{
    uint64_t u = n_pad / ((uint64_t)q1 + 1);
    if (u > b) u = b;
    return (uint32_t)(u < 256 ? u : 256);
}

void drop_graphs(bsort_t h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (auto &g : h->batch_graphs) {
        cudaGraphExecDestroy(g.exec);
        if (g.desc) cudaFreeHost(g.desc);
    }
    h->batch_graphs.clear();
}

bsort_status ensure_workspace(bsort_t h, uint64_t bytes)
{
    if (bytes <= h->ws_bytes) return BSORT_OK;
    if (h->ws_fixed)
        return fail(h, BSORT_ENOMEM, "job needs %llu workspace bytes, handle has %llu",
                    (unsigned long long)bytes, (unsigned long long)h->ws_bytes);
    drop_graphs(h);  // they point into the old workspace
    if (h->ws_owned && h->ws) {
        cudaError_t e = cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFree(workspace)");
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, BSORT_ENOMEM, "cudaMalloc(%llu) failed: %s", (unsigned long long)bytes,
                    cudaGetErrorString(e));
    }
    h->ws = p;
    h->ws_bytes = bytes;
    h->ws_owned = true;
    // the error word starts cleared
    e = cudaMemset(p, 0, kAlign);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset(header)");
    return BSORT_OK;
}

bsort_status prepare(bsort_t h)
{
    if (!h) return BSORT_EINVAL;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!h->kernels_ready) {
        e = init_kernels();
        if (e != cudaSuccess) return cuda_fail(h, e, "kernel attributes");
        h->kernels_ready = true;
    }
    if (h->num_sms == 0) {
        e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return cuda_fail(h, e, "multiprocessor count");
    }
    if ((h->flags & BSORT_FLAG_TIMING) && !h->events_made) {
        for (int r = 0; r < kRing; ++r)
            for (int i = 0; i <= kMaxTimed; ++i) {
                e = cudaEventCreate(&h->ev[r][i]);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
            }
        h->events_made = true;
    }
    return BSORT_OK;
}

// Launch-sequence helper: with BSORT_FLAG_TIMING, records an event before
// the first launch and after each launch of the call, in the next slot of
// the handle's ring.
struct Seq {
    bsort_t h;
    cudaStream_t st;
    bool timing;
    int slot = 0;
    int n = 0;
    Seq(bsort_t h_, cudaStream_t st_)
        : h(h_), st(st_), timing((h_->flags & BSORT_FLAG_TIMING) != 0 && !h_->capturing)
    {
        if (!timing) return;
        slot = (int)(h->call_seq % kRing);
        ++h->call_seq;
        if (h->calls_recorded < (uint64_t)kRing) ++h->calls_recorded;
        h->n_ev[slot] = 0;
        cudaEventRecord(h->ev[slot][0], st);
    }
    bsort_status after(cudaError_t e, const char *name)
    {
        if (e != cudaSuccess) return cuda_fail(h, e, name);
        if (timing && n < kMaxTimed) {
            h->ev_name[n] = name;
            cudaEventRecord(h->ev[slot][n + 1], st);
            ++n;
            h->n_ev[slot] = n;
        }
        return BSORT_OK;
    }
};

#define SEQ(call, name)                                  \
    do {                                                 \
        bsort_status s_ = seq.after((call), (name));     \
        if (s_ != BSORT_OK) return s_;                   \
    } while (0)

// Host buffers of bsort_sort_keys_host, overlapped with the sort: the keys
// arrive in G chunks of whole sublists and Steps 1-3 start on each chunk
// once it is on the device; Step 9 runs in G groups, group g sorting the
// units that begin in position slice [g n'/G, (g+1) n'/G), and that
// slice goes back to the host while the next group sorts (every position of
// the slice lies in a unit that begins at or before it).  Copies run on the
// handle's copy stream, ordered against the caller's stream by events.
struct HostPipe {
    const void *h_in;
    void *h_out;
    void *d_keys;      // device staging of the keys (the sort runs in place)
    uint32_t *ranges;  // device: 2 (kPipe + 1) unit indices
    int groups;        // chunks in and slices out, at most kPipe
};

// Chunks of the overlapped host entry for n 32-bit keys: one per 8 MiB of
// keys, at most kPipe; 0 below 32 MiB, where the copies are too short for
// the extra calls (about a hundred) to pay.
int host_pipe_groups(uint64_t n)
{
    const uint64_t g = n * 4 / (8ull << 20);
    if (g < 4) return 0;
    return g > (uint64_t)kPipe ? kPipe : (int)g;
}

bsort_status ensure_pipe(bsort_t h)
{
    if (h->xfer) return BSORT_OK;
    cudaError_t e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "multiprocessor count");
    // all or nothing: a failed call leaves no events behind to leak on the next
    cudaEvent_t ev[2 * kPipe + 2] = {};
    cudaStream_t xs = nullptr;
    for (int i = 0; i < 2 * kPipe + 2 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        return cuda_fail(h, e, "copy stream and events of the host entry");
    }
    for (int i = 0; i < 2 * kPipe + 2; ++i) h->xev[i] = ev[i];
    h->xfer = xs;
    return BSORT_OK;
}

// the stream `to` waits for the work issued so far on `from`
cudaError_t stream_after(cudaStream_t to, cudaStream_t from, cudaEvent_t ev)
{
    cudaError_t e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    return e;
}

// Algorithm 1 on 64-bit keys (keys only): the same steps with 64-bit sorted
// sublists and buckets and 16-byte sample records merged in L2 (Step 4).
bsort_status run_sort(bsort_t h, bsort_key_type kt, const void *kin, const void *vin, void *kout,
                      void *vout, uint32_t vb, uint64_t n, cudaStream_t st,
                      const HostPipe *hp = nullptr);

// A two-level plan (n' >= 2^32, keys-only 32-bit keys): Steps 1-6 as in
// run_sort over sublists of 32768 keys, Steps 7-8 with 64-bit offsets
// (relocation by source: the top-level runs are long), then the b bucket
// sizes are read back (one wait for the stream) and Step 9 sorts every
// bucket with a plan of its own, in a slice of the workspace, as 32-bit
// keys (float keys are still in their order-preserving code and are decoded
// in the output).
bsort_status run_sort_two_level(bsort_t h, const Plan &P, bsort_key_type kt, const void *kin,
                                void *kout, uint64_t n, cudaStream_t st, Seq &seq)
{
    const bsort_plan_info &I = P.info;
    unsigned char *ws = static_cast<unsigned char *>(h->ws);
    int *err = reinterpret_cast<int *>(ws + P.off_hdr);
    const int is_f32 = kt == BSORT_F32;
    uint32_t *tiles_k = reinterpret_cast<uint32_t *>(ws + P.off_tiles_k);
    uint32_t *reloc_k = reinterpret_cast<uint32_t *>(ws + P.off_reloc_k);
    uint64_t *samples = reinterpret_cast<uint64_t *>(ws + P.off_samples);
    uint64_t *rec_a = reinterpret_cast<uint64_t *>(ws + P.off_rec_a);
    uint64_t *rec_b = reinterpret_cast<uint64_t *>(ws + P.off_rec_b);
    uint64_t *spl = reinterpret_cast<uint64_t *>(ws + P.off_spl);
    uint32_t *cum = reinterpret_cast<uint32_t *>(ws + P.off_cum);
    uint32_t *jr = reinterpret_cast<uint32_t *>(ws + P.off_jr);
    uint64_t *off64 = reinterpret_cast<uint64_t *>(ws + P.off_off64);
    uint32_t *csum = reinterpret_cast<uint32_t *>(ws + P.off_csum);
    uint64_t *cpre = reinterpret_cast<uint64_t *>(ws + P.off_cpre);
    uint64_t *starts = reinterpret_cast<uint64_t *>(ws + P.off_starts);
    unsigned char *child_ws = ws + P.off_child;
    // Steps 1-3
    SEQ(launch_sublist_sort_keys(P.tile_chunk, 1, kin, n, I.m, is_f32, I.s, tiles_k, samples, st,
                                 0, P.radix),
        "step1_3_sublist_sort");
    // Steps 4-5
    const bool one_chunk = P.n_rec_pad == (uint32_t)kRecordChunk;
    SEQ(launch_records_chunk_sort(samples, rec_a, P.n_rec, P.n_rec_pad, one_chunk ? spl : nullptr,
                                  I.s, I.b, st),
        "step4_sample_chunks");
    if (!one_chunk) {
        uint64_t *src = rec_a, *dst = rec_b;
        for (uint32_t L = kRecordChunk; L < P.n_rec_pad; L <<= 1) {
            SEQ(launch_merge_pass(src, dst, P.n_rec_pad, L, st), "step4_sample_merge");
            std::swap(src, dst);
        }
        SEQ(launch_select_splitters(src, P.n_rec, I.b, spl, st), "step5_splitters");
    }
    // Step 6
    SEQ(launch_sample_index(tiles_k, spl, I.t, I.s, I.b, I.m, jr, cum, st), "step6_sample_index");
    // Step 7 (64-bit offsets) and Step 8 (by source)
    SEQ(launch_scan_cum64(cum, I.m, P.n_runs, csum, cpre, I.n_padded, off64, st),
        "step7_prefix_sum");
    SEQ(launch_relocate_src64(tiles_k, cum, off64, I.m, I.b, I.t, reloc_k, st), "step8_relocate");
    SEQ(launch_bucket_starts64(off64, I.m, I.b, I.n_padded, starts, st), "step9_bucket_starts");
    std::vector<uint64_t> hs(I.b + 1);
    cudaError_t e = cudaMemcpyAsync(hs.data(), starts, hs.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "read the bucket sizes");
    // Step 9: every bucket by a plan of its own
    bsort_ctx child;
    child.device = h->device;
    child.flags = h->flags & (BSORT_FLAG_MERGE_SORT | BSORT_FLAG_PLAN_MODEL);
    child.ws = child_ws;
    child.ws_bytes = P.child_bytes;
    child.ws_fixed = true;
    child.kernels_ready = true;
    e = cudaMemsetAsync(child_ws, 0, sizeof(int), st);  // its error word
    if (e != cudaSuccess) return cuda_fail(h, e, "memset(error word)");
    // The padding is the relocated array's tail [n, n'): its keys are the
    // last sublist's largest items, which end the last run of the last
    // bucket.  So bucket j sorts positions [L, min(R, n)) straight into the
    // output (the relocated array stays as Step 8 left it), float codes
    // decoded there afterwards.
    uint32_t *out = static_cast<uint32_t *>(kout);
    for (uint32_t j = 0; j < I.b; ++j) {
        const uint64_t L = hs[j], R = hs[j + 1];
        if (R < L || R > I.n_padded || R - L > I.bucket_bound)
            return fail(h, BSORT_EINTERNAL, "bucket %u spans [%llu, %llu)", j,
                        (unsigned long long)L, (unsigned long long)R);
        const uint64_t end = R < n ? R : n;
        if (end <= L) continue;
        bsort_status rs = run_sort(&child, BSORT_U32, reloc_k + L, nullptr, out + L, nullptr, 0,
                                   end - L, st);
        if (rs != BSORT_OK)
            return fail(h, rs, "bucket %u (%llu keys): %s", j, (unsigned long long)(end - L),
                        child.err);
        if (is_f32) {
            e = launch_f32_decode(out + L, out + L, end - L, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "decode a bucket");
        }
    }
    e = launch_merge_error(reinterpret_cast<const int *>(child_ws), err, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "merge error words");
    return BSORT_OK;
}

// Key-value pairs with 64-bit keys: two stable passes of the 32-bit pair
// sort, the least significant half first (an LSD sort over the halves, each
// pass Algorithm 1 on 32-bit keys carrying positions): pass A orders the
// low halves carrying the input index, pass B orders the high halves
// (gathered in pass A's order) carrying pass A's position, and the output
// takes key and value from input p1[p2[y]].  Stability of both passes makes
// the result the stable order by the full key.  Scratch: five arrays of n
// words after the passes' own workspace (plus n keys and values when
// sorting in place).
bsort_status run_pairs_u64(bsort_t h, const void *kin, const void *vin, void *kout, void *vout,
                           uint32_t vb, uint64_t n, cudaStream_t st)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    if (n >= kMaxN) return fail(h, BSORT_EUNSUPPORTED, "n = %llu exceeds 2^32 - 2^16", (unsigned long long)n);
    if (n == 0) return BSORT_OK;
    Plan PA;
    rs = make_plan(h, BSORT_U32, 4, n, &PA);
    if (rs != BSORT_OK) return rs;
    const uint64_t words = align_up(n * 4);
    const bool in_place = kin == kout || vin == vout;
    const uint64_t keep = in_place ? align_up(n * 8) + align_up(n * (uint64_t)vb) : 0;
    const uint64_t base = align_up(PA.total);
    rs = ensure_workspace(h, base + 5 * words + keep);
    if (rs != BSORT_OK) return rs;
    unsigned char *ws = static_cast<unsigned char *>(h->ws) + base;
    uint32_t *lo = reinterpret_cast<uint32_t *>(ws);
    uint32_t *iota = reinterpret_cast<uint32_t *>(ws + words);
    uint32_t *scratch = reinterpret_cast<uint32_t *>(ws + 2 * words);
    uint32_t *p1 = reinterpret_cast<uint32_t *>(ws + 3 * words);
    uint32_t *p2 = reinterpret_cast<uint32_t *>(ws + 4 * words);
    const uint64_t *k64 = static_cast<const uint64_t *>(kin);
    const void *v = vin;
    cudaError_t e;
    if (in_place) {  // keep the input: the last gather reads it while writing
        unsigned char *kk = ws + 5 * words;
        unsigned char *vv = kk + align_up(n * 8);
        e = cudaMemcpyAsync(kk, kin, n * 8, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vv, vin, n * vb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy the input aside");
        k64 = reinterpret_cast<const uint64_t *>(kk);
        v = vv;
    }
    e = launch_u64_split(k64, lo, iota, n, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "split 64-bit keys");
    rs = run_sort(h, BSORT_U32, lo, iota, scratch, p1, 4, n, st);  // pass A: low halves
    if (rs != BSORT_OK) return rs;
    e = launch_u64_gather_hi(k64, p1, lo, n, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "gather high halves");
    rs = run_sort(h, BSORT_U32, lo, iota, scratch, p2, 4, n, st);  // pass B: high halves
    if (rs != BSORT_OK) return rs;
    e = launch_u64_final(k64, v, (int)vb, p1, p2, static_cast<uint64_t *>(kout), vout, n, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply the permutations");
    return BSORT_OK;
}

bsort_status run_sort_u64(bsort_t h, const Plan &P, const void *kin, void *kout, uint64_t n,
                          cudaStream_t st, Seq &seq)
{
    const bsort_plan_info &I = P.info;
    unsigned char *ws = static_cast<unsigned char *>(h->ws);
    int *err = reinterpret_cast<int *>(ws + P.off_hdr);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(ws + P.off_hdr + 64);
    if (I.single_tile) {
        if (n == 1) {
            if (kout != kin) {
                cudaError_t e = cudaMemcpyAsync(kout, kin, 8, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "copy n=1");
            }
            return BSORT_OK;
        }
        SEQ(launch_bucket_sort_u64(P.unit_chunk, (int)I.unit_ctas, kin, nullptr, 1, n, n, kout,
                                   err, st),
            "step9_single_unit");
        return BSORT_OK;
    }
    uint64_t *tiles = reinterpret_cast<uint64_t *>(ws + P.off_tiles_k);
    uint64_t *reloc = reinterpret_cast<uint64_t *>(ws + P.off_reloc_k);
    Rec128 *samples = reinterpret_cast<Rec128 *>(ws + P.off_samples);
    Rec128 *rec_a = reinterpret_cast<Rec128 *>(ws + P.off_rec_a);
    Rec128 *rec_b = reinterpret_cast<Rec128 *>(ws + P.off_rec_b);
    Rec128 *spl = reinterpret_cast<Rec128 *>(ws + P.off_spl);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(ws + P.off_offsets);
    uint32_t *srcb = reinterpret_cast<uint32_t *>(ws + P.off_srcb);
    uint32_t *blk = reinterpret_cast<uint32_t *>(ws + P.off_blk);
    uint32_t *units = reinterpret_cast<uint32_t *>(ws + P.off_units);
    // Steps 1-3
    SEQ(launch_sublist_sort_u64(P.tile_chunk, (int)I.tile_ctas, kin, n, I.m, I.s, tiles, samples,
                                st),
        "step1_3_sublist_sort");
    // Step 4: merge the m sorted runs of s records (the samples stay intact)
    const Rec128 *src = samples;
    Rec128 *dst = rec_a;
    for (uint64_t L = I.s; L < P.n_rec; L <<= 1) {
        SEQ(launch_rec_merge(src, dst, P.n_rec, (uint32_t)L, st), "step4_sample_merge");
        src = dst;
        dst = dst == rec_a ? rec_b : rec_a;
    }
    // Step 5
    SEQ(launch_select_splitters_u64(src, P.n_rec, I.b, spl, st), "step5_splitters");
    // Step 6
    uint32_t *cum = reinterpret_cast<uint32_t *>(ws + P.off_cum);
    uint32_t *jr = reinterpret_cast<uint32_t *>(ws + P.off_jr);
    SEQ(launch_sample_index_seg_u64(tiles, spl, I.t, I.b, I.m, jr, cum, st),
        "step6_sample_index");
    // Step 7 (one scan per bucket row; also the run starts)
    SEQ(launch_row_scan(cum, I.m, I.t, I.b, nullptr, srcb, offsets, st), "step7_prefix_sum");
    // Step 8
    SEQ(launch_block_index(offsets, P.n_runs, (uint32_t)I.n_padded, blk, st), "step8_run_index");
    SEQ(launch_relocate_u64(tiles, offsets, srcb, blk, P.n_runs, (uint32_t)I.n_padded, reloc, st),
        "step8_relocate");
    // Step 9 (two tiers: one-CTA units, then cluster units for larger buckets)
    uint32_t *units2 = P.small_chunk ? reinterpret_cast<uint32_t *>(ws + P.off_units2) : nullptr;
    const uint32_t q1 = P.small_chunk ? (uint32_t)P.small_chunk : (uint32_t)I.unit_capacity;
    // two tiers: a unit per bucket; one tier: buckets packed greedily
    SEQ(P.small_chunk ? launch_units_each(offsets, I.m, I.b, (uint32_t)I.n_padded, q1,
                                          (uint32_t)I.unit_capacity, units, units2, err, st)
                      : launch_pack_units(offsets, I.m, I.b, (uint32_t)I.n_padded, q1,
                                          (uint32_t)I.unit_capacity, units, units2, err, st),
        "step9_pack_units");
    SEQ(launch_bucket_sort_u64(P.small_chunk ? P.small_chunk : P.unit_chunk,
                               P.small_chunk ? 1 : (int)I.unit_ctas, reloc, units, I.b, n,
                               I.n_padded, kout, err, st),
        "step9_bucket_sort");
    if (P.small_chunk)
        SEQ(launch_bucket_sort_u64(P.unit_chunk, (int)I.unit_ctas, reloc, units2,
                                   large_units_max(I.n_padded, q1, I.b), n, I.n_padded, kout, err,
                                   st),
            "step9_bucket_sort_large");
    return BSORT_OK;
}

bsort_status run_sort(bsort_t h, bsort_key_type kt, const void *kin, const void *vin, void *kout,
                      void *vout, uint32_t vb, uint64_t n, cudaStream_t st, const HostPipe *hp)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    if (hp && (h->flags & BSORT_FLAG_TEST_STALL_SCAN))
        return fail(h, BSORT_EINVAL, "BSORT_FLAG_TEST_STALL_SCAN is for device-buffer calls");
    Plan P;
    rs = make_plan(h, kt, vb, n, &P);
    if (rs != BSORT_OK) return rs;
    rs = ensure_workspace(h, P.total);
    if (rs != BSORT_OK) return rs;
    h->last = P;
    h->have_last = true;
    unsigned char *ws = static_cast<unsigned char *>(h->ws);
    int *err = reinterpret_cast<int *>(ws + P.off_hdr);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(ws + P.off_hdr + 64);
    const int is_f32 = kt == BSORT_F32;
    const bsort_plan_info &I = P.info;
    Seq seq(h, st);
    if (n == 0) return BSORT_OK;
    if (I.levels == 2) {
        if (hp) return fail(h, BSORT_EINTERNAL, "two-level plans take no host pipeline");
        return run_sort_two_level(h, P, kt, kin, kout, n, st, seq);
    }
    if (P.wide) return run_sort_u64(h, P, kin, kout, n, st, seq);
    if (I.single_tile) {
        if (n == 1) {
            if (kout != kin) {
                cudaError_t e = cudaMemcpyAsync(kout, kin, 4, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "copy n=1");
                if (vb) {
                    e = cudaMemcpyAsync(vout, vin, vb, cudaMemcpyDeviceToDevice, st);
                    if (e != cudaSuccess) return cuda_fail(h, e, "copy n=1");
                }
            }
            return BSORT_OK;
        }
        const GatherSrc none;
        SEQ(P.pairs ? launch_bucket_sort_pairs(P.unit_chunk, (int)I.unit_ctas, kin, vin, nullptr,
                                               1, n, n, is_f32, (int)vb, kout, vout, err, none,
                                               st)
                    : launch_bucket_sort_keys(P.unit_chunk, (int)I.unit_ctas, kin, nullptr, 1, n,
                                              n, is_f32, kout, err, none, st, P.radix),
            "step9_single_unit");
        return BSORT_OK;
    }
    uint32_t *tiles_k = reinterpret_cast<uint32_t *>(ws + P.off_tiles_k);
    void *tiles_v = ws + P.off_tiles_v;
    uint32_t *reloc_k = reinterpret_cast<uint32_t *>(ws + P.off_reloc_k);
    void *reloc_v = ws + P.off_reloc_v;
    uint64_t *samples = reinterpret_cast<uint64_t *>(ws + P.off_samples);
    uint64_t *rec_a = reinterpret_cast<uint64_t *>(ws + P.off_rec_a);
    uint64_t *rec_b = reinterpret_cast<uint64_t *>(ws + P.off_rec_b);
    uint64_t *spl = reinterpret_cast<uint64_t *>(ws + P.off_spl);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(ws + P.off_offsets);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + P.off_status);

    // look-back state must start at zero (only the stalled-scan test flag
    // runs the look-back scan here)
    cudaError_t e = cudaSuccess;
    if (h->flags & BSORT_FLAG_TEST_STALL_SCAN) {
        e = cudaMemsetAsync(status, 0, (size_t)P.scan_chunks * 8, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan status)");
        e = cudaMemsetAsync(ticket, 0, 4, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan ticket)");
    }

    // Steps 1-3
    if (hp) {
        // chunk c: copy its sublists' keys in, then sort them
        e = stream_after(h->xfer, st, h->xev[2 * kPipe]);
        if (e != cudaSuccess) return cuda_fail(h, e, "order copy stream");
        const uint32_t per = (I.m + hp->groups - 1) / hp->groups;
        for (uint32_t t0 = 0, c = 0; t0 < I.m; t0 += per, ++c) {
            const uint32_t mc = std::min(per, I.m - t0);
            const uint64_t p0 = (uint64_t)t0 * I.t;
            const uint64_t p1 = std::min<uint64_t>((uint64_t)(t0 + mc) * I.t, n);
            if (p1 > p0) {
                e = cudaMemcpyAsync(static_cast<unsigned char *>(hp->d_keys) + p0 * 4,
                                    static_cast<const unsigned char *>(hp->h_in) + p0 * 4,
                                    (p1 - p0) * 4, cudaMemcpyHostToDevice, h->xfer);
                if (e == cudaSuccess) e = stream_after(st, h->xfer, h->xev[c]);
                if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
            }
            SEQ(launch_sublist_sort_keys(P.tile_chunk, (int)I.tile_ctas, kin, n, mc, is_f32,
                                         I.s, tiles_k, samples, st, t0, P.radix),
                "step1_3_sublist_sort");
        }
    } else {
        SEQ(P.pairs ? launch_sublist_sort_pairs(P.tile_chunk, (int)I.tile_ctas, kin, vin, n,
                                                I.m, is_f32, (int)vb, I.s, tiles_k, tiles_v,
                                                samples, st)
                    : launch_sublist_sort_keys(P.tile_chunk, (int)I.tile_ctas, kin, n, I.m,
                                               is_f32, I.s, tiles_k, samples, st, 0, P.radix),
            "step1_3_sublist_sort");
    }
    // Steps 4-5: the records by digits (large sample sets), or in chunks
    // then merged
    const bool one_chunk = P.n_rec_pad == (uint32_t)kRecordChunk;
    if (P.rec_radix) {
        void *rs = ws + P.off_rs;
        SEQ(launch_records_hist(samples, P.n_rec, rs, h->num_sms, st), "step4_sample_hist");
        SEQ(launch_records_pass(0, samples, rec_a, P.n_rec, I.b, nullptr, rs, err, st),
            "step4_sample_radix");
        SEQ(launch_records_pass(1, rec_a, rec_b, P.n_rec, I.b, nullptr, rs, err, st),
            "step4_sample_radix");
        SEQ(launch_records_pass(2, rec_b, rec_a, P.n_rec, I.b, nullptr, rs, err, st),
            "step4_sample_radix");
        SEQ(launch_records_pass(3, rec_a, nullptr, P.n_rec, I.b, spl, rs, err, st),
            "step4_5_radix_splitters");
    } else {
        SEQ(launch_records_chunk_sort(samples, rec_a, P.n_rec, P.n_rec_pad,
                                      one_chunk ? spl : nullptr, I.s, I.b, st),
            "step4_sample_chunks");
    }
    if (!P.rec_radix && !one_chunk) {
        uint64_t *src = rec_a, *dst = rec_b;
        for (uint32_t L = kRecordChunk; L < P.n_rec_pad; L <<= 1) {
            SEQ(launch_merge_pass(src, dst, P.n_rec_pad, L, st), "step4_sample_merge");
            uint64_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        SEQ(launch_select_splitters(src, P.n_rec, I.b, spl, st), "step5_splitters");
    }
    uint32_t *srcb = reinterpret_cast<uint32_t *>(ws + P.off_srcb);
    uint32_t *blk = reinterpret_cast<uint32_t *>(ws + P.off_blk);
    // Step 6
    uint32_t *cum = reinterpret_cast<uint32_t *>(ws + P.off_cum);
    uint32_t *jr = reinterpret_cast<uint32_t *>(ws + P.off_jr);
    SEQ(launch_sample_index(tiles_k, spl, I.t, I.s, I.b, I.m, jr, cum, st), "step6_sample_index");
    // Step 7: one independent scan per bucket row of the cumulative counts.
    // The run starts are materialised only for the gathering load of Step 9
    // (the relocation derives them from the cumulative counts).  The
    // stalled-scan test flag takes the decoupled look-back scan instead,
    // with its first chunk held back.
    if (h->flags & BSORT_FLAG_TEST_STALL_SCAN) {
        SEQ(launch_scan_cum(cum, I.m, I.t, nullptr, srcb, offsets, P.n_runs, status, ticket, err,
                            st, true),
            "step7_prefix_sum");
        // a stalled scan leaves inconsistent offsets: Steps 8-9 must not read them
        return BSORT_OK;
    }
    // Step 8: materialised, unless BSORT_FLAG_LOW_MEMORY fuses it into the
    // load of Step 9, which then gathers every unit from the runs A_ij.  A
    // materialised relocation of rows that one CTA holds runs together with
    // Step 7, a CTA per bucket.
    GatherSrc g;
    if (P.relocate && bucket_relocate_fits(I.m)) {
        SEQ(launch_bucket_relocate(cum, I.m, I.t, I.b, (uint32_t)I.n_padded, tiles_k, tiles_v,
                                   (int)vb, offsets, reloc_k, reloc_v, st),
            "step7_8_scan_relocate");
    } else {
        SEQ(launch_row_scan(cum, I.m, I.t, I.b, nullptr, P.relocate ? nullptr : srcb, offsets,
                            st),
            "step7_prefix_sum");
        SEQ(launch_block_index(offsets, P.n_runs, (uint32_t)I.n_padded, blk, st),
            "step8_run_index");
        if (P.relocate) {
            SEQ(launch_relocate(tiles_k, tiles_v, offsets, nullptr, blk, P.n_runs,
                                (uint32_t)I.n_padded, (int)vb, reloc_k, reloc_v, st, cum, I.m,
                                I.t),
                "step8_relocate");
        }
    }
    // Step 9: buckets packed into units (two tiers: one-CTA units of
    // small_chunk items, cluster units of unit_capacity for larger buckets)
    uint32_t *units = reinterpret_cast<uint32_t *>(ws + P.off_units);
    uint32_t *units2 = P.small_chunk ? reinterpret_cast<uint32_t *>(ws + P.off_units2) : nullptr;
    const uint32_t q1 = P.small_chunk ? (uint32_t)P.small_chunk : (uint32_t)I.unit_capacity;
    // two tiers: a unit per bucket; one tier: buckets packed greedily
    SEQ(P.small_chunk ? launch_units_each(offsets, I.m, I.b, (uint32_t)I.n_padded, q1,
                                          (uint32_t)I.unit_capacity, units, units2, err, st)
                      : launch_pack_units(offsets, I.m, I.b, (uint32_t)I.n_padded, q1,
                                          (uint32_t)I.unit_capacity, units, units2, err, st),
        "step9_pack_units");
    if (!P.relocate) {
        g.offsets = offsets;
        g.srcb = srcb;
        g.blk = blk;
        g.runs = P.n_runs;
    }
    const void *s9k = P.relocate ? (const void *)reloc_k : (const void *)tiles_k;
    const void *s9v = P.relocate ? (const void *)reloc_v : (const void *)tiles_v;
    const int c1 = P.small_chunk ? P.small_chunk : P.unit_chunk;
    const int k1 = P.small_chunk ? 1 : (int)I.unit_ctas;
    if (hp) {
        // group g: the units of both tiers that begin in slice g, then the
        // slice's keys to the host
        const uint32_t np = (uint32_t)I.n_padded;
        uint32_t *r1 = hp->ranges, *r2 = hp->ranges + kPipe + 1;
        const int G = hp->groups;
        SEQ(launch_unit_ranges(units, np, (uint32_t)G, r1, st), "step9_unit_ranges");
        if (units2) SEQ(launch_unit_ranges(units2, np, (uint32_t)G, r2, st), "step9_unit_ranges");
        // resident CTAs (clusters: 7/8 of the SMs can hold them) loop over
        // the group's units, none of them in a late wave
        const int sms = std::max(h->num_sms, 8);
        const uint32_t g1 = std::max(
            1u, std::min<uint32_t>(I.b, (uint32_t)(k1 == 1 ? sms : (sms * 7 / 8) / k1)));
        const uint32_t g2 = std::max(1u, (uint32_t)((sms * 7 / 8) / (int)I.unit_ctas));
        for (int g = 0; g < G; ++g) {
            SEQ(launch_bucket_sort_keys_range(c1, k1, s9k, units, r1 + g, g1, n, I.n_padded,
                                              is_f32, kout, err, st, P.radix),
                "step9_bucket_sort");
            if (units2)
                SEQ(launch_bucket_sort_keys_range(P.unit_chunk, (int)I.unit_ctas, s9k, units2,
                                                  r2 + g, g2, n, I.n_padded, is_f32, kout, err,
                                                  st, P.radix),
                    "step9_bucket_sort_large");
            const uint64_t p0 = std::min<uint64_t>((uint64_t)g * np / G, n);
            const uint64_t p1 = std::min<uint64_t>((uint64_t)(g + 1) * np / G, n);
            if (p1 > p0) {
                e = stream_after(h->xfer, st, h->xev[kPipe + g]);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(static_cast<unsigned char *>(hp->h_out) + p0 * 4,
                                        static_cast<const unsigned char *>(hp->d_keys) + p0 * 4,
                                        (p1 - p0) * 4, cudaMemcpyDeviceToHost, h->xfer);
                if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
            }
        }
        e = stream_after(st, h->xfer, h->xev[2 * kPipe + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "order copy stream");
        return BSORT_OK;
    }
    SEQ(P.pairs ? launch_bucket_sort_pairs(c1, k1, s9k, s9v, units, I.b, n, I.n_padded, is_f32,
                                           (int)vb, kout, vout, err, g, st)
                : launch_bucket_sort_keys(c1, k1, s9k, units, I.b, n, I.n_padded, is_f32, kout,
                                          err, g, st, P.radix),
        "step9_bucket_sort");
    if (P.small_chunk) {
        const uint32_t u2 = large_units_max(I.n_padded, q1, I.b);
        SEQ(P.pairs ? launch_bucket_sort_pairs(P.unit_chunk, (int)I.unit_ctas, s9k, s9v, units2,
                                               u2, n, I.n_padded, is_f32, (int)vb, kout, vout,
                                               err, g, st)
                    : launch_bucket_sort_keys(P.unit_chunk, (int)I.unit_ctas, s9k, units2, u2, n,
                                              I.n_padded, is_f32, kout, err, g, st, P.radix),
            "step9_bucket_sort_large");
    }
    return BSORT_OK;
}

// run_sort through the handle's graph cache (BSORT_FLAG_GRAPHS): the plan
// and the workspace are settled first, outside any capture; a call seen
// before is one graph launch, a new one is captured from the stream,
// instantiated and launched.
bsort_status run_sort_graph(bsort_t h, bsort_key_type kt, const void *kin, const void *vin,
                            void *kout, void *vout, uint32_t vb, uint64_t n, cudaStream_t st)
{
    // (the legacy default stream cannot be captured: its calls launch as usual)
    if (!(h->flags & BSORT_FLAG_GRAPHS) || n == 0 || st == nullptr || st == cudaStreamLegacy)
        return run_sort(h, kt, kin, vin, kout, vout, vb, n, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)  // the caller is capturing: part of its graph
        return run_sort(h, kt, kin, vin, kout, vout, vb, n, st);
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    Plan P;
    rs = make_plan(h, kt, vb, n, &P);
    if (rs != BSORT_OK) return rs;
    if (P.info.levels == 2)  // waits for the stream mid-call: not capturable
        return run_sort(h, kt, kin, vin, kout, vout, vb, n, st);
    rs = ensure_workspace(h, P.total);
    if (rs != BSORT_OK) return rs;
    for (auto &g : h->graphs) {
        if (g.kt == (int)kt && g.vb == vb && g.n == n && g.kin == kin && g.vin == vin &&
            g.kout == kout && g.vout == vout && g.ws == h->ws && g.st == st) {
            g.used = ++h->graph_clock;
            h->last = P;
            h->have_last = true;
            e = cudaGraphLaunch(g.exec, st);
            return e == cudaSuccess ? BSORT_OK : cuda_fail(h, e, "cudaGraphLaunch");
        }
    }
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    h->capturing = true;
    rs = run_sort(h, kt, kin, vin, kout, vout, vb, n, st);
    h->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rs != BSORT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rs != BSORT_OK ? rs : cuda_fail(h, e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    constexpr size_t kGraphs = 16;
    if (h->graphs.size() >= kGraphs) {  // drop the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < h->graphs.size(); ++i)
            if (h->graphs[i].used < h->graphs[lru].used) lru = i;
        cudaGraphExecDestroy(h->graphs[lru].exec);
        h->graphs.erase(h->graphs.begin() + (long)lru);
    }
    bsort_ctx::Graph g;
    g.kt = (int)kt;
    g.vb = vb;
    g.n = n;
    g.kin = kin;
    g.vin = vin;
    g.kout = kout;
    g.vout = vout;
    g.ws = h->ws;
    g.st = st;
    g.exec = exec;
    g.used = ++h->graph_clock;
    h->graphs.push_back(g);
    e = cudaGraphLaunch(exec, st);
    return e == cudaSuccess ? BSORT_OK : cuda_fail(h, e, "cudaGraphLaunch");
}

// ---------------------------------------------------------------- batches
// Direct unit shapes, smallest first: (chunk, ctas); 64-bit keys use CTAs
// of at most 16384 keys.
constexpr int kNumDirect = 8;
const int kDirectShapes[kNumDirect][2] = {{2048, 1},  {4096, 1},  {8192, 1},  {16384, 1},
                                          {32768, 1}, {32768, 2}, {32768, 4}, {32768, 8}};
const char *const kDirectNames[kNumDirect] = {
    "batch_direct_2048", "batch_direct_4096", "batch_direct_8192", "batch_direct_16384",
    "batch_direct_32768", "batch_direct_2x32768", "batch_direct_4x32768", "batch_direct_8x32768"};
// (the last, a 16-CTA cluster, only where the device schedules one)
constexpr int kNumDirectWide = 8;
const int kDirectShapesWide[kNumDirectWide][2] = {{2048, 1},  {4096, 1},  {8192, 1},
                                                  {16384, 1}, {16384, 2}, {16384, 4},
                                                  {16384, 8}, {16384, 16}};
const char *const kDirectNamesWide[kNumDirectWide] = {
    "batch_direct_u64_2048",    "batch_direct_u64_4096",   "batch_direct_u64_8192",
    "batch_direct_u64_16384",   "batch_direct_u64_2x16384", "batch_direct_u64_4x16384",
    "batch_direct_u64_8x16384", "batch_direct_u64_16x16384"};

// Direct-segment shapes of 64-bit keys this device runs, and the largest
// 64-bit segment sorted whole: batch_direct_max if set, else every shape.
int wide_direct_shapes() { return batch_wide_cluster16() ? kNumDirectWide : kNumDirectWide - 1; }
uint64_t wide_direct_max(const bsort_t h)
{
    const int ns = wide_direct_shapes();
    const uint64_t largest =
        (uint64_t)kDirectShapesWide[ns - 1][0] * (uint64_t)kDirectShapesWide[ns - 1][1];
    return h->direct_max_set && h->direct_max < largest ? h->direct_max : largest;
}

// Host plan of one batch: direct lists per shape, sampled segments with
// their sublists and buckets, plain-sorted large segments, and the
// workspace layout (descriptors first, copied from pinned staging).
struct BatchPlan {
    bsort_batch_info info;
    bool wide = false;  // 64-bit keys
    std::vector<uint32_t> direct[kNumDirect];  // (begin, end) pairs per shape
    std::vector<SegInfo> segs;
    std::vector<uint32_t> sub_seg;
    std::vector<uint32_t> units;               // (segment, bucket) pairs
    std::vector<std::pair<uint64_t, uint64_t>> large;  // (begin, n)
    uint64_t large_ws = 0;
    uint32_t nrec = 0, nspl = 0, runs = 0, scan_chunks = 0;
    uint64_t n_pad = 0;
    // descriptor words (uint32) and their offsets in it
    uint64_t d_direct[kNumDirect] = {}, d_sub = 0, d_segs = 0, d_units = 0, d_words = 0;
    // workspace offsets (bytes)
    uint64_t off_desc = 0, off_tiles = 0, off_reloc = 0, off_samples = 0, off_spl = 0,
             off_counts = 0, off_offsets = 0, off_srcb = 0, off_status = 0, off_blk = 0,
             total = 0;
};

// One array of a batch: keys [begin, begin + n) of the input and output.
struct SegSpan {
    uint64_t begin, n;
};

// Segments q = [segoff[q], segoff[q+1]) of the public offsets table.
bsort_status spans_from_offsets(bsort_t h, const uint64_t *segoff, uint32_t nsegs,
                                std::vector<SegSpan> *out)
{
    out->clear();
    if (nsegs == 0) return BSORT_OK;
    if (!segoff) return fail(h, BSORT_EINVAL, "null segment offsets");
    out->reserve(nsegs);
    for (uint32_t q = 0; q < nsegs; ++q) {
        if (segoff[q + 1] < segoff[q])
            return fail(h, BSORT_EINVAL, "segment offsets decrease at %u", q);
        out->push_back({segoff[q], segoff[q + 1] - segoff[q]});
    }
    return BSORT_OK;
}

bsort_status make_batch_plan(bsort_t h, bsort_key_type kt, const SegSpan *spans,
                             uint32_t nsegs, BatchPlan *B)
{
    if (kt != BSORT_U32 && kt != BSORT_F32 && kt != BSORT_U64)
        return fail(h, BSORT_EINVAL, "unknown key type %d", (int)kt);
    B->wide = kt == BSORT_U64;
    const int(*shapes)[2] = B->wide ? kDirectShapesWide : kDirectShapes;
    const int nshapes = B->wide ? wide_direct_shapes() : kNumDirect;
    const uint64_t largest = (uint64_t)shapes[nshapes - 1][0] * shapes[nshapes - 1][1];
    if (nsegs && !spans) return fail(h, BSORT_EINVAL, "null segment list");
    bsort_batch_info &I = B->info;
    memset(&I, 0, sizeof(I));
    I.num_segs = nsegs;
    if (nsegs == 0) return BSORT_OK;
    for (uint32_t q = 0; q < nsegs; ++q)
        if (spans[q].begin + spans[q].n >= kMaxN)
            return fail(h, BSORT_EUNSUPPORTED, "segment end %llu exceeds 2^32 - 2^16",
                        (unsigned long long)(spans[q].begin + spans[q].n));
    const uint64_t dmax =
        B->wide ? wide_direct_max(h) : (h->direct_max < largest ? h->direct_max : largest);
    const uint64_t tile = B->wide ? (uint64_t)kSegTileU64 : (uint64_t)kSegTile;
    const uint64_t unit = B->wide ? (uint64_t)kBatchUnitU64 : (uint64_t)kBatchUnit;
    uint64_t g = 0;  // sublists so far
    for (uint32_t q = 0; q < nsegs; ++q) {
        const uint64_t a = spans[q].begin, n = spans[q].n;
        I.n += n;
        if (n <= 1) continue;  // nothing to order (a copy when out != in)
        if (n <= dmax) {
            int c = 0;
            while ((uint64_t)shapes[c][0] * shapes[c][1] < n) ++c;
            B->direct[c].push_back((uint32_t)a);
            B->direct[c].push_back((uint32_t)(a + n));
            ++I.direct_segs;
        } else if (n <= (B->wide ? kBatchSampledMaxU64 : kBatchSampledMax)) {
            SegInfo sg = {};
            sg.g0 = (uint32_t)g;
            sg.m = (uint32_t)((n + tile - 1) / tile);
            sg.s = B->wide ? (sg.m <= 32 ? 256u : 128u) : kBatchSamples;
            const uint64_t np = (uint64_t)sg.m * tile;
            uint64_t lo = 1, hi = (uint64_t)sg.m * sg.s;  // smallest b whose bound fits a unit
            while (lo < hi) {
                const uint64_t mid = (lo + hi) / 2;
                if (bound_for(np, sg.m, sg.s, mid) <= unit) hi = mid;
                else lo = mid + 1;
            }
            sg.b = (uint32_t)lo;
            sg.rec = B->nrec;
            sg.spl = B->nspl;
            sg.run0 = B->runs;
            sg.out = (uint32_t)a;
            sg.n = (uint32_t)n;
            for (uint32_t i = 0; i < sg.m; ++i) B->sub_seg.push_back((uint32_t)B->segs.size());
            for (uint32_t j = 0; j < sg.b; ++j) {
                B->units.push_back((uint32_t)B->segs.size());
                B->units.push_back(j);
            }
            B->nrec += sg.m * sg.s;
            B->nspl += sg.b;
            B->runs += sg.m * sg.b;
            g += sg.m;
            B->segs.push_back(sg);
        } else {
            B->large.push_back({a, n});
        }
    }
    if (g * tile >= kMaxN) return fail(h, BSORT_EUNSUPPORTED, "padded sampled segments exceed 2^32");
    B->n_pad = g * tile;
    I.sampled_segs = (uint32_t)B->segs.size();
    I.large_segs = (uint32_t)B->large.size();
    I.sublists = (uint32_t)g;
    I.buckets = B->nspl;
    B->scan_chunks = (B->runs + kScanChunk - 1) / kScanChunk;
    // plain sorts of the large segments reuse the workspace after the batch
    for (const auto &lg : B->large) {
        Plan P;
        bsort_status st = make_plan(h, kt, 0, lg.second, &P);
        if (st != BSORT_OK) return st;
        if (P.total > B->large_ws) B->large_ws = P.total;
        I.num_kernels += P.info.num_kernels;
    }
    // descriptor words
    uint64_t wds = 0;
    auto words = [&](uint64_t n) {
        const uint64_t at = wds;
        wds += (n + 3) / 4 * 4;  // 16-byte aligned pieces
        return at;
    };
    for (int c = 0; c < kNumDirect; ++c) {
        B->d_direct[c] = words(B->direct[c].size());
        if (!B->direct[c].empty()) ++I.num_kernels;
    }
    B->d_sub = words(B->sub_seg.size());
    B->d_segs = words(B->segs.size() * (sizeof(SegInfo) / 4));
    B->d_units = words(B->units.size());
    B->d_words = wds;
    if (!B->segs.empty()) I.num_kernels += 7;  // Steps 1-3, 4-5, 6, 7, run index, 8, 9
    // workspace
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    take(kAlign);  // error word + scan ticket
    B->off_desc = take(wds * 4);
    if (!B->segs.empty()) {
        const uint64_t kb = B->wide ? 8 : 4;   // key bytes
        const uint64_t rb = B->wide ? 16 : 8;  // sample record bytes
        B->off_tiles = take(B->n_pad * kb);
        B->off_reloc = take(B->n_pad * kb);
        B->off_samples = take((uint64_t)B->nrec * rb);
        B->off_spl = take((uint64_t)B->nspl * rb);
        B->off_counts = take((uint64_t)B->runs * 4);
        B->off_offsets = take(((uint64_t)B->runs + 1) * 4);
        B->off_srcb = take((uint64_t)B->runs * 4);
        B->off_status = take((uint64_t)B->scan_chunks * 8);
        B->off_blk = take((B->n_pad + kBlockItems - 1) / kBlockItems * 4);
    }
    B->total = o > B->large_ws ? o : B->large_ws;
    I.workspace_bytes = B->total;
    return BSORT_OK;
}

// stage: when not null, pinned host memory of at least the plan's
// descriptor bytes that the caller keeps unchanged for as long as the
// upload may run again (a captured graph replays it); the handle's shared
// staging is used otherwise.
bsort_status run_batch(bsort_t h, bsort_key_type kt, const void *kin, void *kout,
                       const SegSpan *spans, uint32_t nsegs, cudaStream_t st,
                       void *stage = nullptr)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    BatchPlan B;
    rs = make_batch_plan(h, kt, spans, nsegs, &B);
    if (rs != BSORT_OK) return rs;
    if (B.info.n == 0) return BSORT_OK;
    rs = ensure_workspace(h, B.total);
    if (rs != BSORT_OK) return rs;
    cudaError_t e;
    // segments of one key: copies
    const uint64_t kb = B.wide ? 8 : 4;
    if (kout != kin)
        for (uint32_t q = 0; q < nsegs; ++q)
            if (spans[q].n == 1) {
                e = cudaMemcpyAsync(static_cast<char *>(kout) + spans[q].begin * kb,
                                    static_cast<const char *>(kin) + spans[q].begin * kb, kb,
                                    cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "copy of a one-key segment");
            }
    unsigned char *ws = static_cast<unsigned char *>(h->ws);
    int *err = reinterpret_cast<int *>(ws);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(ws + 64);
    uint32_t *desc = reinterpret_cast<uint32_t *>(ws + B.off_desc);
    const int is_f32 = kt == BSORT_F32;
    const uint32_t *ki = static_cast<const uint32_t *>(kin);
    uint32_t *ko = static_cast<uint32_t *>(kout);
    Seq seq(h, st);
    if (B.d_words && stage) {
        // descriptors from the caller's pinned buffer (a graph's own)
        uint32_t *hw = static_cast<uint32_t *>(stage);
        const uint64_t bytes = B.d_words * 4;
        memset(hw, 0, bytes);
        for (int c = 0; c < kNumDirect; ++c)
            if (!B.direct[c].empty())
                memcpy(hw + B.d_direct[c], B.direct[c].data(), B.direct[c].size() * 4);
        if (!B.sub_seg.empty()) memcpy(hw + B.d_sub, B.sub_seg.data(), B.sub_seg.size() * 4);
        if (!B.segs.empty()) memcpy(hw + B.d_segs, B.segs.data(), B.segs.size() * sizeof(SegInfo));
        if (!B.units.empty()) memcpy(hw + B.d_units, B.units.data(), B.units.size() * 4);
        e = cudaMemcpyAsync(desc, hw, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of the batch descriptors");
    } else if (B.d_words) {
        // descriptors: pinned staging -> workspace (the staging is reused
        // only after the previous copy out of it has completed)
        const uint64_t bytes = B.d_words * 4;
        if (h->stage_pending) {
            e = cudaEventSynchronize(h->stage_ev);
            if (e != cudaSuccess) return cuda_fail(h, e, "wait for the staging copy");
            h->stage_pending = false;
        }
        if (bytes > h->stage_bytes) {
            // grown geometrically: freeing pinned memory waits for the device,
            // and pinning is slow, so a stream of growing batches (the request
            // loop) must not pay them at every new maximum
            const uint64_t grow = std::max<uint64_t>({bytes, 2 * h->stage_bytes, 1ull << 20});
            if (h->stage) cudaFreeHost(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
            e = cudaHostAlloc(&h->stage, grow, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(h, BSORT_ENOMEM, "pinned staging of %llu bytes: %s",
                            (unsigned long long)grow, cudaGetErrorString(e));
            }
            h->stage_bytes = grow;
        }
        if (!h->stage_ev) {
            e = cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
        }
        uint32_t *hw = static_cast<uint32_t *>(h->stage);
        memset(hw, 0, bytes);
        for (int c = 0; c < kNumDirect; ++c)
            if (!B.direct[c].empty())
                memcpy(hw + B.d_direct[c], B.direct[c].data(), B.direct[c].size() * 4);
        if (!B.sub_seg.empty()) memcpy(hw + B.d_sub, B.sub_seg.data(), B.sub_seg.size() * 4);
        if (!B.segs.empty()) memcpy(hw + B.d_segs, B.segs.data(), B.segs.size() * sizeof(SegInfo));
        if (!B.units.empty()) memcpy(hw + B.d_units, B.units.data(), B.units.size() * 4);
        e = cudaMemcpyAsync(desc, hw, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of the batch descriptors");
        e = cudaEventRecord(h->stage_ev, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
        h->stage_pending = true;
    }
    // direct segments: one launch per unit shape
    for (int c = 0; c < kNumDirect; ++c) {
        const uint32_t cnt = (uint32_t)(B.direct[c].size() / 2);
        if (!cnt) continue;
        const int(*shapes)[2] = B.wide ? kDirectShapesWide : kDirectShapes;
        SEQ(launch_seg_sort(shapes[c][0], shapes[c][1], B.wide, kin, kout, desc + B.d_direct[c],
                            cnt, is_f32, err, st),
            B.wide ? kDirectNamesWide[c] : kDirectNames[c]);
    }
    // sampled segments: Algorithm 1, segment-aware
    if (!B.segs.empty()) {
        const uint32_t nsub = B.info.sublists;
        const uint32_t *sub_seg = desc + B.d_sub;
        const SegInfo *segs = reinterpret_cast<const SegInfo *>(desc + B.d_segs);
        const uint32_t *units = desc + B.d_units;
        uint32_t *counts = reinterpret_cast<uint32_t *>(ws + B.off_counts);
        uint32_t *offsets = reinterpret_cast<uint32_t *>(ws + B.off_offsets);
        uint32_t *srcb = reinterpret_cast<uint32_t *>(ws + B.off_srcb);
        unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + B.off_status);
        uint32_t *blk = reinterpret_cast<uint32_t *>(ws + B.off_blk);
        e = cudaMemsetAsync(status, 0, (size_t)B.scan_chunks * 8, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan status)");
        e = cudaMemsetAsync(ticket, 0, 4, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan ticket)");
        if (B.wide) {
            uint64_t *tiles = reinterpret_cast<uint64_t *>(ws + B.off_tiles);
            uint64_t *reloc = reinterpret_cast<uint64_t *>(ws + B.off_reloc);
            Rec128 *samples = reinterpret_cast<Rec128 *>(ws + B.off_samples);
            Rec128 *spl = reinterpret_cast<Rec128 *>(ws + B.off_spl);
            SEQ(launch_seg_sublist_sort_u64(static_cast<const uint64_t *>(kin), sub_seg, nsub,
                                            segs, tiles, samples, st),
                "batch_u64_step1_3_sublist_sort");
            SEQ(launch_seg_records_u64(samples, segs, B.info.sampled_segs, spl, st),
                "batch_u64_step4_5_samples");
            SEQ(launch_seg_sample_index_u64(tiles, samples, spl, sub_seg, nsub, segs, counts,
                                            srcb, st),
                "batch_u64_step6_sample_index");
            SEQ(launch_scan(counts, offsets, B.runs, status, ticket, err, st),
                "batch_u64_step7_prefix_sum");
            SEQ(launch_block_index(offsets, B.runs, (uint32_t)B.n_pad, blk, st),
                "batch_u64_step8_run_index");
            SEQ(launch_relocate_u64(tiles, offsets, srcb, blk, B.runs, (uint32_t)B.n_pad, reloc,
                                    st),
                "batch_u64_step8_relocate");
            SEQ(launch_seg_bucket_sort_u64(reloc, units, B.info.buckets, segs, offsets,
                                           static_cast<uint64_t *>(kout), err, st),
                "batch_u64_step9_bucket_sort");
        } else {
            uint32_t *tiles = reinterpret_cast<uint32_t *>(ws + B.off_tiles);
            uint32_t *reloc = reinterpret_cast<uint32_t *>(ws + B.off_reloc);
            uint64_t *samples = reinterpret_cast<uint64_t *>(ws + B.off_samples);
            uint64_t *spl = reinterpret_cast<uint64_t *>(ws + B.off_spl);
            SEQ(launch_seg_sublist_sort(ki, is_f32, sub_seg, nsub, segs, tiles, samples, st),
                "batch_step1_3_sublist_sort");
            SEQ(launch_seg_records(samples, segs, B.info.sampled_segs, spl, st),
                "batch_step4_5_samples");
            SEQ(launch_seg_sample_index(tiles, samples, spl, sub_seg, nsub, segs, counts, srcb,
                                        st),
                "batch_step6_sample_index");
            SEQ(launch_scan(counts, offsets, B.runs, status, ticket, err, st),
                "batch_step7_prefix_sum");
            SEQ(launch_block_index(offsets, B.runs, (uint32_t)B.n_pad, blk, st),
                "batch_step8_run_index");
            SEQ(launch_relocate(tiles, nullptr, offsets, srcb, blk, B.runs, (uint32_t)B.n_pad, 0,
                                reloc, nullptr, st),
                "batch_step8_relocate");
            SEQ(launch_seg_bucket_sort((int)kBatchUnit, reloc, units, B.info.buckets, segs,
                                       offsets, is_f32, ko, err, st),
                "batch_step9_bucket_sort");
        }
    }
    // large segments: one plain sort each, after the batch (same stream)
    for (const auto &lg : B.large) {
        rs = run_sort(h, kt, static_cast<const char *>(kin) + lg.first * kb, nullptr,
                      static_cast<char *>(kout) + lg.first * kb, nullptr, 0, lg.second, st);
        if (rs != BSORT_OK) return rs;
    }
    return BSORT_OK;
}

// run_batch through the handle's batch-graph cache (BSORT_FLAG_GRAPHS): a
// call whose segment table, key type, buffers, stream and workspace match a
// cached graph replays it with one graph launch (no planning on the host);
// otherwise the batch is planned, its launch sequence captured with the
// descriptors staged in pinned memory the graph owns, and kept (the 8 most
// recently used).
bsort_status run_batch_graph(bsort_t h, bsort_key_type kt, const void *kin, void *kout,
                             const SegSpan *spans, uint32_t nsegs, cudaStream_t st)
{
    if (!(h->flags & BSORT_FLAG_GRAPHS) || nsegs == 0 || st == nullptr || st == cudaStreamLegacy)
        return run_batch(h, kt, kin, kout, spans, nsegs, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return run_batch(h, kt, kin, kout, spans, nsegs, st);
    uint64_t hash = 0x9E3779B97F4A7C15ull ^ nsegs;
    for (uint32_t q = 0; q < nsegs; ++q) {
        hash = (hash ^ spans[q].begin) * 0xBF58476D1CE4E5B9ull;
        hash = (hash ^ spans[q].n) * 0x94D049BB133111EBull;
    }
    for (auto &g : h->batch_graphs) {
        if (g.kt != (int)kt || g.kin != kin || g.kout != kout || g.st != st || g.ws != h->ws ||
            g.hash != hash || g.table.size() != 2ull * nsegs)
            continue;
        bool same = true;
        for (uint32_t q = 0; q < nsegs && same; ++q)
            same = g.table[2 * q] == spans[q].begin && g.table[2 * q + 1] == spans[q].n;
        if (!same) continue;
        g.used = ++h->graph_clock;
        e = cudaGraphLaunch(g.exec, st);
        return e == cudaSuccess ? BSORT_OK : cuda_fail(h, e, "cudaGraphLaunch");
    }
    // settle the plan and the workspace outside the capture
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    BatchPlan B;
    rs = make_batch_plan(h, kt, spans, nsegs, &B);
    if (rs != BSORT_OK) return rs;
    rs = ensure_workspace(h, B.total);  // (covers the plain sorts of large segments)
    if (rs != BSORT_OK) return rs;
    void *desc = nullptr;
    if (B.d_words) {
        e = cudaHostAlloc(&desc, B.d_words * 4, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, BSORT_ENOMEM, "pinned descriptors of %llu bytes",
                        (unsigned long long)(B.d_words * 4));
        }
    }
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (desc) cudaFreeHost(desc);
        return cuda_fail(h, e, "cudaStreamBeginCapture");
    }
    h->capturing = true;
    rs = run_batch(h, kt, kin, kout, spans, nsegs, st, desc ? desc : nullptr);
    h->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rs != BSORT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (desc) cudaFreeHost(desc);
        cudaGetLastError();
        return rs != BSORT_OK ? rs : cuda_fail(h, e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        if (desc) cudaFreeHost(desc);
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    constexpr size_t kBatchGraphs = 8;
    if (h->batch_graphs.size() >= kBatchGraphs) {  // drop the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < h->batch_graphs.size(); ++i)
            if (h->batch_graphs[i].used < h->batch_graphs[lru].used) lru = i;
        // (its last replay may still be reading the descriptors)
        cudaStreamSynchronize(h->batch_graphs[lru].st);
        cudaGraphExecDestroy(h->batch_graphs[lru].exec);
        if (h->batch_graphs[lru].desc) cudaFreeHost(h->batch_graphs[lru].desc);
        h->batch_graphs.erase(h->batch_graphs.begin() + (long)lru);
    }
    bsort_ctx::BatchGraph g;
    g.kt = (int)kt;
    g.kin = kin;
    g.kout = kout;
    g.ws = h->ws;
    g.st = st;
    g.hash = hash;
    g.table.reserve(2ull * nsegs);
    for (uint32_t q = 0; q < nsegs; ++q) {
        g.table.push_back(spans[q].begin);
        g.table.push_back(spans[q].n);
    }
    g.desc = desc;
    g.exec = exec;
    g.used = ++h->graph_clock;
    h->batch_graphs.push_back(std::move(g));
    e = cudaGraphLaunch(exec, st);
    return e == cudaSuccess ? BSORT_OK : cuda_fail(h, e, "cudaGraphLaunch");
}

}  // namespace

// ---------------------------------------------------------------- serving
// The request loop behind bsort_submit / bsort_poll: continuous batching of
// independent sort jobs.  One worker thread per serving handle owns a
// device arena for admitted jobs' keys (part of the serving budget) and two
// lanes, each with its own streams (copy in, sort, copy out) and workspace:
//   lane A (small jobs: those a batch sorts with one CTA, one cluster or
//       the segment-aware sample sort) sorts everything admitted as one
//       batch (bsort_sort_batch's path, in place in the arena) as soon as
//       its previous batch has finished sorting, on a high-priority stream;
//   lane B (large jobs) sorts them one at a time, in arrival order, on a
//       low-priority stream, so that small jobs are not held behind them.
// Each turn of the loop retires jobs whose results are back in host memory
// (freeing their arena ranges), admits queued jobs in arrival order while
// the arena has room (first fit), and launches lane A's next batch.  Jobs
// that arrive while a batch sorts are copied in meanwhile and form the next
// batch.
struct bsort_server {
    struct Req {
        uint64_t ticket = 0;
        bsort_key_type kt = BSORT_U32;
        const void *in = nullptr;
        void *out = nullptr;
        uint64_t n = 0, bytes = 0, off = 0;
        uint64_t submit_ns = 0, start_ns = 0, done_ns = 0;
        uint32_t batch_size = 0;
        int lane = 0;
        bsort_status status = BSORT_ENOTREADY;
        cudaEvent_t ev = nullptr;  // its result is in host memory
        bool done = false;
    };
    struct Batch {
        std::vector<Req *> reqs;
        cudaEvent_t sorted = nullptr;
        int *err_host = nullptr;  // pinned copy of the lane's device error word
    };
    struct Lane {
        bsort_t ctx = nullptr;  // workspace and error word of the lane
        cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
        std::deque<Batch> running;
    };
    bsort_t h = nullptr;
    bsort_t hb = nullptr;  // lane B's own context
    Lane lane[2];
    uint64_t arena_bytes = 0;
    unsigned char *arena = nullptr;
    std::map<uint64_t, uint64_t> free_list;  // offset -> bytes, coalesced
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::deque<Req *> queue[2];                 // submitted, not admitted, per lane
    uint32_t inflight_large = 0;                // lane-B jobs admitted, not retired
    std::unordered_map<uint64_t, Req *> tickets;
    std::deque<uint64_t> finished;              // done, in completion order
    uint64_t next_ticket = 1;
    std::vector<Req *> staged;   // lane A: keys copied in (or on their way)
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int *> err_pool;
    std::vector<int *> err_blocks;  // pinned blocks the err_pool words come from
    // statistics
    uint64_t used = 0, peak = 0, batches = 0, done_count = 0, max_batch = 0;
    uint64_t large_jobs = 0, busy_ns = 0;
};

namespace {

uint64_t clock_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr uint64_t kServeAlign = 256;
// arena positions of a batch are key indices below 2^32 - 2^16
constexpr uint64_t kServeArenaMax = 15ull << 30;
constexpr uint64_t kServeDefaultBudget = 4ull << 30;

uint64_t key_bytes(bsort_key_type kt) { return kt == BSORT_U64 ? 8 : 4; }

// Lane of a job: 0 when a batch sorts it as a direct or sampled segment.
int lane_of(const bsort_t, bsort_key_type kt, uint64_t n)
{
    return n <= (kt == BSORT_U64 ? kBatchSampledMaxU64 : kBatchSampledMax) ? 0 : 1;
}

bool arena_alloc(bsort_server *S, uint64_t bytes, uint64_t *off)
{
    for (auto it = S->free_list.begin(); it != S->free_list.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const uint64_t rest = it->second - bytes;
        const uint64_t at = it->first + bytes;
        S->free_list.erase(it);
        if (rest) S->free_list[at] = rest;
        S->used += bytes;
        if (S->used > S->peak) S->peak = S->used;
        return true;
    }
    return false;
}

void arena_free(bsort_server *S, uint64_t off, uint64_t bytes)
{
    S->used -= bytes;
    auto it = S->free_list.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != S->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        S->free_list.erase(nx);
    }
    if (it != S->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            S->free_list.erase(it);
        }
    }
}

cudaEvent_t take_event(bsort_server *S)
{
    if (!S->ev_pool.empty()) {
        cudaEvent_t e = S->ev_pool.back();
        S->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// A pinned word for a batch's copy of its lane's error word.  Words come
// in blocks of kErrBlock from one pinned allocation each (pinning host
// memory is slow, and the request loop must not stall on it per batch).
constexpr int kErrBlock = 1024;

int *take_err(bsort_server *S)
{
    if (S->err_pool.empty()) {
        void *p = nullptr;
        if (cudaHostAlloc(&p, sizeof(int) * kErrBlock, cudaHostAllocDefault) != cudaSuccess)
            return nullptr;
        S->err_blocks.push_back(static_cast<int *>(p));
        for (int i = kErrBlock - 1; i >= 0; --i) S->err_pool.push_back(static_cast<int *>(p) + i);
    }
    int *w = S->err_pool.back();
    S->err_pool.pop_back();
    return w;
}

// Retire every job whose result is back in host memory.
bool serve_retire(bsort_server *S)
{
    bool any = false;
    for (auto &L : S->lane) {
        while (!L.running.empty()) {
            bsort_server::Batch &b = L.running.front();
            bool all = true;
            for (auto &r : b.reqs) {
                if (!r) continue;
                if (cudaEventQuery(r->ev) != cudaSuccess) {
                    all = false;
                    continue;
                }
                const uint64_t now = clock_ns();
                const int word = b.err_host ? *b.err_host : 0;
                std::lock_guard<std::mutex> lock(S->mu);
                arena_free(S, r->off, r->bytes);
                S->ev_pool.push_back(r->ev);
                r->ev = nullptr;
                r->done_ns = now;
                if (r->status == BSORT_ENOTREADY)
                    r->status = word == 0 ? BSORT_OK
                                          : (word == BSORT_ETIMEOUT ? BSORT_ETIMEOUT
                                                                   : BSORT_EINTERNAL);
                r->done = true;
                if (r->lane == 1) --S->inflight_large;
                S->finished.push_back(r->ticket);
                ++S->done_count;
                r = nullptr;  // the caller may free it once polled
                any = true;
            }
            if (!all) break;
            S->ev_pool.push_back(b.sorted);
            if (b.err_host) S->err_pool.push_back(b.err_host);
            L.running.pop_front();
        }
    }
    return any;
}

// Sort the jobs of one batch of a lane (in place in the arena), copy the
// lane's error word out, then copy every result out.
void serve_run(bsort_server *S, int li, const std::vector<bsort_server::Req *> &jobs)
{
    bsort_server::Lane &L = S->lane[li];
    bsort_t ctx = L.ctx;
    bsort_server::Batch b;
    b.reqs = jobs;
    b.err_host = take_err(S);
    const uint64_t start = clock_ns();
    const bsort_key_type kinds[3] = {BSORT_U32, BSORT_F32, BSORT_U64};
    for (bsort_key_type kt : kinds) {
        const uint64_t kb = key_bytes(kt);
        std::vector<SegSpan> spans;
        std::vector<bsort_server::Req *> owners;
        for (auto *r : jobs)
            if (r->kt == kt && r->status == BSORT_ENOTREADY) {
                spans.push_back({r->off / kb, r->n});
                owners.push_back(r);
            }
        // sub-batches whose workspace fits the lane's: the largest prefix
        // that fits, found by bisection (the workspace a batch needs grows
        // with its segments); a single job always fits
        auto fits = [&](size_t i, size_t j) {
            BatchPlan B;
            return make_batch_plan(ctx, kt, spans.data() + i, (uint32_t)(j - i), &B) ==
                       BSORT_OK &&
                   B.total <= ctx->ws_bytes;
        };
        size_t i = 0;
        while (i < spans.size()) {
            size_t j = spans.size();
            if (!fits(i, j)) {
                size_t lo = i + 1, hi = j - 1;  // largest end in [lo, hi] that fits
                while (lo < hi) {
                    const size_t mid = (lo + hi + 1) / 2;
                    if (fits(i, mid)) lo = mid;
                    else hi = mid - 1;
                }
                j = lo;
            }
            const bsort_status st = run_batch(ctx, kt, S->arena, S->arena, spans.data() + i,
                                              (uint32_t)(j - i), L.s_run);
            if (st != BSORT_OK)
                for (size_t q = i; q < j; ++q) owners[q]->status = st;
            i = j;
        }
    }
    if (b.err_host) {
        cudaMemcpyAsync(b.err_host, ctx->ws, sizeof(int), cudaMemcpyDeviceToHost, L.s_run);
        cudaMemsetAsync(ctx->ws, 0, sizeof(int), L.s_run);
    }
    b.sorted = take_event(S);
    cudaEventRecord(b.sorted, L.s_run);
    cudaStreamWaitEvent(L.s_out, b.sorted, 0);
    const uint32_t size = (uint32_t)jobs.size();
    for (auto *r : jobs) {
        r->start_ns = start;
        r->batch_size = size;
        if (r->status == BSORT_ENOTREADY)
            cudaMemcpyAsync(r->out, S->arena + r->off, r->n * key_bytes(r->kt),
                            cudaMemcpyDeviceToHost, L.s_out);
        r->ev = take_event(S);
        cudaEventRecord(r->ev, L.s_out);
    }
    ++S->batches;
    if (size > S->max_batch) S->max_batch = size;
    L.running.push_back(b);
}

// Admit queued jobs of each lane in arrival order while the arena has
// room, copying their keys in: small jobs wait for lane A's next batch; a
// large job is sorted on lane B right away (behind the ones before it), with
// at most kLargeDepth of them in flight so that the work queued on the
// device stays short (a deep queue makes enqueueing block in the driver).
constexpr uint32_t kLargeDepth = 4;

bool serve_admit(bsort_server *S)
{
    bool any = false;
    for (;;) {
        bsort_server::Req *r = nullptr;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            int li = -1;
            if (!S->queue[0].empty()) li = 0;
            else if (!S->queue[1].empty() && S->inflight_large < kLargeDepth) li = 1;
            if (li < 0) break;
            bsort_server::Req *head = S->queue[li].front();
            uint64_t off = 0;
            if (!arena_alloc(S, head->bytes, &off)) {
                // the small lane waits for room; the large lane may still go
                if (li == 0 && !S->queue[1].empty() && S->inflight_large < kLargeDepth) {
                    head = S->queue[1].front();
                    if (!arena_alloc(S, head->bytes, &off)) break;
                    li = 1;
                } else {
                    break;
                }
            }
            head->off = off;
            S->queue[li].pop_front();
            if (li == 1) ++S->inflight_large;
            r = head;
        }
        bsort_server::Lane &L = S->lane[r->lane];
        cudaError_t e = cudaMemcpyAsync(S->arena + r->off, r->in, r->n * key_bytes(r->kt),
                                        cudaMemcpyHostToDevice, L.s_in);
        if (e != cudaSuccess) r->status = BSORT_ECUDA;
        if (r->lane == 0) {
            S->staged.push_back(r);
        } else {
            ++S->large_jobs;
            cudaEvent_t in_done = take_event(S);
            cudaEventRecord(in_done, L.s_in);
            cudaStreamWaitEvent(L.s_run, in_done, 0);
            S->ev_pool.push_back(in_done);  // a later record does not affect this wait
            serve_run(S, 1, std::vector<bsort_server::Req *>(1, r));
        }
        any = true;
    }
    return any;
}

// Launch lane A's next batch when its sorting stream is idle.
bool serve_launch(bsort_server *S)
{
    bsort_server::Lane &L = S->lane[0];
    if (S->staged.empty()) return false;
    if (!L.running.empty() && cudaEventQuery(L.running.back().sorted) != cudaSuccess)
        return false;
    cudaEvent_t in_done = take_event(S);
    cudaEventRecord(in_done, L.s_in);
    cudaStreamWaitEvent(L.s_run, in_done, 0);
    S->ev_pool.push_back(in_done);
    serve_run(S, 0, S->staged);
    S->staged.clear();
    return true;
}

void serve_loop(bsort_server *S)
{
    cudaSetDevice(S->h->device);
    for (;;) {
        const uint64_t t0 = clock_ns();
        bool busy = serve_retire(S);
        busy |= serve_admit(S);
        busy |= serve_launch(S);
        if (busy) S->busy_ns += clock_ns() - t0;
        std::unique_lock<std::mutex> lock(S->mu);
        const bool idle = S->queue[0].empty() && S->queue[1].empty() && S->staged.empty() &&
                          S->lane[0].running.empty() &&
                          S->lane[1].running.empty();
        if (S->stop && idle) break;
        if (!busy) {
            if (idle) S->cv.wait_for(lock, std::chrono::milliseconds(5));
            else S->cv.wait_for(lock, std::chrono::microseconds(10));
        }
    }
}

bsort_status serve_start(bsort_t h)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    const uint64_t budget = h->serve_budget ? h->serve_budget : kServeDefaultBudget;
    bsort_server *S = new (std::nothrow) bsort_server();
    if (!S) return fail(h, BSORT_ENOMEM, "server state");
    S->h = h;
    uint64_t arena = budget / 2;
    if (arena > kServeArenaMax) arena = kServeArenaMax;
    arena = arena / kServeAlign * kServeAlign;
    S->arena_bytes = arena;
    // the rest of the budget: the two lanes' workspaces
    const uint64_t ws_lane = (budget - arena) / 2 / kAlign * kAlign;
    S->hb = new (std::nothrow) bsort_ctx();
    if (!S->hb) {
        delete S;
        return fail(h, BSORT_ENOMEM, "server state");
    }
    S->hb->device = h->device;
    S->hb->direct_max = h->direct_max;
    S->hb->direct_max_set = h->direct_max_set;
    if (!h->ws_fixed) {
        rs = ensure_workspace(h, ws_lane);
        if (rs == BSORT_OK) h->ws_fixed = true;
    }
    if (rs == BSORT_OK) rs = prepare(S->hb);
    if (rs == BSORT_OK) rs = ensure_workspace(S->hb, ws_lane);
    if (rs != BSORT_OK) {
        delete S->hb;
        delete S;
        return fail(h, rs, "serving workspace of %llu bytes", (unsigned long long)ws_lane);
    }
    S->hb->ws_fixed = true;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&S->arena), arena);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bsort_destroy(S->hb);
        delete S;
        return fail(h, BSORT_ENOMEM, "serving arena of %llu bytes: %s",
                    (unsigned long long)arena, cudaGetErrorString(e));
    }
    S->free_list[0] = arena;
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    S->lane[0].ctx = h;
    S->lane[1].ctx = S->hb;
    for (int li = 0; li < 2; ++li) {
        bsort_server::Lane &L = S->lane[li];
        const int prio = li == 0 ? hi_prio : lo_prio;
        if (cudaStreamCreateWithPriority(&L.s_in, cudaStreamNonBlocking, prio) != cudaSuccess ||
            cudaStreamCreateWithPriority(&L.s_run, cudaStreamNonBlocking, prio) != cudaSuccess ||
            cudaStreamCreateWithPriority(&L.s_out, cudaStreamNonBlocking, prio) != cudaSuccess) {
            cudaFree(S->arena);
            bsort_destroy(S->hb);
            delete S;
            return fail(h, BSORT_ECUDA, "stream creation failed");
        }
    }
    h->server = S;
    S->worker = std::thread(serve_loop, S);
    return BSORT_OK;
}

void serve_stop(bsort_t h)
{
    bsort_server *S = h->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    S->worker.join();
    cudaSetDevice(h->device);
    for (auto &L : S->lane) {
        cudaStreamSynchronize(L.s_in);
        cudaStreamSynchronize(L.s_run);
        cudaStreamSynchronize(L.s_out);
        cudaStreamDestroy(L.s_in);
        cudaStreamDestroy(L.s_run);
        cudaStreamDestroy(L.s_out);
    }
    for (auto &kv : S->tickets) delete kv.second;
    for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
    for (int *p : S->err_blocks) cudaFreeHost(p);
    cudaFree(S->arena);
    bsort_destroy(S->hb);
    delete S;
    h->server = nullptr;
}

bool overlaps(const void *a, uint64_t abytes, const void *b, uint64_t bbytes)
{
    const char *pa = static_cast<const char *>(a);
    const char *pb = static_cast<const char *>(b);
    return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace

extern "C" {

const char *bsort_status_string(bsort_status st)
{
    switch (st) {
    case BSORT_OK: return "BSORT_OK";
    case BSORT_EINVAL: return "BSORT_EINVAL";
    case BSORT_ENOMEM: return "BSORT_ENOMEM";
    case BSORT_ECUDA: return "BSORT_ECUDA";
    case BSORT_ETIMEOUT: return "BSORT_ETIMEOUT";
    case BSORT_EBUSY: return "BSORT_EBUSY";
    case BSORT_ENOTREADY: return "BSORT_ENOTREADY";
    case BSORT_EUNSUPPORTED: return "BSORT_EUNSUPPORTED";
    case BSORT_EINTERNAL: return "BSORT_EINTERNAL";
    }
    return "BSORT_UNKNOWN";
}

bsort_status bsort_create(const bsort_config *cfg, bsort_t *out)
{
    if (!out) return BSORT_EINVAL;
    *out = nullptr;
    bsort_t h = new (std::nothrow) bsort_ctx();
    if (!h) return BSORT_ENOMEM;
    if (cfg) {
        h->device = cfg->device;
        h->flags = cfg->flags;
        h->force_t = cfg->tile;
        h->force_s = cfg->samples;
        h->auto_b = cfg->buckets == BSORT_BUCKETS_AUTO;
        h->force_b = h->auto_b ? 0u : cfg->buckets;
        h->serve_budget = cfg->serve_budget_bytes;
        if (cfg->batch_direct_max) {
            if (cfg->batch_direct_max > 8u * (uint32_t)kMaxCapKeys) {
                delete h;
                return BSORT_EINVAL;
            }
            h->direct_max = cfg->batch_direct_max;
            h->direct_max_set = true;
        }
        if (cfg->flags &
            ~(uint32_t)(BSORT_FLAG_TIMING | BSORT_FLAG_LOW_MEMORY | BSORT_FLAG_GRAPHS |
                        BSORT_FLAG_MERGE_SORT | BSORT_FLAG_TEST_STALL_SCAN |
                        BSORT_FLAG_PLAN_MODEL | BSORT_FLAG_TEST_TWO_LEVEL)) {
            delete h;
            return BSORT_EINVAL;
        }
        if (cfg->workspace) {
            if (cfg->workspace_bytes < kAlign || (reinterpret_cast<uintptr_t>(cfg->workspace) % kAlign)) {
                delete h;
                return BSORT_EINVAL;
            }
            h->ws = cfg->workspace;
            h->ws_bytes = cfg->workspace_bytes;
            h->ws_fixed = true;
            cudaError_t e = cudaSetDevice(h->device);
            if (e == cudaSuccess) e = cudaMemset(h->ws, 0, kAlign);
            if (e != cudaSuccess) {
                delete h;
                return BSORT_ECUDA;
            }
        } else if (cfg->mem_budget_bytes) {
            cudaError_t e = cudaSetDevice(h->device);
            if (e != cudaSuccess) {
                delete h;
                return BSORT_ECUDA;
            }
            h->ws_fixed = false;
            bsort_status st = ensure_workspace(h, align_up(cfg->mem_budget_bytes));
            if (st != BSORT_OK) {
                delete h;
                return st;
            }
            h->ws_fixed = true;
        }
    }
    *out = h;
    return BSORT_OK;
}

bsort_status bsort_destroy(bsort_t h)
{
    if (!h) return BSORT_EINVAL;
    serve_stop(h);
    if (h->ws_owned && h->ws) {
        cudaSetDevice(h->device);
        cudaFree(h->ws);
    }
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    if (h->stage) cudaFreeHost(h->stage);
    drop_graphs(h);
    if (h->xfer) cudaStreamDestroy(h->xfer);
    for (int i = 0; i < 2 * kPipe + 2; ++i)
        if (h->xev[i]) cudaEventDestroy(h->xev[i]);
    if (h->events_made)
        for (int r = 0; r < kRing; ++r)
            for (int i = 0; i <= kMaxTimed; ++i) cudaEventDestroy(h->ev[r][i]);
    delete h;
    return BSORT_OK;
}

bsort_status bsort_plan(bsort_t h, bsort_key_type kt, uint32_t val_bytes, uint64_t n,
                        bsort_plan_info *out)
{
    if (!out) return fail(h, BSORT_EINVAL, "null plan pointer");
    Plan P;
    if (kt == BSORT_U64 && val_bytes != 0) {
        // pairs with 64-bit keys: two passes of the 32-bit pair sort (this
        // plan) and the scratch of run_pairs_u64, in-place case included
        if (val_bytes != 4 && val_bytes != 8)
            return fail(h, BSORT_EINVAL, "val_bytes must be 0, 4 or 8");
        if (n >= kMaxN)
            return fail(h, BSORT_EUNSUPPORTED, "n = %llu exceeds 2^32 - 2^16", (unsigned long long)n);
        bsort_status st = make_plan(h, BSORT_U32, 4, n, &P);
        if (st != BSORT_OK) return st;
        *out = P.info;
        out->workspace_bytes = align_up(P.total) + 5 * align_up(n * 4) + align_up(n * 8) +
                               align_up(n * (uint64_t)val_bytes);
        out->num_kernels = 2 * P.info.num_kernels + 3;
        return BSORT_OK;
    }
    bsort_status st = make_plan(h, kt, val_bytes, n, &P);
    if (st != BSORT_OK) return st;
    *out = P.info;
    return BSORT_OK;
}

bsort_status bsort_sort_keys(bsort_t h, bsort_key_type kt, const void *d_keys_in, void *d_keys_out,
                             uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (h->server) return fail(h, BSORT_EBUSY, "the handle serves requests (bsort_submit)");
    if (n && (!d_keys_in || !d_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    const uint64_t kb = kt == BSORT_U64 ? 8 : 4;
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * kb, d_keys_out, n * kb))
        return fail(h, BSORT_EINVAL, "input and output overlap partially");
    return run_sort_graph(h, kt, d_keys_in, nullptr, d_keys_out, nullptr, 0, n,
                          static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_sort_pairs(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              const void *d_vals_in, void *d_keys_out, void *d_vals_out,
                              uint32_t val_bytes, uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (h->server) return fail(h, BSORT_EBUSY, "the handle serves requests (bsort_submit)");
    if (val_bytes != 4 && val_bytes != 8) return fail(h, BSORT_EINVAL, "val_bytes must be 4 or 8");
    if (n && (!d_keys_in || !d_keys_out || !d_vals_in || !d_vals_out))
        return fail(h, BSORT_EINVAL, "null key/value pointer");
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 4, d_keys_out, n * 4))
        return fail(h, BSORT_EINVAL, "key input and output overlap partially");
    if (n && d_vals_in != d_vals_out &&
        overlaps(d_vals_in, n * val_bytes, d_vals_out, n * val_bytes))
        return fail(h, BSORT_EINVAL, "value input and output overlap partially");
    if (kt == BSORT_U64) {
        if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 8, d_keys_out, n * 8))
            return fail(h, BSORT_EINVAL, "key input and output overlap partially");
        return run_pairs_u64(h, d_keys_in, d_vals_in, d_keys_out, d_vals_out, val_bytes, n,
                             static_cast<cudaStream_t>(cuda_stream));
    }
    return run_sort_graph(h, kt, d_keys_in, d_vals_in, d_keys_out, d_vals_out, val_bytes, n,
                          static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_plan_batch(bsort_t h, bsort_key_type kt, const uint64_t *seg_offsets,
                              uint32_t num_segs, bsort_batch_info *out)
{
    if (!h || !out) return BSORT_EINVAL;
    std::vector<SegSpan> spans;
    bsort_status st = spans_from_offsets(h, seg_offsets, num_segs, &spans);
    if (st != BSORT_OK) return st;
    BatchPlan B;
    st = make_batch_plan(h, kt, spans.data(), num_segs, &B);
    if (st != BSORT_OK) return st;
    *out = B.info;
    return BSORT_OK;
}

bsort_status bsort_sort_batch(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              void *d_keys_out, const uint64_t *seg_offsets, uint32_t num_segs,
                              void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (h->server) return fail(h, BSORT_EBUSY, "the handle serves requests (bsort_submit)");
    if (num_segs && !seg_offsets) return fail(h, BSORT_EINVAL, "null segment offsets");
    const uint64_t end = num_segs ? seg_offsets[num_segs] : 0;
    const uint64_t kb = kt == BSORT_U64 ? 8 : 4;
    if (end && (!d_keys_in || !d_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    if (end && d_keys_in != d_keys_out && overlaps(d_keys_in, end * kb, d_keys_out, end * kb))
        return fail(h, BSORT_EINVAL, "input and output overlap partially");
    std::vector<SegSpan> spans;
    bsort_status st = spans_from_offsets(h, seg_offsets, num_segs, &spans);
    if (st != BSORT_OK) return st;
    return run_batch_graph(h, kt, d_keys_in, d_keys_out, spans.data(), num_segs,
                           static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_submit(bsort_t h, const bsort_request *req, uint64_t *ticket)
{
    if (!h || !req || !ticket) return BSORT_EINVAL;
    const bsort_key_type kt = req->key_type;
    if (kt != BSORT_U32 && kt != BSORT_F32 && kt != BSORT_U64)
        return fail(h, BSORT_EINVAL, "unknown key type %d", (int)kt);
    if (req->n && (!req->h_keys_in || !req->h_keys_out))
        return fail(h, BSORT_EINVAL, "null key pointer");
    if (req->n >= kMaxN) return fail(h, BSORT_EUNSUPPORTED, "n = %llu too large",
                                     (unsigned long long)req->n);
    if (!h->server) {
        bsort_status rs = serve_start(h);
        if (rs != BSORT_OK) return rs;
    }
    bsort_server *S = h->server;
    const uint64_t kb = key_bytes(kt);
    const uint64_t bytes = (req->n * kb + kServeAlign - 1) / kServeAlign * kServeAlign;
    if (bytes > S->arena_bytes)
        return fail(h, BSORT_ENOMEM, "request of %llu bytes exceeds the serving arena (%llu)",
                    (unsigned long long)bytes, (unsigned long long)S->arena_bytes);
    const int lane = lane_of(h, kt, req->n);
    if (req->n > 1) {  // its batch alone must fit the lane's workspace
        SegSpan one = {0, req->n};
        BatchPlan B;
        bsort_status rs = make_batch_plan(h, kt, &one, 1, &B);
        if (rs != BSORT_OK) return rs;
        const uint64_t ws = S->lane[lane].ctx->ws_bytes;
        if (B.total > ws)
            return fail(h, BSORT_ENOMEM, "request needs %llu workspace bytes, serving has %llu",
                        (unsigned long long)B.total, (unsigned long long)ws);
    }
    auto *r = new (std::nothrow) bsort_server::Req();
    if (!r) return fail(h, BSORT_ENOMEM, "request state");
    r->kt = kt;
    r->in = req->h_keys_in;
    r->out = req->h_keys_out;
    r->n = req->n;
    r->lane = lane;
    r->bytes = bytes ? bytes : kServeAlign;
    r->submit_ns = clock_ns();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        r->ticket = S->next_ticket++;
        S->tickets[r->ticket] = r;
        S->queue[r->lane].push_back(r);
    }
    S->cv.notify_one();
    *ticket = r->ticket;
    return BSORT_OK;
}

bsort_status bsort_poll(bsort_t h, uint64_t ticket, bsort_result *out)
{
    if (!h || !out) return BSORT_EINVAL;
    bsort_server *S = h->server;
    if (!S) return fail(h, BSORT_EINVAL, "no request was submitted on this handle");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return BSORT_EINVAL;
    bsort_server::Req *r = it->second;
    if (!r->done) return BSORT_ENOTREADY;
    out->status = r->status;
    out->batch_size = r->batch_size;
    out->submit_ns = r->submit_ns;
    out->start_ns = r->start_ns;
    out->done_ns = r->done_ns;
    S->tickets.erase(it);
    delete r;
    return BSORT_OK;
}

bsort_status bsort_poll_any(bsort_t h, uint64_t *tickets, bsort_result *results, uint32_t cap,
                            uint32_t *count)
{
    if (!h || !count || (cap && (!tickets || !results))) return BSORT_EINVAL;
    *count = 0;
    bsort_server *S = h->server;
    if (!S) return BSORT_OK;
    std::lock_guard<std::mutex> lock(S->mu);
    uint32_t k = 0;
    while (k < cap && !S->finished.empty()) {
        const uint64_t t = S->finished.front();
        S->finished.pop_front();
        auto it = S->tickets.find(t);
        if (it == S->tickets.end()) continue;  // already released by bsort_poll
        bsort_server::Req *r = it->second;
        tickets[k] = t;
        results[k].status = r->status;
        results[k].batch_size = r->batch_size;
        results[k].submit_ns = r->submit_ns;
        results[k].start_ns = r->start_ns;
        results[k].done_ns = r->done_ns;
        ++k;
        S->tickets.erase(it);
        delete r;
    }
    *count = k;
    return BSORT_OK;
}

bsort_status bsort_serve_stats(bsort_t h, bsort_serve_info *out)
{
    if (!h || !out) return BSORT_EINVAL;
    memset(out, 0, sizeof(*out));
    bsort_server *S = h->server;
    if (!S) return BSORT_OK;
    std::lock_guard<std::mutex> lock(S->mu);
    out->arena_bytes = S->arena_bytes;
    out->workspace_bytes = h->ws_bytes + S->hb->ws_bytes;
    out->arena_used_bytes = S->used;
    out->arena_peak_bytes = S->peak;
    out->queued = S->queue[0].size() + S->queue[1].size();
    out->completed = S->done_count;
    out->batches = S->batches;
    out->max_batch = S->max_batch;
    out->large_jobs = S->large_jobs;
    out->worker_busy_ns = S->busy_ns;
    return BSORT_OK;
}

uint64_t bsort_clock_ns(void) { return clock_ns(); }

bsort_status bsort_sort_keys_host(bsort_t h, bsort_key_type kt, const void *h_keys_in,
                                  void *h_keys_out, uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (h->server) return fail(h, BSORT_EBUSY, "the handle serves requests (bsort_submit)");
    if (n && (!h_keys_in || !h_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    if (n == 0) return BSORT_OK;
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    Plan P;
    rs = make_plan(h, kt, 0, n, &P);
    if (rs != BSORT_OK) return rs;
    // staging: one device copy of the keys placed after the job's workspace
    const uint64_t stage = P.total;
    const uint64_t bytes = n * (uint64_t)P.kb;
    rs = ensure_workspace(h, stage + align_up(bytes));
    if (rs != BSORT_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void *d_buf = static_cast<unsigned char *>(h->ws) + stage;
    const int groups = host_pipe_groups(n);
    if (P.kb == 4 && !P.wide && !P.info.single_tile && P.relocate && groups > 0 &&
        P.info.levels == 1) {
        // several sublists: copies overlap Steps 1-3 and Step 9
        rs = ensure_workspace(h, stage + align_up(bytes) + kAlign);
        if (rs != BSORT_OK) return rs;
        rs = ensure_pipe(h);
        if (rs != BSORT_OK) return rs;
        d_buf = static_cast<unsigned char *>(h->ws) + stage;
        HostPipe hp;
        hp.h_in = h_keys_in;
        hp.h_out = h_keys_out;
        hp.d_keys = d_buf;
        hp.ranges = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(h->ws) + stage +
                                                 align_up(bytes));
        hp.groups = groups;
        return run_sort(h, kt, d_buf, nullptr, d_buf, nullptr, 0, n, st, &hp);
    }
    cudaError_t e = cudaMemcpyAsync(d_buf, h_keys_in, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
    rs = run_sort(h, kt, d_buf, nullptr, d_buf, nullptr, 0, n, st);
    if (rs != BSORT_OK) return rs;
    e = cudaMemcpyAsync(h_keys_out, d_buf, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
    return BSORT_OK;
}

bsort_status bsort_sync(bsort_t h, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    if (!h->ws) return BSORT_OK;
    int word = 0;
    e = cudaMemcpy(&word, h->ws, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "read error word");
    if (word == 0) return BSORT_OK;
    int zero = 0;
    e = cudaMemcpy(h->ws, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "clear error word");
    if (word == BSORT_ETIMEOUT)
        return fail(h, BSORT_ETIMEOUT, "a bounded device wait ran out (scan look-back)");
    return fail(h, BSORT_EINTERNAL, "device consistency check failed (code %d)", word);
}

bsort_status bsort_get_intermediate(bsort_t h, bsort_intermediate which, void *h_dst,
                                    uint64_t bytes)
{
    if (!h || !h_dst) return BSORT_EINVAL;
    if (!h->have_last || h->last.info.single_tile || h->last.info.n == 0)
        return fail(h, BSORT_ENOTREADY, "no intermediates: no multi-sublist call yet");
    const Plan &P = h->last;
    uint64_t off = 0, size = 0;
    switch (which) {
    case BSORT_IM_TILES: off = P.off_tiles_k; size = P.info.n_padded * P.kb; break;
    case BSORT_IM_SAMPLES: off = P.off_samples; size = (uint64_t)P.n_rec * (P.wide ? 16 : 8); break;
    case BSORT_IM_SPLITTERS: off = P.off_spl; size = (uint64_t)P.info.b * (P.wide ? 16 : 8); break;
    case BSORT_IM_COUNTS: off = P.off_offsets; size = (uint64_t)P.n_runs * 4; break;
    case BSORT_IM_OFFSETS: off = P.off_offsets; size = (uint64_t)P.n_runs * 4; break;
    case BSORT_IM_RELOCATED:
        if (!P.relocate)
            return fail(h, BSORT_ENOTREADY,
                        "the relocated array is not materialised under BSORT_FLAG_LOW_MEMORY");
        off = P.off_reloc_k;
        size = P.info.n_padded * P.kb;
        break;
    default: return fail(h, BSORT_EINVAL, "unknown intermediate %d", (int)which);
    }
    if (bytes != size)
        return fail(h, BSORT_EINVAL, "intermediate %d has %llu bytes, %llu requested", (int)which,
                    (unsigned long long)size, (unsigned long long)bytes);
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (P.info.levels == 2 && (which == BSORT_IM_COUNTS || which == BSORT_IM_OFFSETS)) {
        // 64-bit offsets (ending with n' at index m*b), reported as uint32
        // where they fit
        if (P.info.n_padded >= (1ull << 32))
            return fail(h, BSORT_EUNSUPPORTED, "offsets of n' >= 2^32 do not fit uint32");
        std::vector<uint64_t> l((size_t)P.n_runs + 1);
        if (e == cudaSuccess)
            e = cudaMemcpy(l.data(), static_cast<unsigned char *>(h->ws) + P.off_off64,
                           l.size() * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy intermediate");
        uint32_t *a = static_cast<uint32_t *>(h_dst);
        for (uint32_t x = 0; x < P.n_runs; ++x)
            a[x] = (uint32_t)(which == BSORT_IM_COUNTS ? l[x + 1] - l[x] : l[x]);
        return BSORT_OK;
    }
    if (which == BSORT_IM_COUNTS) {
        // a_ij = l_(next run) - l_ij: the offsets array ends with n' at
        // index m*b (written with the run index of Step 8)
        std::vector<uint32_t> l((size_t)P.n_runs + 1);
        if (e == cudaSuccess)
            e = cudaMemcpy(l.data(), static_cast<unsigned char *>(h->ws) + off,
                           l.size() * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy intermediate");
        uint32_t *a = static_cast<uint32_t *>(h_dst);
        for (uint32_t x = 0; x < P.n_runs; ++x) a[x] = l[x + 1] - l[x];
        return BSORT_OK;
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(h_dst, static_cast<unsigned char *>(h->ws) + off, size,
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy intermediate");
    if (!P.wide && (which == BSORT_IM_SAMPLES || which == BSORT_IM_SPLITTERS)) {
        // records hold key << 32 | q (q = i*s + k); report key << 32 | p with
        // p = i*t + (k+1)w - 1, the sample's position in the sorted sublists
        const uint64_t s = P.info.s, t = P.info.t, w = P.info.w;
        uint64_t *rec = static_cast<uint64_t *>(h_dst);
        for (uint64_t x = 0; x < size / 8; ++x) {
            const uint64_t q = rec[x] & 0xFFFFFFFFull;
            const uint64_t pos = q / s * t + (q % s + 1) * w - 1;
            rec[x] = (rec[x] & ~0xFFFFFFFFull) | (pos & 0xFFFFFFFFull);
        }
    }
    return BSORT_OK;
}

bsort_status bsort_kernel_times(bsort_t h, float *ms, uint32_t count, uint32_t *written,
                                uint32_t *calls)
{
    if (!h || !written) return BSORT_EINVAL;
    *written = 0;
    if (calls) *calls = 0;
    if (!(h->flags & BSORT_FLAG_TIMING)) return fail(h, BSORT_EINVAL, "handle has no TIMING flag");
    if (h->calls_recorded == 0) return fail(h, BSORT_ENOTREADY, "no timed call yet");
    const int last = (int)((h->call_seq - 1) % kRing);
    const int nk = h->n_ev[last];
    cudaError_t e = cudaEventSynchronize(h->ev[last][nk]);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    uint32_t k = 0;
    for (; k < (uint32_t)nk && k < count; ++k)
        if (ms) ms[k] = 0.f;
    uint32_t used = 0;
    for (uint64_t c = 0; c < h->calls_recorded; ++c) {
        const int slot = (int)((h->call_seq - 1 - c) % kRing);
        if (h->n_ev[slot] != nk) continue;  // a call with another launch sequence
        for (uint32_t q = 0; q < k; ++q) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, h->ev[slot][q], h->ev[slot][q + 1]);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventElapsedTime");
            if (ms) ms[q] += t;
        }
        ++used;
    }
    h->calls_recorded = 0;
    *written = k;
    if (calls) *calls = used;
    return BSORT_OK;
}

const char *bsort_kernel_name(bsort_t h, uint32_t index)
{
    if (!h || index >= (uint32_t)kMaxTimed || !h->ev_name[index]) return "";
    return h->ev_name[index];
}

const char *bsort_last_error(bsort_t h)
{
    if (!h) return "null handle";
    return h->err;
}

}  // extern "C"

// ---------------------------------------------------------------- no-alloc entry
// Scratch for bsort_sort_keys_noalloc: a fixed device array in this file,
// sized for the largest plan of at most BSORT_NOALLOC_MAX_KEYS keys (about
// 8.5 MiB).  Host code may not use the symbol as a device address; its
// device address is looked up with cudaGetSymbolAddress once per CUDA
// context (the set-up also configures the kernels' attributes), keyed by the
// context's id, so that a device reset, which makes a new context and may
// place the array elsewhere, is noticed and the set-up done again.
namespace {
constexpr size_t kNoallocScratchBytes = (size_t)12 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
struct NoallocSetup {
    unsigned long long ctx_id = 0;  // context the entry below belongs to (0: none)
    void *scratch = nullptr;        // device address of g_noalloc_scratch there
};
NoallocSetup g_noalloc[kNoallocMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the calling thread's current CUDA context, or 0 when there is none
// or it cannot be read (the driver entry points are fetched through the
// runtime, so the library needs no link against the driver library).
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}
}  // namespace

extern "C" bsort_status bsort_sort_keys_noalloc(bsort_key_type kt, const void *d_keys_in,
                                                void *d_keys_out, uint64_t n,
                                                void *cuda_stream, int wait)
{
    if (n > BSORT_NOALLOC_MAX_KEYS) return BSORT_EINVAL;
    if (kt == BSORT_U64) return BSORT_EUNSUPPORTED;
    if (kt != BSORT_U32 && kt != BSORT_F32) return BSORT_EINVAL;
    if (n && (!d_keys_in || !d_keys_out)) return BSORT_EINVAL;
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 4, d_keys_out, n * 4))
        return BSORT_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices)
        return BSORT_ECUDA;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocSetup &S = g_noalloc[dev];
        const unsigned long long id = current_context_id();
        if (id == 0 || S.ctx_id != id) {
            // set-up for this context: the array's device address (this also
            // makes the context current if it was not) and kernel attributes
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return BSORT_ECUDA;
            if (init_kernels() != cudaSuccess) return BSORT_ECUDA;
            S.scratch = p;
            S.ctx_id = current_context_id();  // 0 if unreadable: set up again next call
        }
        scratch = S.scratch;
    }
    // a handle on the stack whose fixed workspace is the scratch array
    bsort_ctx ctx;
    ctx.device = dev;
    ctx.ws = scratch;
    ctx.ws_bytes = kNoallocScratchBytes;
    ctx.ws_fixed = true;
    ctx.ws_owned = false;
    ctx.kernels_ready = true;
    Plan P;
    bsort_status st = make_plan(&ctx, kt, 0, n, &P);
    if (st != BSORT_OK) return st;
    if (P.total > kNoallocScratchBytes) return BSORT_ENOMEM;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // The error word at the start of the array is not cleared here: kernels
    // only ever set it (first error wins), so a failure of a call made with
    // wait = 0 stays recorded until a call with wait != 0 reports and clears
    // it.  The array starts at zero when the library's device code is loaded.
    st = run_sort(&ctx, kt, d_keys_in, nullptr, d_keys_out, nullptr, 0, n, stream);
    if (st != BSORT_OK || !wait) return st;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return BSORT_ECUDA;
    int word = 0;
    if (cudaMemcpy(&word, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BSORT_ECUDA;
    if (word == 0) return BSORT_OK;
    if (cudaMemsetAsync(scratch, 0, sizeof(int), stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return BSORT_ECUDA;
    return word == BSORT_ETIMEOUT ? BSORT_ETIMEOUT : BSORT_EINTERNAL;
}
