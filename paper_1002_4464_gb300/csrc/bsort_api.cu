// bsort_api.cu -- host runtime behind include/bsort.h: the planner (Step 1
// parameters and the Step-9 unit), the workspace layout, the launch sequence
// of Algorithm 1 (Dehne & Zaboli, Section 4) and the error word.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/bsort.h"
#include "bsort_internal.h"

namespace {

using namespace bsort;

constexpr uint64_t kAlign = 256;
constexpr uint64_t kMaxN = (1ull << 32) - (1ull << 16);
constexpr uint64_t kMaxSamples = 8192;  // s per sublist (Step 6 keeps 12*s bytes in SMEM)
constexpr int kMaxTimed = 40;   // launches recorded per call
// Batches: segments up to kBatchDirectMax keys (default) are sorted whole by
// one unit; up to kBatchSampledMax by segment-aware sampling with sublists
// of kSegTile keys and s = kBatchSamples (m*s <= kRecordChunk); larger ones
// by one plain sort each.
constexpr uint32_t kBatchDirectMax = 131072;
constexpr uint32_t kBatchSampledMax = (uint32_t)kRecordChunk / 1024 * (uint32_t)kSegTile;
constexpr uint32_t kBatchSamples = 1024;
constexpr uint32_t kBatchUnit = 32768;  // Step-9 unit of sampled segments
constexpr int kRing = 64;       // calls kept for bsort_kernel_times

uint64_t align_up(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Full plan of one job, including the workspace layout.
struct Plan {
    bsort_plan_info info;
    bool pairs;
    int vb;          // value bytes (0 keys only)
    int tile_chunk;  // items per CTA in Step 2 (t = tile_ctas * tile_chunk)
    int unit_chunk;  // items per CTA in Step 9 (capacity = unit_ctas * unit_chunk)
    uint32_t n_rec;      // m*s sample records
    uint32_t n_runs;     // m*b runs A_ij (counts, offsets)
    uint32_t n_rec_pad;  // rounded up to kRecordChunk
    uint32_t scan_chunks;
    // workspace offsets (bytes)
    uint64_t off_hdr, off_tiles_k, off_tiles_v, off_reloc_k, off_reloc_v, off_samples,
        off_rec_a, off_rec_b, off_spl, off_counts, off_cum, off_offsets, off_status,
        off_units, off_srcb, off_blk, total;
    bool relocate;  // materialise Step 8 (else fused into Step 9's load)
};

}  // namespace

struct bsort_ctx {
    int device = 0;
    uint32_t flags = 0;
    uint32_t force_t = 0, force_s = 0, force_b = 0;
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
    void *stage = nullptr;           // pinned staging of batch descriptors
    uint64_t stage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;  // last copy out of stage
    bool stage_pending = false;
    uint64_t calls_recorded = 0;  // calls since the last bsort_kernel_times
    uint64_t call_seq = 0;
    bool events_made = false;
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

// Modelled cost of a plan, in units of one single-CTA sort pass over the
// items.  The factors are measured on GB300 at n = 2^28 uint32 keys: a
// Step-2 sublist sorted by a cluster of 2 / 4 / 8 CTAs costs 1.24 / 1.68 /
// 2.5 passes (distributed-shared-memory merge rounds; 8-CTA clusters also
// leave SMs idle), a Step-9 unit of 2 / 4 / 8 CTAs costs 1.65 / 2.1 / 3.1
// passes (rounds plus unit fill); the samples cost about 1.6e-2 passes per
// sample per key-equivalent (sorting, searching and scanning m*s records),
// and Step 8 about 0.35 passes (0.3 with runs of w >= 32 items).
double plan_cost(uint64_t np, uint64_t s, int tchunk, int tctas, int uchunk, int uctas)
{
    const double n = (double)np;
    auto f1 = [](int c) { return c == 1 ? 1.0 : c == 2 ? 1.24 : c == 4 ? 1.68 : 2.5; };
    auto f9 = [](int c) { return c == 1 ? 1.3 : c == 2 ? 1.65 : c == 4 ? 2.1 : 3.1; };
    const double chunk_levels = log2d(tchunk) / 15.0;  // smaller chunks sort faster
    const double unit_levels = log2d(uchunk) / 15.0;
    const double t = (double)tchunk * tctas;
    const double w = t / (double)s;
    const double samples = n / w;
    return n * (f1(tctas) * chunk_levels + f9(uctas) * unit_levels +
                (w >= 32 ? 0.3 : 0.35)) + samples * 0.45;
}

bsort_status make_plan(bsort_t h, bsort_key_type kt, uint32_t vb, uint64_t n, Plan *P)
{
    memset(P, 0, sizeof(*P));
    if (kt == BSORT_U64) return fail(h, BSORT_EUNSUPPORTED, "64-bit keys are not served by this build");
    if (kt != BSORT_U32 && kt != BSORT_F32) return fail(h, BSORT_EINVAL, "unknown key type %d", (int)kt);
    if (vb != 0 && vb != 4 && vb != 8) return fail(h, BSORT_EINVAL, "val_bytes must be 0, 4 or 8");
    if (n >= kMaxN) return fail(h, BSORT_EUNSUPPORTED, "n = %llu exceeds 2^32 - 2^16", (unsigned long long)n);
    const bool pairs = vb != 0;
    const int cm = max_chunk(pairs);
    P->pairs = pairs;
    P->vb = (int)vb;
    bsort_plan_info &I = P->info;
    I.n = n;
    const uint64_t forced_t = h ? h->force_t : 0;
    const uint64_t forced_s = h ? h->force_s : 0;
    const uint64_t forced_b = h ? h->force_b : 0;
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
        // candidates: forced t or every sublist shape; forced s or every
        // power of two with w = t/s >= 16 and s <= kMaxSamples.  The unit is
        // sized for b = s (or the forced b); the bucket count is chosen after.
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
                const double c = plan_cost(np, sv, tc, tk, uc, uk);
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
        uint64_t b = bs;  // the paper's rule, kept when s is given
        if (forced_b) {
            b = forced_b;
        } else if (!forced_s) {
            const uint64_t bmax = m * bs < (uint64_t)kMaxBuckets ? m * bs : (uint64_t)kMaxBuckets;
            const uint64_t bc = choose_buckets(I.n_padded, m, bs, I.unit_capacity, bmax);
            if (bc) b = bc;
        }
        I.b = (uint32_t)b;
        I.bucket_bound = bound_for(I.n_padded, m, bs, b);
        P->n_rec = (uint32_t)(m * bs);
        P->n_runs = (uint32_t)(m * b);
        P->n_rec_pad = (uint32_t)((P->n_rec + kRecordChunk - 1) / kRecordChunk * kRecordChunk);
        P->scan_chunks = (P->n_runs + kScanChunk - 1) / kScanChunk;
        uint32_t merges = 0;
        for (uint32_t L = kRecordChunk; L < P->n_rec_pad; L <<= 1) ++merges;
        const bool reloc = !(h && (h->flags & BSORT_FLAG_LOW_MEMORY));
        I.num_kernels = 1 /*S2-3*/ + 1 /*S4 chunks*/ + merges + (merges ? 1 : 0) /*S5*/ +
                        1 /*S6*/ + 1 /*S7*/ + 1 /*run index*/ + (reloc ? 1 : 0) /*S8*/ +
                        1 /*units*/ + 1 /*S9*/;
    }

    // workspace layout
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P->relocate = !(h && (h->flags & BSORT_FLAG_LOW_MEMORY));
    P->off_hdr = take(kAlign);  // error word (int) + scan ticket (uint32)
    if (!I.single_tile) {
        const uint64_t np = I.n_padded;
        P->off_tiles_k = take(np * 4);
        P->off_tiles_v = take(np * (uint64_t)vb);
        P->off_reloc_k = take(P->relocate ? np * 4 : 0);
        P->off_reloc_v = take(P->relocate ? np * (uint64_t)vb : 0);
        P->off_samples = take((uint64_t)P->n_rec * 8);
        P->off_rec_a = take((uint64_t)P->n_rec_pad * 8);
        P->off_rec_b = take(P->n_rec_pad > (uint32_t)kRecordChunk ? (uint64_t)P->n_rec_pad * 8 : 0);
        P->off_spl = take((uint64_t)I.b * 8);
        P->off_counts = take((uint64_t)P->n_runs * 4);
        P->off_cum = take((uint64_t)P->n_runs * 4);
        P->off_offsets = take(((uint64_t)P->n_runs + 1) * 4);
        P->off_status = take((uint64_t)P->scan_chunks * 8);
        P->off_units = take((1 + 2 * (uint64_t)I.b) * 4);
        P->off_srcb = take((uint64_t)P->n_runs * 4);
        P->off_blk = take((np + kBlockItems - 1) / kBlockItems * 4);
    }
    P->total = o;
    I.workspace_bytes = o;
    return BSORT_OK;
}

bsort_status ensure_workspace(bsort_t h, uint64_t bytes)
{
    if (bytes <= h->ws_bytes) return BSORT_OK;
    if (h->ws_fixed)
        return fail(h, BSORT_ENOMEM, "job needs %llu workspace bytes, handle has %llu",
                    (unsigned long long)bytes, (unsigned long long)h->ws_bytes);
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
    Seq(bsort_t h_, cudaStream_t st_) : h(h_), st(st_), timing((h_->flags & BSORT_FLAG_TIMING) != 0)
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

bsort_status run_sort(bsort_t h, bsort_key_type kt, const void *kin, const void *vin, void *kout,
                      void *vout, uint32_t vb, uint64_t n, cudaStream_t st)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
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
                                              n, is_f32, kout, err, none, st),
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
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + P.off_counts);
    uint32_t *cum = reinterpret_cast<uint32_t *>(ws + P.off_cum);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(ws + P.off_offsets);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + P.off_status);

    // look-back state must start at zero
    cudaError_t e = cudaMemsetAsync(status, 0, (size_t)P.scan_chunks * 8, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan status)");
    e = cudaMemsetAsync(ticket, 0, 4, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan ticket)");

    // Steps 1-3
    SEQ(P.pairs ? launch_sublist_sort_pairs(P.tile_chunk, (int)I.tile_ctas, kin, vin, n, I.m,
                                            is_f32, (int)vb, I.s, tiles_k, tiles_v, samples, st)
                : launch_sublist_sort_keys(P.tile_chunk, (int)I.tile_ctas, kin, n, I.m, is_f32,
                                           I.s, tiles_k, samples, st),
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
            uint64_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        SEQ(launch_select_splitters(src, P.n_rec, I.b, spl, st), "step5_splitters");
    }
    uint32_t *srcb = reinterpret_cast<uint32_t *>(ws + P.off_srcb);
    uint32_t *blk = reinterpret_cast<uint32_t *>(ws + P.off_blk);
    // Step 6
    SEQ(launch_sample_index(tiles_k, samples, spl, I.t, I.s, I.b, I.m, counts, cum, srcb, st),
        "step6_sample_index");
    // Step 7
    SEQ(launch_scan(counts, offsets, P.n_runs, status, ticket, err, st), "step7_prefix_sum");
    // Step 8: materialised, unless BSORT_FLAG_LOW_MEMORY fuses it into the
    // load of Step 9, which then gathers every unit from the runs A_ij
    GatherSrc g;
    SEQ(launch_block_index(offsets, P.n_runs, (uint32_t)I.n_padded, blk, st), "step8_run_index");
    if (P.relocate) {
        SEQ(launch_relocate(tiles_k, tiles_v, offsets, srcb, blk, P.n_runs,
                            (uint32_t)I.n_padded, (int)vb, reloc_k, reloc_v, st),
            "step8_relocate");
    }
    // Step 9: buckets packed into units of at most unit_capacity items
    uint32_t *units = reinterpret_cast<uint32_t *>(ws + P.off_units);
    SEQ(launch_pack_units(offsets, I.m, I.b, (uint32_t)I.n_padded, (uint32_t)I.unit_capacity,
                          units, err, st),
        "step9_pack_units");
    if (!P.relocate) {
        g.offsets = offsets;
        g.srcb = srcb;
        g.blk = blk;
        g.runs = P.n_runs;
    }
    const void *s9k = P.relocate ? (const void *)reloc_k : (const void *)tiles_k;
    const void *s9v = P.relocate ? (const void *)reloc_v : (const void *)tiles_v;
    SEQ(P.pairs ? launch_bucket_sort_pairs(P.unit_chunk, (int)I.unit_ctas, s9k, s9v, units, I.b,
                                           n, I.n_padded, is_f32, (int)vb, kout, vout, err, g,
                                           st)
                : launch_bucket_sort_keys(P.unit_chunk, (int)I.unit_ctas, s9k, units, I.b, n,
                                          I.n_padded, is_f32, kout, err, g, st),
        "step9_bucket_sort");
    return BSORT_OK;
}

// ---------------------------------------------------------------- batches
// Direct unit shapes, smallest first: (chunk, ctas).
const int kDirectShapes[][2] = {{2048, 1}, {4096, 1}, {8192, 1}, {16384, 1}, {32768, 1},
                                {32768, 2}, {32768, 4}, {32768, 8}};
constexpr int kNumDirect = 8;
const char *const kDirectNames[kNumDirect] = {
    "batch_direct_2048", "batch_direct_4096", "batch_direct_8192", "batch_direct_16384",
    "batch_direct_32768", "batch_direct_2x32768", "batch_direct_4x32768", "batch_direct_8x32768"};

// Host plan of one batch: direct lists per shape, sampled segments with
// their sublists and buckets, plain-sorted large segments, and the
// workspace layout (descriptors first, copied from pinned staging).
struct BatchPlan {
    bsort_batch_info info;
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

bsort_status make_batch_plan(bsort_t h, bsort_key_type kt, const uint64_t *segoff,
                             uint32_t nsegs, BatchPlan *B)
{
    if (kt == BSORT_U64) return fail(h, BSORT_EUNSUPPORTED, "64-bit keys are not served by this build");
    if (kt != BSORT_U32 && kt != BSORT_F32) return fail(h, BSORT_EINVAL, "unknown key type %d", (int)kt);
    if (nsegs && !segoff) return fail(h, BSORT_EINVAL, "null segment offsets");
    bsort_batch_info &I = B->info;
    memset(&I, 0, sizeof(I));
    I.num_segs = nsegs;
    if (nsegs == 0) return BSORT_OK;
    if (segoff[nsegs] >= kMaxN)
        return fail(h, BSORT_EUNSUPPORTED, "segment end %llu exceeds 2^32 - 2^16",
                    (unsigned long long)segoff[nsegs]);
    const uint32_t dmax = h->direct_max;
    uint64_t g = 0;  // sublists so far
    for (uint32_t q = 0; q < nsegs; ++q) {
        if (segoff[q + 1] < segoff[q])
            return fail(h, BSORT_EINVAL, "segment offsets decrease at %u", q);
        const uint64_t a = segoff[q], n = segoff[q + 1] - segoff[q];
        I.n += n;
        if (n <= 1) continue;  // nothing to order (a copy when out != in)
        if (n <= dmax) {
            int c = 0;
            while ((uint64_t)kDirectShapes[c][0] * kDirectShapes[c][1] < n) ++c;
            B->direct[c].push_back((uint32_t)a);
            B->direct[c].push_back((uint32_t)(a + n));
            ++I.direct_segs;
        } else if (n <= kBatchSampledMax) {
            SegInfo sg = {};
            sg.g0 = (uint32_t)g;
            sg.m = (uint32_t)((n + kSegTile - 1) / kSegTile);
            sg.s = kBatchSamples;
            const uint64_t np = (uint64_t)sg.m * kSegTile;
            uint64_t lo = 1, hi = (uint64_t)sg.m * sg.s;  // smallest b whose bound fits a unit
            while (lo < hi) {
                const uint64_t mid = (lo + hi) / 2;
                if (bound_for(np, sg.m, sg.s, mid) <= kBatchUnit) hi = mid;
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
    if (g * kSegTile >= kMaxN) return fail(h, BSORT_EUNSUPPORTED, "padded sampled segments exceed 2^32");
    B->n_pad = g * kSegTile;
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
        B->off_tiles = take(B->n_pad * 4);
        B->off_reloc = take(B->n_pad * 4);
        B->off_samples = take((uint64_t)B->nrec * 8);
        B->off_spl = take((uint64_t)B->nspl * 8);
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

bsort_status run_batch(bsort_t h, bsort_key_type kt, const void *kin, void *kout,
                       const uint64_t *segoff, uint32_t nsegs, cudaStream_t st)
{
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    BatchPlan B;
    rs = make_batch_plan(h, kt, segoff, nsegs, &B);
    if (rs != BSORT_OK) return rs;
    if (B.info.n == 0) return BSORT_OK;
    rs = ensure_workspace(h, B.total);
    if (rs != BSORT_OK) return rs;
    cudaError_t e;
    // segments of one key: copies
    if (kout != kin)
        for (uint32_t q = 0; q < nsegs; ++q)
            if (segoff[q + 1] - segoff[q] == 1) {
                e = cudaMemcpyAsync(static_cast<uint32_t *>(kout) + segoff[q],
                                    static_cast<const uint32_t *>(kin) + segoff[q], 4,
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
    if (B.d_words) {
        // descriptors: pinned staging -> workspace (the staging is reused
        // only after the previous copy out of it has completed)
        const uint64_t bytes = B.d_words * 4;
        if (h->stage_pending) {
            e = cudaEventSynchronize(h->stage_ev);
            if (e != cudaSuccess) return cuda_fail(h, e, "wait for the staging copy");
            h->stage_pending = false;
        }
        if (bytes > h->stage_bytes) {
            if (h->stage) cudaFreeHost(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
            e = cudaHostAlloc(&h->stage, bytes, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(h, BSORT_ENOMEM, "pinned staging of %llu bytes: %s",
                            (unsigned long long)bytes, cudaGetErrorString(e));
            }
            h->stage_bytes = bytes;
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
        SEQ(launch_seg_sort(kDirectShapes[c][0], kDirectShapes[c][1], ki, ko, desc + B.d_direct[c],
                            cnt, is_f32, err, st),
            kDirectNames[c]);
    }
    // sampled segments: Algorithm 1, segment-aware
    if (!B.segs.empty()) {
        const uint32_t nsub = B.info.sublists;
        const uint32_t *sub_seg = desc + B.d_sub;
        const SegInfo *segs = reinterpret_cast<const SegInfo *>(desc + B.d_segs);
        const uint32_t *units = desc + B.d_units;
        uint32_t *tiles = reinterpret_cast<uint32_t *>(ws + B.off_tiles);
        uint32_t *reloc = reinterpret_cast<uint32_t *>(ws + B.off_reloc);
        uint64_t *samples = reinterpret_cast<uint64_t *>(ws + B.off_samples);
        uint64_t *spl = reinterpret_cast<uint64_t *>(ws + B.off_spl);
        uint32_t *counts = reinterpret_cast<uint32_t *>(ws + B.off_counts);
        uint32_t *offsets = reinterpret_cast<uint32_t *>(ws + B.off_offsets);
        uint32_t *srcb = reinterpret_cast<uint32_t *>(ws + B.off_srcb);
        unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + B.off_status);
        uint32_t *blk = reinterpret_cast<uint32_t *>(ws + B.off_blk);
        e = cudaMemsetAsync(status, 0, (size_t)B.scan_chunks * 8, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan status)");
        e = cudaMemsetAsync(ticket, 0, 4, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset(scan ticket)");
        SEQ(launch_seg_sublist_sort(ki, is_f32, sub_seg, nsub, segs, tiles, samples, st),
            "batch_step1_3_sublist_sort");
        SEQ(launch_seg_records(samples, segs, B.info.sampled_segs, spl, st),
            "batch_step4_5_samples");
        SEQ(launch_seg_sample_index(tiles, samples, spl, sub_seg, nsub, segs, counts, srcb, st),
            "batch_step6_sample_index");
        SEQ(launch_scan(counts, offsets, B.runs, status, ticket, err, st), "batch_step7_prefix_sum");
        SEQ(launch_block_index(offsets, B.runs, (uint32_t)B.n_pad, blk, st), "batch_step8_run_index");
        SEQ(launch_relocate(tiles, nullptr, offsets, srcb, blk, B.runs, (uint32_t)B.n_pad, 0,
                            reloc, nullptr, st),
            "batch_step8_relocate");
        SEQ(launch_seg_bucket_sort((int)kBatchUnit, reloc, units, B.info.buckets, segs, offsets,
                                   is_f32, ko, err, st),
            "batch_step9_bucket_sort");
    }
    // large segments: one plain sort each, after the batch (same stream)
    for (const auto &lg : B.large) {
        rs = run_sort(h, kt, ki + lg.first, nullptr, ko + lg.first, nullptr, 0, lg.second, st);
        if (rs != BSORT_OK) return rs;
    }
    return BSORT_OK;
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
        h->force_b = cfg->buckets;
        if (cfg->batch_direct_max) {
            if (cfg->batch_direct_max > 8u * (uint32_t)kMaxCapKeys) {
                delete h;
                return BSORT_EINVAL;
            }
            h->direct_max = cfg->batch_direct_max;
        }
        if (cfg->flags & ~(uint32_t)(BSORT_FLAG_TIMING | BSORT_FLAG_LOW_MEMORY)) {
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
    if (h->ws_owned && h->ws) {
        cudaSetDevice(h->device);
        cudaFree(h->ws);
    }
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    if (h->stage) cudaFreeHost(h->stage);
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
    bsort_status st = make_plan(h, kt, val_bytes, n, &P);
    if (st != BSORT_OK) return st;
    *out = P.info;
    return BSORT_OK;
}

bsort_status bsort_sort_keys(bsort_t h, bsort_key_type kt, const void *d_keys_in, void *d_keys_out,
                             uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (n && (!d_keys_in || !d_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 4, d_keys_out, n * 4))
        return fail(h, BSORT_EINVAL, "input and output overlap partially");
    return run_sort(h, kt, d_keys_in, nullptr, d_keys_out, nullptr, 0, n,
                    static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_sort_pairs(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              const void *d_vals_in, void *d_keys_out, void *d_vals_out,
                              uint32_t val_bytes, uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (val_bytes != 4 && val_bytes != 8) return fail(h, BSORT_EINVAL, "val_bytes must be 4 or 8");
    if (n && (!d_keys_in || !d_keys_out || !d_vals_in || !d_vals_out))
        return fail(h, BSORT_EINVAL, "null key/value pointer");
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 4, d_keys_out, n * 4))
        return fail(h, BSORT_EINVAL, "key input and output overlap partially");
    if (n && d_vals_in != d_vals_out &&
        overlaps(d_vals_in, n * val_bytes, d_vals_out, n * val_bytes))
        return fail(h, BSORT_EINVAL, "value input and output overlap partially");
    return run_sort(h, kt, d_keys_in, d_vals_in, d_keys_out, d_vals_out, val_bytes, n,
                    static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_plan_batch(bsort_t h, bsort_key_type kt, const uint64_t *seg_offsets,
                              uint32_t num_segs, bsort_batch_info *out)
{
    if (!h || !out) return BSORT_EINVAL;
    BatchPlan B;
    bsort_status st = make_batch_plan(h, kt, seg_offsets, num_segs, &B);
    if (st != BSORT_OK) return st;
    *out = B.info;
    return BSORT_OK;
}

bsort_status bsort_sort_batch(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              void *d_keys_out, const uint64_t *seg_offsets, uint32_t num_segs,
                              void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (num_segs && !seg_offsets) return fail(h, BSORT_EINVAL, "null segment offsets");
    const uint64_t end = num_segs ? seg_offsets[num_segs] : 0;
    if (end && (!d_keys_in || !d_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    if (end && d_keys_in != d_keys_out && overlaps(d_keys_in, end * 4, d_keys_out, end * 4))
        return fail(h, BSORT_EINVAL, "input and output overlap partially");
    return run_batch(h, kt, d_keys_in, d_keys_out, seg_offsets, num_segs,
                     static_cast<cudaStream_t>(cuda_stream));
}

bsort_status bsort_sort_keys_host(bsort_t h, bsort_key_type kt, const void *h_keys_in,
                                  void *h_keys_out, uint64_t n, void *cuda_stream)
{
    if (!h) return BSORT_EINVAL;
    if (n && (!h_keys_in || !h_keys_out)) return fail(h, BSORT_EINVAL, "null key pointer");
    if (n == 0) return BSORT_OK;
    bsort_status rs = prepare(h);
    if (rs != BSORT_OK) return rs;
    Plan P;
    rs = make_plan(h, kt, 0, n, &P);
    if (rs != BSORT_OK) return rs;
    // staging: one device copy of the keys placed after the job's workspace
    const uint64_t stage = P.total;
    rs = ensure_workspace(h, stage + align_up(n * 4));
    if (rs != BSORT_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void *d_buf = static_cast<unsigned char *>(h->ws) + stage;
    cudaError_t e = cudaMemcpyAsync(d_buf, h_keys_in, n * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
    rs = run_sort(h, kt, d_buf, nullptr, d_buf, nullptr, 0, n, st);
    if (rs != BSORT_OK) return rs;
    e = cudaMemcpyAsync(h_keys_out, d_buf, n * 4, cudaMemcpyDeviceToHost, st);
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
    case BSORT_IM_TILES: off = P.off_tiles_k; size = P.info.n_padded * 4; break;
    case BSORT_IM_SAMPLES: off = P.off_samples; size = (uint64_t)P.n_rec * 8; break;
    case BSORT_IM_SPLITTERS: off = P.off_spl; size = (uint64_t)P.info.b * 8; break;
    case BSORT_IM_COUNTS: off = P.off_counts; size = (uint64_t)P.n_runs * 4; break;
    case BSORT_IM_OFFSETS: off = P.off_offsets; size = (uint64_t)P.n_runs * 4; break;
    case BSORT_IM_RELOCATED:
        if (!P.relocate)
            return fail(h, BSORT_ENOTREADY,
                        "the relocated array is not materialised under BSORT_FLAG_LOW_MEMORY");
        off = P.off_reloc_k;
        size = P.info.n_padded * 4;
        break;
    default: return fail(h, BSORT_EINVAL, "unknown intermediate %d", (int)which);
    }
    if (bytes != size)
        return fail(h, BSORT_EINVAL, "intermediate %d has %llu bytes, %llu requested", (int)which,
                    (unsigned long long)size, (unsigned long long)bytes);
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(h_dst, static_cast<unsigned char *>(h->ws) + off, size,
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy intermediate");
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
// 8.5 MiB).  Host code may not use the symbol as a device address; the
// device address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr size_t kNoallocScratchBytes = (size_t)12 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoallocMaxDevices] = {};
}  // namespace

extern "C" bsort_status bsort_sort_keys_noalloc(bsort_key_type kt, const void *d_keys_in,
                                                void *d_keys_out, uint64_t n,
                                                void *cuda_stream, int wait)
{
    if (n > BSORT_NOALLOC_MAX_KEYS) return BSORT_EINVAL;
    if (n && (!d_keys_in || !d_keys_out)) return BSORT_EINVAL;
    if (n && d_keys_in != d_keys_out && overlaps(d_keys_in, n * 4, d_keys_out, n * 4))
        return BSORT_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices)
        return BSORT_ECUDA;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return BSORT_ECUDA;
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // a handle on the stack whose fixed workspace is the scratch array
    bsort_ctx ctx;
    ctx.device = dev;
    ctx.ws = scratch;
    ctx.ws_bytes = kNoallocScratchBytes;
    ctx.ws_fixed = true;
    ctx.ws_owned = false;
    Plan P;
    bsort_status st = make_plan(&ctx, kt, 0, n, &P);
    if (st != BSORT_OK) return st;
    if (P.total > kNoallocScratchBytes) return BSORT_ENOMEM;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // the array keeps the previous call's contents: the error word must start
    // at zero (the scan's state is cleared by the sort itself)
    if (cudaMemsetAsync(scratch, 0, kAlign, stream) != cudaSuccess) return BSORT_ECUDA;
    st = run_sort(&ctx, kt, d_keys_in, nullptr, d_keys_out, nullptr, 0, n, stream);
    if (st != BSORT_OK || !wait) return st;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return BSORT_ECUDA;
    int word = 0;
    if (cudaMemcpy(&word, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BSORT_ECUDA;
    if (word == 0) return BSORT_OK;
    return word == BSORT_ETIMEOUT ? BSORT_ETIMEOUT : BSORT_EINTERNAL;
}
