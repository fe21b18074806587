// bsort_internal.h -- launch interface between the host runtime (bsort_api.cu)
// and the kernels (bsort_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bsort {

// Sort-unit shapes: one CTA sorts `cap` items, T threads x E items each.
// Keys-only units sort uint32 keys; pair units sort uint64 composite keys
// (key << 32 | local index) and gather the values afterwards.
constexpr int kMaxCapKeys = 32768;   // 1024 threads x 32 keys, 132 KB SMEM
constexpr int kMaxCapPairs = 16384;  // 1024 threads x 16 records, 136 KB SMEM
constexpr int kRecordChunk = 16384;  // Step-4 chunk sorted by one CTA
constexpr int kMergeTile = 4096;     // outputs per CTA in a Step-4 merge pass
constexpr int kScanChunk = 4096;     // items per CTA of the Step-7 scan

int smem_bytes_for_cap(int cap, bool pairs);

// Configure kernel attributes (max dynamic SMEM, cluster sizes) once per
// device.
cudaError_t init_kernels();
cudaError_t init_misc_kernels();
cudaError_t init_sort_keys_kernels();
cudaError_t init_sort_pairs_kernels();

// Steps 1-3: sort every sublist of t = ctas * chunk items with a cluster of
// `ctas` CTAs of `chunk` items each; write the sorted sublists (keys, and
// values for pairs) and s sample records per sublist.
// Steps 1-3 for sublists tile0 .. tile0 + m - 1.
// radix: a sublist of 32768 keys sorted by one CTA is sorted by digits
// (cta_radix_sort) instead of by comparisons; both give the same sublists.
cudaError_t launch_sublist_sort_keys(int chunk, int ctas, const void *keys_in, uint64_t n,
                                     uint32_t m, int is_f32, uint32_t s, uint32_t *tiles_k,
                                     uint64_t *samples, cudaStream_t st, uint32_t tile0 = 0,
                                     bool radix = false);
// The radix-sorting forms (bsort_sort_keys_radix.cu) that the functions
// above call for units of 32768 keys sorted by one CTA when `radix` is set.
cudaError_t init_sort_keys_radix_kernels();
cudaError_t launch_sublist_sort_keys_radix(int ctas, const void *keys_in, uint64_t n, uint32_t m,
                                           int is_f32, uint32_t s, uint32_t *tiles_k,
                                           uint64_t *samples, cudaStream_t st, uint32_t tile0);
struct GatherSrc;
cudaError_t launch_bucket_sort_keys_radix(int ctas, const void *src_k, const uint32_t *units,
                                          uint32_t max_units, uint64_t n, uint64_t n_pad,
                                          int is_f32, void *out_k, int *err, const GatherSrc &g,
                                          cudaStream_t st);
cudaError_t launch_bucket_sort_keys_range_radix(int ctas, const void *src_k,
                                                const uint32_t *units, const uint32_t *range,
                                                uint32_t grid_units, uint64_t n, uint64_t n_pad,
                                                int is_f32, void *out_k, int *err,
                                                cudaStream_t st);
cudaError_t launch_sublist_sort_pairs(int chunk, int ctas, const void *keys_in,
                                      const void *vals_in, uint64_t n, uint32_t m, int is_f32,
                                      int val_bytes, uint32_t s, uint32_t *tiles_k,
                                      void *tiles_v, uint64_t *samples, cudaStream_t st);

// Step 9: sort every unit with a cluster of `ctas` CTAs of `chunk` items
// (grid = max_units clusters, surplus clusters exit) and write the first n
// positions of the result.  With units == nullptr the whole input [0, n)
// is one unit read from src (raw keys, transformed on load).
// Where Step 9 reads its items: either a materialised relocated array
// (src_k/src_v, Step 8 run before), or, with runs != nullptr, straight from
// the sorted sublists: position y of the relocated order lies in the
// bucket-major run q (offsets[q] <= y < offsets[q+1]) of sublist i = q mod m,
// at rank srcb[q] + (y - offsets[q]).
struct GatherSrc {
    const uint32_t *offsets = nullptr;  // l_q, runs + 1 words
    const uint32_t *srcb = nullptr;     // sorted-sublist position of run q's first item
    const uint32_t *blk = nullptr;      // run index per kBlockItems positions
    uint32_t runs = 0;
};

// Step 9 launches over at most kLoopUnits units with clusters use a grid of
// that many clusters that loop over the device-side unit count.
constexpr uint32_t kLoopUnits = 256;

cudaError_t launch_bucket_sort_keys(int chunk, int ctas, const void *src_k, const uint32_t *units,
                                    uint32_t max_units, uint64_t n, uint64_t n_pad, int is_f32,
                                    void *out_k, int *err, const GatherSrc &g, cudaStream_t st,
                                    bool radix = false);
// Step 9 (keys) over units range[0] .. range[1] - 1 of a list, range in
// device memory, by a grid of grid_units units that loop over them.
cudaError_t launch_bucket_sort_keys_range(int chunk, int ctas, const void *src_k,
                                          const uint32_t *units, const uint32_t *range,
                                          uint32_t grid_units, uint64_t n, uint64_t n_pad,
                                          int is_f32, void *out_k, int *err, cudaStream_t st,
                                          bool radix = false);
// For G position slices [g*n_pad/G, (g+1)*n_pad/G): ranges[g] = first unit of
// the list whose begin is at or above g*n_pad/G (ranges[G] = the count).
cudaError_t launch_unit_ranges(const uint32_t *units, uint32_t n_pad, uint32_t G,
                               uint32_t *ranges, cudaStream_t st);
cudaError_t launch_bucket_sort_pairs(int chunk, int ctas, const void *src_k, const void *src_v,
                                     const uint32_t *units, uint32_t max_units, uint64_t n,
                                     uint64_t n_pad, int is_f32, int val_bytes, void *out_k,
                                     void *out_v, int *err, const GatherSrc &g, cudaStream_t st);

constexpr int kMaxBuckets = 12288;  // b (Step-9 unit packing keeps 16 b bytes in SMEM)
constexpr int kMaxBucketsTiers = 32768;  // b of a two-tier Step 9 (a unit per bucket: 4 b bytes)

// Step 4 (chunks): sort the n_rec records of src in chunks of kRecordChunk
// into dst (which holds n_pad = chunks * kRecordChunk records, the tail
// filled with all-ones); runs of s records are already sorted.  If the whole
// array is one chunk and spl != nullptr, also writes the b splitters (Step 5).
cudaError_t launch_records_chunk_sort(const uint64_t *src, uint64_t *dst, uint32_t n_rec,
                                      uint32_t n_pad, uint64_t *spl, uint32_t s,
                                      uint32_t b, cudaStream_t st);
// Step 4 (merges): merge sorted runs of length L of src into dst.
cudaError_t launch_merge_pass(const uint64_t *src, uint64_t *dst, uint32_t n_pad,
                              uint32_t L, cudaStream_t st);
// Step 5: b splitters g_j = sorted[floor((j+1) n_rec / b) - 1].
cudaError_t launch_select_splitters(const uint64_t *sorted, uint32_t n_rec, uint32_t b,
                                    uint64_t *spl, cudaStream_t st);

// Step 6: cum[j*m + i] = c_ij, the items of sorted sublist i at or below
// splitter j (bucket-major); jr: m * max(1, t / 1024) words of scratch.
// (sample records are key << 32 | q, q = i*s + k the sample's index)
cudaError_t launch_sample_index(const uint32_t *tiles_k, const uint64_t *spl, uint32_t t,
                                uint32_t s, uint32_t b, uint32_t m, uint32_t *jr, uint32_t *cum,
                                cudaStream_t st);
// Number of scratch words launch_sample_index (segments of 1024 keys) or
// launch_sample_index_seg_u64 (4096) needs for m sublists of t.
inline uint64_t sample_index_scratch_words(uint32_t t, uint32_t m, uint32_t seg_items = 1024u)
{
    return (uint64_t)m * (t > seg_items ? t / seg_items : 1u);
}

// Step 7: exclusive scan of n_items uint32 counts (decoupled look-back);
// status must hold ceil(n_items / kScanChunk) words and ticket one word,
// both zero on entry.
cudaError_t launch_scan(const uint32_t *in, uint32_t *out, uint32_t n_items,
                        unsigned long long *status, uint32_t *ticket, int *err,
                        cudaStream_t st);
// Step 7 from Step 6's cumulative counts (item e = j*m + i): counts[e] =
// a_ij = cum[e] - cum[e - m] (0 for j = 0; not written when counts is
// null), srcb[e] = i*t + cum[e - m] (the start of run A_ij), out = the
// exclusive prefix of a in bucket-major order.
// stall_first (a test of the bounded look-back wait): chunk 0 never
// publishes its prefix and the waits give up after a few thousand polls,
// recording DEV_TIMEOUT in *err (the offsets are then wrong).
cudaError_t launch_scan_cum(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t *counts,
                            uint32_t *srcb, uint32_t *out, uint32_t n_items,
                            unsigned long long *status, uint32_t *ticket, int *err,
                            cudaStream_t st, bool stall_first = false);

// Step 7 from the cumulative counts, one CTA per bucket row and no waits
// between CTAs: out[j*m + i] = l_ij for the b rows of m sublists (n' <
// 2^32); counts (a_ij) and srcb (i*t + c_i,j-1) are written when not null.
cudaError_t launch_row_scan(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t b,
                            uint32_t *counts, uint32_t *srcb, uint32_t *out, cudaStream_t st);

// Steps 4-5 by a radix sort of the records (bsort_records.cu), for
// records_radix_fits(m*s, b): launch_records_hist (zeroes the scratch of
// records_radix_scratch_bytes, then the four digit histograms), then
// launch_records_pass for p = 0 .. 3: samples -> rec_a -> rec_b -> rec_a,
// and the last pass (out null) writes the b splitters to spl.
bool records_radix_fits(uint32_t n_rec, uint32_t b);
uint64_t records_radix_scratch_bytes(uint32_t n_rec);
cudaError_t init_records_kernels();
cudaError_t launch_records_hist(const uint64_t *samples, uint32_t n_rec, void *scratch, int sms,
                                cudaStream_t st);
cudaError_t launch_records_pass(int p, const uint64_t *in, uint64_t *out, uint32_t n_rec,
                                uint32_t b, uint64_t *spl, void *scratch, int *err,
                                cudaStream_t st);

// Steps 7 and 8 in one kernel, one CTA per bucket (m <= 8192 sublists, m
// a multiple of 4): offsets[j*m + i] = l_ij (and offsets[m*b] = n_pad) and
// the relocated keys (values: val_bytes 0, 4 or 8), read from the sorted
// sublists by the cumulative counts alone.
bool bucket_relocate_fits(uint32_t m);
cudaError_t launch_bucket_relocate(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t b,
                                  uint32_t n_pad, const uint32_t *tiles_k, const void *tiles_v,
                                  int val_bytes, uint32_t *offsets, uint32_t *reloc_k,
                                  void *reloc_v, cudaStream_t st);

// Steps 7-8 of plans whose padded size reaches 2^32 (keys-only 32-bit keys,
// two levels): off64[e] = bucket-major exclusive prefix of a_ij (from the
// cumulative counts; off64[n_items] = n_pad; chunk_sums / chunk_pre hold one
// word per kScanChunk items), the relocation by source run by run, and
// the b + 1 bucket starts.
cudaError_t launch_scan_cum64(const uint32_t *cum, uint32_t m, uint32_t n_items,
                              uint32_t *chunk_sums, uint64_t *chunk_pre, uint64_t n_pad,
                              uint64_t *off64, cudaStream_t st);
cudaError_t launch_relocate_src64(const uint32_t *tiles_k, const uint32_t *cum,
                                  const uint64_t *off64, uint32_t m, uint32_t b, uint32_t t,
                                  uint32_t *reloc, cudaStream_t st);
cudaError_t launch_bucket_starts64(const uint64_t *off64, uint32_t m, uint32_t b, uint64_t n_pad,
                                   uint64_t *starts, cudaStream_t st);
// dst[x] = the float32 bits of the order-preserving code src[x].
cudaError_t launch_f32_decode(const uint32_t *src, uint32_t *dst, uint64_t n, cudaStream_t st);
// *to takes *from's error code if it has none yet.
cudaError_t launch_merge_error(const int *from, int *to, cudaStream_t st);

// Pairs with 64-bit keys as two stable passes of the 32-bit pair sort:
// lo[x] = low half of k64[x] and iota[x] = x; hi[x] = high half of
// k64[p1[x]]; out[y] = (k64, vals)[p1[p2[y]]].
cudaError_t launch_u64_split(const uint64_t *k64, uint32_t *lo, uint32_t *iota, uint64_t n,
                             cudaStream_t st);
cudaError_t launch_u64_gather_hi(const uint64_t *k64, const uint32_t *p1, uint32_t *hi,
                                 uint64_t n, cudaStream_t st);
cudaError_t launch_u64_final(const uint64_t *k64, const void *vals, int val_bytes,
                             const uint32_t *p1, const uint32_t *p2, uint64_t *out_k,
                             void *out_v, uint64_t n, cudaStream_t st);

constexpr int kRelocateSmemMax = 220 * 1024;
constexpr int kRelocPart = 8192;  // sublist items per Step-8 CTA

// Step 8: fill the relocated array B_1 ... B_b position by position from
// the runs A_ij (offsets: l in run order with the sentinel offsets[runs] =
// n_pad; srcb: sorted-sublist position of each run's first item, i*t +
// c_i(j-1), or null with cum, m and t given: then it is derived from the
// cumulative counts; blk: run index).
cudaError_t launch_relocate(const uint32_t *tiles_k, const void *tiles_v, const uint32_t *offsets,
                            const uint32_t *srcb, const uint32_t *blk, uint32_t runs,
                            uint32_t n_pad, int val_bytes, uint32_t *reloc_k, void *reloc_v,
                            cudaStream_t st, const uint32_t *cum = nullptr, uint32_t m = 0,
                            uint32_t t = 0);

// Positions per entry of the run index used by Step 9's gathering load.
constexpr int kBlockItems = 1024;

// Run index for the gathering load of Step 9: blk[b] = bucket-major run
// containing position b*kBlockItems of the relocated order; also writes
// offsets[runs] = n_pad (offsets must hold runs + 1 words).
cudaError_t launch_block_index(uint32_t *offsets, uint32_t runs, uint32_t n_pad, uint32_t *blk,
                               cudaStream_t st);

// Step 9 units: pack consecutive buckets into units of at most Q1 items; a
// bucket above Q1 (at most Q2) is a unit of its own, listed in units2 (when
// units2 == nullptr, Q1 = Q2 and all units are in units).  Each list holds
// 1 + 2*b words (count, then begin/end pairs).
// Step 9 units of a two-tier plan: one unit per bucket, in `units` (at
// most Q1 items) or `units2`; b <= kMaxBucketsTiers.
cudaError_t launch_units_each(const uint32_t *offsets, uint32_t m, uint32_t b, uint32_t n_pad,
                              uint32_t Q1, uint32_t Q2, uint32_t *units, uint32_t *units2,
                              int *err, cudaStream_t st);
cudaError_t launch_pack_units(const uint32_t *offsets, uint32_t m, uint32_t b,
                              uint32_t n_pad, uint32_t Q1, uint32_t Q2, uint32_t *units,
                              uint32_t *units2, int *err, cudaStream_t st);

// ---------------------------------------------------------------- 64-bit keys
// A sample record of a 64-bit-key sort: (key, p = i*t + r), compared key
// first, then p.
struct __align__(16) Rec128 {
    uint64_t key, p;
};

cudaError_t init_u64_kernels();
cudaError_t launch_sublist_sort_u64(int chunk, int ctas, const void *keys_in, uint64_t n,
                                    uint32_t m, uint32_t s, uint64_t *tiles, Rec128 *samples,
                                    cudaStream_t st);
// Step 4: merge runs of L records of src (N in all) pairwise into dst.
cudaError_t launch_rec_merge(const Rec128 *src, Rec128 *dst, uint32_t N, uint32_t L,
                             cudaStream_t st);
// Step 5: b splitters sorted[floor((j+1) N / b) - 1].
cudaError_t launch_select_splitters_u64(const Rec128 *sorted, uint32_t N, uint32_t b, Rec128 *spl,
                                        cudaStream_t st);
// Step 6: counts a_ij (bucket-major) and run starts i*t + c_i(j-1).
// Step 6 of 64-bit keys by segments of 4096 keys: cum[j*m + i] = c_ij
// (as launch_sample_index); jr: sample_index_scratch_words(t, m, 4096).
cudaError_t launch_sample_index_seg_u64(const uint64_t *tiles, const Rec128 *spl, uint32_t t,
                                        uint32_t b, uint32_t m, uint32_t *jr, uint32_t *cum,
                                        cudaStream_t st);
// Step 8 for 64-bit keys (no values).
cudaError_t launch_relocate_u64(const uint64_t *tiles_k, const uint32_t *offsets,
                                const uint32_t *srcb, const uint32_t *blk, uint32_t runs,
                                uint32_t n_pad, uint64_t *reloc_k, cudaStream_t st);
// Step 9 for 64-bit keys; units == nullptr sorts the whole input [0, n).
cudaError_t launch_bucket_sort_u64(int chunk, int ctas, const void *src, const uint32_t *units,
                                   uint32_t max_units, uint64_t n, uint64_t n_pad, void *out,
                                   int *err, cudaStream_t st);

// ---------------------------------------------------------------- batches
// Sublist size of sampled segments (one 1024 x 32 CTA per sublist).
constexpr int kSegTile = 32768;
// Sublist size of sampled segments of 64-bit keys (one 1024 x 16 CTA).
constexpr int kSegTileU64 = 16384;

// One sampled segment of a batch: sublists g0 .. g0+m-1 (padded positions
// [g0*t, (g0+m)*t)), s samples per sublist at records [rec, rec + m*s),
// b splitters at spl, runs (bucket-major) at [run0, run0 + m*b), n items at
// input / output offset out.
struct SegInfo {
    uint32_t g0, m, s, b, rec, spl, run0, out, n, pad;
};

cudaError_t init_batch_kernels();
// Whether the device schedules the 16-CTA cluster shape of 64-bit direct
// segments (known after init_batch_kernels).
bool batch_wide_cluster16();
// Direct segments: unit u = [seg[2u], seg[2u+1]) sorted by one unit of
// `ctas` CTAs of `chunk` keys (wide: 64-bit keys).
cudaError_t launch_seg_sort(int chunk, int ctas, bool wide, const void *keys_in, void *keys_out,
                            const uint32_t *seg, uint32_t nseg, int is_f32, int *err,
                            cudaStream_t st);
// Sampled segments, Steps 1-3 (sub_seg[g] = segment of sublist g).
cudaError_t launch_seg_sublist_sort(const uint32_t *keys_in, int is_f32, const uint32_t *sub_seg,
                                    uint32_t nsub, const SegInfo *segs, uint32_t *tiles_k,
                                    uint64_t *samples, cudaStream_t st);
// Steps 4-5, one CTA per segment (m*s <= kRecordChunk).
cudaError_t launch_seg_records(const uint64_t *samples, const SegInfo *segs, uint32_t nsegs,
                               uint64_t *spl, cudaStream_t st);
// Step 6: counts a_ij and run starts for every run of every segment.
cudaError_t launch_seg_sample_index(const uint32_t *tiles_k, const uint64_t *samples,
                                    const uint64_t *spl, const uint32_t *sub_seg, uint32_t nsub,
                                    const SegInfo *segs, uint32_t *counts, uint32_t *srcb,
                                    cudaStream_t st);
// Step 9: unit u = bucket units[2u+1] of segment units[2u], `chunk` keys max.
cudaError_t launch_seg_bucket_sort(int chunk, const uint32_t *reloc_k, const uint32_t *units,
                                   uint32_t nunits, const SegInfo *segs, const uint32_t *offsets,
                                   int is_f32, uint32_t *keys_out, int *err, cudaStream_t st);
// Sampled segments of 64-bit keys: the same steps with sublists of
// kSegTileU64 keys, sample records (key, p) of 16 bytes (Steps 4-5 need
// m*s <= 8192) and Step-9 units of at most kSegTileU64 keys; Steps 7-8 are
// the 32-bit path's scan and block index with launch_relocate_u64.
cudaError_t launch_seg_sublist_sort_u64(const uint64_t *keys_in, const uint32_t *sub_seg,
                                        uint32_t nsub, const SegInfo *segs, uint64_t *tiles_k,
                                        Rec128 *samples, cudaStream_t st);
cudaError_t launch_seg_records_u64(const Rec128 *samples, const SegInfo *segs, uint32_t nsegs,
                                   Rec128 *spl, cudaStream_t st);
cudaError_t launch_seg_sample_index_u64(const uint64_t *tiles_k, const Rec128 *samples,
                                        const Rec128 *spl, const uint32_t *sub_seg,
                                        uint32_t nsub, const SegInfo *segs, uint32_t *counts,
                                        uint32_t *srcb, cudaStream_t st);
cudaError_t launch_seg_bucket_sort_u64(const uint64_t *reloc_k, const uint32_t *units,
                                       uint32_t nunits, const SegInfo *segs,
                                       const uint32_t *offsets, uint64_t *keys_out, int *err,
                                       cudaStream_t st);
// Largest m*s of a sampled 64-bit segment (its records in shared memory).
constexpr uint32_t kSegRecordsU64 = 8192;

}  // namespace bsort
