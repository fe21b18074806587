// bsort_kernels.cu -- the kernels of GPU Bucket Sort (Dehne & Zaboli,
// Section 4, Algorithm 1) for sm_103a, and their launch wrappers.
//
//   Steps 1-3  k_sublist_sort      (bsort_sort.cuh) sort each sublist, emit samples
//   Step 4     k_rec_hist, k_rec_pass  (bsort_records.cu) radix sort of the
//                                  sample records, splitters from its last pass;
//              k_records_sort      or: sort the s*m samples in chunks of 16K ...
//              k_merge_pass        ... then merge-path passes through L2
//   Step 5     k_select_splitters  b evenly spaced sorted samples
//   Step 6     k_seg_ranges        splitters per sublist segment ...
//              k_sample_index_grp  ... located in the segment (shared memory)
//   Step 7-8   k_bucket_relocate   per bucket: scan of its count row, then its runs moved
//   Step 7     k_row_scan          or: one scan per bucket row of the counts,
//              k_scan              or (batches): bucket-major scan with look-back
//   Step 8     k_relocate          then: move each run A_ij to l_ij
//   Step 9     k_units_each / k_pack_units  a unit per bucket, or buckets packed
//              k_bucket_sort       (bsort_sort.cuh) sort each unit
//
// Items are compared in composite order (key, position): keys-only sorts
// compare keys (equal keys are indistinguishable), pair sorts compare the
// 64-bit word key << 32 | local index, which makes them stable, and the
// sample records of Steps 3-6 are key << 32 | q with q = i*s + k, the
// sample's index (its position i*t + (k+1)w - 1 grows with q).
#include "bsort_device.cuh"
#include "bsort_internal.h"

namespace bsort {

// ============================================================ Step 4 (chunks)
// The records of one sublist (s consecutive records) are already sorted, so
// when s >= 32*E the chunk is loaded as sorted runs (odd runs reversed) and
// only the remaining merge levels run; otherwise the chunk is sorted whole.
template <int T, int E>
__global__ void __launch_bounds__(T, 1)
k_records_sort(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, uint32_t n_rec,
               uint64_t *__restrict__ spl, uint32_t s, uint32_t b)
{
    constexpr int CAP = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * CAP;
    if (s >= 32u * E && s < (uint32_t)CAP) {
        // all E loads of a thread are issued before its first store
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const uint64_t g = base + (uint64_t)(k * T + tid);
            r[k] = g < n_rec ? src[g] : 0xFFFFFFFFFFFFFFFFull;
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            const int q = x / (int)s, o = x % (int)s;
            const int pos = (q & 1) ? q * (int)s + (int)s - 1 - o : x;
            sm[pidx<uint64_t>(pos)] = r[k];
        }
        __syncthreads();
        cta_merge_runs<uint64_t, T, E>(sm, (int)s);
    } else {
        uint64_t v[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const uint64_t x = base + wb_pos<E>(warp, lane, k);
            v[k] = x < n_rec ? src[x] : 0xFFFFFFFFFFFFFFFFull;
        }
        cta_sort<uint64_t, T, E>(v, sm);
    }
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        dst[base + x] = sm[pidx<uint64_t>(x)];
    }
    if (spl != nullptr) {  // whole sample array in this one chunk: Step 5
        for (uint32_t j = tid; j < b; j += T)
            spl[j] = sm[pidx<uint64_t>((int)((uint64_t)(j + 1) * n_rec / b - 1))];
    }
}

// ============================================================ Step 4 (merges)
// Co-rank of a merge path (items of A among the first d outputs, A first on
// ties) found by one warp: each round the 32 lanes test 32 evenly spaced
// candidates and the range shrinks to one gap (about 32x).
__device__ __forceinline__ uint32_t merge_path_warp(const uint64_t *A, uint32_t la,
                                                    const uint64_t *B, uint32_t lb, uint32_t d,
                                                    int lane)
{
    uint32_t lo = d > lb ? d - lb : 0;
    uint32_t hi = d < la ? d : la;
    // invariant: the answer i is in [lo, hi]; pred(i) = A[i] > B[d-1-i] is
    // monotone (false ... true) on [lo, hi), and the answer is the first true
    while (hi - lo > 32) {
        const uint32_t span = hi - lo;
        const uint32_t c = lo + (uint32_t)(((uint64_t)span * (lane + 1)) / 33);  // in [lo, hi)
        const bool pred = A[c] > B[d - 1 - c];
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
        if (ball == 0) {
            lo = lo + (uint32_t)(((uint64_t)span * 32) / 33) + 1;
        } else {
            const int f = __ffs(ball) - 1;  // first candidate where pred holds
            const uint32_t cf = lo + (uint32_t)(((uint64_t)span * (f + 1)) / 33);
            const uint32_t cp = f ? lo + (uint32_t)(((uint64_t)span * f) / 33) + 1 : lo;
            lo = cp;
            hi = cf;
        }
    }
    // final: at most 32 candidates lo .. hi-1, one per lane
    const uint32_t c = lo + lane;
    const bool pred = c < hi ? (A[c] > B[d - 1 - c]) : true;
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
    return ball ? lo + (uint32_t)(__ffs(ball) - 1) : hi;
}

// One CTA produces kMergeTile outputs of the merge of two runs: it finds
// the input ranges of its outputs by merge path in global memory, stages
// them in SMEM, merges per thread, and writes back through SMEM.
template <int T, int E>
__global__ void __launch_bounds__(T, 4)
k_merge_pass(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, uint32_t n_pad,
             uint32_t L)
{
    constexpr int TILE = T * E;
    __shared__ uint64_t sm[padded_elems<uint64_t>(TILE)];
    __shared__ uint32_t s_split[2];
    const int tid = threadIdx.x;
    const uint32_t o0 = blockIdx.x * TILE;
    const uint32_t a0 = o0 / (2 * L) * (2 * L);
    const uint32_t b0 = a0 + L;
    const uint32_t la = min(L, n_pad - a0);
    const uint32_t lb = b0 < n_pad ? min(L, n_pad - b0) : 0;
    const uint32_t d0 = o0 - a0;
    const uint32_t d1 = min(d0 + TILE, la + lb);
    if (tid < 64) {
        const uint32_t dd = tid < 32 ? d0 : d1;
        const uint32_t r = merge_path_warp(src + a0, la, src + b0, lb, dd, tid & 31);
        if ((tid & 31) == 0) s_split[tid >> 5] = r;
    }
    __syncthreads();
    const uint32_t i0 = s_split[0], i1 = s_split[1];
    const uint32_t j0 = d0 - i0, j1 = d1 - i1;
    const int na = (int)(i1 - i0), nb = (int)(j1 - j0);
    const int cnt = na + nb;  // <= TILE = T*E
    {
        // all E loads of a thread are issued before its first store
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            r[k] = 0;
            if (x < na) r[k] = src[a0 + i0 + x];
            else if (x < cnt) r[k] = src[b0 + j0 + (x - na)];
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            if (x < cnt) sm[pidx<uint64_t>(x)] = r[k];
        }
    }
    __syncthreads();
    const int d = tid * E;
    uint64_t v[E];
    if (d < cnt) {
        int i = merge_path_smem<uint64_t>(sm, 0, na, na, nb, d);
        merge_serial_smem<uint64_t, E, true>(sm, 0, na, na, nb, i, d - i, v);
    }
    __syncthreads();
    if (d < cnt) {
#pragma unroll
        for (int k = 0; k < E; ++k)
            if (d + k < cnt) sm[pidx<uint64_t>(d + k)] = v[k];
    }
    __syncthreads();
    for (int x = tid; x < cnt; x += T) dst[o0 + x] = sm[pidx<uint64_t>(x)];
}

// ============================================================ Step 5
// g_j = S[r_j], r_j = floor((j+1) * n_rec / b) - 1 (n_rec = m*s; with b = s
// this is the paper's S[(j+1)m - 1]).
__global__ void k_select_splitters(const uint64_t *__restrict__ sorted, uint32_t n_rec,
                                   uint32_t b, uint64_t *__restrict__ spl)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < b) spl[j] = sorted[(uint64_t)(j + 1) * n_rec / b - 1];
}

// ============================================================ Step 6
// c_ij = the number of items of sorted sublist i that are <= splitter g_j
// (items compare as key << 32 | position, position = i*t + rank), so that
// the run A_ij holds ranks [c_i,j-1, c_ij) of sublist i.  Every sublist is
// cut into segments of `seg` items; splitter j belongs to the segment
// [S, S + seg) that holds c_ij (the last segment also takes c_ij = t).
// k_seg_ranges finds, per segment, the first splitter that belongs to it:
// c_ij >= S exactly when g_j >= item S - 1, so it is the number of
// splitters below item S - 1 (binary search over the b sorted splitters).
// k_sample_index_grp then takes segment k of kSub6 consecutive sublists:
// it stages the segments in shared memory with coalesced loads (the
// sublists are read from HBM once, whole), and its threads take the
// (splitter, sublist) pairs splitter-major, so that the kSub6 counts of one
// splitter, stored bucket-major at cum[j*m + i], leave as one 32-byte
// sector; each count is a binary search in the staged segment.  It writes
// the cumulative c_ij, which Step 7 turns into the run sizes a_ij and
// starts.  (The paper locates g_j in sublist i through the sublist's
// samples and a w-item window; that reads one window per splitter with
// accesses no warp can coalesce.  The counts are the same.)
constexpr int kSegItems = 1024;  // items of one sublist's segment
constexpr int kSub6 = 8;         // sublists per CTA: 8 counts = one 32-byte sector
constexpr int kSegRow = kSegItems + 4;  // staged row: rows start in different banks

// Position p = i*t + (k+1)w - 1 of the sample whose record holds q = i*s + k.
__device__ __forceinline__ uint64_t sample_pos(uint32_t q, uint32_t s, uint32_t t, uint32_t w)
{
    return (uint64_t)(q / s) * t + (uint64_t)(q % s + 1) * w - 1;
}

__global__ void k_seg_ranges(const uint32_t *__restrict__ tiles_k, const uint64_t *__restrict__ spl,
                             uint32_t t, uint32_t s, uint32_t b, uint32_t m, uint32_t nseg,
                             uint32_t seg, uint32_t *__restrict__ jr)
{
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * nseg) return;
    const uint32_t i = idx / nseg, k = idx % nseg;
    const uint32_t w = t / s;
    uint32_t r = 0;
    if (k > 0) {
        const uint64_t x = (uint64_t)i * t + k * seg - 1;  // item S - 1 of sublist i
        const uint32_t key = tiles_k[x];
        uint32_t lo = 0, hi = b;
        while (lo < hi) {  // splitters below item x in (key, position) order
            const uint32_t mid = (lo + hi) >> 1;
            const uint64_t g = spl[mid];
            const uint32_t gk = (uint32_t)(g >> 32);
            const bool below = gk < key || (gk == key && sample_pos((uint32_t)g, s, t, w) < x);
            if (below) lo = mid + 1;
            else hi = mid;
        }
        r = lo;
    }
    jr[idx] = r;
}

template <int T, int SEG>  // SEG: the segment length at compile time (0: seg)
__global__ void __launch_bounds__(T, 5)
k_sample_index_grp(const uint32_t *__restrict__ tiles_k, const uint64_t *__restrict__ spl,
                   uint32_t t, uint32_t s, uint32_t b, uint32_t m, uint32_t nseg, uint32_t seg_rt,
                   const uint32_t *__restrict__ jr, uint32_t *__restrict__ cum)
{
    const uint32_t seg = SEG ? (uint32_t)SEG : seg_rt;
    __shared__ __align__(16) uint32_t sk[kSub6 * kSegRow];
    __shared__ uint32_t s_lo[kSub6], s_hi[kSub6];
    const uint32_t i0 = (blockIdx.x / nseg) * kSub6, k = blockIdx.x % nseg;
    const uint32_t ns = min((uint32_t)kSub6, m - i0);  // sublists of this group
    const uint32_t S = k * seg;
    const int tid = threadIdx.x;
    if (tid < kSub6) {
        const uint32_t ii = (uint32_t)tid;
        s_lo[ii] = ii < ns ? jr[(i0 + ii) * nseg + k] : 0u;
        s_hi[ii] = ii < ns ? (k + 1 < nseg ? jr[(i0 + ii) * nseg + k + 1] : b) : 0u;
    }
    // stage segment k of every sublist: seg/4 uint4 per sublist, all loads
    // of a thread issued before its first store
    const uint32_t q4 = seg / 4;
    constexpr int Q = kSub6 * kSegItems / 4 / T;
    uint4 r[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t v = (uint32_t)(q * T + tid);
        const uint32_t ii = v / q4, o = v % q4;
        if (ii < ns)
            r[q] = reinterpret_cast<const uint4 *>(tiles_k + (uint64_t)(i0 + ii) * t + S)[o];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t v = (uint32_t)(q * T + tid);
        const uint32_t ii = v / q4, o = v % q4;
        if (ii < ns) reinterpret_cast<uint4 *>(sk + ii * kSegRow)[o] = r[q];
    }
    __syncthreads();
    uint32_t J0 = 0xFFFFFFFFu, J1 = 0;
#pragma unroll
    for (int ii = 0; ii < kSub6; ++ii) {
        if ((uint32_t)ii < ns && s_lo[ii] < s_hi[ii]) {
            J0 = min(J0, s_lo[ii]);
            J1 = max(J1, s_hi[ii]);
        }
    }
    if (J0 >= J1) return;
    // Thread (c, ii) = (tid / 8, tid mod 8) takes sublist i0 + ii and the
    // c-th of T/8 consecutive chunks of the splitters [J0, J1), in order, so
    // that at every step the 8 threads of a chunk write the 8 counts of one
    // splitter (bucket-major cum[j*m + i]) as one 32-byte sector.
    // Splitter g = (gk, q) is the sample at rank gr = (q mod s + 1)w - 1 of
    // sublist gi = q / s; in (key, position) order sublist i holds
    // upper_bound(gk) items <= g if i < gi (all its positions are lower),
    // lower_bound(gk) if i > gi, and exactly gr + 1 if i == gi.  Both bounds
    // count the keys below a threshold (gk + 1, resp. gk; all keys when gk
    // is the largest key and i < gi).  For one sublist the thresholds do not
    // decrease with j (splitters ascend in (gk, q), and gi with q), so the
    // previous count bounds the next from below: the next search covers the
    // 16 keys from there when the count lies among them (branch-free, five
    // probes), else the whole power-of-two segment.
    const uint32_t ls = 31u - (uint32_t)__clz(s);  // s and t are powers of two
    const uint32_t w = t >> ls;
    constexpr uint32_t kChunks = (uint32_t)T / kSub6;
    const uint32_t ii = (uint32_t)tid % kSub6, c = (uint32_t)tid / kSub6;
    if (ii >= ns) return;  // (no barrier follows)
    const uint32_t per = (J1 - J0 + kChunks - 1) / kChunks;
    const uint32_t ja = max(J0 + c * per, s_lo[ii]);
    const uint32_t jb = min(min(J0 + (c + 1) * per, J1), s_hi[ii]);
    const uint32_t i = i0 + ii;
    const uint32_t *row = sk + ii * kSegRow;
    uint32_t lb = 0;  // keys of the segment below the previous threshold
    for (uint32_t j = ja; j < jb; ++j) {
        const uint64_t g = spl[j];
        const uint32_t gk = (uint32_t)(g >> 32), q = (uint32_t)g;
        const uint32_t gi = q >> ls;
        uint32_t res;
        if (i == gi) {
            res = ((q & (s - 1u)) + 1u) * w;  // gr + 1
        } else if (i < gi && gk == 0xFFFFFFFFu) {
            lb = seg;
            res = S + seg;  // every key is <= the largest key
        } else {
            const uint32_t thr = gk + (i < gi ? 1u : 0u);
            uint32_t bpos;
            if (lb + 16u <= seg && row[lb + 15u] >= thr) {
                bpos = lb;
#pragma unroll
                for (uint32_t hh = 8; hh > 0; hh >>= 1)
                    if (row[bpos + hh - 1] < thr) bpos += hh;
            } else {
                bpos = 0;
#pragma unroll
                for (uint32_t hh = seg >> 1; hh > 0; hh >>= 1)
                    if (row[bpos + hh - 1] < thr) bpos += hh;
                bpos += row[bpos] < thr ? 1u : 0u;
            }
            lb = bpos;
            res = S + bpos;
        }
        cum[(uint64_t)j * m + i] = res;
    }
}

// ============================================================ Step 7
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;  // ~0.5-1 s with the back-off below
constexpr int kTestSpinLimit = 4096;  // the stalled-scan test: well under a millisecond

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

template <int T, int ITEMS>
__global__ void __launch_bounds__(T)
k_scan(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint32_t n_items,
       unsigned long long *status, uint32_t *ticket, int *err, const uint32_t *__restrict__ cum,
       uint32_t m, uint32_t t, uint32_t *__restrict__ counts, uint32_t *__restrict__ srcb,
       int spin_limit, int stall_first)
{
    __shared__ uint32_t s_chunk;
    __shared__ uint32_t s_warp[T / 32];
    __shared__ uint32_t s_prefix;
    __shared__ uint32_t s_last;
    // the chunk's items, staged so that global loads and stores are
    // coalesced while each thread scans ITEMS consecutive items (padded:
    // one spare word per 32, so the per-thread runs hit distinct banks)
    __shared__ uint32_t s_items[T * ITEMS + T * ITEMS / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_chunk = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t chunk = s_chunk;
    const uint64_t cbase = (uint64_t)chunk * (T * ITEMS);
    auto spad = [](int x) { return x + (x >> 5); };
    if (cum == nullptr) {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const uint64_t e = cbase + (uint64_t)(k * T + tid);
            s_items[spad(k * T + tid)] = e < n_items ? in[e] : 0u;
        }
    } else {
        // item e = j*m + i from the cumulative counts of Step 6:
        // a_ij = c_ij - c_i,j-1 and A_ij starts at position i*t + c_i,j-1
        uint32_t i = (uint32_t)((cbase + (uint64_t)tid) % m);
        const uint32_t di = (uint32_t)T % m;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const uint64_t e = cbase + (uint64_t)(k * T + tid);
            uint32_t a = 0u;
            if (e < n_items) {
                const uint32_t c = cum[e];
                const uint32_t p = e >= m ? cum[e - m] : 0u;
                a = c - p;
                if (counts != nullptr) counts[e] = a;
                srcb[e] = i * t + p;
            }
            s_items[spad(k * T + tid)] = a;
            i += di;
            if (i >= m) i -= m;
        }
    }
    __syncthreads();
    uint32_t x[ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        x[k] = s_items[spad(tid * ITEMS + k)];
        sum += x[k];
    }
    // block-wide exclusive scan of the per-thread sums
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t wv = lane < T / 32 ? s_warp[lane] : 0u;
        uint32_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < T / 32) s_warp[lane] = wi - wv;  // exclusive warp offsets
        if (lane == T / 32 - 1) s_last = wv;
    }
    __syncthreads();
    if (warp == 0) {
        // decoupled look-back by the whole first warp (bounded waits): lane l
        // inspects chunk p - l; the nearest inclusive prefix ends the walk
        const uint32_t agg = s_warp[T / 32 - 1] + s_last;
        uint32_t prefix = 0;
        if (chunk == 0) {
            // (stall_first, a test of the bounded wait: chunk 0 never
            // publishes, so the look-back of every later chunk that reaches
            // it gives up after spin_limit polls and records DEV_TIMEOUT)
            if (lane == 0 && !stall_first) atomicExch(&status[0], kFlagInc | agg);
        } else {
            if (lane == 0) atomicExch(&status[chunk], kFlagAgg | agg);
            int p = (int)chunk - 1;
            int spins = 0;
            bool timed_out = false;
            while (p >= 0) {
                const int q = p - lane;
                unsigned long long st = q >= 0 ? ld_volatile(&status[q]) : (kFlagInc | 0ull);
                // wait until every inspected chunk has published something
                while (__any_sync(0xFFFFFFFFu, (st >> 62) == 0)) {
                    if (++spins > spin_limit) {
                        timed_out = true;
                        break;
                    }
                    __nanosleep(64);
                    if ((st >> 62) == 0) st = ld_volatile(&status[q]);
                }
                if (timed_out) break;
                const unsigned inc = __ballot_sync(0xFFFFFFFFu, (st >> 62) == 2);
                const int stop = inc ? __ffs(inc) - 1 : 31;  // nearest inclusive lane
                uint32_t val = (lane <= stop) ? (uint32_t)(st & kValMask) : 0u;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) val += __shfl_xor_sync(0xFFFFFFFFu, val, o);
                prefix += val;
                if (inc) break;
                p -= 32;
            }
            if (timed_out && lane == 0) set_error(err, DEV_TIMEOUT);
            if (lane == 0) {
                __threadfence();
                atomicExch(&status[chunk], kFlagInc | (unsigned long long)(prefix + agg));
            }
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t run = s_prefix + s_warp[warp] + (incl - sum);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        s_items[spad(tid * ITEMS + k)] = run;
        run += x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint64_t e = cbase + (uint64_t)(k * T + tid);
        if (e < n_items) out[e] = s_items[spad(k * T + tid)];
    }
}

// Step 7 by rows.  With the cumulative counts c_ij of Step 6 the
// bucket-major exclusive scan splits into independent rows: the items
// before run A_ij are all items of buckets 0 .. j-1, which number
// sum_i' c_i',j-1 (the start of bucket j), plus the runs A_i'j of the
// sublists i' < i, so
//   l_ij = sum_i' c_i',j-1 + sum_{i' < i} (c_i'j - c_i',j-1).
// One CTA per bucket j computes row j from rows j and j-1 of the cumulative
// counts, and no CTA waits for another.  A row of at most T*V sublists is
// one piece: the bucket start and the prefix of the run sizes come from one
// block-wide scan of the pair (sum of c_i,j-1, sum of a_ij) packed in 64
// bits (each half stays below n' < 2^32, so no carry crosses).  Longer rows
// take the bucket start from a first pass over row j-1 and are scanned in
// pieces with a running carry.  counts (a_ij) and srcb (i*t + c_i,j-1, the
// run's first sorted-sublist position) are written when not null.
template <int T, int V>
__global__ void __launch_bounds__(T)
k_row_scan(const uint32_t *__restrict__ cum, uint32_t m, uint32_t t, uint32_t *__restrict__ out,
           uint32_t *__restrict__ counts, uint32_t *__restrict__ srcb)
{
    constexpr int N = T * V;
    constexpr int W = T / 32;
    __shared__ uint32_t s_items[N + N / 32];
    __shared__ unsigned long long s_warp[W];
    __shared__ unsigned long long s_total;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t j = blockIdx.x;
    const uint64_t r0 = (uint64_t)j * m;
    const uint32_t *row = cum + r0;
    const uint32_t *prev = j ? row - m : nullptr;
    auto spad = [](int x) { return x + (x >> 5); };
    // inclusive block scan of one 64-bit value per thread; s_total = sum
    auto block_scan = [&](unsigned long long v) -> unsigned long long {
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long wv = lane < W ? s_warp[lane] : 0ull;
            unsigned long long wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < W) s_warp[lane] = wi - wv;
            if (lane == W - 1) s_total = wi;
        }
        __syncthreads();
        return s_warp[warp] + inc;
    };
    const bool pieces = m > (uint32_t)N;
    if (!pieces && (m & 3u) == 0) {
        // one piece, rows of whole 16-byte words: thread tid takes items
        // [tid*V, tid*V + V) straight from global memory as 16-byte words
        // (all loads in flight before the first use), no staging
        static_assert(V % 4 == 0, "V must be a multiple of 4");
        const uint32_t i0 = (uint32_t)tid * V;
        uint4 c4[V / 4], p4[V / 4];
#pragma unroll
        for (int k = 0; k < V / 4; ++k) {
            const uint32_t i = i0 + 4u * k;
            c4[k] = make_uint4(0u, 0u, 0u, 0u);
            p4[k] = make_uint4(0u, 0u, 0u, 0u);
            if (i < m) {
                c4[k] = *reinterpret_cast<const uint4 *>(row + i);
                if (prev != nullptr) p4[k] = *reinterpret_cast<const uint4 *>(prev + i);
            }
        }
        uint32_t x[V];
        uint32_t sum = 0, ps = 0;
#pragma unroll
        for (int k = 0; k < V / 4; ++k) {
            x[4 * k + 0] = c4[k].x - p4[k].x;
            x[4 * k + 1] = c4[k].y - p4[k].y;
            x[4 * k + 2] = c4[k].z - p4[k].z;
            x[4 * k + 3] = c4[k].w - p4[k].w;
            ps += p4[k].x + p4[k].y + p4[k].z + p4[k].w;
        }
#pragma unroll
        for (int k = 0; k < V; ++k) sum += x[k];
        const unsigned long long v = ((unsigned long long)ps << 32) | (unsigned long long)sum;
        const unsigned long long excl = block_scan(v) - v;
        uint32_t run = (uint32_t)(s_total >> 32) + (uint32_t)excl;
#pragma unroll
        for (int k = 0; k < V / 4; ++k) {
            const uint32_t i = i0 + 4u * k;
            if (i >= m) break;
            uint4 o;
            o.x = run;
            o.y = o.x + x[4 * k + 0];
            o.z = o.y + x[4 * k + 1];
            o.w = o.z + x[4 * k + 2];
            run = o.w + x[4 * k + 3];
            *reinterpret_cast<uint4 *>(out + r0 + i) = o;
            if (counts != nullptr)
                *reinterpret_cast<uint4 *>(counts + r0 + i) =
                    make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
            if (srcb != nullptr)
                *reinterpret_cast<uint4 *>(srcb + r0 + i) =
                    make_uint4(i * t + p4[k].x, (i + 1) * t + p4[k].y, (i + 2) * t + p4[k].z,
                               (i + 3) * t + p4[k].w);
        }
        return;
    }
    uint32_t start = 0;
    if (pieces && prev != nullptr) {
        uint32_t ps = 0;
        for (uint32_t i = (uint32_t)tid; i < m; i += T) ps += prev[i];
        block_scan(ps);
        start = (uint32_t)s_total;
        __syncthreads();  // s_warp and s_total are reused below
    }
    uint32_t carry = 0;
    for (uint32_t base = 0; base < m; base += N) {
        uint32_t ps = 0;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int idx = k * T + tid;
            const uint32_t i = base + (uint32_t)idx;
            uint32_t a = 0;
            if (i < m) {
                const uint32_t p = prev != nullptr ? prev[i] : 0u;
                a = row[i] - p;
                ps += p;
                if (counts != nullptr) counts[r0 + i] = a;
                if (srcb != nullptr) srcb[r0 + i] = i * t + p;
            }
            s_items[spad(idx)] = a;
        }
        __syncthreads();
        uint32_t x[V];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            x[k] = s_items[spad(tid * V + k)];
            sum += x[k];
        }
        const unsigned long long v =
            ((unsigned long long)(pieces ? 0u : ps) << 32) | (unsigned long long)sum;
        const unsigned long long excl = block_scan(v) - v;
        const unsigned long long tot = s_total;
        if (!pieces) start = (uint32_t)(tot >> 32);
        uint32_t run = start + carry + (uint32_t)excl;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            s_items[spad(tid * V + k)] = run;
            run += x[k];
        }
        carry += (uint32_t)tot;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int idx = k * T + tid;
            const uint32_t i = base + (uint32_t)idx;
            if (i < m) out[r0 + i] = s_items[spad(idx)];
        }
        __syncthreads();  // s_items, s_warp and s_total are reused by the next piece
    }
}

// ============================================================ Step 8
// Relocation by destination: CTA c fills positions [c*kRelocPart,
// (c+1)*kRelocPart) of the relocated array, so every CTA moves the same
// number of items whatever the key distribution.  Position y lies in the
// run q (offsets[q] <= y < offsets[q+1]) and comes from position srcb[q] +
// (y - offsets[q]) of the sorted sublists (with srcb null, the run start
// i*t + c_i,j-1 of run q = j*m + i is taken from the cumulative counts).  Each warp covers kBlockItems
// consecutive positions, its lanes on consecutive positions (coalesced
// stores).  The runs meeting a warp's block are blk[b] .. blk[b+1] (the run
// index); when they are few (the usual case) the warp stages them in shared
// memory as a list of the non-empty runs in order, each as the difference
// srcb - offsets (so that position y of the run comes from that + y), and
// a bitmap of the block with a bit at every run start after the first:
// the run of position y is then the number of bits set up to y (one
// population count and a prefix over the bitmap's words, held one word per
// lane), with no per-position walk; a lane resolves sixteen positions and
// then issues their loads together.  Otherwise each lane walks the runs in
// global memory (skipping stretches of empty runs by a search bounded by
// the run index).
constexpr int kRelocRunsCap = 512;  // runs a warp stages in shared memory

// Sorted-sublist position of the first item of run q = j*m + i: srcb[q],
// or i*t + c_i,j-1 from the cumulative counts when srcb is null.
__device__ __forceinline__ uint32_t run_first(const uint32_t *__restrict__ srcb,
                                              const uint32_t *__restrict__ cum, uint32_t m,
                                              uint32_t t, uint32_t q)
{
    if (srcb != nullptr) return srcb[q];
    return (q % m) * t + (q >= m ? cum[q - m] : 0u);
}

template <int T, typename KT>
__global__ void __launch_bounds__(T, 4)
k_relocate(const KT *__restrict__ tiles_k, const void *__restrict__ tiles_v,
           const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ srcb,
           const uint32_t *__restrict__ cum, uint32_t m, uint32_t t,
           const uint32_t *__restrict__ blk, uint32_t runs,
           uint32_t n_pad, int val_bytes, KT *__restrict__ reloc_k,
           void *__restrict__ reloc_v)
{
    constexpr int W = T / 32;
    constexpr int P = kBlockItems / 32;  // positions per lane
    __shared__ uint32_t s_off[W][kRelocRunsCap + 1];
    __shared__ uint32_t s_src[W][kRelocRunsCap];  // then: srcb - offsets of the non-empty runs
    __shared__ uint32_t s_bm[W][32];              // run starts in the warp's block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wy = blockIdx.x * (uint32_t)kRelocPart + (uint32_t)warp * kBlockItems;
    if (wy >= n_pad) return;  // whole warp
    const uint32_t b = wy / kBlockItems;
    const uint32_t nblk = (n_pad + kBlockItems - 1) / kBlockItems;
    const uint32_t q0 = blk[b];
    const uint32_t q1 = b + 1 < nblk ? blk[b + 1] : runs - 1;
    const uint32_t yend = min(wy + (uint32_t)kBlockItems, n_pad);
    if (q1 - q0 < (uint32_t)kRelocRunsCap) {
        const uint32_t R = q1 - q0 + 1;  // runs q0 .. q1; offsets[q1 + 1] exists
        uint32_t *so = s_off[warp];
        uint32_t *sd = s_src[warp];
        for (uint32_t i = lane; i <= R; i += 32) so[i] = offsets[q0 + i];
        if (srcb != nullptr) {
            for (uint32_t i = lane; i < R; i += 32) sd[i] = srcb[q0 + i];
        } else {
            // run q = j*m + i starts at i*t + c_i,j-1 of the sorted sublists
            const uint32_t step = 32u % m;
            uint32_t si = (q0 + lane) % m;
            for (uint32_t i = lane; i < R; i += 32) {
                const uint32_t q = q0 + i;
                sd[i] = si * t + (q >= m ? cum[q - m] : 0u);
                si += step;
                if (si >= m) si -= m;
            }
        }
        __syncwarp();
        // run q0 holds wy; a later run counts if it is non-empty and starts
        // inside the block.  Compact them in order (in place: entry k of
        // the list is written at or below the entry it comes from) and set
        // the bitmap bit of each start.
        uint32_t *bm = s_bm[warp];
        bm[lane] = 0u;
        __syncwarp();
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t nk = 0;
        for (uint32_t r0 = 0; r0 < R; r0 += 32) {
            const uint32_t r = r0 + lane;
            uint32_t st = 0, d = 0;
            bool keep = false;
            if (r < R) {
                st = so[r];
                d = sd[r] - st;
                keep = r == 0 || (so[r + 1] > st && st < yend);
            }
            const unsigned kb = __ballot_sync(0xFFFFFFFFu, keep);
            __syncwarp();  // every entry of this round is read before any is rewritten
            if (keep) {
                sd[nk + (uint32_t)__popc(kb & lt)] = d;
                if (r > 0) atomicOr(&bm[(st - wy) >> 5], 1u << ((st - wy) & 31u));
            }
            nk += (uint32_t)__popc(kb);
            __syncwarp();  // this round's writes land before the next round's reads
        }
        const uint32_t word = bm[lane];  // lane w holds bitmap word w
        // runs before word w: exclusive prefix of the words' bit counts
        const uint32_t cnt = (uint32_t)__popc(word);
        uint32_t pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, pre, o);
            if (lane >= o) pre += y;
        }
        pre -= cnt;
        const uint32_t upto = lane == 31 ? 0xFFFFFFFFu : (2u << lane) - 1u;  // bits 0 .. lane
        constexpr int G = 16;  // positions resolved, then loaded, at a time
#pragma unroll 1
        for (int k0 = 0; k0 < P; k0 += G) {
            uint32_t src[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                // position y = wy + 32 (k0 + k) + lane is bit `lane` of word k0 + k
                const uint32_t wk = __shfl_sync(0xFFFFFFFFu, word, k0 + k);
                const uint32_t pk = __shfl_sync(0xFFFFFFFFu, pre, k0 + k);
                const uint32_t idx = pk + (uint32_t)__popc(wk & upto);
                const uint32_t y = wy + (uint32_t)lane + 32u * (uint32_t)(k0 + k);
                src[k] = sd[idx] + y;
            }
            KT v[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint32_t y = wy + (uint32_t)lane + 32u * (uint32_t)(k0 + k);
                v[k] = y < yend ? tiles_k[src[k]] : (KT)0;
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint32_t y = wy + (uint32_t)lane + 32u * (uint32_t)(k0 + k);
                if (y < yend) reloc_k[y] = v[k];
            }
            if (val_bytes == 4) {
                const uint32_t *tv = static_cast<const uint32_t *>(tiles_v);
                uint32_t *rv = static_cast<uint32_t *>(reloc_v);
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const uint32_t y = wy + (uint32_t)lane + 32u * (uint32_t)(k0 + k);
                    if (y < yend) rv[y] = tv[src[k]];
                }
            } else if (val_bytes == 8) {
                const uint64_t *tv = static_cast<const uint64_t *>(tiles_v);
                uint64_t *rv = static_cast<uint64_t *>(reloc_v);
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const uint32_t y = wy + (uint32_t)lane + 32u * (uint32_t)(k0 + k);
                    if (y < yend) rv[y] = tv[src[k]];
                }
            }
        }
        return;
    }
    uint32_t y = wy + lane;
    uint32_t lo = q0, hi = q1;
    while (lo < hi) {  // last run q with offsets[q] <= y
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= y) lo = mid;
        else hi = mid - 1;
    }
    uint32_t q = lo;
    uint32_t rs = offsets[q], re = offsets[q + 1];
    uint32_t base = run_first(srcb, cum, m, t, q);
    for (; y < yend; y += 32) {
        if (y >= re) {
            run_advance<kBlockItems>(offsets, blk, nblk, runs, y, q, rs, re);
            base = run_first(srcb, cum, m, t, q);
        }
        const uint32_t src = base + (y - rs);
        reloc_k[y] = tiles_k[src];
        if (val_bytes == 4)
            static_cast<uint32_t *>(reloc_v)[y] = static_cast<const uint32_t *>(tiles_v)[src];
        else if (val_bytes == 8)
            static_cast<uint64_t *>(reloc_v)[y] = static_cast<const uint64_t *>(tiles_v)[src];
    }
}

// Steps 7-8 fused, one CTA per bucket j (rows of at most T*V sublists, m a
// multiple of 4).  The CTA scans row j of the cumulative counts as
// k_row_scan does (bucket start B_j = sum_i c_i,j-1, run offsets l_ij,
// written to `offsets` for Step 9 and for inspection), lists the non-empty
// runs of the bucket in shared memory (local start, and sorted-sublist start
// minus local start), and then moves the bucket itself: its warps take
// blocks of kBlockItems consecutive positions y of the bucket, find the run
// holding the block's first position by a 32-way search of the list, mark
// the later run starts of the block in a bitmap and resolve each position's
// run by a population count, as k_relocate does, with coalesced stores to
// B_j + y.  Nothing is read back from global memory but the keys (and
// values) themselves: no run offsets, run starts or run index.
constexpr int kFuseT = 512, kFuseV = 16;
constexpr uint32_t kFuseMaxM = (uint32_t)(kFuseT * kFuseV);

template <int T, int V>
__global__ void __launch_bounds__(T, 2)
k_bucket_relocate(const uint32_t *__restrict__ cum, uint32_t m, uint32_t t, uint32_t b,
                  uint32_t n_pad, const uint32_t *__restrict__ tiles_k,
                  const void *__restrict__ tiles_v, int val_bytes, uint32_t *__restrict__ offsets,
                  uint32_t *__restrict__ reloc_k, void *__restrict__ reloc_v)
{
    constexpr int W = T / 32;
    constexpr int P = kBlockItems / 32;  // positions per lane in a block
    static_assert(V % 4 == 0, "V must be a multiple of 4");
    extern __shared__ uint32_t s_dyn[];
    uint32_t *s_loc = s_dyn;              // [T*V + 1] local start of non-empty run k
    uint32_t *s_d = s_dyn + T * V + 1;    // [T*V] its sorted-sublist start - local start
    __shared__ unsigned long long s_warp[W];
    __shared__ unsigned long long s_total;
    __shared__ uint32_t s_bm[W][32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t j = blockIdx.x;
    const uint64_t r0 = (uint64_t)j * m;
    const uint32_t *row = cum + r0;
    const uint32_t *prev = j ? row - m : nullptr;
    auto block_scan = [&](unsigned long long v) -> unsigned long long {
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long wv = lane < W ? s_warp[lane] : 0ull;
            unsigned long long wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < W) s_warp[lane] = wi - wv;
            if (lane == W - 1) s_total = wi;
        }
        __syncthreads();
        const unsigned long long r = s_warp[warp] + inc;
        __syncthreads();  // s_warp is free again (s_total is read before the next scan ends)
        return r;
    };
    // ---- Step 7 for row j: thread tid holds sublists [tid*V, tid*V + V)
    const uint32_t i0 = (uint32_t)tid * V;
    uint4 c4[V / 4], p4[V / 4];
#pragma unroll
    for (int k = 0; k < V / 4; ++k) {
        const uint32_t i = i0 + 4u * k;
        c4[k] = make_uint4(0u, 0u, 0u, 0u);
        p4[k] = make_uint4(0u, 0u, 0u, 0u);
        if (i < m) {
            c4[k] = *reinterpret_cast<const uint4 *>(row + i);
            if (prev != nullptr) p4[k] = *reinterpret_cast<const uint4 *>(prev + i);
        }
    }
    uint32_t x[V], pv[V];
    uint32_t sum = 0, ps = 0, nz = 0;
#pragma unroll
    for (int k = 0; k < V / 4; ++k) {
        pv[4 * k + 0] = p4[k].x;
        pv[4 * k + 1] = p4[k].y;
        pv[4 * k + 2] = p4[k].z;
        pv[4 * k + 3] = p4[k].w;
        x[4 * k + 0] = c4[k].x - p4[k].x;
        x[4 * k + 1] = c4[k].y - p4[k].y;
        x[4 * k + 2] = c4[k].z - p4[k].z;
        x[4 * k + 3] = c4[k].w - p4[k].w;
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        sum += x[k];
        ps += pv[k];
        nz += x[k] != 0u ? 1u : 0u;
    }
    const unsigned long long v = ((unsigned long long)ps << 32) | (unsigned long long)sum;
    const unsigned long long excl = block_scan(v) - v;
    const unsigned long long tot = s_total;
    const uint32_t Bj = (uint32_t)(tot >> 32);  // bucket start
    const uint32_t Sj = (uint32_t)tot;          // bucket size
    const uint32_t kz = (uint32_t)(block_scan(nz) - nz);
    const uint32_t K = (uint32_t)s_total;       // non-empty runs
    uint32_t run = (uint32_t)excl, k = kz;
#pragma unroll
    for (int q = 0; q < V / 4; ++q) {
        const uint32_t i = i0 + 4u * q;
        if (i < m) {
            uint4 o;
            o.x = Bj + run;
            o.y = o.x + x[4 * q + 0];
            o.z = o.y + x[4 * q + 1];
            o.w = o.z + x[4 * q + 2];
            *reinterpret_cast<uint4 *>(offsets + r0 + i) = o;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (x[4 * q + e] != 0u) {
                s_loc[k] = run;
                s_d[k] = (i + e) * t + pv[4 * q + e] - run;
                ++k;
            }
            run += x[4 * q + e];
        }
    }
    if (tid == 0) {
        s_loc[K] = Sj;
        if (j == b - 1) offsets[(uint64_t)b * m] = n_pad;
    }
    __syncthreads();
    // ---- Step 8 for bucket j
    const uint32_t nblk = (Sj + kBlockItems - 1) / kBlockItems;
    uint32_t *bm = s_bm[warp];
    for (uint32_t bi = (uint32_t)warp; bi < nblk; bi += W) {
        const uint32_t y0 = bi * (uint32_t)kBlockItems;
        const uint32_t yend = min(y0 + (uint32_t)kBlockItems, Sj);
        // last run k0 with s_loc[k0] <= y0 (s_loc[0] = 0)
        uint32_t lo = 0, hi = K;
        while (hi - lo > 1) {
            const uint32_t step = (hi - lo + 31) >> 5;
            const uint32_t idx = lo + (uint32_t)lane * step;
            const bool le = idx < hi && s_loc[idx] <= y0;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, le);  // lane 0 always
            lo += (uint32_t)(31 - __clz((int)bal)) * step;
            hi = min(hi, lo + step);
        }
        const uint32_t k0 = lo;
        bm[lane] = 0u;
        __syncwarp();
        // runs after k0 that start inside the block (starts increase with k)
        for (uint32_t kb = k0 + 1;; kb += 32) {
            const uint32_t kk = kb + (uint32_t)lane;
            const uint32_t st = kk < K ? s_loc[kk] : 0xFFFFFFFFu;
            const bool in = st < yend;
            if (in) atomicOr(&bm[(st - y0) >> 5], 1u << ((st - y0) & 31u));
            if (__ballot_sync(0xFFFFFFFFu, in) != 0xFFFFFFFFu) break;
        }
        __syncwarp();
        const uint32_t word = bm[lane];
        const uint32_t cnt = (uint32_t)__popc(word);
        uint32_t pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yv = __shfl_up_sync(0xFFFFFFFFu, pre, o);
            if (lane >= o) pre += yv;
        }
        pre = pre - cnt + k0;
        const uint32_t upto = lane == 31 ? 0xFFFFFFFFu : (2u << lane) - 1u;
        constexpr int G = 16;
#pragma unroll 1
        for (int k1 = 0; k1 < P; k1 += G) {
            uint32_t src[G];
#pragma unroll
            for (int e = 0; e < G; ++e) {
                const uint32_t wk = __shfl_sync(0xFFFFFFFFu, word, k1 + e);
                const uint32_t pk = __shfl_sync(0xFFFFFFFFu, pre, k1 + e);
                const uint32_t y = y0 + (uint32_t)lane + 32u * (uint32_t)(k1 + e);
                src[e] = s_d[pk + (uint32_t)__popc(wk & upto)] + y;
            }
            uint32_t kv[G];
#pragma unroll
            for (int e = 0; e < G; ++e) {
                const uint32_t y = y0 + (uint32_t)lane + 32u * (uint32_t)(k1 + e);
                kv[e] = y < yend ? tiles_k[src[e]] : 0u;
            }
#pragma unroll
            for (int e = 0; e < G; ++e) {
                const uint32_t y = y0 + (uint32_t)lane + 32u * (uint32_t)(k1 + e);
                if (y < yend) reloc_k[Bj + y] = kv[e];
            }
            if (val_bytes == 4) {
                const uint32_t *tv = static_cast<const uint32_t *>(tiles_v);
                uint32_t *rv = static_cast<uint32_t *>(reloc_v);
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    const uint32_t y = y0 + (uint32_t)lane + 32u * (uint32_t)(k1 + e);
                    if (y < yend) rv[Bj + y] = tv[src[e]];
                }
            } else if (val_bytes == 8) {
                const uint64_t *tv = static_cast<const uint64_t *>(tiles_v);
                uint64_t *rv = static_cast<uint64_t *>(reloc_v);
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    const uint32_t y = y0 + (uint32_t)lane + 32u * (uint32_t)(k1 + e);
                    if (y < yend) rv[Bj + y] = tv[src[e]];
                }
            }
        }
        __syncwarp();  // the bitmap is rewritten by the warp's next block
    }
}

// Block-wide exclusive scan of one value per thread (T threads); *total
// receives the sum.  Uses s_warp[T / 32].
template <int T>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp,
                                                         uint32_t *s_total)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();  // s_warp may still be read by a previous scan
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t wv = lane < T / 32 ? s_warp[lane] : 0u;
        uint32_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < T / 32) s_warp[lane] = wi - wv;
        if (lane == T / 32 - 1) *s_total = wi;
    }
    __syncthreads();
    return s_warp[warp] + incl - v;
}

// Step 9 units of a two-tier plan: every bucket is a unit of its own (the
// bucket count puts the average bucket four sigmas below one CTA's unit, so
// no two buckets would fit one), listed in bucket order in `units` when it
// has at most Q1 items and in `units2` otherwise; a bucket above Q2 (the
// bound allows none) sets the error word.  One CTA; the b + 1 bucket starts
// are staged in shared memory (4 (b + 1) bytes), so b is not held to the
// greedy packing's limit.
template <int T>
__global__ void __launch_bounds__(T)
k_units_each(const uint32_t *__restrict__ offsets, uint32_t m, uint32_t b, uint32_t n_pad,
             uint32_t Q1, uint32_t Q2, uint32_t *__restrict__ units,
             uint32_t *__restrict__ units2, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem_raw);  // b + 1
    __shared__ uint32_t s_warp[T / 32];
    __shared__ uint32_t s_total[2];
    const int tid = threadIdx.x;
    for (uint32_t j0 = tid; j0 <= b; j0 += 4 * T) {  // four strided loads in flight
        uint32_t l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + (uint32_t)u * T;
            l[u] = j < b ? offsets[(uint64_t)j * m] : n_pad;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + (uint32_t)u * T;
            if (j <= b) Lb[j] = l[u];
        }
    }
    __syncthreads();
    uint32_t n1 = 0, n2 = 0;
    for (uint32_t j0 = 0; j0 < b; j0 += T) {
        const uint32_t j = j0 + (uint32_t)tid;
        uint32_t L = 0, R = 0;
        bool small = false, large = false;
        if (j < b) {
            L = Lb[j];
            R = Lb[j + 1];
            if (R - L > Q2) set_error(err, DEV_INTERNAL);  // a bucket exceeds the bound
            small = R - L <= Q1;
            large = !small;
        }
        const uint32_t u1 = block_exclusive_scan<T>(small ? 1u : 0u, s_warp, &s_total[0]);
        const uint32_t u2 = block_exclusive_scan<T>(large ? 1u : 0u, s_warp, &s_total[1]);
        if (small) {
            units[1 + 2 * (n1 + u1)] = L;
            units[2 + 2 * (n1 + u1)] = R;
        }
        if (large) {
            units2[1 + 2 * (n2 + u2)] = L;
            units2[2 + 2 * (n2 + u2)] = R;
        }
        n1 += s_total[0];
        n2 += s_total[1];
    }
    if (tid == 0) {
        units[0] = n1;
        units2[0] = n2;
    }
}

// Step 9 units: consecutive buckets packed greedily into units of at most
// Q1 items; a bucket larger than Q1 (at most the bound, Q2) forms a unit of
// its own.  One CTA: nxt[j] = the bucket after the longest run of buckets
// from j that fits Q1 (at least bucket j itself), the chain 0, nxt[0],
// nxt[nxt[0]], ... marks the unit starts (found by pointer doubling), and
// two scans number the units of at most Q1 items (written to units) and
// the larger ones (written to units2; with units2 == nullptr, Q1 = Q2 and
// every unit goes to units).  Each list: count, then (begin, end) pairs.
template <int T>
__global__ void __launch_bounds__(T, 1)
k_pack_units(const uint32_t *__restrict__ offsets, uint32_t m, uint32_t b, uint32_t n_pad,
             uint32_t Q1, uint32_t Q2, uint32_t *__restrict__ units,
             uint32_t *__restrict__ units2, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem_raw);  // b + 1
    uint32_t *nxt = Lb + (b + 1);                             // b + 1
    uint32_t *jmp = nxt + (b + 1);                            // b + 1
    uint32_t *on = jmp + (b + 1);                             // b + 1
    __shared__ uint32_t s_warp[T / 32];
    __shared__ uint32_t s_total[2];
    const int tid = threadIdx.x;
    // bucket starts (one strided load each): four loads in flight per thread
    for (uint32_t j0 = tid; j0 <= b; j0 += 4 * T) {
        uint32_t l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + (uint32_t)u * T;
            l[u] = j < b ? offsets[(uint64_t)j * m] : n_pad;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + (uint32_t)u * T;
            if (j <= b) {
                Lb[j] = l[u];
                on[j] = j == 0 ? 1u : 0u;
            }
        }
    }
    __syncthreads();
    // largest e in [j+1, b] with Lb[e] - Lb[j] <= Q1, else j + 1
    auto successor = [&](uint32_t j) {
        uint32_t lo = j + 1, hi = b;
        const uint32_t lim = Lb[j] + Q1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (Lb[mid] <= lim) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    for (uint32_t j = tid; j <= b; j += T) {
        uint32_t e = j;
        if (j < b) {
            e = successor(j);
            if (Lb[e] - Lb[j] > Q2) set_error(err, DEV_INTERNAL);  // a bucket exceeds the bound
        }
        nxt[j] = e;
        jmp[j] = e;
    }
    __syncthreads();
    for (uint32_t span = 1; span <= b; span <<= 1) {
        for (uint32_t j = tid; j <= b; j += T)
            if (on[j]) on[jmp[j]] = 1u;
        __syncthreads();
        for (uint32_t j = tid; j <= b; j += T) {
            const uint32_t a = jmp[j];
            nxt[j] = jmp[a];  // use nxt as scratch for the doubled jump
        }
        __syncthreads();
        for (uint32_t j = tid; j <= b; j += T) jmp[j] = nxt[j];
        __syncthreads();
    }
    // recompute the single-step successor (nxt was used as scratch)
    for (uint32_t j = tid; j <= b; j += T) nxt[j] = j < b ? successor(j) : j;
    __syncthreads();
    // number the unit starts (chain members j < b) in order, per list
    const uint32_t per = (b + T - 1) / T;
    const uint32_t j0 = tid * per;
    uint32_t c_small = 0, c_large = 0;
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t j = j0 + q;
        if (j < b && on[j]) {
            if (units2 == nullptr || Lb[nxt[j]] - Lb[j] <= Q1) ++c_small;
            else ++c_large;
        }
    }
    uint32_t u1 = block_exclusive_scan<T>(c_small, s_warp, &s_total[0]);
    uint32_t u2 = block_exclusive_scan<T>(c_large, s_warp, &s_total[1]);
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t j = j0 + q;
        if (j < b && on[j]) {
            if (units2 == nullptr || Lb[nxt[j]] - Lb[j] <= Q1) {
                units[1 + 2 * u1] = Lb[j];
                units[2 + 2 * u1] = Lb[nxt[j]];
                ++u1;
            } else {
                units2[1 + 2 * u2] = Lb[j];
                units2[2 + 2 * u2] = Lb[nxt[j]];
                ++u2;
            }
        }
    }
    if (tid == 0) {
        units[0] = s_total[0];
        if (units2 != nullptr) units2[0] = s_total[1];
    }
}

// Run index of every block of kBlockItems positions of the (virtual)
// relocated array: blk[b] = the bucket-major run q = j*m + i containing
// position b*kBlockItems (last q with l_q <= position; runs are in position
// order, empty runs share their start with the next one).  Also writes the
// sentinel l_{m*s} = n'.
__global__ void k_block_index(uint32_t *__restrict__ offsets, uint32_t runs, uint32_t n_pad,
                              uint32_t *__restrict__ blk, uint32_t nblk)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) offsets[runs] = n_pad;
    if (b >= nblk) return;
    const uint32_t y = b * (uint32_t)kBlockItems;
    uint32_t lo = 0, hi = runs - 1;  // last q in [0, runs) with offsets[q] <= y
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= y) lo = mid;
        else hi = mid - 1;
    }
    blk[b] = lo;
}

// ============================================================ Steps 7-8, n' >= 2^32
// Plans whose padded size reaches 2^32 (two levels: a few buckets of about
// 2^28 keys at the top, each then sorted by a plan of its own) keep counts
// and sublist ranks in 32 bits but need 64-bit bucket offsets.  Step 7 runs
// in three passes over the m*b cumulative counts (item e = j*m + i): the
// sum of a_ij over each chunk of kScanChunk items (each a_ij <= t, so a
// chunk's sum, at most kScanChunk * t, fits 32 bits), one CTA's 64-bit scan
// of the chunk sums, and each chunk's rescan into off64.
template <int T, int ITEMS>
__global__ void __launch_bounds__(T)
k_cum_chunk_sums(const uint32_t *__restrict__ cum, uint32_t m, uint32_t n_items,
                 uint32_t *__restrict__ sums)
{
    __shared__ uint32_t s_warp[T / 32];
    const uint64_t e0 = (uint64_t)blockIdx.x * (T * ITEMS);
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint64_t e = e0 + (uint64_t)(k * T + threadIdx.x);
        if (e < n_items) acc += cum[e] - (e >= m ? cum[e - m] : 0u);
    }
    acc = __reduce_add_sync(0xFFFFFFFFu, acc);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < T / 32; ++w) t += s_warp[w];
        sums[blockIdx.x] = t;
    }
}

// pre[c] = sum of sums[0 .. c) in 64 bits, by one CTA.
template <int T>
__global__ void __launch_bounds__(T)
k_chunk_prefix64(const uint32_t *__restrict__ sums, uint32_t chunks, uint64_t *__restrict__ pre)
{
    __shared__ unsigned long long s_warp[T / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < chunks; c0 += T) {
        const uint32_t c = c0 + (uint32_t)tid;
        const unsigned long long v = c < chunks ? sums[c] : 0ull;
        unsigned long long inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        unsigned long long wpre = 0, tot = 0;
        for (int w = 0; w < T / 32; ++w) {
            wpre += w < warp ? s_warp[w] : 0ull;
            tot += s_warp[w];
        }
        const unsigned long long base = s_base;
        if (c < chunks) pre[c] = base + wpre + inc - v;
        __syncthreads();
        if (tid == 0) s_base = base + tot;
        __syncthreads();
    }
}

// off64[e] = exclusive prefix of a_ij in bucket-major order; off64[n_items] = n_pad.
template <int T, int ITEMS>
__global__ void __launch_bounds__(T)
k_offsets64(const uint32_t *__restrict__ cum, uint32_t m, uint32_t n_items,
            const uint64_t *__restrict__ pre, uint64_t n_pad, uint64_t *__restrict__ off64)
{
    __shared__ uint32_t s_items[T * ITEMS];
    __shared__ uint32_t s_warp[T / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t e0 = (uint64_t)blockIdx.x * (T * ITEMS);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {  // coalesced loads, staged
        const uint64_t e = e0 + (uint64_t)(k * T + tid);
        s_items[k * T + tid] = e < n_items ? cum[e] - (e >= m ? cum[e - m] : 0u) : 0u;
    }
    __syncthreads();
    uint32_t x[ITEMS], sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {  // thread-blocked: items tid*ITEMS .. + ITEMS
        x[k] = s_items[tid * ITEMS + k];
        sum += x[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_warp[w];
    uint64_t run = pre[blockIdx.x] + wpre + inc - sum;
    const uint64_t eb = e0 + (uint64_t)tid * ITEMS;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (eb + k < n_items) off64[eb + k] = run;
        run += x[k];
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) off64[n_items] = n_pad;
}

// Step 8 by source: CTA i copies the runs A_i1 .. A_ib of sorted sublist i
// (ranks [c_i,j-1, c_ij)) to their offsets (runs of a two-level plan are
// long: t/b items on average, so the copies are coalesced).
template <int T>
__global__ void __launch_bounds__(T)
k_relocate_src64(const uint32_t *__restrict__ tiles_k, const uint32_t *__restrict__ cum,
                 const uint64_t *__restrict__ off64, uint32_t m, uint32_t b, uint32_t t,
                 uint32_t *__restrict__ reloc)
{
    const uint32_t i = blockIdx.x;
    const uint32_t *src = tiles_k + (uint64_t)i * t;
    uint32_t lo = 0;
    for (uint32_t j = 0; j < b; ++j) {
        const uint64_t e = (uint64_t)j * m + i;
        const uint32_t hi = cum[e];
        uint32_t *dst = reloc + off64[e] - lo;
        for (uint32_t r = lo + threadIdx.x; r < hi; r += T) dst[r] = src[r];
        lo = hi;
    }
}

// starts[j] = off64[j*m] (bucket j's first position), starts[b] = n_pad.
__global__ void k_bucket_starts64(const uint64_t *__restrict__ off64, uint32_t m, uint32_t b,
                                  uint64_t n_pad, uint64_t *__restrict__ starts)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < b) starts[j] = off64[(uint64_t)j * m];
    if (j == b) starts[b] = n_pad;
}

__global__ void k_f32_decode(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                             uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x)
        dst[x] = f32_decode(src[x]);
}

// First error of a nested sort (its own error word) into the caller's.
__global__ void k_merge_error(const int *__restrict__ from, int *to)
{
    if (threadIdx.x == 0 && *from != 0) atomicCAS(to, 0, *from);
}

// ============================================================ pairs with 64-bit keys
// Key-value pairs with 64-bit keys are sorted as two stable passes of the
// 32-bit pair sort (least significant half first, carrying positions):
// these kernels split the keys, make the index values, gather the high
// halves in the first pass's order, and apply both permutations.
__global__ void k_u64_split(const uint64_t *__restrict__ k64, uint32_t *__restrict__ lo,
                            uint32_t *__restrict__ iota, uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        lo[x] = (uint32_t)k64[x];
        iota[x] = (uint32_t)x;
    }
}

__global__ void k_u64_gather_hi(const uint64_t *__restrict__ k64, const uint32_t *__restrict__ p1,
                                uint32_t *__restrict__ hi, uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x)
        hi[x] = (uint32_t)(k64[p1[x]] >> 32);
}

template <typename V>
__global__ void k_u64_final(const uint64_t *__restrict__ k64, const V *__restrict__ vals,
                            const uint32_t *__restrict__ p1, const uint32_t *__restrict__ p2,
                            uint64_t *__restrict__ out_k, V *__restrict__ out_v, uint64_t n)
{
    for (uint64_t y = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; y < n;
         y += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t src = p1[p2[y]];
        out_k[y] = k64[src];
        out_v[y] = vals[src];
    }
}

// ============================================================ launch wrappers
int smem_bytes_for_cap(int cap, bool pairs)
{
    return pairs ? padded_elems<uint64_t>(cap) * 8 : padded_elems<uint32_t>(cap) * 4;
}

template <typename KernelT>
static cudaError_t set_smem(KernelT kern, int bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

#define BSORT_TRY(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

cudaError_t init_misc_kernels()
{
    BSORT_TRY(set_smem(k_records_sort<1024, 16>, smem_bytes_for_cap(kRecordChunk, true)));
    BSORT_TRY(set_smem(k_pack_units<1024>, 16 * (kMaxBuckets + 1)));
    BSORT_TRY(set_smem(k_units_each<1024>, 4 * (kMaxBucketsTiers + 1)));
    BSORT_TRY(set_smem(k_bucket_relocate<kFuseT, kFuseV>, (int)(8 * kFuseMaxM + 4)));
    return cudaSuccess;
}

cudaError_t launch_records_chunk_sort(const uint64_t *src, uint64_t *dst, uint32_t n_rec,
                                      uint32_t n_pad, uint64_t *spl, uint32_t s, uint32_t b,
                                      cudaStream_t st)
{
    const uint32_t chunks = n_pad / kRecordChunk;
    k_records_sort<1024, 16><<<chunks, 1024, smem_bytes_for_cap(kRecordChunk, true), st>>>(
        src, dst, n_rec, chunks == 1 ? spl : nullptr, s, b);
    return cudaGetLastError();
}

cudaError_t launch_merge_pass(const uint64_t *src, uint64_t *dst, uint32_t n_pad, uint32_t L,
                              cudaStream_t st)
{
    // a CTA's outputs never span two pairs of runs: L and n_pad are
    // multiples of kRecordChunk, itself a multiple of kMergeTile
    static_assert(kRecordChunk % kMergeTile == 0, "merge tiles must divide record chunks");
    if (n_pad % kRecordChunk != 0 || L % kRecordChunk != 0) return cudaErrorInvalidValue;
    k_merge_pass<256, 16><<<n_pad / kMergeTile, 256, 0, st>>>(src, dst, n_pad, L);
    return cudaGetLastError();
}

cudaError_t launch_select_splitters(const uint64_t *sorted, uint32_t n_rec, uint32_t b,
                                    uint64_t *spl, cudaStream_t st)
{
    k_select_splitters<<<(b + 255) / 256, 256, 0, st>>>(sorted, n_rec, b, spl);
    return cudaGetLastError();
}

cudaError_t launch_sample_index(const uint32_t *tiles_k, const uint64_t *spl, uint32_t t,
                                uint32_t s, uint32_t b, uint32_t m, uint32_t *jr, uint32_t *cum,
                                cudaStream_t st)
{
    if (s == 0 || (s & (s - 1)) != 0 || (t & (t - 1)) != 0) return cudaErrorInvalidValue;
    const uint32_t seg = t < (uint32_t)kSegItems ? t : (uint32_t)kSegItems;
    const uint32_t nseg = t / seg;
    const uint32_t ns = m * nseg;
    k_seg_ranges<<<(ns + 255) / 256, 256, 0, st>>>(tiles_k, spl, t, s, b, m, nseg, seg, jr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t groups = (m + kSub6 - 1) / kSub6;
    if (seg == (uint32_t)kSegItems)
        k_sample_index_grp<256, kSegItems><<<groups * nseg, 256, 0, st>>>(tiles_k, spl, t, s, b,
                                                                         m, nseg, seg, jr, cum);
    else
        k_sample_index_grp<256, 0><<<groups * nseg, 256, 0, st>>>(tiles_k, spl, t, s, b, m, nseg,
                                                                 seg, jr, cum);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *in, uint32_t *out, uint32_t n_items,
                        unsigned long long *status, uint32_t *ticket, int *err, cudaStream_t st)
{
    const uint32_t chunks = (n_items + kScanChunk - 1) / kScanChunk;
    k_scan<256, 16><<<chunks, 256, 0, st>>>(in, out, n_items, status, ticket, err, nullptr, 1u,
                                            0u, nullptr, nullptr, kSpinLimit, 0);
    return cudaGetLastError();
}

cudaError_t launch_scan_cum(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t *counts,
                            uint32_t *srcb, uint32_t *out, uint32_t n_items,
                            unsigned long long *status, uint32_t *ticket, int *err,
                            cudaStream_t st, bool stall_first)
{
    const uint32_t chunks = (n_items + kScanChunk - 1) / kScanChunk;
    k_scan<256, 16><<<chunks, 256, 0, st>>>(nullptr, out, n_items, status, ticket, err, cum, m,
                                            t, counts, srcb,
                                            stall_first ? kTestSpinLimit : kSpinLimit,
                                            stall_first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_relocate(const uint32_t *tiles_k, const void *tiles_v, const uint32_t *offsets,
                            const uint32_t *srcb, const uint32_t *blk, uint32_t runs,
                            uint32_t n_pad, int val_bytes, uint32_t *reloc_k, void *reloc_v,
                            cudaStream_t st, const uint32_t *cum, uint32_t m, uint32_t t)
{
    constexpr int T = (kRelocPart / kBlockItems) * 32;
    const uint32_t grid = (n_pad + kRelocPart - 1) / kRelocPart;
    if (srcb == nullptr && (cum == nullptr || m == 0)) return cudaErrorInvalidValue;
    k_relocate<T, uint32_t><<<grid, T, 0, st>>>(tiles_k, tiles_v, offsets, srcb, cum, m, t, blk,
                                                runs, n_pad, val_bytes, reloc_k, reloc_v);
    return cudaGetLastError();
}

bool bucket_relocate_fits(uint32_t m) { return m > 0 && m <= kFuseMaxM && (m & 3u) == 0; }

cudaError_t launch_bucket_relocate(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t b,
                                  uint32_t n_pad, const uint32_t *tiles_k, const void *tiles_v,
                                  int val_bytes, uint32_t *offsets, uint32_t *reloc_k,
                                  void *reloc_v, cudaStream_t st)
{
    if (!bucket_relocate_fits(m) || b == 0) return cudaErrorInvalidValue;
    k_bucket_relocate<kFuseT, kFuseV><<<b, kFuseT, 8 * kFuseMaxM + 4, st>>>(
        cum, m, t, b, n_pad, tiles_k, tiles_v, val_bytes, offsets, reloc_k, reloc_v);
    return cudaGetLastError();
}

cudaError_t launch_row_scan(const uint32_t *cum, uint32_t m, uint32_t t, uint32_t b,
                            uint32_t *counts, uint32_t *srcb, uint32_t *out, cudaStream_t st)
{
    if (m == 0 || b == 0) return cudaSuccess;
    if (m <= 2048u)
        k_row_scan<128, 16><<<b, 128, 0, st>>>(cum, m, t, out, counts, srcb);
    else
        k_row_scan<512, 16><<<b, 512, 0, st>>>(cum, m, t, out, counts, srcb);
    return cudaGetLastError();
}

cudaError_t launch_relocate_u64(const uint64_t *tiles_k, const uint32_t *offsets,
                                const uint32_t *srcb, const uint32_t *blk, uint32_t runs,
                                uint32_t n_pad, uint64_t *reloc_k, cudaStream_t st)
{
    constexpr int T = (kRelocPart / kBlockItems) * 32;
    const uint32_t grid = (n_pad + kRelocPart - 1) / kRelocPart;
    k_relocate<T, uint64_t><<<grid, T, 0, st>>>(tiles_k, nullptr, offsets, srcb, nullptr, 1u, 0u,
                                                blk, runs,
                                                n_pad, 0, reloc_k, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_block_index(uint32_t *offsets, uint32_t runs, uint32_t n_pad, uint32_t *blk,
                               cudaStream_t st)
{
    const uint32_t nblk = (n_pad + kBlockItems - 1) / kBlockItems;
    k_block_index<<<(nblk + 255) / 256, 256, 0, st>>>(offsets, runs, n_pad, blk, nblk);
    return cudaGetLastError();
}

cudaError_t launch_units_each(const uint32_t *offsets, uint32_t m, uint32_t b, uint32_t n_pad,
                              uint32_t Q1, uint32_t Q2, uint32_t *units, uint32_t *units2,
                              int *err, cudaStream_t st)
{
    if (b > (uint32_t)kMaxBucketsTiers || units2 == nullptr) return cudaErrorInvalidValue;
    const int sm = (int)(4 * (b + 1));
    k_units_each<1024><<<1, 1024, sm, st>>>(offsets, m, b, n_pad, Q1, Q2, units, units2, err);
    return cudaGetLastError();
}

cudaError_t launch_pack_units(const uint32_t *offsets, uint32_t m, uint32_t b, uint32_t n_pad,
                              uint32_t Q1, uint32_t Q2, uint32_t *units, uint32_t *units2,
                              int *err, cudaStream_t st)
{
    const int sm = (int)(4 * (b + 1) * 4);
    k_pack_units<1024><<<1, 1024, sm, st>>>(offsets, m, b, n_pad, Q1, Q2, units, units2, err);
    return cudaGetLastError();
}

// ranges[g] = first unit (of count units, sorted by begin) whose begin is
// >= g * n_pad / G; ranges[G] = count.
__global__ void k_unit_ranges(const uint32_t *__restrict__ units, uint32_t n_pad, uint32_t G,
                              uint32_t *__restrict__ ranges)
{
    const uint32_t g = threadIdx.x;
    if (g > G) return;
    const uint32_t count = units[0];
    if (g == G) {
        ranges[g] = count;
        return;
    }
    const uint32_t pos = (uint32_t)((uint64_t)g * n_pad / G);
    uint32_t lo = 0, hi = count;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (units[1 + 2 * mid] < pos) lo = mid + 1;
        else hi = mid;
    }
    ranges[g] = lo;
}

cudaError_t launch_unit_ranges(const uint32_t *units, uint32_t n_pad, uint32_t G,
                               uint32_t *ranges, cudaStream_t st)
{
    if (G + 1 > 32) return cudaErrorInvalidValue;  // one thread per slice boundary
    k_unit_ranges<<<1, 32, 0, st>>>(units, n_pad, G, ranges);
    return cudaGetLastError();
}

cudaError_t launch_scan_cum64(const uint32_t *cum, uint32_t m, uint32_t n_items,
                              uint32_t *chunk_sums, uint64_t *chunk_pre, uint64_t n_pad,
                              uint64_t *off64, cudaStream_t st)
{
    const uint32_t chunks = (n_items + kScanChunk - 1) / kScanChunk;
    k_cum_chunk_sums<256, 16><<<chunks, 256, 0, st>>>(cum, m, n_items, chunk_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_chunk_prefix64<1024><<<1, 1024, 0, st>>>(chunk_sums, chunks, chunk_pre);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_offsets64<256, 16><<<chunks, 256, 0, st>>>(cum, m, n_items, chunk_pre, n_pad, off64);
    return cudaGetLastError();
}

cudaError_t launch_relocate_src64(const uint32_t *tiles_k, const uint32_t *cum,
                                  const uint64_t *off64, uint32_t m, uint32_t b, uint32_t t,
                                  uint32_t *reloc, cudaStream_t st)
{
    k_relocate_src64<256><<<m, 256, 0, st>>>(tiles_k, cum, off64, m, b, t, reloc);
    return cudaGetLastError();
}

cudaError_t launch_bucket_starts64(const uint64_t *off64, uint32_t m, uint32_t b, uint64_t n_pad,
                                   uint64_t *starts, cudaStream_t st)
{
    k_bucket_starts64<<<(b + 256) / 256, 256, 0, st>>>(off64, m, b, n_pad, starts);
    return cudaGetLastError();
}

cudaError_t launch_f32_decode(const uint32_t *src, uint32_t *dst, uint64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    k_f32_decode<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_merge_error(const int *from, int *to, cudaStream_t st)
{
    k_merge_error<<<1, 32, 0, st>>>(from, to);
    return cudaGetLastError();
}

static unsigned elementwise_grid(uint64_t n)
{
    const uint64_t blocks = (n + 255) / 256;
    return (unsigned)(blocks < 65536 ? (blocks ? blocks : 1) : 65536);
}

cudaError_t launch_u64_split(const uint64_t *k64, uint32_t *lo, uint32_t *iota, uint64_t n,
                             cudaStream_t st)
{
    k_u64_split<<<elementwise_grid(n), 256, 0, st>>>(k64, lo, iota, n);
    return cudaGetLastError();
}

cudaError_t launch_u64_gather_hi(const uint64_t *k64, const uint32_t *p1, uint32_t *hi,
                                 uint64_t n, cudaStream_t st)
{
    k_u64_gather_hi<<<elementwise_grid(n), 256, 0, st>>>(k64, p1, hi, n);
    return cudaGetLastError();
}

cudaError_t launch_u64_final(const uint64_t *k64, const void *vals, int val_bytes,
                             const uint32_t *p1, const uint32_t *p2, uint64_t *out_k,
                             void *out_v, uint64_t n, cudaStream_t st)
{
    if (val_bytes == 4)
        k_u64_final<uint32_t><<<elementwise_grid(n), 256, 0, st>>>(
            k64, static_cast<const uint32_t *>(vals), p1, p2, out_k,
            static_cast<uint32_t *>(out_v), n);
    else
        k_u64_final<uint64_t><<<elementwise_grid(n), 256, 0, st>>>(
            k64, static_cast<const uint64_t *>(vals), p1, p2, out_k,
            static_cast<uint64_t *>(out_v), n);
    return cudaGetLastError();
}

cudaError_t init_kernels()
{
    cudaError_t e = init_misc_kernels();
    if (e == cudaSuccess) e = init_records_kernels();
    if (e == cudaSuccess) e = init_sort_keys_kernels();
    if (e == cudaSuccess) e = init_sort_pairs_kernels();
    if (e == cudaSuccess) e = init_batch_kernels();
    if (e == cudaSuccess) e = init_u64_kernels();
    return e;
}

}  // namespace bsort
