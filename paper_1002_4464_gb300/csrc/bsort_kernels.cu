// bsort_kernels.cu -- the kernels of GPU Bucket Sort (Dehne & Zaboli,
// Section 4, Algorithm 1) for sm_103a, and their launch wrappers.
//
//   Steps 1-3  k_sublist_sort      sort each sublist in SMEM, emit samples
//   Step 4     k_records_sort      sort the s*m samples (chunks of 16K) ...
//              k_merge_pass        ... then merge-path passes through L2
//   Step 5     k_select_splitters  every m-th sorted sample
//   Step 6     k_sample_index      locate the s splitters in every sublist
//   Step 7     k_scan              bucket-major exclusive scan (look-back)
//   Step 8     k_relocate          move each run A_ij to l_ij
//   Step 9     k_bucket_sort       sort each bucket B_j in SMEM
//
// Items are compared in composite order (key, position): keys-only sorts
// compare keys (equal keys are indistinguishable), pair sorts compare the
// 64-bit word key << 32 | local index, which makes them stable, and the
// sample records of Steps 3-6 are key << 32 | p with p = i*t + r.
#include "bsort_device.cuh"
#include "bsort_internal.h"

namespace bsort {

// ============================================================ Steps 1-3
// One CTA per sublist i of t = T*E items.  Loads are striped (coalesced);
// a keys-only sort needs no particular assignment of keys to threads, and a
// pair sort carries the local index inside the composite key.
template <int T, int E, bool PAIRS>
__global__ void __launch_bounds__(T, 1)
k_sublist_sort(const uint32_t *__restrict__ keys_in, const void *__restrict__ vals_in,
               uint64_t n, int is_f32, int val_bytes, uint32_t s,
               uint32_t *__restrict__ tiles_k, void *__restrict__ tiles_v,
               uint64_t *__restrict__ samples)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    constexpr int CAP = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const uint64_t base = (uint64_t)blockIdx.x * CAP;
    const uint64_t avail = n > base ? n - base : 0;

    const int lane = tid & 31, warp = tid >> 5;
    K v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = wb_pos<E>(warp, lane, k);
        uint32_t key = 0xFFFFFFFFu;  // pad sentinel (position >= n)
        if ((uint64_t)x < avail) {
            key = keys_in[base + x];
            if (is_f32) key = f32_encode(key);
        }
        if constexpr (PAIRS) v[k] = ((uint64_t)key << 32) | (uint32_t)x;
        else v[k] = (K)key;
    }
    cta_sort<K, T, E>(v, sm, avail < (uint64_t)CAP ? (int)avail : CAP);

#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        const K e = sm[pidx<K>(x)];
        if constexpr (PAIRS) {
            const uint32_t idx = (uint32_t)(e & 0xFFFFFFFFull);
            tiles_k[base + x] = (uint32_t)((uint64_t)e >> 32);
            if (val_bytes == 4) {
                uint32_t val = (uint64_t)idx < avail
                                   ? static_cast<const uint32_t *>(vals_in)[base + idx] : 0u;
                static_cast<uint32_t *>(tiles_v)[base + x] = val;
            } else {
                uint64_t val = (uint64_t)idx < avail
                                   ? static_cast<const uint64_t *>(vals_in)[base + idx] : 0ull;
                static_cast<uint64_t *>(tiles_v)[base + x] = val;
            }
        } else {
            tiles_k[base + x] = (uint32_t)e;
        }
    }
    // Step 3: samples at ranks (k+1)w - 1 as (key, p = i*t + r).
    const uint32_t w = CAP / s;
    for (uint32_t k = tid; k < s; k += T) {
        const uint32_t r = (k + 1) * w - 1;
        const K e = sm[pidx<K>(r)];
        const uint32_t key = PAIRS ? (uint32_t)((uint64_t)e >> 32) : (uint32_t)e;
        samples[(uint64_t)blockIdx.x * s + k] = ((uint64_t)key << 32) | (uint32_t)(base + r);
    }
}

// ============================================================ Step 4 (chunks)
// The records of one sublist (s consecutive records) are already sorted, so
// when s >= 32*E the chunk is loaded as sorted runs (odd runs reversed) and
// only the remaining merge levels run; otherwise the chunk is sorted whole.
template <int T, int E>
__global__ void __launch_bounds__(T, 1)
k_records_sort(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, uint32_t n_rec,
               uint64_t *__restrict__ spl, uint32_t m, uint32_t s)
{
    constexpr int CAP = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * CAP;
    if (s >= 32u * E && s < (uint32_t)CAP) {
        for (int x = tid; x < CAP; x += T) {
            const uint64_t g = base + x;
            const uint64_t r = g < n_rec ? src[g] : 0xFFFFFFFFFFFFFFFFull;
            const int q = x / (int)s, o = x % (int)s;
            const int pos = (q & 1) ? q * (int)s + (int)s - 1 - o : x;
            sm[pidx<uint64_t>(pos)] = r;
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
        for (uint32_t j = tid; j < s; j += T) spl[j] = sm[pidx<uint64_t>((j + 1) * m - 1)];
    }
}

// ============================================================ Step 4 (merges)
__device__ __forceinline__ uint32_t merge_path_global(const uint64_t *A, uint32_t la,
                                                      const uint64_t *B, uint32_t lb,
                                                      uint32_t d)
{
    uint32_t lo = d > lb ? d - lb : 0;
    uint32_t hi = d < la ? d : la;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One CTA produces kMergeTile outputs of the merge of two runs: it finds
// the input ranges of its outputs by merge path in global memory, stages
// them in SMEM, merges per thread, and writes back through SMEM.
template <int T, int E>
__global__ void __launch_bounds__(T)
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
    if (tid == 0) s_split[0] = merge_path_global(src + a0, la, src + b0, lb, d0);
    if (tid == 32) s_split[1] = merge_path_global(src + a0, la, src + b0, lb, d1);
    __syncthreads();
    const uint32_t i0 = s_split[0], i1 = s_split[1];
    const uint32_t j0 = d0 - i0, j1 = d1 - i1;
    const int na = (int)(i1 - i0), nb = (int)(j1 - j0);
    for (int x = tid; x < na; x += T) sm[pidx<uint64_t>(x)] = src[a0 + i0 + x];
    for (int x = tid; x < nb; x += T) sm[pidx<uint64_t>(na + x)] = src[b0 + j0 + x];
    __syncthreads();
    const int cnt = na + nb;
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
__global__ void k_select_splitters(const uint64_t *__restrict__ sorted, uint32_t m,
                                   uint32_t s, uint64_t *__restrict__ spl)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < s) spl[j] = sorted[(uint64_t)(j + 1) * m - 1];
}

// ============================================================ Step 6
// One CTA per sublist i.  The sublist's own s samples (sorted, every w-th
// item) index the sorted sublist: for splitter g, q = #samples <= g gives
// c in [q*w, q*w + w - 1], and a binary search over the w - 1 items of that
// window gives c exactly.  Items compare as key << 32 | (i*t + r).
template <int T>
__global__ void __launch_bounds__(T)
k_sample_index(const uint32_t *__restrict__ tiles_k, const uint64_t *__restrict__ samples,
               const uint64_t *__restrict__ spl, uint32_t t, uint32_t s, uint32_t m,
               uint32_t *__restrict__ counts, uint32_t *__restrict__ cum)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_samp = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *s_c = reinterpret_cast<uint32_t *>(s_samp + s);
    const uint32_t i = blockIdx.x;
    const uint64_t base = (uint64_t)i * t;
    const uint32_t w = t / s;
    for (uint32_t k = threadIdx.x; k < s; k += T) s_samp[k] = samples[(uint64_t)i * s + k];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < s; j += T) {
        const uint64_t g = spl[j];
        uint32_t lo = 0, hi = s;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (s_samp[mid] <= g) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t q = lo;
        uint32_t c;
        if (q == s) {
            c = t;
        } else {
            uint32_t a = q * w, b = q * w + w - 1;  // item at rank b is > g
            while (a < b) {
                uint32_t mid = (a + b) >> 1;
                uint64_t item = ((uint64_t)tiles_k[base + mid] << 32) | (uint32_t)(base + mid);
                if (item <= g) a = mid + 1;
                else b = mid;
            }
            c = a;
        }
        s_c[j] = c;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < s; j += T) {
        const uint32_t c = s_c[j];
        const uint32_t prev = j ? s_c[j - 1] : 0u;
        counts[(uint64_t)j * m + i] = c - prev;
        cum[(uint64_t)i * s + j] = c;
    }
}

// ============================================================ Step 7
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;  // ~0.5-1 s with the back-off below

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

template <int T, int ITEMS>
__global__ void __launch_bounds__(T)
k_scan(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint32_t n_items,
       unsigned long long *status, uint32_t *ticket, int *err)
{
    __shared__ uint32_t s_chunk;
    __shared__ uint32_t s_warp[T / 32];
    __shared__ uint32_t s_prefix;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_chunk = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t chunk = s_chunk;
    const uint64_t base = (uint64_t)chunk * (T * ITEMS) + (uint64_t)tid * ITEMS;
    uint32_t x[ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        x[k] = (base + k < n_items) ? in[base + k] : 0u;
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
        if (lane == T / 32 - 1) {
            const uint32_t agg = wi;
            // decoupled look-back (bounded waits)
            uint32_t prefix = 0;
            if (chunk == 0) {
                atomicExch(&status[0], kFlagInc | agg);
            } else {
                atomicExch(&status[chunk], kFlagAgg | agg);
                int p = (int)chunk - 1;
                while (p >= 0) {
                    unsigned long long st = ld_volatile(&status[p]);
                    int spins = 0;
                    while ((st >> 62) == 0) {
                        if (++spins > kSpinLimit) break;
                        __nanosleep(128);
                        st = ld_volatile(&status[p]);
                    }
                    if ((st >> 62) == 0) {
                        set_error(err, DEV_TIMEOUT);
                        break;
                    }
                    prefix += (uint32_t)(st & kValMask);
                    if ((st & kFlagInc) == kFlagInc && (st >> 62) == 2) break;
                    --p;
                }
                __threadfence();
                atomicExch(&status[chunk], kFlagInc | (unsigned long long)(prefix + agg));
            }
            s_prefix = prefix;
        }
    }
    __syncthreads();
    uint32_t run = s_prefix + s_warp[warp] + (incl - sum);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (base + k < n_items) out[base + k] = run;
        run += x[k];
    }
}

// ============================================================ Step 8
// One CTA per sublist: the sorted sublist (keys, and values when they fit),
// its cumulative counts c_i. and its offsets l_.i are staged in shared memory
// with coalesced loads; then each warp copies whole runs A_ij to l_ij
// (lanes in parallel, coalesced stores).
template <int T>
__global__ void __launch_bounds__(T, 1)
k_relocate(const uint32_t *__restrict__ tiles_k, const void *__restrict__ tiles_v,
           const uint32_t *__restrict__ cum, const uint32_t *__restrict__ offsets,
           uint32_t t, uint32_t s, uint32_t m, uint64_t n_pad, int val_bytes, int stage_vals,
           uint32_t *__restrict__ reloc_k, void *__restrict__ reloc_v, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_k = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *s_cum = s_k + t;
    uint32_t *s_off = s_cum + s;
    unsigned char *s_v = reinterpret_cast<unsigned char *>(s_off + s);
    const uint32_t i = blockIdx.x;
    const uint64_t base = (uint64_t)i * t;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    {
        const uint4 *src4 = reinterpret_cast<const uint4 *>(tiles_k + base);
        uint4 *dst4 = reinterpret_cast<uint4 *>(s_k);
        for (uint32_t x = tid; x < t / 4; x += T) dst4[x] = src4[x];
        if (stage_vals) {
            const uint4 *v4 = reinterpret_cast<const uint4 *>(
                static_cast<const unsigned char *>(tiles_v) + base * val_bytes);
            uint4 *d4 = reinterpret_cast<uint4 *>(s_v);
            for (uint32_t x = tid; x < t * val_bytes / 16; x += T) d4[x] = v4[x];
        }
        for (uint32_t j = tid; j < s; j += T) {
            s_cum[j] = cum[(uint64_t)i * s + j];
            s_off[j] = offsets[(uint64_t)j * m + i];
        }
    }
    __syncthreads();
    for (uint32_t j = warp; j < s; j += T / 32) {
        const uint32_t start = j ? s_cum[j - 1] : 0u;
        const uint32_t end = s_cum[j];
        const uint64_t dst = s_off[j];
        if (end < start || end > t || dst + (end - start) > n_pad) {  // never for a valid plan
            if (lane == 0) set_error(err, DEV_INTERNAL);
            continue;
        }
        for (uint32_t x = start + lane; x < end; x += 32) {
            reloc_k[dst + (x - start)] = s_k[x];
            if (val_bytes == 4) {
                const uint32_t val = stage_vals ? reinterpret_cast<const uint32_t *>(s_v)[x]
                                                : static_cast<const uint32_t *>(tiles_v)[base + x];
                static_cast<uint32_t *>(reloc_v)[dst + (x - start)] = val;
            } else if (val_bytes == 8) {
                const uint64_t val = stage_vals ? reinterpret_cast<const uint64_t *>(s_v)[x]
                                                : static_cast<const uint64_t *>(tiles_v)[base + x];
                static_cast<uint64_t *>(reloc_v)[dst + (x - start)] = val;
            }
        }
    }
}

// Step 9 units: consecutive buckets packed greedily into units of at most Q
// items (every bucket fits one unit, since |B_j| <= bound <= Q).  One CTA:
// nxt[j] = the bucket after the longest run of buckets from j that fits, the
// chain 0, nxt[0], nxt[nxt[0]], ... marks the unit starts (found by pointer
// doubling), and a scan numbers them.  units[0] = U, then (begin, end) pairs.
template <int T>
__global__ void __launch_bounds__(T, 1)
k_pack_units(const uint32_t *__restrict__ offsets, uint32_t m, uint32_t s, uint32_t n_pad,
             uint32_t Q, uint32_t *__restrict__ units, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem_raw);  // s + 1
    uint32_t *nxt = Lb + (s + 1);                             // s + 1
    uint32_t *jmp = nxt + (s + 1);                            // s + 1
    uint32_t *on = jmp + (s + 1);                             // s + 1
    __shared__ uint32_t s_warp[T / 32];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x;
    for (uint32_t j = tid; j <= s; j += T) {
        Lb[j] = j < s ? offsets[(uint64_t)j * m] : n_pad;
        on[j] = j == 0 ? 1u : 0u;
    }
    __syncthreads();
    for (uint32_t j = tid; j <= s; j += T) {
        uint32_t e = j;
        if (j < s) {
            uint32_t lo = j + 1, hi = s;  // largest e in [j+1, s] with Lb[e] - Lb[j] <= Q
            const uint32_t lim = Lb[j] + Q;
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (Lb[mid] <= lim) lo = mid;
                else hi = mid - 1;
            }
            e = lo;
            if (Lb[e] - Lb[j] > Q) set_error(err, DEV_INTERNAL);  // a bucket exceeds Q
        }
        nxt[j] = e;
        jmp[j] = e;
    }
    __syncthreads();
    for (uint32_t span = 1; span <= s; span <<= 1) {
        for (uint32_t j = tid; j <= s; j += T)
            if (on[j]) on[jmp[j]] = 1u;
        __syncthreads();
        for (uint32_t j = tid; j <= s; j += T) {
            const uint32_t a = jmp[j];
            nxt[j] = jmp[a];  // use nxt as scratch for the doubled jump
        }
        __syncthreads();
        for (uint32_t j = tid; j <= s; j += T) jmp[j] = nxt[j];
        __syncthreads();
    }
    // recompute the single-step successor (nxt was used as scratch)
    for (uint32_t j = tid; j <= s; j += T) {
        uint32_t e = j;
        if (j < s) {
            uint32_t lo = j + 1, hi = s;
            const uint32_t lim = Lb[j] + Q;
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (Lb[mid] <= lim) lo = mid;
                else hi = mid - 1;
            }
            e = lo;
        }
        nxt[j] = e;
    }
    __syncthreads();
    // number the unit starts (chain members j < s) in order: block scan
    const uint32_t per = (s + T - 1) / T;
    const uint32_t j0 = tid * per;
    uint32_t cnt = 0;
    for (uint32_t q = 0; q < per; ++q)
        if (j0 + q < s && on[j0 + q]) ++cnt;
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t incl = cnt;
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
        if (lane < T / 32) s_warp[lane] = wi - wv;
        if (lane == T / 32 - 1) s_total = wi;
    }
    __syncthreads();
    uint32_t u = s_warp[warp] + incl - cnt;
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t j = j0 + q;
        if (j < s && on[j]) {
            units[1 + 2 * u] = Lb[j];
            units[2 + 2 * u] = Lb[nxt[j]];
            ++u;
        }
    }
    if (tid == 0) units[0] = s_total;
}

// ============================================================ Step 9
template <int T, int E, bool PAIRS>
__global__ void __launch_bounds__(T, 1)
k_bucket_sort(const uint32_t *__restrict__ src_k, const void *__restrict__ src_v,
              const uint32_t *__restrict__ units, uint64_t n, uint64_t n_pad, int is_f32,
              int val_bytes, uint32_t *__restrict__ out_k, void *__restrict__ out_v, int *err)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    constexpr int CAP = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t u = blockIdx.x;
    const bool direct = units == nullptr;
    uint64_t L = 0, R = n;
    if (!direct) {
        if (u >= units[0]) return;  // fewer units than the grid
        L = units[1 + 2 * u];
        R = units[2 + 2 * u];
    }
    const uint64_t len = R - L;
    if (R < L || R > n_pad || len > (uint64_t)CAP) {  // the plan guarantees a unit fits
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;
    }
    if (len == 0) return;
    K v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = wb_pos<E>(warp, lane, k);
        uint32_t key = 0xFFFFFFFFu;
        if ((uint64_t)x < len) {
            key = src_k[L + x];
            if (direct && is_f32) key = f32_encode(key);
        }
        if constexpr (PAIRS) v[k] = ((uint64_t)key << 32) | (uint32_t)x;
        else v[k] = (K)key;
    }
    cta_sort<K, T, E>(v, sm, (int)len);
    const uint64_t lim = min((unsigned long long)len, (unsigned long long)(n > L ? n - L : 0));
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        if ((uint64_t)x < lim) {
            const K e = sm[pidx<K>(x)];
            uint32_t key = PAIRS ? (uint32_t)((uint64_t)e >> 32) : (uint32_t)e;
            if (is_f32) key = f32_decode(key);
            out_k[L + x] = key;
            if constexpr (PAIRS) {
                const uint32_t idx = (uint32_t)((uint64_t)e & 0xFFFFFFFFull);
                if (val_bytes == 4)
                    static_cast<uint32_t *>(out_v)[L + x] =
                        static_cast<const uint32_t *>(src_v)[L + idx];
                else
                    static_cast<uint64_t *>(out_v)[L + x] =
                        static_cast<const uint64_t *>(src_v)[L + idx];
            }
        }
    }
}

// ============================================================ launch wrappers
bool cap_supported(int cap, bool pairs)
{
    if (pairs) return cap == 2048 || cap == 4096 || cap == 8192 || cap == 16384;
    return cap == 2048 || cap == 4096 || cap == 8192 || cap == 16384 || cap == 32768;
}

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

cudaError_t init_kernels()
{
    BSORT_TRY(set_smem(k_sublist_sort<128, 16, false>, smem_bytes_for_cap(2048, false)));
    BSORT_TRY(set_smem(k_sublist_sort<128, 16, true>, smem_bytes_for_cap(2048, true)));
    BSORT_TRY(set_smem(k_bucket_sort<128, 16, false>, smem_bytes_for_cap(2048, false)));
    BSORT_TRY(set_smem(k_bucket_sort<128, 16, true>, smem_bytes_for_cap(2048, true)));
    BSORT_TRY(set_smem(k_sublist_sort<256, 16, false>, smem_bytes_for_cap(4096, false)));
    BSORT_TRY(set_smem(k_sublist_sort<512, 16, false>, smem_bytes_for_cap(8192, false)));
    BSORT_TRY(set_smem(k_sublist_sort<1024, 16, false>, smem_bytes_for_cap(16384, false)));
    BSORT_TRY(set_smem(k_sublist_sort<1024, 32, false>, smem_bytes_for_cap(32768, false)));
    BSORT_TRY(set_smem(k_sublist_sort<256, 16, true>, smem_bytes_for_cap(4096, true)));
    BSORT_TRY(set_smem(k_sublist_sort<512, 16, true>, smem_bytes_for_cap(8192, true)));
    BSORT_TRY(set_smem(k_sublist_sort<1024, 16, true>, smem_bytes_for_cap(16384, true)));
    BSORT_TRY(set_smem(k_bucket_sort<256, 16, false>, smem_bytes_for_cap(4096, false)));
    BSORT_TRY(set_smem(k_bucket_sort<512, 16, false>, smem_bytes_for_cap(8192, false)));
    BSORT_TRY(set_smem(k_bucket_sort<1024, 16, false>, smem_bytes_for_cap(16384, false)));
    BSORT_TRY(set_smem(k_bucket_sort<1024, 32, false>, smem_bytes_for_cap(32768, false)));
    BSORT_TRY(set_smem(k_bucket_sort<256, 16, true>, smem_bytes_for_cap(4096, true)));
    BSORT_TRY(set_smem(k_bucket_sort<512, 16, true>, smem_bytes_for_cap(8192, true)));
    BSORT_TRY(set_smem(k_bucket_sort<1024, 16, true>, smem_bytes_for_cap(16384, true)));
    BSORT_TRY(set_smem(k_records_sort<1024, 16>, smem_bytes_for_cap(kRecordChunk, true)));
    BSORT_TRY(set_smem(k_sample_index<256>, 64 * 1024));
    BSORT_TRY(set_smem(k_relocate<1024>, kRelocateSmemMax));
    BSORT_TRY(set_smem(k_pack_units<1024>, 16 * 4097));
    return cudaSuccess;
}

cudaError_t launch_sublist_sort(int cap, bool pairs, const void *keys_in, const void *vals_in,
                                uint64_t n, uint32_t m, int is_f32, int val_bytes, uint32_t s,
                                uint32_t *tiles_k, void *tiles_v, uint64_t *samples,
                                cudaStream_t st)
{
    const int sm = smem_bytes_for_cap(cap, pairs);
    const uint32_t *kin = static_cast<const uint32_t *>(keys_in);
#define BSORT_L1(T_, E_, P_)                                                                \
    k_sublist_sort<T_, E_, P_><<<m, T_, sm, st>>>(kin, vals_in, n, is_f32, val_bytes, s,   \
                                                   tiles_k, tiles_v, samples)
    if (!pairs) {
        switch (cap) {
        case 2048: BSORT_L1(128, 16, false); break;
        case 4096: BSORT_L1(256, 16, false); break;
        case 8192: BSORT_L1(512, 16, false); break;
        case 16384: BSORT_L1(1024, 16, false); break;
        case 32768: BSORT_L1(1024, 32, false); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (cap) {
        case 2048: BSORT_L1(128, 16, true); break;
        case 4096: BSORT_L1(256, 16, true); break;
        case 8192: BSORT_L1(512, 16, true); break;
        case 16384: BSORT_L1(1024, 16, true); break;
        default: return cudaErrorInvalidValue;
        }
    }
#undef BSORT_L1
    return cudaGetLastError();
}

cudaError_t launch_records_chunk_sort(const uint64_t *src, uint64_t *dst, uint32_t n_rec,
                                      uint32_t n_pad, uint64_t *spl, uint32_t m, uint32_t s,
                                      cudaStream_t st)
{
    const uint32_t chunks = n_pad / kRecordChunk;
    k_records_sort<1024, 16><<<chunks, 1024, smem_bytes_for_cap(kRecordChunk, true), st>>>(
        src, dst, n_rec, chunks == 1 ? spl : nullptr, m, s);
    return cudaGetLastError();
}

cudaError_t launch_merge_pass(const uint64_t *src, uint64_t *dst, uint32_t n_pad, uint32_t L,
                              cudaStream_t st)
{
    k_merge_pass<256, 16><<<n_pad / kMergeTile, 256, 0, st>>>(src, dst, n_pad, L);
    return cudaGetLastError();
}

cudaError_t launch_select_splitters(const uint64_t *sorted, uint32_t m, uint32_t s,
                                    uint64_t *spl, cudaStream_t st)
{
    k_select_splitters<<<(s + 255) / 256, 256, 0, st>>>(sorted, m, s, spl);
    return cudaGetLastError();
}

cudaError_t launch_sample_index(const uint32_t *tiles_k, const uint64_t *samples,
                                const uint64_t *spl, uint32_t t, uint32_t s, uint32_t m,
                                uint32_t *counts, uint32_t *cum, cudaStream_t st)
{
    const int sm = (int)(s * 12);
    if (sm > 64 * 1024) return cudaErrorInvalidValue;
    k_sample_index<256><<<m, 256, sm, st>>>(tiles_k, samples, spl, t, s, m, counts, cum);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *in, uint32_t *out, uint32_t n_items,
                        unsigned long long *status, uint32_t *ticket, int *err, cudaStream_t st)
{
    const uint32_t chunks = (n_items + kScanChunk - 1) / kScanChunk;
    k_scan<256, 16><<<chunks, 256, 0, st>>>(in, out, n_items, status, ticket, err);
    return cudaGetLastError();
}

int relocate_smem_bytes(uint32_t t, uint32_t s, int val_bytes, int *stage_vals)
{
    int bytes = (int)(t * 4 + 2 * s * 4);
    bytes = (bytes + 15) / 16 * 16;
    const int with_vals = bytes + (int)(t * val_bytes);
    *stage_vals = (val_bytes > 0 && with_vals <= kRelocateSmemMax) ? 1 : 0;
    return *stage_vals ? with_vals : bytes;
}

cudaError_t launch_relocate(const uint32_t *tiles_k, const void *tiles_v, const uint32_t *cum,
                            const uint32_t *offsets, uint32_t t, uint32_t s, uint32_t m,
                            int val_bytes, uint32_t *reloc_k, void *reloc_v, int *err,
                            cudaStream_t st)
{
    int stage_vals = 0;
    const int sm = relocate_smem_bytes(t, s, val_bytes, &stage_vals);
    if (sm > kRelocateSmemMax) return cudaErrorInvalidValue;
    k_relocate<1024><<<m, 1024, sm, st>>>(tiles_k, tiles_v, cum, offsets, t, s, m,
                                          (uint64_t)m * t, val_bytes, stage_vals, reloc_k,
                                          reloc_v, err);
    return cudaGetLastError();
}

cudaError_t launch_pack_units(const uint32_t *offsets, uint32_t m, uint32_t s, uint32_t n_pad,
                              uint32_t Q, uint32_t *units, int *err, cudaStream_t st)
{
    const int sm = (int)(4 * (s + 1) * 4);
    k_pack_units<1024><<<1, 1024, sm, st>>>(offsets, m, s, n_pad, Q, units, err);
    return cudaGetLastError();
}

cudaError_t launch_bucket_sort(int cap, bool pairs, const void *src_k, const void *src_v,
                               const uint32_t *units, uint32_t max_units, uint64_t n,
                               uint64_t n_pad, int is_f32, int val_bytes, void *out_k,
                               void *out_v, int *err, cudaStream_t st)
{
    const int sm = smem_bytes_for_cap(cap, pairs);
    const uint32_t grid = units ? max_units : 1u;
    const uint32_t *sk = static_cast<const uint32_t *>(src_k);
    uint32_t *ok = static_cast<uint32_t *>(out_k);
#define BSORT_L9(T_, E_, P_)                                                                 \
    k_bucket_sort<T_, E_, P_><<<grid, T_, sm, st>>>(sk, src_v, units, n, n_pad, is_f32,      \
                                                    val_bytes, ok, out_v, err)
    if (!pairs) {
        switch (cap) {
        case 2048: BSORT_L9(128, 16, false); break;
        case 4096: BSORT_L9(256, 16, false); break;
        case 8192: BSORT_L9(512, 16, false); break;
        case 16384: BSORT_L9(1024, 16, false); break;
        case 32768: BSORT_L9(1024, 32, false); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (cap) {
        case 2048: BSORT_L9(128, 16, true); break;
        case 4096: BSORT_L9(256, 16, true); break;
        case 8192: BSORT_L9(512, 16, true); break;
        case 16384: BSORT_L9(1024, 16, true); break;
        default: return cudaErrorInvalidValue;
        }
    }
#undef BSORT_L9
    return cudaGetLastError();
}

}  // namespace bsort
