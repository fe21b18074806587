// bsort_sort.cuh -- the two sorting kernels of GPU Bucket Sort (Dehne &
// Zaboli, Section 4, Algorithm 1): Steps 1-3 (sort every sublist, take its
// samples) and Step 9 (sort every bucket).  Both sort one unit of C*T*E
// items with a thread-block cluster of C CTAs: every CTA sorts a chunk of
// T*E items in shared memory (cta_sort), then the cluster merges the chunks
// through distributed shared memory (cluster_merge).  C = 1 is a plain CTA.
//
// Keys-only units sort uint32 keys; pair units sort the 64-bit words
// key << 32 | position-in-unit, which makes the order stable, and gather
// each value from its position afterwards.
#pragma once

#include "bsort_device.cuh"
#include "bsort_internal.h"
#include "bsort_radix.cuh"

namespace bsort {

// Digit width of the radix-sorting CTAs (128 digits per pass).
constexpr int kRadixBits = 7;

// Dynamic shared memory of one sorting CTA: the padded tile, plus the radix
// sort's counters when the CTA sorts 32-bit keys by digits (RADIX).
template <typename K, int T, int E, bool RADIX>
constexpr int sort_smem_bytes()
{
    return RADIX ? RadixSmem<T, E, kRadixBits>::kBytes : padded_elems<K>(T * E) * (int)sizeof(K);
}

// The in-CTA sort of one chunk: the comparison sort (cta_sort) or, for
// 32-bit keys, the radix sort (cta_radix_sort); both leave the same result.
template <typename K, int T, int E, bool RADIX>
__device__ __forceinline__ void chunk_sort(K (&v)[E], K *sm, int len)
{
    if constexpr (RADIX) {
        static_assert(sizeof(K) == 4, "the radix sort takes 32-bit keys");
        cta_radix_sort<T, E, kRadixBits>(v, sm, len);
    } else {
        cta_sort<K, T, E>(v, sm, len);
    }
}

// ============================================================ Steps 1-3
// Cluster c sorts sublist i = tile0 + c (t = C*T*E items); CTA r loads positions
// [r*T*E, (r+1)*T*E) of the sublist and, after the merge, holds its ranks
// [r*T*E, (r+1)*T*E): it writes them to the sorted-sublist array and emits
// the samples (ranks (k+1)w - 1) that fall in that range as key << 32 | p,
// p = i*t + r.
template <int T, int E, bool PAIRS, int C, bool RADIX = false>
__global__ void __launch_bounds__(T, 1)
k_sublist_sort(const uint32_t *__restrict__ keys_in, const void *__restrict__ vals_in,
               uint64_t n, int is_f32, int val_bytes, uint32_t s,
               uint32_t *__restrict__ tiles_k, void *__restrict__ tiles_v,
               uint64_t *__restrict__ samples, uint32_t tile0)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    constexpr int CH = T * E;
    constexpr uint32_t TT = (uint32_t)C * CH;  // sublist size t
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = tile0 + blockIdx.x / C;
    const int r = (int)(blockIdx.x % C);
    const uint64_t base = (uint64_t)tile * TT;
    const uint64_t avail = n > base ? n - base : 0;  // real items of the sublist
    const int len = avail < (uint64_t)TT ? (int)avail : (int)TT;
    const int off = r * CH;  // this CTA's chunk in the sublist
    if (tid == 0) {  // the same chunk of the sublist this SM will most likely sort next
        const uint64_t nb = base + (uint64_t)(num_sms() / C) * TT + off;
        if (nb < n) prefetch_l2(keys_in + nb, 4 * min((uint64_t)CH, n - nb));
    }

    K v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = off + wb_pos<E>(warp, lane, k);
        uint32_t key = 0xFFFFFFFFu;  // pad sentinel (position >= n)
        if (x < len) {
            key = keys_in[base + x];
            if (is_f32) key = f32_encode(key);
        }
        if constexpr (PAIRS) v[k] = ((uint64_t)key << 32) | (uint32_t)x;
        else v[k] = (K)key;
    }
    const int clen = len - off;
    chunk_sort<K, T, E, RADIX>(v, sm, clen < 0 ? 0 : (clen > CH ? CH : clen));
    cluster_merge<K, T, E, C>(sm, len);

#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        const K e = sm[pidx<K>(x)];
        if constexpr (PAIRS) {
            const uint32_t idx = (uint32_t)(e & 0xFFFFFFFFull);
            tiles_k[base + off + x] = (uint32_t)((uint64_t)e >> 32);
            if (val_bytes == 4) {
                uint32_t val = (uint64_t)idx < avail
                                   ? static_cast<const uint32_t *>(vals_in)[base + idx] : 0u;
                static_cast<uint32_t *>(tiles_v)[base + off + x] = val;
            } else {
                uint64_t val = (uint64_t)idx < avail
                                   ? static_cast<const uint64_t *>(vals_in)[base + idx] : 0ull;
                static_cast<uint64_t *>(tiles_v)[base + off + x] = val;
            }
        } else {
            tiles_k[base + off + x] = (uint32_t)e;
        }
    }
    // Step 3: samples at ranks (k+1)w - 1 in [off, off + CH), as the record
    // key << 32 | q with q = i*s + k, the sample's index: its position
    // p = i*t + (k+1)w - 1 grows with q, so records order by (key, q) exactly
    // as by (key, p), and q fits 32 bits whatever the size of the input.
    const uint32_t w = TT / s;
    const uint32_t k0 = (uint32_t)off / w;                // first sample in range
    const uint32_t k1 = (uint32_t)(off + CH) / w;         // one past the last
    for (uint32_t k = k0 + tid; k < k1 && k < s; k += T) {
        const uint32_t rank = (k + 1) * w - 1;
        const K e = sm[pidx<K>((int)(rank - off))];
        const uint32_t key = PAIRS ? (uint32_t)((uint64_t)e >> 32) : (uint32_t)e;
        samples[(uint64_t)tile * s + k] = ((uint64_t)key << 32) | (tile * s + k);
    }
}

// ============================================================ Step 9
// A cluster sorts unit u = [units[1+2u], units[2+2u]) of the relocated order
// (consecutive whole buckets, at most C*T*E items) and writes the positions
// below n of the result.  With units == nullptr there is one unit, [0, n),
// read from the caller's input (raw keys, transformed on load).
//
// The unit's items are read either from a materialised relocated array
// (src_k / src_v) or, when g.offsets != nullptr, gathered straight from the
// sorted sublists (Step 8 fused into this load): every lane walks the
// bucket-major runs as its position grows.  Pair units then sort
// key << 32 | (position in the sorted-sublist array), which orders equal
// keys by original index exactly as the relocated order does, and fetch
// each value from that position.
// prefetch_stride: units between this one and the next this CTA's SM will
// most likely sort (0: no prefetch), whose keys are then fetched into L2.
template <int T, int E, bool PAIRS, int C, bool RADIX>
__device__ __forceinline__ void
bucket_sort_unit(uint32_t u, const uint32_t *__restrict__ src_k, const void *__restrict__ src_v,
                 const uint32_t *__restrict__ units, uint64_t n, uint64_t n_pad, int is_f32,
                 int val_bytes, uint32_t *__restrict__ out_k, void *__restrict__ out_v,
                 int *err, const GatherSrc &g, uint32_t prefetch_stride)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    constexpr int CH = T * E;
    constexpr uint64_t CAP = (uint64_t)C * CH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r = (int)(blockIdx.x % C);
    const bool direct = units == nullptr;
    const bool gather = g.offsets != nullptr;
    uint64_t L = 0, R = n;
    if (!direct) {
        if (u >= units[0]) return;  // fewer units than clusters (uniform per cluster)
        L = units[1 + 2 * u];
        R = units[2 + 2 * u];
    }
    const uint64_t len64 = R - L;
    if (R < L || R > n_pad || len64 > CAP) {  // the plan guarantees a unit fits
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;  // uniform per cluster: no CTA of it reaches a cluster barrier
    }
    if (len64 == 0) return;
    if (!direct && !gather && tid == 0 && r == 0 && prefetch_stride) {
        // the unit this SM will most likely sort next
        const uint32_t un = u + prefetch_stride;
        if (un < units[0]) {
            const uint32_t pl = units[1 + 2 * un], pr = units[2 + 2 * un];
            if (pl < pr && pr <= n_pad) prefetch_l2(src_k + pl, 4ull * (pr - pl));
        }
    }
    const int len = (int)len64;
    const int off = r * CH;  // ranks of the sorted unit this CTA writes
    // the unit's real items are spread evenly over the cluster's CTAs, so
    // that padding (skipped by whole warps) is shared by all of them
    const int per = C == 1 ? CH : (len + C - 1) / C;
    const int ustart = r * per;
    const int uend = min(ustart + per, len);
    K v[E];
    if (!gather) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = ustart + wb_pos<E>(warp, lane, k);
            uint32_t key = 0xFFFFFFFFu;
            uint32_t idx = 0xFFFFFFFFu;  // pads sort after every real item
            if (x < uend) {
                key = src_k[L + x];
                if (direct && is_f32) key = f32_encode(key);
                idx = (uint32_t)x;
            }
            if constexpr (PAIRS) v[k] = ((uint64_t)key << 32) | idx;
            else v[k] = (K)key;
        }
    } else {
        // lane's first position, and the run containing it: search the runs
        // of its block and the next (positions of a warp span < 2 blocks)
        const uint32_t y0 = (uint32_t)(L + ustart + wb_pos<E>(warp, lane, 0));
        uint32_t q = 0;
        const uint32_t nblk = (uint32_t)((n_pad + kBlockItems - 1) / kBlockItems);
        if (ustart + wb_pos<E>(warp, 0, 0) < uend) {  // the warp holds real items
            const uint32_t wy = (uint32_t)(L + ustart + wb_pos<E>(warp, 0, 0));
            const uint32_t b = wy / (uint32_t)kBlockItems;  // < nblk since wy < R <= n_pad
            uint32_t lo = g.blk[b];
            uint32_t hi = b + 2 < nblk ? g.blk[b + 2] : g.runs - 1;
            while (lo < hi) {  // last q with offsets[q] <= y0
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (g.offsets[mid] <= y0) lo = mid;
                else hi = mid - 1;
            }
            q = lo;
        }
        uint32_t rs = g.offsets[q], re = g.offsets[q + 1];
        uint32_t base = g.srcb[q];  // position of run q's first item
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = ustart + wb_pos<E>(warp, lane, k);
            const uint32_t y = y0 + 32u * (uint32_t)k;
            uint32_t key = 0xFFFFFFFFu;
            uint32_t pos = 0xFFFFFFFFu;  // pads sort after every real item
            if (x < uend) {
                if (y >= re) {
                    run_advance<kBlockItems>(g.offsets, g.blk, nblk, g.runs, y, q, rs, re);
                    base = g.srcb[q];
                }
                pos = base + (y - rs);
                key = src_k[pos];
            }
            if constexpr (PAIRS) v[k] = ((uint64_t)key << 32) | pos;
            else v[k] = (K)key;
        }
    }
    chunk_sort<K, T, E, RADIX>(v, sm, uend > ustart ? uend - ustart : 0);
    cluster_merge<K, T, E, C>(sm, len, per);
    const uint64_t lim64 = min((unsigned long long)len, (unsigned long long)(n > L ? n - L : 0));
    const int lim = (int)lim64;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        if (off + x < lim) {
            const K e = sm[pidx<K>(x)];
            uint32_t key = PAIRS ? (uint32_t)((uint64_t)e >> 32) : (uint32_t)e;
            if (is_f32) key = f32_decode(key);
            out_k[L + off + x] = key;
            if constexpr (PAIRS) {
                const uint32_t idx = (uint32_t)((uint64_t)e & 0xFFFFFFFFull);
                const uint64_t from = gather ? (uint64_t)idx : L + idx;
                if (val_bytes == 4)
                    static_cast<uint32_t *>(out_v)[L + off + x] =
                        static_cast<const uint32_t *>(src_v)[from];
                else
                    static_cast<uint64_t *>(out_v)[L + off + x] =
                        static_cast<const uint64_t *>(src_v)[from];
            }
        }
    }
}

// Cluster u of the grid sorts unit u (clusters beyond the unit count exit).
template <int T, int E, bool PAIRS, int C, bool RADIX = false>
__global__ void __launch_bounds__(T, 1)
k_bucket_sort(const uint32_t *__restrict__ src_k, const void *__restrict__ src_v,
              const uint32_t *__restrict__ units, uint64_t n, uint64_t n_pad, int is_f32,
              int val_bytes, uint32_t *__restrict__ out_k, void *__restrict__ out_v, int *err,
              GatherSrc g)
{
    bucket_sort_unit<T, E, PAIRS, C, RADIX>(blockIdx.x / C, src_k, src_v, units, n, n_pad, is_f32,
                                     val_bytes, out_k, out_v, err, g, num_sms() / C);
}

// The same for a unit list whose length only the device knows (the cluster
// tier of a two-tier Step 9, mostly empty, or a range of units given in
// device memory, range[0] .. range[1] - 1): a small grid whose cluster c
// sorts units lo + c, lo + c + G, ... (G clusters; every CTA of a cluster
// takes the same units).
template <int T, int E, bool PAIRS, int C, bool RADIX = false>
__global__ void __launch_bounds__(T, 1)
k_bucket_sort_loop(const uint32_t *__restrict__ src_k, const void *__restrict__ src_v,
                   const uint32_t *__restrict__ units, uint64_t n, uint64_t n_pad, int is_f32,
                   int val_bytes, uint32_t *__restrict__ out_k, void *__restrict__ out_v,
                   int *err, GatherSrc g, const uint32_t *__restrict__ range)
{
    const uint32_t lo = range != nullptr ? range[0] : 0u;
    const uint32_t count = range != nullptr ? range[1] : units[0];
#pragma unroll 1
    for (uint32_t u = lo + blockIdx.x / C; u < count; u += gridDim.x / C) {
        bucket_sort_unit<T, E, PAIRS, C, RADIX>(u, src_k, src_v, units, n, n_pad, is_f32, val_bytes,
                                         out_k, out_v, err, g, gridDim.x / C);
        __syncthreads();  // shared memory is reused by the next unit
    }
}

// ============================================================ launching
template <typename KernelT, typename... Args>
inline cudaError_t launch_maybe_cluster(KernelT kern, unsigned grid, int block, int smem,
                                        int csize, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = csize > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int T, int E, bool PAIRS, int C, bool RADIX = false>
inline cudaError_t init_sort_pair_of_kernels()
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    const int sm = sort_smem_bytes<K, T, E, RADIX>();
    cudaError_t e = cudaFuncSetAttribute(k_sublist_sort<T, E, PAIRS, C, RADIX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_bucket_sort<T, E, PAIRS, C, RADIX>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_bucket_sort_loop<T, E, PAIRS, C, RADIX>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(k_sublist_sort<T, E, PAIRS, C, RADIX>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_bucket_sort<T, E, PAIRS, C, RADIX>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    return e;
}

template <int T, int E, bool PAIRS, int C, bool RADIX = false>
inline cudaError_t launch_sublist_sort_t(const void *keys_in, const void *vals_in, uint64_t n,
                                         uint32_t m, int is_f32, int val_bytes, uint32_t s,
                                         uint32_t *tiles_k, void *tiles_v, uint64_t *samples,
                                         uint32_t tile0, cudaStream_t st)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    const int sm = sort_smem_bytes<K, T, E, RADIX>();
    return launch_maybe_cluster(k_sublist_sort<T, E, PAIRS, C, RADIX>, m * C, T, sm, C, st,
                                static_cast<const uint32_t *>(keys_in), vals_in, n, is_f32,
                                val_bytes, s, tiles_k, tiles_v, samples, tile0);
}

template <int T, int E, bool PAIRS, int C, bool RADIX = false>
inline cudaError_t launch_bucket_sort_t(const void *src_k, const void *src_v,
                                        const uint32_t *units, uint32_t max_units, uint64_t n,
                                        uint64_t n_pad, int is_f32, int val_bytes, void *out_k,
                                        void *out_v, int *err, const GatherSrc &g,
                                        cudaStream_t st)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    const int sm = sort_smem_bytes<K, T, E, RADIX>();
    const unsigned grid = (units ? max_units : 1u) * C;
    if (C > 1 && units != nullptr && max_units <= kLoopUnits)
        return launch_maybe_cluster(k_bucket_sort_loop<T, E, PAIRS, C, RADIX>, grid, T, sm, C, st,
                                    static_cast<const uint32_t *>(src_k), src_v, units, n, n_pad,
                                    is_f32, val_bytes, static_cast<uint32_t *>(out_k), out_v,
                                    err, g, (const uint32_t *)nullptr);
    return launch_maybe_cluster(k_bucket_sort<T, E, PAIRS, C, RADIX>, grid, T, sm, C, st,
                                static_cast<const uint32_t *>(src_k), src_v, units, n, n_pad,
                                is_f32, val_bytes, static_cast<uint32_t *>(out_k), out_v, err, g);
}

// Step 9 over the units range[0] .. range[1] - 1 of a list (device memory),
// by a grid of grid_units clusters (C > 1) or of grid_units SMs' worth of
// CTAs (C = 1) that loop over them.
template <int T, int E, bool PAIRS, int C, bool RADIX = false>
inline cudaError_t launch_bucket_sort_range_t(const void *src_k, const uint32_t *units,
                                              const uint32_t *range, uint32_t grid_units,
                                              uint64_t n, uint64_t n_pad, int is_f32,
                                              void *out_k, int *err, cudaStream_t st)
{
    using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
    const int sm = sort_smem_bytes<K, T, E, RADIX>();
    const GatherSrc none;
    if (C == 1) {
        // grid_units counts SMs: as many CTAs as fit on them at once
        static const int per_sm = [sm] {
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &o, k_bucket_sort_loop<T, E, PAIRS, C, RADIX>, T, sm) != cudaSuccess)
                o = 1;
            return o < 1 ? 1 : o;
        }();
        grid_units *= (uint32_t)per_sm;
    }
    return launch_maybe_cluster(k_bucket_sort_loop<T, E, PAIRS, C, RADIX>, grid_units * C, T, sm, C, st,
                                static_cast<const uint32_t *>(src_k), (const void *)nullptr, units,
                                n, n_pad, is_f32, 0, static_cast<uint32_t *>(out_k),
                                (void *)nullptr, err, none, range);
}

}  // namespace bsort
