// bsort_u64.cu -- GPU Bucket Sort (Dehne & Zaboli, Section 4, Algorithm 1)
// for 64-bit keys, keys only.  The steps are those of the 32-bit path; what
// changes is the width of what they move:
//
//   sorted sublists and buckets hold 64-bit keys (a CTA sorts 16,384 of
//     them; clusters of 2, 4, 8 CTAs for larger units);
//   a sample record is the pair (key, p), p = i*t + r, stored as two 64-bit
//     words (16 bytes), compared key first, then p (the composite order);
//   Step 4 merges the m sorted runs of s records (one per sublist) in
//     log2(m) merge-path passes through L2 instead of sorting chunks in SMEM.
#include "bsort_device.cuh"
#include "bsort_internal.h"
#include "bsort_sort.cuh"

namespace bsort {

__device__ __forceinline__ bool rec_lt(const Rec128 &a, const Rec128 &b)
{
    return a.key < b.key || (a.key == b.key && a.p < b.p);
}

// ============================================================ Steps 1-3
// Cluster i sorts sublist i (t = C*T*E keys) and emits the samples of its
// ranks, as k_sublist_sort does for 32-bit keys.
template <int T, int E, int C>
__global__ void __launch_bounds__(T, 1)
k_sublist_sort_u64(const uint64_t *__restrict__ keys_in, uint64_t n, uint32_t s,
                   uint64_t *__restrict__ tiles_k, Rec128 *__restrict__ samples)
{
    constexpr int CH = T * E;
    constexpr uint32_t TT = (uint32_t)C * CH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = blockIdx.x / C;
    const int r = (int)(blockIdx.x % C);
    const uint64_t base = (uint64_t)tile * TT;
    const uint64_t avail = n > base ? n - base : 0;
    const int len = avail < (uint64_t)TT ? (int)avail : (int)TT;
    const int off = r * CH;
    uint64_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = off + wb_pos<E>(warp, lane, k);
        v[k] = x < len ? keys_in[base + x] : 0xFFFFFFFFFFFFFFFFull;
    }
    const int clen = len - off;
    cta_sort<uint64_t, T, E>(v, sm, clen < 0 ? 0 : (clen > CH ? CH : clen));
    cluster_merge<uint64_t, T, E, C>(sm, len);
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        tiles_k[base + off + x] = sm[pidx<uint64_t>(x)];
    }
    const uint32_t w = TT / s;
    const uint32_t k0 = (uint32_t)off / w;
    const uint32_t k1 = (uint32_t)(off + CH) / w;
    for (uint32_t k = k0 + tid; k < k1 && k < s; k += T) {
        const uint32_t rank = (k + 1) * w - 1;
        Rec128 rec;
        rec.key = sm[pidx<uint64_t>((int)(rank - off))];
        rec.p = base + rank;
        samples[(uint64_t)tile * s + k] = rec;
    }
}

// ============================================================ Step 4
// One merge-path pass: runs of length L of src (N records) merged pairwise
// into runs of 2L in dst.  Thread x writes outputs [x*IT, (x+1)*IT).
template <int T, int IT>
__global__ void __launch_bounds__(T)
k_rec_merge(const Rec128 *__restrict__ src, Rec128 *__restrict__ dst, uint32_t N, uint32_t L)
{
    const uint64_t o = ((uint64_t)blockIdx.x * T + threadIdx.x) * IT;
    if (o >= N) return;
    const uint64_t a0 = o / (2ull * L) * (2ull * L);
    const uint32_t la = (uint32_t)min((uint64_t)L, N - a0);
    const uint32_t lb = a0 + L < N ? (uint32_t)min((uint64_t)L, N - a0 - L) : 0u;
    const Rec128 *A = src + a0;
    const Rec128 *B = A + la;
    const uint32_t d = (uint32_t)(o - a0);
    // co-rank: i items of A among the first d outputs (A first on ties)
    uint32_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (rec_lt(B[d - 1 - mid], A[mid])) hi = mid;
        else lo = mid + 1;
    }
    uint32_t i = lo, j = d - lo;
    const uint32_t end = min(d + (uint32_t)IT, la + lb);  // d < la + lb since o < N
    for (uint32_t x = d; x < end; ++x) {
        const bool takeA = j >= lb || (i < la && !rec_lt(B[j], A[i]));
        dst[a0 + x] = takeA ? A[i++] : B[j++];
    }
}

// The same merge by tiles, when a pair of runs spans whole tiles (2L a
// multiple of T*E): one CTA produces T*E outputs.  A warp finds the tile's
// co-ranks by a 32-ary search in global memory, the CTA stages its A and B
// ranges in shared memory with coalesced loads (all issued before the first
// store), each thread merges E outputs there, and the tile goes back
// through shared memory with coalesced stores.
__device__ __forceinline__ uint32_t rec_corank_warp(const Rec128 *A, uint32_t la, const Rec128 *B,
                                                    uint32_t lb, uint32_t d, int lane)
{
    // i = A items among the first d outputs: the first c in [lo, hi] with
    // B[d-1-c] < A[c] (false ... true on [lo, hi)), hi if none
    uint32_t lo = d > lb ? d - lb : 0;
    uint32_t hi = d < la ? d : la;
    while (hi - lo > 32) {
        const uint32_t span = hi - lo;
        const uint32_t c = lo + (uint32_t)(((uint64_t)span * (lane + 1)) / 33);
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, rec_lt(B[d - 1 - c], A[c]));
        if (ball == 0) {
            lo = lo + (uint32_t)(((uint64_t)span * 32) / 33) + 1;
        } else {
            const int f = __ffs(ball) - 1;
            const uint32_t cf = lo + (uint32_t)(((uint64_t)span * (f + 1)) / 33);
            const uint32_t cp = f ? lo + (uint32_t)(((uint64_t)span * f) / 33) + 1 : lo;
            lo = cp;
            hi = cf;
        }
    }
    const uint32_t c = lo + lane;
    const bool pred = c < hi ? rec_lt(B[d - 1 - c], A[c]) : true;
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
    return ball ? lo + (uint32_t)(__ffs(ball) - 1) : hi;
}

template <int T, int E>
__global__ void __launch_bounds__(T)
k_rec_merge_tiled(const Rec128 *__restrict__ src, Rec128 *__restrict__ dst, uint32_t N,
                  uint32_t L)
{
    constexpr int TILE = T * E;
    __shared__ Rec128 sm[TILE];
    __shared__ uint32_t s_split[2];
    const int tid = threadIdx.x;
    const uint64_t o0 = (uint64_t)blockIdx.x * TILE;
    const uint64_t a0 = o0 / (2ull * L) * (2ull * L);
    const uint32_t la = (uint32_t)min((uint64_t)L, (uint64_t)N - a0);
    const uint32_t lb = a0 + L < N ? (uint32_t)min((uint64_t)L, (uint64_t)N - a0 - L) : 0u;
    const Rec128 *A = src + a0;
    const Rec128 *B = A + la;
    const uint32_t d0 = (uint32_t)(o0 - a0);
    const uint32_t d1 = min(d0 + (uint32_t)TILE, la + lb);
    if (tid < 64) {
        const uint32_t dd = tid < 32 ? d0 : d1;
        const uint32_t r = rec_corank_warp(A, la, B, lb, dd, tid & 31);
        if ((tid & 31) == 0) s_split[tid >> 5] = r;
    }
    __syncthreads();
    const uint32_t i0 = s_split[0], i1 = s_split[1];
    const int na = (int)(i1 - i0), cnt = (int)(d1 - d0);
    const int nb = cnt - na;
    const uint32_t j0 = d0 - i0;
    {
        Rec128 r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            if (x < na) r[k] = A[i0 + x];
            else if (x < cnt) r[k] = B[j0 + (x - na)];
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            if (x < cnt) sm[x] = r[k];
        }
    }
    __syncthreads();
    // thread t: outputs [tE, tE + E) of the tile, A = sm[0, na), B = sm[na, cnt)
    const int d = tid * E;
    Rec128 v[E];
    if (d < cnt) {
        int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rec_lt(sm[na + d - 1 - mid], sm[mid])) hi = mid;
            else lo = mid + 1;
        }
        int i = lo, j = d - lo;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const bool takeA = j >= nb || (i < na && !rec_lt(sm[na + j], sm[i]));
            // an exhausted run is never read: indices stay in [0, cnt)
            v[k] = takeA ? sm[min(i, cnt - 1)] : sm[na + min(j, nb - 1)];
            i += takeA ? 1 : 0;
            j += takeA ? 0 : 1;
        }
    }
    __syncthreads();
    if (d < cnt) {
#pragma unroll
        for (int k = 0; k < E; ++k)
            if (d + k < cnt) sm[d + k] = v[k];
    }
    __syncthreads();
    for (int x = tid; x < cnt; x += T) dst[o0 + x] = sm[x];
}

// ============================================================ Step 5
__global__ void k_select_splitters_u64(const Rec128 *__restrict__ sorted, uint32_t N, uint32_t b,
                                       Rec128 *__restrict__ spl)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < b) spl[j] = sorted[(uint64_t)(j + 1) * N / b - 1];
}

// ============================================================ Step 6 (segments)
// As the 32-bit path's Step 6: c_ij = items of sorted sublist i at or below
// splitter j in (key, position) order, found in the segment of the sublist
// that holds it.  Segments of 4096 keys (32 KB of shared memory); the first
// splitter of segment [S, S + seg) is the number of splitters below item
// S - 1.  Writes the cumulative c_ij bucket-major (Step 7 forms a_ij).
constexpr int kSegItemsU64 = 4096;

__global__ void k_seg_ranges_u64(const uint64_t *__restrict__ tiles, const Rec128 *__restrict__ spl,
                                 uint32_t t, uint32_t b, uint32_t m, uint32_t nseg, uint32_t seg,
                                 uint32_t *__restrict__ jr)
{
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * nseg) return;
    const uint32_t i = idx / nseg, k = idx % nseg;
    uint32_t r = 0;
    if (k > 0) {
        Rec128 v;
        v.p = (uint64_t)i * t + (uint64_t)k * seg - 1;  // item S - 1 of sublist i
        v.key = tiles[v.p];
        uint32_t lo = 0, hi = b;
        while (lo < hi) {  // splitters below v
            const uint32_t mid = (lo + hi) >> 1;
            if (rec_lt(spl[mid], v)) lo = mid + 1;
            else hi = mid;
        }
        r = lo;
    }
    jr[idx] = r;
}

template <int T>
__global__ void __launch_bounds__(T)
k_sample_index_seg_u64(const uint64_t *__restrict__ tiles, const Rec128 *__restrict__ spl,
                       uint32_t t, uint32_t b, uint32_t m, uint32_t nseg, uint32_t seg,
                       const uint32_t *__restrict__ jr, uint32_t *__restrict__ cum)
{
    static_assert(kSegItemsU64 % (2 * T) == 0, "whole uint4 loads per thread");
    __shared__ __align__(16) uint64_t sk[kSegItemsU64];
    const uint32_t i = blockIdx.x / nseg, k = blockIdx.x % nseg;
    const uint32_t S = k * seg;
    const uint64_t p0 = (uint64_t)i * t + S;  // position of the segment's first item
    const uint32_t j_lo = jr[blockIdx.x];
    const uint32_t j_hi = k + 1 < nseg ? jr[blockIdx.x + 1] : b;
    const uint4 *src = reinterpret_cast<const uint4 *>(tiles + p0);
    uint4 *dst = reinterpret_cast<uint4 *>(sk);
    constexpr int Q = kSegItemsU64 / 2 / T;  // all loads before the first store
    uint4 r[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t v = (uint32_t)(q * T) + threadIdx.x;
        if (v < seg / 2) r[q] = src[v];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t v = (uint32_t)(q * T) + threadIdx.x;
        if (v < seg / 2) dst[v] = r[q];
    }
    __syncthreads();
    for (uint32_t j = j_lo + threadIdx.x; j < j_hi; j += T) {
        const Rec128 g = spl[j];
        uint32_t lo = 0, hi = seg;
        while (lo < hi) {  // segment items <= g
            const uint32_t mid = (lo + hi) >> 1;
            Rec128 item;
            item.key = sk[mid];
            item.p = p0 + mid;
            if (!rec_lt(g, item)) lo = mid + 1;
            else hi = mid;
        }
        cum[(uint64_t)j * m + i] = S + lo;
    }
}

// ============================================================ Step 9
// Cluster u sorts unit u = [units[1+2u], units[2+2u]) of the relocated
// array (or, with units == nullptr, the whole input [0, n)) and writes the
// positions below n.
template <int T, int E, int C>
__device__ __forceinline__ void
bucket_sort_unit_u64(uint32_t u, const uint64_t *__restrict__ src,
                     const uint32_t *__restrict__ units, uint64_t n, uint64_t n_pad,
                     uint64_t *__restrict__ out, int *err)
{
    constexpr int CH = T * E;
    constexpr uint64_t CAP = (uint64_t)C * CH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r = (int)(blockIdx.x % C);
    uint64_t L = 0, R = n;
    if (units != nullptr) {
        if (u >= units[0]) return;
        L = units[1 + 2 * u];
        R = units[2 + 2 * u];
    }
    if (R < L || R > n_pad || R - L > CAP) {
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;
    }
    if (R == L) return;
    const int len = (int)(R - L);
    const int per = C == 1 ? CH : (len + C - 1) / C;
    const int ustart = r * per;
    const int uend = min(ustart + per, len);
    uint64_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = ustart + wb_pos<E>(warp, lane, k);
        v[k] = x < uend ? src[L + x] : 0xFFFFFFFFFFFFFFFFull;
    }
    cta_sort<uint64_t, T, E>(v, sm, uend > ustart ? uend - ustart : 0);
    cluster_merge<uint64_t, T, E, C>(sm, len, per);
    const int off = r * CH;
    const uint64_t lim64 = min((unsigned long long)len, (unsigned long long)(n > L ? n - L : 0));
    const int lim = (int)lim64;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        if (off + x < lim) out[L + off + x] = sm[pidx<uint64_t>(x)];
    }
}

template <int T, int E, int C>
__global__ void __launch_bounds__(T, 1)
k_bucket_sort_u64(const uint64_t *__restrict__ src, const uint32_t *__restrict__ units,
                  uint64_t n, uint64_t n_pad, uint64_t *__restrict__ out, int *err)
{
    bucket_sort_unit_u64<T, E, C>(blockIdx.x / C, src, units, n, n_pad, out, err);
}

// Cluster c of a small grid sorts units c, c + G, ... of a device-sized list.
template <int T, int E, int C>
__global__ void __launch_bounds__(T, 1)
k_bucket_sort_u64_loop(const uint64_t *__restrict__ src, const uint32_t *__restrict__ units,
                       uint64_t n, uint64_t n_pad, uint64_t *__restrict__ out, int *err)
{
    const uint32_t count = units[0];
#pragma unroll 1
    for (uint32_t u = blockIdx.x / C; u < count; u += gridDim.x / C) {
        bucket_sort_unit_u64<T, E, C>(u, src, units, n, n_pad, out, err);
        __syncthreads();  // shared memory is reused by the next unit
    }
}

// ============================================================ launching
namespace {

template <int T, int E, int C>
cudaError_t init_u64_t()
{
    const int sm = padded_elems<uint64_t>(T * E) * 8;
    cudaError_t e = cudaFuncSetAttribute(k_sublist_sort_u64<T, E, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bucket_sort_u64<T, E, C>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess && C > 1)
        e = cudaFuncSetAttribute(k_bucket_sort_u64_loop<T, E, C>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

template <int T, int E, int C>
cudaError_t launch_sublist_u64_t(const void *keys_in, uint64_t n, uint32_t m, uint32_t s,
                                 uint64_t *tiles, Rec128 *samples, cudaStream_t st)
{
    const int sm = padded_elems<uint64_t>(T * E) * 8;
    return launch_maybe_cluster(k_sublist_sort_u64<T, E, C>, m * C, T, sm, C, st,
                                static_cast<const uint64_t *>(keys_in), n, s, tiles, samples);
}

template <int T, int E, int C>
cudaError_t launch_bucket_u64_t(const void *src, const uint32_t *units, uint32_t max_units,
                                uint64_t n, uint64_t n_pad, void *out, int *err, cudaStream_t st)
{
    const int sm = padded_elems<uint64_t>(T * E) * 8;
    const unsigned grid = (units ? max_units : 1u) * C;
    if (C > 1 && units != nullptr && max_units <= kLoopUnits)
        return launch_maybe_cluster(k_bucket_sort_u64_loop<T, E, C>, grid, T, sm, C, st,
                                    static_cast<const uint64_t *>(src), units, n, n_pad,
                                    static_cast<uint64_t *>(out), err);
    return launch_maybe_cluster(k_bucket_sort_u64<T, E, C>, grid, T, sm, C, st,
                                static_cast<const uint64_t *>(src), units, n, n_pad,
                                static_cast<uint64_t *>(out), err);
}

}  // namespace

cudaError_t init_u64_kernels()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = init_u64_t<128, 16, 1>();
    if (e == cudaSuccess) e = init_u64_t<256, 16, 1>();
    if (e == cudaSuccess) e = init_u64_t<512, 16, 1>();
    if (e == cudaSuccess) e = init_u64_t<1024, 16, 1>();
    if (e == cudaSuccess) e = init_u64_t<1024, 16, 2>();
    if (e == cudaSuccess) e = init_u64_t<1024, 16, 4>();
    if (e == cudaSuccess) e = init_u64_t<1024, 16, 8>();
    return e;
}

cudaError_t launch_sublist_sort_u64(int chunk, int ctas, const void *keys_in, uint64_t n,
                                    uint32_t m, uint32_t s, uint64_t *tiles, Rec128 *samples,
                                    cudaStream_t st)
{
#define L(T_, E_, C_) return launch_sublist_u64_t<T_, E_, C_>(keys_in, n, m, s, tiles, samples, st)
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(128, 16, 1);
        case 4096: L(256, 16, 1);
        case 8192: L(512, 16, 1);
        case 16384: L(1024, 16, 1);
        }
    } else if (chunk == 16384) {
        switch (ctas) {
        case 2: L(1024, 16, 2);
        case 4: L(1024, 16, 4);
        case 8: L(1024, 16, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_sort_u64(int chunk, int ctas, const void *src, const uint32_t *units,
                                   uint32_t max_units, uint64_t n, uint64_t n_pad, void *out,
                                   int *err, cudaStream_t st)
{
#define L(T_, E_, C_) \
    return launch_bucket_u64_t<T_, E_, C_>(src, units, max_units, n, n_pad, out, err, st)
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(128, 16, 1);
        case 4096: L(256, 16, 1);
        case 8192: L(512, 16, 1);
        case 16384: L(1024, 16, 1);
        }
    } else if (chunk == 16384) {
        switch (ctas) {
        case 2: L(1024, 16, 2);
        case 4: L(1024, 16, 4);
        case 8: L(1024, 16, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_rec_merge(const Rec128 *src, Rec128 *dst, uint32_t N, uint32_t L,
                             cudaStream_t st)
{
    constexpr int T = 256, IT = 8;
    const uint32_t grid = (uint32_t)(((uint64_t)N + T * IT - 1) / (T * IT));
    if ((2ull * L) % (T * IT) == 0) {  // pairs of runs span whole tiles
        k_rec_merge_tiled<T, IT><<<grid, T, 0, st>>>(src, dst, N, L);
        return cudaGetLastError();
    }
    k_rec_merge<T, IT><<<grid, T, 0, st>>>(src, dst, N, L);
    return cudaGetLastError();
}

cudaError_t launch_select_splitters_u64(const Rec128 *sorted, uint32_t N, uint32_t b, Rec128 *spl,
                                        cudaStream_t st)
{
    k_select_splitters_u64<<<(b + 255) / 256, 256, 0, st>>>(sorted, N, b, spl);
    return cudaGetLastError();
}


cudaError_t launch_sample_index_seg_u64(const uint64_t *tiles, const Rec128 *spl, uint32_t t,
                                        uint32_t b, uint32_t m, uint32_t *jr, uint32_t *cum,
                                        cudaStream_t st)
{
    const uint32_t seg = t < (uint32_t)kSegItemsU64 ? t : (uint32_t)kSegItemsU64;
    const uint32_t nseg = t / seg;
    const uint32_t ns = m * nseg;
    k_seg_ranges_u64<<<(ns + 255) / 256, 256, 0, st>>>(tiles, spl, t, b, m, nseg, seg, jr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sample_index_seg_u64<256><<<ns, 256, 0, st>>>(tiles, spl, t, b, m, nseg, seg, jr, cum);
    return cudaGetLastError();
}

}  // namespace bsort
