// bsort_batch.cu -- batched sorting of many independent arrays (segments)
// of uint32 / float32 / uint64 keys in one launch sequence.  The paper
// sorts one array (Section 4, Algorithm 1); here each segment gets the part
// of the method its size calls for:
//
//   direct segments (up to one Step-9 unit): sorted whole by one CTA or one
//     thread-block cluster, as Step 9 sorts a bucket (k_seg_sort, one launch
//     per unit shape);
//   sampled segments (larger): Algorithm 1 with segment-aware sublists,
//     samples and splitters.  Every sublist lies in one segment (the last
//     sublist of a segment is padded), every segment sorts its own m*s
//     samples and picks its own b splitters, buckets never cross segments,
//     and Step 9 writes each bucket back into its segment's output range.
//
// 64-bit keys take the same two routes with the 64-bit path's widths
// (sublists and Step-9 units of 16,384 keys, 16-byte sample records).
//
// Sublists of all sampled segments are numbered globally (g); sublist g
// occupies positions [g*t, (g+1)*t) of the padded sublist space, so the
// composite position p = g*t + r orders each segment's items by index, as
// p = i*t + r does for one array.  Runs A_ij of all segments are numbered
// segment by segment (bucket-major inside a segment), so one exclusive scan
// over all counts gives every run its place in the padded space.
#include "bsort_device.cuh"
#include "bsort_internal.h"
#include "bsort_radix.cuh"

namespace bsort {

// ============================================================ direct segments
// Cluster u sorts segment u = [seg[2u], seg[2u+1]) of the input (at most
// C*T*E keys, guaranteed by the host) into the same range of the output.
// K: uint32_t (uint32 / float32 keys) or uint64_t (64-bit keys).
template <typename K, int T, int E, int C>
__global__ void __launch_bounds__(T, 1)
k_seg_sort(const K *__restrict__ keys_in, K *__restrict__ keys_out,
           const uint32_t *__restrict__ seg, int is_f32, int *err)
{
    constexpr int CH = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t u = blockIdx.x / C;
    const int r = (int)(blockIdx.x % C);
    const uint32_t L = seg[2 * u], R = seg[2 * u + 1];
    if (R < L || R - L > (uint32_t)(C * CH)) {
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;  // uniform per cluster
    }
    const int len = (int)(R - L);
    if (len == 0) return;
    const int per = C == 1 ? CH : (len + C - 1) / C;
    const int ustart = r * per;
    const int uend = min(ustart + per, len);
    K v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = ustart + wb_pos<E>(warp, lane, k);
        K key = KeyMax<K>::v;
        if (x < uend) {
            key = keys_in[L + x];
            if constexpr (sizeof(K) == 4)
                if (is_f32) key = f32_encode(key);
        }
        v[k] = key;
    }
    cta_sort<K, T, E>(v, sm, uend > ustart ? uend - ustart : 0);
    cluster_merge<K, T, E, C>(sm, len, per);
    const int off = r * CH;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        if (off + x < len) {
            K key = sm[pidx<K>(x)];
            if constexpr (sizeof(K) == 4)
                if (is_f32) key = f32_decode(key);
            keys_out[L + off + x] = key;
        }
    }
}

// ============================================================ Steps 1-3
// CTA g sorts sublist g (kSegTile keys): items [i*t, min((i+1)*t, n)) of its
// segment, i = g - g0, padded with the maximal key; writes the sorted
// sublist to tiles[g*t ...] and its s samples (ranks (k+1)w - 1) as
// key << 32 | (g*t + rank) to the segment's record array.  The sublist is
// sorted by digits (cta_radix_sort, 7-bit digits over the bits that vary
// in it): 6.3 against 6.6 ms by comparisons for the 25,000 sublists of the
// 20,000-array workload; its buckets, whose keys span most of the 32 bits
// (few buckets per segment), sort as fast by comparisons, so Step 9 keeps
// them.
constexpr int kSegRadixBits = 7;

template <int T, int E>
__global__ void __launch_bounds__(T, 1)
k_seg_sublist_sort(const uint32_t *__restrict__ keys_in, int is_f32,
                   const uint32_t *__restrict__ sub_seg, const SegInfo *__restrict__ segs,
                   uint32_t *__restrict__ tiles_k, uint64_t *__restrict__ samples)
{
    constexpr int TT = T * E;  // t
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sm = reinterpret_cast<uint32_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t g = blockIdx.x;
    const SegInfo sg = segs[sub_seg[g]];
    const uint32_t i = g - sg.g0;
    const uint32_t first = i * (uint32_t)TT;  // item offset inside the segment
    const int len = sg.n - first < (uint32_t)TT ? (int)(sg.n - first) : TT;
    const uint64_t src = (uint64_t)sg.out + first;
    uint32_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = wb_pos<E>(warp, lane, k);
        uint32_t key = 0xFFFFFFFFu;
        if (x < len) {
            key = keys_in[src + x];
            if (is_f32) key = f32_encode(key);
        }
        v[k] = key;
    }
    cta_radix_sort<T, E, kSegRadixBits>(v, sm, len);
    const uint64_t base = (uint64_t)g * TT;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        tiles_k[base + x] = sm[pidx<uint32_t>(x)];
    }
    const uint32_t w = (uint32_t)TT / sg.s;
    uint64_t *rec = samples + sg.rec + (uint64_t)i * sg.s;
    for (uint32_t k = tid; k < sg.s; k += T) {
        const uint32_t rank = (k + 1) * w - 1;
        rec[k] = ((uint64_t)sm[pidx<uint32_t>((int)rank)] << 32) | (uint32_t)(base + rank);
    }
}

// ============================================================ Steps 4-5
// CTA q sorts the m*s sample records of sampled segment q (at most T*E;
// every sublist's s records are already a sorted run) and writes its b
// splitters g_j = S[floor((j+1) m s / b) - 1].
template <int T, int E>
__global__ void __launch_bounds__(T, 1)
k_seg_records(const uint64_t *__restrict__ samples, const SegInfo *__restrict__ segs,
              uint64_t *__restrict__ spl)
{
    constexpr int CAP = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const SegInfo sg = segs[blockIdx.x];
    const uint32_t nrec = sg.m * sg.s;
    const uint64_t *src = samples + sg.rec;
    if (sg.s >= 32u * E && sg.s < (uint32_t)CAP) {
        const int s = (int)sg.s;
        for (int x = tid; x < CAP; x += T) {
            const uint64_t r = (uint32_t)x < nrec ? src[x] : 0xFFFFFFFFFFFFFFFFull;
            const int q = x / s, o = x % s;
            const int pos = (q & 1) ? q * s + s - 1 - o : x;
            sm[pidx<uint64_t>(pos)] = r;
        }
        __syncthreads();
        cta_merge_runs<uint64_t, T, E>(sm, s);
    } else {
        uint64_t v[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const uint32_t x = (uint32_t)wb_pos<E>(warp, lane, k);
            v[k] = x < nrec ? src[x] : 0xFFFFFFFFFFFFFFFFull;
        }
        cta_sort<uint64_t, T, E>(v, sm);
    }
    for (uint32_t j = tid; j < sg.b; j += T)
        spl[sg.spl + j] = sm[pidx<uint64_t>((int)((uint64_t)(j + 1) * nrec / sg.b - 1))];
}

// ============================================================ Step 6
// CTA g locates its segment's b splitters in sorted sublist g: c_j = #items
// <= g_j (binary search over the sublist's s samples, then its w-item
// window), T splitters per round, and writes for run (j, i) of the segment
// the count a_ij = c_j - c_{j-1} and the run's first position g*t + c_{j-1}.
template <int T>
__global__ void __launch_bounds__(T)
k_seg_sample_index(const uint32_t *__restrict__ tiles_k, const uint64_t *__restrict__ samples,
                   const uint64_t *__restrict__ spl, const uint32_t *__restrict__ sub_seg,
                   const SegInfo *__restrict__ segs, uint32_t t, uint32_t *__restrict__ counts,
                   uint32_t *__restrict__ srcb)
{
    __shared__ uint32_t c[T + 1];
    const int tid = threadIdx.x;
    const uint32_t g = blockIdx.x;
    const SegInfo sg = segs[sub_seg[g]];
    const uint32_t i = g - sg.g0;
    const uint32_t s = sg.s, w = t / s;
    const uint64_t base = (uint64_t)g * t;
    const uint64_t *smp = samples + sg.rec + (uint64_t)i * s;
    const uint64_t *gs = spl + sg.spl;
    if (tid == 0) c[0] = 0;
    for (uint32_t j0 = 0; j0 < sg.b; j0 += T) {
        const uint32_t j = j0 + tid;
        uint32_t cj = t;
        if (j < sg.b) {
            const uint64_t gj = gs[j];
            uint32_t lo = 0, hi = s;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (smp[mid] <= gj) lo = mid + 1;
                else hi = mid;
            }
            cj = window_count(tiles_k, base, lo, w, t, s, gj);
        }
        c[tid + 1] = cj;
        __syncthreads();
        if (j < sg.b) {
            const uint64_t q = sg.run0 + (uint64_t)j * sg.m + i;
            counts[q] = cj - c[tid];
            srcb[q] = (uint32_t)base + c[tid];
        }
        const uint32_t carry = c[T];  // c of the round's last splitter
        __syncthreads();
        if (tid == 0) c[0] = carry;
    }
}

// ============================================================ Step 9
// CTA u sorts bucket j of sampled segment q (units[2u] = q, units[2u+1] =
// j): positions [offsets[run0 + j*m], next bucket's first position) of the
// relocated array, and writes its ranks that hold real items (position -
// g0*t < n) to the segment's output range.  K: uint32_t (uint32 / float32
// keys) or uint64_t (64-bit keys).
template <typename K, int T, int E>
__global__ void __launch_bounds__(T, 1)
k_seg_bucket_sort(const K *__restrict__ reloc_k, const uint32_t *__restrict__ units,
                  const SegInfo *__restrict__ segs, const uint32_t *__restrict__ offsets,
                  uint32_t t, int is_f32, K *__restrict__ keys_out, int *err)
{
    constexpr int CH = T * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sm = reinterpret_cast<K *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t u = blockIdx.x;
    const SegInfo sg = segs[units[2 * u]];
    const uint32_t j = units[2 * u + 1];
    const uint32_t P = sg.g0 * t;  // the segment's first padded position
    const uint32_t L = offsets[sg.run0 + j * sg.m];
    const uint32_t R = j + 1 < sg.b ? offsets[sg.run0 + (j + 1) * sg.m] : P + sg.m * t;
    if (R < L || R - L > (uint32_t)CH) {
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;
    }
    const int len = (int)(R - L);
    if (len == 0) return;
    K v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = wb_pos<E>(warp, lane, k);
        v[k] = x < len ? reloc_k[L + x] : KeyMax<K>::v;
    }
    cta_sort<K, T, E>(v, sm, len);
    // ranks below lim hold real items of the segment (its padding sorts last)
    const uint32_t rel = L - P;
    const int lim = rel >= sg.n ? 0 : (sg.n - rel < (uint32_t)len ? (int)(sg.n - rel) : len);
    const uint64_t dst = (uint64_t)sg.out + rel;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        if (x < lim) {
            K key = sm[pidx<K>(x)];
            if constexpr (sizeof(K) == 4)
                if (is_f32) key = f32_decode(key);
            keys_out[dst + x] = key;
        }
    }
}

// ============================================================ 64-bit keys
// Sampled segments of 64-bit keys take the steps above with the widths of
// the 64-bit path: sublists of kSegTileU64 keys sorted by comparisons, and
// sample records (key, p) of two 64-bit words, ordered key first, then p
// (the composite order).
__device__ __forceinline__ bool seg_rec_lt(const Rec128 &a, const Rec128 &b)
{
    return a.key < b.key || (a.key == b.key && a.p < b.p);
}

// Steps 1-3: CTA g sorts sublist g of its segment and writes the samples
// of ranks (k+1)w - 1 as (key, g*t + rank).
template <int T, int E>
__global__ void __launch_bounds__(T, 1)
k_seg_sublist_sort_u64(const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ sub_seg,
                       const SegInfo *__restrict__ segs, uint64_t *__restrict__ tiles_k,
                       Rec128 *__restrict__ samples)
{
    constexpr int TT = T * E;  // t
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t g = blockIdx.x;
    const SegInfo sg = segs[sub_seg[g]];
    const uint32_t i = g - sg.g0;
    const uint32_t first = i * (uint32_t)TT;  // item offset inside the segment
    const int len = sg.n - first < (uint32_t)TT ? (int)(sg.n - first) : TT;
    const uint64_t src = (uint64_t)sg.out + first;
    uint64_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int x = wb_pos<E>(warp, lane, k);
        v[k] = x < len ? keys_in[src + x] : KeyMax<uint64_t>::v;
    }
    cta_sort<uint64_t, T, E>(v, sm, len);
    const uint64_t base = (uint64_t)g * TT;
#pragma unroll 4
    for (int k = 0; k < E; ++k) {
        const int x = k * T + tid;
        tiles_k[base + x] = sm[pidx<uint64_t>(x)];
    }
    const uint32_t w = (uint32_t)TT / sg.s;
    Rec128 *rec = samples + sg.rec + (uint64_t)i * sg.s;
    for (uint32_t k = tid; k < sg.s; k += T) {
        const uint32_t rank = (k + 1) * w - 1;
        Rec128 r;
        r.key = sm[pidx<uint64_t>((int)rank)];
        r.p = base + rank;
        rec[k] = r;
    }
}

// Steps 4-5: CTA q ranks the N = m*s sample records of sampled segment q
// in shared memory instead of sorting them.  Every sublist's s records are
// a sorted run and no two records are equal (their positions differ), so
// the rank of a record is its index in its own run plus, for each other
// run, the number of that run's records below it (a binary search).  The
// record of rank floor((j+1) N / b) - 1 is splitter j, the same choice as
// the 32-bit path's sorted records; each rank is the splitter of at most
// one j (b <= N), namely j = ceil((rank+1) b / N) - 1 when that j maps back.
template <int T>
__global__ void __launch_bounds__(T, 1)
k_seg_records_u64(const Rec128 *__restrict__ samples, const SegInfo *__restrict__ segs,
                  Rec128 *__restrict__ spl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Rec128 *sm = reinterpret_cast<Rec128 *>(smem_raw);
    const SegInfo sg = segs[blockIdx.x];
    const uint32_t s = sg.s, N = sg.m * sg.s;
    const Rec128 *src = samples + sg.rec;
    for (uint32_t x = threadIdx.x; x < N; x += T) sm[x] = src[x];
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < N; x += T) {
        const Rec128 r = sm[x];
        const uint32_t own = x / s;
        uint64_t rank = x - own * s;
        for (uint32_t i = 0; i < sg.m; ++i) {
            if (i == own) continue;
            const Rec128 *run = sm + (uint64_t)i * s;
            uint32_t lo = 0, hi = s;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (seg_rec_lt(run[mid], r)) lo = mid + 1;
                else hi = mid;
            }
            rank += lo;
        }
        const uint64_t j = ((rank + 1) * sg.b + N - 1) / N - 1;
        if (j < sg.b && (j + 1) * N / sg.b - 1 == rank) spl[sg.spl + j] = r;
    }
}

// Step 6: CTA g locates its segment's b splitters in sorted sublist g, as
// k_seg_sample_index does: the samples at or below g_j (binary search over
// the sublist's s records) fix a window of w ranks that holds c_j, which a
// binary search over the window's items (key, g*t + rank) finds.
template <int T>
__global__ void __launch_bounds__(T)
k_seg_sample_index_u64(const uint64_t *__restrict__ tiles_k, const Rec128 *__restrict__ samples,
                       const Rec128 *__restrict__ spl, const uint32_t *__restrict__ sub_seg,
                       const SegInfo *__restrict__ segs, uint32_t t, uint32_t *__restrict__ counts,
                       uint32_t *__restrict__ srcb)
{
    __shared__ uint32_t c[T + 1];
    const int tid = threadIdx.x;
    const uint32_t g = blockIdx.x;
    const SegInfo sg = segs[sub_seg[g]];
    const uint32_t i = g - sg.g0;
    const uint32_t s = sg.s, w = t / s;
    const uint64_t base = (uint64_t)g * t;
    const Rec128 *smp = samples + sg.rec + (uint64_t)i * s;
    const Rec128 *gs = spl + sg.spl;
    if (tid == 0) c[0] = 0;
    for (uint32_t j0 = 0; j0 < sg.b; j0 += T) {
        const uint32_t j = j0 + tid;
        uint32_t cj = t;
        if (j < sg.b) {
            const Rec128 gj = gs[j];
            uint32_t lo = 0, hi = s;  // samples at or below g_j
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (!seg_rec_lt(gj, smp[mid])) lo = mid + 1;
                else hi = mid;
            }
            if (lo < s) {
                // ranks below lo*w are at or below g_j, rank (lo+1)w - 1 is above
                uint32_t a = lo * w, e = lo * w + w - 1;
                while (a < e) {
                    const uint32_t mid = (a + e) >> 1;
                    Rec128 item;
                    item.key = tiles_k[base + mid];
                    item.p = base + mid;
                    if (!seg_rec_lt(gj, item)) a = mid + 1;
                    else e = mid;
                }
                cj = a;
            }
        }
        c[tid + 1] = cj;
        __syncthreads();
        if (j < sg.b) {
            const uint64_t q = sg.run0 + (uint64_t)j * sg.m + i;
            counts[q] = cj - c[tid];
            srcb[q] = (uint32_t)base + c[tid];
        }
        const uint32_t carry = c[T];  // c of the round's last splitter
        __syncthreads();
        if (tid == 0) c[0] = carry;
    }
}

// ============================================================ launching
namespace {

template <typename KernelT>
cudaError_t set_smem_attr(KernelT k, int bytes, bool nonportable = false)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && nonportable)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename K, int T, int E, int C>
cudaError_t launch_seg_sort_t(const void *keys_in, void *keys_out, const uint32_t *seg,
                              uint32_t nseg, int is_f32, int *err, cudaStream_t st)
{
    const int sm = padded_elems<K>(T * E) * (int)sizeof(K);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nseg * C, 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = (size_t)sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_seg_sort<K, T, E, C>, static_cast<const K *>(keys_in),
                              static_cast<K *>(keys_out), seg, is_f32, err);
}

template <typename K, int T, int E, int C>
cudaError_t init_seg_sort_t()
{
    return set_smem_attr(k_seg_sort<K, T, E, C>, padded_elems<K>(T * E) * (int)sizeof(K));
}

}  // namespace

namespace {
int g_wide16 = -1;  // the 16-CTA 64-bit shape: -1 not asked yet, 0 no, 1 yes
}  // namespace

// Asked once per process, on the current device (no device: no).
bool batch_wide_cluster16()
{
    if (g_wide16 < 0) {
        // non-portable cluster size: usable only if the device schedules it
        const int sm = padded_elems<uint64_t>(16384) * 8;
        int n = 0;
        cudaError_t q = set_smem_attr(k_seg_sort<uint64_t, 1024, 16, 16>, sm, true);
        if (q == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16, 1, 1);
            cfg.blockDim = dim3(1024, 1, 1);
            cfg.dynamicSmemBytes = (size_t)sm;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 16;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            q = cudaOccupancyMaxActiveClusters(&n, k_seg_sort<uint64_t, 1024, 16, 16>, &cfg);
        }
        if (q != cudaSuccess) cudaGetLastError();  // (not an error: the shape is left out)
        g_wide16 = q == cudaSuccess && n >= 1 ? 1 : 0;
    }
    return g_wide16 == 1;
}

cudaError_t init_batch_kernels()
{
    cudaError_t e = cudaSuccess;
    batch_wide_cluster16();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 128, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 256, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 512, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 1024, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 1024, 32, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 1024, 32, 2>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 1024, 32, 4>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint32_t, 1024, 32, 8>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 128, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 256, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 512, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 1024, 16, 1>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 1024, 16, 2>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 1024, 16, 4>();
    if (e == cudaSuccess) e = init_seg_sort_t<uint64_t, 1024, 16, 8>();
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_sublist_sort<256, 128>, RadixSmem<256, 128, kSegRadixBits>::kBytes);
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_records<1024, 16>, padded_elems<uint64_t>(kRecordChunk) * 8);
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_bucket_sort<uint32_t, 1024, 16>,
                          padded_elems<uint32_t>(16384) * 4);
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_bucket_sort<uint32_t, 1024, 32>,
                          padded_elems<uint32_t>(32768) * 4);
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_sublist_sort_u64<1024, 16>,
                          padded_elems<uint64_t>(kSegTileU64) * 8);
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_records_u64<1024>, (int)(kSegRecordsU64 * sizeof(Rec128)));
    if (e == cudaSuccess)
        e = set_smem_attr(k_seg_bucket_sort<uint64_t, 1024, 16>,
                          padded_elems<uint64_t>(kSegTileU64) * 8);
    return e;
}

cudaError_t launch_seg_sort(int chunk, int ctas, bool wide, const void *keys_in, void *keys_out,
                            const uint32_t *seg, uint32_t nseg, int is_f32, int *err,
                            cudaStream_t st)
{
    if (nseg == 0) return cudaSuccess;
#define L(K_, T_, E_, C_) \
    return launch_seg_sort_t<K_, T_, E_, C_>(keys_in, keys_out, seg, nseg, is_f32, err, st)
    if (wide) {
        if (ctas == 1) {
            switch (chunk) {
            case 2048: L(uint64_t, 128, 16, 1);
            case 4096: L(uint64_t, 256, 16, 1);
            case 8192: L(uint64_t, 512, 16, 1);
            case 16384: L(uint64_t, 1024, 16, 1);
            }
        } else if (chunk == 16384) {
            switch (ctas) {
            case 2: L(uint64_t, 1024, 16, 2);
            case 4: L(uint64_t, 1024, 16, 4);
            case 8: L(uint64_t, 1024, 16, 8);
            case 16:
                if (!batch_wide_cluster16()) return cudaErrorInvalidValue;
                L(uint64_t, 1024, 16, 16);
            }
        }
        return cudaErrorInvalidValue;
    }
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(uint32_t, 128, 16, 1);
        case 4096: L(uint32_t, 256, 16, 1);
        case 8192: L(uint32_t, 512, 16, 1);
        case 16384: L(uint32_t, 1024, 16, 1);
        case 32768: L(uint32_t, 1024, 32, 1);
        }
    } else if (chunk == 32768) {
        switch (ctas) {
        case 2: L(uint32_t, 1024, 32, 2);
        case 4: L(uint32_t, 1024, 32, 4);
        case 8: L(uint32_t, 1024, 32, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_seg_sublist_sort(const uint32_t *keys_in, int is_f32, const uint32_t *sub_seg,
                                    uint32_t nsub, const SegInfo *segs, uint32_t *tiles_k,
                                    uint64_t *samples, cudaStream_t st)
{
    if (nsub == 0) return cudaSuccess;
    static_assert(kSegTile == 256 * 128, "a sublist is one radix CTA's unit");
    const int sm = RadixSmem<256, 128, kSegRadixBits>::kBytes;
    k_seg_sublist_sort<256, 128><<<nsub, 256, sm, st>>>(keys_in, is_f32, sub_seg, segs, tiles_k,
                                                        samples);
    return cudaGetLastError();
}

cudaError_t launch_seg_records(const uint64_t *samples, const SegInfo *segs, uint32_t nsegs,
                               uint64_t *spl, cudaStream_t st)
{
    if (nsegs == 0) return cudaSuccess;
    const int sm = padded_elems<uint64_t>(kRecordChunk) * 8;
    k_seg_records<1024, 16><<<nsegs, 1024, sm, st>>>(samples, segs, spl);
    return cudaGetLastError();
}

cudaError_t launch_seg_sample_index(const uint32_t *tiles_k, const uint64_t *samples,
                                    const uint64_t *spl, const uint32_t *sub_seg, uint32_t nsub,
                                    const SegInfo *segs, uint32_t *counts, uint32_t *srcb,
                                    cudaStream_t st)
{
    if (nsub == 0) return cudaSuccess;
    k_seg_sample_index<128><<<nsub, 128, 0, st>>>(tiles_k, samples, spl, sub_seg, segs,
                                                  (uint32_t)kSegTile, counts, srcb);
    return cudaGetLastError();
}

cudaError_t launch_seg_bucket_sort(int chunk, const uint32_t *reloc_k, const uint32_t *units,
                                   uint32_t nunits, const SegInfo *segs, const uint32_t *offsets,
                                   int is_f32, uint32_t *keys_out, int *err, cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    if (chunk == 16384) {
        k_seg_bucket_sort<uint32_t, 1024, 16>
            <<<nunits, 1024, padded_elems<uint32_t>(16384) * 4, st>>>(
                reloc_k, units, segs, offsets, (uint32_t)kSegTile, is_f32, keys_out, err);
    } else if (chunk == 32768) {
        k_seg_bucket_sort<uint32_t, 1024, 32>
            <<<nunits, 1024, padded_elems<uint32_t>(32768) * 4, st>>>(
                reloc_k, units, segs, offsets, (uint32_t)kSegTile, is_f32, keys_out, err);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seg_sublist_sort_u64(const uint64_t *keys_in, const uint32_t *sub_seg,
                                        uint32_t nsub, const SegInfo *segs, uint64_t *tiles_k,
                                        Rec128 *samples, cudaStream_t st)
{
    if (nsub == 0) return cudaSuccess;
    static_assert(kSegTileU64 == 1024 * 16, "a sublist is one CTA's unit");
    k_seg_sublist_sort_u64<1024, 16><<<nsub, 1024, padded_elems<uint64_t>(kSegTileU64) * 8, st>>>(
        keys_in, sub_seg, segs, tiles_k, samples);
    return cudaGetLastError();
}

cudaError_t launch_seg_records_u64(const Rec128 *samples, const SegInfo *segs, uint32_t nsegs,
                                   Rec128 *spl, cudaStream_t st)
{
    if (nsegs == 0) return cudaSuccess;
    k_seg_records_u64<1024><<<nsegs, 1024, kSegRecordsU64 * sizeof(Rec128), st>>>(samples, segs,
                                                                                  spl);
    return cudaGetLastError();
}

cudaError_t launch_seg_sample_index_u64(const uint64_t *tiles_k, const Rec128 *samples,
                                        const Rec128 *spl, const uint32_t *sub_seg,
                                        uint32_t nsub, const SegInfo *segs, uint32_t *counts,
                                        uint32_t *srcb, cudaStream_t st)
{
    if (nsub == 0) return cudaSuccess;
    k_seg_sample_index_u64<128><<<nsub, 128, 0, st>>>(tiles_k, samples, spl, sub_seg, segs,
                                                      (uint32_t)kSegTileU64, counts, srcb);
    return cudaGetLastError();
}

cudaError_t launch_seg_bucket_sort_u64(const uint64_t *reloc_k, const uint32_t *units,
                                       uint32_t nunits, const SegInfo *segs,
                                       const uint32_t *offsets, uint64_t *keys_out, int *err,
                                       cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    k_seg_bucket_sort<uint64_t, 1024, 16>
        <<<nunits, 1024, padded_elems<uint64_t>(kSegTileU64) * 8, st>>>(
            reloc_k, units, segs, offsets, (uint32_t)kSegTileU64, 0, keys_out, err);
    return cudaGetLastError();
}

}  // namespace bsort
