// bsort_device.cuh -- device building blocks of GPU Bucket Sort on sm_103a.
//
// The comparison sort used inside one CTA (Algorithm 1, Step 2 "local sort"
// and Step 9 "sublist sort") is built in three layers:
//   1. every thread sorts E keys in registers with Batcher's odd-even merge
//      network (compare-exchange = one min and one max instruction);
//   2. runs are merged pairwise in shared memory with merge-path partitioning
//      (each thread finds its split by binary search along its diagonal and
//      merges E outputs into registers), log2(T) levels;
//   3. the sorted tile is read back from shared memory in a coalesced order.
// Shared memory holds T*E keys in a padded layout (one spare word per 32
// 4-byte words) so that the blocked register<->SMEM transfers are free of
// bank conflicts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bsort {

// ---------------------------------------------------------------- error word
enum DevErr : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 4,   // matches BSORT_ETIMEOUT
    DEV_INTERNAL = 8   // matches BSORT_EINTERNAL
};

__device__ __forceinline__ void set_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- key codecs
// Order-preserving map of binary32 bits to uint32 (negative: invert all bits;
// non-negative: set the sign bit), and its inverse.
__device__ __forceinline__ uint32_t f32_encode(uint32_t b)
{
    uint32_t mask = (uint32_t)((int32_t)b >> 31) | 0x80000000u;
    return b ^ mask;
}

__device__ __forceinline__ uint32_t f32_decode(uint32_t u)
{
    uint32_t mask = (u & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu;
    return u ^ mask;
}

template <typename K> struct KeyMax;
template <> struct KeyMax<uint32_t> { static constexpr uint32_t v = 0xFFFFFFFFu; };
template <> struct KeyMax<uint64_t> { static constexpr uint64_t v = 0xFFFFFFFFFFFFFFFFull; };

// Padded shared-memory index: one spare slot per 128 bytes.
template <typename K>
__device__ __forceinline__ int pidx(int x)
{
    return sizeof(K) == 4 ? x + (x >> 5) : x + (x >> 4);
}

template <typename K>
__host__ __device__ constexpr int padded_elems(int cap)
{
    return sizeof(K) == 4 ? cap + (cap >> 5) + 1 : cap + (cap >> 4) + 1;
}

// ---------------------------------------------------------------- register sort
template <typename K>
__device__ __forceinline__ void cmp_swap(K &a, K &b)
{
    K lo = a < b ? a : b;
    K hi = a < b ? b : a;
    a = lo;
    b = hi;
}

template <>
__device__ __forceinline__ void cmp_swap<uint32_t>(uint32_t &a, uint32_t &b)
{
    uint32_t lo = min(a, b);
    uint32_t hi = max(a, b);
    a = lo;
    b = hi;
}

// Batcher's odd-even merge sort network on E (power of two) registers.
template <int E, typename K>
__device__ __forceinline__ void sort_network(K (&v)[E])
{
#pragma unroll
    for (int p = 1; p < E; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
#pragma unroll
            for (int j = k % p; j + k < E; j += 2 * k) {
#pragma unroll
                for (int i = 0; i < k; ++i) {
                    if (i + j + k < E && (i + j) / (2 * p) == (i + j + k) / (2 * p))
                        cmp_swap(v[i + j], v[i + j + k]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- merge path
// Number of items of run A among the first d outputs of the stable merge of
// A (length la, at sm index a0) and B (length lb, at b0): smallest i with
// A[i] > B[d-1-i].  Ties go to A.
template <typename K>
__device__ __forceinline__ int merge_path_smem(const K *sm, int a0, int la, int b0,
                                               int lb, int d)
{
    int lo = d > lb ? d - lb : 0;
    int hi = d < la ? d : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        K am = sm[pidx<K>(a0 + mid)];
        K bm = sm[pidx<K>(b0 + d - 1 - mid)];
        if (am <= bm) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Serial merge of E outputs starting at split (i, j) of runs A, B into v.
// MAY_EXHAUST: the caller may ask for more outputs than la + lb - (i + j)
// (the extra outputs are garbage); every load index is then clamped into
// [a0, a0 + la) / [b0, b0 + lb) or to a0 for an empty run.
template <typename K, int E, bool MAY_EXHAUST = false>
__device__ __forceinline__ void merge_serial_smem(const K *sm, int a0, int la, int b0,
                                                  int lb, int i, int j, K (&v)[E])
{
    K a = sm[pidx<K>(a0 + max(min(i, la - 1), 0))];
    K b = sm[pidx<K>(b0 + max(min(j, lb - 1), 0))];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        bool take_a = (j >= lb) || ((i < la) && (a <= b));
        v[k] = take_a ? a : b;
        int ni = i + (take_a ? 1 : 0);
        int nj = j + (take_a ? 0 : 1);
        int idx;
        if (MAY_EXHAUST)
            idx = take_a ? (a0 + max(min(ni, la - 1), 0)) : (b0 + max(min(nj, lb - 1), 0));
        else
            idx = take_a ? (a0 + min(ni, la - 1)) : (b0 + min(nj, lb - 1));
        K nxt = sm[pidx<K>(idx)];
        a = take_a ? nxt : a;
        b = take_a ? b : nxt;
        i = ni;
        j = nj;
    }
}

// Sort T*E keys held E per thread (any assignment of keys to threads) into
// shared memory sm (padded layout).  On return sm[pidx(x)] is the x-th
// smallest key and v holds positions [tid*E, tid*E + E) of the sorted tile.
template <typename K, int T, int E>
__device__ __forceinline__ void cta_sort(K (&v)[E], K *sm)
{
    const int tid = threadIdx.x;
    sort_network<E>(v);
#pragma unroll
    for (int k = 0; k < E; ++k) sm[pidx<K>(tid * E + k)] = v[k];
    __syncthreads();
#pragma unroll 1
    for (int L = E; L < T * E; L <<= 1) {
        const int dg = tid * E;
        const int a0 = dg & ~(2 * L - 1);
        const int d = dg - a0;
        const int b0 = a0 + L;
        int i = merge_path_smem<K>(sm, a0, L, b0, L, d);
        merge_serial_smem<K, E>(sm, a0, L, b0, L, i, d - i, v);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < E; ++k) sm[pidx<K>(tid * E + k)] = v[k];
        __syncthreads();
    }
}

}  // namespace bsort
