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
#include <type_traits>
#include <utility>

#include <cooperative_groups.h>
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

// ---------------------------------------------------------------- L2 prefetch
// Number of SMs of this GPU (the %nsmid special register).
__device__ __forceinline__ uint32_t num_sms()
{
    uint32_t n;
    asm("mov.u32 %0, %%nsmid;" : "=r"(n));
    return n;
}

// Ask the L2 to fetch the 16-byte-aligned interior of [p, p + bytes) (a
// hint: nothing is written, nothing outside the range is touched).  The
// sorting kernels issue it for the unit the SM will most likely take next,
// so that its keys stream from HBM while the current unit sorts in shared
// memory.
__device__ __forceinline__ void prefetch_l2(const void *p, uint64_t bytes)
{
    const uint64_t a = reinterpret_cast<uint64_t>(p);
    const uint64_t lo = (a + 15) & ~15ull;
    const uint64_t hi = (a + bytes) & ~15ull;
    for (uint64_t x = lo; x < hi; x += (1u << 20)) {
        const uint32_t len = (uint32_t)(hi - x < (1u << 20) ? hi - x : (1u << 20));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(x), "r"(len) : "memory");
    }
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

// Batcher's odd-even merge sort network on E (power of two) registers,
// expanded at compile time (p: merged run size, k: comparator distance,
// j: block start, i: offset in block) so that every register index is a
// constant.
template <int E, int P, int K, int J, int I, typename KT>
__device__ __forceinline__ void oem_ce(KT (&v)[E])
{
    if constexpr (I + J + K < E && (I + J) / (2 * P) == (I + J + K) / (2 * P))
        cmp_swap(v[I + J], v[I + J + K]);
}
template <int E, int P, int K, int J, typename KT, int... I>
__device__ __forceinline__ void oem_i(KT (&v)[E], std::integer_sequence<int, I...>)
{
    (oem_ce<E, P, K, J, I>(v), ...);
}
template <int E, int P, int K, int J, typename KT>
__device__ __forceinline__ void oem_j(KT (&v)[E])
{
    if constexpr (J + K < E) {
        oem_i<E, P, K, J>(v, std::make_integer_sequence<int, K>{});
        oem_j<E, P, K, J + 2 * K>(v);
    }
}
template <int E, int P, int K, typename KT>
__device__ __forceinline__ void oem_k(KT (&v)[E])
{
    if constexpr (K >= 1) {
        oem_j<E, P, K, K % P>(v);
        oem_k<E, P, K / 2>(v);
    }
}
template <int E, int P, typename KT>
__device__ __forceinline__ void oem_p(KT (&v)[E])
{
    if constexpr (P < E) {
        oem_k<E, P, P>(v);
        oem_p<E, 2 * P>(v);
    }
}
template <int E, typename K>
__device__ __forceinline__ void sort_network(K (&v)[E])
{
    oem_p<E, 1>(v);
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

// ---------------------------------------------------------------- warp merges
template <typename K>
__device__ __forceinline__ K kmin(K a, K b) { return a < b ? a : b; }
template <typename K>
__device__ __forceinline__ K kmax(K a, K b) { return a < b ? b : a; }
template <>
__device__ __forceinline__ uint32_t kmin<uint32_t>(uint32_t a, uint32_t b) { return min(a, b); }
template <>
__device__ __forceinline__ uint32_t kmax<uint32_t>(uint32_t a, uint32_t b) { return max(a, b); }

// Bitonic merge network across the lanes of a warp.  On entry every lane
// holds E keys sorted ascending; on exit the warp holds 32*E keys sorted
// ascending in blocked order (lane l holds ranks [l*E, l*E + E)).  Level l
// merges runs of 2^(l-1) lanes: one "flip" stage (element x against
// element 2M-1-x), half-cleaners at lane distances 2^(l-2)..1 (shuffles),
// then half-cleaners at register distances E/2..1.
template <typename K, int E>
__device__ __forceinline__ void warp_merge_levels(K (&v)[E], int lane)
{
#pragma unroll
    for (int l = 1; l <= 5; ++l) {
        const int fm = (1 << l) - 1;
        const bool lo_f = (lane & (1 << (l - 1))) == 0;
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            K x1 = __shfl_xor_sync(0xFFFFFFFFu, v[E - 1 - k], fm);
            K x2 = __shfl_xor_sync(0xFFFFFFFFu, v[k], fm);
            v[k] = lo_f ? kmin(v[k], x1) : kmax(v[k], x1);
            v[E - 1 - k] = lo_f ? kmin(v[E - 1 - k], x2) : kmax(v[E - 1 - k], x2);
        }
#pragma unroll
        for (int d = (1 << l) >> 2; d >= 1; d >>= 1) {
            const bool lo = (lane & d) == 0;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                K x = __shfl_xor_sync(0xFFFFFFFFu, v[k], d);
                v[k] = lo ? kmin(v[k], x) : kmax(v[k], x);
            }
        }
#pragma unroll
        for (int h = E / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int k = 0; k < E; ++k)
                if ((k & h) == 0) cmp_swap(v[k], v[k + h]);
        }
    }
}

// ---------------------------------------------------------------- block merges
// Runs of one block level alternate direction: run q is stored ascending if
// q is even and descending if q is odd, so every pair (A ascending, B
// descending) is a bitonic sequence.  A thread producing outputs [d, d+E) of
// the merge walks A upwards and B "downwards in storage" from its co-rank:
// the two pointers converge and never cross, so no bounds checks are needed
// (an exhausted run's pointer reads the other run's extreme element, which
// never wins a comparison it should lose).
template <typename K>
__device__ __forceinline__ int corank_bitonic(const K *sm, int a0, int bend, int L, int d)
{
    // number of A items among the first d outputs; A = sm[a0 .. a0+L)
    // ascending, B = sm[bend-L .. bend) descending (B[j] at bend-1-j)
    int lo = d > L ? d - L : 0;
    int hi = d < L ? d : L;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const K am = sm[pidx<K>(a0 + mid)];
        const K bm = sm[pidx<K>(bend - d + mid)];  // B[d-1-mid]
        if (am <= bm) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename K, int E>
__device__ __forceinline__ void merge_bitonic_pair(const K *sm, int ia, int ib, K (&v)[E])
{
    // ia: storage index of the next A item (moving up);
    // ib: storage index of the next B item (moving down)
    K a = sm[pidx<K>(ia)];
    K b = sm[pidx<K>(ib)];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const bool p = a <= b;
        v[k] = p ? a : b;
        if (k + 1 < E) {
            ia += p ? 1 : 0;
            ib -= p ? 0 : 1;
            const K nxt = sm[pidx<K>(p ? ia : ib)];
            a = p ? nxt : a;
            b = p ? b : nxt;
        }
    }
}

// Store E keys (ranks [r, r+E) of a run of length RL stored at base) in
// the run's direction.
template <typename K, int E>
__device__ __forceinline__ void store_run(K *sm, int base, int RL, int r, bool desc,
                                          const K (&v)[E])
{
    if (!desc) {
#pragma unroll
        for (int k = 0; k < E; ++k) sm[pidx<K>(base + r + k)] = v[k];
    } else {
#pragma unroll
        for (int k = 0; k < E; ++k) sm[pidx<K>(base + RL - 1 - r - k)] = v[k];
    }
}

// Number of A items among the first d outputs of the merge of A = sm[0..la)
// ascending with B stored descending at sm[la .. la+lb) (B[j] at
// la + lb - 1 - j): the unequal-length form of corank_bitonic.
template <typename K>
__device__ __forceinline__ int corank_bitonic_gen(const K *sm, int la, int lb, int d)
{
    const int end = la + lb;
    int lo = d > lb ? d - lb : 0;
    int hi = d < la ? d : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const K am = sm[pidx<K>(mid)];
        const K bm = sm[pidx<K>(end - d + mid)];  // B[d-1-mid]
        if (am <= bm) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Outputs [d, d + E) of the merge of A = sm[0 .. la) ascending with B
// stored descending at sm[la .. la + lb), as S independent merges of E/S
// outputs each (each from its own co-rank), advanced in lockstep so that
// their shared-memory loads overlap: a thread with many outputs and few
// warps beside it is otherwise bound by one long chain of dependent loads.
template <typename K, int E, int S>
__device__ __forceinline__ void merge_bitonic_split(const K *sm, int la, int lb, int d,
                                                    K (&v)[E])
{
    static_assert(E % S == 0, "S divides E");
    constexpr int P = E / S;
    const int end = la + lb;
    int ia[S], ib[S];
    K a[S], b[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int dq = d + q * P;
        const int i = corank_bitonic_gen<K>(sm, la, lb, dq);
        ia[q] = i;
        ib[q] = end - 1 - (dq - i);
        a[q] = sm[pidx<K>(ia[q])];
        b[q] = sm[pidx<K>(ib[q])];
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
            const bool p = a[q] <= b[q];
            v[q * P + k] = p ? a[q] : b[q];
            if (k + 1 < P) {
                ia[q] += p ? 1 : 0;
                ib[q] -= p ? 0 : 1;
                const K nxt = sm[pidx<K>(p ? ia[q] : ib[q])];
                a[q] = p ? nxt : a[q];
                b[q] = p ? b[q] : nxt;
            }
        }
    }
}

// Position of register k of thread (warp, lane) in the CTA's tile under the
// "warp-blocked" layout: warp w owns the contiguous chunk [w*32E, (w+1)*32E)
// and lane l its items l, l+32, l+64, ... of that chunk, so that global
// loads are coalesced and padding (items >= len) fills whole trailing warps.
template <int E>
__device__ __forceinline__ int wb_pos(int warp, int lane, int k)
{
    return warp * (32 * E) + k * 32 + lane;
}

// Sort T*E keys held E per thread into shared memory sm (padded layout),
// ascending.  Items at tile positions >= len are padding holding the
// maximal key (the caller loads them that way, in the warp-blocked layout);
// warps and merge pairs made only of padding skip their work.  On return
// sm[pidx(x)] is the x-th smallest key.
template <typename K, int T, int E>
__device__ __forceinline__ void cta_sort(K (&v)[E], K *sm, int len = T * E)
{
    static_assert(T % 32 == 0 && T >= 32, "whole warps");
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int W = 32 * E;  // warp run
    if (warp * W < len) {
        sort_network<E>(v);
        warp_merge_levels<K, E>(v, lane);
    }
    store_run<K, E>(sm, warp * W, W, lane * E, (warp & 1) != 0, v);
    __syncthreads();
#pragma unroll 1
    for (int L = W; L < T * E; L <<= 1) {
        const int dg = tid * E;
        const int a0 = dg & ~(2 * L - 1);  // start of the pair
        const bool work = a0 < len;
        if (work) {
            const int d = dg - a0;
            const int bend = a0 + 2 * L;
            const int i = corank_bitonic<K>(sm, a0, bend, L, d);
            merge_bitonic_pair<K, E>(sm, a0 + i, bend - 1 - (d - i), v);
        }
        __syncthreads();
        if (work) {
            const bool desc = ((a0 / (2 * L)) & 1) != 0;
            store_run<K, E>(sm, a0, 2 * L, dg - a0, desc, v);
        }
        __syncthreads();
    }
}

// The same sort when the tile already consists of sorted runs of length R
// (R a power of two, 32*E <= R < T*E) stored in sm with run q ascending if q
// is even and descending if q is odd: only the block levels from R run.
template <typename K, int T, int E>
__device__ __forceinline__ void cta_merge_runs(K *sm, int R)
{
    const int tid = threadIdx.x;
    K v[E];
#pragma unroll 1
    for (int L = R; L < T * E; L <<= 1) {
        const int dg = tid * E;
        const int a0 = dg & ~(2 * L - 1);
        const int d = dg - a0;
        const int bend = a0 + 2 * L;
        const int i = corank_bitonic<K>(sm, a0, bend, L, d);
        merge_bitonic_pair<K, E>(sm, a0 + i, bend - 1 - (d - i), v);
        __syncthreads();
        const bool desc = ((a0 / (2 * L)) & 1) != 0;
        store_run<K, E>(sm, a0, 2 * L, d, desc, v);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- cluster merges
// C CTAs of a thread-block cluster each hold a sorted chunk of `chunk` items
// (ascending, padded layout).  log2(C) rounds of pairwise merges through
// distributed shared memory leave CTA r holding ranks [r*chunk, (r+1)*chunk)
// of the cluster's items.  In the round with groups of G CTAs, the first G/2
// CTAs of a group hold run A and the rest run B; CTA r finds the co-ranks of
// its output range by a 32-ary search over the remote chunks, gathers the
// A and B pieces into registers (each piece spans at most two chunks, read
// through distributed shared memory with ordinary loads so that many are in
// flight at once), waits for the whole cluster, stores them as a bitonic
// sequence in its own SMEM, and merges locally.
__device__ __forceinline__ uint32_t smem_u32addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Generic pointer to CTA `rank`'s copy of the shared array sm (distributed
// shared memory).  Loads through it are ordinary loads: the compiler keeps
// many in flight, and the cluster barriers order them.
template <typename K>
__device__ __forceinline__ const K *cluster_ptr(K *sm, int rank)
{
    return cooperative_groups::this_cluster().map_shared_rank(sm, (unsigned)rank);
}

// Item x of the run held by CTAs first_cta, first_cta+1, ... (chunks of
// 2^chunk_shift items), read through distributed shared memory.
template <typename K>
__device__ __forceinline__ K cl_load(K *sm, int first_cta, int chunk_shift, int x)
{
    const int cta = first_cta + (x >> chunk_shift);
    const int off = x & ((1 << chunk_shift) - 1);
    return cluster_ptr(sm, cta)[pidx<K>(off)];
}

template <typename K>
__device__ __forceinline__ int corank_cluster(K *sm, int a_cta, int b_cta, int chunk_shift,
                                              int la, int lb, int d, int lane)
{
    int lo = d > lb ? d - lb : 0;
    int hi = d < la ? d : la;
    while (hi - lo > 32) {
        const int span = hi - lo;
        const int c = lo + (int)(((long long)span * (lane + 1)) / 33);
        const bool pred = cl_load<K>(sm, a_cta, chunk_shift, c) >
                          cl_load<K>(sm, b_cta, chunk_shift, d - 1 - c);
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
        if (ball == 0) {
            lo = lo + (int)(((long long)span * 32) / 33) + 1;
        } else {
            const int f = __ffs(ball) - 1;
            const int cf = lo + (int)(((long long)span * (f + 1)) / 33);
            const int cp = f ? lo + (int)(((long long)span * f) / 33) + 1 : lo;
            lo = cp;
            hi = cf;
        }
    }
    const int c = lo + lane;
    bool pred = true;
    if (c < hi)
        pred = cl_load<K>(sm, a_cta, chunk_shift, c) >
               cl_load<K>(sm, b_cta, chunk_shift, d - 1 - c);
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
    return ball ? lo + __ffs(ball) - 1 : hi;
}

// One contiguous piece [x0, ...) of a run held by CTAs first_cta, ...: at
// most two chunks.  Item z of the piece is at p0[pidx(off0 + z)] for
// z < split, else at p1[pidx(z - split)] (p0, p1: the two chunks, clamped to
// the cluster; a chunk the piece does not reach is never read).
template <typename K>
struct Piece {
    const K *p0, *p1;
    int off0, split;
};

template <typename K, int C>
__device__ __forceinline__ Piece<K> make_piece(K *sm, int first_cta, int chunk_shift, int x0)
{
    const int c0 = first_cta + (x0 >> chunk_shift);
    Piece<K> p;
    p.off0 = x0 & ((1 << chunk_shift) - 1);
    p.split = (1 << chunk_shift) - p.off0;
    p.p0 = cluster_ptr(sm, c0 < C ? c0 : C - 1);
    p.p1 = cluster_ptr(sm, c0 + 1 < C ? c0 + 1 : C - 1);
    return p;
}

template <typename K>
__device__ __forceinline__ const K *piece_addr(const Piece<K> &pc, int z)
{
    return z < pc.split ? pc.p0 + pidx<K>(pc.off0 + z) : pc.p1 + pidx<K>(z - pc.split);
}

// len: number of real items of the whole cluster; before the first round
// CTA r holds the real items [r*per, min((r+1)*per, len)) followed by
// padding (the maximal key), so a group of CTAs starting at g0 holds real
// items iff g0*per < len, and groups made only of padding skip their work.
template <typename K, int T, int E, int C>
__device__ __forceinline__ void cluster_merge(K *sm, int len, int per = T * E)
{
    if constexpr (C > 1) {
        constexpr int CH = T * E;
        constexpr int SH = __builtin_ctz(CH);
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        const int r = (int)cl.block_rank();
        const int tid = threadIdx.x;
        const int lane = tid & 31, warp = tid >> 5;
        __shared__ int s_split[2];
#pragma unroll 1
        for (int G = 2; G <= C; G <<= 1) {
            cl.sync();  // every chunk of the previous round is final
            const int g0 = r & ~(G - 1);
            const int h = G / 2;
            const bool work = g0 * per < len;
            K v[E];
            int na = 0;
            if (work) {
                const int d0 = (r - g0) * CH;
                if (warp < 2) {
                    const int i = corank_cluster<K>(sm, g0, g0 + h, SH, h * CH, h * CH,
                                                    d0 + warp * CH, lane);
                    if (lane == 0) s_split[warp] = i;
                }
                __syncthreads();
                const int i0 = s_split[0], i1 = s_split[1];
                const int j0 = d0 - i0;
                na = i1 - i0;
                const Piece<K> pa = make_piece<K, C>(sm, g0, SH, i0);
                const Piece<K> pb = make_piece<K, C>(sm, g0 + h, SH, j0);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int z = k * T + tid;
                    v[k] = *(z < na ? piece_addr(pa, z) : piece_addr(pb, z - na));
                }
            }
            cl.sync();  // all reads of this round are done
            if (work) {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int z = k * T + tid;
                    const int pos = z < na ? z : CH - 1 - (z - na);
                    sm[pidx<K>(pos)] = v[k];
                }
                __syncthreads();
                const int d = tid * E;
                if constexpr (E > 32) {
                    merge_bitonic_split<K, E, E / 32>(sm, na, CH - na, d, v);
                } else {
                    const int i = corank_bitonic_gen<K>(sm, na, CH - na, d);
                    merge_bitonic_pair<K, E>(sm, i, CH - 1 - (d - i), v);
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < E; ++k) sm[pidx<K>(d + k)] = v[k];
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------- run walking
// The runs of the relocated order are position ranges [offsets[q],
// offsets[q+1]) (offsets[runs] = n_pad), often short and sometimes long
// stretches of empty ones; blk[b] is the run holding position b*BI.  A
// walker at position y in run q with re = offsets[q+1] <= y steps over up to
// kRunSteps runs one by one, then finds the run holding y (< n_pad) by a
// binary search bounded by y's block.
constexpr int kRunSteps = 4;

template <int BI>
__device__ __forceinline__ void run_advance(const uint32_t *__restrict__ offsets,
                                            const uint32_t *__restrict__ blk, uint32_t nblk,
                                            uint32_t runs, uint32_t y, uint32_t &q,
                                            uint32_t &rs, uint32_t &re)
{
    int steps = 0;
    do {
        ++q;
        rs = re;
        re = offsets[q + 1];
    } while (y >= re && ++steps < kRunSteps);
    if (y < re) return;
    // offsets[q + 1] <= y: the run holding y is after q
    const uint32_t b = y / (uint32_t)BI;
    uint32_t lo = max(q + 1, blk[b]);
    uint32_t hi = b + 1 < nblk ? blk[b + 1] : runs - 1;
    while (lo < hi) {  // last run with offsets[run] <= y
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= y) lo = mid;
        else hi = mid - 1;
    }
    q = lo;
    rs = offsets[q];
    re = offsets[q + 1];
}

// ---------------------------------------------------------------- Step 6 window
// c = #items of the sorted sublist at base (t items) that are <= g in
// composite order (key << 32 | position), given q = #samples <= g (sample k
// is rank (k+1)w - 1): c lies in [q*w, q*w + w - 1] and only that window of
// w items is read.
__device__ __forceinline__ uint32_t window_count(const uint32_t *__restrict__ tiles_k,
                                                 uint64_t base, uint32_t q, uint32_t w,
                                                 uint32_t t, uint32_t s, uint64_t g)
{
    if (q >= s) return t;
    const uint32_t r0 = q * w;
    const uint32_t gk = (uint32_t)(g >> 32);
    const uint32_t gp = (uint32_t)g;
    uint32_t cnt = 0;
    if (w <= 64 && (w & 3) == 0) {  // 16-byte aligned: base and q*w are multiples of 4
        const uint4 *p = reinterpret_cast<const uint4 *>(tiles_k + base + r0);
        for (uint32_t v = 0; v < w / 4; ++v) {
            const uint4 x = p[v];
            const uint32_t pos = (uint32_t)(base + r0 + 4 * v);
            cnt += (x.x < gk || (x.x == gk && pos + 0 <= gp)) ? 1u : 0u;
            cnt += (x.y < gk || (x.y == gk && pos + 1 <= gp)) ? 1u : 0u;
            cnt += (x.z < gk || (x.z == gk && pos + 2 <= gp)) ? 1u : 0u;
            cnt += (x.w < gk || (x.w == gk && pos + 3 <= gp)) ? 1u : 0u;
        }
        return r0 + cnt;
    }
    uint32_t a = r0, b = r0 + w - 1;  // the item at rank b is > g
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        const uint64_t item = ((uint64_t)tiles_k[base + mid] << 32) | (uint32_t)(base + mid);
        if (item <= g) a = mid + 1;
        else b = mid;
    }
    return a;
}

}  // namespace bsort
