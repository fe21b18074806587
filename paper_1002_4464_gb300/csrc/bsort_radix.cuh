// bsort_radix.cuh -- least-significant-digit radix sort of the 32-bit keys
// held by one CTA: the in-CTA sort of Step 2 (sort every sublist) and Step 9
// (sort every bucket) of GPU Bucket Sort (Dehne & Zaboli, Section 4,
// Algorithm 1) for uint32 and transformed float32 keys.  Both steps may use
// any exact sort; this one costs a fixed number of instructions per key and
// digit instead of one merge level per doubling of the unit.
//
// Only the bits that vary inside the unit are sorted: the keys become
// key - kmin (kmin, kmax: the unit's smallest and largest real key) and the
// nb = bits(kmax - kmin) low bits are sorted in ceil(nb / DB) passes of at
// most DB-bit digits (a bucket of Step 9 spans about 2^32 / b key values, so
// it needs two or three 7-bit passes; a unit of equal keys needs none).
//
// One pass over the T*E keys, which thread t holds as ranks [t*E, t*E + E)
// of the current order ("thread-blocked"):
//   1. count: every thread counts its keys per digit in its own column of
//      16-bit counters (two digits per 32-bit word: digit d sits in row
//      d mod 2^(w-1), low half if d < 2^(w-1), else high half) with
//      shared-memory reductions (no read-modify-write chain per key);
//   2. scan: one exclusive scan over the words in (row, thread) order gives
//      every (digit, thread) the number of keys of smaller digits or of the
//      same digit in earlier threads (high halves are offset by the total of
//      the low halves);
//   3. rank: every thread walks its keys again in order, and an atomic add
//      on its own counter returns each key's rank (the prefix plus the
//      thread's earlier keys of that digit): a stable counting sort; the key
//      is stored at its rank in the key area at once;
//   4. the keys are reloaded thread-blocked for the next pass.
// A 32K-key unit with 7-bit digits takes 135 KB of keys and 68 KB of
// counters.  No instruction depends on how many distinct digits a warp
// holds (no match.any), so the cost is the same on every key distribution.
#pragma once

#include <cstdint>

#include "bsort_device.cuh"

namespace bsort {

// Shared memory of cta_radix_sort<T, E, DB> (digits of at most DB bits):
// the keys in the padded layout, then the counters (2^(DB-1) rows of T
// words, four spare words after every 64 so that a thread's 64-word scan
// chunk is read with conflict-free 16-byte loads).
template <int T, int E, int DB>
struct RadixSmem {
    static constexpr int kKeyWords = T * E + ((T * E) >> 5) + 1;
    static constexpr int kCounterOff = (kKeyWords + 3) & ~3;  // 16-byte aligned
    static constexpr int kRowWords = T + T / 16;
    static constexpr int kCounterWords = (1 << (DB - 1)) * kRowWords;
    static constexpr int kBytes = (kCounterOff + kCounterWords) * 4;
};

// Layout of the keys between passes: E + 1 words per thread, so that the
// thread-blocked reload (lane stride E + 1, odd) is free of bank conflicts.
template <int E>
__device__ __forceinline__ int radix_phys(int x)
{
    return x + x / E;
}

// Exclusive prefix of x over the CTA's threads in thread order, and the
// total.  s_wt holds one word per warp; the caller synchronises before
// s_wt is written again.
template <int T>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t *s_wt,
                                                        uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_wt[warp] = inc;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) {
        const uint32_t v = s_wt[w];
        pre += w < warp ? v : 0u;
        tot += v;
    }
    total = tot;
    return pre + inc - x;
}

__device__ __forceinline__ void red_add_shared(uint32_t saddr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t atom_add_shared(uint32_t saddr, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(saddr), "r"(v) : "memory");
    return old;
}

// Sort the CTA's T*E keys v ascending into sm (padded layout pidx, T*E
// slots, followed by the counters: RadixSmem<T, E, DB>::kBytes in all).
// On entry v holds the keys in the warp-blocked layout (register k of
// (warp, lane) is position wb_pos<E>(warp, lane, k)); positions >= len are
// padding, whatever they hold.  On return sm[pidx(x)] is the x-th smallest
// real key for x < len and 0xFFFFFFFF for x >= len, as cta_sort leaves it.
// Equal keys are indistinguishable (keys only), so the first pass may take
// the keys in any order.  Ends with __syncthreads().
template <int T, int E, int DB>
__device__ __forceinline__ void cta_radix_sort(uint32_t (&v)[E], uint32_t *sm, int len)
{
    static_assert(T % 64 == 0 && E % 16 == 0, "T a multiple of 64, E of 16");
    static_assert(T * E <= 32768 && (T * E & (T * E - 1)) == 0,
                  "ranks and per-half totals must fit 16 bits; T*E a power of two");
    static_assert(DB >= 1 && DB <= 7, "at most 64 counter rows");
    using S = RadixSmem<T, E, DB>;
    constexpr int W = 32 * E;  // positions of one warp
    constexpr int G = 8;      // keys ranked per batch of atomics
    __shared__ uint32_t s_wt[T / 32];
    __shared__ uint32_t s_mm[2][T / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t *cnt = sm + S::kCounterOff;

    // smallest and largest real key
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    if ((warp + 1) * W <= len) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            lo = min(lo, v[k]);
            hi = max(hi, v[k]);
        }
    } else if (warp * W < len) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if (wb_pos<E>(warp, lane, k) < len) {
                lo = min(lo, v[k]);
                hi = max(hi, v[k]);
            }
        }
    }
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    if (lane == 0) {
        s_mm[0][warp] = lo;
        s_mm[1][warp] = hi;
    }
    __syncthreads();
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) {
        kmin = min(kmin, s_mm[0][w]);
        kmax = max(kmax, s_mm[1][w]);
    }
    const uint32_t range = kmax - kmin;
    const int nb = (len > 0 && kmax > kmin) ? 32 - __clz(range) : 0;
    if (nb == 0) {  // no real key, or all of them equal
#pragma unroll 4
        for (int k = 0; k < E; ++k) {
            const int x = k * T + tid;
            sm[pidx<uint32_t>(x)] = x < len ? kmin : 0xFFFFFFFFu;
        }
        __syncthreads();
        return;
    }
    // keys relative to kmin; padding becomes the largest real key (it then
    // ranks at or after every real key, and is rewritten at the end)
    if ((warp + 1) * W <= len) {
#pragma unroll
        for (int k = 0; k < E; ++k) v[k] -= kmin;
    } else {
#pragma unroll
        for (int k = 0; k < E; ++k)
            v[k] = wb_pos<E>(warp, lane, k) < len ? v[k] - kmin : range;
    }

    // Warps past the last real key hold only padding: they skip every pass
    // (pass 1 takes the keys warp-blocked, later passes thread-blocked, and
    // in both layouts the first aw warps hold the first aw*W positions, the
    // boundary warp's padding included).
    const int aw = (len + W - 1) / W;
    const bool act = warp < aw;
    const int passes = (nb + DB - 1) / DB;
    // this thread's counter in row 0 (shared-window address); rows are
    // kRowWords apart
    const uint32_t c0 = smem_u32addr(cnt + tid + 4 * (tid >> 6));
    constexpr uint32_t kRowBytes = 4u * (uint32_t)S::kRowWords;
    uint4 *chunk = reinterpret_cast<uint4 *>(cnt + 68 * tid);
    int sh = 0;
#pragma unroll 1
    for (int p = 0; p < passes; ++p) {
        const int wd = (nb - sh + (passes - p) - 1) / (passes - p);  // digit bits, <= DB
        const int hs = wd - 1;
        const uint32_t rmask = (1u << hs) - 1u;
        const int owners = (1 << hs) * (T / 64);  // threads owning a 64-word scan chunk
        if (tid < owners) {
#pragma unroll
            for (int i = 0; i < 16; ++i) chunk[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        // 1. count, each thread in its own column
        if (act) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const uint32_t dg = v[k] >> sh;
                const uint32_t h16 = ((dg >> hs) & 1u) << 4;
                red_add_shared(c0 + (dg & rmask) * kRowBytes, 1u << h16);
            }
        }
        __syncthreads();
        // 2. exclusive scan of the counter words in (row, thread) order
        // (four 16-byte words at a time: the keys stay live in registers)
        uint32_t sum = 0;
        if (tid < owners) {
#pragma unroll 1
            for (int i0 = 0; i0 < 16; i0 += 4) {
#pragma unroll
                for (int i = i0; i < i0 + 4; ++i) {
                    const uint4 a = chunk[i];
                    sum += a.x + a.y + a.z + a.w;
                }
            }
        }
        uint32_t total;
        uint32_t run = block_exclusive_sum<T>(sum, s_wt, total);
        run += (total & 0xFFFFu) << 16;  // high-half digits follow every low-half one
        if (tid < owners) {
#pragma unroll 1
            for (int i = 0; i < 16; ++i) {
                const uint4 a = chunk[i];
                uint4 o;
                o.x = run;
                run += a.x;
                o.y = run;
                run += a.y;
                o.z = run;
                run += a.z;
                o.w = run;
                run += a.w;
                chunk[i] = o;
            }
        }
        __syncthreads();
        // 3. rank and scatter: batches of G atomics, then their stores
        const bool last = p + 1 == passes;
#pragma unroll
        for (int k0 = 0; k0 < (act ? E : 0); k0 += G) {
            uint32_t r[G];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const uint32_t dg = v[k0 + j] >> sh;
                const uint32_t h16 = ((dg >> hs) & 1u) << 4;
                const uint32_t old = atom_add_shared(c0 + (dg & rmask) * kRowBytes, 1u << h16);
                // (a rank is below T*E; the mask keeps every store inside the
                // key area whatever the counters hold)
                r[j] = (old >> h16) & (uint32_t)(T * E - 1);
            }
            if (last) {
#pragma unroll
                for (int j = 0; j < G; ++j) sm[pidx<uint32_t>((int)r[j])] = v[k0 + j] + kmin;
            } else {
#pragma unroll
                for (int j = 0; j < G; ++j) sm[radix_phys<E>((int)r[j])] = v[k0 + j];
            }
        }
        __syncthreads();
        // 4. reload thread-blocked (the counters are separate: the next
        // pass's barriers order these loads before its stores)
        if (!last && act) {
#pragma unroll
            for (int k = 0; k < E; ++k) v[k] = sm[radix_phys<E>(tid * E + k)];
        }
        sh += wd;
    }
    // padding back to the maximal key, after the len real keys
    for (int x = len + tid; x < T * E; x += T) sm[pidx<uint32_t>(x)] = 0xFFFFFFFFu;
    __syncthreads();
}

}  // namespace bsort
