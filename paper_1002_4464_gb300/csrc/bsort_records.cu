// bsort_records.cu -- Steps 4-5 of GPU Bucket Sort (Dehne & Zaboli,
// Section 4, Algorithm 1: sort the m*s samples, then take the b evenly
// spaced ones as splitters) by a least-significant-digit radix sort of the
// sample records, for sample sets of many tiles.
//
// The records are key << 32 | q, q = i*s + k the sample's index, written by
// Step 3 at index q: the array starts in q order.  A stable sort by the
// 32-bit key alone then leaves it in (key, q) order, the order Step 4
// defines.  Four passes over 8-bit digits of the key; each pass is one
// kernel over tiles of 8192 records (16 warps of 512 consecutive records,
// 32 consecutive records per warp instruction) in which
//   1. every warp counts its records per digit in its own 256 counters;
//   2. an exclusive scan of the counters in (digit, warp) order gives each
//      warp the first tile rank of each digit, and the tile's digit counts;
//   3. each record's tile rank is its warp's running counter of its digit
//      plus the number of lower lanes holding that digit (found with eight
//      ballots, one per digit bit): a stable order; it is staged there;
//   4. the tile publishes its 256 digit counts and adds up those of the
//      earlier tiles (a decoupled look-back per digit, one thread each,
//      bounded waits); with the global digit histogram (one kernel before
//      the passes) this places the tile's digit-d records in the output,
//      which they reach from the staged order in runs of equal digit.
// The last pass writes no array: a record whose final rank is a splitter
// rank r_j = floor((j+1) m s / b) - 1 (Step 5) is stored as g_j.
#include <cstdint>

#include "bsort_device.cuh"
#include "bsort_internal.h"
#include "bsort_radix.cuh"

namespace bsort {

namespace {

constexpr int kRsT = 512;                              // threads per tile
constexpr int kRsE = 16;                               // records per thread
constexpr int kRsW = kRsT / 32;                        // warps per tile
constexpr int kRsTile = kRsT * kRsE;                   // 8192 records per tile
constexpr int kRsRecSlots = kRsTile + kRsTile / 32;    // staged records, one spare per 32
constexpr int kRsSmemBytes = kRsRecSlots * 8 + kRsW * 256 * 4;
constexpr uint32_t kRsFlagAgg = 1u << 30;  // tile count published
constexpr uint32_t kRsFlagInc = 2u << 30;  // count of this and every earlier tile published
constexpr uint32_t kRsValMask = (1u << 30) - 1u;
constexpr int kRsSpinLimit = 1 << 22;      // polls of one look-back wait (about a second)

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p)
{
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

// staged slot of tile rank x: one spare word after every 32, so that the
// 32 lanes reading ranks 32c .. 32c+31 never share a bank pair
__device__ __forceinline__ int rs_phys(int x)
{
    return x + (x >> 5);
}

// Lanes of the warp (among `valid`) whose 8-bit digit equals this lane's.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, uint32_t valid)
{
    uint32_t m = valid;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
        const bool on = (d >> bit) & 1u;
        const uint32_t bl = __ballot_sync(0xFFFFFFFFu, on);
        m &= on ? bl : ~bl;
    }
    return m;
}

// Digit histograms of all four passes: hist[p*256 + d] = records whose key
// has digit d at bits [8p, 8p + 8).  Warps take 32 consecutive records at a
// time; a digit that all 32 lanes share (runs of equal digits are common:
// the records of one sublist are sorted) is added once.
// The CTA that finishes last (a ticket taken after its counts are in)
// also turns the four histograms into the digits' first global ranks,
// gbase[p*256 + d] = the records whose digit p is below d.
template <int T>
__global__ void __launch_bounds__(T)
k_rec_hist(const uint64_t *__restrict__ rec, uint32_t n, uint32_t *__restrict__ hist,
           uint32_t *__restrict__ done, uint32_t *__restrict__ gbase)
{
    static_assert(T == 256, "one thread per digit in the final scan");
    __shared__ uint32_t sh[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += T) sh[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (T / 32);
    const uint32_t groups = (n + 31) / 32;
    constexpr int U = 4;  // groups in flight per warp
    for (uint32_t g0 = blockIdx.x * (T / 32) + (threadIdx.x >> 5); g0 < groups; g0 += warps * U) {
        uint32_t key[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t x = (uint64_t)(g0 + (uint64_t)u * warps) * 32 + lane;
            ok[u] = g0 + (uint64_t)u * warps < groups && x < n;
            key[u] = ok[u] ? (uint32_t)(rec[x] >> 32) : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + (uint64_t)u * warps >= groups) break;  // warp-uniform
            const bool full = __all_sync(0xFFFFFFFFu, ok[u]);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const uint32_t d = (key[u] >> (8 * p)) & 255u;
                const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, d, 0);
                if (full && __all_sync(0xFFFFFFFFu, d == d0)) {
                    if (lane == 0) atomicAdd(&sh[p * 256 + d0], 32u);
                } else if (ok[u]) {
                    atomicAdd(&sh[p * 256 + d], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += T)
        if (sh[i] != 0u) atomicAdd(&hist[i], sh[i]);
    __threadfence();
    __syncthreads();
    __shared__ uint32_t s_last;
    __shared__ uint32_t s_wt[T / 32];
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
        uint32_t tot;
        const uint32_t c = __ldcg(&hist[p * 256 + (int)threadIdx.x]);
        gbase[p * 256 + (int)threadIdx.x] = block_exclusive_sum<T>(c, s_wt, tot);
        __syncthreads();  // s_wt is reused by the next digit position
    }
}

// One stable pass over the digit at key bits [shift, shift + 8).  gfirst:
// the 256 digits' first global ranks; status: tiles*256 words, ticket: one
// word, both zero at launch.  spl == nullptr: out receives the n records in
// the new order; otherwise only spl[j] = the record of final rank r_j.
template <int T, int E>
__global__ void __launch_bounds__(T, 2)
k_rec_pass(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, uint32_t n, int shift,
           const uint32_t *__restrict__ gfirst, uint32_t *status, uint32_t *ticket, int *err,
           uint64_t *__restrict__ spl, uint32_t b)
{
    static_assert(T == 512 && T * E == kRsTile, "16 warps, one thread per digit in the first 8");
    constexpr int W = T / 32;
    extern __shared__ __align__(16) uint32_t s_dyn[];
    uint64_t *srec = reinterpret_cast<uint64_t *>(s_dyn);  // kRsRecSlots staged records
    uint32_t *whist = s_dyn + 2 * kRsRecSlots;             // [W][256] warp counters
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_wt[W];
    __shared__ uint32_t s_start[257];
    __shared__ uint32_t s_gpos[256];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = tid; i < W * 256; i += T) whist[i] = 0u;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t base = tile * (uint32_t)kRsTile;
    const uint32_t len = min((uint32_t)kRsTile, n - base);
    const int sh = 32 + shift;
    // warp w holds tile ranks [512 w, 512 w + 512), 32 consecutive per step
    const uint32_t xw = (uint32_t)warp * (32u * E) + (uint32_t)lane;
    uint64_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const uint32_t x = xw + 32u * k;
        v[k] = x < len ? in[base + x] : 0ull;
    }
    uint32_t *wh = whist + warp * 256;
    const uint32_t lt = (1u << lane) - 1u;
    // 1. warp counts per digit (shared-memory atomics; a digit held by all
    // 32 lanes is added once)
    uint32_t dg4[E / 4];  // the digits, four to a register
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const bool ok = xw + 32u * k < len;
        const uint32_t d = (uint32_t)(v[k] >> sh) & 255u;
        if (k % 4 == 0) dg4[k / 4] = 0u;
        dg4[k / 4] |= d << (8 * (k % 4));
        const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, d, 0);
        if (__all_sync(0xFFFFFFFFu, ok && d == d0)) {
            if (lane == 0) atomicAdd(&wh[d0], 32u);
        } else if (ok) {
            atomicAdd(&wh[d], 1u);
        }
    }
    __syncthreads();
    // 2. exclusive scan in (digit, warp) order: thread t takes digit t/2,
    // warps [8 (t mod 2), 8 (t mod 2) + 8)
    {
        const uint32_t d = (uint32_t)tid >> 1;
        const int w0 = (tid & 1) * (W / 2);
        uint32_t c[W / 2];
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < W / 2; ++w) {
            c[w] = whist[(w0 + w) * 256 + d];
            sum += c[w];
        }
        uint32_t total;
        uint32_t run = block_exclusive_sum<T>(sum, s_wt, total);
        if ((tid & 1) == 0) s_start[d] = run;
        if (tid == 0) s_start[256] = len;
#pragma unroll
        for (int w = 0; w < W / 2; ++w) {
            whist[(w0 + w) * 256 + d] = run;
            run += c[w];
        }
    }
    // global first rank of each digit (the histogram kernel's scan)
    const uint32_t gbase = tid < 256 ? gfirst[tid] : 0u;
    __syncthreads();  // warp bases and s_start complete
    // 3. rank and stage
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const bool ok = xw + 32u * k < len;
        const uint32_t valid = __ballot_sync(0xFFFFFFFFu, ok);
        if (valid == 0u) break;  // warp-uniform
        const uint32_t d = (dg4[k / 4] >> (8 * (k % 4))) & 255u;
        const uint32_t pm = digit_peers(d, valid);
        const uint32_t r = wh[d] + (uint32_t)__popc(pm & lt);
        __syncwarp();
        if (ok) {
            if ((pm & lt) == 0u) wh[d] += (uint32_t)__popc(pm);
            // (a rank is below the tile size; the mask keeps every store
            // inside the staging area whatever the counters hold)
            srec[rs_phys((int)(r & (uint32_t)(kRsTile - 1)))] = v[k];
        }
        __syncwarp();
    }
    // 4. look-back for digit d over the earlier tiles (threads 0 .. 255)
    uint32_t prefix = 0;
    const uint32_t d = (uint32_t)tid;
    if (tid < 256) {
        const uint32_t cd = s_start[d + 1] - s_start[d];
        uint32_t *mine = status + (uint64_t)tile * 256u + d;
        if (tile == 0) {
            atomicExch(mine, kRsFlagInc | cd);
        } else {
            atomicExch(mine, kRsFlagAgg | cd);
            // LB predecessors per round trip: their words are loaded
            // together, then taken in order (a word not yet published is
            // polled, bounded)
            constexpr int LB = 8;
            int spins = 0;
            bool timed_out = false, done = false;
            for (int64_t tp0 = (int64_t)tile - 1; !done && !timed_out; tp0 -= LB) {
                uint32_t sv[LB];
#pragma unroll
                for (int k = 0; k < LB; ++k)
                    sv[k] = tp0 - k >= 0
                                ? ld_volatile_u32(status + (uint64_t)(tp0 - k) * 256u + d)
                                : kRsFlagInc;  // (tile 0 is inclusive: never reached)
#pragma unroll
                for (int k = 0; k < LB; ++k) {
                    if (done || timed_out) break;
                    while ((sv[k] >> 30) == 0u) {
                        if (++spins > kRsSpinLimit) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(64);
                        sv[k] = ld_volatile_u32(status + (uint64_t)(tp0 - k) * 256u + d);
                    }
                    if (timed_out) break;
                    prefix += sv[k] & kRsValMask;
                    if ((sv[k] >> 30) == 2u) done = true;
                }
            }
            if (timed_out) set_error(err, DEV_TIMEOUT);
            atomicExch(mine, kRsFlagInc | ((prefix + cd) & kRsValMask));
        }
        s_gpos[d] = gbase + prefix - s_start[d];
    }
    __syncthreads();  // staged records and s_gpos complete
    if (spl == nullptr) {
#pragma unroll 4
        for (uint32_t x = (uint32_t)tid; x < len; x += T) {
            const uint64_t rec = srec[rs_phys((int)x)];
            const uint32_t dg = (uint32_t)(rec >> sh) & 255u;
            const uint32_t g = s_gpos[dg] + x;
            if (g < n) out[g] = rec;  // (always, unless a look-back wait gave up)
        }
    } else if (tid < 256) {
        // the splitters among this tile's digit-d records: final ranks
        // [G0, G0 + cd) hold the records staged at [s_start[d], s_start[d+1]);
        // j0 = the first j with r_j = floor((j+1) n / b) - 1 >= G0
        const uint32_t cd = s_start[d + 1] - s_start[d];
        const uint64_t G0 = (uint64_t)gbase + prefix;
        uint64_t j = (((G0 + 1) * b + n - 1) / n) - 1;
        for (; j < b; ++j) {
            const uint64_t r = ((j + 1) * n) / b - 1;
            if (r >= G0 + cd) break;
            spl[j] = srec[rs_phys((int)(r - G0 + s_start[d]))];
        }
    }
}

}  // namespace

// Scratch layout (32-bit words): the four digit histograms (4 * 256), the
// digits' first global ranks (4 * 256), 16 tickets (one per digit pass, one
// for the histogram's last CTA), then 4 * tiles * 256 look-back words; all
// zeroed before the histogram.
namespace {
struct RsScratch {
    uint32_t *hist, *gfirst, *tickets, *status;
};
RsScratch rs_layout(void *scratch)
{
    uint32_t *w = static_cast<uint32_t *>(scratch);
    return {w, w + 4 * 256, w + 8 * 256, w + 8 * 256 + 16};
}
}  // namespace

uint64_t records_radix_scratch_bytes(uint32_t n_rec)
{
    const uint64_t tiles = (n_rec + kRsTile - 1) / kRsTile;
    return 4ull * (8 * 256 + 16 + 4 * tiles * 256);
}

bool records_radix_fits(uint32_t n_rec, uint32_t b)
{
    return n_rec > (uint32_t)kRsTile && b >= 1 && b <= n_rec && n_rec < (1u << 30);
}

cudaError_t init_records_kernels()
{
    return cudaFuncSetAttribute(k_rec_pass<kRsT, kRsE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kRsSmemBytes);
}

cudaError_t launch_records_hist(const uint64_t *samples, uint32_t n_rec, void *scratch, int sms,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(scratch, 0, records_radix_scratch_bytes(n_rec), st);
    if (e != cudaSuccess) return e;
    const RsScratch r = rs_layout(scratch);
    k_rec_hist<256><<<4 * (sms > 0 ? sms : 1), 256, 0, st>>>(samples, n_rec, r.hist,
                                                              r.tickets + 8, r.gfirst);
    return cudaGetLastError();
}

cudaError_t launch_records_pass(int p, const uint64_t *in, uint64_t *out, uint32_t n_rec,
                                uint32_t b, uint64_t *spl, void *scratch, int *err,
                                cudaStream_t st)
{
    if (!records_radix_fits(n_rec, b) || p < 0 || p > 3) return cudaErrorInvalidValue;
    if ((p < 3) != (out != nullptr) || (p == 3) != (spl != nullptr)) return cudaErrorInvalidValue;
    const uint32_t tiles = (n_rec + kRsTile - 1) / kRsTile;
    const RsScratch r = rs_layout(scratch);
    k_rec_pass<kRsT, kRsE><<<tiles, kRsT, kRsSmemBytes, st>>>(
        in, out, n_rec, 8 * p, r.gfirst + 256 * p, r.status + (uint64_t)p * tiles * 256u,
        r.tickets + p, err, spl, b);
    return cudaGetLastError();
}

}  // namespace bsort
