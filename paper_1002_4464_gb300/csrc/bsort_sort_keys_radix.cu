// bsort_sort_keys_radix.cu -- instantiations of the Step 1-3 and Step 9
// sorting kernels whose 32768-key units are sorted by one CTA by digits
// (cta_radix_sort: 256 threads x 128 keys, 7-bit digits), for keys-only
// sorts of uint32 / transformed float32 keys: Step-9 units and Step-2
// sublists of one CTA.
#include "bsort_internal.h"
#include "bsort_sort.cuh"

namespace bsort {

cudaError_t init_sort_keys_radix_kernels()
{
    cudaError_t e;
#define I(C_)                                                    \
    e = init_sort_pair_of_kernels<256, 128, false, C_, true>();  \
    if (e != cudaSuccess) return e
    I(1);
#undef I
    return cudaSuccess;
}

cudaError_t launch_sublist_sort_keys_radix(int ctas, const void *keys_in, uint64_t n, uint32_t m,
                                           int is_f32, uint32_t s, uint32_t *tiles_k,
                                           uint64_t *samples, cudaStream_t st, uint32_t tile0)
{
#define L(C_)                                                                                \
    return launch_sublist_sort_t<256, 128, false, C_, true>(keys_in, nullptr, n, m, is_f32, 0, \
                                                            s, tiles_k, nullptr, samples,      \
                                                            tile0, st)
    if (ctas == 1) L(1);
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_sort_keys_radix(int ctas, const void *src_k, const uint32_t *units,
                                          uint32_t max_units, uint64_t n, uint64_t n_pad,
                                          int is_f32, void *out_k, int *err, const GatherSrc &g,
                                          cudaStream_t st)
{
#define L(C_)                                                                                 \
    return launch_bucket_sort_t<256, 128, false, C_, true>(src_k, nullptr, units, max_units, n, \
                                                           n_pad, is_f32, 0, out_k, nullptr,    \
                                                           err, g, st)
    if (ctas == 1) L(1);
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_sort_keys_range_radix(int ctas, const void *src_k,
                                                const uint32_t *units, const uint32_t *range,
                                                uint32_t grid_units, uint64_t n, uint64_t n_pad,
                                                int is_f32, void *out_k, int *err,
                                                cudaStream_t st)
{
#define L(C_)                                                                               \
    return launch_bucket_sort_range_t<256, 128, false, C_, true>(src_k, units, range,         \
                                                                 grid_units, n, n_pad, is_f32, \
                                                                 out_k, err, st)
    if (ctas == 1) L(1);
#undef L
    return cudaErrorInvalidValue;
}

}  // namespace bsort
