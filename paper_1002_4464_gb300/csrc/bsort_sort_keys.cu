// bsort_sort_keys.cu -- instantiations of the Step 1-3 and Step 9 sorting
// kernels for keys-only sorts (uint32 / transformed float32 keys).
#include "bsort_internal.h"
#include "bsort_sort.cuh"

namespace bsort {

// chunk shapes: 2048 = 128x16, 4096 = 256x16, 8192 = 512x16, 16384 = 1024x16,
// 32768 = 1024x32; clusters of 2, 4, 8 CTAs on the 32768-item chunk.  The
// 32768-item chunk also has a radix-sorting form (256 threads x 128 keys,
// cta_radix_sort), chosen with `radix`.
cudaError_t init_sort_keys_kernels()
{
    cudaError_t e;
#define I(T_, E_, C_)                                            \
    e = init_sort_pair_of_kernels<T_, E_, false, C_>();          \
    if (e != cudaSuccess) return e
    I(128, 16, 1); I(256, 16, 1); I(512, 16, 1); I(1024, 16, 1); I(1024, 32, 1);
    I(1024, 32, 2); I(1024, 32, 4); I(1024, 32, 8);
#undef I
    return init_sort_keys_radix_kernels();
}

cudaError_t launch_sublist_sort_keys(int chunk, int ctas, const void *keys_in, uint64_t n,
                                     uint32_t m, int is_f32, uint32_t s, uint32_t *tiles_k,
                                     uint64_t *samples, cudaStream_t st, uint32_t tile0,
                                     bool radix)
{
    if (radix && chunk == 32768 && ctas == 1)
        return launch_sublist_sort_keys_radix(ctas, keys_in, n, m, is_f32, s, tiles_k, samples,
                                              st, tile0);
#define L(T_, E_, C_)                                                                       \
    return launch_sublist_sort_t<T_, E_, false, C_>(keys_in, nullptr, n, m, is_f32, 0, s,   \
                                                    tiles_k, nullptr, samples, tile0, st)
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(128, 16, 1);
        case 4096: L(256, 16, 1);
        case 8192: L(512, 16, 1);
        case 16384: L(1024, 16, 1);
        case 32768: L(1024, 32, 1);
        }
    } else if (chunk == 32768) {
        switch (ctas) {
        case 2: L(1024, 32, 2);
        case 4: L(1024, 32, 4);
        case 8: L(1024, 32, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_sort_keys(int chunk, int ctas, const void *src_k, const uint32_t *units,
                                    uint32_t max_units, uint64_t n, uint64_t n_pad, int is_f32,
                                    void *out_k, int *err, const GatherSrc &g, cudaStream_t st,
                                    bool radix)
{
    if (radix && chunk == 32768 && ctas == 1)
        return launch_bucket_sort_keys_radix(ctas, src_k, units, max_units, n, n_pad, is_f32,
                                             out_k, err, g, st);
#define L(T_, E_, C_)                                                                        \
    return launch_bucket_sort_t<T_, E_, false, C_>(src_k, nullptr, units, max_units, n,      \
                                                   n_pad, is_f32, 0, out_k, nullptr, err, g, st)
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(128, 16, 1);
        case 4096: L(256, 16, 1);
        case 8192: L(512, 16, 1);
        case 16384: L(1024, 16, 1);
        case 32768: L(1024, 32, 1);
        }
    } else if (chunk == 32768) {
        switch (ctas) {
        case 2: L(1024, 32, 2);
        case 4: L(1024, 32, 4);
        case 8: L(1024, 32, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_sort_keys_range(int chunk, int ctas, const void *src_k,
                                          const uint32_t *units, const uint32_t *range,
                                          uint32_t grid_units, uint64_t n, uint64_t n_pad,
                                          int is_f32, void *out_k, int *err, cudaStream_t st,
                                          bool radix)
{
    if (radix && chunk == 32768 && ctas == 1)
        return launch_bucket_sort_keys_range_radix(ctas, src_k, units, range, grid_units, n,
                                                   n_pad, is_f32, out_k, err, st);
#define L(T_, E_, C_)                                                                         \
    return launch_bucket_sort_range_t<T_, E_, false, C_>(src_k, units, range, grid_units, n, \
                                                         n_pad, is_f32, out_k, err, st)
    if (ctas == 1) {
        switch (chunk) {
        case 2048: L(128, 16, 1);
        case 4096: L(256, 16, 1);
        case 8192: L(512, 16, 1);
        case 16384: L(1024, 16, 1);
        case 32768: L(1024, 32, 1);
        }
    } else if (chunk == 32768) {
        switch (ctas) {
        case 2: L(1024, 32, 2);
        case 4: L(1024, 32, 4);
        case 8: L(1024, 32, 8);
        }
    }
#undef L
    return cudaErrorInvalidValue;
}

}  // namespace bsort
