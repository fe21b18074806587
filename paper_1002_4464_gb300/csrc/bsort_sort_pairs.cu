// bsort_sort_pairs.cu -- instantiations of the Step 1-3 and Step 9 sorting
// kernels for key-value sorts (64-bit words key << 32 | position).
#include "bsort_internal.h"
#include "bsort_sort.cuh"

namespace bsort {

// chunk shapes: 2048 = 128x16, 4096 = 256x16, 8192 = 512x16, 16384 = 1024x16;
// clusters of 2, 4, 8 CTAs on the 16384-item chunk.
cudaError_t init_sort_pairs_kernels()
{
    cudaError_t e;
#define I(T_, E_, C_)                                           \
    e = init_sort_pair_of_kernels<T_, E_, true, C_>();          \
    if (e != cudaSuccess) return e
    I(128, 16, 1); I(256, 16, 1); I(512, 16, 1); I(1024, 16, 1);
    I(1024, 16, 2); I(1024, 16, 4); I(1024, 16, 8);
#undef I
    return cudaSuccess;
}

cudaError_t launch_sublist_sort_pairs(int chunk, int ctas, const void *keys_in,
                                      const void *vals_in, uint64_t n, uint32_t m, int is_f32,
                                      int val_bytes, uint32_t s, uint32_t *tiles_k,
                                      void *tiles_v, uint64_t *samples, cudaStream_t st)
{
#define L(T_, E_, C_)                                                                      \
    return launch_sublist_sort_t<T_, E_, true, C_>(keys_in, vals_in, n, m, is_f32,          \
                                                   val_bytes, s, tiles_k, tiles_v, samples, \
                                                   0u, st)
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

cudaError_t launch_bucket_sort_pairs(int chunk, int ctas, const void *src_k, const void *src_v,
                                     const uint32_t *units, uint32_t max_units, uint64_t n,
                                     uint64_t n_pad, int is_f32, int val_bytes, void *out_k,
                                     void *out_v, int *err, const GatherSrc &g, cudaStream_t st)
{
#define L(T_, E_, C_)                                                                          \
    return launch_bucket_sort_t<T_, E_, true, C_>(src_k, src_v, units, max_units, n, n_pad,    \
                                                  is_f32, val_bytes, out_k, out_v, err, g, st)
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

}  // namespace bsort
