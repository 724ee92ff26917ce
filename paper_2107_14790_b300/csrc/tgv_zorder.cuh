// Z-order (Morton) codes and the device radix sort of 64-bit keys, shared by the
// octree build and the treetop of the composite grid.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// bits 0..20 of v to every third bit
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Morton code: bit 3k of x, 3k+1 of y, 3k+2 of z (21 bits per axis)
__host__ __device__ __forceinline__ uint64_t morton3(uint64_t x, uint64_t y, uint64_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

__host__ __device__ __forceinline__ uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x1f00000000ffffull;
    v = (v | (v >> 32)) & 0x1fffffull;
    return v;
}

// Stable LSD radix sort of n keys by bits [lo_bit, lo_bit + nbits), 8-bit digits; `tmp`
// holds n keys, `hist` tgv_radix_hist_words(n) counts; adds the kernels it launches to
// *launches (nullable).  With `result` (nullable) the sorted keys are left in keys or tmp,
// whichever the last pass wrote, and *result points there; without it they end in keys.
cudaError_t tgv_radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint32_t* hist, int64_t n, int lo_bit, int nbits,
                               cudaStream_t s, int64_t* launches, uint64_t** result = nullptr);
int64_t tgv_radix_hist_words(int64_t n);
