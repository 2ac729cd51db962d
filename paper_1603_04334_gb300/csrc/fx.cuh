// fx.cuh -- per-column magnitude bounds of FP64 blocks, shared by the FP64 stencil
// (stencil_df.cu), the pair scatter (nonlocal.cu) and the bound pass (bounds.cu). A bound
// is the largest high word (bits 32..62) of |y| over a column; it only grows.
#pragma once
#include <cuda_runtime.h>

namespace sparc {

__device__ __forceinline__ unsigned abs_hi_word(double x)
{
    return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}

// *b = max(*b, m). Bounds only grow, so a value read here that is already >= m makes the
// atomic unnecessary (most warps of a launch find the bound raised by earlier warps).
__device__ __forceinline__ void raise_bound(unsigned *b, unsigned m)
{
    if (m > *(volatile unsigned *)b) atomicMax(b, m);
}

__device__ __forceinline__ unsigned abs_hi_word(float x)
{
    // high word of the FP64 widening of |x| (exponent rebiased; subnormals count as 0)
    const unsigned u = __float_as_uint(x) & 0x7fffffffu;
    const unsigned e = u >> 23;
    if (e == 0u) return 0u;
    if (e == 0xffu) return 0x7ff00000u | ((u & 0x7fffffu) ? 0x80000u : 0u);
    return ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
}

}  // namespace sparc
