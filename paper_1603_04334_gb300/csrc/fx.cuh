// fx.cuh -- per-column magnitude bounds of FP64 blocks and the fixed-point grid they
// define, shared by the FP64 stencil (stencil_df.cu), the nonlocal projection and pair
// scatter (nonlocal.cu) and the bound pass (bounds.cu). A bound is the largest high word
// (bits 32..62) of |y| over a column; it only grows.
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

// Column bound (largest high word of |y|) -> E with |y| < 2^E for every y of the column.
__device__ __forceinline__ int bound_exponent(unsigned b) { return (int)((b >> 20) & 0x7ffu) - 1022; }

// A value on its column's 49-bit grid as two integers: y 2^(49-E) = d 2^23 + r truncated
// toward zero, |d| < 2^26 and |r| < 2^23, both with the sign of y (|y| < 2^E). From
// y = M 2^(e-1075) (M the 53-bit significand): N = M >> s, s = 1026 + E - e >= 4, holds d
// (N >> 23) and r (the low 23 bits); zero and subnormal y give 0.
__device__ __forceinline__ int2 fx_split(double y, int E)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned hw = (unsigned)(b >> 32);
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned long long M =
        e ? ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) : 0ull;
    const unsigned long long N = M >> min(1026 + E - e, 63);
    const int sm = (int)hw >> 31;  // 0 or -1
    const int d = ((int)(unsigned)(N >> 23) ^ sm) - sm;
    const int r = ((int)((unsigned)N & 0x7fffffu) ^ sm) - sm;
    return make_int2(d, r);
}

// FP32: y = m 2^(e-150) (24-bit m) = (m 2^29) 2^(e-179), so s = 130 + E - e.
__device__ __forceinline__ int2 fx_split(float y, int E)
{
    const unsigned u = __float_as_uint(y);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned long long M =
        e ? ((unsigned long long)((u & 0x7fffffu) | 0x800000u) << 29) : 0ull;
    const unsigned long long N = M >> min(130 + E - e, 63);
    const int sm = (int)u >> 31;
    const int d = ((int)(unsigned)(N >> 23) ^ sm) - sm;
    const int r = ((int)((unsigned)N & 0x7fffffu) ^ sm) - sm;
    return make_int2(d, r);
}

}  // namespace sparc
