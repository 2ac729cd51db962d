// fx.cuh -- per-column magnitude bounds of FP64 blocks and the fixed-point grid they
// define, shared by the FP64 stencil (stencil_df.cu), the pair scatter (nonlocal.cu) and
// the bound pass (bounds.cu). A bound is the largest high word (bits 32..62) of |y| over a
// column; it only grows.
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

// A value on the column's grid: .x = d, .y = the bits of r (y 2^(28-E) = d + r).
// From the significand M (53 bits) of y = M 2^(e-1075): d = M >> s and r = the next 23
// bits of M below d, with s = 1047 + E - e >= 25 (|y| < 2^E); zero and subnormal y give 0.
__device__ __forceinline__ int2 to_fx(double y, int E)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned hw = (unsigned)(b >> 32), ml = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned mh = (hw & 0xfffffu) | 0x100000u;
    const int s = 1047 + E - e, s2 = s - 23;
    const unsigned d = s < 32 ? __funnelshift_r(ml, mh, s) : (mh >> min(s - 32, 31));
    const unsigned r23 =
        (s2 < 32 ? __funnelshift_r(ml, mh, s2) : (mh >> min(s2 - 32, 31))) & 0x7fffffu;
    float r = __uint_as_float(0x3F800000u | r23) - 1.0f;  // r23 2^-23, exact
    int di = (int)d;
    if (hw >> 31) {
        di = -di;
        r = -r;
    }
    return e == 0 ? make_int2(0, 0) : make_int2(di, __float_as_int(r));
}

// FP32 input: y = m 2^(e-150) (24-bit m); with M = m 2^27 (< 2^51),
// y 2^(28-E) = M 2^-s, s = 149 + E - e >= 23 (|y| < 2^E), so d = M >> s < 2^28.
__device__ __forceinline__ int2 to_fx(float y, int E)
{
    const unsigned u = __float_as_uint(y);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned long long M = (unsigned long long)((u & 0x7fffffu) | 0x800000u) << 27;
    const int s = 149 + E - e;
    const unsigned d = s < 64 ? (unsigned)(M >> s) : 0u;
    const int s2 = s - 23;
    const unsigned r23 = (s2 < 64 ? (unsigned)(M >> s2) : 0u) & 0x7fffffu;
    float r = __uint_as_float(0x3F800000u | r23) - 1.0f;
    int di = (int)d;
    if (u >> 31) {
        di = -di;
        r = -r;
    }
    return e == 0 ? make_int2(0, 0) : make_int2(di, __float_as_int(r));
}

}  // namespace sparc
