// df.cuh -- FP32-pair ("double-float") helpers shared by the FP64 kernels that run on the
// FP32 pipes (stencil_df.cu, gram_df.cu).
//
// split_double: x -> (hi, lo) with hi = x truncated to 24 significant bits and
// lo = (x - hi) rounded to FP32, built from the bit pattern with integer operations only
// (the FP64 pipe is 1/64 of the FP32 rate on GB300). hi + lo equals x to about 2^-48
// relative. |x| < 2^-126 gives (0, 0); for |x| < 2^-74 lo is dropped (absolute error
// below 2^-98); |x| >= 2^128 gives +-Inf and NaN gives NaN in hi, so they propagate.
// No FP64 or conversion instruction is used on any path (a "rare" conversion branch is
// if-converted by the compiler and would run for every value).
// two_sum: Knuth's error-free sum, s + e = a + b exactly.
// mac: one multiply-add of the compensated dot product (Ogita, Rump & Oishi 2005,
// "Dot2"): the exact product of the hi parts (TwoProduct via FMA) enters the running
// sum sh through two_sum, and the product error, the two_sum error and the cross terms
// ah*bl + al*bh go to the second accumulator sl.
#pragma once
#include <cuda_runtime.h>

namespace sparc {

__device__ __forceinline__ float2 split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned sg = hw & 0x80000000u;
    const bool nan = (e == 2047) && (((hw & 0xfffffu) | lw) != 0u);
    const unsigned big = sg | (nan ? 0x7fc00000u : 0x7f800000u);  // +-Inf or NaN
    const unsigned hb = sg | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned hbits = (e > 1150) ? big : ((e >= 897) ? hb : 0u);
    const int es = e - 948;  // biased FP32 exponent of 2^(e - 1075)
    const float sc = __uint_as_float((unsigned)max(es, 1) << 23);
    float lo = __uint2float_rn(lw & 0x1fffffffu) * sc;
    lo = __uint_as_float(__float_as_uint(lo) ^ sg);
    return make_float2(__uint_as_float(hbits), (es >= 1 && e <= 1150) ? lo : 0.0f);
}

__device__ __forceinline__ float2 split_double(float x) { return make_float2(x, 0.0f); }

// Exact FP32 -> FP64 widening from the bit pattern (integer operations only). FP32
// subnormals become 0 (|f| < 2^-126); Inf and NaN map to FP64 Inf and NaN.
__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned sg = u & 0x80000000u;
    unsigned hi = sg | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (e == 0xffu) {  // Inf / NaN (selected, not branched)
        hi = sg | 0x7ff00000u | (m ? 0x80000u : 0u);
        lo = 0u;
    }
    if (e == 0u) hi = lo = 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// hi + lo of an FP32 pair as one FP64 value (a single FP64 add).
__device__ __forceinline__ double pair_to_double(float h, float l) { return widen(h) + widen(l); }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void mac(float2 a, float2 b, float &sh, float &sl)
{
    const float p = a.x * b.x;
    const float pe = fmaf(a.x, b.x, -p);
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl += e;
    sl += pe;
    sl = fmaf(a.x, b.y, sl);
    sl = fmaf(a.y, b.x, sl);
}

}  // namespace sparc
