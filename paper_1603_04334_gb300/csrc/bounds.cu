// bounds.cu -- helpers of the FP64 path that run once per block or per context:
// per-column magnitude bounds (the FP64 stencil's fixed-point grid), V_eff - shift as FP32
// pairs, and FP64 arrays as FP32 pairs.
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

// Column bounds: b[c] = max(b[c], largest high word of |y| over column c). kColmaxCtas
// CTAs per column stride over it (loads 8 x 256 apart in flight per thread), reduce in
// the CTA and raise the bound once: a few atomics per column, not one per warp.
namespace {
constexpr int kColmaxThreads = 256, kColmaxPer = 8, kColmaxCtas = 8;
}  // namespace

template <typename T>
__global__ void __launch_bounds__(kColmaxThreads)
k_colmax(const T *__restrict__ Y, long ld, long nd, unsigned *b)
{
    __shared__ unsigned red[kColmaxThreads / 32];
    const T *Yc = Y + (long)blockIdx.y * ld;
    constexpr long span = (long)kColmaxThreads * kColmaxPer;
    unsigned m = 0u;
    for (long base = (long)blockIdx.x * span + threadIdx.x; base < nd;
         base += (long)gridDim.x * span) {
#pragma unroll
        for (int t = 0; t < kColmaxPer; ++t) {
            const long p = base + (long)t * kColmaxThreads;
            if (p < nd) m = max(m, abs_hi_word(Yc[p]));
        }
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kColmaxThreads / 32; ++w) m = max(m, red[w]);
        if (m) raise_bound(b + blockIdx.y, m);
    }
}

template <typename T>
static cudaError_t colmax_launch(const T *Y, int ncols, long ld, long nd, unsigned *b,
                                 cudaStream_t st)
{
    if (ncols <= 0 || nd <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    const long per = (long)kColmaxThreads * kColmaxPer;
    const long chunks = (nd + per - 1) / per;
    dim3 grid((unsigned)(chunks < kColmaxCtas ? chunks : kColmaxCtas), (unsigned)ncols);
    k_colmax<T><<<grid, kColmaxThreads, 0, st>>>(Y, ld, nd, b);
    note_launch();
    return cudaGetLastError();
}

cudaError_t colmax_f64(const double *Y, int ncols, long ld, long nd, unsigned *b,
                       cudaStream_t st)
{
    return colmax_launch<double>(Y, ncols, ld, nd, b, st);
}

cudaError_t colmax_f32(const float *Y, int ncols, long ld, long nd, unsigned *b,
                       cudaStream_t st)
{
    return colmax_launch<float>(Y, ncols, ld, nd, b, st);
}

}  // namespace sparc
