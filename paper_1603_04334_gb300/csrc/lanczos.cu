// lanczos.cu -- spectral bounds for the Chebyshev filter (Sec. 4: the extremal
// eigenvalues of H come from a few iterations of the Lanczos method).
//
// Plain Lanczos on one vector, all scalars kept on the device (no host round trip per
// step):  w = H v_j;  alpha_j = <w, v_j>;  w -= alpha_j v_j + beta_{j-1} v_{j-1};
//         beta_j = ||w||;  v_{j+1} = w / beta_j.
// If beta_j is zero or not finite the iteration stops there (an invariant subspace was
// found); the remaining kernels see the stop flag and do nothing.
// Start vector: v0[p] = u(splitmix64(seed ^ p)) - 0.5 with u(z) = (z >> 11) 2^-53, the
// SplitMix64 generator as published by Vigna (mixing constants of Stafford's Mix13).
// Dot products are two-level fixed-order reductions, so results are reproducible.
#include "internal.cuh"

namespace sparc {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_lanczos_start(double *v, long n, unsigned long long seed)
{
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x)
        v[p] = (double)(splitmix64(seed ^ (unsigned long long)p) >> 11) *
                   (1.0 / 9007199254740992.0) - 0.5;
}

cudaError_t lanczos_start(double *v, long n, unsigned long long seed, cudaStream_t st)
{
    k_lanczos_start<<<152 * 8, 256, 0, st>>>(v, n, seed);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_dot_part(const double *__restrict__ x, const double *__restrict__ y, long n, double *part)
{
    __shared__ double red[8];
    double s = 0.0;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x)
        s += x[p] * y[p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_dot_final(const double *part, int nb, double *r)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        *r = t;
    }
}

cudaError_t dot_f64(const double *x, const double *y, long n, double *part, double *r,
                    cudaStream_t st)
{
    k_dot_part<<<kDotBlocks, 256, 0, st>>>(x, y, n, part);
    note_launch();
    k_dot_final<<<1, 256, 0, st>>>(part, kDotBlocks, r);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_scale_rsqrt(double *v, long n, const double *nrm2)
{
    const double f = 1.0 / sqrt(*nrm2);
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x)
        v[p] *= f;
}

cudaError_t scale_rsqrt(double *v, long n, const double *nrm2, cudaStream_t st)
{
    k_scale_rsqrt<<<152 * 8, 256, 0, st>>>(v, n, nrm2);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_lanczos_orth(double *w, const double *v, const double *vp, long n,
                               const double *alpha, const double *beta, int j, const int *stop)
{
    if (*stop) return;
    const double a = alpha[j];
    const double b = j > 0 ? beta[j - 1] : 0.0;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x)
        w[p] = w[p] - a * v[p] - b * vp[p];
}

cudaError_t lanczos_orth(double *w, const double *v, const double *vp, long n,
                         const double *alpha, const double *beta, int j, const int *stop,
                         cudaStream_t st)
{
    k_lanczos_orth<<<152 * 8, 256, 0, st>>>(w, v, vp, n, alpha, beta, j, stop);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_lanczos_beta(double *beta, int j, const double *nrm2, int *stop)
{
    if (*stop) return;
    const double b = sqrt(*nrm2);
    beta[j] = b;
    if (!(b > 0.0) || !isfinite(b)) *stop = j + 1;
}

cudaError_t lanczos_beta(double *beta, int j, const double *nrm2, int *stop, cudaStream_t st)
{
    k_lanczos_beta<<<1, 1, 0, st>>>(beta, j, nrm2, stop);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_lanczos_next(double *v, double *vp, const double *w, long n,
                               const double *beta, int j, const int *stop)
{
    if (*stop) return;
    const double f = 1.0 / beta[j];
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x) {
        vp[p] = v[p];
        v[p] = w[p] * f;
    }
}

cudaError_t lanczos_next(double *v, double *vp, const double *w, long n, const double *beta,
                         int j, const int *stop, cudaStream_t st)
{
    k_lanczos_next<<<152 * 8, 256, 0, st>>>(v, vp, w, n, beta, j, stop);
    note_launch();
    return cudaGetLastError();
}

// T (keff x keff, column-major) from alpha/beta; keff = steps completed.
__global__ void k_lanczos_tridiag(const double *alpha, const double *beta, int k, const int *stop,
                                  double *T, int *keff)
{
    const int m = *stop ? *stop : k;
    if (threadIdx.x == 0) *keff = m;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int i = t % m, j = t / m;
        double v = 0.0;
        if (i == j) v = alpha[i];
        else if (i == j + 1) v = beta[j];
        else if (j == i + 1) v = beta[i];
        T[t] = v;
    }
}

cudaError_t lanczos_tridiag(const double *alpha, const double *beta, int k, const int *stop,
                            double *T, int *keff, cudaStream_t st)
{
    k_lanczos_tridiag<<<1, 256, 0, st>>>(alpha, beta, k, stop, T, keff);
    note_launch();
    return cudaGetLastError();
}

// out[0] = theta_min; out[1] = max(1.01 theta_max, theta_max + |beta_last s_last|).
__global__ void k_lanczos_final(const double *ev, const double *Q, const double *beta, int k,
                                const int *keff, double *out)
{
    const int m = *keff;
    const double tmax = ev[m - 1];
    const double s = Q[(m - 1) + (long)(m - 1) * m];
    const double g = tmax + fabs(beta[m - 1] * s);
    const double b = 1.01 * tmax;
    out[0] = ev[0];
    out[1] = b > g ? b : g;
}

cudaError_t lanczos_bounds_final(const double *ev, const double *Q, const double *beta, int k,
                                 const int *keff, double *out, cudaStream_t st)
{
    k_lanczos_final<<<1, 1, 0, st>>>(ev, Q, beta, k, keff, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
