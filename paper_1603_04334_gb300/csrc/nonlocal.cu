// nonlocal.cu -- Kleinman-Bylander nonlocal operator, Eq. (non-localPS:FD), Sec. 3.1:
//   V_nl f = h^3 sum_J sum_lm gamma_Jlm chi_Jlm (chi_Jlm^T f),
// applied matrix-free (Sec. 3.1) in two deterministic passes:
//   project: C_Jlm,c = sum_{s in supp(J)} chi_Jlm(s) Y(s, c)       (gather + 4 x nsup x ncols)
//   scatter: out(p, c) += alpha sum_{e at p} sum_lm gchi(e, lm) C_atom(e)lm,c
// with gchi = h^3 gamma chi precomputed at setup. The scatter walks the node -> entries
// inverse map (entries of a node in ascending order), so no atomics are used and the
// result does not depend on scheduling.
#include "df.cuh"
#include "internal.cuh"

namespace sparc {

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per (atom, column block of CB). Each thread accumulates 4*CB partial sums over
// a strided share of the atom's support; the block reduces them in a fixed order.
template <typename T, typename TC, int CB, int NT>
__global__ void __launch_bounds__(NT)
k_project(const T *__restrict__ Y, long ld, int ncols, const int *__restrict__ atom_ptr,
          const int *__restrict__ idx, const TC *__restrict__ chi, TC *__restrict__ C, TC alpha)
{
    __shared__ TC red[NT / 32][4 * CB];
    const int J = blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int b = atom_ptr[J], e = atom_ptr[J + 1];
    TC acc[4][CB];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) acc[l][cb] = (TC)0;
    for (int s = b + threadIdx.x; s < e; s += NT) {
        const long p = idx[s];
        const TC x0 = chi[4 * (long)s], x1 = chi[4 * (long)s + 1], x2 = chi[4 * (long)s + 2],
                 x3 = chi[4 * (long)s + 3];
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            if (c0 + cb < ncols) {
                const TC y = (TC)Y[p + (long)(c0 + cb) * ld];
                acc[0][cb] += x0 * y;
                acc[1][cb] += x1 * y;
                acc[2][cb] += x2 * y;
                acc[3][cb] += x3 * y;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const TC v = warp_sum(acc[l][cb]);
            if (lane == 0) red[wid][l * CB + cb] = v;
        }
    __syncthreads();
    if (threadIdx.x < 4 * CB) {
        const int l = threadIdx.x / CB, cb = threadIdx.x % CB;
        TC v = (TC)0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) v += red[w][threadIdx.x];
        if (c0 + cb < ncols) C[(long)(J * 4 + l) * ncols + c0 + cb] = alpha * v;
    }
}

template <typename T, typename TC>
static cudaError_t project(const DevHam &H, const T *Y, int ncols, long ld, const TC *chi,
                           TC *C, TC alpha, cudaStream_t st)
{
    if (H.natoms == 0 || ncols <= 0) return cudaSuccess;
    constexpr int CB = 8, NT = 256;
    dim3 grid(H.natoms, (ncols + CB - 1) / CB);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_project<T, TC, CB, NT><<<grid, NT, 0, st>>>(Y, ld, ncols, H.atom_ptr, H.idx, chi, C, alpha);
    note_launch();
    return cudaGetLastError();
}

cudaError_t project_f32(const DevHam &H, const float *Y, int ncols, long ld, double alpha,
                        float *C, cudaStream_t st)
{
    return project<float, float>(H, Y, ncols, ld, H.chi_f, C, (float)alpha, st);
}
cudaError_t project_f32in_f64(const DevHam &H, const float *Y, int ncols, long ld, double *C,
                              cudaStream_t st)
{
    return project<float, double>(H, Y, ncols, ld, H.chi, C, 1.0, st);
}

// ---- FP64 blocks in FP32-pair arithmetic (see df.cuh) ----------------------------------
// Projection with compensated products; each thread's partial sums over its share of the
// support are combined across the CTA with pair additions (TwoSum). The result is written
// as FP32 pairs, scaled by `alpha` (the filter step's factor), for the pair scatter.
template <int CB, int NT>
__global__ void __launch_bounds__(NT)
k_project_df(const double *__restrict__ Y, long ld, int ncols, const int *__restrict__ atom_ptr,
             const int *__restrict__ idx, const float2 *__restrict__ chi, float2 *__restrict__ C,
             float alh, float all)
{
    __shared__ float2 red[NT / 32][4 * CB];
    const int J = blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int b = atom_ptr[J], e = atom_ptr[J + 1];
    float sh[4][CB], sl[4][CB];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) sh[l][cb] = sl[l][cb] = 0.0f;
    for (int s = b + threadIdx.x; s < e; s += NT) {
        const long p = idx[s];
        float2 x[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) x[l] = chi[4 * (long)s + l];
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            if (c0 + cb < ncols) {
                const float2 y = split_double(Y[p + (long)(c0 + cb) * ld]);
#pragma unroll
                for (int l = 0; l < 4; ++l) mac(x[l], y, sh[l][cb], sl[l][cb]);
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            float h = sh[l][cb], lo = sl[l][cb];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
                const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                float t, err;
                two_sum(h, h2, t, err);
                h = t;
                lo = (lo + l2) + err;
            }
            if (lane == 0) red[wid][l * CB + cb] = make_float2(h, lo);
        }
    __syncthreads();
    if (threadIdx.x < 4 * CB) {
        const int l = threadIdx.x / CB, cb = threadIdx.x % CB;
        float h = 0.0f, lo = 0.0f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            const float2 v = red[w][threadIdx.x];
            float t, err;
            two_sum(h, v.x, t, err);
            h = t;
            lo = (lo + v.y) + err;
        }
        // alpha * (h + lo), renormalised
        float ph = 0.0f, pl = 0.0f;
        mac(make_float2(h, lo), make_float2(alh, all), ph, pl);
        float t, err;
        two_sum(ph, pl, t, err);
        if (c0 + cb < ncols) C[(long)(J * 4 + l) * ncols + c0 + cb] = make_float2(t, err);
    }
}

cudaError_t project_f64_df(const DevHam &H, const double *Y, int ncols, long ld, double alpha,
                           float2 *C, cudaStream_t st)
{
    if (H.natoms == 0 || ncols <= 0) return cudaSuccess;
    constexpr int CB = 8, NT = 256;
    dim3 grid(H.natoms, (ncols + CB - 1) / CB);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    const float alh = (float)alpha, all = (float)(alpha - (double)alh);
    k_project_df<CB, NT><<<grid, NT, 0, st>>>(Y, ld, ncols, H.atom_ptr, H.idx, H.chi_df, C, alh,
                                              all);
    note_launch();
    return cudaGetLastError();
}

// Standalone FP64 scatter (used where H is applied in FP64 to an FP32 block; the filter
// steps fuse the scatter into the stencil kernels). A thread owns one covered node and
// walks a strided subset of the columns, so the node's entry data stays in L1; the 32
// threads of a warp hold 32 consecutive covered nodes of the same column.
__global__ void __launch_bounds__(256)
k_scatter_f64(double *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
              const int *__restrict__ uniq_ptr, const int *__restrict__ ent_list,
              const int *__restrict__ ent_atom, const double *__restrict__ gchi,
              const double *__restrict__ C, double alpha)
{
    const long u = (long)blockIdx.x * 32 + threadIdx.x;
    if (u >= nuniq) return;
    const long node = uniq_node[u];
    const int q0 = uniq_ptr[u], q1 = uniq_ptr[u + 1];
    for (int c = threadIdx.y; c < ncols; c += blockDim.y) {
        double v = 0.0;
        for (int q = q0; q < q1; ++q) {
            const int e = ent_list[q];
            const int J = ent_atom[e];
#pragma unroll
            for (int l = 0; l < 4; ++l)
                v += gchi[4 * (long)e + l] * C[(long)(J * 4 + l) * ncols + c];
        }
        double *o = out + node + (long)c * ld;
        *o = *o + alpha * v;
    }
}

// FP32 blocks: Cs already holds alpha chi^T Y (FP32); same layout as k_scatter_f64.
__global__ void __launch_bounds__(256)
k_scatter_f32(float *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
              const int *__restrict__ uniq_ptr, const int *__restrict__ nl_atom,
              const float *__restrict__ g, const float *__restrict__ Cs)
{
    const long u = (long)blockIdx.x * 32 + threadIdx.x;
    if (u >= nuniq) return;
    const long node = uniq_node[u];
    const int q0 = uniq_ptr[u], q1 = uniq_ptr[u + 1];
    for (int c = threadIdx.y; c < ncols; c += blockDim.y) {
        float v = 0.0f;
        for (int q = q0; q < q1; ++q) {
            const float *cs = Cs + (long)nl_atom[q] * 4 * ncols + c;
#pragma unroll
            for (int l = 0; l < 4; ++l) v += g[4L * q + l] * cs[(long)l * ncols];
        }
        float *o = out + node + (long)c * ld;
        *o = *o + v;
    }
}

cudaError_t scatter_f32(const DevHam &H, const float *Cs, float *out, int ncols, long ld,
                        cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((H.nuniq + 31) / 32)), block(32, 8);
    k_scatter_f32<<<grid, block, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                          H.nl_atom, H.nl_gf, Cs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scatter_f64(const DevHam &H, const double *C, double *out, int ncols, long ld,
                        double alpha, cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((H.nuniq + 31) / 32)), block(32, 8);
    k_scatter_f64<<<grid, block, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                          H.ent_list, H.ent_atom, H.gchi, C, alpha);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
