// nonlocal.cu -- Kleinman-Bylander nonlocal operator, Eq. (non-localPS:FD), Sec. 3.1:
//   V_nl f = h^3 sum_J sum_lm gamma_Jlm chi_Jlm (chi_Jlm^T f),
// applied matrix-free (Sec. 3.1) in two deterministic passes:
//   project: C_Jlm,c = sum_{s in supp(J)} chi_Jlm(s) Y(s, c)       (gather + 4 x nsup x ncols)
//   scatter: out(p, c) += alpha sum_{e at p} sum_lm gchi(e, lm) C_atom(e)lm,c
// with gchi = h^3 gamma chi precomputed at setup. The scatter walks the node -> entries
// inverse map (entries of a node in ascending order), so no atomics are used and the
// result does not depend on scheduling.
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
          const int *__restrict__ idx, const TC *__restrict__ chi, TC *__restrict__ C)
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
        if (c0 + cb < ncols) C[(long)(J * 4 + l) * ncols + c0 + cb] = v;
    }
}

template <typename T, typename TC>
static cudaError_t project(const DevHam &H, const T *Y, int ncols, long ld, const TC *chi,
                           TC *C, cudaStream_t st)
{
    if (H.natoms == 0 || ncols <= 0) return cudaSuccess;
    constexpr int CB = 8, NT = 256;
    dim3 grid(H.natoms, (ncols + CB - 1) / CB);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_project<T, TC, CB, NT><<<grid, NT, 0, st>>>(Y, ld, ncols, H.atom_ptr, H.idx, chi, C);
    note_launch();
    return cudaGetLastError();
}

cudaError_t project_f64(const DevHam &H, const double *Y, int ncols, long ld, double *C,
                        cudaStream_t st)
{
    return project<double, double>(H, Y, ncols, ld, H.chi, C, st);
}
cudaError_t project_f32(const DevHam &H, const float *Y, int ncols, long ld, float *C,
                        cudaStream_t st)
{
    return project<float, float>(H, Y, ncols, ld, H.chi_f, C, st);
}
cudaError_t project_f32in_f64(const DevHam &H, const float *Y, int ncols, long ld, double *C,
                              cudaStream_t st)
{
    return project<float, double>(H, Y, ncols, ld, H.chi, C, st);
}

// One thread per (covered node, column): columns on grid.y, nodes on x.
template <typename TO, typename TC>
__global__ void __launch_bounds__(256)
k_scatter(TO *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
          const int *__restrict__ uniq_ptr, const int *__restrict__ ent_list,
          const int *__restrict__ ent_atom, const TC *__restrict__ gchi,
          const TC *__restrict__ C, TC alpha)
{
    const long u = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (u >= nuniq) return;
    TC v = (TC)0;
    for (int q = uniq_ptr[u]; q < uniq_ptr[u + 1]; ++q) {
        const int e = ent_list[q];
        const int J = ent_atom[e];
#pragma unroll
        for (int l = 0; l < 4; ++l) v += gchi[4 * (long)e + l] * C[(long)(J * 4 + l) * ncols + c];
    }
    TO *o = out + (long)uniq_node[u] + (long)c * ld;
    *o = (TO)((TC)*o + alpha * v);
}

template <typename TO, typename TC>
static cudaError_t scatter(const DevHam &H, const TC *gchi, const TC *C, TO *out, int ncols,
                           long ld, double alpha, cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((H.nuniq + 255) / 256), ncols);
    k_scatter<TO, TC><<<grid, 256, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                            H.ent_list, H.ent_atom, gchi, C, (TC)alpha);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scatter_f64(const DevHam &H, const double *C, double *out, int ncols, long ld,
                        double alpha, cudaStream_t st)
{
    return scatter<double, double>(H, H.gchi, C, out, ncols, ld, alpha, st);
}
cudaError_t scatter_f32(const DevHam &H, const float *C, float *out, int ncols, long ld,
                        double alpha, cudaStream_t st)
{
    return scatter<float, float>(H, H.gchi_f, C, out, ncols, ld, alpha, st);
}

}  // namespace sparc
