// stencil_df.cu -- the FP64 fused stencil step computed with FP32 pair ("double-float")
// arithmetic.
//
// Same operation and blocking as k_stencil in stencil.cu (Eq. FD:Laplacian with the
// weights of Eq. weightsLap, zero-Dirichlet boundaries, V_eff and the Chebyshev
// three-term recurrence of Algorithm ChebychevFilter, Sec. 3.4), for FP64 blocks. GB300
// issues FP64 at 1/64 of its FP32 rate (about 0.6e12 FP64 FMA/s against 37e12 FP32 FMA/s),
// so the native FP64 stencil (about 39 FP64 instructions per point) is bound by the FP64
// pipe at roughly 5% of HBM bandwidth. Here each FP64 value becomes a pair of FP32 values
// (hi, lo) with hi + lo = x to about 2^-48 relative, and the weighted sum runs in FP32
// with error-free transformations:
//   * split: hi = x truncated to 24 significant bits and lo = the remaining bits rounded
//     to FP32, both built with integer operations on the bit pattern (no FP64 pipe);
//   * the six neighbours of each radius are summed with Knuth's TwoSum on the hi parts,
//     the lo parts and the rounding errors collected in a second FP32 accumulator;
//   * each radius sum is scaled with Dekker's exact product (TwoProduct via FMA) and
//     added to the running sum with TwoSum, the error terms again going to the second
//     accumulator (the compensated dot product of Ogita, Rump & Oishi, "Dot2", 2005).
// Per point this leaves four FP64 operations: the centre coefficient alpha*V + c0, the
// recombination hi + lo, and the recurrence term -beta*Y_{j-1}. The rounding error is
// about 2^-48 of sum |terms| instead of FP64's 2^-53 per operation.
#include "df.cuh"
#include "internal.cuh"

namespace sparc {

struct DfCoef {
    float wh[kRadius + 1];  // weights of radius r split as wh + wl
    float wl[kRadius + 1];
    double c0, alpha, beta;
};

template <int BX, int BY>
__global__ void __launch_bounds__(BX *BY)
k_stencil_df(const double *__restrict__ Y, const double *Yprev, double *out,
             const double *__restrict__ V, int n0, int n1, int n2, long ld, int nzc, int zchunk,
             DfCoef cf)
{
    constexpr int R = kRadius;
    __shared__ float2 s[BY + 2 * R][BX + 2 * R];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int i = i0 + tx, j = j0 + ty;
    const int col = blockIdx.z / nzc;
    const int k0 = (blockIdx.z % nzc) * zchunk;
    const int k1 = min(n2, k0 + zchunk);
    const long plane = (long)n0 * n1;
    const double *Yc = Y + (long)col * ld;
    const double *Pc = Yprev ? Yprev + (long)col * ld : nullptr;
    double *Oc = out + (long)col * ld;
    const bool act = (i < n0) && (j < n1);
    const long pij = (long)i + (long)n0 * j;
    const float2 zero = make_float2(0.0f, 0.0f);

    float2 q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? split_double(Yc[pij + (long)kk * plane]) : zero;
    }
    for (int k = k0; k < k1; ++k) {
        const long pk = (long)k * plane;
        __syncthreads();
        s[ty + R][tx + R] = q[R];
        if (tx < R) {
            const int il = i0 - R + tx, ir = i0 + BX + tx;
            const bool okj = j < n1;
            s[ty + R][tx] = (okj && il >= 0) ? split_double(Yc[pk + il + (long)n0 * j]) : zero;
            s[ty + R][tx + BX + R] =
                (okj && ir < n0) ? split_double(Yc[pk + ir + (long)n0 * j]) : zero;
        }
        if (ty < R) {
            const int jt = j0 - R + ty, jb = j0 + BY + ty;
            const bool oki = i < n0;
            s[ty][tx + R] = (oki && jt >= 0) ? split_double(Yc[pk + i + (long)n0 * jt]) : zero;
            s[ty + BY + R][tx + R] =
                (oki && jb < n1) ? split_double(Yc[pk + i + (long)n0 * jb]) : zero;
        }
        __syncthreads();
        if (act) {
            const long p = pij + pk;
            // centre: (c0 + alpha V_p) y_p, coefficient formed in FP64 and split
            const float2 c = split_double(fma(cf.alpha, V[p], cf.c0));
            const float2 y = q[R];
            float ah = c.x * y.x;
            float al = fmaf(c.x, y.x, -ah);
            al = fmaf(c.x, y.y, al);
            al = fmaf(c.y, y.x, al);
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const float2 v[6] = {s[ty + R][tx + R + r], s[ty + R][tx + R - r],
                                     s[ty + R + r][tx + R], s[ty + R - r][tx + R], q[R + r],
                                     q[R - r]};
                float sh = v[0].x, sl = v[0].y;
#pragma unroll
                for (int u = 1; u < 6; ++u) {
                    float t, e;
                    two_sum(sh, v[u].x, t, e);
                    sh = t;
                    sl += e;
                    sl += v[u].y;
                }
                const float pr = cf.wh[r] * sh;
                const float pe = fmaf(cf.wh[r], sh, -pr);
                float t, e;
                two_sum(ah, pr, t, e);
                ah = t;
                al += e;
                al += pe;
                al = fmaf(cf.wh[r], sl, al);
                al = fmaf(cf.wl[r], sh, al);
            }
            double d = (double)ah + (double)al;
            if (Pc) d = fma(-cf.beta, Pc[p], d);
            Oc[p] = d;
        }
#pragma unroll
        for (int t = 0; t < 2 * R; ++t) q[t] = q[t + 1];
        const int kn = k + R + 1;
        q[2 * R] = (act && kn < n2) ? split_double(Yc[pij + (long)kn * plane]) : zero;
    }
}

cudaError_t stencil_f64_df(const DevHam &H, const double *Y, const double *Yprev, double *out,
                           int ncols, long ld, double alpha, double shift, double beta,
                           cudaStream_t st)
{
    constexpr int BX = 32, BY = 16;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    const StepCoef<double> d = make_coef(H, alpha, shift, beta);
    DfCoef cf;
    for (int r = 0; r <= kRadius; ++r) {
        cf.wh[r] = (float)d.w[r];
        cf.wl[r] = (float)(d.w[r] - (double)cf.wh[r]);
    }
    cf.c0 = d.c0;
    cf.alpha = d.alpha;
    cf.beta = d.beta;
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil_df<BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, H.V, H.n0, H.n1, H.n2, ld, nzc,
                                                 zchunk, cf);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
