// stencil.cu -- fused local Hamiltonian + Chebyshev three-term step.
//
// One launch computes, for every node p and column c,
//   out = alpha * ( (-1/2 ks L_h + V_eff - shift) Y )(p) - beta * Yprev(p),
// with L_h the radius-6 central stencil of Eq. (FD:Laplacian) (weights Eq. weightsLap,
// Sec. 3.1) and zero-Dirichlet boundaries (values outside the grid are 0, Sec. 3.1).
// alpha = 1, shift = 0, beta = 0 is the local part of H X; the filter of Algorithm
// ChebychevFilter (Sec. 3.4) uses alpha = 2 sigma_j / e, shift = c, beta =
// sigma_{j-1} sigma_j and writes Y_{j+1} in place over Y_{j-1}.
//
// Layout: column-major block, column c at c*ld, node p = i + n0 (j + n1 k).
// Blocking: a CTA owns a BX x BY tile of (i, j) for one column and streams along k
// (2.5-D blocking). The thread's own z-line lives in a 13-deep register queue
// (k-6 .. k+6); the current plane with its radius-6 x/y halos is staged in shared
// memory, so each value is read from global memory once per tile plus halo.
#include "internal.cuh"

namespace sparc {

StepCoef<double> make_coef(const DevHam &H, double alpha, double shift, double beta)
{
    StepCoef<double> c{};
    const double ks = -0.5 * H.kscale;
    for (int r = 1; r <= kRadius; ++r) c.w[r] = alpha * ks * H.w[r];
    c.w[0] = 0.0;
    c.c0 = alpha * ks * 6.0 * H.w[0] - alpha * shift;
    c.alpha = alpha;
    c.beta = beta;
    return c;
}

template <typename TC>
static StepCoef<TC> cast_coef(const StepCoef<double> &d)
{
    StepCoef<TC> c;
    for (int r = 0; r <= kRadius; ++r) c.w[r] = (TC)d.w[r];
    c.c0 = (TC)d.c0;
    c.alpha = (TC)d.alpha;
    c.beta = (TC)d.beta;
    return c;
}

// One tile: nodes (i0 .. i0+BX-1, j0 .. j0+BY-1, k0 .. k1-1) of one column (Yc, Pc, Oc
// point at the column). Ends with a CTA barrier, so the caller may reuse the shared
// memory for its next tile.
template <typename T, typename TO, typename TC, int BX, int BY>
__device__ __forceinline__ void stencil_tile(const T *__restrict__ Yc, const TO *Pc, TO *Oc,
                                             const TC *__restrict__ V, int n0, int n1, int n2,
                                             int i0, int j0, int k0, int k1,
                                             const StepCoef<TC> &cf)
{
    constexpr int R = kRadius;
    // plane k is read from s[b] while plane k+1 is staged into s[b ^ 1] (one barrier per
    // plane; the global loads of plane k+1 are in flight during the compute of plane k)
    __shared__ TC s[2][BY + 2 * R][BX + 2 * R];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx, j = j0 + ty;
    const long plane = (long)n0 * n1;
    const bool act = (i < n0) && (j < n1);
    const long pij = (long)i + (long)n0 * j;
    const bool hx = tx < R, hy = ty < R;
    const int il = i0 - R + tx, ir = i0 + BX + tx, jt = j0 - R + ty, jb = j0 + BY + ty;
    const bool okl = hx && j < n1 && il >= 0, okr = hx && j < n1 && ir < n0;
    const bool okt = hy && i < n0 && jt >= 0, okb = hy && i < n0 && jb < n1;
    const long offl = il + (long)n0 * j, offr = ir + (long)n0 * j;
    const long offt = i + (long)n0 * jt, offb = i + (long)n0 * jb;

    TC q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? (TC)Yc[pij + (long)kk * plane] : (TC)0;
    }
    {
        const long pk = (long)k0 * plane;
        s[0][ty + R][tx + R] = q[R];
        if (hx) {
            s[0][ty + R][tx] = okl ? (TC)Yc[pk + offl] : (TC)0;
            s[0][ty + R][tx + BX + R] = okr ? (TC)Yc[pk + offr] : (TC)0;
        }
        if (hy) {
            s[0][ty][tx + R] = okt ? (TC)Yc[pk + offt] : (TC)0;
            s[0][ty + BY + R][tx + R] = okb ? (TC)Yc[pk + offb] : (TC)0;
        }
    }
    TC vcur = act ? V[pij + (long)k0 * plane] : (TC)0;
    TC pcur = (act && Pc) ? (TC)Pc[pij + (long)k0 * plane] : (TC)0;
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const int b = (k - k0) & 1;
        const long pk = (long)k * plane;
        const bool more = k + 1 < k1;
        const long pk1 = pk + plane;
        T gl = 0, gr = 0, gt = 0, gb = 0, gq = 0;
        TC vnext = 0, pnext = 0;
        if (more) {
            if (okl) gl = Yc[pk1 + offl];
            if (okr) gr = Yc[pk1 + offr];
            if (okt) gt = Yc[pk1 + offt];
            if (okb) gb = Yc[pk1 + offb];
            if (act) {
                vnext = V[pij + pk1];
                if (Pc) pnext = (TC)Pc[pij + pk1];
            }
        }
        const int kn = k + R + 1;
        if (act && kn < n2) gq = Yc[pij + (long)kn * plane];
        if (act) {
            TC acc = (cf.c0 + cf.alpha * vcur) * q[R];
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const TC t = (s[b][ty + R][tx + R + r] + s[b][ty + R][tx + R - r])
                           + (s[b][ty + R + r][tx + R] + s[b][ty + R - r][tx + R])
                           + (q[R + r] + q[R - r]);
                acc += cf.w[r] * t;
            }
            if (Pc) acc -= cf.beta * pcur;
            Oc[pij + pk] = (TO)acc;
        }
#pragma unroll
        for (int t = 0; t < 2 * R; ++t) q[t] = q[t + 1];
        q[2 * R] = (TC)gq;
        vcur = vnext;
        pcur = pnext;
        if (more) {
            s[b ^ 1][ty + R][tx + R] = q[R];
            if (hx) {
                s[b ^ 1][ty + R][tx] = (TC)gl;
                s[b ^ 1][ty + R][tx + BX + R] = (TC)gr;
            }
            if (hy) {
                s[b ^ 1][ty][tx + R] = (TC)gt;
                s[b ^ 1][ty + BY + R][tx + R] = (TC)gb;
            }
        }
        __syncthreads();
    }
}

template <typename T, typename TO, typename TC, int BX, int BY>
__global__ void __launch_bounds__(BX *BY)
k_stencil(const T *Y, const TO *Yprev, TO *out, const TC *__restrict__ V, int n0, int n1, int n2,
          long ld, int nzc, int zchunk, StepCoef<TC> cf)
{
    const int col = blockIdx.z / nzc;
    const int k0 = (blockIdx.z % nzc) * zchunk;
    const int k1 = min(n2, k0 + zchunk);
    stencil_tile<T, TO, TC, BX, BY>(Y + (long)col * ld, Yprev ? Yprev + (long)col * ld : nullptr,
                                    out + (long)col * ld, V, n0, n1, n2, blockIdx.x * BX,
                                    blockIdx.y * BY, k0, k1, cf);
}

// Work-list form for a batch of clusters: each CTA walks the items (cluster, column, tile,
// z range) with a grid stride; a cluster's pointers, sizes and step coefficients come from
// its BatchStencil entry.
template <int BX, int BY>
__global__ void __launch_bounds__(BX *BY)
k_batch_stencil(const BatchItem *__restrict__ items, int nitems, const BatchStencil *cs)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchStencil &C = cs[w.cluster];
        const long off = (long)w.col * C.ld;
        stencil_tile<float, float, float, BX, BY>(C.Y + off, C.Yprev ? C.Yprev + off : nullptr,
                                                  C.out + off, C.V, C.n0, C.n1, C.n2, w.a * BX,
                                                  w.b * BY, w.k0, w.k1, C.cf);
    }
}

// Picks the number of z-chunks so that small problems still fill the 152 SMs.
void stencil_z_split(int n2, long tiles, int ncols, int &nzc, int &zchunk)
{
    const long want = 152L * 8;
    long per = tiles * ncols;
    nzc = 1;
    while (per * nzc < want && n2 / (nzc * 2) >= 16) nzc *= 2;
    while ((long)nzc * ncols > 65535) nzc /= 2;
    if (nzc < 1) nzc = 1;
    zchunk = (n2 + nzc - 1) / nzc;
}

template <typename T, typename TO, typename TC>
static cudaError_t launch(const DevHam &H, const T *Y, const TO *Yprev, TO *out, const TC *V,
                          int ncols, long ld, const StepCoef<double> &cd, cudaStream_t st)
{
    constexpr int BX = 32, BY = 8;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil<T, TO, TC, BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, V, H.n0, H.n1, H.n2,
                                                         ld, nzc, zchunk, cast_coef<TC>(cd));
    note_launch();
    return cudaGetLastError();
}

int batch_stencil_shapes() { return 3; }
void batch_stencil_tile(int shape, int &bx, int &by)
{
    bx = shape == 2 ? 64 : 32;
    by = shape == 1 ? 16 : 8;
}

cudaError_t batch_stencil(int shape, const BatchItem *items, int nitems, const BatchStencil *cs,
                          int grid, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    switch (shape) {
    case 0: k_batch_stencil<32, 8><<<grid, dim3(32, 8), 0, st>>>(items, nitems, cs); break;
    case 1: k_batch_stencil<32, 16><<<grid, dim3(32, 16), 0, st>>>(items, nitems, cs); break;
    case 2: k_batch_stencil<64, 8><<<grid, dim3(64, 8), 0, st>>>(items, nitems, cs); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

StepCoef<float> coef_f32(const DevHam &H, double alpha, double shift, double beta)
{
    return cast_coef<float>(make_coef(H, alpha, shift, beta));
}

cudaError_t stencil_f32(const DevHam &H, const float *Y, const float *Yprev, float *out,
                        int ncols, long ld, double alpha, double shift, double beta,
                        cudaStream_t st)
{
    if (stencil_tma_ok(H, Y, Yprev, out, ld))
        return stencil_f32_tma(H, Y, Yprev, out, ncols, ld,
                               cast_coef<float>(make_coef(H, alpha, shift, beta)), H.err, st);
    return launch<float, float, float>(H, Y, Yprev, out, H.Vf, ncols, ld,
                                       make_coef(H, alpha, shift, beta), st);
}

}  // namespace sparc
