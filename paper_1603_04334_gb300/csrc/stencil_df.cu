// stencil_df.cu -- the FP64 fused stencil step computed with FP32 pair ("double-float")
// arithmetic.
//
// Same operation and blocking as k_stencil in stencil.cu (Eq. FD:Laplacian with the
// weights of Eq. weightsLap, zero-Dirichlet boundaries, V_eff and the Chebyshev
// three-term recurrence of Algorithm ChebychevFilter, Sec. 3.4), for FP64 blocks. GB300
// issues FP64 at 1/64 of its FP32 rate (about 0.6e12 FP64 FMA/s against 37e12 FP32 FMA/s),
// so the native FP64 stencil (about 39 FP64 instructions per point) is bound by the FP64
// pipe at roughly 5% of HBM bandwidth. Here each FP64 value becomes a pair of FP32 values
// (hi, lo) with hi + lo = x to about 2^-48 relative (split_double, df.cuh), and the
// weighted sum runs in FP32 with error-free transformations:
//   * the six neighbours of each radius are summed pairwise with Knuth's TwoSum on the hi
//     parts, the lo parts and the rounding errors going to a second FP32 accumulator;
//   * each radius sum is scaled with Dekker's exact product (TwoProduct via FMA) and
//     added to the running sum with TwoSum, the error terms again going to the second
//     accumulator (the compensated dot product of Ogita, Rump & Oishi, "Dot2", 2005);
//   * the centre coefficient c0 + alpha V_p (V_eff kept as pairs) and the recurrence term
//     -beta Y_{j-1} are formed in the same pair arithmetic.
// Only the final hi + lo recombination uses the FP64 pipe (one add per point); the pair
// parts are widened to FP64 with integer bit operations. The rounding error is about
// 2^-48 of sum |terms| instead of FP64's 2^-53 per operation.
#include "df.cuh"
#include "internal.cuh"

namespace sparc {

struct DfCoef {
    float wh[kRadius + 1];  // weights of radius r split as wh + wl
    float wl[kRadius + 1];
    float c0h, c0l;         // centre constant c0 as a pair
    float ah, al;           // alpha as a pair
    float bh, bl;           // -beta as a pair
};

// (sh, sl) += (vh, vl) * (wh, wl), with sh updated by TwoSum and all error terms in sl.
__device__ __forceinline__ void acc_mul(float vh, float vl, float wh, float wl, float &sh,
                                        float &sl)
{
    const float p = wh * vh;
    const float pe = fmaf(wh, vh, -p);
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl += e;
    sl += pe;
    sl = fmaf(wh, vl, sl);
    sl = fmaf(wl, vh, sl);
}

// (a.x + a.y) + (b.x + b.y) as a pair whose lo part is not renormalised
__device__ __forceinline__ float2 pair_add(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    return make_float2(s, (a.y + b.y) + e);
}

// TI is the input block's type: FP64, or FP32 (an FP32 value is the exact pair (y, 0); the
// mixed-precision Rayleigh-Ritz step applies H in FP64 to the FP32 filtered block).
template <typename TI, int BX, int BY>
__global__ void __launch_bounds__(BX *BY)
k_stencil_df(const TI *__restrict__ Y, const double *Yprev, double *out,
             const float2 *__restrict__ Vdf, int n0, int n1, int n2, long ld, int nzc, int zchunk,
             DfCoef cf)
{
    constexpr int R = kRadius;
    // plane k is read from s[b] while plane k+1 is staged into s[b ^ 1]: one barrier per
    // plane, and the global loads of plane k+1 are in flight while plane k is computed
    __shared__ float2 s[2][BY + 2 * R][BX + 2 * R];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int i = i0 + tx, j = j0 + ty;
    const int col = blockIdx.z / nzc;
    const int k0 = (blockIdx.z % nzc) * zchunk;
    const int k1 = min(n2, k0 + zchunk);
    const long plane = (long)n0 * n1;
    const TI *Yc = Y + (long)col * ld;
    const double *Pc = Yprev ? Yprev + (long)col * ld : nullptr;
    double *Oc = out + (long)col * ld;
    const bool act = (i < n0) && (j < n1);
    const long pij = (long)i + (long)n0 * j;
    const float2 zero = make_float2(0.0f, 0.0f);
    // halo duties of this thread: x halos (tx < R) and y halos (ty < R)
    const bool hx = tx < R, hy = ty < R;
    const int il = i0 - R + tx, ir = i0 + BX + tx, jt = j0 - R + ty, jb = j0 + BY + ty;
    const bool okl = hx && j < n1 && il >= 0, okr = hx && j < n1 && ir < n0;
    const bool okt = hy && i < n0 && jt >= 0, okb = hy && i < n0 && jb < n1;
    const long offl = il + (long)n0 * j, offr = ir + (long)n0 * j;
    const long offt = i + (long)n0 * jt, offb = i + (long)n0 * jb;

    float2 q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? split_double(Yc[pij + (long)kk * plane]) : zero;
    }
    {
        const long pk = (long)k0 * plane;
        s[0][ty + R][tx + R] = q[R];
        if (hx) {
            s[0][ty + R][tx] = okl ? split_double(Yc[pk + offl]) : zero;
            s[0][ty + R][tx + BX + R] = okr ? split_double(Yc[pk + offr]) : zero;
        }
        if (hy) {
            s[0][ty][tx + R] = okt ? split_double(Yc[pk + offt]) : zero;
            s[0][ty + BY + R][tx + R] = okb ? split_double(Yc[pk + offb]) : zero;
        }
    }
    float2 vcur = act ? Vdf[pij + (long)k0 * plane] : zero;
    double pcur = (act && Pc) ? Pc[pij + (long)k0 * plane] : 0.0;
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const int b = (k - k0) & 1;
        const long pk = (long)k * plane;
        // loads for plane k+1 (and the queue entry k+R+1), consumed after the compute
        const bool more = k + 1 < k1;
        const long pk1 = pk + plane;
        TI gl = 0, gr = 0, gt = 0, gb = 0, gq = 0;
        double pnext = 0.0;
        float2 vnext = zero;
        if (more) {
            if (okl) gl = Yc[pk1 + offl];
            if (okr) gr = Yc[pk1 + offr];
            if (okt) gt = Yc[pk1 + offt];
            if (okb) gb = Yc[pk1 + offb];
            if (act) {
                vnext = Vdf[pij + pk1];
                if (Pc) pnext = Pc[pij + pk1];
            }
        }
        const int kn = k + R + 1;
        if (act && kn < n2) gq = Yc[pij + (long)kn * plane];
        if (act) {
            const long p = pij + pk;
            // centre coefficient cc = c0 + alpha V_p as a pair
            const float2 v = vcur;
            float ch = 0.0f, cl = 0.0f;
            acc_mul(v.x, v.y, cf.ah, cf.al, ch, cl);
            {
                float t, e;
                two_sum(ch, cf.c0h, t, e);
                ch = t;
                cl += e + cf.c0l;
            }
            // running sum (ah, al) starts with cc * y_p
            const float2 y = q[R];
            float ah = 0.0f, al = 0.0f;
            acc_mul(y.x, y.y, ch, cl, ah, al);
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const float2 t0 = pair_add(s[b][ty + R][tx + R + r], s[b][ty + R][tx + R - r]);
                const float2 t1 = pair_add(s[b][ty + R + r][tx + R], s[b][ty + R - r][tx + R]);
                const float2 t2 = pair_add(q[R + r], q[R - r]);
                const float2 t = pair_add(pair_add(t0, t1), t2);
                acc_mul(t.x, t.y, cf.wh[r], cf.wl[r], ah, al);
            }
            if (Pc) {
                const float2 pv = split_double(pcur);
                acc_mul(pv.x, pv.y, cf.bh, cf.bl, ah, al);
            }
            Oc[p] = pair_to_double(ah, al);
        }
#pragma unroll
        for (int t = 0; t < 2 * R; ++t) q[t] = q[t + 1];
        q[2 * R] = (act && kn < n2) ? split_double(gq) : zero;
        vcur = vnext;
        pcur = pnext;
        if (more) {
            s[b ^ 1][ty + R][tx + R] = q[R];
            if (hx) {
                s[b ^ 1][ty + R][tx] = okl ? split_double(gl) : zero;
                s[b ^ 1][ty + R][tx + BX + R] = okr ? split_double(gr) : zero;
            }
            if (hy) {
                s[b ^ 1][ty][tx + R] = okt ? split_double(gt) : zero;
                s[b ^ 1][ty + BY + R][tx + R] = okb ? split_double(gb) : zero;
            }
        }
        __syncthreads();
    }
}

static void split_host(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// Nonlocal scatter for FP64 blocks in pair arithmetic: out(p, c) += sum_{q at p} sum_l
// g(q, l) Cs(atom(q), l, c), Cs = alpha chi^T Y as pairs (k_project_df). A thread owns one
// covered node and a group of kScatCols columns; the grid's x dimension (dispatched first)
// runs over the covered nodes, so the CTAs resident at one time sweep consecutive nodes of
// the same columns (coalesced, DRAM-page-local read-modify-write of the output; the node's
// entries stay in L1). The pair sum is added to the FP64 output with one FP64 add.
namespace {
constexpr int kScatNodes = 256;
constexpr int kScatCols = 8;
}  // namespace

__global__ void __launch_bounds__(kScatNodes)
k_scatter_df(double *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
             const int *__restrict__ uniq_ptr, const int *__restrict__ nl_atom,
             const float2 *__restrict__ g, const float2 *__restrict__ Cs)
{
    const long u = (long)blockIdx.x * kScatNodes + threadIdx.x;
    if (u >= nuniq) return;
    const int c0 = blockIdx.y * kScatCols, c1 = min(ncols, c0 + kScatCols);
    const long node = uniq_node[u];
    const int q0 = uniq_ptr[u], q1 = uniq_ptr[u + 1];
    // all column sums first (coefficients from L1 / L2), then every output read is issued
    // before any store: kScatCols independent DRAM reads in flight per thread
    double v[kScatCols], x[kScatCols];
#pragma unroll
    for (int k = 0; k < kScatCols; ++k) {
        const int c = c0 + k;
        float vh = 0.0f, vl = 0.0f;
        if (c < c1) {
            for (int q = q0; q < q1; ++q) {
                const float2 *cs = Cs + (long)nl_atom[q] * 4 * ncols + c;
#pragma unroll
                for (int l = 0; l < 4; ++l) mac(g[4L * q + l], cs[(long)l * ncols], vh, vl);
            }
        }
        v[k] = pair_to_double(vh, vl);
    }
    double *o = out + node + (long)c0 * ld;
#pragma unroll
    for (int k = 0; k < kScatCols; ++k) x[k] = c0 + k < c1 ? o[(long)k * ld] : 0.0;
#pragma unroll
    for (int k = 0; k < kScatCols; ++k)
        if (c0 + k < c1) o[(long)k * ld] = x[k] + v[k];
}

cudaError_t scatter_f64_df(const DevHam &H, const float2 *Cs, double *out, int ncols, long ld,
                           cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((H.nuniq + kScatNodes - 1) / kScatNodes),
              (unsigned)((ncols + kScatCols - 1) / kScatCols));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_scatter_df<<<grid, kScatNodes, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                              H.nl_atom, H.nl_gdf, Cs);
    note_launch();
    return cudaGetLastError();
}

template <typename TI>
static cudaError_t stencil_df_launch(const DevHam &H, const TI *Y, const double *Yprev,
                                     double *out, int ncols, long ld, double alpha, double shift,
                                     double beta, cudaStream_t st)
{
    constexpr int BX = 32, BY = 16;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    const StepCoef<double> d = make_coef(H, alpha, shift, beta);
    DfCoef cf;
    for (int r = 0; r <= kRadius; ++r) split_host(d.w[r], cf.wh[r], cf.wl[r]);
    split_host(d.c0, cf.c0h, cf.c0l);
    split_host(d.alpha, cf.ah, cf.al);
    split_host(-d.beta, cf.bh, cf.bl);
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil_df<TI, BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, H.Vdf, H.n0, H.n1, H.n2, ld,
                                                     nzc, zchunk, cf);
    note_launch();
    return cudaGetLastError();
}

cudaError_t stencil_f64(const DevHam &H, const double *Y, const double *Yprev, double *out,
                        int ncols, long ld, double alpha, double shift, double beta,
                        cudaStream_t st)
{
    return stencil_df_launch<double>(H, Y, Yprev, out, ncols, ld, alpha, shift, beta, st);
}

cudaError_t stencil_f32in_f64(const DevHam &H, const float *Y, double *out, int ncols, long ld,
                              cudaStream_t st)
{
    return stencil_df_launch<float>(H, Y, nullptr, out, ncols, ld, 1.0, 0.0, 0.0, st);
}

__global__ void k_to_float_pair(const double *in, float2 *out, long n)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x)
        out[q] = split_double(in[q]);
}

cudaError_t to_float_pair(const double *in, float2 *out, long n, cudaStream_t st)
{
    k_to_float_pair<<<152 * 8, 256, 0, st>>>(in, out, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
