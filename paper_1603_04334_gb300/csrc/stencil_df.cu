// stencil_df.cu -- the FP64 fused stencil step on the integer, FP32 and FP64 pipes.
//
// Same operation and blocking as k_stencil in stencil.cu (Eq. FD:Laplacian with the
// weights of Eq. weightsLap, zero-Dirichlet boundaries, V_eff and the Chebyshev
// three-term recurrence of Algorithm ChebychevFilter, Sec. 3.4), for FP64 blocks. GB300
// issues FP64 at 1/64 of its FP32 rate, so a native FP64 stencil (37 FP64 multiply-adds
// per point) is bound by the FP64 pipe at a few per cent of HBM bandwidth. This kernel
// spends four FP64 operations per point:
//   * The Laplacian weights of radius n_o are rationals with one small common
//     denominator D (h^2 w_p = W_p / D, W_p integers, D = 831600 for n_o = 6), so
//     h^2 D L_h y = sum_p W_p S_p is an integer combination of the neighbour sums S_p.
//   * Every value of a column is put on a fixed-point grid: with |y| < 2^E over the
//     column (E from a per-column bound), y 2^(26-E) = d + r with d an integer truncated
//     toward zero (|d| < 2^26) and r the rest (|r| < 1, same sign, kept to 23 bits as
//     FP32).
//   * Each radius sums its six neighbours' d in int32 (exact: |sum| < 6 * 2^26) and
//     applies W_p with one 32 x 32 -> 64-bit integer multiply-add (exact); the r parts are
//     summed and weighted in FP32 and the FP32 sum is rounded to an integer. The total
//     T ~ h^2 D L_h y 2^(26-E) is an int64 below 2^51 in magnitude (sum |W_p| < 2^24.1),
//     converted to FP64 exactly by one FP64 add (the 1.5 * 2^52 offset).
//   * Three more FP64 operations finish the point: out = alpha g 2^(E-26) T +
//     [alpha (V_p - shift)] y_p - beta Y_{j-1}, g = (-1/2) ks / (D h^2), with
//     alpha (V - shift) formed once per launch (k_scaled_v) and y_p read again as FP64.
// Error: the truncation of r (2^-49 of the column's largest value per value) and the FP32
// rounding of the r sum (a few units of 2^(E-26), weighted by g ~ 1e-5 at h = 0.3): about
// 2^-40 of the column's largest value in the worst case, FP64 rounding elsewhere. A column
// whose bound is not finite (Inf or NaN anywhere in Y_j) gives NaN in every output value of
// the column. Each launch can raise the output's column bounds (atomicMax), which is how
// the filter hands the bound of Y_{j+1} to the next step without another pass over the
// block.
#include <type_traits>

#include "df.cuh"
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

struct FxCoef {
    int W[kRadius + 1];    // integer weights: W[0] three-dimensional centre, W[p] radius p
    float Wf[kRadius + 1]; // the same as FP32 (exact: |W| < 2^24)
    double ag;             // alpha (-1/2) ks / (D h^2)
    double mbeta;          // -beta
};

// A value on the column's grid: .x = d, .y = the bits of r (y 2^(26-E) = d + r, |y| < 2^E).
// From y = M 2^(e-1075) (M the 53-bit significand): N = M >> s with s = 1026 + E - e
// (s >= 4 when |y| < 2^E) holds d (N >> 23, below 2^26) and the next 23 bits (r); zero and
// subnormal y give 0; the sign is applied to both parts.
__device__ __forceinline__ int2 to_grid(double y, int E)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned hw = (unsigned)(b >> 32);
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned long long M =
        e ? ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) : 0ull;
    const unsigned long long N = M >> min(1026 + E - e, 63);
    const unsigned sg = hw & 0x80000000u;
    const int sm = (int)hw >> 31;  // 0 or -1
    const int d = ((int)(unsigned)(N >> 23) ^ sm) - sm;
    const float r = __uint_as_float(((unsigned)N & 0x7fffffu) | 0x3F800000u) - 1.0f;
    return make_int2(d, (int)(__float_as_uint(r) ^ sg));
}

// FP32 input: y = m 2^(e-150) (24-bit m) = (m 2^29) 2^(e-179); s = 130 + E - e.
__device__ __forceinline__ int2 to_grid(float y, int E)
{
    const unsigned u = __float_as_uint(y);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned long long M =
        e ? ((unsigned long long)((u & 0x7fffffu) | 0x800000u) << 29) : 0ull;
    const unsigned long long N = M >> min(130 + E - e, 63);
    const unsigned sg = u & 0x80000000u;
    const int sm = (int)u >> 31;
    const int d = ((int)(unsigned)(N >> 23) ^ sm) - sm;
    const float r = __uint_as_float(((unsigned)N & 0x7fffffu) | 0x3F800000u) - 1.0f;
    return make_int2(d, (int)(__float_as_uint(r) ^ sg));
}

__device__ __forceinline__ double as_f64(double y) { return y; }
__device__ __forceinline__ double as_f64(float y) { return (double)y; }

// An integer |t| < 2^51 as FP64, exactly: t added to the significand of 1.5 * 2^52 (whose
// unit in the last place is 1), then 1.5 * 2^52 subtracted.
__device__ __forceinline__ double int51_to_double(long long t)
{
    return __longlong_as_double(t + 0x4338000000000000ll) - 6755399441055744.0;
}

// TI is the input block's type: FP64, or FP32 (the mixed-precision Rayleigh-Ritz step
// applies H in FP64 to the FP32 filtered block). One thread per (x, y) node of a BX x BY
// tile walks the tile's z range of one column; the 13 planes around it stay in registers
// on the column's grid, the current plane's tile with its x and y halos in shared memory.
// The halo strips (2 R (BX + BY) nodes) are loaded and converted by all threads together,
// at most two nodes each, so no warp runs them as a divergent side branch. The next
// plane's halo values, queue entry, alpha (V - shift) and Y_{j-1} are loaded during the
// current plane's compute. u: the launch's alpha (V_eff - shift), Nd values.
template <typename TI, int BX, int BY>
__global__ void __launch_bounds__(BX *BY, 2)
k_stencil_df(const TI *__restrict__ Y, const double *Yprev, double *out,
             const double *__restrict__ u, int n0, int n1, int n2, long ld, int nzc, int zchunk,
             FxCoef cf, const unsigned *__restrict__ bY, unsigned *bOut)
{
    constexpr int R = kRadius, SX = BX + 2 * R, SY = BY + 2 * R, NT = BX * BY;
    constexpr int NH = 2 * R * (BX + BY);  // halo nodes of a plane
    static_assert(NH <= 2 * NT, "at most two halo nodes per thread");
    // plane k is read from buffer b while plane k+1 is staged into buffer b ^ 1: one barrier
    // per plane, and the global loads of plane k+1 are in flight while plane k is computed
    __shared__ int2 s[2 * SY * SX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int i = i0 + tx, j = j0 + ty;
    const int col = blockIdx.z / nzc;
    const int k0 = (blockIdx.z % nzc) * zchunk;
    const int k1 = min(n2, k0 + zchunk);
    const unsigned plane = (unsigned)n0 * (unsigned)n1;  // offsets in a column fit 32 bits
    // the column's offset in Y, Y_{j-1} and out (the base pointers stay kernel parameters)
    const long cb = (long)col * ld;
    const bool hasP = Yprev != nullptr;
    const bool act = (i < n0) && (j < n1);
    const unsigned pij = act ? (unsigned)i + (unsigned)n0 * (unsigned)j : 0u;
    const int2 zero = make_int2(0, 0);
    // the column's scale: grid values in units of 2^(EY-26)
    const unsigned uy = bY[col];
    const bool nonfinite = ((uy >> 20) & 0x7ffu) == 0x7ffu;
    const int EY = bound_exponent(uy);
    // alpha g 2^(EY-26); NaN for a column whose bound is not finite, which makes every output
    // of the column NaN without a test per point
    const double gs =
        nonfinite ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(cf.ag, EY - 26);
    // halo duties: nodes tid and tid + NT of the strips (left, right: R x BY each; top,
    // bottom: BX x R each); hs = shared-memory index (-1: none), hg = offset in the plane
    // (kNoNode: the node lies outside the grid and stays zero)
    constexpr unsigned kNoNode = 0xffffffffu;
    int hs[2];
    unsigned hg[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const int h = tid + v * NT;
        int sx, sy;
        if (h < 2 * R * BY) {
            const int side = h / (R * BY), rr = h % (R * BY);
            sy = R + rr / R;
            sx = side ? BX + R + rr % R : rr % R;
        } else {
            const int w = h - 2 * R * BY;
            const int side = w / (R * BX), rr = w % (R * BX);
            sx = R + rr % BX;
            sy = side ? BY + R + rr / BX : rr / BX;
        }
        const int gx = i0 - R + sx, gy = j0 - R + sy;
        hs[v] = h < NH ? sy * SX + sx : -1;
        const bool in = h < NH && gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
        hg[v] = in ? (unsigned)gx + (unsigned)n0 * (unsigned)gy : kNoNode;
    }
    const int me = (ty + R) * SX + tx + R;  // this thread's node in a plane buffer

    int2 q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? to_grid(Y[cb + pij + (unsigned)kk * plane], EY) : zero;
    }
    {
        const unsigned pk = (unsigned)k0 * plane;
        s[me] = q[R];
#pragma unroll
        for (int v = 0; v < 2; ++v)
            if (hs[v] >= 0) s[hs[v]] = hg[v] != kNoNode ? to_grid(Y[cb + hg[v] + pk], EY) : zero;
    }
    double ucur = act && k0 < k1 ? u[pij + (unsigned)k0 * plane] : 0.0;
    double pcur = act && hasP && k0 < k1 ? Yprev[cb + pij + (unsigned)k0 * plane] : 0.0;
    unsigned omax = 0u;
    __syncthreads();
    // The plane loop is unrolled 13 times, one copy per rotation of the z queue: in the
    // copy of phase PH, logical queue entry t (plane k - R + t) sits in q[(PH + t) % 13], so
    // the queue is never shifted.
    int k = k0;
    auto step = [&](auto phase) {
        constexpr int PH = decltype(phase)::value;
        constexpr int Q = 2 * R + 1;
        const int b = (k - k0) & 1;
        const unsigned pk = (unsigned)k * plane;
        // loads for plane k+1 (and the queue entry k+R+1), consumed after the compute
        const bool more = k + 1 < k1;
        const unsigned pk1 = pk + plane;
        TI g[2] = {0, 0}, gq = 0;
        double unext = 0.0, pnext = 0.0;
        if (more) {
#pragma unroll
            for (int v = 0; v < 2; ++v)
                if (hg[v] != kNoNode) g[v] = Y[cb + hg[v] + pk1];
            if (act) {
                unext = u[pij + pk1];
                if (hasP) pnext = Yprev[cb + pij + pk1];
            }
        }
        const int kn = k + R + 1;
        if (act && kn < n2) gq = Y[cb + pij + (unsigned)kn * plane];
        if (act) {
            const double yc = as_f64(Y[cb + pij + pk]);  // the point's own value (cached)
            // h^2 D L_h y in units of 2^(EY-26): exact integer sums of d, FP32 sums of r
            const int2 c = q[(PH + R) % Q];
            const int2 *row = s + b * (SY * SX) + me;
            long long A = (long long)cf.W[0] * c.x;
            float Rs = cf.Wf[0] * __int_as_float(c.y);
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const int2 xa = row[r], xb = row[-r], ya = row[r * SX], yb = row[-r * SX];
                const int2 za = q[(PH + R + r) % Q], zb = q[(PH + R - r) % Q];
                const int sd = (xa.x + xb.x + ya.x) + (yb.x + za.x + zb.x);
                const float sr = ((__int_as_float(xa.y) + __int_as_float(xb.y)) +
                                  (__int_as_float(ya.y) + __int_as_float(yb.y))) +
                                 (__int_as_float(za.y) + __int_as_float(zb.y));
                A += (long long)cf.W[r] * sd;
                Rs = fmaf(cf.Wf[r], sr, Rs);
            }
            const double T = int51_to_double(A + (long long)__float2int_rn(Rs));
            // pcur is 0 without Y_{j-1} (its loads are guarded), so the term needs no test
            const double o = fma(gs, T, fma(ucur, yc, cf.mbeta * pcur));
            omax = max(omax, abs_hi_word(o));
            out[cb + pij + pk] = o;
        }
        // plane k - R leaves the queue; its slot takes plane k + R + 1 (logical entry 2R
        // of the next phase), and the next phase's centre is plane k + 1
        q[PH % Q] = (act && kn < n2) ? to_grid(gq, EY) : zero;
        ucur = unext;
        pcur = pnext;
        if (more) {
            int2 *nb = s + (b ^ 1) * (SY * SX);
            nb[me] = q[(PH + 1 + R) % Q];
#pragma unroll
            for (int v = 0; v < 2; ++v)
                if (hs[v] >= 0) nb[hs[v]] = hg[v] != kNoNode ? to_grid(g[v], EY) : zero;
        }
        __syncthreads();
        ++k;
    };
#define SPARC_DF_STEP(P)                                                                 \
    if (k >= k1) break;                                                                  \
    step(std::integral_constant<int, P>{});
    for (;;) {
        SPARC_DF_STEP(0) SPARC_DF_STEP(1) SPARC_DF_STEP(2) SPARC_DF_STEP(3) SPARC_DF_STEP(4)
        SPARC_DF_STEP(5) SPARC_DF_STEP(6) SPARC_DF_STEP(7) SPARC_DF_STEP(8) SPARC_DF_STEP(9)
        SPARC_DF_STEP(10) SPARC_DF_STEP(11) SPARC_DF_STEP(12)
    }
#undef SPARC_DF_STEP
    if (bOut) {
        omax = __reduce_max_sync(0xffffffffu, omax);
        if ((tid & 31) == 0 && omax) raise_bound(bOut + col, omax);
    }
}

// u = alpha (V - shift): the per-launch potential factor of the FP64 step.
__global__ void k_scaled_v(const double *__restrict__ V, double alpha, double shift,
                           double *__restrict__ u, long n)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x)
        u[q] = alpha * (V[q] - shift);
}

cudaError_t scaled_v(const double *V, double alpha, double shift, double *u, long n,
                     cudaStream_t st)
{
    const long b = (n + 255) / 256;
    k_scaled_v<<<(unsigned)(b < 152 * 8 ? b : 152 * 8), 256, 0, st>>>(V, alpha, shift, u, n);
    note_launch();
    return cudaGetLastError();
}

template <typename TI>
static cudaError_t stencil_df_launch(const DevHam &H, const TI *Y, const double *Yprev,
                                     double *out, int ncols, long ld, double alpha,
                                     const double *u, double beta, const unsigned *bY,
                                     unsigned *bOut, cudaStream_t st)
{
    constexpr int BX = 32, BY = 16;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535 || !bY || !u) return cudaErrorInvalidValue;
    FxCoef cf;
    for (int r = 0; r <= kRadius; ++r) {
        cf.W[r] = H.wint[r];
        cf.Wf[r] = (float)H.wint[r];
    }
    cf.ag = alpha * (-0.5 * H.kscale * H.wunit);
    cf.mbeta = -beta;
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil_df<TI, BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, u, H.n0, H.n1, H.n2, ld,
                                                     nzc, zchunk, cf, bY, bOut);
    note_launch();
    return cudaGetLastError();
}

cudaError_t stencil_f64(const DevHam &H, const double *Y, const double *Yprev, double *out,
                        int ncols, long ld, double alpha, const double *u, double beta,
                        const unsigned *bY, unsigned *bOut, cudaStream_t st)
{
    return stencil_df_launch<double>(H, Y, Yprev, out, ncols, ld, alpha, u, beta, bY, bOut, st);
}

cudaError_t stencil_f32in_f64(const DevHam &H, const float *Y, double *out, int ncols, long ld,
                              const unsigned *bY, cudaStream_t st)
{
    return stencil_df_launch<float>(H, Y, nullptr, out, ncols, ld, 1.0, H.V, 0.0, bY, nullptr,
                                    st);
}

}  // namespace sparc
