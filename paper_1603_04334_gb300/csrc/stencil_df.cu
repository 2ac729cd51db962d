// stencil_df.cu -- the FP64 fused stencil step on the integer and FP32 pipes.
//
// Same operation and blocking as k_stencil in stencil.cu (Eq. FD:Laplacian with the
// weights of Eq. weightsLap, zero-Dirichlet boundaries, V_eff and the Chebyshev
// three-term recurrence of Algorithm ChebychevFilter, Sec. 3.4), for FP64 blocks. GB300
// issues FP64 at 1/64 of its FP32 rate, so a native FP64 stencil is bound by the FP64
// pipe at a few per cent of HBM bandwidth. This kernel does one FP64 add per point:
//   * The Laplacian weights of radius n_o are rationals with one small common
//     denominator D (h^2 w_p = W_p / D, W_p integers, D = 831600 for n_o = 6), so
//     h^2 D L_h y = sum_p W_p S_p is an integer combination of the neighbour sums S_p.
//   * Every value of a column is put on a fixed-point grid: with |y| < 2^E over the
//     column (E from a per-column bound), y 2^(28-E) = d + r with d an integer truncated
//     toward zero (|d| < 2^28) and r the rest (|r| < 1, same sign, kept to 23 bits as
//     FP32).
//   * Each radius sums its six neighbours' d in int32 (exact: |sum| < 6 * 2^28 < 2^31)
//     and applies W_p with one 32 x 32 -> 64-bit integer multiply-add (exact: the int64
//     accumulator stays below 2^53); the r parts are summed and weighted in FP32. The r
//     parts carry only the bits below 2^(E-28), so FP32 rounding there costs about 2^-51
//     of the largest term.
//   * The integer sum becomes an FP32 pair and the r sum is added; in pair arithmetic
//     (TwoSum / TwoProduct, df.cuh) and in units of 2^(E-28) the kernel forms
//     (-1/2) ks / (D h^2) T + (V_p - shift) y_p and multiplies it by alpha. The pair is
//     widened to FP64 by integer operations on its exponent (no FP64 instruction), then
//     two FP64 operations finish the point: the pair's add and the recurrence term
//     -beta Y_{j-1} as one fused multiply-add.
// Error: the truncation of r (2^-51 of the column's largest value) plus about 2^-47 of the
// largest term in the pair and FP32 arithmetic. A column whose bound is not finite (Inf or
// NaN anywhere in Y_j) gives NaN in every output value of the column, and so does a point
// whose pair overflows FP32 (|alpha (V_p - shift)| or the Laplacian scale near 2^100 and
// beyond). Each launch can raise the output's column bounds (atomicMax), which is how the
// filter hands the bound of Y_{j+1} to the next step without another pass over the block.
#include <type_traits>

#include "df.cuh"
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

struct FxCoef {
    int W[kRadius + 1];    // integer weights: W[0] three-dimensional centre, W[p] radius p
    float Wf[kRadius + 1]; // the same as FP32 (exact: |W| < 2^24)
    float gh, gl;          // (-1/2) ks / (D h^2) as a pair
    float ah, al;          // alpha as a pair
    double mbeta;          // -beta
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

// x (integer, -2^22 <= x < 2^22) as float without a conversion instruction: x is added
// to the significand of 1.5 * 2^23, whose unit in the last place is 1.
__device__ __forceinline__ float small_int_to_float(int x)
{
    return __int_as_float(0x4B400000 + x) - 12582912.0f;
}

// An integer |A| < 2^54 as an FP32 pair (hi + lo = A to about 2^-48 relative): A is cut
// into a signed high word and two 16-bit pieces, each exactly representable; the first
// sum is Fast2Sum (the high piece is zero or larger in magnitude than the middle one).
__device__ __forceinline__ float2 int_to_pair(long long A)
{
    const int hi = (int)(A >> 32);
    const unsigned lo = (unsigned)A;
    const float fh = small_int_to_float(hi) * 4294967296.0f;
    const float fm = small_int_to_float((int)(lo >> 16)) * 65536.0f;
    const float fl = small_int_to_float((int)(lo & 0xffffu));
    const float s = fh + fm;
    const float e = fm - (s - fh);
    return make_float2(s, e + fl);
}

// d + r as an FP32 pair: d = dh 2^16 + dl with exactly representable pieces, Fast2Sum
// (|dh 2^16| >= 2^16 > dl unless dh = 0), then r joins the low part.
__device__ __forceinline__ float2 fx_to_pair(int2 v)
{
    const float fh = small_int_to_float(v.x >> 16) * 65536.0f;
    const float fl = small_int_to_float(v.x & 0xffff);
    const float s = fh + fl;
    const float e = fl - (s - fh);
    return make_float2(s, e + __int_as_float(v.y));
}

// f 2^k as FP64 from the bit pattern: FP32 zero and subnormals, and results below the
// FP64 normal range, give a signed zero; results above it give Inf; Inf / NaN stay so.
__device__ __forceinline__ double widen_scaled(float f, int k)
{
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned m = u & 0x7fffffu, sg = u & 0x80000000u;
    const int E = e + 896 + k;
    unsigned hi = sg | ((unsigned)E << 20) | (m >> 3), lo = m << 29;
    if (e == 0 || E <= 0) hi = sg, lo = 0u;
    if (e != 0 && E >= 2047) hi = sg | 0x7ff00000u, lo = 0u;
    if (e == 0xff) hi = sg | 0x7ff00000u | (m ? 0x80000u : 0u), lo = 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// f 2^k as FP64 for FP32 values the scaled pair arithmetic produces, with
// koff = (896 + k) << 20 and -896 <= k <= 896 (so every normal FP32 exponent lands in the
// FP64 normal range): the exponent field is moved by an integer add; zero and FP32
// subnormals give a signed zero. Inf and NaN are not handled (the caller checks).
__device__ __forceinline__ double widen_fast(float f, unsigned koff)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sg = u & 0x80000000u;
    const bool z = (u & 0x7f800000u) == 0u;
    const unsigned hi = z ? sg : (sg | (((u >> 3) & 0x0fffffffu) + koff));
    return __hiloint2double((int)hi, z ? 0 : (int)(u << 29));
}

// TI is the input block's type: FP64, or FP32 (the mixed-precision Rayleigh-Ritz step
// applies H in FP64 to the FP32 filtered block). One thread per (x, y) node of a BX x BY
// tile walks the tile's z range of one column; the 13 planes around it stay in registers
// on the column's grid, the current plane's tile with its x and y halos in shared memory.
// The halo strips (2 R (BX + BY) nodes) are loaded and converted by all threads together,
// at most two nodes each, so no warp runs them as a divergent side branch.
template <typename TI, int BX, int BY>
__global__ void __launch_bounds__(BX *BY, 2)
k_stencil_df(const TI *__restrict__ Y, const double *Yprev, double *out,
             const float2 *__restrict__ Vc, int n0, int n1, int n2, long ld, int nzc, int zchunk,
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
    const TI *Yc = Y + (long)col * ld;
    const double *Pc = Yprev ? Yprev + (long)col * ld : nullptr;
    double *Oc = out + (long)col * ld;
    const bool act = (i < n0) && (j < n1);
    const unsigned pij = act ? (unsigned)i + (unsigned)n0 * (unsigned)j : 0u;
    const int2 zero = make_int2(0, 0);
    // the column's scale: grid values and the pair arithmetic in units of 2^(EY-28)
    const unsigned uy = bY[col];
    const bool nonfinite = ((uy >> 20) & 0x7ffu) == 0x7ffu;
    const int EY = bound_exponent(uy);
    const int kout = EY - 28;
    const bool fastw = kout >= -896 && kout <= 896;  // uniform over the CTA
    const unsigned koff = (unsigned)(896 + kout) << 20;
    // halo duties: nodes tid and tid + NT of the strips (left, right: R x BY each; top,
    // bottom: BX x R each); hs = shared-memory index (-1: none), hg = offset in the plane
    int hs[2];
    unsigned hg[2];
    bool hv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int h = tid + u * NT;
        int sx, sy;
        if (h < 2 * R * BY) {
            const int side = h / (R * BY), rr = h % (R * BY);
            sy = R + rr / R;
            sx = side ? BX + R + rr % R : rr % R;
        } else {
            const int v = h - 2 * R * BY;
            const int side = v / (R * BX), rr = v % (R * BX);
            sx = R + rr % BX;
            sy = side ? BY + R + rr / BX : rr / BX;
        }
        const int gx = i0 - R + sx, gy = j0 - R + sy;
        hs[u] = h < NH ? sy * SX + sx : -1;
        hv[u] = h < NH && gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
        hg[u] = hv[u] ? (unsigned)gx + (unsigned)n0 * (unsigned)gy : 0u;
    }
    const int me = (ty + R) * SX + tx + R;  // this thread's node in a plane buffer

    int2 q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? to_fx(Yc[pij + (unsigned)kk * plane], EY) : zero;
    }
    {
        const unsigned pk = (unsigned)k0 * plane;
        s[me] = q[R];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (hs[u] >= 0) s[hs[u]] = hv[u] ? to_fx(Yc[hg[u] + pk], EY) : zero;
    }
    float2 vcur = act ? Vc[pij + (unsigned)k0 * plane] : make_float2(0.0f, 0.0f);
    double pcur = (act && Pc) ? Pc[pij + (unsigned)k0 * plane] : 0.0;
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
        double pnext = 0.0;
        float2 vnext = make_float2(0.0f, 0.0f);
        if (more) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (hv[u]) g[u] = Yc[hg[u] + pk1];
            if (act) {
                vnext = Vc[pij + pk1];
                if (Pc) pnext = Pc[pij + pk1];
            }
        }
        const int kn = k + R + 1;
        if (act && kn < n2) gq = Yc[pij + (unsigned)kn * plane];
        if (act) {
            // h^2 D L_h y in units of 2^(EY-28): exact integer sums of d, FP32 sums of r
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
            // T = A + Rs as a pair; (-1/2) ks / (D h^2) T + (V_p - shift) y_p; times alpha
            const float2 tp = int_to_pair(A);
            float th, tl;
            two_sum(tp.x, Rs, th, tl);
            tl += tp.y;
            float ih = cf.gh * th;
            float il = fmaf(cf.gh, th, -ih);
            il = fmaf(cf.gh, tl, il);
            il = fmaf(cf.gl, th, il);
            const float2 y = fx_to_pair(c);
            acc_mul(y.x, y.y, vcur.x, vcur.y, ih, il);
            const float ah = cf.ah * ih;
            float al = fmaf(cf.ah, ih, -ah);
            al = fmaf(cf.ah, il, al);
            al = fmaf(cf.al, ih, al);
            double o;
            if (fastw)
                o = widen_fast(ah, koff) + widen_fast(al, koff);
            else
                o = widen_scaled(ah, kout) + widen_scaled(al, kout);
            if (Pc) o = fma(cf.mbeta, pcur, o);
            if (nonfinite || (__float_as_uint(ah) & 0x7f800000u) == 0x7f800000u)
                o = __longlong_as_double(0x7ff8000000000000ll);
            omax = max(omax, abs_hi_word(o));
            Oc[pij + pk] = o;
        }
        // plane k - R leaves the queue; its slot takes plane k + R + 1 (logical entry 2R
        // of the next phase), and the next phase's centre is plane k + 1
        q[PH % Q] = (act && kn < n2) ? to_fx(gq, EY) : zero;
        vcur = vnext;
        pcur = pnext;
        if (more) {
            int2 *nb = s + (b ^ 1) * (SY * SX);
            nb[me] = q[(PH + 1 + R) % Q];
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (hs[u] >= 0) nb[hs[u]] = hv[u] ? to_fx(g[u], EY) : zero;
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

static void split_host(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

template <typename TI>
static cudaError_t stencil_df_launch(const DevHam &H, const TI *Y, const double *Yprev,
                                     double *out, int ncols, long ld, double alpha,
                                     const float2 *Vc, double beta, const unsigned *bY,
                                     unsigned *bOut, cudaStream_t st)
{
    constexpr int BX = 32, BY = 16;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535 || !bY || !Vc) return cudaErrorInvalidValue;
    FxCoef cf;
    for (int r = 0; r <= kRadius; ++r) {
        cf.W[r] = H.wint[r];
        cf.Wf[r] = (float)H.wint[r];
    }
    split_host(-0.5 * H.kscale * H.wunit, cf.gh, cf.gl);
    split_host(alpha, cf.ah, cf.al);
    cf.mbeta = -beta;
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil_df<TI, BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, Vc, H.n0, H.n1, H.n2, ld,
                                                     nzc, zchunk, cf, bY, bOut);
    note_launch();
    return cudaGetLastError();
}

cudaError_t stencil_f64(const DevHam &H, const double *Y, const double *Yprev, double *out,
                        int ncols, long ld, double alpha, const float2 *Vc, double beta,
                        const unsigned *bY, unsigned *bOut, cudaStream_t st)
{
    return stencil_df_launch<double>(H, Y, Yprev, out, ncols, ld, alpha, Vc, beta, bY, bOut,
                                     st);
}

cudaError_t stencil_f32in_f64(const DevHam &H, const float *Y, double *out, int ncols, long ld,
                              const unsigned *bY, cudaStream_t st)
{
    return stencil_df_launch<float>(H, Y, nullptr, out, ncols, ld, 1.0, H.Vdf, 0.0, bY, nullptr,
                                    st);
}

}  // namespace sparc
