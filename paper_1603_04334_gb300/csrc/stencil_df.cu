// stencil_df.cu -- the FP64 fused stencil step on the FP32 and integer pipes.
//
// Same operation and blocking as k_stencil in stencil.cu (Eq. FD:Laplacian with the
// weights of Eq. weightsLap, zero-Dirichlet boundaries, V_eff and the Chebyshev
// three-term recurrence of Algorithm ChebychevFilter, Sec. 3.4), for FP64 blocks. GB300
// issues FP64 at 1/64 of its FP32 rate, so a native FP64 stencil is bound by the FP64
// pipe at a few per cent of HBM bandwidth. This kernel does no FP64 arithmetic but one
// add per point:
//   * The Laplacian weights of radius n_o are rationals with one small common
//     denominator D (h^2 w_p = W_p / D, W_p integers, D = 831600 for n_o = 6), so
//     h^2 D L_h y = sum_p W_p S_p is an integer combination of the neighbour sums S_p.
//   * Every value of a column is brought to a fixed-point grid: with |y| < 2^E over the
//     column (E from a per-column bound), Q = y 2^(54-E) truncated to an integer
//     (|Q| < 2^54; the dropped part is below 2^(E-54), i.e. 2^-53 of the column's
//     largest value), stored as two int32 digits Q = d1 2^27 + d0 with 0 <= d0 < 2^27.
//   * Each radius sums its six neighbours digit by digit in int32 (exact: |sum| < 2^30)
//     and the weights are applied with 32 x 32 -> 64-bit integer multiply-adds into two
//     int64 accumulators (exact: |acc| < 2^52 because |W_0| + 6 sum |W_p| < 2^25).
//   * The exact integer result is turned into an FP32 pair and scaled by
//     alpha (-1/2) ks / (D h^2); the centre term (c0 + alpha V_p) y_p and the recurrence
//     term -beta Y_{j-1} are formed in pair arithmetic (TwoSum / TwoProduct, df.cuh), all
//     in units of 2^(E_ref - 54) with E_ref the larger of the column bounds of Y_j and
//     Y_{j-1}, so that no FP32 exponent can overflow; the pair is widened to FP64 with
//     that exponent offset (one FP64 add).
// The error is the truncation above (absolute, relative to the column's largest value)
// plus about 2^-47 of the largest term in the pair arithmetic. A column whose bound is
// not finite (Inf or NaN anywhere in Y_j or Y_{j-1}) gives NaN in every output value.
// Each launch can raise the output's column bounds (atomicMax), which is how the filter
// hands the bound of Y_{j+1} to the next step without another pass over the block.
#include "df.cuh"
#include "internal.cuh"

namespace sparc {

struct FxCoef {
    int W[kRadius + 1];  // integer weights: W[0] three-dimensional centre, W[p] radius p
    float gh, gl;        // alpha (-1/2) ks / (D h^2) as a pair
    float c0h, c0l;      // -alpha * shift as a pair
    float ah, al;        // alpha as a pair
    float bh, bl;        // -beta as a pair
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

// Column bound (largest high word of |y|) -> E with |y| < 2^E for every y of the column.
__device__ __forceinline__ int bound_exponent(unsigned b) { return (int)((b >> 20) & 0x7ffu) - 1022; }

// y 2^(54-E) truncated toward zero, as digits (d1, d0): d1 2^27 + d0, 0 <= d0 < 2^27.
// Requires |y| < 2^E; zero and subnormal y give 0.
__device__ __forceinline__ int2 to_digits(double y, int E)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned hw = (unsigned)(b >> 32);
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int rsh = 1021 + E - e;  // y = M 2^(e-1075): Q = M 2^-rsh, rsh >= -1
    unsigned long long Q = rsh < 0 ? (M << 1) : (rsh < 64 ? (M >> rsh) : 0ull);
    if (e == 0) Q = 0ull;
    const long long S = (hw >> 31) ? -(long long)Q : (long long)Q;
    return make_int2((int)(S >> 27), (int)(S & 0x7ffffffll));
}

__device__ __forceinline__ int2 to_digits(float y, int E)
{
    const unsigned u = __float_as_uint(y);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned long long M = (unsigned long long)((u & 0x7fffffu) | 0x800000u);
    const int lsh = e - 96 - E;  // y = M 2^(e-150): Q = M 2^lsh, lsh <= 30
    unsigned long long Q = lsh >= 0 ? (M << lsh) : (-lsh < 64 ? (M >> -lsh) : 0ull);
    if (e == 0) Q = 0ull;
    const long long S = (u >> 31) ? -(long long)Q : (long long)Q;
    return make_int2((int)(S >> 27), (int)(S & 0x7ffffffll));
}

// The digits' value d1 2^27 + d0 (in units of 2^(E-54)) as an FP32 pair.
__device__ __forceinline__ float2 digits_to_pair(int2 d)
{
    return int_to_pair((long long)d.x * 134217728ll + d.y);
}

// FP32 pair (hi, lo) of y 2^k for finite y, from the bit pattern (as split_double in
// df.cuh, with the exponent moved by k): zero for y = 0, subnormal y or |y 2^k| < 2^-126.
__device__ __forceinline__ float2 split_scaled(double y, int k)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu);
    const int ek = e + k;
    const unsigned sg = hw & 0x80000000u;
    const unsigned hb = sg | ((unsigned)(ek - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
    const bool zero = e == 0 || ek < 897;
    const unsigned hbits = zero ? 0u : (ek > 1150 ? (sg | 0x7f800000u) : hb);
    const int es = ek - 948;
    const float sc = __uint_as_float((unsigned)max(es, 1) << 23);
    float lo = __uint2float_rn(lw & 0x1fffffffu) * sc;
    lo = __uint_as_float(__float_as_uint(lo) ^ sg);
    return make_float2(__uint_as_float(hbits), (!zero && es >= 1 && ek <= 1150) ? lo : 0.0f);
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

__device__ __forceinline__ unsigned abs_hi_word(double x)
{
    return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}

// TI is the input block's type: FP64, or FP32 (the mixed-precision Rayleigh-Ritz step
// applies H in FP64 to the FP32 filtered block). One thread per (x, y) node of a BX x BY
// tile walks the tile's z range of one column; the 13 planes around it stay in registers
// as digits, the current plane's tile with its x and y halos in shared memory.
template <typename TI, int BX, int BY>
__global__ void __launch_bounds__(BX *BY, 2)
k_stencil_df(const TI *__restrict__ Y, const double *Yprev, double *out,
             const float2 *__restrict__ Vdf, int n0, int n1, int n2, long ld, int nzc, int zchunk,
             FxCoef cf, const unsigned *__restrict__ bY, const unsigned *__restrict__ bP,
             unsigned *bOut)
{
    constexpr int R = kRadius;
    // plane k is read from s[b] while plane k+1 is staged into s[b ^ 1]: one barrier per
    // plane, and the global loads of plane k+1 are in flight while plane k is computed
    __shared__ int2 s[2][BY + 2 * R][BX + 2 * R];
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
    const int2 zero = make_int2(0, 0);
    // the column's scales: digits in units of 2^(EY-54), results in units of 2^(Eref-54)
    const unsigned uy = bY[col], up = Pc ? bP[col] : 0u;
    const bool nonfinite = ((uy >> 20) & 0x7ffu) == 0x7ffu || ((up >> 20) & 0x7ffu) == 0x7ffu;
    const int EY = bound_exponent(uy);
    const int Eref = Pc ? max(EY, bound_exponent(up)) : EY;
    const int dsc = EY - Eref;  // <= 0
    const float p2 = dsc < -126 ? 0.0f : __uint_as_float((unsigned)(dsc + 127) << 23);
    const float sgh = cf.gh * p2, sgl = cf.gl * p2;
    const float c0h = cf.c0h * p2, c0l = cf.c0l * p2, ah_ = cf.ah * p2, al_ = cf.al * p2;
    const int kout = Eref - 54;
    // halo duties of this thread: x halos (tx < R) and y halos (ty < R)
    const bool hx = tx < R, hy = ty < R;
    const int il = i0 - R + tx, ir = i0 + BX + tx, jt = j0 - R + ty, jb = j0 + BY + ty;
    const bool okl = hx && j < n1 && il >= 0, okr = hx && j < n1 && ir < n0;
    const bool okt = hy && i < n0 && jt >= 0, okb = hy && i < n0 && jb < n1;
    const long offl = il + (long)n0 * j, offr = ir + (long)n0 * j;
    const long offt = i + (long)n0 * jt, offb = i + (long)n0 * jb;

    int2 q[2 * R + 1];
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) {
        const int kk = k0 - R + t;
        q[t] = (act && kk >= 0 && kk < n2) ? to_digits(Yc[pij + (long)kk * plane], EY) : zero;
    }
    {
        const long pk = (long)k0 * plane;
        s[0][ty + R][tx + R] = q[R];
        if (hx) {
            s[0][ty + R][tx] = okl ? to_digits(Yc[pk + offl], EY) : zero;
            s[0][ty + R][tx + BX + R] = okr ? to_digits(Yc[pk + offr], EY) : zero;
        }
        if (hy) {
            s[0][ty][tx + R] = okt ? to_digits(Yc[pk + offt], EY) : zero;
            s[0][ty + BY + R][tx + R] = okb ? to_digits(Yc[pk + offb], EY) : zero;
        }
    }
    float2 vcur = act ? Vdf[pij + (long)k0 * plane] : make_float2(0.0f, 0.0f);
    double pcur = (act && Pc) ? Pc[pij + (long)k0 * plane] : 0.0;
    unsigned omax = 0u;
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const int b = (k - k0) & 1;
        const long pk = (long)k * plane;
        // loads for plane k+1 (and the queue entry k+R+1), consumed after the compute
        const bool more = k + 1 < k1;
        const long pk1 = pk + plane;
        TI gl = 0, gr = 0, gt = 0, gb = 0, gq = 0;
        double pnext = 0.0;
        float2 vnext = make_float2(0.0f, 0.0f);
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
            // h^2 D L_h y in units of 2^(EY-54): two digit planes, exact integer sums
            const int2 c = q[R];
            long long A1 = (long long)cf.W[0] * c.x, A0 = (long long)cf.W[0] * c.y;
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const int2 xa = s[b][ty + R][tx + R + r], xb = s[b][ty + R][tx + R - r];
                const int2 ya = s[b][ty + R + r][tx + R], yb = s[b][ty + R - r][tx + R];
                const int s1 = (xa.x + xb.x + ya.x) + (yb.x + q[R + r].x + q[R - r].x);
                const int s0 = (xa.y + xb.y + ya.y) + (yb.y + q[R + r].y + q[R - r].y);
                A1 += (long long)cf.W[r] * s1;
                A0 += (long long)cf.W[r] * s0;
            }
            // N = A1 2^27 + A0 as a pair, times g = alpha (-1/2) ks / (D h^2) 2^(EY-Eref)
            const float2 n1p = int_to_pair(A1), n0p = int_to_pair(A0);
            float nh, nl;
            two_sum(n1p.x * 134217728.0f, n0p.x, nh, nl);
            nl += n1p.y * 134217728.0f + n0p.y;
            float ah = sgh * nh;
            float al = fmaf(sgh, nh, -ah);
            al = fmaf(sgh, nl, al);
            al = fmaf(sgl, nh, al);
            // centre: (c0 + alpha V_p) y_p
            const float2 v = vcur;
            float ch = 0.0f, cl = 0.0f;
            acc_mul(v.x, v.y, ah_, al_, ch, cl);
            {
                float t, e;
                two_sum(ch, c0h, t, e);
                ch = t;
                cl += e + c0l;
            }
            const float2 y = digits_to_pair(c);
            acc_mul(y.x, y.y, ch, cl, ah, al);
            if (Pc) {
                const float2 pv = split_scaled(pcur, -kout);
                acc_mul(pv.x, pv.y, cf.bh, cf.bl, ah, al);
            }
            double o = widen_scaled(ah, kout) + widen_scaled(al, kout);
            if (nonfinite) o = __longlong_as_double(0x7ff8000000000000ll);
            omax = max(omax, abs_hi_word(o));
            Oc[pij + pk] = o;
        }
#pragma unroll
        for (int t = 0; t < 2 * R; ++t) q[t] = q[t + 1];
        q[2 * R] = (act && kn < n2) ? to_digits(gq, EY) : zero;
        vcur = vnext;
        pcur = pnext;
        if (more) {
            s[b ^ 1][ty + R][tx + R] = q[R];
            if (hx) {
                s[b ^ 1][ty + R][tx] = okl ? to_digits(gl, EY) : zero;
                s[b ^ 1][ty + R][tx + BX + R] = okr ? to_digits(gr, EY) : zero;
            }
            if (hy) {
                s[b ^ 1][ty][tx + R] = okt ? to_digits(gt, EY) : zero;
                s[b ^ 1][ty + BY + R][tx + R] = okb ? to_digits(gb, EY) : zero;
            }
        }
        __syncthreads();
    }
    if (bOut) {
        omax = __reduce_max_sync(0xffffffffu, omax);
        if (((ty * BX + tx) & 31) == 0 && omax) atomicMax(bOut + col, omax);
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
// entries stay in L1). The pair sum is added to the FP64 output with one FP64 add. With
// bOut, the column bounds of the output are raised to cover the updated values.
namespace {
constexpr int kScatNodes = 256;
constexpr int kScatCols = 8;
}  // namespace

__global__ void __launch_bounds__(kScatNodes)
k_scatter_df(double *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
             const int *__restrict__ uniq_ptr, const int *__restrict__ nl_atom,
             const float2 *__restrict__ g, const float2 *__restrict__ Cs, unsigned *bOut)
{
    const long u = (long)blockIdx.x * kScatNodes + threadIdx.x;
    const bool live = u < nuniq;  // no early return: the warp reduces the bounds below
    const int c0 = blockIdx.y * kScatCols, c1 = min(ncols, c0 + kScatCols);
    double o[kScatCols];
    if (live) {
        const long node = uniq_node[u];
        const int q0 = uniq_ptr[u], q1 = uniq_ptr[u + 1];
        // all column sums first (coefficients from L1 / L2), then every output read is
        // issued before any store: kScatCols independent DRAM reads in flight per thread
        double v[kScatCols];
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
        double *op = out + node + (long)c0 * ld;
#pragma unroll
        for (int k = 0; k < kScatCols; ++k) o[k] = c0 + k < c1 ? op[(long)k * ld] : 0.0;
#pragma unroll
        for (int k = 0; k < kScatCols; ++k) {
            o[k] += v[k];
            if (c0 + k < c1) op[(long)k * ld] = o[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScatCols; ++k) o[k] = 0.0;
    }
    if (bOut) {
#pragma unroll
        for (int k = 0; k < kScatCols; ++k) {
            const unsigned m = __reduce_max_sync(0xffffffffu, abs_hi_word(o[k]));
            if ((threadIdx.x & 31) == 0 && m && c0 + k < c1) atomicMax(bOut + c0 + k, m);
        }
    }
}

cudaError_t scatter_f64_df(const DevHam &H, const float2 *Cs, double *out, int ncols, long ld,
                           unsigned *bOut, cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((H.nuniq + kScatNodes - 1) / kScatNodes),
              (unsigned)((ncols + kScatCols - 1) / kScatCols));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_scatter_df<<<grid, kScatNodes, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                              H.nl_atom, H.nl_gdf, Cs, bOut);
    note_launch();
    return cudaGetLastError();
}

// Column bounds: b[c] = max(b[c], largest high word of |y| over column c). A CTA reads
// kColmaxPer consecutive elements per thread of one column; one atomic per warp.
namespace {
constexpr int kColmaxThreads = 256, kColmaxPer = 8;
}  // namespace

__device__ __forceinline__ unsigned abs_hi_word(float x)
{
    // high word of the FP64 widening of |x| (exponent rebiased; subnormals count as 0)
    const unsigned u = __float_as_uint(x) & 0x7fffffffu;
    const unsigned e = u >> 23;
    if (e == 0u) return 0u;
    if (e == 0xffu) return 0x7ff00000u | ((u & 0x7fffffu) ? 0x80000u : 0u);
    return ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
}

template <typename T>
__global__ void __launch_bounds__(kColmaxThreads)
k_colmax(const T *__restrict__ Y, long ld, long nd, unsigned *b)
{
    const T *Yc = Y + (long)blockIdx.y * ld;
    const long base = (long)blockIdx.x * kColmaxThreads * kColmaxPer + threadIdx.x;
    unsigned m = 0u;
#pragma unroll
    for (int t = 0; t < kColmaxPer; ++t) {
        const long p = base + (long)t * kColmaxThreads;
        if (p < nd) m = max(m, abs_hi_word(Yc[p]));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(b + blockIdx.y, m);
}

template <typename T>
static cudaError_t colmax_launch(const T *Y, int ncols, long ld, long nd, unsigned *b,
                                 cudaStream_t st)
{
    if (ncols <= 0 || nd <= 0) return cudaSuccess;
    if (ncols > 65535) return cudaErrorInvalidValue;
    const long per = (long)kColmaxThreads * kColmaxPer;
    dim3 grid((unsigned)((nd + per - 1) / per), (unsigned)ncols);
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

template <typename TI>
static cudaError_t stencil_df_launch(const DevHam &H, const TI *Y, const double *Yprev,
                                     double *out, int ncols, long ld, double alpha, double shift,
                                     double beta, const unsigned *bY, const unsigned *bP,
                                     unsigned *bOut, cudaStream_t st)
{
    constexpr int BX = 32, BY = 16;
    if (ncols <= 0) return cudaSuccess;
    if (ncols > 65535 || !bY || (Yprev && !bP)) return cudaErrorInvalidValue;
    FxCoef cf;
    for (int r = 0; r <= kRadius; ++r) cf.W[r] = H.wint[r];
    split_host(alpha * (-0.5 * H.kscale) * H.wunit, cf.gh, cf.gl);
    split_host(-alpha * shift, cf.c0h, cf.c0l);
    split_host(alpha, cf.ah, cf.al);
    split_host(-beta, cf.bh, cf.bl);
    const int gx = (H.n0 + BX - 1) / BX, gy = (H.n1 + BY - 1) / BY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(BX, BY);
    k_stencil_df<TI, BX, BY><<<grid, block, 0, st>>>(Y, Yprev, out, H.Vdf, H.n0, H.n1, H.n2, ld,
                                                     nzc, zchunk, cf, bY, bP, bOut);
    note_launch();
    return cudaGetLastError();
}

cudaError_t stencil_f64(const DevHam &H, const double *Y, const double *Yprev, double *out,
                        int ncols, long ld, double alpha, double shift, double beta,
                        const unsigned *bY, const unsigned *bP, unsigned *bOut,
                        cudaStream_t st)
{
    return stencil_df_launch<double>(H, Y, Yprev, out, ncols, ld, alpha, shift, beta, bY, bP,
                                     bOut, st);
}

cudaError_t stencil_f32in_f64(const DevHam &H, const float *Y, double *out, int ncols, long ld,
                              const unsigned *bY, cudaStream_t st)
{
    return stencil_df_launch<float>(H, Y, nullptr, out, ncols, ld, 1.0, 0.0, 0.0, bY, nullptr,
                                    nullptr, st);
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
