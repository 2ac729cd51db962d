// rotate_fx.cu -- the rotation X = Y C of the FP64 Rayleigh-Ritz step (Eq.
// OrbitalTransformation, Sec. 3.4; C the Ns x Ns matrix L^-T Q) on the integer and FP32
// pipes, from the per-column fixed-point grids of the FP64 stencil.
//
// Column k of Y has a bound 2^E_k > max_i |y_ik| (fx.cuh). The rows of C are first scaled
// by 2^(E_k - E_max) (E_max the largest E_k), which puts every product Y_ik C_kj on the
// common scale 2^(E_max - 28); each column j of the scaled C is then put on its own grid
// 2^F_j. On these grids y 2^(28 - E) = d + r with d an int32 (|d| < 2^28) and r the next
// 23 bits as FP32, so a product is
//   d_y d_c + (d_y r_c + r_y d_c) + r_y r_c:
// d_y d_c is exact in a 32 x 32 -> 64-bit integer multiply-add; the cross terms (below
// 2^29 each) are summed in FP32 with float(d) (its rounding is 2^-24 of a term that is
// itself 2^-28 of d d); r r < 1 is dropped (2^-56 of the leading term). Every kChunk terms
// the FP32 cross sum is rounded to an integer and joins the chunk's int64 sum
// (|sum| < 2^62 + 2^36), which is added, shifted right by `sh` bits with rounding, to the
// output's int64 sum (sh chosen by the host so nothing overflows). That sum becomes an
// FP32 pair with integer operations and is widened to FP64 with the exponent offset (one
// FP64 add per output). Error about 2^-47 of sum |y c|: the accuracy of an FP64 dot
// product, at three integer / FP32 instructions per multiply-add where FP32-pair
// arithmetic takes twelve.
//
// A CTA walks 64-row tiles of Y for one 64-column tile of C; 256 threads hold 4 x 4
// outputs each (chunk sums in registers, the outputs' int64 sums in shared memory, each
// thread owning its 16 words). K = Ns is staged 16 at a time: the raw FP64 tile of Y and
// the grid-form tile of C of stage s+1 are copied asynchronously (cp.async, two-slot
// rings) while stage s is converted and multiplied. A non-finite column bound of Y gives
// NaN in every output.
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int FT = 64;          // output tile (rows and columns)
constexpr int kChunk = 64;      // terms per exact int64 chunk sum (64 * 2^56 < 2^63)
constexpr int kThreads = 256;
struct __align__(16) FxEl {
    int d;
    float fd, r, pad;
};
constexpr unsigned kSliceBytes = 16u * kThreads * sizeof(long long);  // [entry][thread]
}  // namespace

__device__ __forceinline__ FxEl fx_el(double x, int E)
{
    const int2 v = to_fx(x, E);
    FxEl e;
    e.d = v.x;
    e.fd = (float)v.x;
    e.r = __int_as_float(v.y);
    e.pad = 0.0f;
    return e;
}

// Asynchronous copies global -> shared (cp.async), zero-filled when `ok` is false (the
// source address is then never read; a valid one is passed anyway).
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 8 : 0));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// ---- rotation ---------------------------------------------------------------------
// One CTA: E_max over the bounds of Y's columns, then per column j of C (one warp per
// column) the scaled entries C_kj 2^(E_k - E_max), their bound F_j and their grid values,
// stored row-major ([k][j]) for coalesced staging. meta = {E_max, any bound not finite}.
__global__ void __launch_bounds__(1024)
k_rot_prep(const double *__restrict__ C, int ns, const unsigned *__restrict__ bA, FxEl *Cd,
           unsigned *bC, int *meta)
{
    __shared__ int red[32];
    __shared__ int emax_s, bad_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int em = -2000, bad = 0;
    for (int k = tid; k < ns; k += blockDim.x) {
        const unsigned b = bA[k];
        bad |= ((b >> 20) & 0x7ffu) == 0x7ffu;
        em = max(em, bound_exponent(b));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0) red[w] = em;
    if (tid == 0) bad_s = 0;
    __syncthreads();
    if (lane == 0 && bad) atomicOr(&bad_s, 1);
    if (tid == 0) {
        int m = red[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = max(m, red[q]);
        emax_s = m;
    }
    __syncthreads();
    const int Emax = emax_s;
    for (int j = w; j < ns; j += blockDim.x >> 5) {
        unsigned m = 0u;
        for (int k = lane; k < ns; k += 32) {
            const double v = ldexp(C[k + (long)j * ns], bound_exponent(bA[k]) - Emax);
            m = max(m, abs_hi_word(v));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        const int F = bound_exponent(m);
        for (int k = lane; k < ns; k += 32) {
            const double v = ldexp(C[k + (long)j * ns], bound_exponent(bA[k]) - Emax);
            Cd[(long)k * ns + j] = fx_el(v, F);
        }
        if (lane == 0) bC[j] = m;
    }
    if (tid == 0) {
        meta[0] = Emax;
        meta[1] = bad_s;
    }
}

// x (|x| < 2^63) as an FP32 pair: three 21-bit pieces, each exact, Fast2Sum of the upper
// two (the top piece is zero or larger in magnitude), the last joins the low part.
__device__ __forceinline__ float2 int63_to_pair(long long x)
{
    const int p2 = (int)(x >> 42);
    const int p1 = (int)((x >> 21) & 0x1fffff);
    const int p0 = (int)(x & 0x1fffff);
    const float f2 = (__int_as_float(0x4B400000 + p2) - 12582912.0f) * 4398046511104.0f;  // 2^42
    const float f1 = (__int_as_float(0x4B400000 + p1) - 12582912.0f) * 2097152.0f;        // 2^21
    const float f0 = __int_as_float(0x4B400000 + p0) - 12582912.0f;
    const float s = f2 + f1;
    const float e = f1 - (s - f2);
    return make_float2(s, e + f0);
}

// f 2^k as FP64 from the bit pattern (zero / FP32 subnormal / FP64 underflow -> signed zero,
// overflow -> Inf).
__device__ __forceinline__ double widen_k(float f, int k)
{
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned m = u & 0x7fffffu, sg = u & 0x80000000u;
    const int E = e + 896 + k;
    unsigned hi = sg | ((unsigned)E << 20) | (m >> 3), lo = m << 29;
    if (e == 0 || E <= 0) hi = sg, lo = 0u;
    if (e != 0 && E >= 2047) hi = sg | 0x7ff00000u, lo = 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// out = A C: a CTA walks 64-row tiles of A for one 64-column tile of C (column tiles of a
// row tile run side by side, so A stays in L2), K = ns staged RK at a time. The raw FP64
// tile of A and the grid-form tile of C of stage s+1 are copied asynchronously while
// stage s is converted and multiplied (two-slot rings, no registers held for them).
namespace {
constexpr int RK = 16;
constexpr unsigned kRotSmem = 2u * RK * FT * sizeof(double)     // raw A ring
                              + 2u * RK * FT * sizeof(FxEl)     // C ring
                              + RK * FT * sizeof(FxEl)          // converted A
                              + kSliceBytes;                    // 96 KB
}  // namespace

__global__ void __launch_bounds__(kThreads, 2)
k_rotate_fx(const double *__restrict__ A, long lda, const unsigned *__restrict__ bA, long nd,
            int ns, const FxEl *__restrict__ Cd, const unsigned *__restrict__ bC,
            const int *__restrict__ meta, int sh, double *__restrict__ out, long ldo)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *Araw = reinterpret_cast<double *>(smem);               // [2][RK][FT]
    FxEl *Cs = reinterpret_cast<FxEl *>(Araw + 2 * RK * FT);        // [2][RK][FT]
    FxEl *As = Cs + 2 * RK * FT;                                    // [RK][FT]
    long long *slice = reinterpret_cast<long long *>(As + RK * FT);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int j0 = blockIdx.x * FT;
    const int Emax = meta[0];
    const bool bad = meta[1] != 0;
    const long long half = sh > 0 ? (1LL << (sh - 1)) : 0;
    const int nst = (ns + RK - 1) / RK;
    for (long rt = blockIdx.y; rt * FT < nd; rt += gridDim.y) {
        const long r0 = rt * FT;
        // stage s into slot s & 1: element e = tid + 256 u is (k = e / 64, row / column
        // e % 64) of the RK x 64 tiles
        auto issue = [&](int st) {
            const int k0 = st * RK, b = st & 1;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = tid + kThreads * u, k = e >> 6, q = e & 63;
                const long row = r0 + q;
                const bool oka = row < nd && k0 + k < ns;
                cp_async8(Araw + (b * RK + k) * FT + q, oka ? A + row + (long)(k0 + k) * lda : A,
                          oka);
                const bool okc = k0 + k < ns && j0 + q < ns;
                cp_async16(Cs + (b * RK + k) * FT + q,
                           okc ? Cd + (long)(k0 + k) * ns + j0 + q : Cd, okc);
            }
            cp_async_commit();
        };
        long long acc[4][4];
        float cr[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                acc[x][y] = 0;
                cr[x][y] = 0.0f;
                slice[(x * 4 + y) * kThreads + tid] = 0;
            }
        issue(0);
        int nk = 0;
        for (int st = 0; st < nst; ++st) {
            if (st + 1 < nst)
                issue(st + 1);
            else
                cp_async_commit();  // an empty group keeps the wait count uniform
            cp_async_wait1();
            __syncthreads();
            {   // convert this stage's A elements onto their columns' grids
                const int k0 = st * RK, b = st & 1;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = tid + kThreads * u, k = e >> 6, q = e & 63;
                    const int E = k0 + k < ns ? bound_exponent(bA[k0 + k]) : 0;
                    As[k * FT + q] = fx_el(Araw[(b * RK + k) * FT + q], E);
                }
            }
            __syncthreads();
            const FxEl *cs = Cs + (st & 1) * RK * FT;
#pragma unroll 2
            for (int kk = 0; kk < RK; ++kk) {
                FxEl a[4], c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = As[kk * FT + ty + 16 * u];
                    c[u] = cs[kk * FT + tx + 16 * u];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[x][y]) : "r"(a[x].d), "r"(c[y].d));
                        cr[x][y] = fmaf(a[x].fd, c[y].r, cr[x][y]);
                        cr[x][y] = fmaf(a[x].r, c[y].fd, cr[x][y]);
                    }
            }
            nk += RK;
            if (nk == kChunk || st + 1 == nst) {  // flush the chunk into the slice sums
                nk = 0;
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const long long t = acc[x][y] + __float2ll_rn(cr[x][y]);
                        slice[(x * 4 + y) * kThreads + tid] += (t + half) >> sh;
                        acc[x][y] = 0;
                        cr[x][y] = 0.0f;
                    }
            }
            __syncthreads();  // slot st & 1 and the converted tile are free again
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int c = j0 + tx + 16 * y;
            if (c >= ns) continue;
            const int kf = sh + Emax - 28 + bound_exponent(bC[c]) - 28;
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const long row = r0 + ty + 16 * x;
                if (row >= nd) continue;
                const float2 p = int63_to_pair(slice[(x * 4 + y) * kThreads + tid]);
                double v = widen_k(p.x, kf) + widen_k(p.y, kf);
                if (bad) v = __longlong_as_double(0x7ff8000000000000ll);
                out[row + (long)c * ldo] = v;
            }
        }
    }
}

size_t rotate_fx_workspace(int ns) { return sizeof(FxEl) * (size_t)ns * ns + 16 * (size_t)ns + 64; }

cudaError_t rotate_f64_fx(const double *A, long lda, const unsigned *bA, long nd, int ns,
                          const double *C, double *out, long ldo, void *ws, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_rotate_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRotSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    FxEl *Cd = reinterpret_cast<FxEl *>(ws);
    unsigned *bC = reinterpret_cast<unsigned *>(Cd + (size_t)ns * ns);
    int *meta = reinterpret_cast<int *>(bC + ns);
    k_rot_prep<<<1, 1024, 0, st>>>(C, ns, bA, Cd, bC, meta);
    note_launch();
    const int chunks = (ns + kChunk - 1) / kChunk;
    int sh = 0;
    while ((1 << sh) < chunks + 1) ++sh;
    const long gy = (nd + FT - 1) / FT;
    dim3 grid((ns + FT - 1) / FT, (unsigned)(gy < 65535 ? gy : 65535));
    k_rotate_fx<<<grid, kThreads, kRotSmem, st>>>(A, lda, bA, nd, ns, Cd, bC, meta, sh, out,
                                                   ldo);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
