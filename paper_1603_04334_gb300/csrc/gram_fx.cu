// gram_fx.cu -- the FP64 subspace contractions M_s = Y^T Y, H_s = Y^T (H Y) and the
// rotation Y C of the Rayleigh-Ritz step (Sec. 3.4) on the integer and FP32 pipes, from the
// per-column fixed-point grids of the FP64 stencil.
//
// Column j of an operand has a bound 2^E_j > max_k |x_kj| (fx.cuh). On that grid
// x 2^(28 - E_j) = d + r with d an int32 (|d| < 2^28) and r the next 23 bits as FP32, so
//   a b 2^(56 - E_i - E_j) = da db + (da rb + ra db) + ra rb.
// da db is exact in a 32 x 32 -> 64-bit integer multiply-add; the cross terms (below
// 2^29 each) are summed in FP32 with float(d) (its rounding is 2^-24 of a term that is
// itself 2^-28 of da db); ra rb < 1 is dropped (2^-56 of the leading term). Every kChunk
// rows the FP32 cross sum is rounded to an integer and joins the chunk's int64 sum
// (|sum| < 2^62 + 2^36), which is added, shifted right by `sh` bits with rounding, to the
// slice's int64 sum: the host picks sh so that no slice sum can overflow, and the dropped
// bits are below 2^(sh - 63) of the largest possible chunk sum. The slice sum times
// 2^(sh + E_i + E_j - 56) is the slice's partial; partials are summed in FP64 in a fixed
// order. Error per chunk about 2^-47 of sum |a b| (the FP32 cross sums): the accuracy of
// an FP64 dot product, at three integer / FP32 instructions per multiply-add where the
// FP32-pair Gram (gram_df.cu) takes twelve.
//
// A CTA owns a 64 x 64 tile of G over a slice of rows (split-K); 256 threads hold 4 x 4
// entries each: the chunk sums in registers, the slice sums in shared memory (each
// thread owns its 16 words, no atomics). Operand rows are staged 16 at a time: the raw
// FP64 tiles of stage s+1 are copied asynchronously (cp.async, two-slot rings) while stage
// s is converted to (d, float(d), r) and multiplied. Symmetric mode computes
// the tiles with i0 <= j0 only and the reduction mirrors them. A column whose bound is not
// finite gives NaN in its row and column of G.
//
// The rotation X = Y C (Eq. OrbitalTransformation, C the Ns x Ns matrix of the Rayleigh-
// Ritz step) uses the same arithmetic: the rows of C are first scaled by 2^(E_k - E_max)
// (E_k the bound exponent of column k of Y, E_max the largest), which puts every product
// Y_ik C_kj on the common scale 2^(E_max - 28); each column j of the scaled C is put on its
// own grid 2^F_j. An output's int64 sum becomes an FP32 pair with integer operations and is
// widened to FP64 with the exponent offset (one FP64 add per output).
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int FT = 64;          // tile of G
constexpr int FK = 16;          // rows per stage
constexpr int kChunk = 64;      // rows per exact int64 chunk sum (64 * 2^56 < 2^63)
constexpr int kThreads = 256;
struct __align__(16) FxEl {
    int d;
    float fd, r, pad;
};
constexpr unsigned kSliceBytes = 16u * kThreads * sizeof(long long);  // [entry][thread]
constexpr int kRawCol = FK + 1;  // padded column of a raw tile (doubles)
constexpr unsigned kSmemBytes = 4u * FT * kRawCol * sizeof(double)  // raw A, B rings
                                + 2u * FK * FT * sizeof(FxEl)       // converted A, B
                                + kSliceBytes;                      // 98 KB
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

__global__ void __launch_bounds__(kThreads, 2)
k_gram_fx(const double *__restrict__ A, long lda, const unsigned *__restrict__ bA,
          const double *__restrict__ B, long ldb, const unsigned *__restrict__ bB, long nd,
          int ns, long rows_per, int sh, int sym, double *__restrict__ part)
{
    if (sym && blockIdx.x > blockIdx.y) return;
    extern __shared__ __align__(16) unsigned char smem[];
    // raw tiles column-major with a padded column ([2][FT][FK + 1]): the copies (rows
    // along threads) and the conversion reads (columns along threads) are conflict-free
    double *Araw = reinterpret_cast<double *>(smem);
    double *Braw = Araw + 2 * FT * kRawCol;
    FxEl *As = reinterpret_cast<FxEl *>(Braw + 2 * FT * kRawCol);  // [FK][FT]
    FxEl *Bs = As + FK * FT;                                       // [FK][FT]
    long long *slice = reinterpret_cast<long long *>(Bs + FK * FT);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * FT, j0 = blockIdx.y * FT;
    const long r0 = (long)blockIdx.z * rows_per;
    const long r1 = min(nd, r0 + rows_per);
    // conversion duty: column tid % 64, rows tid / 64 + 4 u of a stage
    const int cc = tid & 63;
    const int EA = i0 + cc < ns ? bound_exponent(bA[i0 + cc]) : 0;
    const int EB = j0 + cc < ns ? bound_exponent(bB[j0 + cc]) : 0;
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
    const long nst = (r1 > r0) ? (r1 - r0 + FK - 1) / FK : 0;
    auto issue = [&](long st) {
        const int b = (int)(st & 1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // copy duty: element e = tid + 256 u is row e % 16,
            const int e = tid + kThreads * u, q = e & 15, c = e >> 4;  // column e / 16
            const long row = r0 + st * FK + q;
            const bool oka = row < r1 && i0 + c < ns, okb = row < r1 && j0 + c < ns;
            cp_async8(Araw + (b * FT + c) * kRawCol + q, oka ? A + row + (long)(i0 + c) * lda : A,
                      oka);
            cp_async8(Braw + (b * FT + c) * kRawCol + q, okb ? B + row + (long)(j0 + c) * ldb : B,
                      okb);
        }
        cp_async_commit();
    };
    const long long half = sh > 0 ? (1LL << (sh - 1)) : 0;
    auto flush = [&]() {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const long long t = acc[x][y] + __float2ll_rn(cr[x][y]);
                slice[(x * 4 + y) * kThreads + tid] += (t + half) >> sh;
                acc[x][y] = 0;
                cr[x][y] = 0.0f;
            }
    };
    if (nst > 0) issue(0);
    int steps = 0;
    for (long st = 0; st < nst; ++st) {
        if (st + 1 < nst)
            issue(st + 1);
        else
            cp_async_commit();  // an empty group keeps the wait count uniform
        cp_async_wait1();
        __syncthreads();
        {   // this stage's elements onto their columns' grids
            const int b = (int)(st & 1);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = (tid >> 6) + 4 * u;
                As[q * FT + cc] = fx_el(Araw[(b * FT + cc) * kRawCol + q], EA);
                Bs[q * FT + cc] = fx_el(Braw[(b * FT + cc) * kRawCol + q], EB);
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < FK; ++kk) {
            FxEl a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk * FT + ty + 16 * u];
                b[u] = Bs[kk * FT + tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    // one 32 x 32 -> 64-bit multiply-add into the chunk sum
                    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[x][y]) : "r"(a[x].d), "r"(b[y].d));
                    cr[x][y] = fmaf(a[x].fd, b[y].r, cr[x][y]);
                    cr[x][y] = fmaf(a[x].r, b[y].fd, cr[x][y]);
                }
        }
        if (++steps == kChunk / FK) {
            steps = 0;
            flush();
        }
        __syncthreads();  // ring slot st & 1 and the converted tiles are free again
    }
    flush();
    double *P = part + (long)blockIdx.z * ns * ns;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = i0 + ty + 16 * x, gj = j0 + tx + 16 * y;
            if (gi < ns && gj < ns) {
                const unsigned ui = bA[gi], uj = bB[gj];
                double v;
                if (((ui >> 20) & 0x7ffu) == 0x7ffu || ((uj >> 20) & 0x7ffu) == 0x7ffu)
                    v = __longlong_as_double(0x7ff8000000000000ll);
                else
                    v = ldexp((double)slice[(x * 4 + y) * kThreads + tid],
                              sh + bound_exponent(ui) + bound_exponent(uj) - 56);
                P[gi + (long)gj * ns] = v;
            }
        }
}

// G(i, j) = sum over slices in a fixed order; in symmetric mode entries of tiles below the
// diagonal are read from the mirrored (j, i) position.
__global__ void k_gram_fx_reduce(const double *__restrict__ part, int nsplit, int ns, int sym,
                                 double *G)
{
    const long nn = (long)ns * ns;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nn;
         q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q % ns), j = (int)(q / ns);
        const long src = (sym && (i / FT) > (j / FT)) ? (long)j + (long)i * ns : q;
        double s = 0.0;
        for (int t = 0; t < nsplit; ++t) s += part[(long)t * nn + src];
        G[q] = s;
    }
}

cudaError_t gram_f64_fx(const double *A, long lda, const unsigned *bA, const double *B,
                        long ldb, const unsigned *bB, long nd, int ns, double *G, double *part,
                        cudaStream_t st, bool sym)
{
    if (ns <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_gram_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // one wave of CTAs: two resident per SM, the active tiles times the slices
    const int nt = (ns + FT - 1) / FT;
    const int tiles = sym ? nt * (nt + 1) / 2 : nt * nt;
    int nsplit = 2 * 152 / tiles;
    const int cap = gram_default_splits(ns, nd);  // the partial buffer holds this many
    if (nsplit > cap) nsplit = cap;
    if ((long)nsplit * kChunk > nd) nsplit = (int)((nd + kChunk - 1) / kChunk);
    if (nsplit < 1) nsplit = 1;
    long rows_per = (nd + nsplit - 1) / nsplit;
    rows_per = (rows_per + FK - 1) / FK * FK;
    // slice sums stay below 2^63: chunks per slice <= 2^sh, each chunk sum < 2^62 + 2^36
    const long chunks = (rows_per + kChunk - 1) / kChunk;
    int sh = 0;
    while ((1L << sh) < chunks + 1) ++sh;
    dim3 grid((ns + FT - 1) / FT, (ns + FT - 1) / FT, nsplit);
    k_gram_fx<<<grid, kThreads, kSmemBytes, st>>>(A, lda, bA, B, ldb, bB, nd, ns, rows_per, sh,
                                                  sym ? 1 : 0, part);
    note_launch();
    const long nn = (long)ns * ns;
    int rb = (int)((nn + 255) / 256);
    if (rb > 152 * 16) rb = 152 * 16;
    k_gram_fx_reduce<<<rb, 256, 0, st>>>(part, nsplit, ns, sym ? 1 : 0, G);
    note_launch();
    return cudaGetLastError();
}

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
