// gram_tc.cu -- the subspace contractions on the tensor cores (tcgen05):
//   M_s = Y^T Y  and  H_s = Y^T (H Y)   (projection onto the filtered block, Sec. 3.4),
// G = A^T B over the Nd grid rows, and the rotation X = Y (L^-T Q) (Eq.
// OrbitalTransformation). Two digit representations share one kernel: 47 bits (six digits;
// the Gram pair of both forms, FP64 or FP32 Y, and the FP64 form's rotation) and 23 bits
// (three digits; sparc_gram_tc and the mixed form's FP32 rotation). The description below
// is of the 23-bit form; the 47-bit form differs as stated at struct Tc47.
//
// The scheme is a fixed-point form of the error-free splitting of a matrix product into
// slices whose products the hardware forms exactly (the Ozaki scheme: K. Ozaki, T. Ogita,
// S. Oishi and S. M. Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applicability", Numer. Algorithms 59,
// 2012), with per-chunk scaling so that the slices are small integers and the tensor
// core's FP32 accumulator sums them exactly, in the manner of the integer-unit emulations of
// FP64 products (H. Ootomo, K. Ozaki and R. Yokota, "DGEMM on integer matrix
// multiplication unit", IJHPCA 2024).
//
// Representation. The rows are cut into chunks of kChunk = 256. For chunk c and column j
// of an operand, e = e(c, j) is the smallest integer with max_{k in c} |x_kj| < 2^e, and
// each entry is rounded to N = round(|x| 2^(23 - e)), an integer in [0, 2^23], written in
// three balanced base-256 digits N = d1 2^16 + d2 2^8 + d3 with 0 <= d1 <= 128 and
// -128 <= d2, d3 <= 127 (signs carried by the digits). Every digit is an integer of at most
// 8 bits, held exactly by BF16. So x = 2^(e - 23) (d1 2^16 + d2 2^8 + d3) up to 2^-24 of
// the chunk's largest entry (about the rounding the FP32 block already carries).
//
// Exact accumulation. A product of two digits is an integer below 2^14 in magnitude,
// exact in the tensor core's FP32 accumulator. The digit pairs (s, t) are grouped by
// class w = s + t (0-based digits), whose weight is 2^(-8 w) relative to class 0; classes
// 0, 1, 2 are kept (6 digit products per 16 rows, one tensor-memory accumulator per class)
// and classes 3, 4 (products below 2^-22 of the leading term) are dropped. Per chunk a class
// accumulator holds at most 3 x 2^14 x 256 < 2^24 in magnitude, so its FP32 sums are
// exact integers. After each chunk the epilogue warps read the three accumulators from
// tensor memory, combine them exactly into an FP32 pair (TwoSum), scale the pair by the
// chunk's power of two 2^(e_i + e_j - 14) and add it to FP32-pair running sums (error about
// 2^-48 relative). The result is the Gram matrix of the 23-bit rounded block with no error
// growth along Nd; the FP32-pair Gram of gram_df.cu remains the exact one.
//
// Layout and pipeline. A pre-pass (k_tc_digits) writes the digits of an operand in the
// shared-memory order the MMA reads (no swizzle, K-major, 8-row x 16-byte core matrices)
// as 8 KB blobs, one per (128-column block, 32-row step, digit), plus the exponents
// e(c, j). A CTA owns one 128 x 128 tile of G over a range of chunks (split-K): warp 0
// streams the blobs of A and B into a three-stage ring with untiled bulk copies (48 KB a
// stage; B's digits side by side along N), one thread of warp 1 issues the tcgen05.mma
// (M = 128, K = 16): per A digit s one MMA over the B digits 0 .. 2 - s at once (N = 384 as
// 256 + 128, then 256, then 128), which writes the class accumulators s .. 2 side by side
// (384 tensor-memory columns) and reads the A digit once instead of once per product; it
// commits stage releases and chunk completions to mbarriers, and eight epilogue warps (two per tensor-memory lane quarter,
// 64 columns each; high parts of the running sums in registers, low parts in shared
// memory) flush every chunk. Partial tiles of the K splits are summed by a
// second kernel in a fixed order (deterministic). Every wait is bounded; on a timeout the
// kernel raises *err, drains its copies and MMAs (bounded), frees its tensor memory and
// returns.
#include "internal.cuh"

#include <atomic>
#include "tma.cuh"

#include <cstdint>
#include <cuda_bf16.h>

namespace sparc {

namespace {
constexpr int kTile = 128;                     // MMA M (A columns per tile)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr unsigned kWaitLimit = 1u << 22;
constexpr int kTmemCols = 512;
constexpr int kNonFinite = INT32_MIN;          // exponent sentinel of a chunk with Inf/NaN
// core-matrix offsets inside a blob (elements): K-adjacent cores 2048 B apart, M/N-adjacent
// cores 128 B apart
constexpr unsigned kLbo = 2048, kSbo = 128;
}  // namespace

// The representations. Tc23: entries rounded to 23 bits of the chunk's largest, three
// base-256 digits, classes 0..2, 256-row chunks, 128 x 128 tiles (sparc_gram_tc, the mixed
// form's rotation). Tc47: 47 bits, six base-256 digits, classes 0..5 (21 digit products per
// 16 rows, issued as 8 MMAs of N = 64 .. 256 over the digit-concatenated B; a class sums at
// most six digit products, so 128-row chunks keep it below 2^24), 128 x 64 half tiles (six
// class accumulators of 64 columns fit the 512 tensor-memory columns): the Gram pairs of
// both forms and the FP64 form's rotation. The digit base is a
// parameter (kBase bits); kScale = kBits - kBase (kDigits - 1), so that
// x = 2^(e - kScale) sum_s d_s 2^(-kBase s).
struct Tc23 {
    static constexpr int kDigits = 3, kClasses = 3, kBits = 23, kChunk = 256, kStep = 32,
                         kN = 128, kStages = 3, kBase = 8;
};
struct Tc47 {
    static constexpr int kDigits = 6, kClasses = 6, kBits = 47, kChunk = 128, kStep = 16,
                         kN = 64, kStages = 4, kBase = 8;
};
// A stage holds A's blobs (all 128 columns of each digit) and the kN columns of B's blobs
// this CTA multiplies. B is stored digit-concatenated: per 8-row K group, the kN / 8 core
// matrices of digit 0, then those of digit 1, ... (kDigits kN columns, each piece copied
// from one contiguous run of a blob's K group), so that one MMA with N = nb kN multiplies
// an A digit by nb consecutive B digits at once and writes the nb class accumulators that
// sit side by side in tensor memory. B's K-adjacent cores are kDigits kN 16 B apart.
template <class C> struct TcDims {
    static constexpr int kStepsPerChunk = C::kChunk / C::kStep;
    static constexpr int kBlobElems = kTile * C::kStep;                    // BF16 per blob
    static constexpr unsigned kOperandBytes = C::kDigits * kBlobElems * 2;
    static constexpr unsigned kBPiece = C::kN * 16;            // one digit's cores of a K group
    static constexpr unsigned kBLbo = C::kDigits * kBPiece;     // B K-group stride
    static constexpr unsigned kBOperandBytes = C::kDigits * C::kN * C::kStep * 2;
    static constexpr unsigned kStageBytes = kOperandBytes + kBOperandBytes;
    static constexpr int kHalves = kTile / C::kN;                          // CTAs per tile
    static constexpr int kEpiCols = C::kN / 2;                             // per epilogue warp
    // ring, then the low parts of the epilogue's running pair sums ([warp][column][lane])
    static constexpr unsigned kLowBytes = kEpiWarps * kEpiCols * 32 * 4;
    static constexpr unsigned kSmemBytes = C::kStages * kStageBytes + kLowBytes + 1024;
    static_assert(kSmemBytes <= 227 * 1024, "shared memory of one CTA");
    static_assert(C::kClasses * C::kN <= kTmemCols, "class accumulators exceed tensor memory");
    static_assert(C::kBits <= C::kBase * C::kDigits - 1,
                  "top digit must stay within [0, 2^(kBase - 1)]");
    // a class sums at most kClasses digit products of magnitude <= 2^(2 kBase - 2) per row:
    // exact in the FP32 accumulator over a chunk
    static_assert(((long)C::kClasses << (2 * C::kBase - 2)) * C::kChunk < (1L << 24),
                  "class sums of a chunk must stay exact in FP32");
    static constexpr int kScale = C::kBits - C::kBase * (C::kDigits - 1);
};

namespace {
template <class C>
__device__ __forceinline__ long blob_offset(int cb, long step, int s, long nstep)
{
    return (((long)cb * nstep + step) * C::kDigits + s) * TcDims<C>::kBlobElems;
}

__device__ __forceinline__ int in_blob(int k, int c)  // k: row in step, c: column (0..127)
{
    return ((((k >> 3) * 16 + (c >> 3)) * 8 + (c & 7)) * 8) + (k & 7);
}

// |x| as an unsigned integer (monotonic in |x| for finite x), exponent bits and significand
template <typename T> struct FBits;
template <> struct FBits<float> {
    using U = uint32_t;
    static constexpr int kMant = 23, kBias = 127, kExpMask = 0xFF;
    __device__ static U mag(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
    __device__ static bool neg(float x) { return (__float_as_uint(x) >> 31) != 0; }
};
template <> struct FBits<double> {
    using U = unsigned long long;
    static constexpr int kMant = 52, kBias = 1023, kExpMask = 0x7FF;
    __device__ static U mag(double x) { return (U)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull; }
    __device__ static bool neg(double x) { return __double_as_longlong(x) < 0; }
};
}  // namespace

// Digits and exponents of one operand. CTA: one chunk (blockIdx.y) x 8 columns
// (blockIdx.x), one warp per column, kChunk / 32 rows per lane. Rows past nd and columns
// past ns are zero; a chunk column holding Inf or NaN gets the exponent kNonFinite.
template <class C, typename T>
__global__ void __launch_bounds__(256)
k_tc_digits(const T *__restrict__ X, long ld, long nd, int ns, long nstep,
            __nv_bfloat16 *__restrict__ D, int *__restrict__ E, int ns_pad)
{
    using B = FBits<T>;
    using U = typename B::U;
    constexpr int R = C::kChunk / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = blockIdx.x * 8 + warp;
    const long chunk = blockIdx.y;
    const long k0 = chunk * C::kChunk;
    U mag[R];
    bool ng[R];
    U mx = 0;
    bool bad = false;
    const U inf = (U)B::kExpMask << B::kMant;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const long k = k0 + lane + 32 * u;
        T x = (T)0;
        if (col < ns && k < nd) x = X[k + (long)col * ld];
        mag[u] = B::mag(x);
        ng[u] = B::neg(x);
        bad |= mag[u] >= inf;
        mx = mag[u] > mx ? mag[u] : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U t = (U)__shfl_xor_sync(0xffffffffu, (unsigned long long)mx, o);
        mx = t > mx ? t : mx;
    }
    bad = __any_sync(0xffffffffu, bad);
    // max |x| < 2^e: e = unbiased exponent of the max + 1 (normal), 1 - bias + 1 for
    // subnormals; 0 for an all-zero chunk column
    const int bxm = (int)(mx >> B::kMant);
    const int e = mx == 0 ? 0 : (bxm == 0 ? 2 - B::kBias : bxm - B::kBias + 1);
    if (lane == 0 && col < ns_pad) E[chunk * ns_pad + col] = bad ? kNonFinite : e;
    const int cb = col >> 7, c = col & 127;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const long k = k0 + lane + 32 * u;
        long N = 0;
        if (!bad && mag[u] != 0) {
            const int bx = (int)(mag[u] >> B::kMant);
            const U m = (mag[u] & (((U)1 << B::kMant) - 1)) | (bx ? ((U)1 << B::kMant) : 0);
            const int ebx = bx ? bx : 1;
            // N = round(m 2^(ebx - bias - mant + kBits - e)) in [0, 2^kBits]
            const int sh = e + B::kBias + B::kMant - C::kBits - ebx;
            if (sh <= 0)
                N = (long)m << (-sh);  // exact: FP32 inputs of the 47-bit form
            else if (sh < 8 * (int)sizeof(U))
                N = (long)((m + ((U)1 << (sh - 1))) >> sh);
        }
        // balanced base-2^kBase digits from the bottom; the top one lies in
        // [0, 2^(kBase - 1)]
        constexpr long kHalf = 1L << (C::kBase - 1), kMask = (1L << C::kBase) - 1;
        int d[C::kDigits];
#pragma unroll
        for (int s = C::kDigits - 1; s > 0; --s) {
            d[s] = (int)(((N + kHalf) & kMask) - kHalf);
            N = (N - d[s]) >> C::kBase;
        }
        d[0] = (int)N;
        const int sg = ng[u] ? -1 : 1;
        const long step = k / C::kStep;
        const int kl = (int)(k % C::kStep);
        if (col < ns_pad) {
            const long base = blob_offset<C>(cb, step, 0, nstep) + in_blob(kl, c);
#pragma unroll
            for (int s = 0; s < C::kDigits; ++s)
                D[base + (long)s * TcDims<C>::kBlobElems] = __float2bfloat16_rn((float)(sg * d[s]));
        }
    }
}

// 2^(e - kScale) as an FP32 factor (the chunk scale 2^(e_i + e_j - 2 kScale) is applied as
// two such factors, each exact); 0 below the FP32 normal range, NaN for a non-finite chunk.
template <class C>
__device__ __forceinline__ float pow2_factor(int e)
{
    if (e == kNonFinite) return __int_as_float(0x7FC00000);
    const int b = e - TcDims<C>::kScale + 127;
    if (b <= 0) return 0.0f;
    if (b >= 255) return __int_as_float(0x7F800000);
    return __int_as_float(b << 23);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// FP32 -> FP64 by moving the exponent field (integer operations; FP32 subnormals count as
// zero, Inf / NaN stay so): the rotation writes one output per thread and column, where an
// FP64 conversion instruction per value would load the FP64 pipe.
__device__ __forceinline__ double widen_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sg = u & 0x80000000u;
    unsigned hi = sg | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0u) hi = sg, lo = 0u;
    if (e == 0xffu) hi = sg | 0x7ff00000u | (m ? 0x80000u : 0u), lo = 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// Digits of the transposed operand: B = Y^T for the rotation, so the K dimension runs over
// Y's columns and each Y row gets its own exponent per chunk of kChunk columns. CTA: 32
// rows (lanes) x the chunk's kChunk / 8 groups of 8 columns (warps): loads are coalesced
// across lanes, the row's largest entry is reduced through shared memory, and each thread
// writes its 8 values of a digit as one 16-byte store (the 8 K-adjacent elements of a core
// matrix row are contiguous, and the 32 rows of a warp fill 512 contiguous bytes). Rows past
// nd and columns past ns are zero.
template <class C, typename T>
__global__ void __launch_bounds__(32 * (C::kChunk / 8))
k_tc_digits_t(const T *__restrict__ Y, long ld, long nd, int ns, long nstep,
              __nv_bfloat16 *__restrict__ D, int *__restrict__ E, long nd_pad)
{
    using B = FBits<T>;
    using U = typename B::U;
    constexpr int G = C::kChunk / 8;  // column groups (warps)
    __shared__ U red[G][32];
    __shared__ int bad_s[G][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long row = (long)blockIdx.x * 32 + lane;
    const long chunk = blockIdx.y;
    const int kb = (int)(chunk * C::kChunk) + g * 8;  // first column of this thread's group
    const bool live = row < nd;
    T x[8];
    U mx = 0;
    int bad = 0;
    const U inf = (U)B::kExpMask << B::kMant;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        x[t] = (live && kb + t < ns) ? Y[row + (long)(kb + t) * ld] : (T)0;
        const U m = B::mag(x[t]);
        bad |= m >= inf;
        mx = m > mx ? m : mx;
    }
    red[g][lane] = mx;
    bad_s[g][lane] = bad;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < G; ++q) {
        mx = red[q][lane] > mx ? red[q][lane] : mx;
        bad |= bad_s[q][lane];
    }
    const int bxm = (int)(mx >> B::kMant);
    const int e = mx == 0 ? 0 : (bxm == 0 ? 2 - B::kBias : bxm - B::kBias + 1);
    if (g == 0 && row < nd_pad) E[chunk * nd_pad + row] = bad ? kNonFinite : e;
    if (row >= nd_pad) return;
    // each value's magnitude on the grid and its sign; the digits are then peeled off from
    // the bottom and each digit's 8 values stored at once (16 bytes: the 8 K-adjacent
    // elements of a core-matrix row; the 32 rows of a warp fill 512 contiguous bytes)
    long N[8];
    unsigned neg = 0u;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const U mag = B::mag(x[t]);
        N[t] = 0;
        if (!bad && mag != 0) {
            const int bx = (int)(mag >> B::kMant);
            const U m = (mag & (((U)1 << B::kMant) - 1)) | (bx ? ((U)1 << B::kMant) : 0);
            const int ebx = bx ? bx : 1;
            const int sh = e + B::kBias + B::kMant - C::kBits - ebx;
            if (sh <= 0)
                N[t] = (long)m << (-sh);
            else if (sh < 8 * (int)sizeof(U))
                N[t] = (long)((m + ((U)1 << (sh - 1))) >> sh);
        }
        neg |= (B::neg(x[t]) ? 1u : 0u) << t;
    }
    // the 8 columns kb .. kb+7 lie in one K-step (kStep is a multiple of 8) and one core
    const int cb = (int)(row >> 7), c = (int)(row & 127);
    const long base = blob_offset<C>(cb, kb / C::kStep, 0, nstep) + in_blob(kb % C::kStep, c);
    constexpr long kHalf = 1L << (C::kBase - 1), kMask = (1L << C::kBase) - 1;
#pragma unroll
    for (int s2 = C::kDigits - 1; s2 >= 0; --s2) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int dv;
            if (s2 > 0) {
                dv = (int)(((N[t] + kHalf) & kMask) - kHalf);
                N[t] = (N[t] - dv) >> C::kBase;
            } else {
                dv = (int)N[t];
            }
            v[t] = __float2bfloat16_rn((float)(((neg >> t) & 1u) ? -dv : dv));
        }
        *reinterpret_cast<uint4 *>(D + base + (long)s2 * TcDims<C>::kBlobElems) =
            *reinterpret_cast<const uint4 *>(v);
    }
}

// tiles[t] = (A column block, B column block); a tile is computed by kHalves CTAs, each
// for kN of its 128 B columns. part: nsplit x ntiles x 128 x 128 doubles, element (r, c) of
// a tile at r * 128 + c (r: A column, c: B column).
// Work units: a unit is one tile half (kN of the tile's 128 B columns) over a range of
// chunks. Gram mode: CTA b owns unit b (units = halves x tiles x splits). ROT (the rotation,
// see rotate_tc below): tile t is (t / mblk, t % mblk) over all chunks (mblk = B blocks, so
// the units that share an A block run side by side and find it in L2), the CTAs are
// persistent and walk units b, b + gridDim.x, ... with the ring, the MMAs and the epilogue
// running on across units; A's and B's exponents have the row strides ea_ld and eb_ld, and
// the epilogue writes out[i + j ldo] (i: A column, j: B column) for i < nrow, j < ncol, a
// warp's lanes covering 32 consecutive i (coalesced).
template <class C, bool ROT, typename TO = double>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const __nv_bfloat16 *__restrict__ DA, const int *__restrict__ EA,
          const __nv_bfloat16 *__restrict__ DB, const int *__restrict__ EB, int ns_pad, long nstep,
          const int2 *__restrict__ tiles, int ntiles, int nsplit, double *__restrict__ part,
          int *err, int eb_ld = 0, int mblk = 1, TO *__restrict__ out = nullptr, long ldo = 0,
          long nrow = 0, int ncol = 0, long ea_ld = 0)
{
    using Dm = TcDims<C>;
    constexpr int kStages = C::kStages, kStepsPerChunk = Dm::kStepsPerChunk;
    constexpr unsigned kStageBytes = Dm::kStageBytes, kOperandBytes = Dm::kOperandBytes;
    constexpr unsigned kBLbo = Dm::kBLbo, kBPiece = Dm::kBPiece;
    constexpr int kGroups = C::kStep / 8;  // 8-row K groups of a step
    constexpr int kEpiCols = Dm::kEpiCols;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full, acc_empty, drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    unsigned char *smem =
        (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long nchunk = nstep / kStepsPerChunk;
    const long ea_stride = ROT ? ea_ld : ns_pad;
    const int nunits = ROT ? ntiles * Dm::kHalves : (int)gridDim.x;
    const int ustride = ROT ? (int)gridDim.x : nunits;
    struct Unit {
        int hf, tile, split;
        int2 tb;
        long c0, c1;
    };
    auto unit = [&](int u) {
        Unit w;
        w.hf = u % Dm::kHalves;
        w.tile = (u / Dm::kHalves) % ntiles;
        w.split = u / (Dm::kHalves * ntiles);
        w.tb = ROT ? make_int2(w.tile / mblk, w.tile % mblk) : tiles[w.tile];
        w.c0 = ROT ? 0 : (long)w.split * nchunk / nsplit;
        w.c1 = ROT ? nchunk : (long)(w.split + 1) * nchunk / nsplit;
        return w;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, kEpiWarps);
        mbar_init(&drain, 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    if (warp == 1) tmem_alloc(&tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    auto fail = [&]() {
        abort_flag = 1;
        atomicExch(err, 1);
    };

    if (warp == 0) {
        // ---- producer: A and B blobs of each step into the ring, unit after unit ----
        if (lane == 0) {
            long j = 0, issued = 0;  // steps handed to the ring over all units
            for (int u = blockIdx.x; u < nunits && !abort_flag; u += ustride) {
                const Unit w = unit(u);
                for (long st = w.c0 * kStepsPerChunk; st < w.c1 * kStepsPerChunk && !abort_flag;
                     ++st, ++j) {
                    const int s = (int)(j % kStages);
                    if (j >= kStages &&
                        !mbar_wait(&empty[s], (unsigned)(((j / kStages) & 1) ^ 1), kWaitLimit)) {
                        fail();
                        break;
                    }
                    unsigned char *dst = smem + (size_t)s * kStageBytes;
                    mbar_arrive_expect_tx(&full[s], kStageBytes);
                    bulk_load(dst, DA + blob_offset<C>(w.tb.x, st, 0, nstep), kOperandBytes,
                              &full[s]);
                    // this unit's kN columns of every digit and K group of B, digit-concatenated
#pragma unroll
                    for (int d = 0; d < C::kDigits; ++d)
#pragma unroll
                        for (int g = 0; g < kGroups; ++g)
                            bulk_load(dst + kOperandBytes + g * kBLbo + d * kBPiece,
                                      DB + blob_offset<C>(w.tb.y, st, d, nstep) + g * (kTile * 8) +
                                          w.hf * (C::kN * 8),
                                      kBPiece, &full[s]);
                    issued = j + 1;
                }
            }
            if (abort_flag) {
                // wait (bounded) for the last copy issued into each stage
                for (int s = 0; s < kStages; ++s) {
                    long last = -1;
                    for (long q = s; q < issued; q += kStages) last = q;
                    if (last >= 0)
                        mbar_wait(&full[s], (unsigned)((last / kStages) & 1), kWaitLimit);
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            long j = 0, cc = 0;  // steps and chunks over all units
            for (int u = blockIdx.x; u < nunits && !abort_flag; u += ustride) {
                const Unit w = unit(u);
                const long st0 = w.c0 * kStepsPerChunk;
                for (long st = st0; st < w.c1 * kStepsPerChunk && !abort_flag; ++st, ++j) {
                    const int s = (int)(j % kStages);
                    const int kin = (int)((st - st0) % kStepsPerChunk);
                    if (kin == 0 && cc > 0) {
                        if (!mbar_wait(&acc_empty, (unsigned)((cc - 1) & 1), kWaitLimit)) {
                            fail();
                            break;
                        }
                        tc_fence_after();
                    }
                    if (!mbar_wait(&full[s], (unsigned)((j / kStages) & 1), kWaitLimit)) {
                        fail();
                        break;
                    }
                    tc_fence_after();
                    const unsigned char *a = smem + (size_t)s * kStageBytes;
                    const unsigned char *b = a + kOperandBytes;
#pragma unroll
                    for (int ks = 0; ks < C::kStep / 16; ++ks) {
#pragma unroll
                        for (int sa = 0; sa < C::kDigits; ++sa) {
                            // A digit sa times B digits 0 .. nb-1 (classes sa .. sa+nb-1, the
                            // kept ones), as MMAs of N <= 256 over the digit-concatenated B
                            const int nb = C::kClasses - sa < C::kDigits ? C::kClasses - sa
                                                                         : C::kDigits;
                            const uint64_t ad =
                                smem_desc(a + sa * Dm::kBlobElems * 2 + ks * 2 * kLbo, kLbo, kSbo);
#pragma unroll
                            for (int n0 = 0; n0 < nb * C::kN; n0 += 256) {
                                const int nl = nb * C::kN - n0 < 256 ? nb * C::kN - n0 : 256;
                                const uint64_t bd =
                                    smem_desc(b + ks * 2 * kBLbo + (n0 / 8) * kSbo, kBLbo, kSbo);
                                // the sa = 0 MMAs cover every class: at a chunk start they
                                // overwrite the accumulators, all later ones accumulate
                                const bool first = kin == 0 && ks == 0 && sa == 0;
                                tc_mma_bf16(tmem + (uint32_t)(sa * C::kN + n0), ad, bd,
                                            idesc_bf16_f32(kTile, nl), !first);
                            }
                        }
                    }
                    tc_commit(&empty[s]);  // stage free once these MMAs are done
                    if (kin == kStepsPerChunk - 1) {
                        tc_commit(&acc_full);  // chunk complete
                        ++cc;
                    }
                }
            }
            // all MMAs issued by this thread are complete before tensor memory is freed
            tc_commit(&drain);
            if (!mbar_wait(&drain, 0u, kWaitLimit)) fail();
        }
    } else {
        // ---- epilogue: flush each chunk's class accumulators into FP32-pair sums ----
        const int q = warp & 3;                 // tensor-memory lane quarter of this warp
        const int hw = (warp - 2) >> 2;         // columns kEpiCols hw .. of this CTA's kN
        const int r = q * 32 + lane;            // tile row = A column within the block
        float H[kEpiCols];
        float *Lw = reinterpret_cast<float *>(smem + (size_t)kStages * kStageBytes) +
                    (size_t)(warp - 2) * kEpiCols * 32 + lane;  // Lw[u * 32]: column u
        long cc = 0;  // chunks over all units
        bool ok = true;
        // the chunk exponents are loaded one chunk ahead (they do not depend on the MMAs):
        // this thread's A column, and kEpiCols / 32 of the warp's B columns per lane, whose
        // factors reach the other lanes by shuffle
        constexpr int kEB = kEpiCols / 32;
        const long eb_stride = ROT ? eb_ld : ns_pad;
        for (int u = blockIdx.x; u < nunits && ok; u += ustride) {
            const Unit w = unit(u);
            const long colA = (long)w.tb.x * kTile + r;
            const int *ebw = EB + (long)w.tb.y * kTile + w.hf * C::kN + hw * kEpiCols + lane;
#pragma unroll
            for (int x = 0; x < kEpiCols; ++x) {
                H[x] = 0.0f;
                Lw[x * 32] = 0.0f;
            }
            int ea_n = EA[w.c0 * ea_stride + colA], eb_n[kEB];
#pragma unroll
            for (int k = 0; k < kEB; ++k) eb_n[k] = ebw[w.c0 * eb_stride + 32 * k];
            for (long c = w.c0; c < w.c1; ++c, ++cc) {
                const float fA = pow2_factor<C>(ea_n);
                float fb[kEB];
#pragma unroll
                for (int k = 0; k < kEB; ++k) fb[k] = pow2_factor<C>(eb_n[k]);
                if (c + 1 < w.c1) {
                    ea_n = EA[(c + 1) * ea_stride + colA];
#pragma unroll
                    for (int k = 0; k < kEB; ++k) eb_n[k] = ebw[(c + 1) * eb_stride + 32 * k];
                }
                ok = mbar_wait(&acc_full, (unsigned)(cc & 1), kWaitLimit) && !abort_flag;
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) fail();
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int g = 0; g < kEpiCols / 8; ++g) {
                    const uint32_t ta =
                        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hw * kEpiCols + g * 8);
                    uint32_t v[C::kClasses][8];
#pragma unroll
                    for (int cl = 0; cl < C::kClasses; ++cl)
                        tmem_ld8(ta + (uint32_t)(cl * C::kN), v[cl]);
                    tmem_wait_ld();
#pragma unroll
                    for (int x = 0; x < 8; ++x) {
                        // sum_w class_w 2^(-8 w) as a pair (each class value an exact integer)
                        float h = __uint_as_float(v[0][x]), l = 0.0f;
                        float wt = 1.0f;
#pragma unroll
                        for (int cl = 1; cl < C::kClasses; ++cl) {
                            wt *= 1.0f / (float)(1 << C::kBase);  // 2^-kBase
                            float t, e2;
                            two_sum_f(h, __uint_as_float(v[cl][x]) * wt, t, e2);
                            h = t;
                            l += e2;
                        }
                        const float f =
                            fA * __shfl_sync(0xffffffffu, fb[(g * 8 + x) / 32], (g * 8 + x) % 32);
                        const float ph = h * f, pl = l * f;
                        float sh, se;
                        two_sum_f(H[g * 8 + x], ph, sh, se);
                        H[g * 8 + x] = sh;
                        Lw[(g * 8 + x) * 32] += se + pl;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty);
            }
            if (!ok) break;
            if (ROT) {
                const long i = (long)w.tb.x * kTile + r;
                const long j0 = (long)w.tb.y * kTile + w.hf * C::kN + hw * kEpiCols;
                if (i < nrow) {
                    TO *o = out + i + j0 * ldo;
#pragma unroll
                    for (int x = 0; x < kEpiCols; ++x) {
                        if (j0 + x >= ncol) continue;
                        if constexpr (sizeof(TO) == 4)
                            o[(long)x * ldo] = H[x] + Lw[x * 32];  // the pair rounded to FP32
                        else
                            o[(long)x * ldo] = widen_int(H[x]) + widen_int(Lw[x * 32]);
                    }
                }
            } else {
                double *o = part + ((long)w.split * ntiles + w.tile) * kTile * kTile +
                            (long)r * kTile + w.hf * C::kN + hw * kEpiCols;
#pragma unroll
                for (int x = 0; x < kEpiCols; ++x) o[x] = (double)H[x] + (double)Lw[x * 32];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// G from the split partials, summed in split order; sym mirrors each off-diagonal tile.
__global__ void k_gram_tc_reduce(const double *__restrict__ part, const int2 *__restrict__ tiles,
                                 int ntiles, int nsplit, int ns, bool sym, double *G)
{
    const long tot = (long)ntiles * kTile * kTile;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (long)gridDim.x * blockDim.x) {
        const int tile = (int)(t / (kTile * kTile));
        const int e = (int)(t % (kTile * kTile));
        const int r = e / kTile, c = e % kTile;
        const int2 tb = tiles[tile];
        const int i = tb.x * kTile + r, j = tb.y * kTile + c;
        if (i >= ns || j >= ns) continue;
        double v = 0.0;
        for (int s = 0; s < nsplit; ++s) v += part[((long)s * ntiles + tile) * kTile * kTile + e];
        G[i + (long)j * ns] = v;
        if (sym && tb.x != tb.y) G[j + (long)i * ns] = v;
    }
}

// ---- host side -------------------------------------------------------------------------

namespace {
struct TcPlan {
    int ns_pad, nblk, ntiles, nsplit;
    long nstep, nchunk;
    size_t digits_bytes, exps_bytes, part_bytes, tiles_bytes;
};

template <class C>
TcPlan tc_plan(long nd, int ns, bool sym)
{
    TcPlan p;
    p.nblk = (ns + kTile - 1) / kTile;
    p.ns_pad = p.nblk * kTile;
    p.nchunk = (nd + C::kChunk - 1) / C::kChunk;
    p.nstep = p.nchunk * TcDims<C>::kStepsPerChunk;
    p.ntiles = sym ? p.nblk * (p.nblk + 1) / 2 : p.nblk * p.nblk;
    // K splits: one CTA per SM (the ring and the class accumulators fill an SM), so the
    // kernel takes (waves of 152 CTAs) x (chunks per split). Pick the split count with the
    // fewest chunk-times, counting about two chunks of fixed cost per CTA (set-up and the
    // partial tile's store), and keep the partial tiles within 256 MB.
    const long ctas = (long)p.ntiles * TcDims<C>::kHalves;
    const long smax_mem = ((long)256 << 20) / ((long)p.ntiles * kTile * kTile * 8);
    long smax = p.nchunk < smax_mem ? p.nchunk : smax_mem;
    if (smax > 1024) smax = 1024;
    long best_s = 1, best = -1;
    for (long s = 1; s <= smax; ++s) {
        const long waves = (ctas * s + 151) / 152;
        const long cost = waves * ((p.nchunk + s - 1) / s + 2);
        if (best < 0 || cost < best) best = cost, best_s = s;
    }
    p.nsplit = (int)best_s;
    p.digits_bytes = (size_t)C::kDigits * p.ns_pad * p.nstep * C::kStep * 2;
    p.exps_bytes = (size_t)p.nchunk * p.ns_pad * sizeof(int);
    p.part_bytes = (size_t)p.nsplit * p.ntiles * kTile * kTile * sizeof(double);
    p.tiles_bytes = (size_t)p.ntiles * sizeof(int2);
    return p;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class C>
size_t tc_workspace(long nd, int ns, bool same_operand, bool sym)
{
    const TcPlan p = tc_plan<C>(nd, ns, sym);
    const int nops = same_operand ? 1 : 2;
    return nops * (align256(p.digits_bytes) + align256(p.exps_bytes)) + align256(p.part_bytes) +
           align256(p.tiles_bytes);
}
}  // namespace

size_t gram_tc_workspace(long nd, int ns, bool same_operand, bool sym)
{
    return tc_workspace<Tc23>(nd, ns, same_operand, sym);
}
size_t gram_tc47_workspace(long nd, int ns) { return tc_workspace<Tc47>(nd, ns, false, true); }

template <class C, typename T>
static cudaError_t tc_digits(const T *X, long ld, long nd, int ns, const TcPlan &p,
                             __nv_bfloat16 *D, int *E, cudaStream_t st)
{
    if (p.nchunk > 65535) return cudaErrorInvalidValue;
    dim3 grid(p.ns_pad / 8, (unsigned)p.nchunk);
    k_tc_digits<C, T><<<grid, 256, 0, st>>>(X, ld, nd, ns, p.nstep, D, E, p.ns_pad);
    note_launch();
    return cudaGetLastError();
}

// Tile list (host-built, uploaded) and the kernel's shared-memory attribute.
template <class C>
static cudaError_t tc_prepare(const TcPlan &p, bool sym, int2 *tiles, cudaStream_t st)
{
    static std::atomic<bool> attr_set{false};  // set once (several host threads may launch)
    cudaError_t e;
    if (!attr_set.load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(k_gram_tc<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcDims<C>::kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set.store(true, std::memory_order_release);
    }
    static thread_local int2 host_tiles[64 * 65 / 2 + 64 * 64];
    if (p.ntiles > (int)(sizeof(host_tiles) / sizeof(int2))) return cudaErrorInvalidValue;
    int n = 0;
    for (int a = 0; a < p.nblk; ++a)
        for (int b = (sym ? a : 0); b < p.nblk; ++b) host_tiles[n++] = make_int2(a, b);
    return cudaMemcpyAsync(tiles, host_tiles, p.tiles_bytes, cudaMemcpyHostToDevice, st);
}

template <class C>
static cudaError_t tc_run(const TcPlan &p, const __nv_bfloat16 *DA, const int *EA,
                          const __nv_bfloat16 *DB, const int *EB, const int2 *tiles,
                          double *part, int ns, bool sym, double *G, int *err, cudaStream_t st)
{
    const int ctas = p.ntiles * p.nsplit * TcDims<C>::kHalves;
    k_gram_tc<C, false><<<ctas, kThreads, TcDims<C>::kSmemBytes, st>>>(DA, EA, DB, EB, p.ns_pad, p.nstep,
                                                                tiles, p.ntiles, p.nsplit, part,
                                                                err);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gram_tc_reduce<<<152 * 4, 256, 0, st>>>(part, tiles, p.ntiles, p.nsplit, ns, sym, G);
    note_launch();
    return cudaGetLastError();
}

template <class C, typename TA, typename TB>
static cudaError_t gram_tc_impl(const TA *A, long lda, const TB *B, long ldb, long nd, int ns,
                                double *G, void *ws, size_t ws_bytes, bool sym, int *err,
                                cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaErrorInvalidValue;
    const bool same = (const void *)A == (const void *)B && sizeof(TA) == sizeof(TB) && lda == ldb;
    const TcPlan p = tc_plan<C>(nd, ns, sym);
    if (ws_bytes < tc_workspace<C>(nd, ns, same, sym)) return cudaErrorInvalidValue;
    unsigned char *w = (unsigned char *)ws;
    auto take = [&](size_t b) {
        unsigned char *r = w;
        w += align256(b);
        return r;
    };
    __nv_bfloat16 *DA = (__nv_bfloat16 *)take(p.digits_bytes);
    int *EA = (int *)take(p.exps_bytes);
    __nv_bfloat16 *DB = DA;
    int *EB = EA;
    if (!same) {
        DB = (__nv_bfloat16 *)take(p.digits_bytes);
        EB = (int *)take(p.exps_bytes);
    }
    double *part = (double *)take(p.part_bytes);
    int2 *tiles = (int2 *)take(p.tiles_bytes);

    cudaError_t e;
    if ((e = tc_prepare<C>(p, sym, tiles, st)) != cudaSuccess) return e;
    if ((e = tc_digits<C, TA>(A, lda, nd, ns, p, DA, EA, st)) != cudaSuccess) return e;
    if (!same && (e = tc_digits<C, TB>(B, ldb, nd, ns, p, DB, EB, st)) != cudaSuccess) return e;
    return tc_run<C>(p, DA, EA, DB, EB, tiles, part, ns, sym, G, err, st);
}

template <class C, typename TA, typename TB>
static cudaError_t gram_tc_pair_impl(const TA *A, long lda, const TB *B, long ldb, long nd,
                                     int ns, double *M, double *Hm, void *ws, size_t ws_bytes,
                                     int *err, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaErrorInvalidValue;
    const TcPlan p = tc_plan<C>(nd, ns, true);
    if (ws_bytes < tc_workspace<C>(nd, ns, false, true)) return cudaErrorInvalidValue;
    unsigned char *w = (unsigned char *)ws;
    auto take = [&](size_t b) {
        unsigned char *r = w;
        w += align256(b);
        return r;
    };
    __nv_bfloat16 *DA = (__nv_bfloat16 *)take(p.digits_bytes);
    int *EA = (int *)take(p.exps_bytes);
    __nv_bfloat16 *DB = (__nv_bfloat16 *)take(p.digits_bytes);
    int *EB = (int *)take(p.exps_bytes);
    double *part = (double *)take(p.part_bytes);
    int2 *tiles = (int2 *)take(p.tiles_bytes);
    cudaError_t e;
    if ((e = tc_prepare<C>(p, true, tiles, st)) != cudaSuccess) return e;
    if ((e = tc_digits<C, TA>(A, lda, nd, ns, p, DA, EA, st)) != cudaSuccess) return e;
    if ((e = tc_digits<C, TB>(B, ldb, nd, ns, p, DB, EB, st)) != cudaSuccess) return e;
    if ((e = tc_run<C>(p, DA, EA, DA, EA, tiles, part, ns, true, M, err, st)) != cudaSuccess)
        return e;
    return tc_run<C>(p, DA, EA, DB, EB, tiles, part, ns, true, Hm, err, st);
}

template <typename TA, typename TB>
cudaError_t gram_tc(const TA *A, long lda, const TB *B, long ldb, long nd, int ns, double *G,
                    void *ws, size_t ws_bytes, bool sym, int *err, cudaStream_t st)
{
    return gram_tc_impl<Tc23, TA, TB>(A, lda, B, ldb, nd, ns, G, ws, ws_bytes, sym, err, st);
}


template <typename TA>
cudaError_t gram_tc47_pair(const TA *A, long lda, const double *B, long ldb, long nd, int ns,
                           double *M, double *Hm, void *ws, size_t ws_bytes, int *err,
                           cudaStream_t st)
{
    return gram_tc_pair_impl<Tc47, TA, double>(A, lda, B, ldb, nd, ns, M, Hm, ws, ws_bytes, err,
                                               st);
}
template cudaError_t gram_tc47_pair<double>(const double *, long, const double *, long, long, int,
                                            double *, double *, void *, size_t, int *,
                                            cudaStream_t);
template cudaError_t gram_tc47_pair<float>(const float *, long, const double *, long, long, int,
                                           double *, double *, void *, size_t, int *,
                                           cudaStream_t);

// ---- rotation out = Y C on the tensor cores -----------------------------------------------
// Written as the contraction G = A^T B with A = Y^T (K = Ns: Y's columns, M = Nd: Y's rows)
// and B = C (N = Ns): G(i, j) = sum_k Y_ik C_kj = out(i, j). Y gets exponents per (K chunk,
// row), C per (K chunk, column), so every product in a class accumulator shares one scale.
// K = Ns is short, so a unit is one tile (Tc47: a 128 x 64 half tile) over all of K; the
// tensor-memory lanes hold Y's rows, so each store of the epilogue covers 32 consecutive rows
// of a column. The FP64 form uses the 47-bit digits (FP64 blocks, FP64 output); the mixed
// form the 23-bit digits (FP32 block or the FP64 H Y of its residuals, FP32 output): each
// entry of Y and C is rounded to 2^-24 of its chunk's largest, the rounding an FP32 result
// carries anyway, for 6 digit products per 16 K instead of 21.
namespace {
struct RotPlan {
    int ns_pad, mblk;
    long nblk, nd_pad, nchunk, nstep;
    size_t da_bytes, ea_bytes, db_bytes, eb_bytes;
};
template <class C>
RotPlan rot_plan(long nd, int ns)
{
    RotPlan p;
    p.mblk = (ns + kTile - 1) / kTile;
    p.ns_pad = p.mblk * kTile;
    p.nblk = (nd + kTile - 1) / kTile;
    p.nd_pad = p.nblk * kTile;
    p.nchunk = (ns + C::kChunk - 1) / C::kChunk;
    p.nstep = p.nchunk * TcDims<C>::kStepsPerChunk;
    p.da_bytes = (size_t)C::kDigits * p.ns_pad * p.nstep * C::kStep * 2;
    p.ea_bytes = (size_t)p.nchunk * p.ns_pad * sizeof(int);
    p.db_bytes = (size_t)C::kDigits * p.nd_pad * p.nstep * C::kStep * 2;
    p.eb_bytes = (size_t)p.nchunk * p.nd_pad * sizeof(int);
    return p;
}
template <class C>
size_t rot_workspace(long nd, int ns)
{
    const RotPlan p = rot_plan<C>(nd, ns);
    return align256(p.da_bytes) + align256(p.ea_bytes) + align256(p.db_bytes) +
           align256(p.eb_bytes);
}

template <class C, typename TY, typename TO>
cudaError_t rotate_tc_impl(const TY *Y, long ldy, long nd, int ns, const double *Cm, TO *out,
                           long ldo, void *ws, size_t ws_bytes, int *err, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaSuccess;
    const RotPlan p = rot_plan<C>(nd, ns);
    if (ws_bytes < rot_workspace<C>(nd, ns)) return cudaErrorInvalidValue;
    const long ctas = (long)p.mblk * p.nblk * TcDims<C>::kHalves;
    if (p.nchunk > 65535 || ctas > 0x7fffffffL || p.nd_pad / 32 > 0x7fffffffL)
        return cudaErrorInvalidValue;
    unsigned char *w = (unsigned char *)ws;
    auto take = [&](size_t b) {
        unsigned char *r = w;
        w += align256(b);
        return r;
    };
    __nv_bfloat16 *DA = (__nv_bfloat16 *)take(p.da_bytes);
    int *EA = (int *)take(p.ea_bytes);
    __nv_bfloat16 *DB = (__nv_bfloat16 *)take(p.db_bytes);
    int *EB = (int *)take(p.eb_bytes);
    static std::atomic<bool> attr_set{false};  // set once (several host threads may launch)
    cudaError_t e;
    if (!attr_set.load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(k_gram_tc<C, true, TO>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcDims<C>::kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set.store(true, std::memory_order_release);
    }
    {   // A = C: K = Ns rows, M = Ns columns
        dim3 grid(p.ns_pad / 8, (unsigned)p.nchunk);
        k_tc_digits<C, double><<<grid, 256, 0, st>>>(Cm, ns, ns, ns, p.nstep, DA, EA, p.ns_pad);
        note_launch();
    }
    {   // B = Y^T: K = Ns (Y's columns), N = Nd (Y's rows)
        dim3 grid((unsigned)(p.nd_pad / 32), (unsigned)p.nchunk);
        k_tc_digits_t<C, TY><<<grid, 32 * (C::kChunk / 8), 0, st>>>(Y, ldy, nd, ns, p.nstep, DB,
                                                                    EB, p.nd_pad);
        note_launch();
    }
    const unsigned grid = (unsigned)(ctas < 152 ? ctas : 152);  // persistent, one per SM
    // A: Y's digits (nblk row blocks, exponent stride nd_pad); B: C's (mblk column blocks,
    // the fastest tile index)
    k_gram_tc<C, true, TO><<<grid, kThreads, TcDims<C>::kSmemBytes, st>>>(
        DB, EB, DA, EA, p.ns_pad, p.nstep, nullptr, (int)(p.mblk * p.nblk), 1, nullptr, err,
        p.ns_pad, p.mblk, out, ldo, nd, ns, p.nd_pad);
    note_launch();
    return cudaGetLastError();
}
}  // namespace

size_t rotate_tc_workspace(long nd, int ns) { return rot_workspace<Tc47>(nd, ns); }
size_t rotate_tc23_workspace(long nd, int ns) { return rot_workspace<Tc23>(nd, ns); }

cudaError_t rotate_tc(const double *Y, long ldy, long nd, int ns, const double *Cm, double *out,
                      long ldo, void *ws, size_t ws_bytes, int *err, cudaStream_t st)
{
    return rotate_tc_impl<Tc47, double, double>(Y, ldy, nd, ns, Cm, out, ldo, ws, ws_bytes, err,
                                                st);
}

template <typename TY>
cudaError_t rotate_tc23(const TY *Y, long ldy, long nd, int ns, const double *Cm, float *out,
                        long ldo, void *ws, size_t ws_bytes, int *err, cudaStream_t st)
{
    return rotate_tc_impl<Tc23, TY, float>(Y, ldy, nd, ns, Cm, out, ldo, ws, ws_bytes, err, st);
}
template cudaError_t rotate_tc23<float>(const float *, long, long, int, const double *, float *,
                                        long, void *, size_t, int *, cudaStream_t);
template cudaError_t rotate_tc23<double>(const double *, long, long, int, const double *, float *,
                                         long, void *, size_t, int *, cudaStream_t);

__global__ void k_add_into(double *__restrict__ dst, const double *__restrict__ src, long n)
{
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long)gridDim.x * blockDim.x)
        dst[t] += src[t];
}

cudaError_t add_into(double *dst, const double *src, long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long b = (n + 255) / 256;
    k_add_into<<<(unsigned)(b < 1216 ? b : 1216), 256, 0, st>>>(dst, src, n);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t gram_tc<float, float>(const float *, long, const float *, long, long, int,
                                           double *, void *, size_t, bool, int *, cudaStream_t);
template cudaError_t gram_tc<float, double>(const float *, long, const double *, long, long, int,
                                            double *, void *, size_t, bool, int *, cudaStream_t);
template cudaError_t gram_tc<double, double>(const double *, long, const double *, long, long,
                                             int, double *, void *, size_t, bool, int *,
                                             cudaStream_t);

}  // namespace sparc
