// gram.cu -- subspace contractions of CheFSI (Sec. 3.4):
//   projection  M_s = Psi_f^T Psi_f,  H_s = Psi_f^T (H Psi_f)   (Eq. after
//               SubspaceGeneralizedEigenproblem), G = A^T B over Nd rows;
//   rotation    Psi = Psi_f Y  (Eq. OrbitalTransformation);
//   residuals   r_n = || H x_n - lambda_n x_n ||_2.
// All accumulate in FP64. A product of two FP32 values is exact in FP64, so the FP32
// blocks of the mixed-precision form lose nothing at the product step.
//
// Gram: a CTA computes a 64 x 64 tile of G over one slice of the Nd rows (split-K);
// the slices are summed by a second kernel in a fixed order (deterministic).
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int GT = 64;     // Gram tile (rows and columns of G)
constexpr int GK = 16;     // rows of A/B staged per step
constexpr int kSplitTarget = 152 * 4;  // CTAs wanted per launch
constexpr long kMinRowsPerSplit = 2048;

int gram_splits(int ns, long nd)
{
    const long tiles = (long)((ns + GT - 1) / GT) * ((ns + GT - 1) / GT);
    long s = (kSplitTarget + tiles - 1) / tiles;
    const long smax = (nd + kMinRowsPerSplit - 1) / kMinRowsPerSplit;
    if (s > smax) s = smax;
    if (s < 1) s = 1;
    if (s > 4096) s = 4096;
    return (int)s;
}
}  // namespace

long gram_part_elems(int ns, long nd) { return (long)gram_splits(ns, nd) * ns * ns; }

// All Gram contractions run in FP32-pair arithmetic (gram_df.cu); for FP32 inputs the
// products are exact there.
template <typename TA, typename TB>
static cudaError_t gram(const TA *A, long lda, const TB *B, long ldb, long nd, int ns, double *G,
                        double *part, cudaStream_t st, bool sym)
{
    return gram_df_launch<TA, TB>(A, lda, B, ldb, nd, ns, G, part, gram_splits(ns, nd), sym, st);
}

cudaError_t gram_f64(const double *A, long lda, const double *B, long ldb, long nd, int ns,
                     double *G, double *part, cudaStream_t st, bool sym)
{
    return gram<double, double>(A, lda, B, ldb, nd, ns, G, part, st, sym);
}
int gram_default_splits(int ns, long nd) { return gram_splits(ns, nd); }

cudaError_t gram_f64_nsplit(const double *A, long lda, const double *B, long ldb, long nd, int ns,
                            double *G, double *part, int nsplit, cudaStream_t st)
{
    return gram_df_launch<double, double>(A, lda, B, ldb, nd, ns, G, part, nsplit, false, st);
}

cudaError_t gram_f32_f32(const float *A, long lda, const float *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st, bool sym)
{
    return gram<float, float>(A, lda, B, ldb, nd, ns, G, part, st, sym);
}
cudaError_t gram_f32_f64(const float *A, long lda, const double *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st, bool sym)
{
    return gram<float, double>(A, lda, B, ldb, nd, ns, G, part, st, sym);
}

// ---- rotation of FP32 blocks: out = A Q in FP32 arithmetic (the rotated block is stored
// in FP32, and span(A Q') = span(A) for any invertible Q' close to Q, so the subspace the
// next filter starts from does not depend on this rounding). Tile 64 rows x 64 columns,
// Q staged 16 rows at a time. FP64 blocks use k_rotate_df (gram_df.cu). TA = double reads
// an FP64 block (rounded to FP32 on load): the FP32 form's rotated H Y_f for the residuals.
template <typename TA>
__global__ void __launch_bounds__(256)
k_rotate_f32(const TA *__restrict__ A, long lda, long nd, int ns, const double *__restrict__ Q,
             float *__restrict__ out, long ldo)
{
    __shared__ float As[GK][GT + 1];   // [k][row]
    __shared__ float Qs[GK][GT + 1];   // [k][col]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // the column tiles of one row tile are neighbours in the grid (x fastest), so the
    // row slice of A they share is read from DRAM once and from L2 by the others
    const int j0 = blockIdx.x * GT;
    for (long rt = blockIdx.y; rt * GT < nd; rt += gridDim.y) {
    const long r0 = rt * GT;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < ns; k0 += GK) {
        // A tile: 16 columns (k) x 64 rows; thread loads rows (t % 64), columns t/64 + 4u
        {
            const int rr = threadIdx.x & 63, kc = threadIdx.x >> 6;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kc + 4 * u;
                const long row = r0 + rr;
                As[k][rr] = (row < nd && k0 + k < ns) ? (float)A[row + (long)(k0 + k) * lda] : 0.0f;
            }
        }
        // Q tile: 16 rows (k) x 64 columns; thread loads k = t % 16, columns t/16 + 16u
        {
            const int kk = threadIdx.x & 15, cc = threadIdx.x >> 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = cc + 16 * u;
                Qs[kk][c] = (k0 + kk < ns && j0 + c < ns) ? (float)Q[(k0 + kk) + (long)(j0 + c) * ns]
                                                          : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                q[u] = Qs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], q[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const long row = r0 + ty + 16 * x;
            const int c = j0 + tx + 16 * y;
            if (row < nd && c < ns) out[row + (long)c * ldo] = acc[x][y];
        }
    __syncthreads();  // the next row tile reuses the shared tiles
    }
}

cudaError_t rotate_f64(const double *A, long lda, long nd, int ns, const double *Q, double *out,
                       long ldo, cudaStream_t st)
{
    return rotate_f64_df(A, lda, nd, ns, Q, out, ldo, st);
}
// Register-blocked form for large blocks: a CTA computes a 128 x 128 tile of out with 256
// threads, each an 8 x 8 sub-block (rows ty*4 + {0..3, 64..67}, columns tx*4 + {0..3,
// 64..67}); K (the columns of A) is staged 8 at a time through double-buffered shared
// memory, the next slice's global loads in flight during the current slice's FMAs.
constexpr int RT = 128, RK = 8;

template <typename TA>
__global__ void __launch_bounds__(256)
k_rotate_f32_big(const TA *__restrict__ A, long lda, long nd, int ns, const double *__restrict__ Q,
                 float *__restrict__ out, long ldo)
{
    __shared__ __align__(16) float As[2][RK][RT];   // [k][row]
    __shared__ __align__(16) float Qs[2][RK][RT];   // [k][col]
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int j0 = blockIdx.x * RT;  // column tiles of a row tile run side by side (L2 reuse)
    for (long rt = blockIdx.y; rt * RT < nd; rt += gridDim.y) {
    const long r0 = rt * RT;
    // global -> register staging: A slice 128 rows x 8 k, Q slice 8 k x 128 columns
    const int ar = t & 127, ak = t >> 7;        // rows ar, k = ak + 2u (u = 0..3)
    const int qk = t & 7, qc = t >> 3;          // k = qk, columns qc + 32u
    float ga[4], gq[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = ak + 2 * u;
            const long row = r0 + ar;
            ga[u] = (row < nd && k0 + k < ns) ? (float)A[row + (long)(k0 + k) * lda] : 0.0f;
            const int c = qc + 32 * u;
            gq[u] = (k0 + qk < ns && j0 + c < ns) ? (float)Q[(k0 + qk) + (long)(j0 + c) * ns] : 0.0f;
        }
    };
    auto stage = [&](int b) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[b][ak + 2 * u][ar] = ga[u];
            Qs[b][qk][qc + 32 * u] = gq[u];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.0f;
    load(0);
    stage(0);
    __syncthreads();
    int b = 0;
    for (int k0 = 0; k0 < ns; k0 += RK) {
        const bool more = k0 + RK < ns;
        if (more) load(k0 + RK);
#pragma unroll
        for (int kk = 0; kk < RK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[b][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[b][kk][64 + ty * 4]);
            const float4 q0 = *reinterpret_cast<const float4 *>(&Qs[b][kk][tx * 4]);
            const float4 q1 = *reinterpret_cast<const float4 *>(&Qs[b][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], q[y], acc[x][y]);
        }
        if (more) stage(b ^ 1);
        __syncthreads();
        b ^= 1;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const long row = r0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + x - 4);
        if (row >= nd) continue;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int c = j0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + y - 4);
            if (c < ns) out[row + (long)c * ldo] = acc[x][y];
        }
    }
    __syncthreads();  // the next row tile reuses the shared buffers
    }
}

template <typename TA>
static cudaError_t rotate_to_f32(const TA *A, long lda, long nd, int ns, const double *Q,
                                 float *out, long ldo, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaSuccess;
    if (ns >= 256) {
        const long gy = (nd + RT - 1) / RT;
        dim3 grid((ns + RT - 1) / RT, (unsigned)(gy < 65535 ? gy : 65535));
        k_rotate_f32_big<TA><<<grid, 256, 0, st>>>(A, lda, nd, ns, Q, out, ldo);
    } else {
        const long gy = (nd + GT - 1) / GT;
        dim3 grid((ns + GT - 1) / GT, (unsigned)(gy < 65535 ? gy : 65535));
        k_rotate_f32<TA><<<grid, 256, 0, st>>>(A, lda, nd, ns, Q, out, ldo);
    }
    note_launch();
    return cudaGetLastError();
}
cudaError_t rotate_f32(const float *A, long lda, long nd, int ns, const double *Q, float *out,
                       long ldo, cudaStream_t st)
{
    return rotate_to_f32<float>(A, lda, nd, ns, Q, out, ldo, st);
}
cudaError_t rotate_f64in_f32(const double *A, long lda, long nd, int ns, const double *Q,
                             float *out, long ldo, cudaStream_t st)
{
    return rotate_to_f32<double>(A, lda, nd, ns, Q, out, ldo, st);
}

// ---- residual norms: one CTA per column, fixed-order reduction -----------------------
template <typename T, typename TH>
__global__ void __launch_bounds__(256)
k_resid(const T *__restrict__ X, const TH *__restrict__ HX, long ld, long nd,
        const double *__restrict__ ritz, double *__restrict__ resid)
{
    __shared__ double red[8];
    const int c = blockIdx.x;
    const double lam = ritz[c];
    const T *x = X + (long)c * ld;
    const TH *hx = HX + (long)c * ld;
    double s = 0.0;
    for (long p = threadIdx.x; p < nd; p += 256) {
        const double r = (double)hx[p] - lam * (double)x[p];
        s += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        resid[c] = sqrt(t);
    }
}

cudaError_t resid_f64(const double *X, const double *HX, long ld, long nd, int ncols,
                      const double *ritz, double *resid, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    k_resid<double, double><<<ncols, 256, 0, st>>>(X, HX, ld, nd, ritz, resid);
    note_launch();
    return cudaGetLastError();
}
cudaError_t resid_f32(const float *X, const float *HX, long ld, long nd, int ncols,
                      const double *ritz, double *resid, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    k_resid<float, float><<<ncols, 256, 0, st>>>(X, HX, ld, nd, ritz, resid);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_check_finite(const double *a, long n, int *flag)
{
    int bad = 0;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x)
        if (!isfinite(a[q])) bad = 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t check_finite(const double *a, long n, int *flag, cudaStream_t st)
{
    int b = (int)((n + 255) / 256);
    if (b > 152 * 4) b = 152 * 4;
    if (b < 1) b = 1;
    k_check_finite<<<b, 256, 0, st>>>(a, n, flag);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
