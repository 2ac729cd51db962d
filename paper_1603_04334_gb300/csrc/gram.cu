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

template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_gram(const TA *__restrict__ A, long lda, const TB *__restrict__ B, long ldb, long nd, int ns,
       long rows_per, double *__restrict__ part)
{
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    const long r0 = (long)blockIdx.z * rows_per;
    const long r1 = min(nd, r0 + rows_per);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    // loader mapping: thread t loads row (t % 16) of columns (t / 16) + 16*u, u = 0..3
    const int lr = threadIdx.x & 15, lc = threadIdx.x >> 4;
    for (long r = r0; r < r1; r += GK) {
        const long row = r + lr;
        const bool okr = row < r1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = lc + 16 * u;
            As[lr][c] = (okr && i0 + c < ns) ? (double)A[row + (long)(i0 + c) * lda] : 0.0;
            Bs[lr][c] = (okr && j0 + c < ns) ? (double)B[row + (long)(j0 + c) * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                b[u] = Bs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
    double *P = part + (long)blockIdx.z * ns * ns;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = i0 + ty + 16 * x, gj = j0 + tx + 16 * y;
            if (gi < ns && gj < ns) P[gi + (long)gj * ns] = acc[x][y];
        }
}

__global__ void k_gram_reduce(const double *__restrict__ part, int nsplit, long nn, double *G)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nn;
         q += (long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < nsplit; ++t) s += part[(long)t * nn + q];
        G[q] = s;
    }
}

template <typename TA, typename TB>
static cudaError_t gram(const TA *A, long lda, const TB *B, long ldb, long nd, int ns, double *G,
                        double *part, cudaStream_t st)
{
    if (ns <= 0) return cudaSuccess;
    const int nsplit = gram_splits(ns, nd);
    long rows_per = (nd + nsplit - 1) / nsplit;
    rows_per = (rows_per + GK - 1) / GK * GK;
    dim3 grid((ns + GT - 1) / GT, (ns + GT - 1) / GT, nsplit);
    k_gram<TA, TB><<<grid, 256, 0, st>>>(A, lda, B, ldb, nd, ns, rows_per, part);
    note_launch();
    const long nn = (long)ns * ns;
    int rb = (int)((nn + 255) / 256);
    if (rb > 152 * 16) rb = 152 * 16;
    k_gram_reduce<<<rb, 256, 0, st>>>(part, nsplit, nn, G);
    note_launch();
    return cudaGetLastError();
}

cudaError_t gram_f64(const double *A, long lda, const double *B, long ldb, long nd, int ns,
                     double *G, double *part, cudaStream_t st)
{
    return gram<double, double>(A, lda, B, ldb, nd, ns, G, part, st);
}
cudaError_t gram_f32_f32(const float *A, long lda, const float *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st)
{
    return gram<float, float>(A, lda, B, ldb, nd, ns, G, part, st);
}
cudaError_t gram_f32_f64(const float *A, long lda, const double *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st)
{
    return gram<float, double>(A, lda, B, ldb, nd, ns, G, part, st);
}

// ---- rotation: out = A Q, tile 64 rows x 64 columns, Q staged 16 rows at a time ------
template <typename T>
__global__ void __launch_bounds__(256)
k_rotate(const T *__restrict__ A, long lda, long nd, int ns, const double *__restrict__ Q,
         T *__restrict__ out, long ldo)
{
    __shared__ double As[GK][GT + 1];   // [k][row]
    __shared__ double Qs[GK][GT + 1];   // [k][col]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long r0 = (long)blockIdx.x * GT;
    const int j0 = blockIdx.y * GT;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < ns; k0 += GK) {
        // A tile: 16 columns (k) x 64 rows; thread loads rows (t % 64), columns t/64 + 4u
        {
            const int rr = threadIdx.x & 63, kc = threadIdx.x >> 6;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kc + 4 * u;
                const long row = r0 + rr;
                As[k][rr] = (row < nd && k0 + k < ns) ? (double)A[row + (long)(k0 + k) * lda] : 0.0;
            }
        }
        // Q tile: 16 rows (k) x 64 columns; thread loads k = t % 16, columns t/16 + 16u
        {
            const int kk = threadIdx.x & 15, cc = threadIdx.x >> 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = cc + 16 * u;
                Qs[kk][c] = (k0 + kk < ns && j0 + c < ns) ? Q[(k0 + kk) + (long)(j0 + c) * ns] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                q[u] = Qs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], q[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const long row = r0 + ty + 16 * x;
            const int c = j0 + tx + 16 * y;
            if (row < nd && c < ns) out[row + (long)c * ldo] = (T)acc[x][y];
        }
}

template <typename T>
static cudaError_t rotate(const T *A, long lda, long nd, int ns, const double *Q, T *out,
                          long ldo, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaSuccess;
    const long gx = (nd + GT - 1) / GT;
    if (gx > 2147483647L) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (ns + GT - 1) / GT);
    k_rotate<T><<<grid, 256, 0, st>>>(A, lda, nd, ns, Q, out, ldo);
    note_launch();
    return cudaGetLastError();
}

cudaError_t rotate_f64(const double *A, long lda, long nd, int ns, const double *Q, double *out,
                       long ldo, cudaStream_t st)
{
    return rotate<double>(A, lda, nd, ns, Q, out, ldo, st);
}
cudaError_t rotate_f32(const float *A, long lda, long nd, int ns, const double *Q, float *out,
                       long ldo, cudaStream_t st)
{
    return rotate<float>(A, lda, nd, ns, Q, out, ldo, st);
}

// ---- residual norms: one CTA per column, fixed-order reduction -----------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_resid(const T *__restrict__ X, const double *__restrict__ HX, long ld, long nd,
        const double *__restrict__ ritz, double *__restrict__ resid)
{
    __shared__ double red[8];
    const int c = blockIdx.x;
    const double lam = ritz[c];
    const T *x = X + (long)c * ld;
    const double *hx = HX + (long)c * ld;
    double s = 0.0;
    for (long p = threadIdx.x; p < nd; p += 256) {
        const double r = hx[p] - lam * (double)x[p];
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
    k_resid<double><<<ncols, 256, 0, st>>>(X, HX, ld, nd, ritz, resid);
    note_launch();
    return cudaGetLastError();
}
cudaError_t resid_f32(const float *X, const double *HX, long ld, long nd, int ncols,
                      const double *ritz, double *resid, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    k_resid<float><<<ncols, 256, 0, st>>>(X, HX, ld, nd, ritz, resid);
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
