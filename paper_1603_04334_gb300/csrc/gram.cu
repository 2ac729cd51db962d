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

cudaError_t rotate_f64(const double *A, long lda, long nd, int ns, const double *Q, double *out,
                       long ldo, cudaStream_t st)
{
    return rotate_f64_df(A, lda, nd, ns, Q, out, ldo, st);
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
