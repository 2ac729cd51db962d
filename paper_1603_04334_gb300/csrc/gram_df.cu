// gram_df.cu -- FP64 subspace contractions in FP32-pair arithmetic (Sec. 3.4 projection
// M_s = Y^T Y, H_s = Y^T (H Y), and the rotation of Eq. OrbitalTransformation).
//
// GB300's FP64 pipe issues at 1/64 of the FP32 rate, so a native FP64 Gram of a
// 884736 x 128 block takes ~23 ms. Here every FP64 input is split into an FP32 pair
// (hi, lo) (see split_double in stencil_df.cu) and each product a*b is accumulated as
//   p = ah*bh exactly via TwoProduct (FMA), p added to the running sum with TwoSum, and
//   the product error, the TwoSum error and the cross terms ah*bl + al*bh collected in a
//   second FP32 accumulator
// (compensated dot product, Ogita-Rump-Oishi 2005). One multiply-add costs 12 FP32
// instructions. The FP32 error accumulator would lose about n u^2 sum|a_i b_i| over n
// products (u = 2^-24), so the pair is added into an FP64 accumulator every 64 rows and
// restarted; the result is then as accurate as an FP64 dot product. Row slices are summed
// in FP64 in a fixed order. For FP32 inputs lo = 0 and the products are exact.
//
// Symmetric mode (M_s and H_s, both symmetric in exact arithmetic): only tiles with
// i0 <= j0 are computed and the reduction mirrors them.
#include "df.cuh"
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int GT = 64;
constexpr int GK = 16;
constexpr int kFlush = 64;  // rows per FP32-pair partial before it is added in FP64
}  // namespace

template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_gram_df(const TA *__restrict__ A, long lda, const TB *__restrict__ B, long ldb, long nd, int ns,
          long rows_per, int sym, double *__restrict__ part)
{
    if (sym && blockIdx.x > blockIdx.y) return;
    // chunk c is read from buffer c & 1 while chunk c+1 is split into the other one; the
    // global loads of chunk c+1 are issued before the compute of chunk c
    __shared__ float2 As[2][GK][GT + 1];
    __shared__ float2 Bs[2][GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    const long r0 = (long)blockIdx.z * rows_per;
    const long r1 = min(nd, r0 + rows_per);
    float sh[4][4], sl[4][4];
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            sh[a][b] = sl[a][b] = 0.0f;
            acc[a][b] = 0.0;
        }
    const int lr = threadIdx.x & 15, lc = threadIdx.x >> 4;
    const float2 z = make_float2(0.0f, 0.0f);
    TA ra[4];
    TB rb[4];
    auto load = [&](long r) {
        const long row = r + lr;
        const bool okr = row < r1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = lc + 16 * u;
            ra[u] = (okr && i0 + c < ns) ? A[row + (long)(i0 + c) * lda] : (TA)0;
            rb[u] = (okr && j0 + c < ns) ? B[row + (long)(j0 + c) * ldb] : (TB)0;
        }
    };
    auto stage = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[buf][lr][lc + 16 * u] = split_double(ra[u]);
            Bs[buf][lr][lc + 16 * u] = split_double(rb[u]);
        }
    };
    if (r0 < r1) {
        load(r0);
        stage(0);
    }
    __syncthreads();
    int chunk = 0, buf = 0;
    for (long r = r0; r < r1; r += GK) {
        const bool more = r + GK < r1;
        if (more) load(r + GK);
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[buf][kk][ty + 16 * u];
                b[u] = Bs[buf][kk][tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) mac(a[x], b[y], sh[x][y], sl[x][y]);
        }
        // every kFlush rows the FP32 pair is added into FP64 and restarted, so the FP32
        // error accumulator never sums more than kFlush products
        if (++chunk == kFlush / GK) {
            chunk = 0;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    acc[x][y] += pair_to_double(sh[x][y], sl[x][y]);
                    sh[x][y] = sl[x][y] = 0.0f;
                }
        }
        if (more) stage(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    double *P = part + (long)blockIdx.z * ns * ns;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = i0 + ty + 16 * x, gj = j0 + tx + 16 * y;
            if (gi < ns && gj < ns)
                P[gi + (long)gj * ns] = acc[x][y] + pair_to_double(sh[x][y], sl[x][y]);
        }
}

// G(i, j) = sum over slices; in symmetric mode entries of tiles below the diagonal are
// read from the mirrored (j, i) position.
__global__ void k_gram_df_reduce(const double *__restrict__ part, int nsplit, int ns, int sym,
                                 double *G)
{
    const long nn = (long)ns * ns;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nn;
         q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q % ns), j = (int)(q / ns);
        const long src = (sym && (i / GT) > (j / GT)) ? (long)j + (long)i * ns : q;
        double s = 0.0;
        for (int t = 0; t < nsplit; ++t) s += part[(long)t * nn + src];
        G[q] = s;
    }
}

template <typename TA, typename TB>
cudaError_t gram_df_launch(const TA *A, long lda, const TB *B, long ldb, long nd, int ns,
                           double *G, double *part, int nsplit, bool sym, cudaStream_t st)
{
    if (ns <= 0) return cudaSuccess;
    if (nsplit < 1) return cudaErrorInvalidValue;
    long rows_per = (nd + nsplit - 1) / nsplit;
    rows_per = (rows_per + GK - 1) / GK * GK;
    dim3 grid((ns + GT - 1) / GT, (ns + GT - 1) / GT, nsplit);
    k_gram_df<TA, TB><<<grid, 256, 0, st>>>(A, lda, B, ldb, nd, ns, rows_per, sym ? 1 : 0, part);
    note_launch();
    const long nn = (long)ns * ns;
    int rb = (int)((nn + 255) / 256);
    if (rb > 152 * 16) rb = 152 * 16;
    k_gram_df_reduce<<<rb, 256, 0, st>>>(part, nsplit, ns, sym ? 1 : 0, G);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t gram_df_launch<double, double>(const double *, long, const double *, long,
                                                    long, int, double *, double *, int, bool,
                                                    cudaStream_t);
template cudaError_t gram_df_launch<float, float>(const float *, long, const float *, long, long,
                                                  int, double *, double *, int, bool,
                                                  cudaStream_t);
template cudaError_t gram_df_launch<float, double>(const float *, long, const double *, long,
                                                   long, int, double *, double *, int, bool,
                                                   cudaStream_t);

// ---- rotation out = A Q in FP32-pair arithmetic (FP64 blocks) ------------------------
__global__ void __launch_bounds__(256)
k_rotate_df(const double *__restrict__ A, long lda, long nd, int ns, const double *__restrict__ Q,
            double *__restrict__ out, long ldo)
{
    __shared__ float2 As[GK][GT + 1];
    __shared__ float2 Qs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int j0 = blockIdx.x * GT;  // column tiles of a row tile run side by side (L2 reuse)
    for (long rt = blockIdx.y; rt * GT < nd; rt += gridDim.y) {
    const long r0 = rt * GT;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.0f;
    const float2 z = make_float2(0.0f, 0.0f);
    for (int k0 = 0; k0 < ns; k0 += GK) {
        {
            const int rr = threadIdx.x & 63, kc = threadIdx.x >> 6;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kc + 4 * u;
                const long row = r0 + rr;
                As[k][rr] = (row < nd && k0 + k < ns) ? split_double(A[row + (long)(k0 + k) * lda]) : z;
            }
        }
        {
            const int kk = threadIdx.x & 15, cc = threadIdx.x >> 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = cc + 16 * u;
                Qs[kk][c] = (k0 + kk < ns && j0 + c < ns) ? split_double(Q[(k0 + kk) + (long)(j0 + c) * ns])
                                                          : z;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            float2 a[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                q[u] = Qs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) mac(a[x], q[y], sh[x][y], sl[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const long row = r0 + ty + 16 * x;
            const int c = j0 + tx + 16 * y;
            if (row < nd && c < ns) out[row + (long)c * ldo] = (double)sh[x][y] + (double)sl[x][y];
        }
    }
}

cudaError_t rotate_f64_df(const double *A, long lda, long nd, int ns, const double *Q, double *out,
                          long ldo, cudaStream_t st)
{
    if (ns <= 0 || nd <= 0) return cudaSuccess;
    const long gy = (nd + GT - 1) / GT;
    dim3 grid((ns + GT - 1) / GT, (unsigned)(gy < 65535 ? gy : 65535));
    k_rotate_df<<<grid, 256, 0, st>>>(A, lda, nd, ns, Q, out, ldo);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
