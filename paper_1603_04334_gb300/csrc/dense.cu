// dense.cu -- the Ns x Ns steps of CheFSI on the device (Sec. 3.4; the paper solves
// the generalized eigenproblem H_s y = lambda M_s y with LAPACK, Sec. 4, serially on
// the host, and names it the next bottleneck in Sec. 5).
//
// Reduction (the one LAPACK's dsygv performs): M_s = L L^T (Cholesky), A = L^-1 H_s L^-T,
// A = Q diag(lambda) Q^T, and the coefficient matrix of the rotation Y = L^-T Q.
// The symmetric eigensolve is the cyclic Jacobi method with the round-robin (chess
// tournament) parallel ordering of Brent & Luk (1985): in each round the Ns/2 disjoint
// (p, q) pairs are rotated at once; rotation angles follow Golub & Van Loan's symmetric
// Schur decomposition (Algorithm 8.4.1, "sym.schur2"); a rotation is skipped when
// |a_pq| <= 4 eps ||A||_F (an absolute threshold, so rounding noise near zero diagonal
// entries cannot keep the sweeps going) and the sweeps stop when a sweep skips all of
// them. Off-diagonal entries left below that threshold move the eigenvalues only at
// second order (|a_pq|^2 / gap).
// Eigenvalues are sorted ascending and each eigenvector column is signed so that its
// largest-magnitude entry is positive (lowest index on ties).
//
// Matrices are column-major in global memory (L2-resident for the sizes used). The k x k
// Lanczos eigensolve and the final sort run in one CTA of 1024 threads; the Ns x Ns
// reduction runs on many SMs (below). All loops and waits are bounded.
#include "grid.cuh"
#include "internal.cuh"

#include <atomic>

namespace sparc {

namespace {
constexpr int NT = 1024;
constexpr int kMaxSweeps = 60;
constexpr double kEps = 2.220446049250313e-16;

template <typename T>
struct PairsT {
    int p[kMaxDense / 2];
    int q[kMaxDense / 2];
    T c[kMaxDense / 2];
    T s[kMaxDense / 2];
};
using Pairs = PairsT<double>;

__device__ void pair_of(int r, int k, int m, int &p, int &q)
{
    // circle method: player m-1 is fixed; round r pairs (r, m-1) and
    // ((r + k) mod (m-1), (r - k) mod (m-1)) for k = 1..m/2-1.
    if (k == 0) {
        p = r;
        q = m - 1;
    } else {
        p = (r + k) % (m - 1);
        q = (r - k + (m - 1)) % (m - 1);
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// Sum over the CTA (fixed order, same result in every thread).
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Cyclic Jacobi on A (n x n, column-major, symmetric) in the arithmetic of T; V
// accumulates the rotations. Returns (to all threads) the number of sweeps used, or -1 if
// it did not converge within max_sweeps.
template <typename T>
__device__ int jacobi(T *A, T *V, int n, PairsT<T> &P, int *sh_flag, double eps,
                      int max_sweeps = kMaxSweeps)
{
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    double f = 0.0;
    for (long t = tid; t < (long)n * n; t += NT) {
        V[t] = ((t % n) == (t / n)) ? (T)1 : (T)0;
        f += (double)A[t] * (double)A[t];
    }
    const T thr = (T)(4.0 * eps * sqrt(block_sum(f, red)));
    __syncthreads();
    if (n == 1) return 0;
    const int m = (n % 2 == 0) ? n : n + 1;
    const int half = m / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) *sh_flag = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < half; k += NT) {
                int p, q;
                pair_of(r, k, m, p, q);
                T c = (T)1, s = (T)0;
                if (q < n) {
                    const T apq = A[p + (long)q * n];
                    const T app = A[p + (long)p * n], aqq = A[q + (long)q * n];
                    if (fabs(apq) > thr) {
                        const T tau = (aqq - app) / ((T)2 * apq);
                        const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
                        c = (T)1 / sqrt((T)1 + t * t);
                        s = t * c;
                        *sh_flag = 1;
                    }
                }
                P.p[k] = p;
                P.q[k] = q < n ? q : p;
                P.c[k] = c;
                P.s[k] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (long t = tid; t < (long)half * n; t += NT) {
                const int k = (int)(t / n), col = (int)(t % n);
                const T s = P.s[k];
                if (s == (T)0) continue;
                const T c = P.c[k];
                const int p = P.p[k], q = P.q[k];
                const T ap = A[p + (long)col * n], aq = A[q + (long)col * n];
                A[p + (long)col * n] = c * ap - s * aq;
                A[q + (long)col * n] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long t = tid; t < (long)half * n; t += NT) {
                const int k = (int)(t / n), row = (int)(t % n);
                const T s = P.s[k];
                if (s == (T)0) continue;
                const T c = P.c[k];
                const int p = P.p[k], q = P.q[k];
                const T ap = A[row + (long)p * n], aq = A[row + (long)q * n];
                A[row + (long)p * n] = c * ap - s * aq;
                A[row + (long)q * n] = s * ap + c * aq;
                const T vp = V[row + (long)p * n], vq = V[row + (long)q * n];
                V[row + (long)p * n] = c * vp - s * vq;
                V[row + (long)q * n] = s * vp + c * vq;
            }
            __syncthreads();
        }
        const int any = *sh_flag;
        __syncthreads();
        if (!any) return sweep + 1;
    }
    return -1;
}

// ev[rank(i)] = dg[i * ds] sorted ascending (ds = n + 1 reads the diagonal of an n x n
// matrix); Q[:, rank(i)] = V[:, i], signed so its largest |.| entry is positive.
__device__ void sort_and_sign(const double *dg, long ds, const double *V, int n, double *ev,
                              double *Q, int *rank)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += NT) {
        const double di = dg[i * ds];
        int r = 0;
        for (int j = 0; j < n; ++j) {
            const double dj = dg[j * ds];
            if (dj < di || (dj == di && j < i)) ++r;
        }
        rank[i] = r;
        ev[r] = di;
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
        const int r = rank[i];
        int arg = 0;
        double best = -1.0;
        for (int row = 0; row < n; ++row) {
            const double a = fabs(V[row + (long)i * n]);
            if (a > best) {
                best = a;
                arg = row;
            }
        }
        const double sg = V[arg + (long)i * n] < 0.0 ? -1.0 : 1.0;
        for (int row = 0; row < n; ++row) Q[row + (long)r * n] = sg * V[row + (long)i * n];
    }
    __syncthreads();
}
}  // namespace

long dense_work_elems(int ns) { return 11L * ns * ns + 8L * ns + 64; }

// ---- multi-SM reduction of the generalized problem ----------------------------------
// Cholesky M_s = L L^T on a cooperative grid (right-looking, one bounded grid barrier per
// column), the triangular inverse U = L^-T (one warp per column, no barrier), and the
// products A = U^T (H_s U) and Cf = U Q as FP32-pair GEMMs (gram_df.cu); the eigensolve
// in between is the multi-SM Jacobi of jacobi.cu. Same reduction and pivot rule as the
// dsygv-style single-CTA path it replaces, with the dense products spread over all SMs.
namespace {
constexpr int CT = 256;       // threads per CTA of the cooperative Cholesky
constexpr int kInvWarps = 4;  // columns per CTA of the triangular inverse
}  // namespace

// Symmetrise M_s and H_s and check them for non-finite entries (status 2); Cholesky with
// the pivot rule pivot_j > 4 n eps M_jj (status 1 otherwise); writes L row-major into Lr
// (Lr[k + r n] = L_rk, zero above the diagonal) and 1 / L_jj into dinv. Every CTA reads
// the same pivot after the barrier, so all take the same decision. M is overwritten by the
// Schur complements; odiag holds the original diagonal. A barrier that times out sets
// status 4.
__global__ void __launch_bounds__(CT)
k_chol_grid(double *M, double *Hs, int n, double *Lr, double *dinv, double *odiag,
            GridBarrier *bar, int *status)
{
    const unsigned nb = gridDim.x;
    const long gtid = (long)blockIdx.x * CT + threadIdx.x, gs = (long)nb * CT;
    const long nn = (long)n * n;
    auto sync = [&]() -> bool {
        if (grid_barrier(bar, nb)) return true;
        if (threadIdx.x == 0) atomicExch(status, 4);
        return false;
    };
    for (long t = gtid; t < nn; t += gs) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (i < j) {
            const long tt = j + (long)i * n;
            const double m = 0.5 * (M[t] + M[tt]), h = 0.5 * (Hs[t] + Hs[tt]);
            M[t] = m;
            M[tt] = m;
            Hs[t] = h;
            Hs[tt] = h;
            if (!isfinite(m) || !isfinite(h)) atomicExch(status, 2);
        } else if (i == j) {
            if (!isfinite(M[t]) || !isfinite(Hs[t])) atomicExch(status, 2);
            odiag[i] = M[t];
        }
    }
    if (!sync()) return;
    if (*((volatile int *)status) != 0) return;
    for (int j = 0; j < n; ++j) {
        const double d = __ldcg(M + j + (long)j * n);
        if (!(d > 4.0 * n * kEps * __ldcg(odiag + j)) || !isfinite(d)) {
            if (gtid == 0) atomicExch(status, 1);
            return;
        }
        const double inv = 1.0 / d;
        const int m = n - 1 - j;
        for (long t = gtid; t < (long)m * m; t += gs) {
            const int rr = j + 1 + (int)(t % m), cc = j + 1 + (int)(t / m);
            if (rr >= cc) {
                const double a = __ldcg(M + rr + (long)j * n), b = __ldcg(M + cc + (long)j * n);
                M[rr + (long)cc * n] = __ldcg(M + rr + (long)cc * n) - a * b * inv;
            }
        }
        if (!sync()) return;
    }
    // L_jj = sqrt(pivot_j), L_rj = M_rj / L_jj
    for (long t = gtid; t < n; t += gs) {
        const double l = sqrt(__ldcg(M + t + t * n));
        odiag[t] = l;
        dinv[t] = 1.0 / l;
    }
    if (!sync()) return;
    for (long t = gtid; t < nn; t += gs) {
        const int r = (int)(t % n), k = (int)(t / n);  // column-major walk of M
        double v = 0.0;
        if (k < r)
            v = __ldcg(M + t) * __ldcg(dinv + k);
        else if (k == r)
            v = __ldcg(odiag + r);
        Lr[k + (long)r * n] = v;
    }
}

// U = L^-T: warp c solves L x = e_c by forward substitution (rows c .. n-1; each row's dot
// product is split over the lanes in a fixed order and lane 0's sum is used), then writes
// row c of U (U_cr = x_r, zero for r < c).
__global__ void __launch_bounds__(32 * kInvWarps)
k_tri_inv(const double *__restrict__ Lr, const double *__restrict__ dinv, int n, double *U,
          const int *status)
{
    __shared__ double xs[kInvWarps][kMaxDense];
    if (*((volatile const int *)status) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kInvWarps + warp;
    if (c >= n) return;
    double *x = xs[warp];
    for (int r = c; r < n; ++r) {
        const double *row = Lr + (long)r * n;
        double sum = 0.0;
        for (int k = c + lane; k < r; k += 32) sum += row[k] * x[k];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        sum = __shfl_sync(0xffffffffu, sum, 0);
        if (lane == 0) x[r] = ((r == c ? 1.0 : 0.0) - sum) * dinv[r];
        __syncwarp();
    }
    for (int r = lane; r < n; r += 32) U[c + (long)r * n] = r >= c ? x[r] : 0.0;
}

// After the multi-SM Jacobi: sort the eigenvalues ascending and sign the eigenvectors
// (largest |entry| positive, lowest index on ties) into Q.
__global__ void __launch_bounds__(NT)
k_dense_sort(int n, const double *diag, const double *V, double *ritz, double *Q, int *status,
             const GridBarrier *bar)
{
    __shared__ int rank[kMaxDense];
    if (*status != 0) return;
    if (bar->err) {
        if (threadIdx.x == 0) *status = 4;
        return;
    }
    sort_and_sign(diag, 1, V, n, ritz, Q, rank);
}

// ---- mixed-precision eigensolve of A = U^T H_s U (Ns > kMixedFrom) ----------------------
// Block Jacobi in FP32 first (jacobi.cu; 64x the FP64 rate on GB300), its eigenvectors P made
// orthogonal to FP64 accuracy by two Newton-Schulz steps P <- P (3 I - P^T P) / 2, then the
// FP64 Jacobi on A' = P^T A P, which is already diagonal to the FP32 level and converges in
// a few sweeps (quadratically); the eigenvectors of A are P V'. The result is the FP64
// eigendecomposition; the FP32 phase only shortens the FP64 phase.
constexpr int kMixedFrom = 256;     // Ns above this: FP32 phase first
constexpr int kMaxSweeps32 = 20;

__global__ void k_f64_to_f32(const double *a, float *b, long n)
{
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}
__global__ void k_f32_to_f64(const float *a, double *b, long n)
{
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        b[t] = (double)a[t];
}
// A grid barrier of the FP32 phase that gave up makes the whole eigensolve report a
// timeout (its eigenvectors would be partial); the FP64 phase resets the barrier.
__global__ void k_keep_barrier_error(const GridBarrier *bar, int *status)
{
    if (threadIdx.x == 0 && bar->err && *status == 0) *status = 4;
}

// C <- 1.5 I - 0.5 C (the Newton-Schulz coefficient matrix from C = P^T P)
__global__ void k_newton_schulz_coef(double *C, int n)
{
    const long nn = (long)n * n;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long)gridDim.x * blockDim.x)
        C[t] = ((t % n) == (t / n) ? 1.5 : 0.0) - 0.5 * C[t];
}

static std::atomic<int> g_chol_blocks{0};  // co-resident CTAs of k_chol_grid (queried once)

cudaError_t dense_rr(double *M, double *Hs, int ns, double *ritz, double *Cf, double *work,
                     int *status, cudaStream_t st)
{
    if (ns <= 0 || ns > kMaxDense) return cudaErrorInvalidValue;
    const long nn = (long)ns * ns;
    double *R0 = work;            // L row-major, then H_s U, then Jacobi's second copy, then Q
    double *A = work + nn;        // U^T H_s U, then A' = P^T A P (Jacobi's working copy)
    double *V = work + 2 * nn;    // FP64 Jacobi eigenvectors of A'
    double *U = work + 3 * nn;    // L^-T
    double *part = work + 4 * nn; // Gram partials (one row slice for ns <= 2048 rows)
    double *P = work + 5 * nn;    // FP32-phase eigenvectors, then orthogonalised
    double *G = work + 6 * nn;    // P^T P / Newton-Schulz coefficients / A P / P V'
    double *P2 = work + 7 * nn;   // Newton-Schulz ping-pong
    float *A32 = (float *)(work + 8 * nn), *V32 = A32 + nn;
    float *A32b = (float *)(work + 9 * nn);
    double *diag = work + 10 * nn, *dinv = diag + ns, *odiag = dinv + ns;
    GridBarrier *bar = (GridBarrier *)(status + 8);
    int *status32 = status + 13;  // FP32 phase: running out of sweeps only shortens its help
    cudaError_t e;
    if (g_chol_blocks.load(std::memory_order_acquire) == 0) {
        int dev = 0, sms = 0, per = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_grid, CT, 0)) !=
            cudaSuccess)
            return e;
        g_chol_blocks.store(sms * (per > 0 ? per : 1), std::memory_order_release);
    }
    long want = (nn / 2 + CT - 1) / CT;
    if (want < 1) want = 1;
    const int cb = g_chol_blocks.load(std::memory_order_acquire);
    int G0 = (int)(want < cb ? want : cb);
    if (G0 > 152) G0 = 152;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
    {
        void *args[] = {&M, &Hs, &ns, &R0, &dinv, &odiag, &bar, &status};
        e = cudaLaunchCooperativeKernel((const void *)k_chol_grid, dim3(G0), dim3(CT), args, 0, st);
        note_launch();
        if (e != cudaSuccess) return e;
    }
    k_tri_inv<<<(ns + kInvWarps - 1) / kInvWarps, 32 * kInvWarps, 0, st>>>(R0, dinv, ns, U,
                                                                            status);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rotate_f64(Hs, ns, ns, ns, U, R0, ns, st)) != cudaSuccess) return e;  // H_s U
    if ((e = gram_f64(U, ns, R0, ns, ns, ns, A, part, st, true)) != cudaSuccess) return e;
    if (ns <= kMixedFrom) {
        // small Ns: the FP64 Jacobi alone is cheaper than the FP32 phase and the extra
        // products (its rounds are bound by the grid barrier, not by arithmetic)
        if ((e = jacobi_grid(A, R0, V, diag, ns, bar, status, status + 12, st)) != cudaSuccess)
            return e;
        k_dense_sort<<<1, NT, 0, st>>>(ns, diag, V, ritz, R0, status, bar);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return rotate_f64(U, ns, ns, ns, R0, Cf, ns, st);  // Cf = U Q
    }
    // FP32 phase -> P
    const int cg = (int)((nn + 255) / 256 < 152 * 4 ? (nn + 255) / 256 : 152 * 4);
    {
        k_f64_to_f32<<<cg, 256, 0, st>>>(A, A32, nn);
        note_launch();
        if ((e = cudaMemsetAsync(status32, 0, sizeof(int), st)) != cudaSuccess) return e;
        // the block form (its scratch in the second FP32 buffer, which it does not need)
        if ((e = block_jacobi_f32(A32, V32, ns, A32b, status + 14 + 1, kMaxSweeps32, st)) !=
            cudaSuccess)
            return e;
        k_f32_to_f64<<<cg, 256, 0, st>>>(V32, P, nn);
        note_launch();
        k_keep_barrier_error<<<1, 32, 0, st>>>(bar, status);
        note_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // two Newton-Schulz steps: P <- P (1.5 I - 0.5 P^T P)
    double *Pc = P, *Pn = P2;
    for (int it = 0; it < 2; ++it) {
        if ((e = gram_f64(Pc, ns, Pc, ns, ns, ns, G, part, st, true)) != cudaSuccess) return e;
        k_newton_schulz_coef<<<cg, 256, 0, st>>>(G, ns);
        note_launch();
        if ((e = rotate_f64(Pc, ns, ns, ns, G, Pn, ns, st)) != cudaSuccess) return e;
        double *t = Pc;
        Pc = Pn;
        Pn = t;
    }
    // A' = P^T (A P), then the FP64 Jacobi on A'
    if ((e = rotate_f64(A, ns, ns, ns, Pc, G, ns, st)) != cudaSuccess) return e;
    if ((e = gram_f64(Pc, ns, G, ns, ns, ns, A, part, st, true)) != cudaSuccess) return e;
    if ((e = jacobi_grid(A, R0, V, diag, ns, bar, status, status + 12, st)) != cudaSuccess)
        return e;
    if ((e = rotate_f64(Pc, ns, ns, ns, V, G, ns, st)) != cudaSuccess) return e;  // P V'
    k_dense_sort<<<1, NT, 0, st>>>(ns, diag, G, ritz, R0, status, bar);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return rotate_f64(U, ns, ns, ns, R0, Cf, ns, st);  // Cf = U Q
}

__global__ void __launch_bounds__(NT)
k_dense_syev(double *A, int nmax, const int *n_dev, double *ev, double *Q, double *work,
             int *status)
{
    const int n = n_dev ? *n_dev : nmax;
    if (n < 1 || n > nmax) {
        if (threadIdx.x == 0) *status = 2;
        return;
    }
    __shared__ Pairs P;
    __shared__ int flag;
    __shared__ int rank[kMaxDense];
    double *V = work;
    const int sweeps = jacobi<double>(A, V, n, P, &flag, kEps);
    if (sweeps < 0) {
        if (threadIdx.x == 0) *status = 3;
        return;
    }
    sort_and_sign(A, (long)n + 1, V, n, ev, Q, rank);
    if (threadIdx.x == 0) *status = 0;
}

cudaError_t dense_syev(double *A, int ns, const int *ns_dev, double *ev, double *Q,
                       double *work, int *status, cudaStream_t st)
{
    if (ns <= 0 || ns > kMaxDense) return cudaErrorInvalidValue;
    k_dense_syev<<<1, NT, 0, st>>>(A, ns, ns_dev, ev, Q, work, status);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
