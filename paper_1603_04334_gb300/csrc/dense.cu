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
// Every kernel here is one CTA of 1024 threads working on column-major matrices in
// global memory (L1/L2 resident for the sizes used). All loops are bounded.
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int NT = 1024;
constexpr int kMaxSweeps = 60;
constexpr double kEps = 2.220446049250313e-16;

struct Pairs {
    int p[kMaxDense / 2];
    int q[kMaxDense / 2];
    double c[kMaxDense / 2];
    double s[kMaxDense / 2];
};

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

// Cyclic Jacobi on A (n x n, column-major, symmetric); V accumulates the rotations.
// Returns (to all threads) the number of sweeps used, or -1 if it did not converge.
__device__ int jacobi(double *A, double *V, int n, Pairs &P, int *sh_flag)
{
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    double f = 0.0;
    for (long t = tid; t < (long)n * n; t += NT) {
        V[t] = ((t % n) == (t / n)) ? 1.0 : 0.0;
        f += A[t] * A[t];
    }
    const double thr = 4.0 * kEps * sqrt(block_sum(f, red));
    __syncthreads();
    if (n == 1) return 0;
    const int m = (n % 2 == 0) ? n : n + 1;
    const int half = m / 2;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        if (tid == 0) *sh_flag = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < half; k += NT) {
                int p, q;
                pair_of(r, k, m, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[p + (long)q * n];
                    const double app = A[p + (long)p * n], aqq = A[q + (long)q * n];
                    if (fabs(apq) > thr) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
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
                const double s = P.s[k];
                if (s == 0.0) continue;
                const double c = P.c[k];
                const int p = P.p[k], q = P.q[k];
                const double ap = A[p + (long)col * n], aq = A[q + (long)col * n];
                A[p + (long)col * n] = c * ap - s * aq;
                A[q + (long)col * n] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long t = tid; t < (long)half * n; t += NT) {
                const int k = (int)(t / n), row = (int)(t % n);
                const double s = P.s[k];
                if (s == 0.0) continue;
                const double c = P.c[k];
                const int p = P.p[k], q = P.q[k];
                const double ap = A[row + (long)p * n], aq = A[row + (long)q * n];
                A[row + (long)p * n] = c * ap - s * aq;
                A[row + (long)q * n] = s * ap + c * aq;
                const double vp = V[row + (long)p * n], vq = V[row + (long)q * n];
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

long dense_work_elems(int ns) { return 3L * ns * ns + 8L * ns + 64; }

// Symmetrise, Cholesky M = L L^T (L overwrites M), A = L^-1 H_s L^-T into work + n^2.
__global__ void __launch_bounds__(NT)
k_dense_pre(double *M, double *Hs, int n, double *work, int *status)
{
    __shared__ int flag;
    const int tid = threadIdx.x;
    const long nn = (long)n * n;
    double *W = work;            // L^-1 H_s
    double *A = work + nn;       // L^-1 H_s L^-T, then Jacobi working copy
    double *V = work + 2 * nn;   // Jacobi eigenvectors
    if (tid == 0) flag = 0;
    __syncthreads();
    // 1. symmetrise, check finiteness
    for (long t = tid; t < nn; t += NT) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (i < j) {
            const double m = 0.5 * (M[i + (long)j * n] + M[j + (long)i * n]);
            const double h = 0.5 * (Hs[i + (long)j * n] + Hs[j + (long)i * n]);
            M[i + (long)j * n] = m;
            M[j + (long)i * n] = m;
            Hs[i + (long)j * n] = h;
            Hs[j + (long)i * n] = h;
        }
        if (!isfinite(M[t]) || !isfinite(Hs[t])) flag = 2;
    }
    __syncthreads();
    if (flag) {
        if (tid == 0) *status = flag;
        return;
    }
    // 2. Cholesky M = L L^T (lower, in place), right-looking. M_s counts as numerically
    //    positive definite when every pivot exceeds 4 n eps times its original diagonal
    //    entry (pivot / diagonal = squared sine of the angle between a column and the span
    //    of the previous ones). The diagonal is saved in V before it is overwritten.
    for (int j = tid; j < n; j += NT) V[j] = M[j + (long)j * n];
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = M[j + (long)j * n];
            if (!(d > 4.0 * n * kEps * V[j]) || !isfinite(d))
                flag = 1;
            else
                M[j + (long)j * n] = sqrt(d);
        }
        __syncthreads();
        if (flag) {
            if (tid == 0) *status = 1;
            return;
        }
        const double djj = M[j + (long)j * n];
        for (int i = j + 1 + tid; i < n; i += NT) M[i + (long)j * n] /= djj;
        __syncthreads();
        const int mrem = n - j - 1;
        for (long t = tid; t < (long)mrem * mrem; t += NT) {
            const int rr = j + 1 + (int)(t % mrem), cc = j + 1 + (int)(t / mrem);
            if (rr >= cc) M[rr + (long)cc * n] -= M[rr + (long)j * n] * M[cc + (long)j * n];
        }
        __syncthreads();
    }
    // 3. W = L^-1 H_s (forward substitution, one thread per column)
    for (int c = tid; c < n; c += NT) {
        for (int r = 0; r < n; ++r) {
            double s = Hs[r + (long)c * n];
            for (int k = 0; k < r; ++k) s -= M[r + (long)k * n] * W[k + (long)c * n];
            W[r + (long)c * n] = s / M[r + (long)r * n];
        }
    }
    __syncthreads();
    // 4. A = L^-1 W^T  (= L^-1 H_s L^-T), then symmetrise
    for (int c = tid; c < n; c += NT) {
        for (int r = 0; r < n; ++r) {
            double s = W[c + (long)r * n];
            for (int k = 0; k < r; ++k) s -= M[r + (long)k * n] * A[k + (long)c * n];
            A[r + (long)c * n] = s / M[r + (long)r * n];
        }
    }
    __syncthreads();
    for (long t = tid; t < nn; t += NT) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (i < j) {
            const double a = 0.5 * (A[i + (long)j * n] + A[j + (long)i * n]);
            A[i + (long)j * n] = a;
            A[j + (long)i * n] = a;
        }
    }
    if (tid == 0) *status = 0;
}

// After the multi-SM Jacobi (jacobi.cu): sort and sign the eigenpairs (Q into W) and form
// Cf = L^-T Q by backward substitution, one thread per column.
__global__ void __launch_bounds__(NT)
k_dense_post(const double *L, int n, const double *diag, const double *V, double *ritz,
             double *Cf, double *W, int *status, const GridBarrier *bar)
{
    __shared__ int rank[kMaxDense];
    const int tid = threadIdx.x;
    if (*status != 0) return;
    if (bar->err) {
        if (tid == 0) *status = 4;
        return;
    }
    sort_and_sign(diag, 1, V, n, ritz, W, rank);
    const double *M = L;
    for (int c = tid; c < n; c += NT) {
        for (int r = n - 1; r >= 0; --r) {
            double s = W[r + (long)c * n];
            for (int k = r + 1; k < n; ++k) s -= M[k + (long)r * n] * Cf[k + (long)c * n];
            Cf[r + (long)c * n] = s / M[r + (long)r * n];
        }
    }
    if (tid == 0) *status = 0;
}

cudaError_t dense_rr(double *M, double *Hs, int ns, double *ritz, double *Cf, double *work,
                     int *status, cudaStream_t st)
{
    if (ns <= 0 || ns > kMaxDense) return cudaErrorInvalidValue;
    const long nn = (long)ns * ns;
    double *W = work, *A = work + nn, *V = work + 2 * nn, *diag = work + 3 * nn;
    GridBarrier *bar = (GridBarrier *)(status + 8);
    k_dense_pre<<<1, NT, 0, st>>>(M, Hs, ns, work, status);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = jacobi_grid(A, W, V, diag, ns, bar, status, status + 12, st);
    if (e != cudaSuccess) return e;
    k_dense_post<<<1, NT, 0, st>>>(M, ns, diag, V, ritz, Cf, W, status, bar);
    note_launch();
    return cudaGetLastError();
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
    const int sweeps = jacobi(A, V, n, P, &flag);
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
