// jacobi.cu -- the symmetric eigensolve of the Rayleigh-Ritz step (Sec. 3.4, the
// standard problem L^-1 H_s L^-T q = lambda q) spread over many SMs.
//
// Cyclic Jacobi with the round-robin parallel ordering of Brent & Luk (1985): each round
// rotates n/2 disjoint (p, q) pairs. The two-sided update A <- J^T A J factors into
// independent 2 x 2 blocks A[{p1,q1},{p2,q2}] <- J_1^T A[...] J_2, so a round is one pass
// over all blocks with no ordering between them. A is double-buffered (read the current
// copy, write the next), and every CTA recomputes all of the round's rotation angles from
// the current copy, so a round needs a single grid-wide barrier and every CTA reaches the
// same convergence decision without further communication. V <- V J updates columns p, q
// of V in place (each (row, pair) belongs to one thread).
//
// Rotation angles follow Golub & Van Loan's symmetric Schur decomposition (Algorithm
// 8.4.1); a rotation is skipped when |a_pq| <= 4 eps ||A||_F, and the sweeps stop after a
// sweep that skipped all of them (as in dense.cu's single-CTA version). A round that
// skips all of its rotations changes nothing, so it needs neither the update pass nor the
// barrier (every CTA takes that decision from the same data).
//
// The grid barrier is an arrival counter in global memory (grid.cuh); the kernel is launched
// cooperatively (all CTAs co-resident), and every wait is bounded: after kBarrierSpins
// polls the waiting CTA raises an error flag, every CTA leaves at its next barrier and the
// host reports SPARC_ERR_TIMEOUT.
#include "grid.cuh"
#include "internal.cuh"

#include <atomic>

namespace sparc {

namespace {
constexpr int NT = 256;
constexpr int kMaxSweeps = 60;
constexpr double kEps = 2.220446049250313e-16;
// CTAs of the grid Jacobi, at most: its FP64 rounds are bound by the FP64 pipe and gain
// nothing from a second CTA per SM.
constexpr int kJacobiCtas = 152;

__device__ __forceinline__ void pair_of(int r, int k, int m, int &p, int &q)
{
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

// Returns false (to every thread of the CTA) once any CTA has hit the spin limit.
}  // namespace

// T: the arithmetic (the eigensolve runs it in FP64), eps the unit roundoff of T.
template <typename T>
__global__ void __launch_bounds__(NT, 1)
k_jacobi_grid(T *A0, T *A1, T *V, T *diag, int n, GridBarrier *bar, int *status,
              int *sweeps_out, double eps, int max_sweeps)
{
    __shared__ int sp[kMaxDense / 2], sq[kMaxDense / 2];
    __shared__ T sc[kMaxDense / 2], ss[kMaxDense / 2];
    __shared__ double red[NT / 32];
    __shared__ int any_rot, round_rot;
    if (*((volatile int *)status) != 0) return;  // the reduction step failed
    const unsigned nb = gridDim.x;
    const long nn = (long)n * n;
    const long gtid = (long)blockIdx.x * NT + threadIdx.x, gstride = (long)nb * NT;
    for (long t = gtid; t < nn; t += gstride) V[t] = ((t % n) == (t / n)) ? (T)1 : (T)0;
    double f = 0.0;
    for (long t = threadIdx.x; t < nn; t += NT) f += (double)A0[t] * (double)A0[t];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
    __syncthreads();
    double fro = 0.0;
    for (int w = 0; w < NT / 32; ++w) fro += red[w];
    const T thr = (T)(4.0 * eps * sqrt(fro));
    if (!grid_barrier(bar, nb)) return;

    T *cur = A0, *nxt = A1;
    const int m = n + (n & 1), half = m / 2;
    int sweeps = -1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) any_rot = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            if (threadIdx.x == 0) round_rot = 0;
            __syncthreads();
            for (int k = threadIdx.x; k < half; k += NT) {
                int p, q;
                pair_of(r, k, m, p, q);
                T c = (T)1, s = (T)0;
                if (q < n) {
                    const T apq = __ldcg(cur + p + (long)q * n);
                    if (fabs(apq) > thr) {
                        const T app = __ldcg(cur + p + (long)p * n);
                        const T aqq = __ldcg(cur + q + (long)q * n);
                        const T tau = (aqq - app) / ((T)2 * apq);
                        const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
                        c = (T)1 / sqrt((T)1 + t * t);
                        s = t * c;
                        any_rot = 1;
                        round_rot = 1;
                    }
                }
                sp[k] = p;
                sq[k] = q;
                sc[k] = c;
                ss[k] = s;
            }
            __syncthreads();
            // a round without rotations leaves A and V as they are; every CTA computed the
            // same angles from the same copy, so all of them skip it (and its barrier)
            if (!round_rot) continue;
            // 2 x 2 blocks: next = J_1^T cur J_2. A is symmetric, so block (k2, k1) of next is
            // the transpose of block (k1, k2): only k1 <= k2 is computed and written to both
            // places (every entry of next is written; half the FP64 work of computing all
            // blocks, and next stays exactly symmetric)
            for (long b = gtid; b < (long)half * half; b += gstride) {
                const int k1 = (int)(b % half), k2 = (int)(b / half);
                if (k1 > k2) continue;
                const int p1 = sp[k1], q1 = sq[k1], p2 = sp[k2], q2 = sq[k2];
                const bool v1 = q1 < n, v2 = q2 < n;
                const T c1 = sc[k1], s1 = ss[k1], c2 = sc[k2], s2 = ss[k2];
                const T app = __ldcg(cur + p1 + (long)p2 * n);
                const T apq = v2 ? __ldcg(cur + p1 + (long)q2 * n) : (T)0;
                const T aqp = v1 ? __ldcg(cur + q1 + (long)p2 * n) : (T)0;
                const T aqq = (v1 && v2) ? __ldcg(cur + q1 + (long)q2 * n) : (T)0;
                const T bpp = c1 * app - s1 * aqp, bpq = c1 * apq - s1 * aqq;
                const T bqp = s1 * app + c1 * aqp, bqq = s1 * apq + c1 * aqq;
                const T npp = c2 * bpp - s2 * bpq, npq = s2 * bpp + c2 * bpq;
                const T nqp = c2 * bqp - s2 * bqq, nqq = s2 * bqp + c2 * bqq;
                nxt[p1 + (long)p2 * n] = npp;
                if (v2) nxt[p1 + (long)q2 * n] = npq;
                if (v1) nxt[q1 + (long)p2 * n] = nqp;
                if (v1 && v2) nxt[q1 + (long)q2 * n] = nqq;
                if (k1 != k2) {
                    nxt[p2 + (long)p1 * n] = npp;
                    if (v2) nxt[q2 + (long)p1 * n] = npq;
                    if (v1) nxt[p2 + (long)q1 * n] = nqp;
                    if (v1 && v2) nxt[q2 + (long)q1 * n] = nqq;
                }
            }
            // V <- V J, columns p, q of each rotated pair
            for (long t = gtid; t < (long)half * n; t += gstride) {
                const int k = (int)(t / n), row = (int)(t % n);
                const T s = ss[k];
                if (s == (T)0) continue;
                const T c = sc[k];
                const int p = sp[k], q = sq[k];
                const T vp = __ldcg(V + row + (long)p * n), vq = __ldcg(V + row + (long)q * n);
                V[row + (long)p * n] = c * vp - s * vq;
                V[row + (long)q * n] = s * vp + c * vq;
            }
            if (!grid_barrier(bar, nb)) return;
            T *t = cur;
            cur = nxt;
            nxt = t;
        }
        const int any = any_rot;
        __syncthreads();
        if (!any) {
            sweeps = sweep + 1;
            break;
        }
    }
    for (long i = gtid; i < n; i += gstride) diag[i] = __ldcg(cur + i + i * n);
    if (gtid == 0) {
        *sweeps_out = sweeps;
        if (sweeps < 0) *status = 3;
    }
}

template <typename T>
static cudaError_t jacobi_grid_t(T *A0, T *A1, T *V, T *diag, int n, GridBarrier *bar,
                                 int *status, int *sweeps_out, double eps, int max_sweeps,
                                 cudaStream_t st)
{
    static std::atomic<int> coop_blocks{0};  // co-resident CTAs of this instance (queried once)
    if (n <= 0 || n > kMaxDense) return cudaErrorInvalidValue;
    if (coop_blocks.load(std::memory_order_acquire) == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_jacobi_grid<T>, NT, 0);
        if (e != cudaSuccess) return e;
        coop_blocks.store(sms * (per > 0 ? per : 1), std::memory_order_release);
    }
    const long half = (n + 1) / 2;
    // a round's FP64 work (the 2 x 2 blocks and the columns of V) spread over four times
    // the CTAs that one block per thread would take: the FP64 pipes of more SMs, at the
    // cost of a barrier over more CTAs
    long want = 4 * ((half * half + NT - 1) / NT);
    if (want < 1) want = 1;
    const int cb = coop_blocks.load(std::memory_order_acquire);
    int G = (int)(want < cb ? want : cb);
    if (G > kJacobiCtas) G = kJacobiCtas;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&A0, &A1, &V, &diag, &n, &bar, &status, &sweeps_out, &eps, &max_sweeps};
    e = cudaLaunchCooperativeKernel((const void *)k_jacobi_grid<T>, dim3(G), dim3(NT), args, 0,
                                    st);
    note_launch();
    return e;
}

cudaError_t jacobi_grid(double *A0, double *A1, double *V, double *diag, int n, GridBarrier *bar,
                        int *status, int *sweeps_out, cudaStream_t st)
{
    return jacobi_grid_t<double>(A0, A1, V, diag, n, bar, status, sweeps_out, kEps, kMaxSweeps,
                                 st);
}


// Failure-detection self-test: every CTA of a cooperative grid waits at a barrier that
// expects one CTA more than the grid holds, so the wait can only end through its spin
// limit (~65 ms here). status[0] = 4 when every CTA left through the timeout path, 0 if
// the barrier (wrongly) completed.
__global__ void __launch_bounds__(32) k_barrier_selftest(GridBarrier *bar, int *status)
{
    const bool ok = grid_barrier(bar, gridDim.x + 1u, 1ull << 20);
    if (threadIdx.x == 0 && !ok) atomicExch(status, 4);
}

cudaError_t barrier_selftest(GridBarrier *bar, int *status, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&bar, &status};
    e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(2), dim3(32), args, 0,
                                    st);
    note_launch();
    return e;
}


// ---- block Jacobi for the FP32 pre-solve ---------------------------------------------
// The two-sided cyclic Jacobi method by blocks (the block form of the same Brent-Luk
// round-robin ordering): the columns are cut into blocks of kBjB = 32, and in each round
// the blocks are paired round-robin. For a pair (I, J) one CTA diagonalises the symmetric
// subproblem S = A[I u J, I u J] (at most 64 x 64) in shared memory by kBjInner sweeps of
// the scalar cyclic Jacobi (same angle formula and threshold as above) and stores the
// accumulated rotation Q_IJ. A second kernel then applies all the round's rotations at
// once: A[P, P'] <- Q_P^T A[P, P'] Q_P' for every pair of pairs (P <= P', the transpose
// written to [P', P]) and V[R, P] <- V[R, P] Q_P for every 64-row block R, as 64 x 64
// products in shared memory. Each tile is read and written by one CTA, so A and V are
// updated in place. A sweep takes nb - 1 rounds of two launches for nb blocks (31 at
// Ns = 1024, against 1023 barrier-separated rounds of the scalar form, each of which
// streams all of A and V through L2). A sweep whose inner solves made no rotation ends
// the solve: the kernels of later sweeps see the done flag and return at once.
namespace {
constexpr int kBjB = 32;                 // block size
constexpr int kBjM = 2 * kBjB;           // largest subproblem
constexpr int kBjLd = kBjM + 1;          // shared-memory row stride (no bank conflicts)
constexpr int kBjThreads = 256;
constexpr int kBjInner = 1;              // inner sweeps per subproblem and round

struct BjState {
    float thr;   // 4 eps ||A||_F
    int rot;     // a rotation happened in the current sweep
    int done;    // the solve has converged
    int sweeps;  // sweeps used
};

// Round r of the round-robin over nbe (even) blocks: pair k of the round holds blocks
// (bi, bj); blocks >= nb are empty.
__device__ __forceinline__ void bj_pair(int r, int k, int nbe, int &bi, int &bj)
{
    pair_of(r, k, nbe, bi, bj);
}

// global index of local position i of the pair's index set (block bi then block bj)
__device__ __forceinline__ int bj_index(int i, int bi, int ni, int bj)
{
    return i < ni ? bi * kBjB + i : bj * kBjB + (i - ni);
}

__device__ __forceinline__ int bj_size(int blk, int n)
{
    const int lo = blk * kBjB;
    return lo >= n ? 0 : min(kBjB, n - lo);
}
}  // namespace

__global__ void __launch_bounds__(1024) k_bj_init(const float *__restrict__ A, float *V, int n,
                                                  BjState *st, double eps)
{
    __shared__ double red[32];
    double f = 0.0;
    const long nn = (long)n * n;
    for (long t = threadIdx.x; t < nn; t += blockDim.x) {
        f += (double)A[t] * (double)A[t];
        V[t] = ((t % n) == (t / n)) ? 1.0f : 0.0f;
    }
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        st->thr = (float)(4.0 * eps * sqrt(s));
        st->rot = 0;
        st->done = 0;
        st->sweeps = -1;
    }
}

// sweep bookkeeping: phase 0 starts sweep s, phase 1 ends it
__global__ void k_bj_sweep(BjState *st, int s, int phase)
{
    if (st->done) return;
    if (phase == 0) {
        st->rot = 0;
    } else if (!st->rot) {
        st->done = 1;
        st->sweeps = s + 1;
    }
}

// Inner solve of each pair of round r: S = A[P, P] in shared memory, kBjInner cyclic
// sweeps, Q (the accumulated rotation, kBjM x kBjM with an identity outside the subproblem)
// to Qs[pair].
__global__ void __launch_bounds__(kBjThreads)
k_bj_solve(const float *__restrict__ A, int n, int nbe, int r, float *__restrict__ Qs,
           BjState *st)
{
    __shared__ float S[kBjM * kBjLd], Q[kBjM * kBjLd];
    __shared__ int sp[kBjB], sq[kBjB];
    __shared__ float sc[kBjB], ss[kBjB];
    __shared__ int any;
    if (*(volatile int *)&st->done) return;
    int bi, bj;
    bj_pair(r, blockIdx.x, nbe, bi, bj);
    const int ni = bj_size(bi, n), nj = bj_size(bj, n), m = ni + nj;
    const float thr = st->thr;
    for (int t = threadIdx.x; t < kBjM * kBjM; t += kBjThreads) {
        const int i = t % kBjM, j = t / kBjM;
        float v = 0.0f;
        if (i < m && j < m) v = A[bj_index(i, bi, ni, bj) + (long)bj_index(j, bi, ni, bj) * n];
        S[i + j * kBjLd] = v;
        Q[i + j * kBjLd] = i == j ? 1.0f : 0.0f;
    }
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int me = m + (m & 1), half = me / 2;
    for (int sw = 0; sw < kBjInner && m > 1; ++sw) {
        for (int rr = 0; rr < me - 1; ++rr) {
            if (threadIdx.x < half) {
                const int k = threadIdx.x;
                int p, q;
                pair_of(rr, k, me, p, q);
                float c = 1.0f, s = 0.0f;
                if (q < m) {
                    const float apq = S[p + q * kBjLd];
                    if (fabsf(apq) > thr) {
                        const float app = S[p + p * kBjLd], aqq = S[q + q * kBjLd];
                        const float tau = (aqq - app) / (2.0f * apq);
                        const float tt = (tau >= 0.0f ? 1.0f : -1.0f) /
                                         (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        c = 1.0f / sqrtf(1.0f + tt * tt);
                        s = tt * c;
                        any = 1;
                    }
                }
                sp[k] = p;
                sq[k] = q < m ? q : p;
                sc[k] = c;
                ss[k] = s;
            }
            __syncthreads();
            // rows: S <- J^T S
            for (int t = threadIdx.x; t < half * m; t += kBjThreads) {
                const int k = t / m, col = t % m;
                const float s = ss[k];
                if (s == 0.0f) continue;
                const float c = sc[k];
                const int p = sp[k], q = sq[k];
                const float ap = S[p + col * kBjLd], aq = S[q + col * kBjLd];
                S[p + col * kBjLd] = c * ap - s * aq;
                S[q + col * kBjLd] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: S <- S J, Q <- Q J
            for (int t = threadIdx.x; t < half * m; t += kBjThreads) {
                const int k = t / m, row = t % m;
                const float s = ss[k];
                if (s == 0.0f) continue;
                const float c = sc[k];
                const int p = sp[k], q = sq[k];
                const float ap = S[row + p * kBjLd], aq = S[row + q * kBjLd];
                S[row + p * kBjLd] = c * ap - s * aq;
                S[row + q * kBjLd] = s * ap + c * aq;
                const float vp = Q[row + p * kBjLd], vq = Q[row + q * kBjLd];
                Q[row + p * kBjLd] = c * vp - s * vq;
                Q[row + q * kBjLd] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    float *qg = Qs + (long)blockIdx.x * kBjM * kBjM;
    for (int t = threadIdx.x; t < kBjM * kBjM; t += kBjThreads) {
        const int i = t % kBjM, j = t / kBjM;
        qg[t] = Q[i + j * kBjLd];
    }
    if (threadIdx.x == 0 && any) atomicExch(&st->rot, 1);
}

// Application of round r's rotations. CTAs [0, npairs (npairs + 1) / 2): A tiles (P, P'),
// P <= P'; then npairs x ceil(n / 64) V tiles (pair P, rows 64 R ..). Each computes a
// 64 x 64 product (two for A) in shared memory, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(kBjThreads)
k_bj_apply(float *A, float *V, int n, int nbe, int r, const float *__restrict__ Qs,
           const BjState *st)
{
    __shared__ float T[kBjM * kBjLd], Qa[kBjM * kBjLd], Qb[kBjM * kBjLd];
    if (*(volatile const int *)&st->done) return;
    const int npairs = nbe / 2;
    const int nat = npairs * (npairs + 1) / 2;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 each
    int b = blockIdx.x;
    if (b < nat) {
        // tile (pa, pb), pa <= pb, row-major over the upper triangle
        int pa = 0;
        while (b >= npairs - pa) {
            b -= npairs - pa;
            ++pa;
        }
        const int pb = pa + b;
        int ai, aj, bi, bj;
        bj_pair(r, pa, nbe, ai, aj);
        bj_pair(r, pb, nbe, bi, bj);
        const int nai = bj_size(ai, n), ma = nai + bj_size(aj, n);
        const int nbi = bj_size(bi, n), mb = nbi + bj_size(bj, n);
        if (ma == 0 || mb == 0) return;
        const float *qa = Qs + (long)pa * kBjM * kBjM, *qb = Qs + (long)pb * kBjM * kBjM;
        for (int t = threadIdx.x; t < kBjM * kBjM; t += kBjThreads) {
            const int i = t % kBjM, j = t / kBjM;
            T[i + j * kBjLd] = (i < ma && j < mb)
                                   ? A[bj_index(i, ai, nai, aj) + (long)bj_index(j, bi, nbi, bj) * n]
                                   : 0.0f;
            Qa[i + j * kBjLd] = qa[t];
            Qb[i + j * kBjLd] = qb[t];
        }
        __syncthreads();
        // W = T Qb (4 x 4 per thread), kept in registers, then T <- W
        float w[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) w[u][v] = 0.0f;
        for (int k = 0; k < kBjM; ++k) {
            float x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = T[(ty * 4 + u) + k * kBjLd];
#pragma unroll
            for (int v = 0; v < 4; ++v) y[v] = Qb[k + (tx * 4 + v) * kBjLd];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) w[u][v] = fmaf(x[u], y[v], w[u][v]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) T[(ty * 4 + u) + (tx * 4 + v) * kBjLd] = w[u][v];
        __syncthreads();
        // T' = Qa^T W
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) w[u][v] = 0.0f;
        for (int k = 0; k < kBjM; ++k) {
            float x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = Qa[k + (ty * 4 + u) * kBjLd];
#pragma unroll
            for (int v = 0; v < 4; ++v) y[v] = T[k + (tx * 4 + v) * kBjLd];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) w[u][v] = fmaf(x[u], y[v], w[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = ty * 4 + u, j = tx * 4 + v;
                if (i < ma && j < mb) {
                    const int gi = bj_index(i, ai, nai, aj), gj = bj_index(j, bi, nbi, bj);
                    A[gi + (long)gj * n] = w[u][v];
                    if (pa != pb) A[gj + (long)gi * n] = w[u][v];
                }
            }
        return;
    }
    // V tile: V[rows, P] <- V[rows, P] Q_P
    b -= nat;
    const int nrb = (n + kBjM - 1) / kBjM;
    const int p = b / nrb, rb = b % nrb;
    int pi, pj;
    bj_pair(r, p, nbe, pi, pj);
    const int npi = bj_size(pi, n), mp = npi + bj_size(pj, n);
    const int r0 = rb * kBjM, nr = min(kBjM, n - r0);
    if (mp == 0 || nr <= 0) return;
    const float *q = Qs + (long)p * kBjM * kBjM;
    for (int t = threadIdx.x; t < kBjM * kBjM; t += kBjThreads) {
        const int i = t % kBjM, j = t / kBjM;
        T[i + j * kBjLd] = (i < nr && j < mp) ? V[(r0 + i) + (long)bj_index(j, pi, npi, pj) * n] : 0.0f;
        Qb[i + j * kBjLd] = q[t];
    }
    __syncthreads();
    float w[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) w[u][v] = 0.0f;
    for (int k = 0; k < kBjM; ++k) {
        float x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = T[(ty * 4 + u) + k * kBjLd];
#pragma unroll
        for (int v = 0; v < 4; ++v) y[v] = Qb[k + (tx * 4 + v) * kBjLd];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) w[u][v] = fmaf(x[u], y[v], w[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = ty * 4 + u, j = tx * 4 + v;
            if (i < nr && j < mp) V[(r0 + i) + (long)bj_index(j, pi, npi, pj) * n] = w[u][v];
        }
}

size_t block_jacobi_f32_scratch(int n)
{
    const int nb = (n + kBjB - 1) / kBjB, nbe = nb + (nb & 1);
    return (size_t)(nbe / 2) * kBjM * kBjM * sizeof(float) + 256;
}

cudaError_t block_jacobi_f32(float *A, float *V, int n, void *scratch, int *sweeps_out,
                             int max_sweeps, cudaStream_t st)
{
    if (n <= 0 || n > kMaxDense) return cudaErrorInvalidValue;
    const int nb = (n + kBjB - 1) / kBjB, nbe = nb + (nb & 1), npairs = nbe / 2;
    BjState *bs = reinterpret_cast<BjState *>(scratch);
    float *Qs = reinterpret_cast<float *>(reinterpret_cast<char *>(scratch) + 256);
    k_bj_init<<<1, 1024, 0, st>>>(A, V, n, bs, 1.1920928955078125e-07);
    note_launch();
    const int nrb = (n + kBjM - 1) / kBjM;
    const int napply = npairs * (npairs + 1) / 2 + npairs * nrb;
    cudaError_t e;
    for (int s = 0; s < max_sweeps; ++s) {
        k_bj_sweep<<<1, 1, 0, st>>>(bs, s, 0);
        note_launch();
        for (int r = 0; r < nbe - 1; ++r) {
            k_bj_solve<<<npairs, kBjThreads, 0, st>>>(A, n, nbe, r, Qs, bs);
            note_launch();
            k_bj_apply<<<napply, kBjThreads, 0, st>>>(A, V, n, nbe, r, Qs, bs);
            note_launch();
        }
        k_bj_sweep<<<1, 1, 0, st>>>(bs, s, 1);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (s >= 2) {
            // from the third sweep on the host looks at the done flag (one small copy and a
            // stream synchronisation per sweep) instead of queueing sweeps that would return
            int done = 0;
            if ((e = cudaMemcpyAsync(&done, &bs->done, sizeof(int), cudaMemcpyDeviceToHost,
                                     st)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            if (done) break;
        }
    }
    if (sweeps_out)
        e = cudaMemcpyAsync(sweeps_out, &bs->sweeps, sizeof(int), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace sparc
