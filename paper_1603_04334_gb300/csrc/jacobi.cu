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
// The grid barrier is a counter/generation pair in global memory; the kernel is launched
// cooperatively (all CTAs co-resident), and every wait is bounded: after kBarrierSpins
// polls the waiting CTA raises an error flag, every CTA leaves at its next barrier and the
// host reports SPARC_ERR_TIMEOUT.
#include "grid.cuh"
#include "internal.cuh"

#include <atomic>
#include <type_traits>

namespace sparc {

namespace {
constexpr int NT = 256;
constexpr int kMaxSweeps = 60;
constexpr double kEps = 2.220446049250313e-16;
// CTAs of a grid Jacobi, at most. A round streams all of A and V through L2; the FP32
// pre-solve's rounds go faster with two CTAs per SM (more loads in flight: 197 against
// 213 ms per Ns = 1024 dense step; one per SM: 274 ms with 76 CTAs), the FP64 ones, bound
// by the FP64 pipe, gain nothing from a second CTA per SM.
constexpr int kJacobiCtasF32 = 304;
constexpr int kJacobiCtasF64 = 152;

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

// T = double: the eigensolve; T = float: the FP32 pre-solve of the mixed-precision
// eigensolve (dense.cu), with eps the unit roundoff of T.
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
    const int cap = std::is_same<T, float>::value ? kJacobiCtasF32 : kJacobiCtasF64;
    if (G > cap) G = cap;
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

cudaError_t jacobi_grid_f32(float *A0, float *A1, float *V, float *diag, int n, GridBarrier *bar,
                            int *status, int *sweeps_out, int max_sweeps, cudaStream_t st)
{
    return jacobi_grid_t<float>(A0, A1, V, diag, n, bar, status, sweeps_out,
                                1.1920928955078125e-07, max_sweeps, st);
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

}  // namespace sparc
