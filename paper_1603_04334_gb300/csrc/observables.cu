// observables.cu -- the steps after the subspace rotation: occupations and the Fermi level
// (Eq. FermiEnergyConstraintFormulation), the electron density (Sec. 3.4, the equation
// after Eq. OrbitalTransformation) and the non-local atomic force (Eq. NonlocForce:Discrete
// with Y and W of Eq. NonLocForce:U:W, Algorithm non-localForceCalculation), all in FP64.
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int kFermiThreads = 256;
constexpr int kFermiMaxIter = 200;
constexpr int kDensityThreads = 256;
constexpr int kForceThreads = 256;

// Sums of a and b over the block in a fixed order (same result on every launch).
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[NT])
{
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    a = sh[0][0];
    b = sh[1][0];
    __syncthreads();
}
}  // namespace

// One CTA. F(mu) = 2 sum_n g_n(mu) - N_e increases with mu; F' = (2 / kT) sum g (1 - g).
// A bracket [lo, hi] with F(lo) <= 0 <= F(hi) is grown from [min lambda - 1, max lambda + 1];
// from its midpoint, Newton steps are taken while they land inside the bracket and the
// bracket at least halves every two steps, bisection otherwise (the paper finds the same
// root with Brent's method, Sec. 4). Stops when the Newton step is below 2 ulp of mu,
// F(mu) = 0, or the bracket is 4 ulp wide. status: 0 converged, 1 no convergence, 2 a
// non-finite eigenvalue.
__global__ void __launch_bounds__(kFermiThreads)
k_fermi(const double *__restrict__ lam, int ns, double nelec, double kT, double *mu_out,
        double *g, int *status)
{
    __shared__ double red[2][kFermiThreads];
    const double eps = 2.220446049250313e-16;
    auto eval = [&](double mu, double &F, double &dF) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < ns; i += kFermiThreads) {
            const double gi = 1.0 / (1.0 + exp((lam[i] - mu) / kT));
            a += gi;
            b += gi * (1.0 - gi);
        }
        block_sum2<kFermiThreads>(a, b, red);
        F = 2.0 * a - nelec;
        dF = 2.0 * b / kT;
    };
    // extremes of the spectrum
    double lmin = INFINITY, lmax = -INFINITY;
    bool finite = true;
    for (int i = threadIdx.x; i < ns; i += kFermiThreads) {
        const double v = lam[i];
        finite = finite && isfinite(v);
        lmin = fmin(lmin, v);
        lmax = fmax(lmax, v);
    }
    finite = __syncthreads_and(finite);
    red[0][threadIdx.x] = lmin;
    red[1][threadIdx.x] = lmax;
    __syncthreads();
    for (int s = kFermiThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] = fmin(red[0][threadIdx.x], red[0][threadIdx.x + s]);
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
        }
        __syncthreads();
    }
    lmin = red[0][0];
    lmax = red[1][0];
    __syncthreads();
    if (!finite) {
        if (threadIdx.x == 0) *status = 2;
        return;
    }
    double lo = lmin - 1.0, hi = lmax + 1.0, F, dF;
    double width = hi - lo;
    for (int t = 0; t < 64; ++t) {  // F(lo) <= 0 (N_e > 0)
        eval(lo, F, dF);
        if (F <= 0.0) break;
        lo -= width;
        width *= 2.0;
    }
    width = hi - lo;
    for (int t = 0; t < 64; ++t) {  // F(hi) >= 0 (N_e < 2 Ns)
        eval(hi, F, dF);
        if (F >= 0.0) break;
        hi += width;
        width *= 2.0;
    }
    double mu = 0.5 * (lo + hi);
    eval(mu, F, dF);
    double w_prev2 = INFINITY, w_prev = INFINITY;
    int st = 1;
    for (int it = 0; it < kFermiMaxIter; ++it) {
        if (F == 0.0) {
            st = 0;
            break;
        }
        if (F < 0.0)
            lo = mu;
        else
            hi = mu;
        const double w = hi - lo;
        if (w <= 4.0 * eps * fmax(fabs(lo), fabs(hi))) {
            st = 0;
            break;
        }
        const double nx = dF > 0.0 ? mu - F / dF : NAN;  // NaN fails the range test
        const bool newton = nx > lo && nx < hi && (it < 2 || w <= 0.5 * w_prev2);
        if (newton && fabs(nx - mu) <= 2.0 * eps * fabs(mu)) {
            mu = nx;
            st = 0;
            break;
        }
        w_prev2 = w_prev;
        w_prev = w;
        mu = newton ? nx : 0.5 * (lo + hi);
        eval(mu, F, dF);
    }
    for (int i = threadIdx.x; i < ns; i += kFermiThreads)
        g[i] = 1.0 / (1.0 + exp((lam[i] - mu) / kT));
    if (threadIdx.x == 0) {
        *mu_out = mu;
        *status = st;
    }
}

cudaError_t fermi_level(const double *lam, int ns, double nelec, double kT, double *mu,
                        double *g, int *status, cudaStream_t st)
{
    k_fermi<<<1, kFermiThreads, 0, st>>>(lam, ns, nelec, kT, mu, g, status);
    note_launch();
    return cudaGetLastError();
}

// rho[p] = scale * sum_n g_n x_n[p]^2, columns in ascending order; one node per thread, eight
// column loads in flight.
template <typename T>
__global__ void __launch_bounds__(kDensityThreads)
k_density(const T *__restrict__ X, long ld, int ncols, long nd, const double *__restrict__ g,
          double scale, double *__restrict__ rho)
{
    const long p = (long)blockIdx.x * kDensityThreads + threadIdx.x;
    if (p >= nd) return;
    const T *x = X + p;
    double acc = 0.0;
    int n = 0;
    for (; n + 8 <= ncols; n += 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = x[(long)(n + u) * ld];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double d = (double)v[u];
            acc = fma(g[n + u] * d, d, acc);
        }
    }
    for (; n < ncols; ++n) {
        const double d = (double)x[(long)n * ld];
        acc = fma(g[n] * d, d, acc);
    }
    rho[p] = scale * acc;
}

template <typename T>
cudaError_t density(const T *X, long ld, int ncols, long nd, const double *g, double h,
                    double *rho, cudaStream_t st)
{
    const long blocks = (nd + kDensityThreads - 1) / kDensityThreads;
    k_density<T><<<(unsigned)blocks, kDensityThreads, 0, st>>>(X, ld, ncols, nd, g,
                                                               2.0 / (h * h * h), rho);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t density<double>(const double *, long, int, long, const double *, double,
                                     double *, cudaStream_t);
template cudaError_t density<float>(const float *, long, int, long, const double *, double,
                                    double *, cudaStream_t);

// One CTA per (atom J, column n). Over the atom's support entries: y_l = sum x chi_l and
// w_dl = sum (grad_h x)_d chi_l, with grad_h of Eq. (gradient:approximate) evaluated at the
// entry's node from the column (zero outside the grid); out[(J ncols + n) 16 + k]:
// k = l (y), 4 + 4 d + l (w).
template <typename T>
__global__ void __launch_bounds__(kForceThreads)
k_force_yw(const T *__restrict__ X, long ld, const int *__restrict__ atom_ptr,
           const int *__restrict__ idx, const double *__restrict__ chi, int n0, int n1, int n2,
           int radius, GradCoef wg, double *__restrict__ out)
{
    __shared__ double red[2][kForceThreads];
    const int J = blockIdx.x, n = blockIdx.y, ncols = gridDim.y;
    const T *x = X + (long)n * ld;
    const int e0 = atom_ptr[J], e1 = atom_ptr[J + 1];
    const long plane = (long)n0 * n1;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += kForceThreads) {
        const long p = idx[e];
        const int i = (int)(p % n0), j = (int)((p / n0) % n1), k = (int)(p / plane);
        double gd[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int r = 1; r <= kRadius; ++r) {
            if (r > radius) break;
            const double ax = (i + r < n0 ? (double)x[p + r] : 0.0) -
                              (i - r >= 0 ? (double)x[p - r] : 0.0);
            const double ay = (j + r < n1 ? (double)x[p + (long)r * n0] : 0.0) -
                              (j - r >= 0 ? (double)x[p - (long)r * n0] : 0.0);
            const double az = (k + r < n2 ? (double)x[p + r * plane] : 0.0) -
                              (k - r >= 0 ? (double)x[p - r * plane] : 0.0);
            gd[0] = fma(wg.w[r], ax, gd[0]);
            gd[1] = fma(wg.w[r], ay, gd[1]);
            gd[2] = fma(wg.w[r], az, gd[2]);
        }
        const double xc = (double)x[p];
        const double *c = chi + 4L * e;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const double cl = c[l];
            acc[l] = fma(xc, cl, acc[l]);
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[4 + 4 * d + l] = fma(gd[d], cl, acc[4 + 4 * d + l]);
        }
    }
    double *o = out + ((long)J * ncols + n) * 16;
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        double a = acc[k], b = acc[k + 1];
        block_sum2<kForceThreads>(a, b, red);
        if (threadIdx.x == 0) {
            o[k] = a;
            o[k + 1] = b;
        }
    }
}

// f_Jd = -4 h^3 sum_n g_n sum_lm gamma_Jl y_nl w_ndl (columns in ascending order); one thread
// per (atom, direction).
__global__ void k_force_sum(const double *__restrict__ yw, const double *__restrict__ g,
                            const double *__restrict__ gamma, int natoms, int ncols, double h3,
                            double *__restrict__ f)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * natoms) return;
    const int J = t / 3, d = t % 3;
    const double *gm = gamma + 4L * J;
    double s = 0.0;
    for (int n = 0; n < ncols; ++n) {
        const double *v = yw + ((long)J * ncols + n) * 16;
        double a = 0.0;
#pragma unroll
        for (int l = 0; l < 4; ++l) a = fma(gm[l] * v[l], v[4 + 4 * d + l], a);
        s = fma(g[n], a, s);
    }
    f[t] = -4.0 * h3 * s;
}

template <typename T>
cudaError_t nonlocal_force(const DevHam &H, const T *X, long ld, int ncols, const double *g,
                           const double *gamma, const GradCoef &wg, double *yw, double *f,
                           cudaStream_t st)
{
    if (H.natoms <= 0) return cudaSuccess;
    dim3 grid(H.natoms, ncols);
    k_force_yw<T><<<grid, kForceThreads, 0, st>>>(X, ld, H.atom_ptr, H.idx, H.chi, H.n0, H.n1,
                                                  H.n2, H.radius, wg, yw);
    note_launch();
    const int nt = 3 * H.natoms;
    k_force_sum<<<(nt + 127) / 128, 128, 0, st>>>(yw, g, gamma, H.natoms, ncols,
                                                  H.h * H.h * H.h, f);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t nonlocal_force<double>(const DevHam &, const double *, long, int,
                                            const double *, const double *, const GradCoef &,
                                            double *, double *, cudaStream_t);
template cudaError_t nonlocal_force<float>(const DevHam &, const float *, long, int,
                                           const double *, const double *, const GradCoef &,
                                           double *, double *, cudaStream_t);

GradCoef grad_coef(int radius, double h)
{
    // w~_p = (-1)^(p+1) / (h p) (n_o!)^2 / ((n_o - p)! (n_o + p)!), the ratio formed as the
    // product over q = 1..p of (n_o - q + 1) / (n_o + q)
    GradCoef c;
    for (int p = 0; p <= kRadius; ++p) c.w[p] = 0.0;
    for (int p = 1; p <= radius; ++p) {
        double ratio = 1.0;
        for (int q = 1; q <= p; ++q) ratio *= (double)(radius - q + 1) / (double)(radius + q);
        c.w[p] = ((p % 2) ? 1.0 : -1.0) * ratio / (h * p);
    }
    return c;
}

}  // namespace sparc
