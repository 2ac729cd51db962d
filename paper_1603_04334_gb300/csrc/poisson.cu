// poisson.cu -- the electrostatic potential (Sec. 3.3): pseudocharges (Eq.
// PseudochargeDiscrete, Algorithm PseudochargeCalculation), multipole boundary values (Eq.
// phi:BC:discrete, l_max = 6 as in Sec. 4), the charge correction (Eq. Phi:correction)
// and the linear system -(1/4 pi) L_h phi = rho + b - d (Eq. FD:PoissonDiscrete) solved by
// conjugate gradients with a Jacobi preconditioner, all in FP64 on the device.
//
// The multipole terms use real solid harmonics R_lm(x) = |x|^l Y_lm(x/|x|), evaluated as
// polynomials: with Pi_l^m(z, r^2) the associated-Legendre recurrence in solid form
// (Pi_m^m = (2m-1)!!, Pi_{m+1}^m = (2m+1) z Pi_m^m, (l-m) Pi_l^m = (2l-1) z Pi_{l-1}^m -
// (l+m-1) r^2 Pi_{l-2}^m) and (x + iy)^m = A_m + i B_m, R_l0 = N_l0 Pi_l^0, R_lm = N_lm
// Pi_l^m A_m and R_l,-m = N_lm Pi_l^m B_m (m > 0), N the orthonormalisation constants.
// The boundary potential sum_m Y_lm(x) Q_lm depends only on the span of the degree-l
// harmonics, so any orthonormal real basis gives the same values.
//
// Every reduction (moments, CG dot products) runs in a fixed order: a block-level tree,
// then one CTA over the block partials, so results repeat bit for bit.
#include "internal.cuh"

namespace sparc {

namespace {
constexpr int kLmax = 6;
constexpr int kNQ = (kLmax + 1) * (kLmax + 1);  // 49 moments
constexpr int kPT = 256;                         // threads of the grid-wide kernels
constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)
constexpr double kSqrtPi = 1.7724538509055159;
constexpr int kVecGrid = 152 * 8;                // CTAs of the vector kernels and dot products
}  // namespace

// R_lm(x, y, z) for l <= 6 into S[l*l + l + m] (N: the 49 normalisation constants, same
// index).
__device__ __forceinline__ void solid_harmonics(double x, double y, double z, const double *N,
                                                double *S)
{
    const double r2 = x * x + y * y + z * z;
    double A = 1.0, B = 0.0;  // Re and Im of (x + iy)^m
    double pmm = 1.0;         // Pi_m^m = (2m-1)!!
#pragma unroll
    for (int m = 0; m <= kLmax; ++m) {
        if (m > 0) {
            const double a = A * x - B * y, b = A * y + B * x;
            A = a;
            B = b;
            pmm *= (double)(2 * m - 1);
        }
        double p2 = 0.0, p1 = pmm;  // Pi_{l-2}^m, Pi_{l-1}^m
#pragma unroll
        for (int l = m; l <= kLmax; ++l) {
            double pl;
            if (l == m)
                pl = pmm;
            else if (l == m + 1)
                pl = (double)(2 * m + 1) * z * pmm;
            else
                pl = ((double)(2 * l - 1) * z * p1 - (double)(l + m - 1) * r2 * p2) /
                     (double)(l - m);
            if (l > m) {
                p2 = p1;
                p1 = pl;
            }
            const int c = l * l + l;
            if (m == 0) {
                S[c] = N[c] * pl;
            } else {
                S[c + m] = N[c + m] * pl * A;
                S[c - m] = N[c + m] * pl * B;
            }
        }
    }
}

struct PoisCoef {
    double w[kRadius + 1];  // Laplacian weights (1/h^2 included); 6 w[0] is the centre's
    double N[kNQ];          // solid-harmonic normalisation
    double cx, cy, cz;      // expansion centre
    double h;
    int radius;
};

// V_ext on the grid extended by `radius` nodes beyond each face: sum_J -Z_J erf(r/rc)/r
// (r -> 0: -2 Z_J / (sqrt(pi) rc); r >= 6 rc: -Z_J / r, where erf rounds to 1).
__global__ void __launch_bounds__(kPT)
k_vext(double *__restrict__ Ve, int e0, int e1, int e2, int radius, double h,
       const double *__restrict__ R, const double *__restrict__ Z, int natoms, double rc)
{
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    const long ne = (long)e0 * e1 * e2;
    if (t >= ne) return;
    const int i = (int)(t % e0) - radius, j = (int)((t / e0) % e1) - radius,
              k = (int)(t / ((long)e0 * e1)) - radius;
    const double x = i * h, y = j * h, z = k * h;
    double v = 0.0;
    for (int J = 0; J < natoms; ++J) {
        const double dx = x - R[3 * J], dy = y - R[3 * J + 1], dz = z - R[3 * J + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < 1e-12)
            v -= 2.0 * Z[J] / (kSqrtPi * rc);
        else if (r >= 6.0 * rc)
            v -= Z[J] / r;
        else
            v -= Z[J] * erf(r / rc) / r;
    }
    Ve[t] = v;
}

// b = -(1/4 pi) L_h V_ext at the grid nodes (Eq. PseudochargeDiscrete).
__global__ void __launch_bounds__(kPT)
k_pseudocharge(const double *__restrict__ Ve, double *__restrict__ b, int n0, int n1, int n2,
               PoisCoef pc)
{
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    const long nd = (long)n0 * n1 * n2;
    if (t >= nd) return;
    const int R = pc.radius;
    const int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / ((long)n0 * n1));
    const long e0 = n0 + 2 * R, e01 = e0 * (n1 + 2 * R);
    const long c = (i + R) + (j + R) * e0 + (k + R) * e01;
    double L = 6.0 * pc.w[0] * Ve[c];
    for (int p = 1; p <= R; ++p)
        L += pc.w[p] * (Ve[c + p] + Ve[c - p] + Ve[c + p * e0] + Ve[c - p * e0] +
                        Ve[c + p * e01] + Ve[c - p * e01]);
    b[t] = -kInv4Pi * L;
}

// Block partials of sum (rho + b) R_lm(x - centre) over the grid: part[block * 49 + q].
__global__ void __launch_bounds__(kPT)
k_moments(const double *__restrict__ rho, const double *__restrict__ b, int n0, int n1, int n2,
          PoisCoef pc, double *__restrict__ part)
{
    __shared__ double sh[kPT / 32][kNQ];
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    const long nd = (long)n0 * n1 * n2;
    double S[kNQ];
    double f = 0.0;
    if (t < nd) {
        f = (rho ? rho[t] : 0.0) + b[t];
        const int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / ((long)n0 * n1));
        solid_harmonics(i * pc.h - pc.cx, j * pc.h - pc.cy, k * pc.h - pc.cz, pc.N, S);
    } else {
#pragma unroll
        for (int q = 0; q < kNQ; ++q) S[q] = 0.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
        double v = f * S[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kNQ; q += kPT) {
        double v = 0.0;
        for (int w = 0; w < kPT / 32; ++w) v += sh[w][q];
        part[(long)blockIdx.x * kNQ + q] = v;
    }
}

// out[q] = scale * sum_b part[b * stride + q] over nblk blocks (one CTA, fixed order).
__global__ void __launch_bounds__(kPT)
k_sum_partials(const double *__restrict__ part, int nblk, int nq, double scale, double *out)
{
    __shared__ double sh[kPT];
    for (int q = 0; q < nq; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblk; b += kPT) v += part[(long)b * nq + q];
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int s = kPT / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = scale * sh[0];
        __syncthreads();
    }
}

// phi at the nodes outside the grid that a grid node's stencil reaches: face f (0: i < 0,
// 1: i >= n0, 2: j < 0, 3: j >= n1, 4: k < 0, 5: k >= n2), layer p = 1..radius, and the
// face's two in-grid coordinates (a fastest). Eq. (phi:BC:discrete):
// phi = sum_l 4 pi / (2l + 1) r^-(2l+1) sum_m R_lm(x) Q_lm.
__global__ void __launch_bounds__(kPT)
k_phi_ext(double *__restrict__ pe, int n0, int n1, int n2, PoisCoef pc,
          const double *__restrict__ Q, long total)
{
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    if (t >= total) return;
    const int R = pc.radius;
    const long s01 = (long)n1 * n2 * R, s23 = (long)n0 * n2 * R;
    int f;
    long u;
    if (t < 2 * s01) {
        f = (int)(t / s01);
        u = t % s01;
    } else if (t < 2 * s01 + 2 * s23) {
        f = 2 + (int)((t - 2 * s01) / s23);
        u = (t - 2 * s01) % s23;
    } else {
        const long s45 = (long)n0 * n1 * R;
        f = 4 + (int)((t - 2 * s01 - 2 * s23) / s45);
        u = (t - 2 * s01 - 2 * s23) % s45;
    }
    const int na = f < 2 ? n1 : n0, nb = f < 4 ? n2 : n1;
    const int a = (int)(u % na), bb = (int)((u / na) % nb), p = (int)(u / ((long)na * nb)) + 1;
    int i, j, k;
    switch (f) {
    case 0: i = -p; j = a; k = bb; break;
    case 1: i = n0 - 1 + p; j = a; k = bb; break;
    case 2: i = a; j = -p; k = bb; break;
    case 3: i = a; j = n1 - 1 + p; k = bb; break;
    case 4: i = a; j = bb; k = -p; break;
    default: i = a; j = bb; k = n2 - 1 + p; break;
    }
    const double x = i * pc.h - pc.cx, y = j * pc.h - pc.cy, z = k * pc.h - pc.cz;
    double S[kNQ];
    solid_harmonics(x, y, z, pc.N, S);
    const double r2 = x * x + y * y + z * z, r = sqrt(r2);
    double phi = 0.0, rp = r;  // rp = r^(2l+1)
#pragma unroll
    for (int l = 0; l <= kLmax; ++l) {
        double s = 0.0;
#pragma unroll
        for (int m = -l; m <= l; ++m) s += S[l * l + l + m] * Q[l * l + l + m];
        phi += 4.0 * M_PI / (double)(2 * l + 1) * s / rp;
        rp *= r2;
    }
    pe[t] = phi;
}

// rhs = rho + b - d, d = -(1/4 pi) sum_p w_p (phi at the outside neighbours at distance p)
// (Eq. Phi:correction).
__global__ void __launch_bounds__(kPT)
k_poisson_rhs(const double *__restrict__ rho, const double *__restrict__ b,
              const double *__restrict__ pe, int n0, int n1, int n2, PoisCoef pc,
              double *__restrict__ rhs)
{
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    const long nd = (long)n0 * n1 * n2;
    if (t >= nd) return;
    const int R = pc.radius;
    const int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / ((long)n0 * n1));
    const long s01 = (long)n1 * n2 * R, s23 = (long)n0 * n2 * R, s45 = (long)n0 * n1 * R;
    const long o[6] = {0, s01, 2 * s01, 2 * s01 + s23, 2 * s01 + 2 * s23,
                       2 * s01 + 2 * s23 + s45};
    // the neighbour at distance p beyond a face lies in that face's layer q (1..R): q = p - i
    // below the grid, q = i + p - (n0 - 1) above it (likewise for j, k)
    double d = 0.0;
    for (int p = 1; p <= R; ++p) {
        double s = 0.0;
        if (i - p < 0) s += pe[o[0] + (long)(p - i - 1) * n1 * n2 + j + (long)k * n1];
        if (i + p >= n0) s += pe[o[1] + (long)(i + p - n0) * n1 * n2 + j + (long)k * n1];
        if (j - p < 0) s += pe[o[2] + (long)(p - j - 1) * n0 * n2 + i + (long)k * n0];
        if (j + p >= n1) s += pe[o[3] + (long)(j + p - n1) * n0 * n2 + i + (long)k * n0];
        if (k - p < 0) s += pe[o[4] + (long)(p - k - 1) * n0 * n1 + i + (long)j * n0];
        if (k + p >= n2) s += pe[o[5] + (long)(k + p - n2) * n0 * n1 + i + (long)j * n0];
        d += pc.w[p] * s;
    }
    d *= -kInv4Pi;
    rhs[t] = (rho ? rho[t] : 0.0) + b[t] - d;
}

// out = -(1/4 pi) L_h in (zero Dirichlet), one node per thread; the FP64 stencil of a
// single vector is light enough for the plain form.
__global__ void __launch_bounds__(kPT)
k_poisson_apply(const double *__restrict__ in, double *__restrict__ out, int n0, int n1, int n2,
                PoisCoef pc, const int *done)
{
    if (*(volatile const int *)done) return;
    const long t = (long)blockIdx.x * kPT + threadIdx.x;
    const long nd = (long)n0 * n1 * n2;
    if (t >= nd) return;
    const int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / ((long)n0 * n1));
    const long pl = (long)n0 * n1;
    double L = 6.0 * pc.w[0] * in[t];
    for (int p = 1; p <= pc.radius; ++p) {
        double s = 0.0;
        if (i + p < n0) s += in[t + p];
        if (i - p >= 0) s += in[t - p];
        if (j + p < n1) s += in[t + (long)p * n0];
        if (j - p >= 0) s += in[t - (long)p * n0];
        if (k + p < n2) s += in[t + p * pl];
        if (k - p >= 0) s += in[t - p * pl];
        L += pc.w[p] * s;
    }
    out[t] = -kInv4Pi * L;
}

// Block partials of a.b (and of c.c when c is not null): part[2 block], part[2 block + 1].
__global__ void __launch_bounds__(kPT)
k_dot2(const double *__restrict__ a, const double *__restrict__ b, const double *__restrict__ c,
       long n, double *__restrict__ part, const int *done)
{
    __shared__ double sh[2][kPT / 32];
    if (*(volatile const int *)done) return;
    double u = 0.0, v = 0.0;
    for (long t = (long)blockIdx.x * kPT + threadIdx.x; t < n; t += (long)gridDim.x * kPT) {
        u = fma(a[t], b[t], u);
        if (c) v = fma(c[t], c[t], v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_down_sync(0xffffffffu, u, o);
        v += __shfl_down_sync(0xffffffffu, v, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = u;
        sh[1][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0, sv = 0.0;
        for (int w = 0; w < kPT / 32; ++w) {
            su += sh[0][w];
            sv += sh[1][w];
        }
        part[2 * blockIdx.x] = su;
        part[2 * blockIdx.x + 1] = sv;
    }
}

// CG scalars (device): s[0] = |f|^2, s[1 + (it & 1)] = r.z of iteration it, s[3] = p.Ap,
// s[4] = r.r, s[5] = alpha.
// Sums the dot partials in a fixed order. mode 0: s[3] = p.Ap. mode 1: s[1 + nxt] = r.z,
// s[4] = r.r and done = (r.r <= tol^2 |f|^2), iters = it. mode 2: r.z and |f|^2 at the start.
__global__ void __launch_bounds__(kPT)
k_cg_scalars(const double *__restrict__ part, int nblk, double *s, int mode, int it,
             double tol2, int *done, int *iters)
{
    __shared__ double sh[2][kPT];
    if (*(volatile const int *)done) return;
    double u = 0.0, v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kPT) {
        u += part[2 * b];
        v += part[2 * b + 1];
    }
    sh[0][threadIdx.x] = u;
    sh[1][threadIdx.x] = v;
    __syncthreads();
    for (int q = kPT / 2; q > 0; q >>= 1) {
        if (threadIdx.x < q) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + q];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + q];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        s[3] = sh[0][0];
        s[5] = s[1 + (it & 1)] / s[3];
    } else if (mode == 1) {
        s[1 + ((it + 1) & 1)] = sh[0][0];
        s[4] = sh[1][0];
        *iters = it + 1;
        if (s[4] <= tol2 * s[0]) *done = 1;
    } else {
        s[1] = sh[0][0];
        s[0] = sh[1][0];
        if (s[0] == 0.0) *done = 1;
    }
}

// x += alpha p, r -= alpha Ap, z = r / diag.
__global__ void __launch_bounds__(kPT)
k_cg_update(double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
            const double *__restrict__ p, const double *__restrict__ Ap, long n, double idiag,
            const double *s, const int *done)
{
    if (*(volatile const int *)done) return;
    const double alpha = s[5];
    for (long t = (long)blockIdx.x * kPT + threadIdx.x; t < n; t += (long)gridDim.x * kPT) {
        x[t] = fma(alpha, p[t], x[t]);
        const double rt = fma(-alpha, Ap[t], r[t]);
        r[t] = rt;
        z[t] = rt * idiag;
    }
}

// p = z + beta p, beta = (r.z)_new / (r.z)_old.
__global__ void __launch_bounds__(kPT)
k_cg_direction(double *__restrict__ p, const double *__restrict__ z, long n, const double *s,
               int it, const int *done)
{
    if (*(volatile const int *)done) return;
    const double beta = s[1 + ((it + 1) & 1)] / s[1 + (it & 1)];
    for (long t = (long)blockIdx.x * kPT + threadIdx.x; t < n; t += (long)gridDim.x * kPT)
        p[t] = fma(beta, p[t], z[t]);
}

// r = f, z = f / diag, p = z, x = 0.
__global__ void __launch_bounds__(kPT)
k_cg_init(const double *__restrict__ f, double *__restrict__ x, double *__restrict__ r,
          double *__restrict__ z, double *__restrict__ p, long n, double idiag)
{
    for (long t = (long)blockIdx.x * kPT + threadIdx.x; t < n; t += (long)gridDim.x * kPT) {
        const double v = f[t];
        x[t] = 0.0;
        r[t] = v;
        z[t] = v * idiag;
        p[t] = v * idiag;
    }
}

size_t poisson_workspace(int n0, int n1, int n2, int radius)
{
    const long nd = (long)n0 * n1 * n2;
    const long ne = (long)(n0 + 2 * radius) * (n1 + 2 * radius) * (n2 + 2 * radius);
    const long nshell = 2L * radius * ((long)n1 * n2 + (long)n0 * n2 + (long)n0 * n1);
    const long nblk = (nd + kPT - 1) / kPT;
    const long nparts = nblk * kNQ > 2L * kVecGrid ? nblk * kNQ : 2L * kVecGrid;
    // b, rhs, r, z, p, Ap; V_ext; shell; partials; Q (49) + scalars (8)
    return sizeof(double) * (size_t)(6 * nd + ne + nshell + nparts + kNQ + 8) + 2 * sizeof(int);
}

cudaError_t poisson_solve(const DevHam &H, const double *R, const double *Z, int natoms,
                          double rc, const double *rho, double *phi, double *b_out, double tol,
                          int maxit, void *ws, int *iters_host, double *relres_host,
                          cudaStream_t st)
{
    const int n0 = H.n0, n1 = H.n1, n2 = H.n2, Rr = H.radius;
    const long nd = (long)n0 * n1 * n2;
    const long ne = (long)(n0 + 2 * Rr) * (n1 + 2 * Rr) * (n2 + 2 * Rr);
    const long nshell = 2L * Rr * ((long)n1 * n2 + (long)n0 * n2 + (long)n0 * n1);
    const long nblk = (nd + kPT - 1) / kPT;
    const long nparts = nblk * kNQ > 2L * kVecGrid ? nblk * kNQ : 2L * kVecGrid;
    double *w = (double *)ws;
    double *b = w, *rhs = b + nd, *r = rhs + nd, *z = r + nd, *p = z + nd, *Ap = p + nd;
    double *Ve = Ap + nd, *pe = Ve + ne, *part = pe + nshell, *Q = part + nparts, *s = Q + kNQ;
    int *done = (int *)(s + 8), *iters = done + 1;

    PoisCoef pc;
    for (int q = 0; q <= kRadius; ++q) pc.w[q] = H.w[q];
    pc.h = H.h;
    pc.radius = Rr;
    pc.cx = 0.5 * (n0 - 1) * H.h;
    pc.cy = 0.5 * (n1 - 1) * H.h;
    pc.cz = 0.5 * (n2 - 1) * H.h;
    for (int l = 0; l <= kLmax; ++l) {
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0;  // (l - m)! / (l + m)!
            for (int q = l - m + 1; q <= l + m; ++q) ratio /= (double)q;
            const double nlm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio * (m ? 2.0 : 1.0));
            pc.N[l * l + l + m] = nlm;
            pc.N[l * l + l - m] = nlm;
        }
    }
    const double idiag = 1.0 / (-kInv4Pi * 6.0 * H.w[0]);
    cudaError_t e;
    // pseudocharge, moments, boundary values, right-hand side
    k_vext<<<(unsigned)((ne + kPT - 1) / kPT), kPT, 0, st>>>(Ve, n0 + 2 * Rr, n1 + 2 * Rr,
                                                             n2 + 2 * Rr, Rr, H.h, R, Z, natoms,
                                                             rc);
    note_launch();
    k_pseudocharge<<<(unsigned)nblk, kPT, 0, st>>>(Ve, b, n0, n1, n2, pc);
    note_launch();
    k_moments<<<(unsigned)nblk, kPT, 0, st>>>(rho, b, n0, n1, n2, pc, part);
    note_launch();
    k_sum_partials<<<1, kPT, 0, st>>>(part, (int)nblk, kNQ, H.h * H.h * H.h, Q);
    note_launch();
    k_phi_ext<<<(unsigned)((nshell + kPT - 1) / kPT), kPT, 0, st>>>(pe, n0, n1, n2, pc, Q,
                                                                    nshell);
    note_launch();
    k_poisson_rhs<<<(unsigned)nblk, kPT, 0, st>>>(rho, b, pe, n0, n1, n2, pc, rhs);
    note_launch();
    if (b_out) {
        if ((e = cudaMemcpyAsync(b_out, b, sizeof(double) * nd, cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
            return e;
    }
    // CG from phi = 0
    const unsigned gv = kVecGrid;
    if ((e = cudaMemsetAsync(done, 0, 2 * sizeof(int), st)) != cudaSuccess) return e;
    k_cg_init<<<gv, kPT, 0, st>>>(rhs, phi, r, z, p, nd, idiag);
    note_launch();
    k_dot2<<<gv, kPT, 0, st>>>(r, z, rhs, nd, part, done);
    note_launch();
    k_cg_scalars<<<1, kPT, 0, st>>>(part, gv, s, 2, 0, tol * tol, done, iters);
    note_launch();
    int done_h = 0, it_h = 0;
    const int kBatch = 16;  // iterations between host checks of the done flag
    for (int it = 0; it < maxit; ++it) {
        k_poisson_apply<<<(unsigned)nblk, kPT, 0, st>>>(p, Ap, n0, n1, n2, pc, done);
        k_dot2<<<gv, kPT, 0, st>>>(p, Ap, nullptr, nd, part, done);
        k_cg_scalars<<<1, kPT, 0, st>>>(part, gv, s, 0, it, 0.0, done, iters);
        k_cg_update<<<gv, kPT, 0, st>>>(phi, r, z, p, Ap, nd, idiag, s, done);
        k_dot2<<<gv, kPT, 0, st>>>(r, z, r, nd, part, done);
        k_cg_scalars<<<1, kPT, 0, st>>>(part, gv, s, 1, it, tol * tol, done, iters);
        k_cg_direction<<<gv, kPT, 0, st>>>(p, z, nd, s, it, done);
        for (int q = 0; q < 7; ++q) note_launch();
        if ((it + 1) % kBatch == 0 || it + 1 == maxit) {
            if ((e = cudaMemcpyAsync(&done_h, done, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            if (done_h) break;
        }
    }
    double sc[8];
    if ((e = cudaMemcpyAsync(sc, s, sizeof(sc), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&it_h, iters, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&done_h, done, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    *iters_host = it_h;
    *relres_host = sc[0] > 0.0 ? sqrt(sc[4] / sc[0]) : 0.0;
    return cudaGetLastError();
}

}  // namespace sparc
