/*
 * sparc_oracle.c -- plain FP64 CPU oracle for the Chebyshev-filtered subspace
 * iteration (CheFSI) hot path of SPARC for isolated clusters
 * (Ghosh & Suryanarayana, arXiv:1603.04334).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never loads it.
 *
 * Everything is written as plain loops in double precision, in the order the
 * paper states the operations, and is compiled with -ffp-contract=off so that
 * every a*b+c is two roundings. The only parallelism is an OpenMP loop over
 * independent orbital columns (results do not depend on the thread count).
 *
 * Grid convention: nodes i = 0..n0-1, j = 0..n1-1, k = 0..n2-1 at coordinates
 * (i*h, j*h, k*h); linear index p = i + n0*(j + n1*k) (x fastest). A block of
 * orbitals is column-major: column c starts at X + c*ld, ld >= Nd.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Thread count of the OpenMP loops (for timing the oracle on 1 or all host cores; the
 * results do not depend on it). n <= 0 leaves the count unchanged. Returns the count in
 * effect. */
int orc_threads(int n)
{
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
}

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------
 * Finite-difference Laplacian weights, Eq. (weightsLap), Sec. 3.1:
 *   w_0 = -(1/h^2) sum_{q=1}^{n_o} 1/q^2
 *   w_p = 2 (-1)^{p+1} / (h^2 p^2) * (n_o!)^2 / ((n_o-p)! (n_o+p)!)
 * The factorial ratio is formed as prod_{q=1}^{p} (n_o-q+1)/(n_o+q).
 * ------------------------------------------------------------------------- */
void orc_lap_weights(int no, double h, double *w)
{
    double s = 0.0;
    for (int q = 1; q <= no; ++q)
        s += 1.0 / ((double)q * (double)q);
    w[0] = -s / (h * h);
    for (int p = 1; p <= no; ++p) {
        double ratio = 1.0;
        for (int q = 1; q <= p; ++q)
            ratio *= (double)(no - q + 1) / (double)(no + q);
        double sign = (p % 2 == 1) ? 1.0 : -1.0;
        w[p] = 2.0 * sign / (h * h * (double)p * (double)p) * ratio;
    }
}

/* Zero-Dirichlet read (Sec. 3.1: f = 0 at any index that is not a node). */
static double at(const double *f, int n0, int n1, int n2, int i, int j, int k)
{
    if (i < 0 || i >= n0 || j < 0 || j >= n1 || k < 0 || k >= n2)
        return 0.0;
    return f[(long)i + (long)n0 * ((long)j + (long)n1 * (long)k)];
}

/* ---------------------------------------------------------------------------
 * Discrete Laplacian, Eq. (FD:Laplacian), Sec. 3.1, for one grid function:
 *   (L_h f)(i,j,k) = sum_{p=0}^{n_o} w_p [ f(i+p,j,k) + f(i-p,j,k) + f(i,j+p,k)
 *                     + f(i,j-p,k) + f(i,j,k+p) + f(i,j,k-p) ]
 * The p = 0 term lists f(i,j,k) six times, so the centre weight is 6 w_0.
 * ------------------------------------------------------------------------- */
void orc_laplacian(int n0, int n1, int n2, double h, int no,
                   const double *f, double *out)
{
    double w[64];
    orc_lap_weights(no, h, w);
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                double s = 0.0;
                for (int p = 0; p <= no; ++p) {
                    double t = at(f, n0, n1, n2, i + p, j, k) + at(f, n0, n1, n2, i - p, j, k)
                             + at(f, n0, n1, n2, i, j + p, k) + at(f, n0, n1, n2, i, j - p, k)
                             + at(f, n0, n1, n2, i, j, k + p) + at(f, n0, n1, n2, i, j, k - p);
                    s += w[p] * t;
                }
                out[(long)i + (long)n0 * ((long)j + (long)n1 * (long)k)] = s;
            }
}

/* ---------------------------------------------------------------------------
 * Local potential used by the synthetic clusters:
 *   V_eff(x) = sum_J -Z_J erf(|x - R_J| / rc) / |x - R_J|,
 * with the limit -2 Z_J / (sqrt(pi) rc) at |x - R_J| -> 0 (taken for r < 1e-12).
 * ------------------------------------------------------------------------- */
void orc_veff(int n0, int n1, int n2, double h, int natoms, const double *R,
              const double *Z, double rc, double *V)
{
    /* every node is computed on its own (same sum order at any thread count) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                double x = (double)i * h, y = (double)j * h, z = (double)k * h;
                double v = 0.0;
                for (int J = 0; J < natoms; ++J) {
                    double dx = x - R[3 * J], dy = y - R[3 * J + 1], dz = z - R[3 * J + 2];
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    if (r < 1e-12)
                        v += -Z[J] * 2.0 / (sqrt(M_PI) * rc);
                    else
                        v += -Z[J] * erf(r / rc) / r;
                }
                V[(long)i + (long)n0 * ((long)j + (long)n1 * (long)k)] = v;
            }
}

/* ---------------------------------------------------------------------------
 * Kleinman-Bylander projectors, Sec. 2 (separable form) and Eq.
 * (non-localPS:FD), Sec. 3.1. Each atom J owns the nodes within rcut of R_J
 * (inclusive: r^2 <= rcut^2, with r^2 = dx*dx + dy*dy + dz*dz evaluated in
 * that order); nodes outside the grid do not exist. On each support node:
 *   chi_s  = Y00 exp(-r^2 / (2 sigma^2)),               Y00 = 1 / (2 sqrt(pi))
 *   chi_pd = sqrt(3 / (4 pi)) (x_d - R_d) exp(-r^2 / (2 sigma^2)),  d = x, y, z
 * (r^l exp(-r^2/(2 sigma^2)) Y_lm with real spherical harmonics).
 * Support entries are listed atom by atom, nodes in increasing linear index.
 * ------------------------------------------------------------------------- */
static int lo_index(double c, double rc, double h)
{
    int i = (int)floor((c - rc) / h) - 1;
    return i < 0 ? 0 : i;
}
static int hi_index(double c, double rc, double h, int n)
{
    int i = (int)ceil((c + rc) / h) + 1;
    return i > n - 1 ? n - 1 : i;
}

/* Counts support nodes per atom into counts[natoms]; returns the total. */
long orc_projector_count(int n0, int n1, int n2, double h, int natoms,
                         const double *R, double rcut, long *counts)
{
    long total = 0;
    double rc2 = rcut * rcut;
    for (int J = 0; J < natoms; ++J) {
        long c = 0;
        int i0 = lo_index(R[3 * J], rcut, h), i1 = hi_index(R[3 * J], rcut, h, n0);
        int j0 = lo_index(R[3 * J + 1], rcut, h), j1 = hi_index(R[3 * J + 1], rcut, h, n1);
        int k0 = lo_index(R[3 * J + 2], rcut, h), k1 = hi_index(R[3 * J + 2], rcut, h, n2);
        for (int k = k0; k <= k1; ++k)
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    double dx = (double)i * h - R[3 * J];
                    double dy = (double)j * h - R[3 * J + 1];
                    double dz = (double)k * h - R[3 * J + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 <= rc2)
                        ++c;
                }
        counts[J] = c;
        total += c;
    }
    return total;
}

/* Fills idx[total] (linear node index) and chi[4*total] ((s, px, py, pz) per node). */
void orc_projector_fill(int n0, int n1, int n2, double h, int natoms,
                        const double *R, double sigma, double rcut,
                        long *idx, double *chi)
{
    const double Y00 = 1.0 / (2.0 * sqrt(M_PI));
    const double Y1 = sqrt(3.0 / (4.0 * M_PI));
    double rc2 = rcut * rcut;
    long e = 0;
    for (int J = 0; J < natoms; ++J) {
        int i0 = lo_index(R[3 * J], rcut, h), i1 = hi_index(R[3 * J], rcut, h, n0);
        int j0 = lo_index(R[3 * J + 1], rcut, h), j1 = hi_index(R[3 * J + 1], rcut, h, n1);
        int k0 = lo_index(R[3 * J + 2], rcut, h), k1 = hi_index(R[3 * J + 2], rcut, h, n2);
        for (int k = k0; k <= k1; ++k)
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    double dx = (double)i * h - R[3 * J];
                    double dy = (double)j * h - R[3 * J + 1];
                    double dz = (double)k * h - R[3 * J + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 <= rc2) {
                        double g = exp(-r2 / (2.0 * sigma * sigma));
                        idx[e] = (long)i + (long)n0 * ((long)j + (long)n1 * (long)k);
                        chi[4 * e + 0] = Y00 * g;
                        chi[4 * e + 1] = Y1 * dx * g;
                        chi[4 * e + 2] = Y1 * dy * g;
                        chi[4 * e + 3] = Y1 * dz * g;
                        ++e;
                    }
                }
    }
}

/* ---------------------------------------------------------------------------
 * The discrete Hamiltonian, Sec. 3.1 (after Eq. non-localPS:FD):
 *   H = -1/2 kscale L_h + diag(V) + V_nl,
 *   V_nl f = h^3 sum_J sum_lm gamma_Jlm chi_Jlm (sum_{support} chi_Jlm f).
 * kscale = 1 is the physical operator; kscale = 0 leaves the diagonal part only
 * (used by the Chebyshev pin on a diagonal H).
 * ------------------------------------------------------------------------- */
typedef struct {
    int n0, n1, n2;
    double h;
    int no;
    double kscale;
    const double *V;        /* Nd */
    int natoms;
    const long *atom_ptr;   /* natoms + 1 offsets into idx / chi */
    const long *idx;
    const double *chi;      /* 4 per support entry */
    const double *gamma;    /* 4 per atom: (s, px, py, pz) */
} orc_ham;

static long ham_nd(const orc_ham *H) { return (long)H->n0 * H->n1 * H->n2; }

/* out = H x for one column (x and out are distinct). */
static void ham_apply_col(const orc_ham *H, const double *x, double *out)
{
    long nd = ham_nd(H);
    orc_laplacian(H->n0, H->n1, H->n2, H->h, H->no, x, out);
    for (long p = 0; p < nd; ++p)
        out[p] = -0.5 * H->kscale * out[p] + H->V[p] * x[p];
    double h3 = H->h * H->h * H->h;
    for (int J = 0; J < H->natoms; ++J) {
        long b = H->atom_ptr[J], e = H->atom_ptr[J + 1];
        for (int lm = 0; lm < 4; ++lm) {
            double c = 0.0;
            for (long s = b; s < e; ++s)
                c += H->chi[4 * s + lm] * x[H->idx[s]];
            double f = h3 * H->gamma[4 * J + lm] * c;
            for (long s = b; s < e; ++s)
                out[H->idx[s]] += f * H->chi[4 * s + lm];
        }
    }
}

/* HX = H X for ncols columns (column-major, leading dimension ld). */
void orc_apply_H(const orc_ham *H, const double *X, double *HX, int ncols, long ld)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < ncols; ++c)
        ham_apply_col(H, X + (long)c * ld, HX + (long)c * ld);
}

/* (H X)(p, col) for npts sampled (node, column) pairs, each computed on its own
 * from the definition (stencil at node p plus every atom whose support holds p). */
void orc_apply_H_at(const orc_ham *H, const double *X, long ld, long npts,
                    const long *pts, const int *cols, double *out)
{
    double w[64];
    orc_lap_weights(H->no, H->h, w);
    double h3 = H->h * H->h * H->h;
    int n0 = H->n0, n1 = H->n1, n2 = H->n2;
#pragma omp parallel for schedule(dynamic)
    for (long q = 0; q < npts; ++q) {
        const double *x = X + (long)cols[q] * ld;
        long p = pts[q];
        int i = (int)(p % n0), j = (int)((p / n0) % n1), k = (int)(p / ((long)n0 * n1));
        double s = 0.0;
        for (int r = 0; r <= H->no; ++r) {
            double t = at(x, n0, n1, n2, i + r, j, k) + at(x, n0, n1, n2, i - r, j, k)
                     + at(x, n0, n1, n2, i, j + r, k) + at(x, n0, n1, n2, i, j - r, k)
                     + at(x, n0, n1, n2, i, j, k + r) + at(x, n0, n1, n2, i, j, k - r);
            s += w[r] * t;
        }
        double v = -0.5 * H->kscale * s + H->V[p] * x[p];
        for (int J = 0; J < H->natoms; ++J) {
            long b = H->atom_ptr[J], e = H->atom_ptr[J + 1];
            long hit = -1;
            for (long t = b; t < e; ++t)
                if (H->idx[t] == p) { hit = t; break; }
            if (hit < 0)
                continue;
            for (int lm = 0; lm < 4; ++lm) {
                double c = 0.0;
                for (long t = b; t < e; ++t)
                    c += H->chi[4 * t + lm] * x[H->idx[t]];
                v += h3 * H->gamma[4 * J + lm] * c * H->chi[4 * hit + lm];
            }
        }
        out[q] = v;
    }
}

/* ---------------------------------------------------------------------------
 * Chebyshev filter, Algorithm ChebychevFilter (Sec. 3.4) with Eq. (ChebFilter):
 *   Psi_f = p_m(H) Psi,  p_m(t) = C_m((t - c)/e),  e = (b - a)/2,  c = (b + a)/2,
 * normalised so that p_m(a0) = 1 (scaled three-term recurrence of the CheFSI
 * method the paper cites, Zhou et al. 2006):
 *   sigma_1 = e / (a0 - c)
 *   Y_1 = (sigma_1 / e) (H - c) Y_0
 *   for j = 2..m:  sigma_j = 1 / (2/sigma_1 - sigma_{j-1})
 *                  Y_j = (2 sigma_j / e)(H - c) Y_{j-1} - sigma_{j-1} sigma_j Y_{j-2}
 * The printed algorithm updates sigma from its own previous value and scales the
 * H term with the old sigma; taken literally the result is not proportional to
 * C_m. The recurrence above is the reading that reproduces p_m(t) exactly.
 * a = lambda_c (cutoff), b = upper bound of the spectrum, a0 = lower end
 * (lambda_1 estimate). X is overwritten by Y_m. m counts applications of H.
 * ------------------------------------------------------------------------- */
static void filter_col(const orc_ham *H, double *x, double *y0, double *y1,
                       double *hy, int m, double a, double b, double a0)
{
    long nd = ham_nd(H);
    double e = (b - a) / 2.0, c = (b + a) / 2.0;
    double sigma1 = e / (a0 - c);
    memcpy(y0, x, sizeof(double) * nd);
    ham_apply_col(H, y0, hy);
    for (long p = 0; p < nd; ++p)
        y1[p] = (sigma1 / e) * (hy[p] - c * y0[p]);
    double sigma = sigma1;
    for (int j = 2; j <= m; ++j) {
        double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
        ham_apply_col(H, y1, hy);
        for (long p = 0; p < nd; ++p) {
            double ynew = (2.0 * sigma_new / e) * (hy[p] - c * y1[p]) - sigma * sigma_new * y0[p];
            y0[p] = y1[p];
            y1[p] = ynew;
        }
        sigma = sigma_new;
    }
    memcpy(x, y1, sizeof(double) * nd);
}

int orc_cheb_filter(const orc_ham *H, double *X, int ncols, long ld,
                    int m, double a, double b, double a0)
{
    if (m < 1 || !(a0 < a) || !(a < b))
        return -1;
    long nd = ham_nd(H);
    int bad = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)nd);
        if (!buf) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(static)
        for (int c = 0; c < ncols; ++c)
            if (buf)
                filter_col(H, X + (long)c * ld, buf, buf + nd, buf + 2 * nd, m, a, b, a0);
        free(buf);
    }
    return bad ? -2 : 0;
}

/* ---------------------------------------------------------------------------
 * Spectral bounds by a few Lanczos steps (Sec. 4, CheFSI parameters).
 * Start vector v0[p] = u(splitmix64(seed ^ p)) - 0.5, u(z) = (z >> 11) * 2^-53,
 * normalised; splitmix64 as published by Vigna (Steele, Lea & Flood's SplitMix,
 * 64-bit variant). Plain Lanczos without reorthogonalisation:
 *   w = H v_j;  alpha_j = <w, v_j>;  w -= alpha_j v_j + beta_{j-1} v_{j-1};
 *   beta_j = ||w||;  v_{j+1} = w / beta_j.
 * Writes alpha[0..k-1], beta[0..k-1] (beta[j] couples steps j and j+1) and
 * returns the number of completed steps (fewer than k if beta hits zero).
 * ------------------------------------------------------------------------- */
static uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_lanczos_start(long nd, uint64_t seed, double *v)
{
    for (long p = 0; p < nd; ++p)
        v[p] = (double)(splitmix64(seed ^ (uint64_t)p) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

int orc_lanczos(const orc_ham *H, int k, uint64_t seed, double *alpha, double *beta)
{
    long nd = ham_nd(H);
    double *v = (double *)malloc(sizeof(double) * nd);
    double *vp = (double *)calloc((size_t)nd, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * nd);
    if (!v || !vp || !w) {
        free(v); free(vp); free(w);
        return -2;
    }
    orc_lanczos_start(nd, seed, v);
    double nrm = 0.0;
    for (long p = 0; p < nd; ++p)
        nrm += v[p] * v[p];
    nrm = sqrt(nrm);
    for (long p = 0; p < nd; ++p)
        v[p] /= nrm;
    double bprev = 0.0;
    int done = 0;
    for (int j = 0; j < k; ++j) {
        ham_apply_col(H, v, w);
        double al = 0.0;
        for (long p = 0; p < nd; ++p)
            al += w[p] * v[p];
        for (long p = 0; p < nd; ++p)
            w[p] = w[p] - al * v[p] - bprev * vp[p];
        double be = 0.0;
        for (long p = 0; p < nd; ++p)
            be += w[p] * w[p];
        be = sqrt(be);
        alpha[j] = al;
        beta[j] = be;
        done = j + 1;
        if (be == 0.0)
            break;
        for (long p = 0; p < nd; ++p) {
            vp[p] = v[p];
            v[p] = w[p] / be;
        }
        bprev = be;
    }
    free(v); free(vp); free(w);
    return done;
}
