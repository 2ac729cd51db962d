/*
 * sparc.h -- C ABI of the GB300 (sm_103a) Chebyshev-filtered subspace iteration
 * library for SPARC's real-space Kohn-Sham Hamiltonian of isolated clusters
 * (Ghosh & Suryanarayana, arXiv:1603.04334).
 *
 * The Hamiltonian (Sec. 3.1, text after Eq. non-localPS:FD) is
 *     H = -1/2 L_h + diag(V_eff) + V_nl,
 * with L_h the order-2n_o central finite-difference Laplacian of Eq. (FD:Laplacian),
 * weights of Eq. (weightsLap), n_o = 6, zero-Dirichlet boundaries, and the
 * Kleinman-Bylander nonlocal operator of Eq. (non-localPS:FD),
 *     V_nl f = h^3 sum_J sum_lm gamma_Jlm chi_Jlm (chi_Jlm^T f).
 *
 * Conventions shared by every call:
 *   - Grid nodes (i, j, k), 0 <= i < n[0], ..., at coordinates (i h, j h, k h); the
 *     linear node index is p = i + n[0] (j + n[1] k) (x fastest). Nd = n0 n1 n2.
 *   - A block of orbitals (Psi in Sec. 3.1) is a column-major Nd x ncols array on the
 *     device: column c starts at element c*ld, ld >= Nd. Blocks are owned by the
 *     caller (for instance PyTorch tensors of shape (ncols, ld)); the library never
 *     frees them. Element type is given by a sparc_dtype argument.
 *   - Every call is enqueued on the stream bound at sparc_create. Calls that return
 *     host values (Ritz values, residuals, bounds) synchronise that stream before
 *     returning; the others are asynchronous.
 *   - Every call returns a status; none aborts, traps or prints. On failure the
 *     message is kept per context (sparc_last_error). Arguments are checked on the
 *     host before any work is enqueued.
 *   - One context per stream; a context must not be used by two threads at once.
 */
#ifndef SPARC_GB300_H
#define SPARC_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sparc_ctx sparc_ctx; /* opaque, owned by the library */

typedef enum {
    SPARC_OK = 0,
    SPARC_ERR_ARG = -1,        /* invalid argument (sizes, pointers, bounds order) */
    SPARC_ERR_OOM = -2,        /* device or pinned-host allocation failed */
    SPARC_ERR_CUDA = -3,       /* a CUDA runtime call or kernel launch failed */
    SPARC_ERR_NOT_SPD = -4,    /* overlap matrix M_s not positive definite (Cholesky) */
    SPARC_ERR_NONFINITE = -5,  /* NaN or Inf met in a projected matrix */
    SPARC_ERR_TIMEOUT = -6,    /* a bounded device-side iteration ran out */
    SPARC_ERR_BUDGET = -7      /* a request exceeds a configured memory budget */
} sparc_status;

typedef enum { SPARC_F64 = 0, SPARC_F32 = 1 } sparc_dtype;

/* Uniform grid of Sec. 3.1: n[d] nodes per axis, spacing h (bohr), stencil radius
 * n_o (`radius`, 1..6; the paper uses 6, Sec. 4). */
typedef struct {
    int n[3];
    double h;
    int radius;
} sparc_grid;

/* Atoms of the cluster. R: 3*natoms positions (bohr), host memory. Z: natoms valence
 * charges (only read when sparc_create builds V_eff itself). gamma: 4*natoms KB
 * coefficients for the projectors (s, px, py, pz) of each atom (Sec. 2). Projector
 * radial form: chi_s = Y00 exp(-r^2/(2 sigma^2)), chi_pd = sqrt(3/4pi) (x_d - R_d)
 * exp(-r^2/(2 sigma^2)), truncated to nodes with r^2 <= rcut^2. rc_erf is the width
 * of the synthetic local potential -Z erf(r/rc_erf)/r. natoms may be 0. */
typedef struct {
    int natoms;
    const double *R;
    const double *Z;
    const double *gamma;
    double sigma;
    double rcut;
    double rc_erf;
} sparc_atoms;

/* Creates a context: copies V_eff (or builds it on the device when veff_host is
 * NULL, from V_eff(x) = sum_J -Z_J erf(|x-R_J|/rc_erf)/|x-R_J|), builds the projector
 * support tables on the device (Sec. 3.2's per-atom influence boxes, restricted to
 * the sphere r <= rcut), and binds `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream). veff_host: Nd doubles, x fastest, host memory. */
sparc_status sparc_create(const sparc_grid *grid, const double *veff_host,
                          const sparc_atoms *atoms, void *cuda_stream, sparc_ctx **out);

/* Frees everything the context owns. NULL is accepted. */
sparc_status sparc_destroy(sparc_ctx *ctx);

/* Last error message of the context ("" if none); valid until the next call. */
const char *sparc_last_error(const sparc_ctx *ctx);

/* Copies the context's V_eff (Nd doubles) to host memory; synchronises. */
sparc_status sparc_get_veff(sparc_ctx *ctx, double *veff_host);

/* Number of nodes and of projector support entries (sum over atoms). */
sparc_status sparc_info(const sparc_ctx *ctx, long *nd, long *nsupport, int *natoms);

/* Scales the kinetic term: H = -1/2 kscale L_h + V_eff + V_nl (default 1). kscale = 0
 * gives a diagonal-plus-nonlocal operator, used to check the filter against scalar
 * Chebyshev values. */
sparc_status sparc_set_kinetic_scale(sparc_ctx *ctx, double kscale);

/* HX = H X, Sec. 3.1. X, HX: distinct device blocks of `dtype` (F64 or F32, the
 * arithmetic follows the storage type), ncols columns, leading dimension ld. */
sparc_status sparc_apply_H(sparc_ctx *ctx, sparc_dtype dtype, const void *X, void *HX,
                           int ncols, long ld);

/* Spectral bounds by k Lanczos steps (Sec. 4: extremal eigenvalues of H from "a few
 * iterations of the Lanczos method"), all on the device in FP64. Start vector
 * v0[p] = u(splitmix64(seed ^ p)) - 0.5, u(z) = (z >> 11) 2^-53, normalised; no
 * reorthogonalisation. Returns lo = theta_min(T_k) and
 * hi = max(1.01 theta_max, theta_max + |beta_k s_k|) (s_k: last component of the
 * unit eigenvector of theta_max). 1 <= k <= 64. Synchronises. */
sparc_status sparc_lanczos_bounds(sparc_ctx *ctx, int ksteps, unsigned long long seed,
                                  double *lo, double *hi);

/* Filter interval of the first CheFSI iteration (Sec. 4: the bounds of the spectrum from
 * a few Lanczos steps, and a cutoff lambda_c below which the filter passes the spectrum).
 * Runs sparc_lanczos_bounds(ctx, ksteps, seed, &lo, &hi) and writes
 *     bounds_out[3] = [a, b, a0] = [lo + (hi - lo) / 4, hi, lo]   (host memory),
 * the bounds_inout argument of the first sparc_chefsi_step. The paper's cutoff is
 * lambda_c = E_F + 0.1 Ha, which a fixed Hamiltonian without electrons does not have; the
 * quarter point is this library's choice. Later iterations take a and a0 from the Ritz
 * values (sparc_chefsi_step updates bounds_inout). Errors: those of sparc_lanczos_bounds;
 * SPARC_ERR_ARG for a NULL bounds_out or when lo == hi (no interval). Synchronises. */
sparc_status sparc_first_bounds(sparc_ctx *ctx, int ksteps, unsigned long long seed,
                                double *bounds_out);

/* Chebyshev filter, Algorithm ChebychevFilter with Eq. (ChebFilter), Sec. 3.4:
 * X <- p_m(H) X with p_m(t) = C_m((t - c)/e) / C_m((a0 - c)/e), e = (b - a)/2,
 * c = (b + a)/2, m = degree (number of applications of H), using the scaled
 * three-term recurrence of the CheFSI method the paper cites:
 *   sigma_1 = e/(a0 - c); Y_1 = (sigma_1/e)(H - c)X;
 *   sigma_j = 1/(2/sigma_1 - sigma_{j-1}),
 *   Y_j = (2 sigma_j/e)(H - c) Y_{j-1} - sigma_{j-1} sigma_j Y_{j-2}.
 * a = cutoff lambda_c, b = upper bound of the spectrum, a0 = lower end (lambda_1
 * estimate); requires a0 < a < b, degree >= 1. work: a second device block with the
 * same dtype, ncols and ld, overwritten. FP64 or FP32 arithmetic per dtype. */
sparc_status sparc_cheb_filter(sparc_ctx *ctx, sparc_dtype dtype, void *X, void *work,
                               int ncols, long ld, int degree, double a, double b,
                               double a0);

/* Projection, generalized eigenproblem and rotation, Sec. 3.4 (Eq.
 * SubspaceGeneralizedEigenproblem and Eq. OrbitalTransformation), in FP64 on the
 * device: M_s = Xf^T Xf, H_s = Xf^T (H Xf), M_s = L L^T (Cholesky),
 * Q^T (L^-1 H_s L^-T) Q = diag(ritz) (cyclic Jacobi), Xf <- Xf (L^-T Q).
 * Each column of Q is signed so that its largest-magnitude entry is positive.
 * On return Xf holds Euclidean-orthonormal Ritz vectors (ascending Ritz values),
 * ritz_host[ncols] the Ritz values, and resid_host[ncols] (if not NULL) the residual
 * norms ||H x_n - ritz_n x_n||_2. M_s and H_s are formed on the tensor cores from the
 * operands' 47-bit digits (each entry rounded to 2^-48 of the largest in its 128-row chunk,
 * the digit products summed exactly): FP64-level for both dtypes. For dtype F32 the block
 * stays FP32, H Xf is applied in FP64 and M_s, H_s and the eigensolve are FP64; the rotation
 * and the rotated H X of the residuals run on the tensor cores in the 23-bit digit form with
 * FP32 results (the block's own precision; residuals good to about 1e-7 of ||H x_n||).
 * HXf_or_null: optional FP64 device
 * block (ncols x ld) used as the H Xf workspace; when NULL the context allocates one.
 * Fails with SPARC_ERR_NOT_SPD if M_s is not numerically positive definite and with
 * SPARC_ERR_NONFINITE on NaN/Inf, leaving Xf unrotated. ncols <= 1024. Synchronises. */
sparc_status sparc_orth_rr(sparc_ctx *ctx, sparc_dtype dtype, void *Xf, void *HXf_or_null,
                           int ncols, long ld, double *ritz_host, double *resid_host);

/* Projection contraction of Sec. 3.4 (the relations after Eq.
 * SubspaceGeneralizedEigenproblem): G = A^T B over the context's Nd rows, e.g.
 * M_s = Psi_f^T Psi_f or H_s = Psi_f^T (H Psi_f). A, B: device blocks (ncols columns,
 * leading dimension ld) of types (dtype_a, dtype_b) = (F64, F64), (F32, F32) or
 * (F32, F64); products and sums are FP64. G: device, ncols x ncols, column-major FP64,
 * overwritten. The row slices are summed in a fixed order, so repeated calls are
 * bitwise identical. Uses context workspace (allocated on first use or growth).
 * Asynchronous on the context stream. */
sparc_status sparc_gram(sparc_ctx *ctx, sparc_dtype dtype_a, const void *A, sparc_dtype dtype_b,
                        const void *B, int ncols, long ld, double *G);

/* The same contraction on the tensor cores, as the mixed-precision form uses it for M_s
 * and H_s (Sec. 3.4 with the FP32 filter). Each operand is rounded, per 256-row chunk and
 * column, to 23 bits of that chunk's largest magnitude (three 8-bit digits in BF16), the
 * digit products are summed exactly on the tensor cores (tcgen05), and the chunks are
 * combined in FP32-pair arithmetic. Error bound per entry: |dG_ij| <= 2^-21 sum_k
 * (m_i(k) m_j(k) + m_i(k) |B_kj| + |A_ki| m_j(k)), m_i(k) the largest |A_.i| of row k's
 * chunk (m_j likewise for B) -- the rounding an FP32 block already carries, with no
 * growth along Nd; sparc_gram is exact for FP32 data. Types (F32, F32), (F32, F64) or
 * (F64, F64); a chunk column holding Inf or NaN makes the affected entries NaN. G: device,
 * ncols x ncols, column-major FP64, overwritten; bitwise repeatable. Uses context
 * workspace of about 6 x ncols x Nd bytes per distinct operand (allocated on first use or
 * growth). Asynchronous; a bounded internal wait that expires is reported as
 * SPARC_ERR_TIMEOUT by the next synchronising call. The paper's contractions are FP64
 * throughout; this is the GB300 form of them. */
sparc_status sparc_gram_tc(sparc_ctx *ctx, sparc_dtype dtype_a, const void *A,
                           sparc_dtype dtype_b, const void *B, int ncols, long ld, double *G);

/* One CheFSI iteration, Sec. 3.4: sparc_cheb_filter with bounds_inout = [a, b, a0],
 * then sparc_orth_rr. Afterwards bounds_inout is updated for the next iteration:
 * a = largest Ritz value, a0 = smallest Ritz value, b unchanged. work as in
 * sparc_cheb_filter. Synchronises. */
sparc_status sparc_chefsi_step(sparc_ctx *ctx, sparc_dtype dtype, void *X, void *work,
                               int ncols, long ld, int degree, double *bounds_inout,
                               double *ritz_host, double *resid_host);

/* ---- after the rotation: occupations, density, non-local force ------------------- */

/* Occupations and Fermi level, Eq. (FermiEnergyConstraintFormulation), Sec. 3.4:
 * lambda_f is the root of 2 sum_n g_n = N_e with g_n = 1 / (1 + exp((lambda_n -
 * lambda_f) / kT)) (the paper uses kT = 1e-3 Ha, Sec. 5). lambda_host: ns eigenvalues
 * (host, any order); nelec in (0, 2 ns); kT > 0. Writes *lambda_f_host and, unless
 * g_host is NULL, g_host[ns] (host). The root is found on the device (one CTA: Newton
 * steps safeguarded by bisection; the paper uses Brent's method, Sec. 4). Where all
 * levels sit more than ~37 kT from the root, the occupations round to 0 and 1 and every
 * point of that gap is a root in double precision: g is then exact, lambda_f any point
 * of it. Synchronises. Errors: SPARC_ERR_ARG (NULL pointers, ns <= 0, nelec or kT out of
 * range), SPARC_ERR_NONFINITE (an eigenvalue is NaN or Inf; outputs unset),
 * SPARC_ERR_TIMEOUT (no convergence in 200 steps). */
sparc_status sparc_occupations(sparc_ctx *ctx, const double *lambda_host, int ns, double nelec,
                               double kT, double *lambda_f_host, double *g_host);

/* Electron density, Sec. 3.4 (the equation after Eq. OrbitalTransformation):
 * rho[p] = (2 / h^3) sum_n g_n x_n[p]^2 over the ncols columns x_n of X (Euclidean-
 * normalised orbitals, as sparc_orth_rr returns them; F64 or F32 block, accumulated in
 * FP64). g_host: ncols occupations (host, copied before the call returns); rho: Nd
 * doubles of caller-owned device memory, x fastest. Asynchronous. Errors: SPARC_ERR_ARG. */
sparc_status sparc_density(sparc_ctx *ctx, sparc_dtype dtype, const void *X, int ncols, long ld,
                           const double *g_host, double *rho);

/* Non-local atomic force, Eq. (NonlocForce:Discrete) with Y and W of Eq. (NonLocForce:U:W),
 * Algorithm non-localForceCalculation:
 *     f_J = -4 sum_n g_n sum_lm gamma_Jl Y_Jnlm W_Jnlm,
 *     Y_Jnlm = h^3 sum psi_n chi_Jlm,  W_Jnlm = h^3 sum (grad_h psi_n) chi_Jlm,
 * over the projector support of atom J, grad_h the order-2n_o finite-difference gradient
 * of Eq. (gradient:approximate) with zero-Dirichlet values. psi_n = x_n / h^(3/2), x_n the
 * Euclidean-normalised columns of X: with that normalisation f_J is minus the derivative
 * of E_nl = 2 sum_n g_n x_n^T V_nl x_n in R_J (the paper's density formula uses x_n
 * itself). X: F64 or F32 block; g_host: ncols occupations (host); force_host: 3 natoms
 * doubles (x, y, z per atom; untouched when the cluster has no atoms). FP64 arithmetic.
 * Synchronises. Errors: SPARC_ERR_ARG. */
sparc_status sparc_nonlocal_force(sparc_ctx *ctx, sparc_dtype dtype, const void *X, int ncols,
                                  long ld, const double *g_host, double *force_host);

/* Electrostatic potential, Sec. 3.3: phi solves -(1/4 pi) L_h phi = rho + b - d (Eq.
 * FD:PoissonDiscrete) with zero Dirichlet values, where
 *   b = -(1/4 pi) L_h sum_J V_J (Eq. PseudochargeDiscrete, Algorithm
 *       PseudochargeCalculation), V_J = -Z_J erf(|x - R_J| / rc_erf) / |x - R_J| the atoms'
 *       local potential, evaluated at the grid nodes and at the n_o nodes beyond each
 *       face; it integrates to -Z_J (the sign of the attractive V_J);
 *   d = the charge correction of Eq. (Phi:correction) from the multipole boundary values
 *       of Eq. (phi:BC:discrete), l_max = 6 (Sec. 4), |x| measured from the box centre
 *       ((n_d - 1) h / 2 per axis).
 * Conjugate gradients with a Jacobi preconditioner (the paper's block-Jacobi on one block
 * per processor; here the diagonal) from phi = 0, until ||r|| <= tol ||rhs||.
 * rho: Nd doubles (device, x fastest) or NULL for rho = 0; phi: Nd doubles (device,
 * caller-owned) for the result; b_out: Nd doubles (device) for b, or NULL. Writes the
 * iteration count and the final relative residual to *iters_host / *relres_host (each may
 * be NULL). Needs the atoms' charges Z at sparc_create. Synchronises. Errors:
 * SPARC_ERR_ARG (NULL phi, tol outside (0, 1), maxit <= 0, no Z), SPARC_ERR_TIMEOUT (the
 * tolerance not reached in maxit iterations; phi holds the last iterate). */
sparc_status sparc_poisson(sparc_ctx *ctx, const double *rho, double *phi, double tol, int maxit,
                           double *b_out, int *iters_host, double *relres_host);

/* ---- instrumentation ------------------------------------------------------------ */

/* Phases timed by the context's profiler. */
typedef enum {
    SPARC_PHASE_STENCIL = 0, /* fused stencil + V_eff + recurrence (H X, filter steps) */
    SPARC_PHASE_PROJECT = 1, /* nonlocal projections chi^T Y */
    SPARC_PHASE_SCATTER = 2, /* nonlocal scatter-add */
    SPARC_PHASE_GRAM = 3,    /* M_s and H_s contractions */
    SPARC_PHASE_DENSE = 4,   /* Cholesky, Jacobi eigensolve, back-transform */
    SPARC_PHASE_ROTATE = 5,  /* subspace rotation (and rotated H X for residuals) */
    SPARC_PHASE_OTHER = 6,   /* Lanczos vector kernels, residual norms, copies */
    SPARC_NPHASES = 7
} sparc_phase;

/* Enables (1) or disables (0) per-phase timing: each phase's launches are bracketed by
 * CUDA events recorded on the context stream. Disabling discards pending events. */
sparc_status sparc_profile_enable(sparc_ctx *ctx, int enable);

/* Accumulated launches and device milliseconds of `phase` since the last reset;
 * synchronises the context stream. */
sparc_status sparc_profile_read(sparc_ctx *ctx, int phase, long long *launches, double *ms);

/* Clears the accumulated profile. */
sparc_status sparc_profile_reset(sparc_ctx *ctx);

/* Number of kernels this library has launched in the calling process (all contexts). */
sparc_status sparc_launch_count(long long *count);

/* Upper bound of the device memory the context has held at any time (bytes it allocated,
 * its set-up temporaries counted as if never freed). */
sparc_status sparc_device_bytes(const sparc_ctx *ctx, size_t *peak_bytes);

/* ---- synchronisation and failure detection ------------------------------------------ */

/* Waits for all work enqueued on the context's stream and reports device-side errors
 * that asynchronous calls cannot return. Every wait inside a kernel of this library is
 * bounded; a kernel whose wait expires (a TMA load that never lands) stops, leaves no copy
 * in flight, and raises a sticky device flag. sparc_apply_H and sparc_cheb_filter return
 * before their kernels run, so such a flag is reported by the next synchronising call
 * (this one, sparc_lanczos_bounds, sparc_orth_rr or sparc_chefsi_step) as
 * SPARC_ERR_TIMEOUT, and cleared. The paper has no counterpart. */
sparc_status sparc_sync(sparc_ctx *ctx);

/* Self-test of the bounded waits, for failure-detection tests without a GPU fault.
 * which = 0: an mbarrier that expects two arrivals and receives one (the wait of the TMA
 * stencil pipeline); which = 1: a cooperative two-CTA grid barrier that expects three CTAs
 * (the barrier of the multi-SM Jacobi solver). Neither wait can complete; each gives up
 * after its poll limit (2^20 polls, well under a second). Returns SPARC_ERR_TIMEOUT when the kernel detected the expired wait
 * and reported it through the host (the expected result), SPARC_OK if the wait completed
 * (a defect), SPARC_ERR_ARG for another `which`. The context stays usable afterwards.
 * The paper has no counterpart. */
sparc_status sparc_selftest_timeout(sparc_ctx *ctx, int which);

/* ---- allocation-free variant ---------------------------------------------------- */

/* G = A^T B in FP64 without allocating any memory. The paper has no counterpart: this is a
 * service for callers that cannot let the library call cudaMalloc where they call it --
 * real-time loops that forbid allocation after start-up (an allocation can block and
 * synchronise the device), hosts that carve all device memory out of their own pool, or
 * processes that have already reserved nearly all of it. Same result as sparc_gram for FP64
 * inputs, up to the order of the row-slice sums. A, B: device, nd rows x ncols columns,
 * column-major, leading dimension ld >= nd. G: device, ncols x ncols, column-major,
 * overwritten. Enqueued on `cuda_stream` (a cudaStream_t; NULL = legacy default stream);
 * needs no context. The row-slice partial sums live in a fixed 16 MiB __device__ array that
 * every GPU loading the library keeps until exit: ncols^2 must not exceed 2^21 (any
 * ncols <= 1024 fits), else SPARC_ERR_ARG. The first call on a device looks up that array's
 * address (cudaGetSymbolAddress) with the device current and keeps it for the life of the
 * process; make that first call before any stream capture begins. The kept address belongs
 * to the device's primary context: a process that resets the device (cudaDeviceReset) must
 * not call this entry point on it afterwards. All calls share the array: calls that overlap
 * on the GPU race on it and must be serialised. Each call overwrites every partial it reads,
 * so no clearing is needed. Returns SPARC_ERR_ARG for NULL pointers or bad sizes,
 * SPARC_ERR_CUDA if the lookup or the launch fails. */
sparc_status sparc_gram_noalloc(const double *A, const double *B, long nd, int ncols, long ld,
                                double *G, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SPARC_GB300_H */
