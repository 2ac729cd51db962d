// internal.cuh -- declarations shared by the CUDA translation units of libsparc_gb300.
// Not part of the public ABI (include/sparc.h is).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

struct sparc_ctx;  // include/sparc.h

namespace sparc {

constexpr int kRadius = 6;  // stencil radius the kernels are written for (n_o <= 6)

// Counts kernel launches made by this library (process-wide, read by sparc_launch_count).
void note_launch(int n = 1);
// [a, b, a0] of the first CheFSI iteration from the Lanczos bounds (sparc.cu)
void first_iteration_bounds(double lo, double hi, double *bounds);

// Device copy of the discrete Hamiltonian (Sec. 3.1) and of its projector tables.
struct DevHam {
    int n0 = 0, n1 = 0, n2 = 0;
    long nd = 0;
    double h = 0;
    int radius = 6;
    double kscale = 1.0;
    double w[kRadius + 1] = {0};  // Laplacian weights w_p (1/h^2 included), zero beyond radius
    // the same weights as exact integers over one denominator D: 6 h^2 w_0 = wint[0] / D,
    // h^2 w_p = wint[p] / D (p >= 1); wunit = 1 / (D h^2)
    int wint[kRadius + 1] = {0};
    double wunit = 0;
    int *err = nullptr;           // device word set by a kernel whose bounded wait ran out

    const double *V = nullptr;   // V_eff, Nd
    const float *Vf = nullptr;   // V_eff rounded to float (FP32 filter)

    int natoms = 0;
    long nsup = 0;                   // support entries over all atoms
    const int *atom_ptr = nullptr;   // natoms+1 offsets into the entry arrays
    const int *idx = nullptr;        // node index of each entry
    const double *chi = nullptr;     // 4 per entry: chi_s, chi_px, chi_py, chi_pz
    const float *chi_f = nullptr;
    // chi on a 46-bit grid per (atom, l) for the integer projection: per entry (a_0..a_3),
    // (b_0..b_3) with chi_l = 2^(F-46) (a_l 2^23 + b_l); chi_F: F per (atom, l)
    const int4 *chi_q = nullptr;
    const int *chi_F = nullptr;
    const int *proj_order = nullptr; // natoms: the projections' atom order (spatial)
    const double *gchi = nullptr;    // 4 per entry: h^3 gamma_Jlm chi_Jlm
    const float *gchi_f = nullptr;
    const int *ent_atom = nullptr;   // atom of each entry

    long nuniq = 0;                  // nodes covered by at least one support
    const int *uniq_node = nullptr;  // ascending node indices
    const int *uniq_ptr = nullptr;   // nuniq+1 offsets into ent_list
    const int *ent_list = nullptr;   // entries of each node, ascending entry id

    // node-ordered copies of the entry data read by the scatter kernels
    const int *nl_atom = nullptr;    // per ent_list position: atom
    const float *nl_gf = nullptr;    // per ent_list position: 4 x h^3 gamma chi (FP32)
    const float2 *nl_gdf = nullptr;  // same as FP32 pairs
};

// Coefficients of one fused step  out = alpha*((-1/2 ks L_h + V - c) Y + V_nl Y) - beta*Yprev.
// w[r] = alpha * (-1/2) * ks * w_r (r >= 1); c0 = alpha * (-1/2) * ks * 6 w_0 - alpha * c.
template <typename TC>
struct StepCoef {
    TC w[kRadius + 1];
    TC c0;
    TC alpha;
    TC beta;
};

StepCoef<double> make_coef(const DevHam &H, double alpha, double shift, double beta);

// ---- stencil.cu / stencil_df.cu ----------------------------------------------------
// out = alpha*((-1/2 ks L_h + V - shift) Y + V_nl Y) - beta*Yprev   (one fused step).
// Yprev may be null (beta ignored) and may alias out (in-place recurrence). Cs: the
// projection coefficients alpha * chi^T Y (FP32 pairs for FP64 blocks, FP32 for FP32
// blocks), or null when the Hamiltonian has no atoms.
// FP64 blocks (stencil_df.cu): the neighbour sums are exact integer sums of the values
// scaled by a power of two per column, so each column needs a bound of its magnitude:
// bY[c] = the largest high word (bits 32..62) of |y| over the column, as written by
// colmax_f64 or by the launch that produced the block. bOut, if not null, is raised
// (atomicMax) to the bound of the output's columns. u: alpha (V_eff - shift), Nd values
// (from scaled_v; H.V itself when alpha = 1 and shift = 0).
cudaError_t stencil_f64(const DevHam &H, const double *Y, const double *Yprev, double *out,
                        int ncols, long ld, double alpha, const double *u, double beta,
                        const unsigned *bY, unsigned *bOut, cudaStream_t st);
cudaError_t scaled_v(const double *V, double alpha, double shift, double *u, long n,
                     cudaStream_t st);
// out += V_nl part from Cs = alpha chi^T Y (pairs), for FP64 outputs (nonlocal.cu); bOut
// as for stencil_f64 (raised to the bound of the updated values), or null
cudaError_t scatter_f64_df(const DevHam &H, const float2 *Cs, double *out, int ncols, long ld,
                           unsigned *bOut, cudaStream_t st);
// b[c] = max(b[c], largest high word of |Y| over column c) for FP64 or FP32 blocks (an FP32
// value counts as its FP64 widening); b must be zeroed first to get the bound alone.
cudaError_t colmax_f64(const double *Y, int ncols, long ld, long nd, unsigned *b,
                       cudaStream_t st);
cudaError_t colmax_f32(const float *Y, int ncols, long ld, long nd, unsigned *b,
                       cudaStream_t st);
// out += V_nl part from Cs = alpha chi^T Y, FP32 blocks (nonlocal.cu)
cudaError_t scatter_f32(const DevHam &H, const float *Cs, float *out, int ncols, long ld,
                        cudaStream_t st);
// ---- batched FP32 filter steps over many clusters (batch.cu) --------------------------
// One unit of work of a batched launch. stencil: column `col`, tile (a, b) of the x-y
// plane, planes k0 .. k1-1; projection: atom a, columns col .. col+15; scatter: covered
// nodes a*256 .. a*256+255, columns col .. col+15.
struct BatchItem {
    int cluster, col, a, b, k0, k1;
};
// Per cluster and step: where the stencil reads and writes, and its coefficients.
struct BatchStencil {
    const float *Y;
    const float *Yprev;  // null in the first filter step
    float *out;
    const float *V;
    int n0, n1, n2;
    long ld;
    StepCoef<float> cf;
};
// Per cluster and step: the nonlocal term's tables, input, output and coefficient buffer.
struct BatchNonlocal {
    const float *Y;
    float *out;
    float *C;  // alpha chi^T Y, [atom][column][4]
    const int *atom_ptr, *idx, *uniq_node, *uniq_ptr, *nl_atom;
    const float *chi_f, *nl_gf;
    long ld, nuniq;
    int ncols;
    float alpha;
};
// Per cluster and step for the TMA-fed batched stencil: device addresses of the tensor maps
// of Y_j (halo box) and Y_{j-1} (tile box; null in the first step), and the rest as above.
struct BatchTma {
    const void *mY;
    const void *mP;
    float *out;
    const float *V;
    int n0, n1, n2;
    long ld;
    StepCoef<float> cf;
};
cudaError_t encode_f32_maps(const DevHam &H, const float *base, int ncols, long ld, void *maps);
size_t tensor_map_bytes();
void batch_tma_tile(int &bx, int &by);
cudaError_t batch_stencil_tma(const BatchItem *items, int nitems, const BatchTma *cs, int grid,
                              int *err, cudaStream_t st);
int batch_stencil_shapes();
void batch_stencil_tile(int shape, int &bx, int &by);
cudaError_t batch_stencil(int shape, const BatchItem *items, int nitems, const BatchStencil *cs,
                          int grid, cudaStream_t st);
cudaError_t batch_project(const BatchItem *items, int nitems, const BatchNonlocal *cs, int grid,
                          cudaStream_t st);
cudaError_t batch_scatter(const BatchItem *items, int nitems, const BatchNonlocal *cs, int grid,
                          cudaStream_t st);
StepCoef<float> coef_f32(const DevHam &H, double alpha, double shift, double beta);
// context accessors for the batch layer (sparc.cu)
const DevHam *ctx_ham(const sparc_ctx *ctx);
cudaStream_t ctx_stream(const sparc_ctx *ctx);
float *ctx_coef_buffer(sparc_ctx *ctx, int ncols);  // grows the context's C buffer
constexpr int kBatchCols = 16;     // columns per nonlocal work item
constexpr int kBatchNodes = 256;   // covered nodes per scatter work item

cudaError_t stencil_f32(const DevHam &H, const float *Y, const float *Yprev, float *out,
                        int ncols, long ld, double alpha, double shift, double beta,
                        cudaStream_t st);
void stencil_z_split(int n2, long tiles, int ncols, int &nzc, int &zchunk);
// stencil_tma.cu: TMA-fed FP32 step for shapes with n0, ld multiples of 4 and 16-byte
// aligned blocks (stencil_tma_ok); stencil_f32 picks it when it applies.
bool stencil_tma_ok(const DevHam &H, const void *Y, const void *Yprev, const void *out, long ld);
cudaError_t stencil_f32_tma(const DevHam &H, const float *Y, const float *Yprev, float *out,
                            int ncols, long ld, const StepCoef<float> &cf, int *err,
                            cudaStream_t st);
// FP64 arithmetic on an FP32 block (H applied to FP32 Ritz blocks in FP64).
cudaError_t stencil_f32in_f64(const DevHam &H, const float *Y, double *out, int ncols,
                              long ld, const unsigned *bY, cudaStream_t st);

// ---- nonlocal.cu ------------------------------------------------------------------
// C[(J*4+lm)*ncols + c] = alpha * sum_{s in supp(J)} chi_Jlm(s) Y[idx(s) + c*ld]
// (FP64 blocks: exact integer sums on the columns' grids (bY: the column bounds of Y),
// output as FP32 pairs; FP32 blocks: FP32)
cudaError_t project_f64_fx(const DevHam &H, const double *Y, int ncols, long ld, double alpha,
                           const unsigned *bY, float2 *C, cudaStream_t st);
cudaError_t project_f32(const DevHam &H, const float *Y, int ncols, long ld, double alpha,
                        float *C, cudaStream_t st);
// the FP64 projection of an FP32 block (pairs, alpha = 1), for the pair scatter
cudaError_t project_f32in_f64(const DevHam &H, const float *Y, int ncols, long ld,
                              const unsigned *bY, float2 *C, cudaStream_t st);
// the integer grid of chi (DevHam::chi_q, chi_F) from chi
cudaError_t chi_fixed(int natoms, const int *atom_ptr, const double *chi, int4 *chi_q,
                      int *chi_F, cudaStream_t st);
// node-ordered entry tables of the scatter kernels
cudaError_t build_nl_node_tables(long nuniq, const int *uniq_ptr, const int *ent_list,
                                 const int *ent_atom, const double *gchi, int *nl_atom,
                                 float *nl_gf, float2 *nl_gdf, cudaStream_t st);

// ---- setup.cu -------------------------------------------------------------------
// V_eff(x) = sum_J -Z_J erf(r/rc)/r on the device.
cudaError_t build_veff(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                       const double *Z_dev, double rc, double *V, cudaStream_t st);
// Support counts per atom (r^2 <= rcut^2 within the grid).
cudaError_t support_count(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                          double rcut, int *counts, cudaStream_t st);
// Fills idx/chi (entries atom by atom, ascending node index), ent_atom, gchi (+ float copies).
cudaError_t support_fill(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                         const double *gamma_dev, double sigma, double rcut,
                         const int *atom_ptr, int *idx, double *chi, float *chi_f,
                         double *gchi, float *gchi_f, int *ent_atom, cudaStream_t st);
// Inverse map node -> entries. Scratch buffers sized by the caller (see sparc.cu).
cudaError_t build_inverse_map(long nd, long nsup, const int *idx, int *node_cnt,
                              int *node_start, int *cursor, int *ent_list, int *flags,
                              int *uniq_rank, int *scan_tmp, int *uniq_node, int *uniq_ptr,
                              cudaStream_t st);
cudaError_t exclusive_scan_int(const int *in, int *out, long n, int *tmp, cudaStream_t st);
cudaError_t to_float(const double *in, float *out, long n, cudaStream_t st);

// ---- gram.cu --------------------------------------------------------------------
// G (ns x ns, column-major, FP64) = A^T B over nd rows; A, B column-major with lda/ldb.
// part: workspace of gram_part_elems(ns, nd) doubles.
// sym: A^T B is known to be symmetric (M_s, H_s); only tiles i0 <= j0 are computed.
long gram_part_elems(int ns, long nd);
cudaError_t gram_f64(const double *A, long lda, const double *B, long ldb, long nd, int ns,
                     double *G, double *part, cudaStream_t st, bool sym = false);
cudaError_t gram_f32_f32(const float *A, long lda, const float *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st, bool sym = false);
cudaError_t gram_f32_f64(const float *A, long lda, const double *B, long ldb, long nd, int ns,
                         double *G, double *part, cudaStream_t st, bool sym = false);
// gram_df.cu: FP32-pair kernels behind the entry points above and below.
template <typename TA, typename TB>
cudaError_t gram_df_launch(const TA *A, long lda, const TB *B, long ldb, long nd, int ns,
                           double *G, double *part, int nsplit, bool sym, cudaStream_t st);
cudaError_t rotate_f64_df(const double *A, long lda, long nd, int ns, const double *Q, double *out,
                          long ldo, cudaStream_t st);
// FP64 Gram with a caller-chosen number of row slices (part: nsplit * ns * ns doubles).
int gram_default_splits(int ns, long nd);
// Tensor-core Gram of the mixed-precision form (gram_tc.cu): G = A^T B (ns x ns FP64,
// column-major) from operands rounded to 23 bits of each 256-row chunk's largest entry,
// accumulated exactly on the tensor cores; sym computes the tiles on and above the
// diagonal and mirrors them. ws: at least gram_tc_workspace(nd, ns, A == B, sym) bytes,
// 256-byte aligned. A bounded wait that expires sets *err.
size_t gram_tc_workspace(long nd, int ns, bool same_operand, bool sym);
// The same contractions for FP64 blocks in the 47-bit form (six digits per entry, classes
// 0..5): M = A^T A and Hm = A^T B, both symmetric; ws: gram_tc47_workspace(nd, ns) bytes.
size_t gram_tc47_workspace(long nd, int ns);
// out = Y C (C: ns x ns FP64, column-major) on the tensor cores in the 47-bit digit form;
// ws: rotate_tc_workspace(nd, ns) bytes.
size_t rotate_tc_workspace(long nd, int ns);
// The same in the 23-bit digit form with FP32 output (the mixed-precision form: Y its FP32
// block, or the FP64 H Y of its residuals); ws: rotate_tc23_workspace(nd, ns) bytes.
size_t rotate_tc23_workspace(long nd, int ns);
// Rows per slab of the tensor-core Gram (47-bit digits in both forms) and rotation (47-bit
// digits in the FP64 form, 23-bit in the mixed form): the whole block when the digit
// workspace stays within 24 GB, else the largest multiple of 256 rows, halving from nd,
// that does. Larger blocks are processed slab by slab: the Grams of the slabs are summed
// (slabs start on 128-row chunk boundaries, so every slab's digits are those the
// whole-block call would form) and the rotation's rows are independent.
inline long tc_slab_rows(long nd, int ns, bool mixed)
{
    const size_t cap = (size_t)24 << 30;
    auto rot = [&](long r) { return mixed ? rotate_tc23_workspace(r, ns) : rotate_tc_workspace(r, ns); };
    long rows = nd;
    while (rows > 256 && (gram_tc47_workspace(rows, ns) > cap || rot(rows) > cap))
        rows = (rows / 2 + 255) / 256 * 256;
    return rows;
}
// Bytes of the tensor-core workspace one slab of tc_slab_rows(nd, ns, mixed) rows needs.
inline size_t tc_slab_workspace(long nd, int ns, bool mixed)
{
    const long slab = tc_slab_rows(nd, ns, mixed);
    const size_t wg = gram_tc47_workspace(slab, ns);
    const size_t wr = mixed ? rotate_tc23_workspace(slab, ns) : rotate_tc_workspace(slab, ns);
    return wg > wr ? wg : wr;
}
// dst[i] += src[i], i < n
cudaError_t add_into(double *dst, const double *src, long n, cudaStream_t st);
cudaError_t rotate_tc(const double *Y, long ldy, long nd, int ns, const double *C, double *out,
                      long ldo, void *ws, size_t ws_bytes, int *err, cudaStream_t st);
template <typename TY>
cudaError_t rotate_tc23(const TY *Y, long ldy, long nd, int ns, const double *C, float *out,
                        long ldo, void *ws, size_t ws_bytes, int *err, cudaStream_t st);
// M = A^T A and Hm = A^T B in the 47-bit digit form (A FP64 or FP32, B FP64).
template <typename TA>
cudaError_t gram_tc47_pair(const TA *A, long lda, const double *B, long ldb, long nd, int ns,
                           double *M, double *Hm, void *ws, size_t ws_bytes, int *err,
                           cudaStream_t st);
template <typename TA, typename TB>
cudaError_t gram_tc(const TA *A, long lda, const TB *B, long ldb, long nd, int ns, double *G,
                    void *ws, size_t ws_bytes, bool sym, int *err, cudaStream_t st);
cudaError_t gram_f64_nsplit(const double *A, long lda, const double *B, long ldb, long nd, int ns,
                            double *G, double *part, int nsplit, cudaStream_t st);
// out (nd x ns, ldo) = A (nd x ns, lda) Q (ns x ns, column-major FP64)
cudaError_t rotate_f64(const double *A, long lda, long nd, int ns, const double *Q,
                       double *out, long ldo, cudaStream_t st);

// ---- dense.cu -------------------------------------------------------------------
// Small dense Rayleigh-Ritz on the device (single CTA kernels), ns <= kMaxDense.
constexpr int kMaxDense = 1024;
// Given M and Hs (ns x ns column-major, overwritten), computes ritz (ascending) and
// Cf = L^-T Q (column-major, ns x ns). status: 0 ok, 1 not SPD, 2 non-finite, 3 no
// convergence. work: dense_work_elems(ns) doubles.
long dense_work_elems(int ns);
cudaError_t dense_rr(double *M, double *Hs, int ns, double *ritz, double *Cf, double *work,
                     int *status, cudaStream_t st);
// Symmetric eigensolve (cyclic Jacobi) of A (n x n, column-major, overwritten):
// eigenvalues ascending in ev, eigenvectors (sign-fixed) in Q. n = *ns_dev when ns_dev is
// not null (then n <= ns), else ns. work: dense_work_elems(ns).
cudaError_t dense_syev(double *A, int ns, const int *ns_dev, double *ev, double *Q,
                       double *work, int *status, cudaStream_t st);

// ---- jacobi.cu --------------------------------------------------------------------
// Grid-wide barrier state (zeroed before each cooperative launch).
struct GridBarrier {
    unsigned count;  // arrivals since the barrier was zeroed (grid.cuh)
    unsigned gen;    // unused
    int err;
    int pad;
};
// Multi-SM cyclic Jacobi of A0 (n x n, column-major; A1 is a second n x n buffer):
// eigenvalues (unsorted) in diag, eigenvectors in V. Skipped if *status != 0 on entry;
// sets *status = 3 if the sweeps do not converge; bar->err != 0 after a barrier timeout.
cudaError_t jacobi_grid(double *A0, double *A1, double *V, double *diag, int n, GridBarrier *bar,
                        int *status, int *sweeps_out, cudaStream_t st);
// Block Jacobi in FP32 (jacobi.cu): V = eigenvectors of the symmetric A (n x n, column-
// major, overwritten by the nearly diagonal result); scratch of block_jacobi_f32_scratch(n)
// bytes (device, 8-byte aligned); *sweeps_out (device) = sweeps used or -1. Synchronises
// the stream once per sweep from the third on.
size_t block_jacobi_f32_scratch(int n);
cudaError_t block_jacobi_f32(float *A, float *V, int n, void *scratch, int *sweeps_out,
                             int max_sweeps, cudaStream_t st);
// Self-tests of the bounded waits (failure detection without a fault): a grid barrier
// that can never complete (status <- 4 after its spin limit) and an mbarrier that never
// completes (err <- 1 after its probe limit).
cudaError_t barrier_selftest(GridBarrier *bar, int *status, cudaStream_t st);
cudaError_t mbar_selftest(int *err, cudaStream_t st);

// ---- lanczos.cu -------------------------------------------------------------------
constexpr int kDotBlocks = 608;
// r = <x, y> (FP64, deterministic two-level reduction); part: kDotBlocks doubles.
cudaError_t dot_f64(const double *x, const double *y, long n, double *part, double *r,
                    cudaStream_t st);
cudaError_t lanczos_start(double *v, long n, unsigned long long seed, cudaStream_t st);
// v *= 1/sqrt(*nrm2)
cudaError_t scale_rsqrt(double *v, long n, const double *nrm2, cudaStream_t st);
// w = w - alpha[j] v - beta[j-1] vp   (beta term skipped when j == 0); skipped if *stop
cudaError_t lanczos_orth(double *w, const double *v, const double *vp, long n,
                         const double *alpha, const double *beta, int j, const int *stop,
                         cudaStream_t st);
// beta[j] = sqrt(*nrm2); if beta[j] == 0 or non-finite: *stop = j+1 (once)
cudaError_t lanczos_beta(double *beta, int j, const double *nrm2, int *stop, cudaStream_t st);
// vp = v; v = w / beta[j] (skipped if *stop)
cudaError_t lanczos_next(double *v, double *vp, const double *w, long n, const double *beta,
                         int j, const int *stop, cudaStream_t st);
// T (k x k) from alpha, beta, using keff = (*stop ? *stop : k)
cudaError_t lanczos_tridiag(const double *alpha, const double *beta, int k, const int *stop,
                            double *T, int *keff, cudaStream_t st);
// out[0] = theta_min, out[1] = max(1.01 theta_max, theta_max + |beta_keff s|)
cudaError_t lanczos_bounds_final(const double *ev, const double *Q, const double *beta, int k,
                                 const int *keff, double *out, cudaStream_t st);

// ---- resid (gram.cu) --------------------------------------------------------------
// resid[c] = || HX[:,c] - ritz[c] X[:,c] ||_2 (deterministic per-column reduction)
cudaError_t resid_f64(const double *X, const double *HX, long ld, long nd, int ncols,
                      const double *ritz, double *resid, cudaStream_t st);
cudaError_t resid_f32(const float *X, const float *HX, long ld, long nd, int ncols,
                      const double *ritz, double *resid, cudaStream_t st);
// flag |= 1 if any of n values is NaN or Inf
cudaError_t check_finite(const double *a, long n, int *flag, cudaStream_t st);

// ---- observables.cu -----------------------------------------------------------------
// Fermi level of Eq. (FermiEnergyConstraintFormulation): *mu with 2 sum g_n = nelec, g
// (ns values) the occupations at *mu; *status 0 converged, 1 not converged, 2 non-finite
// eigenvalue. One CTA; lam, mu, g, status on the device.
cudaError_t fermi_level(const double *lam, int ns, double nelec, double kT, double *mu,
                        double *g, int *status, cudaStream_t st);
// rho[p] = (2 / h^3) sum_n g_n X[p + n ld]^2, p < nd (g: ncols values on the device)
template <typename T>
cudaError_t density(const T *X, long ld, int ncols, long nd, const double *g, double h,
                    double *rho, cudaStream_t st);
// Weights w~_p of Eq. (gradient:approximate) for radius n_o (1/h included), zero beyond.
struct GradCoef {
    double w[kRadius + 1];
};
GradCoef grad_coef(int radius, double h);
// Non-local force of Eq. (NonlocForce:Discrete): f (3 natoms) from the columns X, occupations
// g (ncols) and gamma (4 natoms); yw: 16 natoms ncols doubles of workspace.
template <typename T>
cudaError_t nonlocal_force(const DevHam &H, const T *X, long ld, int ncols, const double *g,
                           const double *gamma, const GradCoef &wg, double *yw, double *f,
                           cudaStream_t st);

// ---- poisson.cu -------------------------------------------------------------------
// Bytes of device workspace poisson_solve needs for an n0 x n1 x n2 grid.
size_t poisson_workspace(int n0, int n1, int n2, int radius);
// Electrostatic potential: phi (Nd) from rho (Nd, or null for zero) and the pseudocharges
// of the atoms R (3 natoms), Z (natoms) with the potential -Z erf(r/rc)/r; b_out (Nd, or
// null) receives the pseudocharge density. CG to ||r|| <= tol ||rhs|| or maxit iterations;
// *iters_host and *relres_host report them. Synchronises.
cudaError_t poisson_solve(const DevHam &H, const double *R, const double *Z, int natoms,
                          double rc, const double *rho, double *phi, double *b_out, double tol,
                          int maxit, void *ws, int *iters_host, double *relres_host,
                          cudaStream_t st);

}  // namespace sparc
