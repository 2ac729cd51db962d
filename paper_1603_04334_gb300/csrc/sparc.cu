// sparc.cu -- context, workspaces and the C ABI declared in include/sparc.h.
//
// The context owns the device copy of the Hamiltonian of Sec. 3.1 (V_eff, projector
// tables) and grow-only workspaces; caller blocks (X, HX, work) are never freed here.
// Host code only validates arguments, sizes workspaces and enqueues kernels; every
// arithmetic step of the path runs in the kernels of stencil.cu, nonlocal.cu, gram.cu,
// dense.cu, lanczos.cu and setup.cu.
#include "sparc.h"
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

using namespace sparc;

namespace sparc {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Filter interval of the first CheFSI iteration from the Lanczos bounds [lo, hi] (Sec. 4
// gives the lower end as lambda_c = E_F + 0.1 Ha, which a fixed Hamiltonian without
// electrons lacks): a0 = lo, b = hi and the cutoff a a quarter of the way up,
// a = a0 + (b - a0) / 4. Later iterations take a and a0 from the Ritz values
// (sparc_chefsi_step).
void first_iteration_bounds(double lo, double hi, double *bounds)
{
    bounds[0] = lo + 0.25 * (hi - lo);
    bounds[1] = hi;
    bounds[2] = lo;
}
}  // namespace sparc

// Per-phase CUDA-event timing on the context stream.
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;          // recycled events
    std::vector<cudaEvent_t> used;          // events handed out since the last read
    std::vector<int> phase;                 // phase of each (start, stop) pair in `used`
    long long count[SPARC_NPHASES] = {0};
    double ms[SPARC_NPHASES] = {0};
};

struct sparc_ctx {
    DevHam H;
    cudaStream_t st = nullptr;
    std::string err;

    // owned tables
    double *V = nullptr;
    float *Vf = nullptr;
    int *atom_ptr = nullptr, *idx = nullptr, *ent_atom = nullptr;
    double *chi = nullptr, *gchi = nullptr;
    float *chi_f = nullptr, *gchi_f = nullptr;
    int *uniq_node = nullptr, *uniq_ptr = nullptr, *ent_list = nullptr;
    float2 *nl_gdf = nullptr;
    int4 *chi_q = nullptr;
    int *chi_F = nullptr;
    int *proj_order = nullptr;   // atoms in Morton order of their cells (projections)
    int *nl_atom = nullptr;
    float *nl_gf = nullptr;

    // grow-only workspaces
    void *C = nullptr;       size_t C_bytes = 0;     // projection coefficients
    void *hx = nullptr;      size_t hx_bytes = 0;    // FP64 H Xf
    void *rotx = nullptr;    size_t rotx_bytes = 0;  // rotated block
    void *roth = nullptr;    size_t roth_bytes = 0;  // rotated H block (residuals)
    void *part = nullptr;    size_t part_bytes = 0;  // Gram split-K partials
    void *tcws = nullptr;    size_t tcws_bytes = 0;  // tensor-core Gram digits, exponents, partials
    size_t dev_bytes = 0, dev_peak = 0;  // device bytes allocated (see dmalloc)
    void *dm = nullptr;      size_t dm_bytes = 0;    // M, Hs, Cf, ritz, resid, dense work
    void *lz = nullptr;      size_t lz_bytes = 0;    // Lanczos vectors and scalars
    void *bnd = nullptr;     size_t bnd_bytes = 0;   // column bounds of the FP64 filter's blocks
    void *bsc = nullptr;     size_t bsc_bytes = 0;   // column bounds of other FP64 H applications
    void *vc = nullptr;      size_t vc_bytes = 0;    // alpha (V_eff - shift) of an FP64 step
    int *flags = nullptr;                            // device status words
    void *obs = nullptr;     size_t obs_bytes = 0;   // occupations, density and force data
    std::vector<double> gamma;                       // KB coefficients, 4 per atom (host)
    std::vector<double> atomR, atomZ;                // positions and valence charges (host)
    double rc_erf = 1.0;
    void *pois = nullptr;    size_t pois_bytes = 0;  // electrostatics workspace
    double *pin = nullptr;                           // pinned host staging (2*1024+16)
    int *pin_i = nullptr;
    Profiler prof;
};

namespace {

constexpr int kMaxLanczos = 64;
constexpr int kPinDoubles = 2 * kMaxDense + 16;

sparc_status fail(sparc_ctx *c, sparc_status s, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

sparc_status fail(sparc_ctx *c, sparc_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SPARC_ERR_OOM : SPARC_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define TRY(call)                                                                      \
    do {                                                                               \
        sparc_status s_ = (call);                                                      \
        if (s_ != SPARC_OK) return s_;                                                 \
    } while (0)

cudaEvent_t prof_event(sparc_ctx *ctx)
{
    Profiler &P = ctx->prof;
    cudaEvent_t e = nullptr;
    if (!P.pool.empty()) {
        e = P.pool.back();
        P.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    P.used.push_back(e);
    return e;
}

// Brackets the launches of one phase with events when profiling is on.
struct PhaseScope {
    sparc_ctx *ctx;
    int ph;
    bool live = false;
    PhaseScope(sparc_ctx *c, int p) : ctx(c), ph(p)
    {
        if (!ctx->prof.on) return;
        cudaEvent_t e = prof_event(ctx);
        if (e && cudaEventRecord(e, ctx->st) == cudaSuccess) live = true;
    }
    ~PhaseScope()
    {
        if (!live) return;
        cudaEvent_t e = prof_event(ctx);
        if (e) {
            cudaEventRecord(e, ctx->st);
            ctx->prof.phase.push_back(ph);
        } else {
            ctx->prof.used.pop_back();
        }
    }
};
#define PHASE(p) PhaseScope phase_scope_(ctx, (p))

sparc_status prof_collect(sparc_ctx *ctx)
{
    Profiler &P = ctx->prof;
    if (P.used.empty()) return SPARC_OK;
    CK(cudaStreamSynchronize(ctx->st));
    const size_t pairs = P.phase.size();
    for (size_t q = 0; q < pairs && 2 * q + 1 < P.used.size(); ++q) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, P.used[2 * q], P.used[2 * q + 1]));
        P.count[P.phase[q]] += 1;
        P.ms[P.phase[q]] += t;
    }
    for (cudaEvent_t e : P.used) P.pool.push_back(e);
    P.used.clear();
    P.phase.clear();
    return SPARC_OK;
}

sparc_status ensure(sparc_ctx *ctx, void *&p, size_t &cap, size_t bytes)
{
    if (bytes <= cap) return SPARC_OK;
    if (p) CK(cudaFree(p));
    ctx->dev_bytes -= cap;
    p = nullptr;
    cap = 0;
    CK(cudaMalloc(&p, bytes));
    cap = bytes;
    ctx->dev_bytes += bytes;
    if (ctx->dev_bytes > ctx->dev_peak) ctx->dev_peak = ctx->dev_bytes;
    return SPARC_OK;
}

template <typename T>
sparc_status dmalloc(sparc_ctx *ctx, T *&p, size_t n)
{
    CK(cudaMalloc((void **)&p, sizeof(T) * (n ? n : 1)));
    // counted until the context is destroyed (set-up temporaries included): an upper
    // bound of the context's peak device memory
    ctx->dev_bytes += sizeof(T) * (n ? n : 1);
    if (ctx->dev_bytes > ctx->dev_peak) ctx->dev_peak = ctx->dev_bytes;
    return SPARC_OK;
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

sparc_status check_block(sparc_ctx *ctx, const void *X, int ncols, long ld, const char *name)
{
    if (!X) return fail(ctx, SPARC_ERR_ARG, "%s is NULL", name);
    if (ncols <= 0) return fail(ctx, SPARC_ERR_ARG, "ncols must be positive (got %d)", ncols);
    if (ncols > 65535) return fail(ctx, SPARC_ERR_ARG, "ncols %d exceeds 65535", ncols);
    if (ld < ctx->H.nd)
        return fail(ctx, SPARC_ERR_ARG, "ld (%ld) must be >= Nd (%ld)", ld, ctx->H.nd);
    return SPARC_OK;
}

size_t esize(sparc_dtype t) { return t == SPARC_F32 ? 4 : 8; }

// --- H applications --------------------------------------------------------------------
sparc_status ensure_C(sparc_ctx *ctx, int ncols)
{
    const size_t b = sizeof(double) * 4 * (size_t)(ctx->H.natoms > 0 ? ctx->H.natoms : 1) * ncols;
    return ensure(ctx, ctx->C, ctx->C_bytes, b);
}

// Column bounds of an FP64 or FP32 block into the scratch bound buffer (zeroed, then
// raised by one pass over the block); returns the buffer.
template <typename T>
sparc_status scratch_bounds(sparc_ctx *ctx, const T *Y, int ncols, long ld, unsigned **b)
{
    TRY(ensure(ctx, ctx->bsc, ctx->bsc_bytes, sizeof(unsigned) * (size_t)ncols));
    *b = (unsigned *)ctx->bsc;
    CK(cudaMemsetAsync(*b, 0, sizeof(unsigned) * (size_t)ncols, ctx->st));
    if (std::is_same<T, double>::value)
        CK(colmax_f64((const double *)Y, ncols, ld, ctx->H.nd, *b, ctx->st));
    else
        CK(colmax_f32((const float *)Y, ncols, ld, ctx->H.nd, *b, ctx->st));
    return SPARC_OK;
}

// alpha (V_eff - shift) for one FP64 step (formed on the context stream before the step;
// V_eff itself for alpha = 1, shift = 0).
sparc_status scaled_potential(sparc_ctx *ctx, double alpha, double shift, const double **u)
{
    if (alpha == 1.0 && shift == 0.0) {
        *u = ctx->H.V;
        return SPARC_OK;
    }
    TRY(ensure(ctx, ctx->vc, ctx->vc_bytes, sizeof(double) * (size_t)ctx->H.nd));
    CK(scaled_v(ctx->H.V, alpha, shift, (double *)ctx->vc, ctx->H.nd, ctx->st));
    *u = (const double *)ctx->vc;
    return SPARC_OK;
}

// out = alpha ((H - shift) Y) - beta Yprev  (Yprev may alias out, may be null):
// projection alpha chi^T Y, stencil step, nonlocal scatter-add. bY: column bounds of Y
// (null: taken here by a pass over Y); bOut: raised to the bounds of out when not null.
sparc_status step_f64(sparc_ctx *ctx, const double *Y, const double *Yprev, double *out, int ncols,
                      long ld, double alpha, double shift, double beta,
                      const unsigned *bY = nullptr, unsigned *bOut = nullptr)
{
    const DevHam &H = ctx->H;
    if (!bY) {
        unsigned *b = nullptr;
        TRY(scratch_bounds(ctx, Y, ncols, ld, &b));
        bY = b;
    }
    const double *u = nullptr;
    { PHASE(SPARC_PHASE_OTHER); TRY(scaled_potential(ctx, alpha, shift, &u)); }
    if (H.natoms > 0) {
        TRY(ensure_C(ctx, ncols));
        { PHASE(SPARC_PHASE_PROJECT); CK(project_f64_fx(H, Y, ncols, ld, alpha, bY, (float2 *)ctx->C, ctx->st)); }
    }
    { PHASE(SPARC_PHASE_STENCIL); CK(stencil_f64(H, Y, Yprev, out, ncols, ld, alpha, u, beta, bY, bOut, ctx->st)); }
    if (H.natoms > 0) { PHASE(SPARC_PHASE_SCATTER); CK(scatter_f64_df(H, (const float2 *)ctx->C, out, ncols, ld, bOut, ctx->st)); }
    return SPARC_OK;
}

sparc_status step_f32(sparc_ctx *ctx, const float *Y, const float *Yprev, float *out, int ncols,
                      long ld, double alpha, double shift, double beta)
{
    const DevHam &H = ctx->H;
    if (H.natoms > 0) {
        TRY(ensure_C(ctx, ncols));
        { PHASE(SPARC_PHASE_PROJECT); CK(project_f32(H, Y, ncols, ld, alpha, (float *)ctx->C, ctx->st)); }
    }
    { PHASE(SPARC_PHASE_STENCIL); CK(stencil_f32(H, Y, Yprev, out, ncols, ld, alpha, shift, beta, ctx->st)); }
    if (H.natoms > 0) { PHASE(SPARC_PHASE_SCATTER); CK(scatter_f32(H, (const float *)ctx->C, out, ncols, ld, ctx->st)); }
    return SPARC_OK;
}

// FP64 H applied to an FP32 block (result FP64)
sparc_status apply_f32in_f64(sparc_ctx *ctx, const float *Y, double *out, int ncols, long ld)
{
    const DevHam &H = ctx->H;
    unsigned *bY = nullptr;
    TRY(scratch_bounds(ctx, Y, ncols, ld, &bY));
    if (H.natoms > 0) {
        TRY(ensure_C(ctx, ncols));
        { PHASE(SPARC_PHASE_PROJECT); CK(project_f32in_f64(H, Y, ncols, ld, bY, (float2 *)ctx->C, ctx->st)); }
    }
    { PHASE(SPARC_PHASE_STENCIL); CK(stencil_f32in_f64(H, Y, out, ncols, ld, bY, ctx->st)); }
    if (H.natoms > 0) { PHASE(SPARC_PHASE_SCATTER); CK(scatter_f64_df(H, (const float2 *)ctx->C, out, ncols, ld, nullptr, ctx->st)); }
    return SPARC_OK;
}

// Step t of a filter (Y = Y_t, Yp = Y_{t-1}, out = Y_{t+1}). FP64 blocks: bnd holds one
// row of column bounds per Y_t (row 0 filled before the first step); step t reads row t
// and raises row t+1.
template <typename T>
sparc_status step_t(sparc_ctx *ctx, const T *Y, const T *Yp, T *out, int ncols, long ld,
                    double alpha, double shift, double beta, unsigned *bnd, int t);
template <>
sparc_status step_t<double>(sparc_ctx *ctx, const double *Y, const double *Yp, double *out,
                            int ncols, long ld, double alpha, double shift, double beta,
                            unsigned *bnd, int t)
{
    const size_t n = (size_t)ncols;
    return step_f64(ctx, Y, Yp, out, ncols, ld, alpha, shift, beta, bnd + t * n,
                    bnd + (t + 1) * n);
}
template <>
sparc_status step_t<float>(sparc_ctx *ctx, const float *Y, const float *Yp, float *out,
                           int ncols, long ld, double alpha, double shift, double beta,
                           unsigned *, int)
{
    return step_f32(ctx, Y, Yp, out, ncols, ld, alpha, shift, beta);
}

// --- Chebyshev filter (Algorithm ChebychevFilter, scaled recurrence) -------------------
sparc_status check_bounds(sparc_ctx *ctx, int degree, double a, double b, double a0)
{
    if (degree < 1) return fail(ctx, SPARC_ERR_ARG, "degree must be >= 1 (got %d)", degree);
    if (!(std::isfinite(a) && std::isfinite(b) && std::isfinite(a0)))
        return fail(ctx, SPARC_ERR_ARG, "filter bounds must be finite");
    if (!(a0 < a && a < b))
        return fail(ctx, SPARC_ERR_ARG, "filter bounds need a0 < a < b (a0=%g a=%g b=%g)", a0, a, b);
    return SPARC_OK;
}

// Runs the filter with X as Y_0 and W as the second buffer; *result is the buffer that
// holds Y_m (X when degree is even, W when odd).
template <typename T>
sparc_status filter_impl(sparc_ctx *ctx, T *X, T *W, int ncols, long ld, int m, double a,
                         double b, double a0, T **result)
{
    const double e = (b - a) / 2.0, c = (b + a) / 2.0;
    const double sigma1 = e / (a0 - c);
    unsigned *bnd = nullptr;
    if (std::is_same<T, double>::value) {
        const size_t nb = sizeof(unsigned) * (size_t)(m + 1) * ncols;
        TRY(ensure(ctx, ctx->bnd, ctx->bnd_bytes, nb));
        bnd = (unsigned *)ctx->bnd;
        CK(cudaMemsetAsync(bnd, 0, nb, ctx->st));
        CK(colmax_f64((const double *)X, ncols, ld, ctx->H.nd, bnd, ctx->st));
    }
    TRY(step_t<T>(ctx, X, nullptr, W, ncols, ld, sigma1 / e, c, 0.0, bnd, 0));
    T *cur = W, *prev = X;
    double sigma = sigma1;
    for (int j = 2; j <= m; ++j) {
        const double sn = 1.0 / (2.0 / sigma1 - sigma);
        TRY(step_t<T>(ctx, cur, prev, prev, ncols, ld, 2.0 * sn / e, c, sigma * sn, bnd, j - 1));
        T *t = cur;
        cur = prev;
        prev = t;
        sigma = sn;
    }
    *result = cur;
    return SPARC_OK;
}

template <typename T>
sparc_status copy_block(sparc_ctx *ctx, T *dst, const T *src, int ncols, long ld)
{
    if (dst == src) return SPARC_OK;
    CK(cudaMemcpy2DAsync(dst, ld * sizeof(T), src, ld * sizeof(T), ctx->H.nd * sizeof(T), ncols,
                         cudaMemcpyDeviceToDevice, ctx->st));
    return SPARC_OK;
}

// --- Rayleigh-Ritz --------------------------------------------------------------------
struct DenseBufs {
    double *M, *Hs, *Cf, *ritz, *resid, *work;
};

sparc_status dense_bufs(sparc_ctx *ctx, int ns, DenseBufs &d)
{
    const size_t nn = (size_t)ns * ns;
    const size_t tot = 3 * nn + 2 * (size_t)ns + (size_t)dense_work_elems(ns);
    TRY(ensure(ctx, ctx->dm, ctx->dm_bytes, tot * sizeof(double)));
    double *b = (double *)ctx->dm;
    d.M = b;
    d.Hs = b + nn;
    d.Cf = b + 2 * nn;
    d.ritz = b + 3 * nn;
    d.resid = d.ritz + ns;
    d.work = d.resid + ns;
    return SPARC_OK;
}

// Projection + eigensolve + rotation of the filtered block Yf. The rotated block is
// written to `dst` (which may be Yf itself). HX: FP64 workspace (ncols x ld) or null.
template <typename T>
sparc_status rr_core(sparc_ctx *ctx, T *Yf, T *dst, double *HX, int ns, long ld,
                     double *ritz_host, double *resid_host)
{
    const long nd = ctx->H.nd;
    if (ns > kMaxDense)
        return fail(ctx, SPARC_ERR_ARG, "ncols %d exceeds the dense eigensolver limit %d", ns,
                    kMaxDense);
    if (!ritz_host) return fail(ctx, SPARC_ERR_ARG, "ritz_host is NULL");
    if (!HX) {
        TRY(ensure(ctx, ctx->hx, ctx->hx_bytes, sizeof(double) * (size_t)ns * ld));
        HX = (double *)ctx->hx;
    }
    // H Yf in FP64
    if (sizeof(T) == 8)
        TRY(step_f64(ctx, (const double *)Yf, nullptr, HX, ns, ld, 1.0, 0.0, 0.0));
    else
        TRY(apply_f32in_f64(ctx, (const float *)Yf, HX, ns, ld));
    // M_s = Yf^T Yf, H_s = Yf^T (H Yf)
    DenseBufs d;
    TRY(dense_bufs(ctx, ns, d));
    // Both forms: the two contractions on the tensor cores in the 47-bit digit form
    // (gram_tc.cu; an FP32 block's entries are represented exactly, H Yf to 2^-48 of each
    // chunk's largest: FP64-level M_s and H_s), slab by slab where the whole block's digits
    // would exceed the workspace cap; the rotations below reuse the workspace.
    const bool mixed = sizeof(T) == 4;
    const long slab = tc_slab_rows(nd, ns, mixed);
    {
        TRY(ensure(ctx, ctx->tcws, ctx->tcws_bytes, tc_slab_workspace(nd, ns, mixed)));
        const size_t nn = (size_t)ns * ns;
        if (slab < nd) TRY(ensure(ctx, ctx->part, ctx->part_bytes, sizeof(double) * 2 * nn));
        PHASE(SPARC_PHASE_GRAM);
        for (long r0 = 0; r0 < nd; r0 += slab) {
            const long rows = nd - r0 < slab ? nd - r0 : slab;
            double *Mo = r0 ? (double *)ctx->part : d.M, *Ho = r0 ? (double *)ctx->part + nn : d.Hs;
            CK(gram_tc47_pair<T>(Yf + r0, ld, HX + r0, ld, rows, ns, Mo, Ho, ctx->tcws, ctx->tcws_bytes, ctx->H.err, ctx->st));
            if (r0) {
                CK(add_into(d.M, Mo, (long)nn, ctx->st));
                CK(add_into(d.Hs, Ho, (long)nn, ctx->st));
            }
        }
    }
    { PHASE(SPARC_PHASE_DENSE); CK(dense_rr(d.M, d.Hs, ns, d.ritz, d.Cf, d.work, ctx->flags, ctx->st)); }
    CK(cudaMemcpyAsync(ctx->pin_i, ctx->flags, sizeof(int) * 16, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int status = ctx->pin_i[0];
    if (ctx->pin_i[14] != 0) {
        CK(cudaMemsetAsync(ctx->flags + 14, 0, sizeof(int), ctx->st));
        return fail(ctx, SPARC_ERR_TIMEOUT, "a stencil launch timed out waiting for a TMA load");
    }
    if (status == 4) return fail(ctx, SPARC_ERR_TIMEOUT, "grid barrier of the Jacobi solver timed out");
    if (status == 1)
        return fail(ctx, SPARC_ERR_NOT_SPD, "overlap matrix M_s is not positive definite");
    if (status == 2) return fail(ctx, SPARC_ERR_NONFINITE, "non-finite entries in M_s or H_s");
    if (status == 3) return fail(ctx, SPARC_ERR_TIMEOUT, "Jacobi eigensolver did not converge");
    if (status != 0) return fail(ctx, SPARC_ERR_CUDA, "dense eigensolver status %d", status);
    // rotation X = Yf (L^-T Q)
    T *xout = dst;
    if (dst == Yf) {
        TRY(ensure(ctx, ctx->rotx, ctx->rotx_bytes, sizeof(T) * (size_t)ns * ld));
        xout = (T *)ctx->rotx;
    }
    if (sizeof(T) == 8) {
        PHASE(SPARC_PHASE_ROTATE);
        for (long r0 = 0; r0 < nd; r0 += slab)
            CK(rotate_tc((const double *)Yf + r0, ld, nd - r0 < slab ? nd - r0 : slab, ns, d.Cf, (double *)xout + r0, ld, ctx->tcws, ctx->tcws_bytes, ctx->H.err, ctx->st));
    } else {
        PHASE(SPARC_PHASE_ROTATE);
        for (long r0 = 0; r0 < nd; r0 += slab)
            CK(rotate_tc23<float>((const float *)Yf + r0, ld, nd - r0 < slab ? nd - r0 : slab, ns, d.Cf, (float *)xout + r0, ld, ctx->tcws, ctx->tcws_bytes, ctx->H.err, ctx->st));
    }
    if (resid_host) {
        // H X = (H Y_f) (L^-T Q); residuals against the rotated block. The mixed form rotates
        // H Y_f in the 23-bit digit form to FP32 (the block itself is FP32; about 1e-7
        // relative of |H X|).
        TRY(ensure(ctx, ctx->roth, ctx->roth_bytes, sizeof(T) * (size_t)ns * ld));
        if (sizeof(T) == 8) {
            double *hxr = (double *)ctx->roth;
            {
                PHASE(SPARC_PHASE_ROTATE);
                for (long r0 = 0; r0 < nd; r0 += slab)
                    CK(rotate_tc(HX + r0, ld, nd - r0 < slab ? nd - r0 : slab, ns, d.Cf, hxr + r0, ld, ctx->tcws, ctx->tcws_bytes, ctx->H.err, ctx->st));
            }
            { PHASE(SPARC_PHASE_OTHER); CK(resid_f64((const double *)xout, hxr, ld, nd, ns, d.ritz, d.resid, ctx->st)); }
        } else {
            float *hxr = (float *)ctx->roth;
            {
                PHASE(SPARC_PHASE_ROTATE);
                for (long r0 = 0; r0 < nd; r0 += slab)
                    CK(rotate_tc23<double>(HX + r0, ld, nd - r0 < slab ? nd - r0 : slab, ns, d.Cf, hxr + r0, ld, ctx->tcws, ctx->tcws_bytes, ctx->H.err, ctx->st));
            }
            { PHASE(SPARC_PHASE_OTHER); CK(resid_f32((const float *)xout, hxr, ld, nd, ns, d.ritz, d.resid, ctx->st)); }
        }
    }
    if (xout != dst) TRY(copy_block<T>(ctx, dst, xout, ns, ld));
    CK(cudaMemcpyAsync(ctx->pin, d.ritz, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::memcpy(ritz_host, ctx->pin, sizeof(double) * ns);
    if (resid_host) std::memcpy(resid_host, ctx->pin + ns, sizeof(double) * ns);
    return SPARC_OK;
}

void lap_weights(int no, double h, double *w)
{
    // Eq. (weightsLap), Sec. 3.1.
    double s = 0.0;
    for (int q = 1; q <= no; ++q) s += 1.0 / ((double)q * q);
    w[0] = -s / (h * h);
    for (int p = 1; p <= kRadius; ++p) {
        if (p > no) {
            w[p] = 0.0;
            continue;
        }
        double ratio = 1.0;
        for (int q = 1; q <= p; ++q) ratio *= (double)(no - q + 1) / (double)(no + q);
        w[p] = 2.0 * ((p % 2) ? 1.0 : -1.0) / (h * h * (double)p * p) * ratio;
    }
}

// Eq. (weightsLap) as exact fractions: h^2 w_p = 2 (-1)^(p+1) / p^2 * prod_{q<=p}
// (no-q+1)/(no+q) and the three-dimensional centre 6 h^2 w_0 = -6 sum_{q<=no} 1/q^2, all
// brought to their least common denominator D (831600 for no = 6). The FP64 stencil sums
// 6 neighbours of |value| < 2^27 per radius in int32 and accumulates the weighted sums of
// two such digit planes in int64, so |wint[0]| + 6 sum_p |wint[p]| must stay below 2^25.
bool lap_weights_int(int no, double h, int *wint, double &wunit)
{
    if (no < 1 || no > kRadius) return false;
    auto gcd = [](long long a, long long b) {
        if (a < 0) a = -a;
        while (b) {
            const long long t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    long long num[kRadius + 1], den[kRadius + 1];
    long long cn = 0, cd = 1;  // sum_q 1/q^2
    for (int q = 1; q <= no; ++q) {
        cn = cn * q * q + cd;
        cd *= (long long)q * q;
        const long long g = gcd(cn, cd);
        cn /= g;
        cd /= g;
    }
    num[0] = -6 * cn;
    den[0] = cd;
    for (int p = 1; p <= no; ++p) {
        long long n = 2, d = (long long)p * p;
        for (int q = 1; q <= p; ++q) {
            n *= no - q + 1;
            d *= no + q;
            const long long g = gcd(n, d);
            n /= g;
            d /= g;
        }
        num[p] = (p % 2) ? n : -n;
        den[p] = d;
    }
    long long D = 1;
    for (int p = 0; p <= no; ++p) {
        const long long g = gcd(D, den[p]);
        D = D / g * den[p];
        if (D > (1LL << 40)) return false;
    }
    long long tot = 0;
    for (int p = 0; p <= kRadius; ++p) {
        const long long W = p <= no ? num[p] * (D / den[p]) : 0;
        if (W > INT32_MAX || W < INT32_MIN) return false;
        wint[p] = (int)W;
        tot += (p ? 6 : 1) * (W < 0 ? -W : W);
    }
    if (tot >= (1LL << 25)) return false;
    wunit = 1.0 / ((double)D * h * h);
    return true;
}

void free_ctx(sparc_ctx *c)
{
    if (!c) return;
    void *ps[] = {c->V, c->Vf, c->atom_ptr, c->idx, c->ent_atom, c->chi, c->gchi, c->chi_f,
                  c->gchi_f, c->chi_q, c->chi_F, c->proj_order, c->uniq_node, c->uniq_ptr, c->ent_list, c->nl_atom, c->nl_gf, c->nl_gdf, c->C, c->hx, c->rotx, c->roth, c->part,
                  c->tcws, c->dm, c->lz, c->bnd, c->bsc, c->vc, c->flags, c->obs, c->pois};
    for (void *p : ps) dfree(p);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->prof.used) cudaEventDestroy(e);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->pin_i) cudaFreeHost(c->pin_i);
    delete c;
}

sparc_status build_tables(sparc_ctx *ctx, const sparc_atoms *at)
{
    DevHam &H = ctx->H;
    const int na = at->natoms;
    H.natoms = na;
    if (na == 0) return SPARC_OK;
    ctx->gamma.assign(at->gamma, at->gamma + 4 * (size_t)na);
    ctx->atomR.assign(at->R, at->R + 3 * (size_t)na);
    if (at->Z) ctx->atomZ.assign(at->Z, at->Z + (size_t)na);
    ctx->rc_erf = at->rc_erf;
    double *R = nullptr, *G = nullptr;
    int *counts = nullptr;
    TRY(dmalloc(ctx, R, 3 * (size_t)na));
    TRY(dmalloc(ctx, G, 4 * (size_t)na));
    TRY(dmalloc(ctx, counts, (size_t)na));
    CK(cudaMemcpyAsync(R, at->R, sizeof(double) * 3 * na, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(G, at->gamma, sizeof(double) * 4 * na, cudaMemcpyHostToDevice, ctx->st));
    CK(support_count(H.n0, H.n1, H.n2, H.h, na, R, at->rcut, counts, ctx->st));
    std::vector<int> hc(na);
    CK(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * na, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int> ptr(na + 1, 0);
    long tot = 0;
    for (int J = 0; J < na; ++J) {
        tot += hc[J];
        if (tot > 2000000000L) return fail(ctx, SPARC_ERR_ARG, "too many projector support entries");
        ptr[J + 1] = (int)tot;
    }
    H.nsup = tot;
    {   // the projections' CTA order: atoms sorted by the Morton code of their cell (cells
        // of 2 rcut), so that atoms whose supports overlap are gathered at about the same time
        std::vector<std::pair<unsigned long long, int>> key(na);
        const double cell = 2.0 * at->rcut;
        for (int J = 0; J < na; ++J) {
            unsigned long long code = 0;
            unsigned c3[3];
            for (int d = 0; d < 3; ++d) {
                const double v = at->R[3 * J + d] / cell;
                c3[d] = v <= 0.0 ? 0u : (v >= 1048575.0 ? 1048575u : (unsigned)v);
            }
            for (int b = 19; b >= 0; --b)
                for (int d = 2; d >= 0; --d) code = (code << 1) | ((c3[d] >> b) & 1u);
            key[J] = {code, J};
        }
        std::sort(key.begin(), key.end());
        std::vector<int> order(na);
        for (int J = 0; J < na; ++J) order[J] = key[J].second;
        TRY(dmalloc(ctx, ctx->proj_order, na));
        CK(cudaMemcpyAsync(ctx->proj_order, order.data(), sizeof(int) * na,
                           cudaMemcpyHostToDevice, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        H.proj_order = ctx->proj_order;
    }
    TRY(dmalloc(ctx, ctx->atom_ptr, na + 1));
    CK(cudaMemcpyAsync(ctx->atom_ptr, ptr.data(), sizeof(int) * (na + 1), cudaMemcpyHostToDevice,
                       ctx->st));
    TRY(dmalloc(ctx, ctx->idx, tot));
    TRY(dmalloc(ctx, ctx->ent_atom, tot));
    TRY(dmalloc(ctx, ctx->chi, 4 * tot));
    TRY(dmalloc(ctx, ctx->gchi, 4 * tot));
    TRY(dmalloc(ctx, ctx->chi_f, 4 * tot));
    TRY(dmalloc(ctx, ctx->gchi_f, 4 * tot));
    CK(support_fill(H.n0, H.n1, H.n2, H.h, na, R, G, at->sigma, at->rcut, ctx->atom_ptr, ctx->idx,
                    ctx->chi, ctx->chi_f, ctx->gchi, ctx->gchi_f, ctx->ent_atom, ctx->st));
    // inverse map node -> entries
    const long nd = H.nd;
    const long nu_max = tot < nd ? tot : nd;
    int *node_cnt = nullptr, *node_start = nullptr, *cursor = nullptr, *flags = nullptr,
        *rank = nullptr, *scan_tmp = nullptr;
    TRY(dmalloc(ctx, node_cnt, nd));
    TRY(dmalloc(ctx, node_start, nd + 1));
    TRY(dmalloc(ctx, cursor, nd));
    TRY(dmalloc(ctx, flags, nd));
    TRY(dmalloc(ctx, rank, nd + 1));
    TRY(dmalloc(ctx, scan_tmp, nd / 4096 + 2));
    TRY(dmalloc(ctx, ctx->ent_list, tot));
    TRY(dmalloc(ctx, ctx->uniq_node, nu_max));
    TRY(dmalloc(ctx, ctx->uniq_ptr, nu_max + 1));
    CK(build_inverse_map(nd, tot, ctx->idx, node_cnt, node_start, cursor, ctx->ent_list, flags,
                         rank, scan_tmp, ctx->uniq_node, ctx->uniq_ptr, ctx->st));
    int nuniq = 0;
    CK(cudaMemcpyAsync(&nuniq, rank + nd, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    H.nuniq = nuniq;
    for (void *p : {(void *)R, (void *)G, (void *)counts, (void *)node_cnt, (void *)node_start,
                    (void *)cursor, (void *)flags, (void *)rank, (void *)scan_tmp})
        CK(cudaFree(p));
    // chi on its integer grid (FP64 projection) and the node-ordered entry tables of the
    // scatter kernels
    TRY(dmalloc(ctx, ctx->chi_q, 2 * tot));
    TRY(dmalloc(ctx, ctx->chi_F, 4 * (long)H.natoms));
    CK(chi_fixed(H.natoms, ctx->atom_ptr, ctx->chi, ctx->chi_q, ctx->chi_F, ctx->st));
    TRY(dmalloc(ctx, ctx->nl_atom, tot));
    TRY(dmalloc(ctx, ctx->nl_gf, 4 * tot));
    TRY(dmalloc(ctx, ctx->nl_gdf, 4 * tot));
    CK(build_nl_node_tables(nuniq, ctx->uniq_ptr, ctx->ent_list, ctx->ent_atom, ctx->gchi,
                            ctx->nl_atom, ctx->nl_gf, ctx->nl_gdf, ctx->st));
    H.chi_q = ctx->chi_q;
    H.chi_F = ctx->chi_F;
    H.nl_atom = ctx->nl_atom;
    H.nl_gf = ctx->nl_gf;
    H.nl_gdf = ctx->nl_gdf;
    H.atom_ptr = ctx->atom_ptr;
    H.idx = ctx->idx;
    H.chi = ctx->chi;
    H.chi_f = ctx->chi_f;
    H.gchi = ctx->gchi;
    H.gchi_f = ctx->gchi_f;
    H.ent_atom = ctx->ent_atom;
    H.uniq_node = ctx->uniq_node;
    H.uniq_ptr = ctx->uniq_ptr;
    H.ent_list = ctx->ent_list;
    return SPARC_OK;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

sparc_status sparc_create(const sparc_grid *grid, const double *veff_host,
                          const sparc_atoms *atoms, void *cuda_stream, sparc_ctx **out)
{
    if (!out) return SPARC_ERR_ARG;
    *out = nullptr;
    if (!grid || !atoms) return SPARC_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (grid->n[d] < 1) return SPARC_ERR_ARG;
    const long nd = (long)grid->n[0] * grid->n[1] * grid->n[2];
    if (nd > 2000000000L || !(grid->h > 0.0) || grid->radius < 1 || grid->radius > kRadius)
        return SPARC_ERR_ARG;
    if (atoms->natoms < 0) return SPARC_ERR_ARG;
    if (atoms->natoms > 0 && (!atoms->R || !atoms->gamma || !(atoms->sigma > 0.0) ||
                              !(atoms->rcut >= 0.0)))
        return SPARC_ERR_ARG;
    if (!veff_host && atoms->natoms > 0 && (!atoms->Z || !(atoms->rc_erf > 0.0)))
        return SPARC_ERR_ARG;

    sparc_ctx *ctx = new (std::nothrow) sparc_ctx();
    if (!ctx) return SPARC_ERR_OOM;
    ctx->st = (cudaStream_t)cuda_stream;
    DevHam &H = ctx->H;
    H.n0 = grid->n[0];
    H.n1 = grid->n[1];
    H.n2 = grid->n[2];
    H.nd = nd;
    H.h = grid->h;
    H.radius = grid->radius;
    H.kscale = 1.0;
    lap_weights(grid->radius, grid->h, H.w);
    if (!lap_weights_int(grid->radius, grid->h, H.wint, H.wunit)) {
        delete ctx;
        return SPARC_ERR_ARG;
    }

    sparc_status s = SPARC_OK;
    auto run = [&]() -> sparc_status {
        CK(cudaMallocHost((void **)&ctx->pin, sizeof(double) * kPinDoubles));
        CK(cudaMallocHost((void **)&ctx->pin_i, sizeof(int) * 16));
        TRY(dmalloc(ctx, ctx->flags, 16));
        CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * 16, ctx->st));
        H.err = ctx->flags + 14;
        TRY(dmalloc(ctx, ctx->V, nd));
        TRY(dmalloc(ctx, ctx->Vf, nd));
        if (veff_host) {
            CK(cudaMemcpyAsync(ctx->V, veff_host, sizeof(double) * nd, cudaMemcpyHostToDevice,
                               ctx->st));
        } else if (atoms->natoms == 0) {
            CK(cudaMemsetAsync(ctx->V, 0, sizeof(double) * nd, ctx->st));
        } else {
            double *R = nullptr, *Z = nullptr;
            TRY(dmalloc(ctx, R, 3 * (size_t)atoms->natoms));
            TRY(dmalloc(ctx, Z, (size_t)atoms->natoms));
            CK(cudaMemcpyAsync(R, atoms->R, sizeof(double) * 3 * atoms->natoms,
                               cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(Z, atoms->Z, sizeof(double) * atoms->natoms,
                               cudaMemcpyHostToDevice, ctx->st));
            CK(build_veff(H.n0, H.n1, H.n2, H.h, atoms->natoms, R, Z, atoms->rc_erf, ctx->V,
                          ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            CK(cudaFree(R));
            CK(cudaFree(Z));
        }
        CK(to_float(ctx->V, ctx->Vf, nd, ctx->st));
        H.V = ctx->V;
        H.Vf = ctx->Vf;
        TRY(build_tables(ctx, atoms));
        CK(cudaStreamSynchronize(ctx->st));
        CK(cudaGetLastError());
        return SPARC_OK;
    };
    s = run();
    if (s != SPARC_OK) {
        fprintf(stderr, "sparc_create: %s\n", ctx->err.c_str());
        free_ctx(ctx);
        return s;
    }
    *out = ctx;
    return SPARC_OK;
}

sparc_status sparc_destroy(sparc_ctx *ctx)
{
    if (!ctx) return SPARC_OK;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    free_ctx(ctx);
    return SPARC_OK;
}

const char *sparc_last_error(const sparc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

sparc_status sparc_get_veff(sparc_ctx *ctx, double *veff_host)
{
    if (!ctx || !veff_host) return fail(ctx, SPARC_ERR_ARG, "null argument");
    CK(cudaMemcpyAsync(veff_host, ctx->V, sizeof(double) * ctx->H.nd, cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SPARC_OK;
}

sparc_status sparc_info(const sparc_ctx *ctx, long *nd, long *nsupport, int *natoms)
{
    if (!ctx) return SPARC_ERR_ARG;
    if (nd) *nd = ctx->H.nd;
    if (nsupport) *nsupport = ctx->H.nsup;
    if (natoms) *natoms = ctx->H.natoms;
    return SPARC_OK;
}

sparc_status sparc_set_kinetic_scale(sparc_ctx *ctx, double kscale)
{
    if (!ctx) return SPARC_ERR_ARG;
    if (!std::isfinite(kscale)) return fail(ctx, SPARC_ERR_ARG, "kscale must be finite");
    ctx->H.kscale = kscale;
    return SPARC_OK;
}

sparc_status sparc_apply_H(sparc_ctx *ctx, sparc_dtype dtype, const void *X, void *HX, int ncols,
                           long ld)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, X, ncols, ld, "X"));
    TRY(check_block(ctx, HX, ncols, ld, "HX"));
    if (X == HX) return fail(ctx, SPARC_ERR_ARG, "X and HX must be distinct");
    if (dtype == SPARC_F64)
        return step_f64(ctx, (const double *)X, nullptr, (double *)HX, ncols, ld, 1.0, 0.0, 0.0);
    if (dtype == SPARC_F32)
        return step_f32(ctx, (const float *)X, nullptr, (float *)HX, ncols, ld, 1.0, 0.0, 0.0);
    return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
}

sparc_status sparc_cheb_filter(sparc_ctx *ctx, sparc_dtype dtype, void *X, void *work, int ncols,
                               long ld, int degree, double a, double b, double a0)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, X, ncols, ld, "X"));
    TRY(check_block(ctx, work, ncols, ld, "work"));
    if (X == work) return fail(ctx, SPARC_ERR_ARG, "X and work must be distinct");
    TRY(check_bounds(ctx, degree, a, b, a0));
    if (dtype == SPARC_F64) {
        double *res = nullptr;
        TRY(filter_impl<double>(ctx, (double *)X, (double *)work, ncols, ld, degree, a, b, a0, &res));
        return copy_block<double>(ctx, (double *)X, res, ncols, ld);
    }
    if (dtype == SPARC_F32) {
        float *res = nullptr;
        TRY(filter_impl<float>(ctx, (float *)X, (float *)work, ncols, ld, degree, a, b, a0, &res));
        return copy_block<float>(ctx, (float *)X, res, ncols, ld);
    }
    return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
}

sparc_status sparc_orth_rr(sparc_ctx *ctx, sparc_dtype dtype, void *Xf, void *HXf_or_null,
                           int ncols, long ld, double *ritz_host, double *resid_host)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, Xf, ncols, ld, "Xf"));
    if (dtype == SPARC_F64)
        return rr_core<double>(ctx, (double *)Xf, (double *)Xf, (double *)HXf_or_null, ncols, ld,
                               ritz_host, resid_host);
    if (dtype == SPARC_F32)
        return rr_core<float>(ctx, (float *)Xf, (float *)Xf, (double *)HXf_or_null, ncols, ld,
                              ritz_host, resid_host);
    return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
}

sparc_status sparc_gram(sparc_ctx *ctx, sparc_dtype dtype_a, const void *A, sparc_dtype dtype_b,
                        const void *B, int ncols, long ld, double *G)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, A, ncols, ld, "A"));
    TRY(check_block(ctx, B, ncols, ld, "B"));
    if (!G) return fail(ctx, SPARC_ERR_ARG, "G is NULL");
    const long nd = ctx->H.nd;
    TRY(ensure(ctx, ctx->part, ctx->part_bytes,
               sizeof(double) * (size_t)gram_part_elems(ncols, nd)));
    double *part = (double *)ctx->part;
    PHASE(SPARC_PHASE_GRAM);
    if (dtype_a == SPARC_F64 && dtype_b == SPARC_F64)
        CK(gram_f64((const double *)A, ld, (const double *)B, ld, nd, ncols, G, part, ctx->st));
    else if (dtype_a == SPARC_F32 && dtype_b == SPARC_F32)
        CK(gram_f32_f32((const float *)A, ld, (const float *)B, ld, nd, ncols, G, part, ctx->st));
    else if (dtype_a == SPARC_F32 && dtype_b == SPARC_F64)
        CK(gram_f32_f64((const float *)A, ld, (const double *)B, ld, nd, ncols, G, part, ctx->st));
    else
        return fail(ctx, SPARC_ERR_ARG, "unsupported dtype pair (%d, %d)", (int)dtype_a,
                    (int)dtype_b);
    return SPARC_OK;
}

sparc_status sparc_gram_tc(sparc_ctx *ctx, sparc_dtype dtype_a, const void *A, sparc_dtype dtype_b,
                           const void *B, int ncols, long ld, double *G)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, A, ncols, ld, "A"));
    TRY(check_block(ctx, B, ncols, ld, "B"));
    if (!G) return fail(ctx, SPARC_ERR_ARG, "G is NULL");
    const long nd = ctx->H.nd;
    const bool same = A == B && dtype_a == dtype_b;
    TRY(ensure(ctx, ctx->tcws, ctx->tcws_bytes, gram_tc_workspace(nd, ncols, same, false)));
    PHASE(SPARC_PHASE_GRAM);
    if (dtype_a == SPARC_F32 && dtype_b == SPARC_F32)
        CK((gram_tc<float, float>((const float *)A, ld, (const float *)B, ld, nd, ncols, G,
                                 ctx->tcws, ctx->tcws_bytes, false, ctx->H.err, ctx->st)));
    else if (dtype_a == SPARC_F32 && dtype_b == SPARC_F64)
        CK((gram_tc<float, double>((const float *)A, ld, (const double *)B, ld, nd, ncols, G,
                                  ctx->tcws, ctx->tcws_bytes, false, ctx->H.err, ctx->st)));
    else if (dtype_a == SPARC_F64 && dtype_b == SPARC_F64)
        CK((gram_tc<double, double>((const double *)A, ld, (const double *)B, ld, nd, ncols, G,
                                   ctx->tcws, ctx->tcws_bytes, false, ctx->H.err, ctx->st)));
    else
        return fail(ctx, SPARC_ERR_ARG, "unsupported dtype pair (%d, %d)", (int)dtype_a,
                    (int)dtype_b);
    return SPARC_OK;
}

sparc_status sparc_chefsi_step(sparc_ctx *ctx, sparc_dtype dtype, void *X, void *work, int ncols,
                               long ld, int degree, double *bounds_inout, double *ritz_host,
                               double *resid_host)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (!bounds_inout) return fail(ctx, SPARC_ERR_ARG, "bounds_inout is NULL");
    TRY(check_block(ctx, X, ncols, ld, "X"));
    TRY(check_block(ctx, work, ncols, ld, "work"));
    if (X == work) return fail(ctx, SPARC_ERR_ARG, "X and work must be distinct");
    if (!ritz_host) return fail(ctx, SPARC_ERR_ARG, "ritz_host is NULL");
    const double a = bounds_inout[0], b = bounds_inout[1], a0 = bounds_inout[2];
    TRY(check_bounds(ctx, degree, a, b, a0));
    if (ncols > kMaxDense)
        return fail(ctx, SPARC_ERR_ARG, "ncols %d exceeds the dense eigensolver limit %d", ncols,
                    kMaxDense);
    if (dtype == SPARC_F64) {
        double *res = nullptr;
        TRY(filter_impl<double>(ctx, (double *)X, (double *)work, ncols, ld, degree, a, b, a0, &res));
        double *dst = (res == (double *)work) ? (double *)X : (double *)work;
        TRY(rr_core<double>(ctx, res, dst, nullptr, ncols, ld, ritz_host, resid_host));
        TRY(copy_block<double>(ctx, (double *)X, dst, ncols, ld));
    } else if (dtype == SPARC_F32) {
        float *res = nullptr;
        TRY(filter_impl<float>(ctx, (float *)X, (float *)work, ncols, ld, degree, a, b, a0, &res));
        float *dst = (res == (float *)work) ? (float *)X : (float *)work;
        TRY(rr_core<float>(ctx, res, dst, nullptr, ncols, ld, ritz_host, resid_host));
        TRY(copy_block<float>(ctx, (float *)X, dst, ncols, ld));
    } else {
        return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
    }
    CK(cudaStreamSynchronize(ctx->st));
    double lo = ritz_host[0], hi = ritz_host[0];
    for (int i = 1; i < ncols; ++i) {
        lo = ritz_host[i] < lo ? ritz_host[i] : lo;
        hi = ritz_host[i] > hi ? ritz_host[i] : hi;
    }
    bounds_inout[0] = hi;
    bounds_inout[2] = lo;
    return SPARC_OK;
}

sparc_status sparc_lanczos_bounds(sparc_ctx *ctx, int ksteps, unsigned long long seed, double *lo,
                                  double *hi)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (!lo || !hi) return fail(ctx, SPARC_ERR_ARG, "lo/hi is NULL");
    if (ksteps < 1 || ksteps > kMaxLanczos)
        return fail(ctx, SPARC_ERR_ARG, "ksteps must be in 1..%d (got %d)", kMaxLanczos, ksteps);
    const long nd = ctx->H.nd;
    const int K = kMaxLanczos;
    const size_t nsc = 4 * (size_t)K + 8 + 2 * (size_t)K * K + (size_t)dense_work_elems(K);
    const size_t tot = 3 * (size_t)nd + (size_t)kDotBlocks + nsc;
    TRY(ensure(ctx, ctx->lz, ctx->lz_bytes, tot * sizeof(double)));
    double *v = (double *)ctx->lz, *vp = v + nd, *w = vp + nd, *part = w + nd;
    double *alpha = part + kDotBlocks, *beta = alpha + K, *nrm2 = beta + K, *outb = nrm2 + 2,
           *ev = outb + 4, *T = ev + K + 2, *Q = T + (size_t)K * K, *work = Q + (size_t)K * K;
    int *stop = ctx->flags + 4, *keff = ctx->flags + 5, *status = ctx->flags + 6;
    CK(cudaMemsetAsync(ctx->flags + 4, 0, sizeof(int) * 3, ctx->st));
    CK(cudaMemsetAsync(vp, 0, sizeof(double) * nd, ctx->st));
    CK(cudaMemsetAsync(beta, 0, sizeof(double) * K, ctx->st));
    { PHASE(SPARC_PHASE_OTHER); CK(lanczos_start(v, nd, seed, ctx->st)); }
    { PHASE(SPARC_PHASE_OTHER); CK(dot_f64(v, v, nd, part, nrm2, ctx->st)); }
    { PHASE(SPARC_PHASE_OTHER); CK(scale_rsqrt(v, nd, nrm2, ctx->st)); }
    for (int j = 0; j < ksteps; ++j) {
        TRY(step_f64(ctx, v, nullptr, w, 1, nd, 1.0, 0.0, 0.0));
        { PHASE(SPARC_PHASE_OTHER); CK(dot_f64(w, v, nd, part, alpha + j, ctx->st)); }
        { PHASE(SPARC_PHASE_OTHER); CK(lanczos_orth(w, v, vp, nd, alpha, beta, j, stop, ctx->st)); }
        { PHASE(SPARC_PHASE_OTHER); CK(dot_f64(w, w, nd, part, nrm2, ctx->st)); }
        { PHASE(SPARC_PHASE_OTHER); CK(lanczos_beta(beta, j, nrm2, stop, ctx->st)); }
        { PHASE(SPARC_PHASE_OTHER); CK(lanczos_next(v, vp, w, nd, beta, j, stop, ctx->st)); }
    }
    { PHASE(SPARC_PHASE_OTHER); CK(lanczos_tridiag(alpha, beta, ksteps, stop, T, keff, ctx->st)); }
    { PHASE(SPARC_PHASE_DENSE); CK(dense_syev(T, ksteps, keff, ev, Q, work, status, ctx->st)); }
    { PHASE(SPARC_PHASE_OTHER); CK(lanczos_bounds_final(ev, Q, beta, ksteps, keff, outb, ctx->st)); }
    CK(cudaMemcpyAsync(ctx->pin, outb, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->pin_i, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    TRY(sparc_sync(ctx));
    if (ctx->pin_i[0] != 0)
        return fail(ctx, SPARC_ERR_TIMEOUT, "tridiagonal eigensolve failed (status %d)", ctx->pin_i[0]);
    *lo = ctx->pin[0];
    *hi = ctx->pin[1];
    return SPARC_OK;
}

sparc_status sparc_first_bounds(sparc_ctx *ctx, int ksteps, unsigned long long seed,
                                double *bounds_out)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (!bounds_out) return fail(ctx, SPARC_ERR_ARG, "bounds_out is NULL");
    double lo = 0.0, hi = 0.0;
    TRY(sparc_lanczos_bounds(ctx, ksteps, seed, &lo, &hi));
    first_iteration_bounds(lo, hi, bounds_out);
    if (!(bounds_out[2] < bounds_out[0] && bounds_out[0] < bounds_out[1]))
        return fail(ctx, SPARC_ERR_ARG,
                    "Lanczos bounds lo = %g, hi = %g leave no filter interval (a0 < a < b)", lo, hi);
    return SPARC_OK;
}

sparc_status sparc_profile_enable(sparc_ctx *ctx, int enable)
{
    if (!ctx) return SPARC_ERR_ARG;
    if (!enable && ctx->prof.on) {
        TRY(prof_collect(ctx));
    }
    ctx->prof.on = enable != 0;
    return SPARC_OK;
}

sparc_status sparc_profile_read(sparc_ctx *ctx, int phase, long long *launches, double *ms)
{
    if (!ctx) return SPARC_ERR_ARG;
    if (phase < 0 || phase >= SPARC_NPHASES)
        return fail(ctx, SPARC_ERR_ARG, "phase %d out of range", phase);
    TRY(prof_collect(ctx));
    if (launches) *launches = ctx->prof.count[phase];
    if (ms) *ms = ctx->prof.ms[phase];
    return SPARC_OK;
}

sparc_status sparc_profile_reset(sparc_ctx *ctx)
{
    if (!ctx) return SPARC_ERR_ARG;
    TRY(prof_collect(ctx));
    for (int p = 0; p < SPARC_NPHASES; ++p) {
        ctx->prof.count[p] = 0;
        ctx->prof.ms[p] = 0.0;
    }
    return SPARC_OK;
}

sparc_status sparc_launch_count(long long *count)
{
    if (!count) return SPARC_ERR_ARG;
    *count = g_launches.load(std::memory_order_relaxed);
    return SPARC_OK;
}

}  // extern "C"

namespace sparc {
// accessors for the batch layer (batch.cu)
const DevHam *ctx_ham(const sparc_ctx *ctx) { return &ctx->H; }
cudaStream_t ctx_stream(const sparc_ctx *ctx) { return ctx->st; }
float *ctx_coef_buffer(sparc_ctx *ctx, int ncols)
{
    return ensure_C(ctx, ncols) == SPARC_OK ? (float *)ctx->C : nullptr;
}
}  // namespace sparc

extern "C" {

sparc_status sparc_device_bytes(const sparc_ctx *ctx, size_t *peak_bytes)
{
    if (!ctx || !peak_bytes) return SPARC_ERR_ARG;
    *peak_bytes = ctx->dev_peak;
    return SPARC_OK;
}

sparc_status sparc_sync(sparc_ctx *ctx)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    CK(cudaMemcpyAsync(ctx->pin_i + 14, ctx->flags + 14, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->pin_i[14] != 0) {
        CK(cudaMemsetAsync(ctx->flags + 14, 0, sizeof(int), ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return fail(ctx, SPARC_ERR_TIMEOUT, "a stencil launch timed out waiting for a TMA load");
    }
    return SPARC_OK;
}

sparc_status sparc_selftest_timeout(sparc_ctx *ctx, int which)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (which == 0) {
        CK(mbar_selftest(ctx->flags + 14, ctx->st));
        return sparc_sync(ctx);
    }
    if (which == 1) {
        int *status = ctx->flags + 6;
        CK(barrier_selftest(reinterpret_cast<GridBarrier *>(ctx->flags + 8), status, ctx->st));
        CK(cudaMemcpyAsync(ctx->pin_i, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemsetAsync(ctx->flags + 8, 0, sizeof(GridBarrier), ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if (ctx->pin_i[0] == 4) return fail(ctx, SPARC_ERR_TIMEOUT, "grid barrier timed out");
        return SPARC_OK;
    }
    return fail(ctx, SPARC_ERR_ARG, "which must be 0 (mbarrier) or 1 (grid barrier), got %d", which);
}


// --- after the rotation: occupations, density, non-local force ---------------------------
sparc_status sparc_occupations(sparc_ctx *ctx, const double *lambda_host, int ns, double nelec,
                               double kT, double *lambda_f_host, double *g_host)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (!lambda_host || !lambda_f_host) return fail(ctx, SPARC_ERR_ARG, "lambda and lambda_f must not be NULL");
    if (ns <= 0) return fail(ctx, SPARC_ERR_ARG, "ns must be positive (got %d)", ns);
    if (!(kT > 0.0) || !std::isfinite(kT)) return fail(ctx, SPARC_ERR_ARG, "kT must be positive and finite");
    if (!(nelec > 0.0) || !(nelec < 2.0 * ns))
        return fail(ctx, SPARC_ERR_ARG, "N_e must lie in (0, 2 ns) = (0, %d) (got %g)", 2 * ns, nelec);
    // workspace: lambda, g, mu, status
    TRY(ensure(ctx, ctx->obs, ctx->obs_bytes, sizeof(double) * (2 * (size_t)ns + 2)));
    double *lam = (double *)ctx->obs, *g = lam + ns, *mu = g + ns;
    int *status = (int *)(mu + 1);
    CK(cudaMemcpyAsync(lam, lambda_host, sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->st));
    { PHASE(SPARC_PHASE_OTHER); CK(fermi_level(lam, ns, nelec, kT, mu, g, status, ctx->st)); }
    int st = 0;
    CK(cudaMemcpyAsync(lambda_f_host, mu, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    if (g_host) CK(cudaMemcpyAsync(g_host, g, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (st == 2) return fail(ctx, SPARC_ERR_NONFINITE, "an eigenvalue is NaN or Inf");
    if (st != 0) return fail(ctx, SPARC_ERR_TIMEOUT, "the Fermi-level iteration did not converge");
    return SPARC_OK;
}

sparc_status sparc_density(sparc_ctx *ctx, sparc_dtype dtype, const void *X, int ncols, long ld,
                           const double *g_host, double *rho)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, X, ncols, ld, "X"));
    if (!g_host || !rho) return fail(ctx, SPARC_ERR_ARG, "g and rho must not be NULL");
    if (dtype != SPARC_F64 && dtype != SPARC_F32) return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
    TRY(ensure(ctx, ctx->obs, ctx->obs_bytes, sizeof(double) * (size_t)ncols));
    double *g = (double *)ctx->obs;
    CK(cudaMemcpyAsync(g, g_host, sizeof(double) * ncols, cudaMemcpyHostToDevice, ctx->st));
    PHASE(SPARC_PHASE_OTHER);
    if (dtype == SPARC_F64)
        CK(density<double>((const double *)X, ld, ncols, ctx->H.nd, g, ctx->H.h, rho, ctx->st));
    else
        CK(density<float>((const float *)X, ld, ncols, ctx->H.nd, g, ctx->H.h, rho, ctx->st));
    return SPARC_OK;
}

sparc_status sparc_nonlocal_force(sparc_ctx *ctx, sparc_dtype dtype, const void *X, int ncols,
                                  long ld, const double *g_host, double *force_host)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    TRY(check_block(ctx, X, ncols, ld, "X"));
    if (!g_host || !force_host) return fail(ctx, SPARC_ERR_ARG, "g and force must not be NULL");
    if (dtype != SPARC_F64 && dtype != SPARC_F32) return fail(ctx, SPARC_ERR_ARG, "unknown dtype %d", (int)dtype);
    const int na = ctx->H.natoms;
    if (na == 0) return SPARC_OK;
    // workspace: g, gamma, f, then the per (atom, column) projections y, w
    const size_t nw = (size_t)ncols + 4 * (size_t)na + 3 * (size_t)na + 16 * (size_t)na * ncols;
    TRY(ensure(ctx, ctx->obs, ctx->obs_bytes, sizeof(double) * nw));
    double *g = (double *)ctx->obs, *gam = g + ncols, *f = gam + 4 * (size_t)na,
           *yw = f + 3 * (size_t)na;
    CK(cudaMemcpyAsync(g, g_host, sizeof(double) * ncols, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(gam, ctx->gamma.data(), sizeof(double) * 4 * na, cudaMemcpyHostToDevice,
                       ctx->st));
    const GradCoef wg = grad_coef(ctx->H.radius, ctx->H.h);
    {
        PHASE(SPARC_PHASE_OTHER);
        if (dtype == SPARC_F64)
            CK(nonlocal_force<double>(ctx->H, (const double *)X, ld, ncols, g, gam, wg, yw, f, ctx->st));
        else
            CK(nonlocal_force<float>(ctx->H, (const float *)X, ld, ncols, g, gam, wg, yw, f, ctx->st));
    }
    CK(cudaMemcpyAsync(force_host, f, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SPARC_OK;
}

sparc_status sparc_poisson(sparc_ctx *ctx, const double *rho, double *phi, double tol, int maxit,
                           double *b_out, int *iters_host, double *relres_host)
{
    if (!ctx) return SPARC_ERR_ARG;
    ctx->err.clear();
    if (!phi) return fail(ctx, SPARC_ERR_ARG, "phi must not be NULL");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(ctx, SPARC_ERR_ARG, "tol must lie in (0, 1)");
    if (maxit <= 0) return fail(ctx, SPARC_ERR_ARG, "maxit must be positive (got %d)", maxit);
    const int na = ctx->H.natoms;
    if (na > 0 && ctx->atomZ.size() != (size_t)na)
        return fail(ctx, SPARC_ERR_ARG, "the context was created without valence charges Z");
    const DevHam &H = ctx->H;
    // the solver's workspace, then the atoms' positions and charges
    const size_t wb = (poisson_workspace(H.n0, H.n1, H.n2, H.radius) + 255) & ~(size_t)255;
    TRY(ensure(ctx, ctx->pois, ctx->pois_bytes, wb + sizeof(double) * (4 * (size_t)na + 1)));
    double *R = (double *)((unsigned char *)ctx->pois + wb);
    double *Z = R + 3 * (size_t)na;
    if (na > 0) {
        CK(cudaMemcpyAsync(R, ctx->atomR.data(), sizeof(double) * 3 * na, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(Z, ctx->atomZ.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->st));
    }
    int it = 0;
    double rel = 0.0;
    {
        PHASE(SPARC_PHASE_OTHER);
        CK(poisson_solve(H, R, Z, na, ctx->rc_erf, rho, phi, b_out, tol, maxit, ctx->pois, &it,
                         &rel, ctx->st));
    }
    if (iters_host) *iters_host = it;
    if (relres_host) *relres_host = rel;
    if (!(rel <= tol))
        return fail(ctx, SPARC_ERR_TIMEOUT, "CG stopped at relative residual %.3e after %d iterations", rel, it);
    return SPARC_OK;
}

}  // extern "C"

