// batch.cu -- Chebyshev filter steps of many clusters in shared launches
// (include/sparc_batch.h).
//
// Host side: the work lists (one per kernel, spanning every cluster), the per-step tables
// of pointers and coefficients (the recurrence of Algorithm ChebychevFilter, Sec. 3.4, per
// cluster: sigma_1 = e / (a0 - c), sigma_j = 1 / (2 / sigma_1 - sigma_{j-1}), step j
// writes (2 sigma_j / e)(H - c) Y_{j-1} - sigma_{j-1} sigma_j Y_{j-2} over Y_{j-2}), the
// CUDA graph of the m steps, and the autotuner over tile shape x z split. The kernels are
// k_batch_stencil (stencil.cu) and k_batch_project / k_batch_scatter (nonlocal.cu), which
// share their per-tile code with the single-cluster kernels.
#include "internal.cuh"
#include "sparc.h"
#include "sparc_batch.h"

#include <cstring>
#include <vector>

using namespace sparc;

namespace {
constexpr int kZSplits[3] = {1, 2, 4};
// stencil forms: shared-memory tiles 32 x 8, 32 x 16, 64 x 8; the TMA-fed 32 x 16 on a
// persistent grid (form 3: one ring per CTA across its items) or with one CTA per item
// (form 4: the scheduling of the single-cluster launches); forms 3 and 4 for blocks the TMA
// path accepts. Each with 1, 2 or 4 z ranges per column.
constexpr int kForms = 5, kTmaForm = 3, kTmaItemForm = 4;
constexpr int kVariants = kForms * 3;
constexpr int kDefaultVariant = kTmaItemForm * 3;  // TMA, one CTA per item, whole z range

// Persistent grids: enough resident CTAs to fill the 152 SMs several times.
constexpr int kGridStencil = 152 * 8;
constexpr int kGridTma = 152 * 3;
constexpr int kGridProject = 152 * 2;
constexpr int kGridScatter = 152 * 6;

struct Key {
    std::vector<const void *> X, W;
    std::vector<int> ncols;
    std::vector<long> ld;
    int degree = -1, variant = -1;
    bool operator==(const Key &o) const
    {
        return X == o.X && W == o.W && ncols == o.ncols && ld == o.ld && degree == o.degree &&
               variant == o.variant;
    }
};
}  // namespace

struct sparc_batch {
    std::vector<sparc_ctx *> ctx;
    // batched work runs on a private stream (graph capture needs a non-default stream),
    // ordered after the caller's stream on entry and before it on exit through events
    cudaStream_t user_st = nullptr, st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int variant = kDefaultVariant;
    int form = 0;  // stencil form of the current work lists
    // device work lists
    BatchItem *items = nullptr;
    size_t items_cap = 0;
    int n_st = 0, n_pr = 0, n_sc = 0;
    // per-step tables: pinned host copy and device copy
    BatchStencil *h_st = nullptr, *d_st = nullptr;
    BatchNonlocal *h_nl = nullptr, *d_nl = nullptr;
    BatchTma *h_tm = nullptr, *d_tm = nullptr;
    size_t steps_cap = 0;
    // tensor maps per cluster: X halo, X tile, W halo, W tile (device, 64-byte aligned)
    unsigned char *maps = nullptr;
    size_t maps_cap = 0;
    bool tma = false;  // every block accepted by the TMA path
    cudaGraphExec_t exec = nullptr;
    Key key;
    bool any_atoms = false;
};

namespace {

void free_tables(sparc_batch *b)
{
    if (b->items) cudaFree(b->items);
    if (b->d_st) cudaFree(b->d_st);
    if (b->d_nl) cudaFree(b->d_nl);
    if (b->h_st) cudaFreeHost(b->h_st);
    if (b->h_nl) cudaFreeHost(b->h_nl);
    if (b->d_tm) cudaFree(b->d_tm);
    if (b->h_tm) cudaFreeHost(b->h_tm);
    if (b->maps) cudaFree(b->maps);
    b->d_tm = nullptr;
    b->h_tm = nullptr;
    b->maps = nullptr;
    b->maps_cap = 0;
    b->items = nullptr;
    b->d_st = nullptr;
    b->d_nl = nullptr;
    b->h_st = nullptr;
    b->h_nl = nullptr;
    b->items_cap = b->steps_cap = 0;
}

// Work lists for the current variant and column counts (uploaded synchronously).
sparc_status build_items(sparc_batch *b, const int *ncols)
{
    int bx, by;
    if (b->form >= kTmaForm)
        batch_tma_tile(bx, by);
    else
        batch_stencil_tile(b->form, bx, by);
    const int zs = kZSplits[b->variant % 3];
    std::vector<BatchItem> st, pr, sc;
    b->any_atoms = false;
    for (size_t c = 0; c < b->ctx.size(); ++c) {
        const DevHam &H = *ctx_ham(b->ctx[c]);
        const int gx = (H.n0 + bx - 1) / bx, gy = (H.n1 + by - 1) / by;
        int nzc = zs;
        while (nzc > 1 && H.n2 / nzc < 16) nzc /= 2;
        const int zch = (H.n2 + nzc - 1) / nzc;
        for (int col = 0; col < ncols[c]; ++col)
            for (int z = 0; z < nzc; ++z)
                for (int y = 0; y < gy; ++y)
                    for (int x = 0; x < gx; ++x) {
                        const int k0 = z * zch, k1 = k0 + zch < H.n2 ? k0 + zch : H.n2;
                        if (k0 < k1) st.push_back({(int)c, col, x, y, k0, k1});
                    }
        if (H.natoms > 0) {
            b->any_atoms = true;
            for (int J = 0; J < H.natoms; ++J)
                for (int col = 0; col < ncols[c]; col += kBatchCols)
                    pr.push_back({(int)c, col, J, 0, 0, 0});
            const long chunks = (H.nuniq + kBatchNodes - 1) / kBatchNodes;
            for (long u = 0; u < chunks; ++u)
                for (int col = 0; col < ncols[c]; col += kBatchCols)
                    sc.push_back({(int)c, col, (int)u, 0, 0, 0});
        }
    }
    const size_t tot = st.size() + pr.size() + sc.size();
    if (tot > 0x7fffffff) return SPARC_ERR_ARG;
    if (b->form == kTmaForm) {
        // the persistent TMA kernel numbers the planes of each CTA's items in 32 bits
        std::vector<long long> planes(kGridTma, 0);
        for (size_t i = 0; i < st.size(); ++i)
            planes[i % kGridTma] += (st[i].k1 - st[i].k0) + 2 * kRadius;
        for (long long v : planes)
            if (v >= (1LL << 31)) return SPARC_ERR_ARG;
    }
    if (tot > b->items_cap) {
        if (b->items) cudaFree(b->items);
        b->items = nullptr;
        b->items_cap = 0;
        if (cudaMalloc(&b->items, sizeof(BatchItem) * tot) != cudaSuccess) return SPARC_ERR_OOM;
        b->items_cap = tot;
    }
    std::vector<BatchItem> all;
    all.reserve(tot);
    all.insert(all.end(), st.begin(), st.end());
    all.insert(all.end(), pr.begin(), pr.end());
    all.insert(all.end(), sc.begin(), sc.end());
    if (tot && cudaMemcpy(b->items, all.data(), sizeof(BatchItem) * tot,
                          cudaMemcpyHostToDevice) != cudaSuccess)
        return SPARC_ERR_CUDA;
    b->n_st = (int)st.size();
    b->n_pr = (int)pr.size();
    b->n_sc = (int)sc.size();
    return SPARC_OK;
}

sparc_status ensure_steps(sparc_batch *b, int degree)
{
    const size_t need = (size_t)degree * b->ctx.size();
    if (need <= b->steps_cap) return SPARC_OK;
    if (b->d_st) cudaFree(b->d_st);
    if (b->d_nl) cudaFree(b->d_nl);
    if (b->h_st) cudaFreeHost(b->h_st);
    if (b->h_nl) cudaFreeHost(b->h_nl);
    if (b->d_tm) cudaFree(b->d_tm);
    if (b->h_tm) cudaFreeHost(b->h_tm);
    b->d_st = nullptr;
    b->d_nl = nullptr;
    b->h_st = nullptr;
    b->h_nl = nullptr;
    b->d_tm = nullptr;
    b->h_tm = nullptr;
    b->steps_cap = 0;
    if (cudaMalloc(&b->d_st, sizeof(BatchStencil) * need) != cudaSuccess ||
        cudaMalloc(&b->d_nl, sizeof(BatchNonlocal) * need) != cudaSuccess ||
        cudaMalloc(&b->d_tm, sizeof(BatchTma) * need) != cudaSuccess ||
        cudaMallocHost(&b->h_st, sizeof(BatchStencil) * need) != cudaSuccess ||
        cudaMallocHost(&b->h_nl, sizeof(BatchNonlocal) * need) != cudaSuccess ||
        cudaMallocHost(&b->h_tm, sizeof(BatchTma) * need) != cudaSuccess)
        return SPARC_ERR_OOM;
    b->steps_cap = need;
    return SPARC_OK;
}

// Per step and cluster: pointers (ping-pong between X and W) and coefficients.
void fill_steps(sparc_batch *b, float *const *X, float *const *W, const int *ncols,
                const long *ld, int degree, const double *bounds, float *const *C)
{
    const size_t n = b->ctx.size();
    for (size_t c = 0; c < n; ++c) {
        const DevHam &H = *ctx_ham(b->ctx[c]);
        const double a = bounds[3 * c], bb = bounds[3 * c + 1], a0 = bounds[3 * c + 2];
        const double e = (bb - a) / 2.0, cc = (bb + a) / 2.0;
        const double s1 = e / (a0 - cc);
        float *cur = X[c], *prev = nullptr, *out = W[c];
        double sigma = s1;
        for (int j = 1; j <= degree; ++j) {
            double alpha, beta;
            if (j == 1) {
                alpha = s1 / e;
                beta = 0.0;
            } else {
                const double sn = 1.0 / (2.0 / s1 - sigma);
                alpha = 2.0 * sn / e;
                beta = sigma * sn;
                sigma = sn;
                out = prev;
            }
            BatchStencil &S = b->h_st[(size_t)(j - 1) * n + c];
            S.Y = cur;
            S.Yprev = j == 1 ? nullptr : prev;
            S.out = out;
            S.V = H.Vf;
            S.n0 = H.n0;
            S.n1 = H.n1;
            S.n2 = H.n2;
            S.ld = ld[c];
            S.cf = coef_f32(H, alpha, cc, beta);
            BatchNonlocal &P = b->h_nl[(size_t)(j - 1) * n + c];
            P.Y = cur;
            P.out = out;
            P.C = C[c];
            P.atom_ptr = H.atom_ptr;
            P.idx = H.idx;
            P.uniq_node = H.uniq_node;
            P.uniq_ptr = H.uniq_ptr;
            P.nl_atom = H.nl_atom;
            P.chi_f = H.chi_f;
            P.nl_gf = H.nl_gf;
            P.ld = ld[c];
            P.nuniq = H.nuniq;
            P.ncols = ncols[c];
            P.alpha = (float)alpha;
            if (b->tma) {
                const size_t mb = tensor_map_bytes();
                const unsigned char *m = b->maps + 4 * mb * c;
                BatchTma &M = b->h_tm[(size_t)(j - 1) * n + c];
                M.mY = m + (cur == X[c] ? 0 : 2) * mb;
                M.mP = j == 1 ? nullptr : m + ((prev == X[c] ? 0 : 2) + 1) * mb;
                M.out = out;
                M.V = H.Vf;
                M.n0 = H.n0;
                M.n1 = H.n1;
                M.n2 = H.n2;
                M.ld = ld[c];
                M.cf = S.cf;
            }
            // the step's output becomes the next input; its input the next Y_{j-1}
            float *t = cur;
            cur = out;
            prev = t;
        }
    }
}

// Enqueues (or captures) the m steps and the final copies back into X.
cudaError_t enqueue_steps(sparc_batch *b, float *const *X, float *const *W, const int *ncols,
                          const long *ld, int degree)
{
    const size_t n = b->ctx.size();
    const BatchItem *st_items = b->items, *pr_items = b->items + b->n_st,
                    *sc_items = b->items + b->n_st + b->n_pr;
    cudaError_t e;
    for (int j = 0; j < degree; ++j) {
        const BatchStencil *S = b->d_st + (size_t)j * n;
        const BatchNonlocal *P = b->d_nl + (size_t)j * n;
        if (b->any_atoms && (e = batch_project(pr_items, b->n_pr, P, kGridProject, b->st)))
            return e;
        if (b->form >= kTmaForm) {
            const int grid = b->form == kTmaItemForm ? b->n_st : kGridTma;
            e = batch_stencil_tma(st_items, b->n_st, b->d_tm + (size_t)j * n, grid,
                                  ctx_ham(b->ctx[0])->err, b->st);
        } else {
            e = batch_stencil(b->form, st_items, b->n_st, S, kGridStencil, b->st);
        }
        if (e) return e;
        if (b->any_atoms && (e = batch_scatter(sc_items, b->n_sc, P, kGridScatter, b->st)))
            return e;
    }
    // after m steps the result sits in W for odd m (X for even m)
    if (degree % 2 == 1)
        for (size_t c = 0; c < n; ++c) {
            const long nd = ctx_ham(b->ctx[c])->nd;
            e = cudaMemcpy2DAsync(X[c], ld[c] * sizeof(float), W[c], ld[c] * sizeof(float),
                                  nd * sizeof(float), ncols[c], cudaMemcpyDeviceToDevice, b->st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

sparc_status run_filter(sparc_batch *b, float *const *X, float *const *W, const int *ncols,
                        const long *ld, int degree, const double *bounds)
{
    const size_t n = b->ctx.size();
    if (!X || !W || !ncols || !ld || !bounds || degree < 1) return SPARC_ERR_ARG;
    std::vector<float *> C(n);
    for (size_t c = 0; c < n; ++c) {
        const DevHam &H = *ctx_ham(b->ctx[c]);
        if (!X[c] || !W[c] || X[c] == W[c] || ncols[c] < 1 || ld[c] < H.nd) return SPARC_ERR_ARG;
        const double a = bounds[3 * c], bb = bounds[3 * c + 1], a0 = bounds[3 * c + 2];
        if (!(a0 < a && a < bb)) return SPARC_ERR_ARG;
        C[c] = ctx_coef_buffer(b->ctx[c], ncols[c]);  // allocations happen before any capture
        if (!C[c]) return SPARC_ERR_OOM;
    }
    Key k;
    k.X.assign(X, X + n);
    k.W.assign(W, W + n);
    k.ncols.assign(ncols, ncols + n);
    k.ld.assign(ld, ld + n);
    k.degree = degree;
    k.variant = b->variant;
    const bool same = b->exec && k == b->key;
    sparc_status s;
    if (!same) {
        // the TMA form needs every block in the layout its loads accept; else the
        // shared-memory form with the same tile
        bool ok = true;
        for (size_t c = 0; c < n; ++c)
            ok = ok && stencil_tma_ok(*ctx_ham(b->ctx[c]), X[c], W[c], W[c], ld[c]) &&
                 stencil_tma_ok(*ctx_ham(b->ctx[c]), W[c], X[c], X[c], ld[c]);
        b->form = b->variant / 3;
        if (b->form >= kTmaForm && !ok) b->form = 1;
        b->tma = b->form >= kTmaForm;
        if (b->tma) {
            const size_t mb = tensor_map_bytes(), need = 4 * mb * n;
            if (need > b->maps_cap) {
                if (b->maps) cudaFree(b->maps);
                b->maps = nullptr;
                b->maps_cap = 0;
                if (cudaMalloc(&b->maps, need) != cudaSuccess) return SPARC_ERR_OOM;
                b->maps_cap = need;
            }
            std::vector<unsigned char> hm(need);
            for (size_t c = 0; c < n; ++c) {
                const DevHam &H = *ctx_ham(b->ctx[c]);
                if (encode_f32_maps(H, X[c], ncols[c], ld[c], hm.data() + 4 * mb * c) != cudaSuccess ||
                    encode_f32_maps(H, W[c], ncols[c], ld[c], hm.data() + 4 * mb * c + 2 * mb) != cudaSuccess)
                    return SPARC_ERR_CUDA;
            }
            if (cudaMemcpy(b->maps, hm.data(), need, cudaMemcpyHostToDevice) != cudaSuccess)
                return SPARC_ERR_CUDA;
        }
        if ((s = build_items(b, ncols)) != SPARC_OK) return s;
        if ((s = ensure_steps(b, degree)) != SPARC_OK) return s;
    }
    // the pinned table may still be in flight from the previous call
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return SPARC_ERR_CUDA;
    if (cudaEventRecord(b->ev_in, b->user_st) != cudaSuccess ||
        cudaStreamWaitEvent(b->st, b->ev_in, 0) != cudaSuccess)
        return SPARC_ERR_CUDA;
    fill_steps(b, X, W, ncols, ld, degree, bounds, C.data());
    const size_t bytes_st = sizeof(BatchStencil) * (size_t)degree * n;
    const size_t bytes_nl = sizeof(BatchNonlocal) * (size_t)degree * n;
    if (cudaMemcpyAsync(b->d_st, b->h_st, bytes_st, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_nl, b->h_nl, bytes_nl, cudaMemcpyHostToDevice, b->st) != cudaSuccess)
        return SPARC_ERR_CUDA;
    if (b->tma && cudaMemcpyAsync(b->d_tm, b->h_tm, sizeof(BatchTma) * (size_t)degree * n,
                                  cudaMemcpyHostToDevice, b->st) != cudaSuccess)
        return SPARC_ERR_CUDA;
    if (!same) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return SPARC_ERR_CUDA;
        const cudaError_t e = enqueue_steps(b, X, W, ncols, ld, degree);
        const cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return SPARC_ERR_CUDA;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            b->exec = nullptr;
            return SPARC_ERR_CUDA;
        }
        b->key = k;
    }
    if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return SPARC_ERR_CUDA;
    if (cudaEventRecord(b->ev_out, b->st) != cudaSuccess ||
        cudaStreamWaitEvent(b->user_st, b->ev_out, 0) != cudaSuccess)
        return SPARC_ERR_CUDA;
    return SPARC_OK;
}

}  // namespace

extern "C" {

sparc_status sparc_batch_create(sparc_ctx *const *ctxs, int n, void *cuda_stream,
                                sparc_batch **out)
{
    if (!ctxs || n < 1 || !out) return SPARC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return SPARC_ERR_ARG;
    sparc_batch *b = new (std::nothrow) sparc_batch();
    if (!b) return SPARC_ERR_OOM;
    b->ctx.assign(ctxs, ctxs + n);
    b->user_st = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        sparc_batch_destroy(b);
        return SPARC_ERR_CUDA;
    }
    *out = b;
    return SPARC_OK;
}

sparc_status sparc_batch_filter(sparc_batch *b, float *const *X, float *const *W,
                                const int *ncols, const long *ld, int degree,
                                const double *bounds)
{
    if (!b) return SPARC_ERR_ARG;
    return run_filter(b, X, W, ncols, ld, degree, bounds);
}

sparc_status sparc_batch_variant(sparc_batch *b, int variant, int *count)
{
    if (!b) return SPARC_ERR_ARG;
    if (count) *count = kVariants;
    if (variant < 0) return SPARC_OK;
    if (variant >= kVariants) return SPARC_ERR_ARG;
    b->variant = variant;
    return SPARC_OK;
}

sparc_status sparc_batch_tune(sparc_batch *b, float *const *X, float *const *W,
                              const int *ncols, const long *ld, int degree,
                              const double *bounds, int *variant, double *ms)
{
    if (!b) return SPARC_ERR_ARG;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SPARC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SPARC_ERR_CUDA;
    }
    int best = -1;
    float best_ms = 0.0f;
    sparc_status s = SPARC_OK;
    for (int v = 0; v < kVariants && s == SPARC_OK; ++v) {
        b->variant = v;
        if ((s = run_filter(b, X, W, ncols, ld, degree, bounds)) != SPARC_OK) break;  // warm-up
        float t = 0.0f;
        if (cudaEventRecord(e0, b->st) != cudaSuccess) { s = SPARC_ERR_CUDA; break; }
        for (int r = 0; r < 2 && s == SPARC_OK; ++r) s = run_filter(b, X, W, ncols, ld, degree, bounds);
        if (s != SPARC_OK) break;
        if (cudaEventRecord(e1, b->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            s = SPARC_ERR_CUDA;
            break;
        }
        t /= 2.0f;
        if (best < 0 || t < best_ms) {
            best = v;
            best_ms = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SPARC_OK) return s;
    b->variant = best;
    if (variant) *variant = best;
    if (ms) *ms = best_ms;
    return SPARC_OK;
}

sparc_status sparc_batch_destroy(sparc_batch *b)
{
    if (!b) return SPARC_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_tables(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
    return SPARC_OK;
}

}  // extern "C"
