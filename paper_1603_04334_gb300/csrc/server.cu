// server.cu -- request loop for cluster eigensolves on one GPU (include/sparc_server.h).
//
// A fixed pool of worker threads, one CUDA stream each; an arrival-ordered queue; an HBM
// budget charged with each request's device-memory estimate on admission and credited
// back when it finishes. A worker takes the first queued request that fits what is left
// of the budget, runs its whole solve on its own stream (context, blocks, bounds resident
// on the device throughout), publishes the result and takes the next one, so requests join
// while others run and their kernels overlap on the device. The estimate follows the
// library's own allocation rules (the same size helpers the context uses), and the solve
// reports an upper bound of what it actually held next to it.
#include "internal.cuh"
#include "sparc.h"
#include "sparc_batch.h"
#include "sparc_server.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace sparc {
namespace {

constexpr int kMaxPassOver = 8;
constexpr int kLanczosSteps = 10;
constexpr int kRrThreads = 8;  // host threads running the batched server's per-request steps

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// start block: X[c ld + p] = u(mix64(key ^ (c nd + p))) - 0.5, u(z) = (z >> 11) 2^-53
template <typename T>
__global__ void k_start_block(T *X, long nd, int ns, long ld, unsigned long long key)
{
    const long tot = nd * ns;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
         q += (long)gridDim.x * blockDim.x) {
        const long c = q / nd, p = q % nd;
        const double u = (double)(mix64(key ^ (unsigned long long)q) >> 11) * 0x1.0p-53;
        X[c * ld + p] = (T)(u - 0.5);
    }
}

unsigned long long host_mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Request {
    long long id = 0;
    sparc_request spec{};
    std::vector<double> R, Z, gamma;
    size_t est = 0;
    int passed_over = 0;
    bool done = false;
    sparc_result_info info{};
    std::vector<double> ritz, resid;
};

double now_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

long nodes_in_support_box(double h, double rcut)
{
    const long w = 2 * (long)std::ceil(rcut / h) + 1;  // cube around the sphere
    return w * w * w;
}

}  // namespace
}  // namespace sparc

using namespace sparc;

struct sparc_server {
    size_t budget = 0, reserved = 0, peak_reserved = 0;
    int slots = 0;
    bool simulate = false;
    bool batched = false;  // one scheduler thread, filters of all active requests batched
    int running = 0, max_running = 0;
    int device = 0;  // CUDA device of the creating thread; every worker uses it
    long long completed = 0, next_id = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::map<long long, std::unique_ptr<Request>> all;
    std::vector<std::thread> workers;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

// First queued request that fits what is left of the budget. Each waiting request ahead of
// the one admitted counts one pass-over; a request passed over kMaxPassOver times blocks
// the requests behind it until it fits.
Request *pick(sparc_server *S)
{
    const size_t left = S->budget - S->reserved;
    for (size_t i = 0; i < S->queue.size(); ++i) {
        Request *r = S->queue[i];
        if (r->est <= left) {
            for (size_t j = 0; j < i; ++j) S->queue[j]->passed_over++;
            S->queue.erase(S->queue.begin() + (long)i);
            return r;
        }
        if (r->passed_over >= kMaxPassOver) return nullptr;
    }
    return nullptr;
}

sparc_status solve(const Request &r, cudaStream_t st, sparc_result_info &info,
                   std::vector<double> &ritz, std::vector<double> &resid)
{
    const sparc_request &q = r.spec;
    const long nd = (long)q.n[0] * q.n[1] * q.n[2];
    const size_t es = q.dtype == SPARC_F32 ? 4 : 8;
    sparc_grid g{{q.n[0], q.n[1], q.n[2]}, q.h, kRadius};
    sparc_atoms a{q.natoms, r.R.data(), r.Z.data(), r.gamma.data(), 0.8, 3.0, 1.0};
    sparc_ctx *ctx = nullptr;
    sparc_status s = sparc_create(&g, nullptr, &a, st, &ctx);
    if (s != SPARC_OK) return s;
    void *X = nullptr, *W = nullptr;
    const size_t bb = es * (size_t)nd * q.ns;
    auto finish = [&](sparc_status rs) {
        size_t peak = 0;
        sparc_device_bytes(ctx, &peak);
        info.used_bytes = peak + (X ? bb : 0) + (W ? bb : 0);
        if (X) cudaFree(X);
        if (W) cudaFree(W);
        sparc_destroy(ctx);
        return rs;
    };
    if (cudaMalloc(&X, bb) != cudaSuccess || cudaMalloc(&W, bb) != cudaSuccess) {
        cudaGetLastError();
        return finish(SPARC_ERR_OOM);
    }
    const unsigned long long key = host_mix64(q.seed);
    if (q.dtype == SPARC_F32)
        k_start_block<float><<<152 * 8, 256, 0, st>>>((float *)X, nd, q.ns, nd, key);
    else
        k_start_block<double><<<152 * 8, 256, 0, st>>>((double *)X, nd, q.ns, nd, key);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return finish(SPARC_ERR_CUDA);
    double b[3];  // [a, b, a0] of the first iteration
    s = sparc_first_bounds(ctx, kLanczosSteps, q.seed, b);
    if (s != SPARC_OK) return finish(s);
    ritz.assign(q.ns, 0.0);
    resid.assign(q.ns, 0.0);
    for (int it = 0; it < q.max_iters; ++it) {
        s = sparc_chefsi_step(ctx, q.dtype, X, W, q.ns, nd, q.degree, b, ritz.data(),
                              resid.data());
        if (s != SPARC_OK) return finish(s);
        info.iters = it + 1;
        const double mr = *std::max_element(resid.begin(), resid.end());
        if (mr <= q.tol) {
            info.converged = 1;
            break;
        }
    }
    return finish(SPARC_OK);
}

void worker(sparc_server *S)
{
    cudaStream_t st = nullptr;
    if (!S->simulate && (cudaSetDevice(S->device) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess))
        st = nullptr;
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || (r = pick(S)) != nullptr; });
            if (!r) break;
            S->reserved += r->est;
            S->peak_reserved = std::max(S->peak_reserved, S->reserved);
            S->running++;
            S->max_running = std::max(S->max_running, S->running);
            r->info.t_admit = now_since(S->t0);
        }
        sparc_result_info info = r->info;
        std::vector<double> ritz, resid;
        sparc_status s;
        if (S->simulate) {
            std::this_thread::sleep_for(std::chrono::duration<double>(r->spec.sim_seconds));
            ritz.assign(r->spec.ns, 0.0);
            resid.assign(r->spec.ns, 0.0);
            info.iters = r->spec.max_iters;
            info.converged = 1;
            info.used_bytes = r->est;
            s = SPARC_OK;
        } else if (!st) {
            s = SPARC_ERR_CUDA;
        } else {
            s = solve(*r, st, info, ritz, resid);
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            info.status = s;
            info.t_done = now_since(S->t0);
            r->info = info;
            r->ritz = std::move(ritz);
            r->resid = std::move(resid);
            r->done = true;
            S->reserved -= r->est;
            S->running--;
            S->completed++;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

// ---- continuous batching: one scheduler thread, one stream -------------------------------
// Each round runs one CheFSI iteration of every active request: the Chebyshev filters of
// the FP32-filter requests that share the round's degree go through one sparc_batch (the
// three filter kernels of each step walk one work list over all of them), any other
// request is filtered on its own, then every request's Rayleigh-Ritz step runs. Between
// rounds, finished requests leave (their memory returns to the budget) and waiting
// requests join as the budget and the `slots` limit allow; the batch is rebuilt whenever
// the set of batched requests changes. The batch keeps its default kernel variant (no
// autotuning), so a request's arithmetic does not depend on which others share its
// launches. Each request has its own stream: once the batched filter is done, the
// requests' Rayleigh-Ritz steps (and the filters that were not batched) run side by side
// on a pool of host threads, one request per thread at a time.
struct Active {
    Request *r = nullptr;
    cudaStream_t st = nullptr;
    sparc_ctx *ctx = nullptr;
    void *X = nullptr, *W = nullptr;
    long nd = 0;
    double b[3] = {0, 0, 0};
    sparc_result_info info{};
    std::vector<double> ritz, resid;
    bool done = false;
    sparc_status status = SPARC_OK;
};

// Stream, context, blocks, start block and first-iteration bounds of an admitted request.
sparc_status start_active(Active &a)
{
    const sparc_request &q = a.r->spec;
    a.nd = (long)q.n[0] * q.n[1] * q.n[2];
    const size_t es = q.dtype == SPARC_F32 ? 4 : 8;
    if (cudaStreamCreateWithFlags(&a.st, cudaStreamNonBlocking) != cudaSuccess) {
        a.st = nullptr;
        return SPARC_ERR_CUDA;
    }
    cudaStream_t st = a.st;
    sparc_grid g{{q.n[0], q.n[1], q.n[2]}, q.h, kRadius};
    sparc_atoms at{q.natoms, a.r->R.data(), a.r->Z.data(), a.r->gamma.data(), 0.8, 3.0, 1.0};
    sparc_status s = sparc_create(&g, nullptr, &at, st, &a.ctx);
    if (s != SPARC_OK) return s;
    const size_t bb = es * (size_t)a.nd * q.ns;
    if (cudaMalloc(&a.X, bb) != cudaSuccess || cudaMalloc(&a.W, bb) != cudaSuccess) {
        cudaGetLastError();
        return SPARC_ERR_OOM;
    }
    const unsigned long long key = host_mix64(q.seed);
    if (q.dtype == SPARC_F32)
        k_start_block<float><<<152 * 8, 256, 0, st>>>((float *)a.X, a.nd, q.ns, a.nd, key);
    else
        k_start_block<double><<<152 * 8, 256, 0, st>>>((double *)a.X, a.nd, q.ns, a.nd, key);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return SPARC_ERR_CUDA;
    a.ritz.assign(q.ns, 0.0);
    a.resid.assign(q.ns, 0.0);
    return sparc_first_bounds(a.ctx, kLanczosSteps, q.seed, a.b);
}

void release_active(Active &a)
{
    const sparc_request &q = a.r->spec;
    const size_t bb = (q.dtype == SPARC_F32 ? 4 : 8) * (size_t)a.nd * q.ns;
    size_t peak = 0;
    if (a.ctx) sparc_device_bytes(a.ctx, &peak);
    a.info.used_bytes = peak + (a.X ? bb : 0) + (a.W ? bb : 0);
    if (a.X) cudaFree(a.X);
    if (a.W) cudaFree(a.W);
    if (a.ctx) sparc_destroy(a.ctx);
    if (a.st) cudaStreamDestroy(a.st);
    a.X = a.W = nullptr;
    a.ctx = nullptr;
    a.st = nullptr;
}

// Runs task(i) for i < n on `threads` host threads (the calling thread included), each
// with `device` current; returns when all are done.
template <typename F>
void run_parallel(int n, int threads, int device, F task)
{
    std::atomic<int> next{0};
    auto body = [&](bool set_device) {
        if (set_device) cudaSetDevice(device);
        for (int i; (i = next.fetch_add(1)) < n;) task(i);
    };
    const int extra = std::min(threads, n) - 1;
    std::vector<std::thread> pool;
    for (int t = 0; t < extra; ++t) pool.emplace_back(body, true);
    body(false);
    for (std::thread &t : pool) t.join();
}

// Rayleigh-Ritz of one request after its filter; bounds for the next round as
// sparc_chefsi_step sets them (a = largest, a0 = smallest Ritz value).
void rr_active(Active &a)
{
    const sparc_request &q = a.r->spec;
    sparc_status s = sparc_orth_rr(a.ctx, q.dtype, a.X, nullptr, q.ns, a.nd, a.ritz.data(),
                                   a.resid.data());
    a.info.iters++;
    if (s != SPARC_OK) {
        a.status = s;
        a.done = true;
        return;
    }
    a.b[0] = *std::max_element(a.ritz.begin(), a.ritz.end());
    a.b[2] = *std::min_element(a.ritz.begin(), a.ritz.end());
    if (*std::max_element(a.resid.begin(), a.resid.end()) <= q.tol) {
        a.info.converged = 1;
        a.done = true;
    } else if (a.info.iters >= q.max_iters) {
        a.done = true;
    }
}

void scheduler(sparc_server *S)
{
    cudaStream_t st = nullptr;
    const bool gpu_ok = cudaSetDevice(S->device) == cudaSuccess &&
                        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    std::vector<std::unique_ptr<Active>> act;
    sparc_batch *batch = nullptr;
    std::vector<sparc_ctx *> batch_ctxs;
    for (;;) {
        // admit waiting requests while slots and budget allow (block when nothing runs)
        std::vector<Request *> joined;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (act.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && act.empty()) break;
            Request *r;
            while (!S->stop && (int)act.size() + (int)joined.size() < S->slots &&
                   (r = pick(S)) != nullptr) {
                S->reserved += r->est;
                S->peak_reserved = std::max(S->peak_reserved, S->reserved);
                S->running++;
                S->max_running = std::max(S->max_running, S->running);
                r->info.t_admit = now_since(S->t0);
                joined.push_back(r);
            }
        }
        for (Request *r : joined) {
            auto a = std::make_unique<Active>();
            a->r = r;
            a->info = r->info;
            a->status = gpu_ok ? start_active(*a) : SPARC_ERR_CUDA;
            if (a->status != SPARC_OK) a->done = true;
            act.push_back(std::move(a));
        }
        if (act.empty()) continue;
        // the round: batched filters, then the other filters, then every Rayleigh-Ritz
        int degree = -1;
        std::vector<Active *> bat;
        for (auto &a : act) {
            if (a->done || a->r->spec.dtype != SPARC_F32) continue;
            if (degree < 0) degree = a->r->spec.degree;
            if (a->r->spec.degree == degree) bat.push_back(a.get());
        }
        std::vector<sparc_ctx *> want;
        for (Active *a : bat) want.push_back(a->ctx);
        if (want != batch_ctxs) {
            sparc_batch_destroy(batch);
            batch = nullptr;
            batch_ctxs.clear();
            if (!want.empty() && sparc_batch_create(want.data(), (int)want.size(), st, &batch) ==
                                     SPARC_OK)
                batch_ctxs = want;
        }
        if (!bat.empty()) {
            std::vector<float *> X, W;
            std::vector<int> nc;
            std::vector<long> ld;
            std::vector<double> bounds;
            for (Active *a : bat) {
                X.push_back((float *)a->X);
                W.push_back((float *)a->W);
                nc.push_back(a->r->spec.ns);
                ld.push_back(a->nd);
                bounds.insert(bounds.end(), a->b, a->b + 3);
            }
            sparc_status s =
                batch ? sparc_batch_filter(batch, X.data(), W.data(), nc.data(), ld.data(), degree,
                                           bounds.data())
                      : SPARC_ERR_OOM;
            // the batch ends on the scheduler's stream; the requests' own streams take over
            if (s == SPARC_OK && cudaStreamSynchronize(st) != cudaSuccess) s = SPARC_ERR_CUDA;
            if (s != SPARC_OK)
                for (Active *a : bat) a->status = s, a->done = true;
        }
        std::vector<Active *> todo;
        for (auto &a : act)
            if (!a->done) todo.push_back(a.get());
        run_parallel((int)todo.size(), kRrThreads, S->device, [&](int i) {
            Active &a = *todo[i];
            const bool batched = std::find(bat.begin(), bat.end(), &a) != bat.end();
            if (!batched) {
                const sparc_request &q = a.r->spec;
                const sparc_status s = sparc_cheb_filter(a.ctx, q.dtype, a.X, a.W, q.ns, a.nd,
                                                         q.degree, a.b[0], a.b[1], a.b[2]);
                if (s != SPARC_OK) {
                    a.status = s;
                    a.done = true;
                    return;
                }
            }
            rr_active(a);
        });
        // finished requests leave; the batch over them goes first (it uses their contexts)
        bool left = false;
        for (auto &a : act) left = left || a->done;
        if (!left) continue;
        sparc_batch_destroy(batch);
        batch = nullptr;
        batch_ctxs.clear();
        for (auto it = act.begin(); it != act.end();) {
            Active &a = **it;
            if (!a.done) {
                ++it;
                continue;
            }
            release_active(a);
            {
                std::lock_guard<std::mutex> lk(S->mu);
                Request *r = a.r;
                a.info.status = a.status;
                a.info.t_done = now_since(S->t0);
                r->info = a.info;
                r->ritz = std::move(a.ritz);
                r->resid = std::move(a.resid);
                r->done = true;
                S->reserved -= r->est;
                S->running--;
                S->completed++;
            }
            S->cv_done.notify_all();
            it = act.erase(it);
        }
    }
    sparc_batch_destroy(batch);
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

size_t sparc_request_bytes(const sparc_request *q)
{
    if (!q) return 0;
    const long nd = (long)q->n[0] * q->n[1] * q->n[2];
    const int ns = q->ns;
    const size_t es = q->dtype == SPARC_F32 ? 4 : 8;
    const size_t na = q->natoms > 0 ? (size_t)q->natoms : 1;
    // context: V_eff (FP64, FP32) and set-up scratch per node, projector entries (index,
    // chi and gamma chi in FP64 / FP32 / pairs, inverse map), bounded by the cube around
    // each support sphere
    const size_t per_node = 8 + 4 + 4 * 8 + 8;
    const size_t per_entry = 4 + 4 + 32 + 32 + 16 + 16 + 32 + 4 + 4 + 16 + 32 + 16;
    const size_t entries = na * (size_t)nodes_in_support_box(q->h, 3.0);
    size_t b = per_node * (size_t)nd + per_entry * entries + 4096 * 64;
    // workspaces: projection coefficients, H Y_f (FP64), rotated H X (residuals), the
    // tensor-core Gram of either form, Ns x Ns matrices, Lanczos
    b += sizeof(double) * 4 * na * ns;
    b += sizeof(double) * (size_t)nd * ns;
    b += es * (size_t)nd * ns;
    // tensor-core Gram and rotation (one workspace, sized for a slab of rows, and the slab
    // Grams' sums)
    const bool mixed = q->dtype == SPARC_F32;
    b += tc_slab_workspace(nd, ns, mixed);
    if (tc_slab_rows(nd, ns, mixed) < nd) b += sizeof(double) * 2 * (size_t)ns * ns;
    if (!mixed) {
        // column bounds of the filter's blocks, alpha (V_eff - shift) of a step
        b += sizeof(unsigned) * ((size_t)(q->degree + 1) * ns + (size_t)ns);
        b += 8 * (size_t)nd;
    }
    b += sizeof(double) * (4 * (size_t)ns * ns + 2 * (size_t)ns + (size_t)dense_work_elems(ns));
    b += sizeof(double) * (3 * (size_t)nd + kDotBlocks + 4096);
    // the request's two orbital blocks
    b += 2 * es * (size_t)nd * ns;
    return b + b / 16;  // allocation granularity
}

sparc_status sparc_server_create(size_t hbm_budget_bytes, int slots, int simulate,
                                 sparc_server **out)
{
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes == 0) return SPARC_ERR_ARG;
    sparc_server *S = new (std::nothrow) sparc_server();
    if (!S) return SPARC_ERR_OOM;
    S->budget = hbm_budget_bytes;
    S->slots = slots;
    S->simulate = simulate != 0;
    if (!S->simulate && cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return SPARC_ERR_CUDA;
    }
    for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S);
    *out = S;
    return SPARC_OK;
}

sparc_status sparc_server_create_batched(size_t hbm_budget_bytes, int max_active,
                                         sparc_server **out)
{
    if (!out || max_active < 1 || max_active > 1024 || hbm_budget_bytes == 0)
        return SPARC_ERR_ARG;
    sparc_server *S = new (std::nothrow) sparc_server();
    if (!S) return SPARC_ERR_OOM;
    S->budget = hbm_budget_bytes;
    S->slots = max_active;
    S->batched = true;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return SPARC_ERR_CUDA;
    }
    S->workers.emplace_back(scheduler, S);
    *out = S;
    return SPARC_OK;
}

sparc_status sparc_server_submit(sparc_server *S, const sparc_request *q, long long *id)
{
    if (!S || !q || !id) return SPARC_ERR_ARG;
    if (q->n[0] < 1 || q->n[1] < 1 || q->n[2] < 1 || !(q->h > 0) || q->ns < 1 ||
        q->ns > kMaxDense || q->degree < 1 || q->max_iters < 1 || q->natoms < 0 ||
        (q->natoms > 0 && (!q->R || !q->Z || !q->gamma)) ||
        (q->dtype != SPARC_F32 && q->dtype != SPARC_F64) ||
        (long)q->n[0] * q->n[1] * q->n[2] < q->ns)
        return SPARC_ERR_ARG;
    auto r = std::make_unique<Request>();
    r->spec = *q;
    r->R.assign(q->R ? q->R : nullptr, q->R ? q->R + 3 * (size_t)q->natoms : nullptr);
    r->Z.assign(q->Z ? q->Z : nullptr, q->Z ? q->Z + (size_t)q->natoms : nullptr);
    r->gamma.assign(q->gamma ? q->gamma : nullptr, q->gamma ? q->gamma + 4 * (size_t)q->natoms : nullptr);
    r->spec.R = r->spec.Z = r->spec.gamma = nullptr;
    r->est = sparc_request_bytes(q);
    if (r->est > S->budget) return SPARC_ERR_BUDGET;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return SPARC_ERR_ARG;
        r->id = S->next_id++;
        r->info.ns = q->ns;
        r->info.est_bytes = r->est;
        r->info.t_submit = now_since(S->t0);
        r->info.t_admit = r->info.t_done = -1.0;
        *id = r->id;
        S->queue.push_back(r.get());
        S->all.emplace(r->id, std::move(r));
    }
    S->cv_work.notify_all();
    return SPARC_OK;
}

sparc_status sparc_server_wait(sparc_server *S, long long id, double timeout_s,
                               sparc_result_info *info, double *ritz, double *resid)
{
    if (!S) return SPARC_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return SPARC_ERR_ARG;
    Request *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_s < 0)
        S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        return SPARC_ERR_TIMEOUT;
    if (info) *info = r->info;
    if (ritz && !r->ritz.empty()) std::memcpy(ritz, r->ritz.data(), sizeof(double) * r->ritz.size());
    if (resid && !r->resid.empty())
        std::memcpy(resid, r->resid.data(), sizeof(double) * r->resid.size());
    return SPARC_OK;
}

sparc_status sparc_server_stats(sparc_server *S, long long *completed, int *max_running,
                                size_t *peak_reserved)
{
    if (!S) return SPARC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (completed) *completed = S->completed;
    if (max_running) *max_running = S->max_running;
    if (peak_reserved) *peak_reserved = S->peak_reserved;
    return SPARC_OK;
}

sparc_status sparc_server_destroy(sparc_server *S)
{
    if (!S) return SPARC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request *r : S->queue) {
            r->info.status = SPARC_ERR_ARG;
            r->done = true;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (std::thread &t : S->workers) t.join();
    delete S;
    return SPARC_OK;
}

}  // extern "C"
