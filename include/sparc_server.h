/* sparc_server.h -- request loop for cluster eigensolves on one GPU.
 *
 * The paper solves one cluster at a time (Sec. 3.4, Sec. 4); it has no counterpart of
 * this layer. A server runs CheFSI solves of clusters of different grid sizes and state
 * counts side by side: requests wait in arrival order, and each of `slots` worker threads
 * admits the first waiting request whose device-memory estimate fits in what is left of
 * the HBM budget (a request passed over kMaxPassOver = 8 times blocks later arrivals until
 * it fits). An admitted request owns a context (sparc_create) on its worker's CUDA stream,
 * its orbital blocks, V_eff, projector tables and filter bounds stay resident on the
 * device across its CheFSI iterations, and its kernels overlap with those of the other
 * admitted requests (one stream per worker). When a request finishes, its memory returns
 * to the budget and the next waiting requests are admitted (continuous batching at request
 * granularity). Every kernel of the library is deterministic, so a request's results do
 * not depend on what runs beside it.
 *
 * Solve of one request: Lanczos bounds (10 steps, seed), start block uniform in
 * (-0.5, 0.5) from splitmix64(seed, column, node), then CheFSI iterations
 * (sparc_chefsi_step, degree m, dtype F32 = mixed form or F64) until the largest residual
 * is <= tol or max_iters iterations have run.
 *
 * Thread safety: all calls may be made from any thread. Times are seconds on the host's
 * steady clock since the server was created. */
#ifndef SPARC_SERVER_H
#define SPARC_SERVER_H

#include <stddef.h>

#include "sparc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sparc_server sparc_server; /* opaque, owned by the library */

/* One eigensolve. Arrays are host memory and are copied by sparc_server_submit. */
typedef struct {
    int n[3];             /* grid nodes per axis */
    double h;             /* mesh size (bohr) */
    int natoms;
    const double *R;      /* 3 * natoms positions (bohr) */
    const double *Z;      /* natoms valence charges (V_eff built on the device) */
    const double *gamma;  /* 4 * natoms KB coefficients (s, px, py, pz) */
    int ns;               /* number of states (columns), 1..1024 */
    int degree;           /* Chebyshev degree m >= 1 */
    int max_iters;        /* CheFSI iterations at most (>= 1) */
    double tol;           /* stop once max residual <= tol */
    unsigned long long seed;
    sparc_dtype dtype;    /* SPARC_F32 (FP32 filter, FP64 Rayleigh-Ritz) or SPARC_F64 */
    double sim_seconds;   /* simulated servers only: how long the fake solve takes */
} sparc_request;

typedef struct {
    int status;           /* sparc_status of the solve */
    int iters;            /* CheFSI iterations run */
    int converged;        /* 1 if max residual <= tol */
    int ns;
    double t_submit, t_admit, t_done;  /* steady-clock seconds since server creation */
    size_t est_bytes;     /* device memory reserved from the budget */
    size_t used_bytes;    /* upper bound of what the solve held (context + blocks) */
} sparc_result_info;

/* Creates a server with `slots` worker threads (1..64) and an HBM budget in bytes.
 * simulate = 1 runs no GPU work: a solve sleeps sim_seconds and returns ns zero Ritz
 * values (for testing the admission logic without a GPU). */
sparc_status sparc_server_create(size_t hbm_budget_bytes, int slots, int simulate,
                                 sparc_server **out);

/* Creates a server in continuous-batching mode: one scheduler thread and one CUDA stream
 * run rounds, each one CheFSI iteration of every active request. The Chebyshev filters of
 * the active FP32-filter requests that share a degree run together through one
 * sparc_batch (each filter step's three kernels walk one work list spanning all of them,
 * include/sparc_batch.h); other requests are filtered on their own; then each request's
 * Rayleigh-Ritz step (sparc_orth_rr) runs. After a round, requests that converged or ran
 * out of iterations leave and their memory returns to the budget, and waiting requests
 * join (same admission rule as above) while fewer than max_active (1..1024) are active.
 * The batch uses one fixed kernel variant, so a request's results do not depend on which
 * other requests share its launches. Same solve per request as above; the rest of the API
 * is shared. */
sparc_status sparc_server_create_batched(size_t hbm_budget_bytes, int max_active,
                                         sparc_server **out);

/* Device memory a request will hold while it runs (context tables and workspaces plus its
 * two orbital blocks); the budget is charged this much on admission. */
size_t sparc_request_bytes(const sparc_request *req);

/* Queues a request; *id receives its handle. SPARC_ERR_BUDGET if its estimate exceeds
 * the whole budget, SPARC_ERR_ARG for invalid sizes. */
sparc_status sparc_server_submit(sparc_server *srv, const sparc_request *req, long long *id);

/* Waits up to timeout_s seconds (< 0: no limit) for request `id`. On completion fills
 * *info and, when not NULL, ritz[ns] and resid[ns] (ascending Ritz values of the last
 * iteration and their residual norms) and returns SPARC_OK; SPARC_ERR_TIMEOUT if the
 * request is still queued or running; SPARC_ERR_ARG for an unknown id. A result can be
 * read any number of times. */
sparc_status sparc_server_wait(sparc_server *srv, long long id, double timeout_s,
                               sparc_result_info *info, double *ritz, double *resid);

/* Counters: requests completed, the largest number running at once, and the largest
 * budget reservation seen (bytes). */
sparc_status sparc_server_stats(sparc_server *srv, long long *completed, int *max_running,
                                size_t *peak_reserved);

/* Stops admitting, waits for running requests to finish, marks queued ones as cancelled
 * (status SPARC_ERR_ARG) and frees the server. NULL is accepted. */
sparc_status sparc_server_destroy(sparc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SPARC_SERVER_H */
