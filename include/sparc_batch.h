/* sparc_batch.h -- Chebyshev filter steps of many uneven clusters in shared launches.
 *
 * The paper filters one cluster at a time (Algorithm ChebychevFilter, Sec. 3.4); this
 * layer has no counterpart there. A batch groups contexts (one cluster each, created by
 * sparc_create on the same device) and runs the FP32 filter of all their blocks together:
 * each filter step is three persistent launches -- projection chi^T Y, fused stencil +
 * V_eff + recurrence, nonlocal scatter -- whose CTAs walk one work list spanning every
 * cluster (items: cluster x column x x-y tile x z range for the stencil; cluster x atom x
 * 16 columns for the projection; cluster x 256 covered nodes x 16 columns for the
 * scatter), with each cluster's sizes, tables and step coefficients read from a per-step
 * table. The m steps are captured once into a CUDA graph and replayed while the blocks,
 * column counts and degree stay the same (bounds may change between calls: the
 * coefficient table is uploaded before each replay). Results equal sparc_cheb_filter on
 * each cluster (same arithmetic per point, up to FP32 contraction order).
 *
 * The stencil's tile shape and z split come from a small autotuner (sparc_batch_tune).
 * All calls are asynchronous on the stream given at creation unless stated otherwise. */
#ifndef SPARC_BATCH_H
#define SPARC_BATCH_H

#include "sparc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sparc_batch sparc_batch; /* opaque, owned by the library */

/* Groups n contexts (not owned; they must outlive the batch). cuda_stream: the caller's
 * stream (NULL = legacy default stream); batched work runs on a private stream that waits
 * for the caller's stream on entry and makes it wait on exit, so calls are ordered with
 * the caller's work on that stream. The contexts' coefficient buffers are used by the
 * batched launches: do not run other calls on these contexts concurrently on other
 * streams. */
sparc_status sparc_batch_create(sparc_ctx *const *ctxs, int n, void *cuda_stream,
                                sparc_batch **out);

/* Degree-m filter of every cluster: X[c] (FP32 device block, ncols[c] columns, leading
 * dimension ld[c] >= Nd of cluster c) is replaced by its filtered block, W[c] (same shape)
 * is overwritten; bounds[3c .. 3c+2] = (a, b, a0) with a0 < a < b. */
sparc_status sparc_batch_filter(sparc_batch *b, float *const *X, float *const *W,
                                const int *ncols, const long *ld, int degree,
                                const double *bounds);

/* Autotuner: runs the filter (as sparc_batch_filter, so X is overwritten with filtered
 * data) under every tile shape x z split the library offers, times each with CUDA events
 * after a warm-up, keeps the fastest for later calls and returns its index and time (ms).
 * Synchronises. */
sparc_status sparc_batch_tune(sparc_batch *b, float *const *X, float *const *W,
                              const int *ncols, const long *ld, int degree,
                              const double *bounds, int *variant, double *ms);

/* Selects a variant by index (0 .. count-1); count receives the number of variants.
 * variant < 0 only queries. */
sparc_status sparc_batch_variant(sparc_batch *b, int variant, int *count);

/* Frees the batch (not the contexts). NULL is accepted. */
sparc_status sparc_batch_destroy(sparc_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* SPARC_BATCH_H */
