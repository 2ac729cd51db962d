// noalloc.cu -- an FP64 Gram contraction G = A^T B that allocates no memory.
//
// Who needs it: callers that must not allocate device memory at the point of use --
// real-time or embedded loops that forbid cudaMalloc after start-up (an allocation can
// block and synchronise the whole device), hosts that hand this library pre-allocated
// buffers from their own pool and cannot let it grow one, or processes that have reserved
// nearly all device memory already. sparc_gram keeps its row-slice partial
// sums in context workspace that it may (re)allocate; this variant keeps them in one
// file-scope __device__ array instead, so the caller only supplies A, B and G.
//
// Costs and limits, as a user should know them:
//   * The array is kNoAllocScratchDoubles doubles (16 MiB). Every GPU that loads this
//     library holds it until the process exits, whether or not this call is used.
//   * ncols^2 must fit in the array (ncols <= 1024 always does); larger requests are
//     rejected with SPARC_ERR_ARG before any work is enqueued.
//   * All calls share the one array per device. Calls that overlap on the GPU (for
//     example on two streams at once) race on it and give wrong results; serialise them.
//     Each call overwrites every partial it later reads, so nothing needs clearing and
//     the contents left by an earlier call do not matter.
//   * Host code cannot use the array's name as a device address. The first call on each
//     device looks the address up with cudaGetSymbolAddress (with that device current)
//     and caches it; make that first call before any stream capture begins. The cached
//     address belongs to the device's primary context, so a process that resets the device
//     (cudaDeviceReset) must not call this entry point on it again.
#include "sparc.h"
#include "internal.cuh"

#include <mutex>

namespace {

constexpr long kNoAllocScratchDoubles = 2L * 1024 * 1024;  // 16 MiB of FP64 partials
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch for the current device (looked up once per device).
cudaError_t scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sparc_status sparc_gram_noalloc(const double *A, const double *B, long nd, int ncols,
                                           long ld, double *G, void *cuda_stream)
{
    if (!A || !B || !G || nd < 1 || ncols < 1 || ld < nd) return SPARC_ERR_ARG;
    const long nn = (long)ncols * ncols;
    if (nn > kNoAllocScratchDoubles) return SPARC_ERR_ARG;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return SPARC_ERR_CUDA;
    int nsplit = sparc::gram_default_splits(ncols, nd);
    const long fit = kNoAllocScratchDoubles / nn;
    if (nsplit > fit) nsplit = (int)fit;
    const cudaError_t e = sparc::gram_f64_nsplit(A, ld, B, ld, nd, ncols, G, scratch, nsplit,
                                                 (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? SPARC_OK : SPARC_ERR_CUDA;
}
