// stencil_tma.cu -- the FP32 fused stencil step (Eq. FD:Laplacian, weights Eq. weightsLap,
// zero-Dirichlet boundaries, V_eff, Chebyshev recurrence of Algorithm ChebychevFilter,
// Sec. 3.4) fed by the Tensor Memory Accelerator.
//
// The FP32 filter step moves 12 B per point-orbital and should run at HBM speed. A CTA owns
// a 32 x 16 tile of (x, y) for one column and streams along z. One elected thread keeps a
// ring of kStages shared-memory planes filled with 4-D tiled TMA loads
// (cp.async.bulk.tensor) of the tile plus its radius-6 halo: the box starts 8 nodes left
// of the tile so that the x coordinate stays 16-byte aligned, and nodes outside the grid
// are zero-filled by the TMA unit, which is exactly the zero-Dirichlet boundary. Each
// plane's arrival is signalled through an mbarrier (expect-tx); all waits are bounded and
// report a timeout through a device flag instead of hanging.
//
// Each thread computes 4 consecutive x nodes of one row with 128-bit shared loads
// (5 loads cover x-6 .. x+9 of the four nodes, 12 more the y neighbours) and keeps the
// z neighbours of its four nodes in a 13-deep register queue of float4, filled from each
// newly arrived plane. The queue needs planes t .. t+6 of the ring, so with kStages = 10
// the loads run 4 planes ahead of the compute.
//
// Requirements (checked on the host, else the plain kernel of stencil.cu runs): n0 and ld
// multiples of 4 and 16-byte aligned block pointers (TMA strides and float4 accesses).
#include "internal.cuh"
#include "tma.cuh"

#include <cudaTypedefs.h>

namespace sparc {

namespace {
constexpr int kTX = 8;       // threads along x, 4 nodes each
constexpr int kTY = 16;      // rows per tile
constexpr int kBX = 4 * kTX; // 32 nodes along x
constexpr int kR = kRadius;  // 6
constexpr int kW = kBX + 16; // box width: 8 left (aligned) + 32 + 8 right
constexpr int kH = kTY + 2 * kR;
constexpr int kStages = 10;
constexpr int kPlaneBytes = kW * kH * 4;
constexpr unsigned kWaitLimit = 1u << 22;
}  // namespace

__global__ void __launch_bounds__(kTX *kTY)
k_stencil_f32_tma(const __grid_constant__ CUtensorMap tmY, const float *Yprev, float *out,
                  const float *__restrict__ V, int n0, int n1, int n2, long ld, int nzc,
                  int zchunk, StepCoef<float> cf, int *err)
{
    extern __shared__ __align__(128) float sm[];  // [kStages][kH][kW]
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ int timed_out;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kTY;
    const int col = blockIdx.z / nzc;
    const int k0 = (blockIdx.z % nzc) * zchunk;
    const int k1 = min(n2, k0 + zchunk);
    const int T = (k1 - k0) + 2 * kR;  // planes k0-6 .. k1+5
    const int i = i0 + 4 * tx, j = j0 + ty;
    const bool act = (i < n0) && (j < n1);
    const long plane = (long)n0 * n1;
    const long pij = (long)i + (long)n0 * j;
    const float *Pc = Yprev ? Yprev + (long)col * ld : nullptr;
    float *Oc = out + (long)col * ld;

    if (tid == 0) {
        tma_prefetch_desc(&tmY);
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
        timed_out = 0;
    }
    __syncthreads();
    int issued = 0;  // planes 0 .. issued-1 have been handed to the TMA unit (thread 0)
    auto issue = [&](int t) {  // plane t (z = k0 - 6 + t) into stage t % kStages
        const int s = t % kStages;
        mbar_arrive_expect_tx(&full[s], kPlaneBytes);
        tma_load_4d(sm + (long)s * kH * kW, &tmY, &full[s], i0 - 8, j0 - kR, k0 - kR + t, col);
        issued = t + 1;
    };
    auto wait = [&](int t) -> bool {
        return mbar_wait(&full[t % kStages], (unsigned)((t / kStages) & 1), kWaitLimit);
    };
    auto center = [&](int t) -> float4 {
        return *reinterpret_cast<const float4 *>(sm + ((long)(t % kStages) * kH + kR + ty) * kW +
                                                 8 + 4 * tx);
    };
    if (tid == 0)
        for (int t = 0; t < kStages && t < T; ++t) issue(t);

    bool ok = true;
    float4 q[2 * kR + 1];
    // planes 0..5 only feed the queue: read them, then hand their stages to planes
    // kStages .. kStages+5
    for (int t = 0; t < kR; ++t) {
        ok = ok && wait(t);
        q[t] = center(t);
    }
    if (!ok) timed_out = 1;
    __syncthreads();
    if (tid == 0 && !timed_out)
        for (int t = kStages; t < kStages + kR && t < T; ++t) issue(t);
    for (int t = kR; t < 2 * kR; ++t) {
        ok = ok && wait(t);
        q[t] = center(t);
    }
    if (!ok) timed_out = 1;
    __syncthreads();

    for (int tc = kR; tc < T - kR && !timed_out; ++tc) {  // plane tc is z = k0 - 6 + tc
        const int k = k0 - kR + tc;
        const long p = pij + (long)k * plane;
        float4 vv = make_float4(0.f, 0.f, 0.f, 0.f), pv = vv;
        if (act) {
            vv = *reinterpret_cast<const float4 *>(V + p);
            if (Pc) pv = *reinterpret_cast<const float4 *>(Pc + p);
        }
        if (!wait(tc + kR)) timed_out = 1;
        q[2 * kR] = center(tc + kR);
        const float *pl = sm + (long)(tc % kStages) * kH * kW;
        const float *row = pl + (kR + ty) * kW + 4 * tx;  // x offset 4tx = node i - 8
        float f[20];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const float4 v = *reinterpret_cast<const float4 *>(row + 4 * m);
            f[4 * m] = v.x;
            f[4 * m + 1] = v.y;
            f[4 * m + 2] = v.z;
            f[4 * m + 3] = v.w;
        }
        float acc[4];
        const float *c4 = &q[kR].x;
        const float *v4 = &vv.x;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = (cf.c0 + cf.alpha * v4[u]) * c4[u];
#pragma unroll
        for (int r = 1; r <= kR; ++r) {
            const float4 yp = *reinterpret_cast<const float4 *>(row + r * kW + 8);
            const float4 ym = *reinterpret_cast<const float4 *>(row - r * kW + 8);
            const float *a = &yp.x, *b = &ym.x, *zp = &q[kR + r].x, *zm = &q[kR - r].x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float t = (f[8 + u + r] + f[8 + u - r]) + (a[u] + b[u]) + (zp[u] + zm[u]);
                acc[u] += cf.w[r] * t;
            }
        }
        if (act) {
            const float *p4 = &pv.x;
            float4 o;
            o.x = Pc ? acc[0] - cf.beta * p4[0] : acc[0];
            o.y = Pc ? acc[1] - cf.beta * p4[1] : acc[1];
            o.z = Pc ? acc[2] - cf.beta * p4[2] : acc[2];
            o.w = Pc ? acc[3] - cf.beta * p4[3] : acc[3];
            *reinterpret_cast<float4 *>(Oc + p) = o;
        }
#pragma unroll
        for (int t = 0; t < 2 * kR; ++t) q[t] = q[t + 1];
        __syncthreads();  // every thread is done with plane tc's stage
        if (tid == 0 && !timed_out && tc + kStages < T) issue(tc + kStages);
    }
    if (timed_out) {
        // leave no TMA write in flight into this CTA's shared memory: wait (bounded) for
        // the latest issued plane of every stage, then report
        if (tid == 0) {
            atomicExch(err, 1);
            for (int s = 0; s < kStages; ++s) {
                int last = -1;  // latest plane issued into stage s
                for (int t = s; t < issued; t += kStages) last = t;
                if (last >= 0) mbar_wait(&full[s], (unsigned)((last / kStages) & 1), kWaitLimit);
            }
        }
        __syncthreads();
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encoder()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

bool stencil_tma_ok(const DevHam &H, const void *Y, const void *Yprev, const void *out, long ld)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    return (H.n0 % 4 == 0) && (ld % 4 == 0) && al(Y) && al(out) && (!Yprev || al(Yprev)) &&
           al(H.Vf) && H.n0 <= (1 << 24) && H.n1 <= (1 << 24);
}

cudaError_t stencil_f32_tma(const DevHam &H, const float *Y, const float *Yprev, float *out,
                            int ncols, long ld, const StepCoef<float> &cf, int *err,
                            cudaStream_t st)
{
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    static bool attr_set = false;
    const int smem = kStages * kPlaneBytes;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_stencil_f32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    CUtensorMap map;
    cuuint64_t dims[4] = {(cuuint64_t)H.n0, (cuuint64_t)H.n1, (cuuint64_t)H.n2, (cuuint64_t)ncols};
    cuuint64_t strides[3] = {(cuuint64_t)H.n0 * 4, (cuuint64_t)H.n0 * H.n1 * 4,
                             (cuuint64_t)ld * 4};
    cuuint32_t box[4] = {(cuuint32_t)kW, (cuuint32_t)kH, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)Y, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int gx = (H.n0 + kBX - 1) / kBX, gy = (H.n1 + kTY - 1) / kTY;
    int nzc, zchunk;
    stencil_z_split(H.n2, (long)gx * gy, ncols, nzc, zchunk);
    dim3 grid(gx, gy, ncols * nzc), block(kTX, kTY);
    k_stencil_f32_tma<<<grid, block, smem, st>>>(map, Yprev, out, H.Vf, H.n0, H.n1, H.n2, ld, nzc,
                                                 zchunk, cf, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
