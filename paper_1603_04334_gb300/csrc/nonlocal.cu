// nonlocal.cu -- Kleinman-Bylander nonlocal operator, Eq. (non-localPS:FD), Sec. 3.1:
//   V_nl f = h^3 sum_J sum_lm gamma_Jlm chi_Jlm (chi_Jlm^T f),
// applied matrix-free (Sec. 3.1) in two deterministic passes:
//   project: C_Jlm,c = sum_{s in supp(J)} chi_Jlm(s) Y(s, c)       (gather + 4 x nsup x ncols)
//   scatter: out(p, c) += alpha sum_{e at p} sum_lm gchi(e, lm) C_atom(e)lm,c
// with gchi = h^3 gamma chi precomputed at setup. The scatter walks the node -> entries
// inverse map (entries of a node in ascending order), so the values need no atomics and
// do not depend on scheduling (the FP64 pair scatter also raises per-column magnitude
// bounds with atomicMax, whose result does not depend on order either).
#include "df.cuh"
#include "fx.cuh"
#include "internal.cuh"

namespace sparc {

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per (atom, column block of CB). Each thread accumulates 4*CB partial sums over
// a strided share of the atom's support; the block reduces them in a fixed order.
// C layout: ILV = false: C[(J * 4 + l) * ncols + c]; ILV = true: C[(J * ncols + c) * 4 + l]
// (the four channels of one atom and column contiguous, one 16-byte load in the scatter).
// project_block: atom J (support entries b .. e-1), columns c0 .. c0+CB-1; ends with a CTA
// barrier so the caller may reuse the shared memory.
template <typename T, typename TC, int CB, int NT, bool ILV>
__device__ __forceinline__ void project_block(const T *__restrict__ Y, long ld, int ncols, int J,
                                              int b, int e, int c0,
                                              const int *__restrict__ idx,
                                              const TC *__restrict__ chi, TC *__restrict__ C,
                                              TC alpha)
{
    __shared__ TC red[NT / 32][4 * CB];
    TC acc[4][CB];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) acc[l][cb] = (TC)0;
    // Two support points per trip, their node indices loaded one trip ahead, so a thread
    // has 2 * CB independent loads of Y in flight instead of an index -> value chain.
    auto load_chi = [&](int s, TC x[4]) {
        if constexpr (sizeof(TC) == 4) {
            const float4 v = reinterpret_cast<const float4 *>(chi)[s];
            x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
        } else {
            const double2 a = reinterpret_cast<const double2 *>(chi)[2 * (long)s];
            const double2 q = reinterpret_cast<const double2 *>(chi)[2 * (long)s + 1];
            x[0] = a.x, x[1] = a.y, x[2] = q.x, x[3] = q.y;
        }
    };
    int s = b + threadIdx.x;
    long pa = s < e ? idx[s] : 0, pb = s + NT < e ? idx[s + NT] : 0;
    for (; s < e; s += 2 * NT) {
        const bool vb = s + NT < e;
        TC xa[4], xb[4] = {(TC)0, (TC)0, (TC)0, (TC)0};
        TC ya[CB], yb[CB];
        load_chi(s, xa);
        if (vb) load_chi(s + NT, xb);
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const bool vc = c0 + cb < ncols;
            ya[cb] = vc ? (TC)Y[pa + (long)(c0 + cb) * ld] : (TC)0;
            yb[cb] = (vc && vb) ? (TC)Y[pb + (long)(c0 + cb) * ld] : (TC)0;
        }
        const int sn = s + 2 * NT;
        pa = sn < e ? idx[sn] : 0;
        pb = sn + NT < e ? idx[sn + NT] : 0;
#pragma unroll
        for (int cb = 0; cb < CB; ++cb)
#pragma unroll
            for (int l = 0; l < 4; ++l) acc[l][cb] += xa[l] * ya[cb];
#pragma unroll
        for (int cb = 0; cb < CB; ++cb)
#pragma unroll
            for (int l = 0; l < 4; ++l) acc[l][cb] += xb[l] * yb[cb];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const TC v = warp_sum(acc[l][cb]);
            if (lane == 0) red[wid][l * CB + cb] = v;
        }
    __syncthreads();
    if (threadIdx.x < 4 * CB) {
        const int l = threadIdx.x / CB, cb = threadIdx.x % CB;
        TC v = (TC)0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) v += red[w][threadIdx.x];
        if (c0 + cb < ncols) {
            const long o = ILV ? ((long)J * ncols + c0 + cb) * 4 + l
                               : (long)(J * 4 + l) * ncols + c0 + cb;
            C[o] = alpha * v;
        }
    }
    __syncthreads();
}

// Grid: x = atom (dispatched first: the CTAs resident at one time read the supports of
// many atoms for the same columns, so the nodes that several supports share are read from
// DRAM about once), y = column block. order (optional): the atoms in a spatial order, so
// that CTAs dispatched together gather overlapping supports (and the DRAM granules that the
// short x-runs of one support fetch only in part serve its neighbours).
template <typename T, typename TC, int CB, int NT, bool ILV>
__global__ void __launch_bounds__(NT)
k_project(const T *__restrict__ Y, long ld, int ncols, const int *__restrict__ atom_ptr,
          const int *__restrict__ idx, const TC *__restrict__ chi, TC *__restrict__ C, TC alpha,
          const int *__restrict__ order)
{
    const int J = order ? order[blockIdx.x] : (int)blockIdx.x;
    project_block<T, TC, CB, NT, ILV>(Y, ld, ncols, J, atom_ptr[J], atom_ptr[J + 1],
                                      blockIdx.y * CB, idx, chi, C, alpha);
}

// Work-list form for a batch of clusters (items: cluster, atom, first column).
__global__ void __launch_bounds__(256, 2)
k_batch_project(const BatchItem *__restrict__ items, int nitems, const BatchNonlocal *cs)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchNonlocal &P = cs[w.cluster];
        project_block<float, float, kBatchCols, 256, true>(
            P.Y, P.ld, P.ncols, w.a, P.atom_ptr[w.a], P.atom_ptr[w.a + 1], w.col, P.idx,
            P.chi_f, P.C, P.alpha);
    }
}

cudaError_t batch_project(const BatchItem *items, int nitems, const BatchNonlocal *cs, int grid,
                          cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    k_batch_project<<<grid, 256, 0, st>>>(items, nitems, cs);
    note_launch();
    return cudaGetLastError();
}

template <typename T, typename TC, bool ILV>
static cudaError_t project(const DevHam &H, const T *Y, int ncols, long ld, const TC *chi,
                           TC *C, TC alpha, cudaStream_t st)
{
    if (H.natoms == 0 || ncols <= 0) return cudaSuccess;
    // FP32 accumulators leave room for 16 columns per CTA (32 loads of Y in flight per
    // thread); FP64 ones for 8
    constexpr int CB = sizeof(TC) == 4 ? 16 : 8, NT = 256;
    dim3 grid(H.natoms, (ncols + CB - 1) / CB);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_project<T, TC, CB, NT, ILV>
        <<<grid, NT, 0, st>>>(Y, ld, ncols, H.atom_ptr, H.idx, chi, C, alpha, H.proj_order);
    note_launch();
    return cudaGetLastError();
}

cudaError_t project_f32(const DevHam &H, const float *Y, int ncols, long ld, double alpha,
                        float *C, cudaStream_t st)
{
    return project<float, float, true>(H, Y, ncols, ld, H.chi_f, C, (float)alpha, st);
}
// ---- FP64 projection in exact integer arithmetic ---------------------------------------
// Each column of Y is put on its 49-bit grid (fx_split: y = 2^(E-49) (d 2^23 + r), E from
// the column bound) and each projector l of atom J on a 46-bit grid of its own (chi =
// 2^(F-46) (a 2^23 + b), F from max |chi_Jl| over the support, a and b integers below 2^23
// in magnitude). Then
//   chi y = 2^(E+F-95) (a d 2^46 + (a r + b d) 2^23 + b r),
// and the kernel sums a d and a r + b d exactly in two int64 accumulators per (l, column);
// only b r is dropped (below 2^-49 of the largest product), so C is the projection of the
// two grids to about 2^-48 of sum |chi y|, with no rounding along the support (compensated
// FP32-pair sums lose about 2^-44 of it to cancellation). Integer sums do not depend on
// their order; the per-warp sums are combined across the CTA in FP64 in a fixed order. The
// result is alpha C as an FP32 pair, for the pair scatter.
// chi_q: per entry two int4, (a_0..a_3) then (b_0..b_3); chi_F: per (atom, l) the exponent F.

// chi_q and chi_F from chi. CTA: one atom; F from the largest high word of |chi| per l.
__global__ void __launch_bounds__(256)
k_chi_fixed(const int *__restrict__ atom_ptr, const double *__restrict__ chi, int4 *chi_q,
            int *chi_F)
{
    __shared__ unsigned mx[4];
    const int J = blockIdx.x;
    const int b = atom_ptr[J], e = atom_ptr[J + 1];
    if (threadIdx.x < 4) mx[threadIdx.x] = 0u;
    __syncthreads();
    unsigned m[4] = {0u, 0u, 0u, 0u};
    for (int s = b + threadIdx.x; s < e; s += blockDim.x)
#pragma unroll
        for (int l = 0; l < 4; ++l) m[l] = max(m[l], abs_hi_word(chi[4L * s + l]));
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const unsigned w = __reduce_max_sync(0xffffffffu, m[l]);
        if ((threadIdx.x & 31) == 0) atomicMax(&mx[l], w);
    }
    __syncthreads();
    int F[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) F[l] = mx[l] ? bound_exponent(mx[l]) : 0;
    if (threadIdx.x < 4) chi_F[4 * J + threadIdx.x] = F[threadIdx.x];
    for (int s = b + threadIdx.x; s < e; s += blockDim.x) {
        int qa[4], qb[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            // |chi| 2^(46 - F) < 2^46, rounded to an integer (a power-of-two scaling is exact)
            const double c = chi[4L * s + l];
            const long long A = llrint(fabs(ldexp(c, 46 - F[l])));
            const int sg = c < 0.0 ? -1 : 1;
            qa[l] = sg * (int)(A >> 23);
            qb[l] = sg * (int)(A & 0x7fffff);
        }
        chi_q[2L * s] = make_int4(qa[0], qa[1], qa[2], qa[3]);
        chi_q[2L * s + 1] = make_int4(qb[0], qb[1], qb[2], qb[3]);
    }
}

cudaError_t chi_fixed(int natoms, const int *atom_ptr, const double *chi, int4 *chi_q,
                      int *chi_F, cudaStream_t st)
{
    if (natoms <= 0) return cudaSuccess;
    k_chi_fixed<<<natoms, 256, 0, st>>>(atom_ptr, chi, chi_q, chi_F);
    note_launch();
    return cudaGetLastError();
}

// One CTA per (atom, CB columns); T: the block's type (FP64, or the FP32 block to which the
// mixed-precision Rayleigh-Ritz step applies H in FP64). bY: the columns' bounds.
// Grid as k_project: x = atom (in the spatial order), y = column block.
template <typename T, int CB, int NT>
__global__ void __launch_bounds__(NT, 3)
k_project_fx(const T *__restrict__ Y, long ld, int ncols, const int *__restrict__ atom_ptr,
             const int *__restrict__ idx, const int4 *__restrict__ chi_q,
             const int *__restrict__ chi_F, const unsigned *__restrict__ bY, double alpha,
             float2 *__restrict__ C, const int *__restrict__ order)
{
    __shared__ double red[NT / 32][8 * CB];
    const int J = order ? order[blockIdx.x] : (int)blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int b = atom_ptr[J], e = atom_ptr[J + 1];
    int E[CB];
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) E[cb] = c0 + cb < ncols ? bound_exponent(bY[c0 + cb]) : 0;
    long long hi[4][CB], lo[4][CB];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) hi[l][cb] = lo[l][cb] = 0;
    // two entries per trip, their node indices loaded one trip ahead: 2 CB independent loads
    // of Y in flight per thread instead of an index -> value chain
    auto acc = [&](const T (&y)[CB], int4 qa, int4 qb) {
        const int a[4] = {qa.x, qa.y, qa.z, qa.w}, bb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const int2 q = fx_split(y[cb], E[cb]);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                hi[l][cb] += (long long)a[l] * q.x;
                lo[l][cb] += (long long)a[l] * q.y + (long long)bb[l] * q.x;
            }
        }
    };
    int s = b + threadIdx.x;
    long pa = s < e ? idx[s] : 0, pb = s + NT < e ? idx[s + NT] : 0;
    for (; s < e; s += 2 * NT) {
        const bool vb = s + NT < e;
        T ya[CB], yb[CB];
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const bool vc = c0 + cb < ncols;
            ya[cb] = vc ? Y[pa + (long)(c0 + cb) * ld] : (T)0;
            yb[cb] = (vc && vb) ? Y[pb + (long)(c0 + cb) * ld] : (T)0;
        }
        const int4 qa = chi_q[2L * s], qb = chi_q[2L * s + 1];
        const int4 z = make_int4(0, 0, 0, 0);
        const int4 ra = vb ? chi_q[2L * (s + NT)] : z, rb = vb ? chi_q[2L * (s + NT) + 1] : z;
        const int sn = s + 2 * NT;
        pa = sn < e ? idx[sn] : 0;
        pb = sn + NT < e ? idx[sn + NT] : 0;
        acc(ya, qa, qb);
        acc(yb, ra, rb);
    }
    // |a d| and |a r + b d| are below 2^50: a thread's sums stay below 2^(50 + log2 t) for t
    // entries; before the 32-way warp sum they are shifted right by max(0, log2 t - 7) so that
    // it stays below 2^62 (for supports up to 32768 entries per atom no shift is needed)
    const int t = (e - b + NT - 1) / NT;
    const int sh = t > 128 ? (32 - __clz(t - 1)) - 7 : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            long long h = hi[l][cb] >> sh, g = lo[l][cb] >> sh;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                h += __shfl_xor_sync(0xffffffffu, h, o);
                g += __shfl_xor_sync(0xffffffffu, g, o);
            }
            if (lane == 0) {
                red[wid][(l * CB + cb) * 2] = (double)h;
                red[wid][(l * CB + cb) * 2 + 1] = (double)g;
            }
        }
    __syncthreads();
    if (threadIdx.x < 4 * CB) {
        const int l = threadIdx.x / CB, cb = threadIdx.x % CB;
        double h = 0.0, g = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            h += red[w][threadIdx.x * 2];
            g += red[w][threadIdx.x * 2 + 1];
        }
        if (c0 + cb < ncols) {
            // alpha 2^(E+F-49+sh) (h + 2^-23 g); a column whose bound is not finite gives NaN
            const unsigned u = bY[c0 + cb];
            double v = alpha * ldexp(fma(g, 0x1p-23, h), E[cb] + chi_F[4 * J + l] - 49 + sh);
            if (((u >> 20) & 0x7ffu) == 0x7ffu) v = __longlong_as_double(0x7ff8000000000000ll);
            const float vh = (float)v;
            C[(long)(J * 4 + l) * ncols + c0 + cb] = make_float2(vh, (float)(v - (double)vh));
        }
    }
}

template <typename T>
static cudaError_t project_fx(const DevHam &H, const T *Y, int ncols, long ld, double alpha,
                              const unsigned *bY, float2 *C, cudaStream_t st)
{
    if (H.natoms == 0 || ncols <= 0) return cudaSuccess;
    constexpr int CB = 2, NT = 256;
    dim3 grid(H.natoms, (ncols + CB - 1) / CB);
    if (grid.y > 65535 || !bY) return cudaErrorInvalidValue;
    k_project_fx<T, CB, NT><<<grid, NT, 0, st>>>(Y, ld, ncols, H.atom_ptr, H.idx, H.chi_q,
                                                 H.chi_F, bY, alpha, C, H.proj_order);
    note_launch();
    return cudaGetLastError();
}

cudaError_t project_f64_fx(const DevHam &H, const double *Y, int ncols, long ld, double alpha,
                           const unsigned *bY, float2 *C, cudaStream_t st)
{
    return project_fx<double>(H, Y, ncols, ld, alpha, bY, C, st);
}

cudaError_t project_f32in_f64(const DevHam &H, const float *Y, int ncols, long ld,
                              const unsigned *bY, float2 *C, cudaStream_t st)
{
    return project_fx<float>(H, Y, ncols, ld, 1.0, bY, C, st);
}

constexpr int kScatNodes = 256;     // covered nodes (threads) per CTA of the FP32 scatter
constexpr int kScatF32Cols = 8;     // columns per group
constexpr int kScatF32Groups = 4;   // column groups per thread

// FP32 blocks: Cs holds alpha chi^T Y as one float4 per (atom, column), Cs4[J * ncols + c],
// and g4[q] the four h^3 gamma chi values of entry q. A thread owns one covered node and
// kScatF32Groups groups of kScatF32Cols columns; the grid's x dimension (dispatched first)
// runs over the column ranges, so the CTAs resident at one time share their covered nodes
// and read the node's entry tables from L1/L2 (with the nodes outermost, every column group
// read the tables again from DRAM: about as many bytes as the output itself at 1024
// columns). Per group the thread walks its node's entries (the atoms whose support holds
// it, ascending): per entry one load of the four coefficients and, per column, one 16-byte
// load of Cs (L1/L2-resident). The entry loop runs to the largest entry count of the warp
// with the shorter lanes predicated off, so a warp whose nodes are covered by different
// numbers of atoms stays on one path. Per column the entries are summed in ascending order.
template <int NC>
__device__ __forceinline__ void scatter_f32_group(float *ob, long ld, int ncols, int cg, int q0,
                                                  int n, int nmax, bool live, const float (&x)[NC],
                                                  const int *__restrict__ nl_atom,
                                                  const float4 *__restrict__ g4,
                                                  const float4 *__restrict__ Cs4)
{
    float v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0.0f;
    for (int t = 0; t < nmax; ++t) {
        if (t < n) {
            const float4 g = g4[q0 + t];
            const float4 *cq = Cs4 + (long)nl_atom[q0 + t] * ncols + cg;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (cg + c < ncols) {
                    const float4 cc = cq[c];
                    v[c] += g.x * cc.x;
                    v[c] += g.y * cc.y;
                    v[c] += g.z * cc.z;
                    v[c] += g.w * cc.w;
                }
            }
        }
    }
    if (live) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (cg + c < ncols) ob[(long)(cg + c) * ld] = x[c] + v[c];
    }
}

// Covered node `node` (entries q0 .. q1-1), columns c0 .. c0 + NG NC - 1 (those below ncols)
// in NG groups of NC: the output reads of group g+1 are issued before the sums of group g
// are formed and stored, so a thread keeps NC DRAM reads in flight throughout. All lanes
// of a warp call it together (lanes without a node pass live = false).
template <int NC, int NG>
__device__ __forceinline__ void scatter_f32_node(float *out, long ld, int ncols, long node, int q0,
                                                 int q1, int c0, bool live,
                                                 const int *__restrict__ nl_atom,
                                                 const float4 *__restrict__ g4,
                                                 const float4 *__restrict__ Cs4)
{
    float *ob = out + node;
    const int n = live ? q1 - q0 : 0;
    const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
    float x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = (live && c0 + c < ncols) ? ob[(long)(c0 + c) * ld] : 0.0f;
#pragma unroll 1
    for (int gi = 0; gi < NG; ++gi) {
        const int cg = c0 + gi * NC;
        if (cg >= ncols) break;
        const int cn = cg + NC;
        const bool more = gi + 1 < NG && cn < ncols;
        float xn[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            xn[c] = (more && live && cn + c < ncols) ? ob[(long)(cn + c) * ld] : 0.0f;
        scatter_f32_group<NC>(ob, ld, ncols, cg, q0, n, nmax, live, x, nl_atom, g4, Cs4);
#pragma unroll
        for (int c = 0; c < NC; ++c) x[c] = xn[c];
    }
}

// One covered node per thread, NG groups of NC columns; every lane of a warp reaches the
// entry loop's warp-wide maximum (lanes past nuniq take part with no entries).
template <int NC, int NG>
__global__ void __launch_bounds__(kScatNodes)
k_scatter_f32(float *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
              const int *__restrict__ uniq_ptr, const int *__restrict__ nl_atom,
              const float4 *__restrict__ g4, const float4 *__restrict__ Cs4)
{
    const int c0 = blockIdx.x * NC * NG;
    for (long ub = blockIdx.y; ub * kScatNodes < nuniq; ub += gridDim.y) {
        const long u = ub * kScatNodes + threadIdx.x;
        const bool live = u < nuniq;
        scatter_f32_node<NC, NG>(out, ld, ncols, live ? uniq_node[u] : 0,
                                 live ? uniq_ptr[u] : 0, live ? uniq_ptr[u + 1] : 0, c0, live,
                                 nl_atom, g4, Cs4);
    }
}

// Work-list form for a batch of clusters (items: cluster, node chunk, first column).
__global__ void __launch_bounds__(kScatNodes)
k_batch_scatter(const BatchItem *__restrict__ items, int nitems, const BatchNonlocal *cs)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchNonlocal &P = cs[w.cluster];
        const long u = (long)w.a * kBatchNodes + threadIdx.x;
        const bool live = u < P.nuniq;
        scatter_f32_node<kBatchCols, 1>(P.out, P.ld, P.ncols, live ? P.uniq_node[u] : 0,
                                        live ? P.uniq_ptr[u] : 0, live ? P.uniq_ptr[u + 1] : 0,
                                        w.col, live, P.nl_atom,
                                        reinterpret_cast<const float4 *>(P.nl_gf),
                                        reinterpret_cast<const float4 *>(P.C));
    }
}

cudaError_t batch_scatter(const BatchItem *items, int nitems, const BatchNonlocal *cs, int grid,
                          cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    k_batch_scatter<<<grid, kScatNodes, 0, st>>>(items, nitems, cs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scatter_f32(const DevHam &H, const float *Cs, float *out, int ncols, long ld,
                        cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    constexpr int NC = kScatF32Cols, NG = kScatF32Groups;
    const long nb = (H.nuniq + kScatNodes - 1) / kScatNodes;
    dim3 grid((unsigned)((ncols + NC * NG - 1) / (NC * NG)), (unsigned)(nb < 65535 ? nb : 65535));
    k_scatter_f32<NC, NG><<<grid, kScatNodes, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                               H.nl_atom, reinterpret_cast<const float4 *>(H.nl_gf),
                                               reinterpret_cast<const float4 *>(Cs));
    note_launch();
    return cudaGetLastError();
}

// Nonlocal scatter for FP64 blocks in pair arithmetic: out(p, c) += sum_{q at p} sum_l
// g(q, l) Cs(atom(q), l, c), Cs = alpha chi^T Y as pairs (k_project_df). A thread owns one
// covered node and kScatDfGroups groups of kScatDfCols columns; the grid's x dimension
// (dispatched first) runs over the column ranges, so the CTAs resident at one time share
// their covered nodes (the node's entry tables are read from L1/L2, not once per column
// group from DRAM), and y over blocks of covered nodes (strided when there are more than the
// grid holds). The pair sum is added to the FP64 output with one FP64 add. With bOut, the
// column bounds of the output are raised to cover the updated values.
namespace {
constexpr int kScatDfNodes = 256;
constexpr int kScatDfCols = 4;    // columns per group
constexpr int kScatDfGroups = 4;  // column groups per thread
}  // namespace

__global__ void __launch_bounds__(kScatDfNodes, 4)
k_scatter_df(double *out, long ld, int ncols, long nuniq, const int *__restrict__ uniq_node,
             const int *__restrict__ uniq_ptr, const int *__restrict__ nl_atom,
             const float2 *__restrict__ g, const float2 *__restrict__ Cs, unsigned *bOut)
{
    constexpr int K = kScatDfCols;
    const int c0 = blockIdx.x * K * kScatDfGroups;
    // both loops are uniform over the CTA: every lane reaches the bound reductions
    for (long ub = blockIdx.y; ub * kScatDfNodes < nuniq; ub += gridDim.y) {
        const long u = ub * kScatDfNodes + threadIdx.x;
        const bool live = u < nuniq;
        const long node = live ? uniq_node[u] : 0;
        const int q0 = live ? uniq_ptr[u] : 0, q1 = live ? uniq_ptr[u + 1] : 0;
        double *ob = out + node;
        // the output reads of group g+1 are issued before the sums of group g are formed,
        // so K DRAM reads stay in flight; each entry's atom and coefficients are loaded once
        // per group, and per column the entries are summed in ascending order
        double o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = (live && c0 + k < ncols) ? ob[(long)(c0 + k) * ld] : 0.0;
#pragma unroll 1
        for (int gi = 0; gi < kScatDfGroups; ++gi) {
            const int cg = c0 + gi * K;
            if (cg >= ncols) break;
            const int cn = cg + K;
            const bool more = gi + 1 < kScatDfGroups && cn < ncols;
            double on[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
                on[k] = (more && live && cn + k < ncols) ? ob[(long)(cn + k) * ld] : 0.0;
            float vh[K], vl[K];
#pragma unroll
            for (int k = 0; k < K; ++k) vh[k] = vl[k] = 0.0f;
            for (int q = q0; q < q1; ++q) {
                const float2 *cs = Cs + (long)nl_atom[q] * 4 * ncols + cg;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const float2 gl = g[4L * q + l];
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (cg + k < ncols) mac(gl, cs[(long)l * ncols + k], vh[k], vl[k]);
                }
            }
            unsigned om[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                o[k] += pair_to_double(vh[k], vl[k]);
                om[k] = 0u;
                if (live && cg + k < ncols) {
                    ob[(long)(cg + k) * ld] = o[k];
                    om[k] = abs_hi_word(o[k]);
                }
            }
            if (bOut) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const unsigned m = __reduce_max_sync(0xffffffffu, om[k]);
                    if ((threadIdx.x & 31) == 0 && m && cg + k < ncols) raise_bound(bOut + cg + k, m);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) o[k] = on[k];
        }
    }
}

cudaError_t scatter_f64_df(const DevHam &H, const float2 *Cs, double *out, int ncols, long ld,
                           unsigned *bOut, cudaStream_t st)
{
    if (H.natoms == 0 || H.nuniq == 0 || ncols <= 0) return cudaSuccess;
    const long nb = (H.nuniq + kScatDfNodes - 1) / kScatDfNodes;
    constexpr int cpb = kScatDfCols * kScatDfGroups;
    dim3 grid((unsigned)((ncols + cpb - 1) / cpb), (unsigned)(nb < 65535 ? nb : 65535));
    k_scatter_df<<<grid, kScatDfNodes, 0, st>>>(out, ld, ncols, H.nuniq, H.uniq_node, H.uniq_ptr,
                                              H.nl_atom, H.nl_gdf, Cs, bOut);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
