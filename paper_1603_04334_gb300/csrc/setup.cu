// setup.cu -- once-per-Hamiltonian tables on the device.
//
// * V_eff(x) = sum_J -Z_J erf(|x - R_J| / rc) / |x - R_J| (synthetic local potential;
//   limit -2 Z_J / (sqrt(pi) rc) for |x - R_J| < 1e-12).
// * Kleinman-Bylander projector supports (Sec. 2 separable form; Eq. non-localPS:FD,
//   Sec. 3.1; per-atom influence boxes as in Sec. 3.2): node p belongs to atom J when
//   r^2 <= rcut^2 with r^2 = dx*dx + dy*dy + dz*dz, dx = i*h - R_x, evaluated in that
//   order. This file is compiled with -fmad=false so every product and sum is rounded
//   separately; membership is an exact function of (i, h, R, rcut).
//   chi_s = Y00 exp(-r^2/(2 sigma^2)), chi_pd = sqrt(3/(4 pi)) (x_d - R_d) exp(...).
// * The node -> entries inverse map used by the scatter (counting sort by node, then a
//   per-node sort of the short entry lists so the order is deterministic).
#include "internal.cuh"

namespace sparc {

__global__ void k_veff(int n0, int n1, int n2, double h, int natoms, const double *R,
                       const double *Z, double rc, double *V)
{
    const long nd = (long)n0 * n1 * n2;
    const double lim = 2.0 / (sqrt(3.14159265358979323846) * rc);
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
         p += (long)gridDim.x * blockDim.x) {
        const int i = (int)(p % n0), j = (int)((p / n0) % n1), k = (int)(p / ((long)n0 * n1));
        const double x = (double)i * h, y = (double)j * h, z = (double)k * h;
        double v = 0.0;
        for (int J = 0; J < natoms; ++J) {
            const double dx = x - R[3 * J], dy = y - R[3 * J + 1], dz = z - R[3 * J + 2];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < 1e-12)
                v += -Z[J] * lim;
            else
                v += -Z[J] * erf(r / rc) / r;
        }
        V[p] = v;
    }
}

cudaError_t build_veff(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                       const double *Z_dev, double rc, double *V, cudaStream_t st)
{
    const long nd = (long)n0 * n1 * n2;
    int blocks = (int)((nd + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_veff<<<blocks, 256, 0, st>>>(n0, n1, n2, h, natoms, R_dev, Z_dev, rc, V);
    note_launch();
    return cudaGetLastError();
}

// Inclusive node range of an atom's bounding box along one axis (clipped to the grid).
__device__ __forceinline__ void box_range(double c, double rc, double h, int n, int &lo, int &hi)
{
    lo = (int)floor((c - rc) / h) - 1;
    hi = (int)ceil((c + rc) / h) + 1;
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
}

struct Box {
    int i0, j0, k0, ni, nj, nk;
    __device__ long size() const { return (long)ni * nj * nk; }
};

__device__ __forceinline__ Box atom_box(const double *R, int J, double rcut, double h, int n0,
                                        int n1, int n2)
{
    Box b;
    int i1, j1, k1;
    box_range(R[3 * J], rcut, h, n0, b.i0, i1);
    box_range(R[3 * J + 1], rcut, h, n1, b.j0, j1);
    box_range(R[3 * J + 2], rcut, h, n2, b.k0, k1);
    b.ni = max(0, i1 - b.i0 + 1);
    b.nj = max(0, j1 - b.j0 + 1);
    b.nk = max(0, k1 - b.k0 + 1);
    return b;
}

__device__ __forceinline__ bool member(const double *R, int J, int i, int j, int k, double h,
                                       double rc2, double &dx, double &dy, double &dz,
                                       double &r2)
{
    dx = __dsub_rn(__dmul_rn((double)i, h), R[3 * J]);
    dy = __dsub_rn(__dmul_rn((double)j, h), R[3 * J + 1]);
    dz = __dsub_rn(__dmul_rn((double)k, h), R[3 * J + 2]);
    r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 <= rc2;
}

// One CTA per atom: counts nodes of its box inside the sphere.
__global__ void k_support_count(int n0, int n1, int n2, double h, const double *R, double rcut,
                                int *counts)
{
    __shared__ int red[32];
    const int J = blockIdx.x;
    const Box b = atom_box(R, J, rcut, h, n0, n1, n2);
    const double rc2 = __dmul_rn(rcut, rcut);
    int c = 0;
    for (long t = threadIdx.x; t < b.size(); t += blockDim.x) {
        const int i = b.i0 + (int)(t % b.ni), j = b.j0 + (int)((t / b.ni) % b.nj),
                  k = b.k0 + (int)(t / ((long)b.ni * b.nj));
        double dx, dy, dz, r2;
        if (member(R, J, i, j, k, h, rc2, dx, dy, dz, r2)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        counts[J] = s;
    }
}

cudaError_t support_count(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                          double rcut, int *counts, cudaStream_t st)
{
    if (natoms == 0) return cudaSuccess;
    k_support_count<<<natoms, 256, 0, st>>>(n0, n1, n2, h, R_dev, rcut, counts);
    note_launch();
    return cudaGetLastError();
}

// One CTA per atom: walks the box in (k, j, i) order in chunks of blockDim and compacts
// members with a block-wide exclusive scan, so entries are in ascending node order.
__global__ void k_support_fill(int n0, int n1, int n2, double h, const double *R,
                               const double *gamma, double sigma, double rcut,
                               const int *atom_ptr, int *idx, double *chi, float *chi_f,
                               double *gchi, float *gchi_f, int *ent_atom)
{
    __shared__ int wsum[32];
    __shared__ int base;
    const int J = blockIdx.x;
    const Box b = atom_box(R, J, rcut, h, n0, n1, n2);
    const double rc2 = __dmul_rn(rcut, rcut);
    const double Y00 = 1.0 / (2.0 * sqrt(3.14159265358979323846));
    const double Y1 = sqrt(3.0 / (4.0 * 3.14159265358979323846));
    const double two_s2 = __dmul_rn(__dmul_rn(2.0, sigma), sigma);
    const double h3 = __dmul_rn(__dmul_rn(h, h), h);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = atom_ptr[J];
    __syncthreads();
    for (long t0 = 0; t0 < b.size(); t0 += blockDim.x) {
        const long t = t0 + threadIdx.x;
        int i = 0, j = 0, k = 0;
        double dx = 0, dy = 0, dz = 0, r2 = 0;
        bool in = false;
        if (t < b.size()) {
            i = b.i0 + (int)(t % b.ni);
            j = b.j0 + (int)((t / b.ni) % b.nj);
            k = b.k0 + (int)(t / ((long)b.ni * b.nj));
            in = member(R, J, i, j, k, h, rc2, dx, dy, dz, r2);
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wsum[wid] = __popc(m);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) off += wsum[w];
            tot += wsum[w];
        }
        if (in) {
            const int e = base + off + __popc(m & ((1u << lane) - 1u));
            const double g = exp(-r2 / two_s2);
            const double c4[4] = {Y00 * g, Y1 * dx * g, Y1 * dy * g, Y1 * dz * g};
            idx[e] = i + n0 * (j + n1 * k);
            ent_atom[e] = J;
            for (int l = 0; l < 4; ++l) {
                chi[4L * e + l] = c4[l];
                chi_f[4L * e + l] = (float)c4[l];
                const double gc = h3 * gamma[4 * J + l] * c4[l];
                gchi[4L * e + l] = gc;
                gchi_f[4L * e + l] = (float)gc;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
}

cudaError_t support_fill(int n0, int n1, int n2, double h, int natoms, const double *R_dev,
                         const double *gamma_dev, double sigma, double rcut,
                         const int *atom_ptr, int *idx, double *chi, float *chi_f,
                         double *gchi, float *gchi_f, int *ent_atom, cudaStream_t st)
{
    if (natoms == 0) return cudaSuccess;
    k_support_fill<<<natoms, 256, 0, st>>>(n0, n1, n2, h, R_dev, gamma_dev, sigma, rcut, atom_ptr,
                                           idx, chi, chi_f, gchi, gchi_f, ent_atom);
    note_launch();
    return cudaGetLastError();
}

// ---- exclusive scan of ints (three passes: block sums, scan of sums, local scan) ----
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // items per thread

__device__ int block_excl_scan(int v, int *sh, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    total = sh[nw - 1];
    const int pre = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    __syncthreads();
    return pre;
}

__global__ void k_scan_sums(const int *in, long n, int *sums)
{
    __shared__ int sh[32];
    const long base = (long)blockIdx.x * kScanBlock * kScanItems;
    int v = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const long q = base + (long)threadIdx.x * kScanItems + t;
        if (q < n) v += in[q];
    }
    int total;
    block_excl_scan(v, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_top(int *sums, int nb)
{
    __shared__ int sh[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int q = b0 + threadIdx.x;
        const int v = q < nb ? sums[q] : 0;
        int total;
        const int pre = block_excl_scan(v, sh, total);
        if (q < nb) sums[q] = carry + pre;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void k_scan_local(const int *in, long n, const int *sums, int *out)
{
    __shared__ int sh[32];
    const long base = (long)blockIdx.x * kScanBlock * kScanItems;
    int vals[kScanItems];
    int v = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const long q = base + (long)threadIdx.x * kScanItems + t;
        vals[t] = q < n ? in[q] : 0;
        v += vals[t];
    }
    int total;
    int pre = block_excl_scan(v, sh, total) + sums[blockIdx.x];
    for (int t = 0; t < kScanItems; ++t) {
        const long q = base + (long)threadIdx.x * kScanItems + t;
        if (q < n) out[q] = pre;
        pre += vals[t];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = pre;
}

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total.
// tmp: ceil(n / 4096) ints.
cudaError_t exclusive_scan_int(const int *in, int *out, long n, int *tmp, cudaStream_t st)
{
    const long per = (long)kScanBlock * kScanItems;
    const int nb = (int)((n + per - 1) / per);
    if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
    k_scan_sums<<<nb, kScanBlock, 0, st>>>(in, n, tmp);
    note_launch();
    k_scan_top<<<1, kScanBlock, 0, st>>>(tmp, nb);
    note_launch();
    k_scan_local<<<nb, kScanBlock, 0, st>>>(in, n, tmp, out);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_count_nodes(const int *idx, long nsup, int *node_cnt)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nsup;
         e += (long)gridDim.x * blockDim.x)
        atomicAdd(&node_cnt[idx[e]], 1);
}

__global__ void k_place_entries(const int *idx, long nsup, const int *node_start, int *cursor,
                                int *ent_list)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nsup;
         e += (long)gridDim.x * blockDim.x) {
        const int p = idx[e];
        const int slot = atomicAdd(&cursor[p], 1);
        ent_list[node_start[p] + slot] = (int)e;
    }
}

// Sorts each node's entry list ascending (lists hold a few entries) and marks covered nodes.
__global__ void k_sort_lists(long nd, const int *node_start, int *ent_list, int *flags)
{
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
         p += (long)gridDim.x * blockDim.x) {
        const int b = node_start[p], e = node_start[p + 1];
        flags[p] = e > b ? 1 : 0;
        for (int a = b + 1; a < e; ++a) {
            const int v = ent_list[a];
            int c = a - 1;
            while (c >= b && ent_list[c] > v) {
                ent_list[c + 1] = ent_list[c];
                --c;
            }
            ent_list[c + 1] = v;
        }
    }
}

__global__ void k_compact_nodes(long nd, const int *flags, const int *rank, const int *node_start,
                                int *uniq_node, int *uniq_ptr, long nsup)
{
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
         p += (long)gridDim.x * blockDim.x) {
        if (flags[p]) {
            uniq_node[rank[p]] = (int)p;
            uniq_ptr[rank[p]] = node_start[p];
        }
        if (p == nd - 1) uniq_ptr[rank[nd]] = (int)nsup;
    }
}

cudaError_t build_inverse_map(long nd, long nsup, const int *idx, int *node_cnt,
                              int *node_start, int *cursor, int *ent_list, int *flags,
                              int *uniq_rank, int *scan_tmp, int *uniq_node, int *uniq_ptr,
                              cudaStream_t st)
{
    cudaError_t err;
    const int grid = 152 * 8;
    if ((err = cudaMemsetAsync(node_cnt, 0, sizeof(int) * nd, st)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(cursor, 0, sizeof(int) * nd, st)) != cudaSuccess) return err;
    k_count_nodes<<<grid, 256, 0, st>>>(idx, nsup, node_cnt);
    note_launch();
    if ((err = exclusive_scan_int(node_cnt, node_start, nd, scan_tmp, st)) != cudaSuccess)
        return err;
    k_place_entries<<<grid, 256, 0, st>>>(idx, nsup, node_start, cursor, ent_list);
    note_launch();
    k_sort_lists<<<grid, 256, 0, st>>>(nd, node_start, ent_list, flags);
    note_launch();
    if ((err = exclusive_scan_int(flags, uniq_rank, nd, scan_tmp, st)) != cudaSuccess) return err;
    k_compact_nodes<<<grid, 256, 0, st>>>(nd, flags, uniq_rank, node_start, uniq_node, uniq_ptr,
                                          nsup);
    note_launch();
    return cudaGetLastError();
}

// Node-ordered copies of the entry data for the scatter kernels: for every position q of
// ent_list, the atom and h^3 gamma chi of entry ent_list[q] (FP32 and FP32 pair), so a
// covered node reads its entries contiguously.
__global__ void k_nl_node_tables(long nuniq, const int *uniq_ptr, const int *ent_list,
                                 const int *ent_atom, const double *gchi, int *nl_atom,
                                 float *nl_gf, float2 *nl_gdf)
{
    for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < nuniq;
         u += (long)gridDim.x * blockDim.x) {
        for (int q = uniq_ptr[u]; q < uniq_ptr[u + 1]; ++q) {
            const int e = ent_list[q];
            nl_atom[q] = ent_atom[e];
            for (int l = 0; l < 4; ++l) {
                const double g = gchi[4L * e + l];
                const float gh = (float)g;
                nl_gf[4L * q + l] = gh;
                nl_gdf[4L * q + l] = make_float2(gh, (float)(g - (double)gh));
            }
        }
    }
}

cudaError_t build_nl_node_tables(long nuniq, const int *uniq_ptr, const int *ent_list,
                                 const int *ent_atom, const double *gchi, int *nl_atom,
                                 float *nl_gf, float2 *nl_gdf, cudaStream_t st)
{
    if (nuniq == 0) return cudaSuccess;
    k_nl_node_tables<<<152 * 4, 256, 0, st>>>(nuniq, uniq_ptr, ent_list, ent_atom, gchi, nl_atom,
                                              nl_gf, nl_gdf);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_to_float(const double *in, float *out, long n)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

cudaError_t to_float(const double *in, float *out, long n, cudaStream_t st)
{
    k_to_float<<<152 * 8, 256, 0, st>>>(in, out, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sparc
