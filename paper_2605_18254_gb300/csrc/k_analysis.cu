// k_analysis.cu -- structure descriptors of a generated configuration
// (Section 3.2): nearest neighbours (centre distance and partner, smallest
// surface gap; Fig. 4d), the radial distribution of the centres, and the
// local volume fraction of every particle from a discrete periodic Voronoi
// tessellation (particle volume over the volume of its Voronoi cell, Figs. 5
// and 7).  They read the binary64 copy of P binned on the grid of its own
// scale (the binning of the certification) and evaluate every distance with
// the same binary64 operations as the definitions: minimum-image difference
// per axis, squared distance summed in axis order, correctly rounded root.
//
// Searches grow ring by ring around the home cell: after the cells within H
// of it (per axis), every particle not yet examined is at least H w_min away
// from any point of the home cell, so the search stops once the best
// distance is within that bound (or the whole grid has been examined).
#include "srm_dev.cuh"
#include "srm_launch.h"

namespace srm {

namespace {

__device__ __forceinline__ int wrap_cell(int c, int n)
{
    c %= n;
    return c < 0 ? c + n : c;
}

template <int DIM>
__device__ __forceinline__ double dist2_exact(const double q[3], const double t[3], const double L[3],
                                              const double halfL[3])
{
    double ss = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        double d = __dsub_rn(q[a], t[a]);
        if (d > halfL[a]) d = __dsub_rn(d, L[a]);
        if (d < -halfL[a]) d = __dadd_rn(d, L[a]);
        ss = a == 0 ? __dmul_rn(d, d) : __dadd_rn(ss, __dmul_rn(d, d));
    }
    return ss;
}

// Calls f(j) for every sorted index j in the cells at Chebyshev ring H
// (exactly) around cell (hx, hy, hz); rings larger than the grid visit
// wrapped cells again (harmless for minima).
template <int DIM, typename F>
__device__ __forceinline__ void for_ring(const RveDev *st, int hx, int hy, int hz, int H, F f)
{
    const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
    const uint32_t *cs = st->cell_start;
    const int Hz = DIM == 3 ? H : 0;
    for (int dz = -Hz; dz <= Hz; dz++)
        for (int dy = -H; dy <= H; dy++)
            for (int dx = -H; dx <= H; dx++) {
                const int ring = max(max(abs(dx), abs(dy)), abs(dz));
                if (ring != H) continue;
                const int c = wrap_cell(hx + dx, n0) + n0 * (wrap_cell(hy + dy, n1) + n1 * wrap_cell(hz + dz, n2));
                for (uint32_t j = cs[c]; j < cs[c + 1]; j++) f(j);
            }
}

__device__ __forceinline__ int ring_cap(const RveDev *st, int dim)
{
    int m = 0;
    for (int a = 0; a < dim; a++) m = max(m, st->gn[a] / 2 + 1);
    return m;
}

__device__ __forceinline__ double w_min(const RveDev *st, int dim)
{
    double w = st->gw[0];
    for (int a = 1; a < dim; a++) w = fmin(w, st->gw[a]);
    return w * (1.0 - 1e-12);  // a point may sit an ulp outside its cell
}

}  // namespace

// One thread per particle (sorted order); results by particle id.
template <int DIM>
__global__ void __launch_bounds__(256) k_nearest(const RveDev *st, double *nn_dist, long long *nn_id, double *gap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st->n) return;
    const Slot d = st->slot[st->dst_idx];
    const double4_32a *pos = reinterpret_cast<const double4_32a *>(d.pos);
    const double4_32a p = pos[i];
    const double q[3] = {p.x, p.y, p.z};
    const uint32_t me = d.pid[i];
    const uint32_t c = d.cell[i];
    const int hx = (int)(c % (uint32_t)st->gn[0]), hy = (int)((c / (uint32_t)st->gn[0]) % (uint32_t)st->gn[1]);
    const int hz = (int)(c / ((uint32_t)st->gn[0] * (uint32_t)st->gn[1]));
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double bs = inf, bg = inf;
    uint32_t bj = 0xffffffffu;
    const double wm = w_min(st, DIM), Rmax = __dmul_rn(st->lam_P, st->rmax);
    const int cap = ring_cap(st, DIM);
    for (int H = 0; H <= cap; H++) {
        for_ring<DIM>(st, hx, hy, hz, H, [&](uint32_t j) {
            const uint32_t id = d.pid[j];
            if (id == me) return;
            const double4_32a t = pos[j];
            const double tt[3] = {t.x, t.y, t.z};
            const double S = __dsqrt_rn(dist2_exact<DIM>(q, tt, st->L, st->halfL));
            if (S < bs || (S == bs && id < bj)) {
                bs = S;
                bj = id;
            }
            const double g = __dsub_rn(S, __dadd_rn(p.w, t.w));
            if (g < bg) bg = g;
        });
        // unexamined particles: S >= H wm, gap >= H wm - R_i - R_max
        const double reach = H * wm;
        if (H >= 1 && bs <= reach && bg <= reach - p.w - Rmax) break;
    }
    nn_dist[me] = bs;
    if (nn_id) nn_id[me] = bj == 0xffffffffu ? -1 : (long long)bj;
    gap[me] = bg;
}

// Ordered pairs (i, j), i != j, with S_ij < r_max, by bin floor(S / dr);
// the cell offsets lo_a..hi_a around the home cell hold every such partner
// and visit each cell once (-H..H with H = ceil(r_max / w_a), or the whole
// axis when 2 H + 1 >= n_a).  Block histogram in shared memory, added to the
// global counts.
struct Offs {
    int lo[3], hi[3];
};

template <int DIM>
__global__ void __launch_bounds__(256) k_rdf(const RveDev *st, double r_max, int bins, double dr, Offs o,
                                             unsigned long long *counts)
{
    extern __shared__ unsigned long long hist[];
    for (int b = threadIdx.x; b < bins; b += blockDim.x) hist[b] = 0ull;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < st->n) {
        const Slot d = st->slot[st->dst_idx];
        const double4_32a *pos = reinterpret_cast<const double4_32a *>(d.pos);
        const uint32_t *cs = st->cell_start;
        const double4_32a p = pos[i];
        const double q[3] = {p.x, p.y, p.z};
        const uint32_t c = d.cell[i];
        const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
        const int hx = (int)(c % (uint32_t)n0), hy = (int)((c / (uint32_t)n0) % (uint32_t)n1);
        const int hz = (int)(c / ((uint32_t)n0 * (uint32_t)n1));
        for (int dz = o.lo[2]; dz <= o.hi[2]; dz++)
            for (int dy = o.lo[1]; dy <= o.hi[1]; dy++)
                for (int dx = o.lo[0]; dx <= o.hi[0]; dx++) {
                    const int cc = wrap_cell(hx + dx, n0) + n0 * (wrap_cell(hy + dy, n1) + n1 * wrap_cell(hz + dz, n2));
                    for (uint32_t j = cs[cc]; j < cs[cc + 1]; j++) {
                        if (j == (uint32_t)i) continue;
                        const double4_32a t = pos[j];
                        const double tt[3] = {t.x, t.y, t.z};
                        const double S = __dsqrt_rn(dist2_exact<DIM>(q, tt, st->L, st->halfL));
                        if (!(S < r_max)) continue;
                        const long long b = (long long)floor(__ddiv_rn(S, dr));
                        if (b < bins) atomicAdd(&hist[b], 1ull);
                    }
                }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bins; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], hist[b]);
}

// One thread per voxel (x fastest): the voxel centre ((i_a + 0.5) h_a)
// belongs to the particle with the smallest squared minimum-image distance,
// ties to the smaller id; voxel counts by particle id.
template <int DIM>
__global__ void __launch_bounds__(256) k_voronoi(const RveDev *st, int M0, int M1, int M2, double h0, double h1,
                                                 double h2, long long total, unsigned long long *count)
{
    const Slot d = st->slot[st->dst_idx];
    const double4_32a *pos = reinterpret_cast<const double4_32a *>(d.pos);
    const double wm = w_min(st, DIM);
    const int cap = ring_cap(st, DIM);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const long long ix = v % M0, iy = (v / M0) % M1, iz = DIM == 3 ? v / ((long long)M0 * M1) : 0;
        const double q[3] = {__dmul_rn(__dadd_rn((double)ix, 0.5), h0), __dmul_rn(__dadd_rn((double)iy, 0.5), h1),
                             DIM == 3 ? __dmul_rn(__dadd_rn((double)iz, 0.5), h2) : 0.0};
        const int hx = cell_coord_d(q[0], st->gw[0], st->gn[0]), hy = cell_coord_d(q[1], st->gw[1], st->gn[1]);
        const int hz = DIM == 3 ? cell_coord_d(q[2], st->gw[2], st->gn[2]) : 0;
        double best = inf;
        uint32_t bj = 0xffffffffu;
        for (int H = 0; H <= cap; H++) {
            for_ring<DIM>(st, hx, hy, hz, H, [&](uint32_t j) {
                const double4_32a t = pos[j];
                const double tt[3] = {t.x, t.y, t.z};
                const double s = dist2_exact<DIM>(q, tt, st->L, st->halfL);
                const uint32_t id = d.pid[j];
                if (s < best || (s == best && id < bj)) {
                    best = s;
                    bj = id;
                }
            });
            const double reach = H * wm;
            if (H >= 1 && best <= __dmul_rn(reach, reach)) break;
        }
        if (bj != 0xffffffffu) atomicAdd(&count[bj], 1ull);
    }
}

void launch_nearest(RveDev *d_st, int dim, int64_t n, double *nn_dist, long long *nn_id, double *gap, cudaStream_t s)
{
    const int nb = (int)((n + 255) / 256);
    if (dim == 2) k_nearest<2><<<nb, 256, 0, s>>>(d_st, nn_dist, nn_id, gap);
    else k_nearest<3><<<nb, 256, 0, s>>>(d_st, nn_dist, nn_id, gap);
}

void launch_rdf(RveDev *d_st, int dim, int64_t n, double r_max, int bins, const int lo[3], const int hi[3],
                unsigned long long *counts, cudaStream_t s)
{
    const int nb = (int)((n + 255) / 256);
    const double dr = r_max / (double)bins;
    const size_t smem = sizeof(unsigned long long) * (size_t)bins;
    Offs o;
    for (int a = 0; a < 3; a++) {
        o.lo[a] = a < dim ? lo[a] : 0;
        o.hi[a] = a < dim ? hi[a] : 0;
    }
    if (dim == 2) k_rdf<2><<<nb, 256, smem, s>>>(d_st, r_max, bins, dr, o, counts);
    else k_rdf<3><<<nb, 256, smem, s>>>(d_st, r_max, bins, dr, o, counts);
}

void launch_voronoi(RveDev *d_st, int dim, const int32_t M[3], const double h[3], unsigned long long *count,
                    cudaStream_t s)
{
    const long long total = (long long)M[0] * M[1] * (dim == 3 ? M[2] : 1);
    long long nb = (total + 255) / 256;
    if (nb > 152 * 64) nb = 152 * 64;
    if (dim == 2) k_voronoi<2><<<(int)nb, 256, 0, s>>>(d_st, M[0], M[1], 1, h[0], h[1], 1.0, total, count);
    else k_voronoi<3><<<(int)nb, 256, 0, s>>>(d_st, M[0], M[1], M[2], h[0], h[1], h[2], total, count);
}

}  // namespace srm
