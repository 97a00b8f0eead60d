// srm_stencil.cuh -- the neighbour stencil of one cell, listed and staged
// by one warp in shared memory (used by the sweep and the check kernels).
#pragma once

#include "srm_dev.cuh"

namespace srm {

constexpr int SW_WARPS = 4;
constexpr int MAX_ST = 125;

struct StencilSmem {
    uint32_t b[MAX_ST];  // first sorted index of stencil cell j
    uint32_t o[MAX_ST + 1];  // offset of cell j in the flattened candidate list
    int32_t cell[MAX_ST];    // linear index of stencil cell j (staged path)
    int8_t sh[MAX_ST][3];    // unwrapped shift of cell j from the home cell
    uint8_t low[MAX_ST];     // 1: cell j has a lower colour than the home cell (staged path)
    uint32_t n[MAX_ST];      // particles of cell j (staged path)
};

constexpr size_t ST_HDR = (sizeof(StencilSmem) + 31) / 32 * 32;

// Shared memory of one warp: stencil list, staged positions, staged indices
// (rounded to 32 bytes so that every warp's positions stay 32-byte aligned).
template <typename PT>
__host__ __device__ constexpr size_t warp_smem_bytes(int cap)
{
    return (ST_HDR + (size_t)cap * sizeof(PT) + (size_t)cap * 4 + 31) / 32 * 32;
}

// Lists the stencil cells of home (hx, hy, hz) and returns the candidate
// count; the home cell is stencil cell 0, so its particles are candidates
// 0 .. n_home-1.
__device__ __forceinline__ uint32_t list_stencil(const RveDev *st, const uint32_t *cs, int hx, int hy,
                                                 int hz, StencilSmem &S, int &nst, int &center)
{
    const int lane = threadIdx.x & 31;
    const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
    const int w0 = 2 * H0 + 1, w1 = 2 * H1 + 1, w2 = 2 * H2 + 1;
    nst = w0 * w1 * w2;
    center = H0 + w0 * (H1 + w1 * H2);
    const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
    uint32_t carry = 0;
    for (int base = 0; base < nst; base += 32) {
        const int j = base + lane;
        uint32_t cnt = 0;
        if (j < nst) {
            // the home cell is listed first: stencil position 0 <-> offset
            // index `center`, so the home particles lead the candidate list
            const int jj = j == 0 ? center : (j == center ? 0 : j);
            const int dx = jj % w0 - H0, dy = (jj / w0) % w1 - H1, dz = jj / (w0 * w1) - H2;
            int cx = hx + dx, cy = hy + dy, cz = hz + dz;
            cx = cx < 0 ? cx + n0 : (cx >= n0 ? cx - n0 : cx);
            cy = cy < 0 ? cy + n1 : (cy >= n1 ? cy - n1 : cy);
            cz = cz < 0 ? cz + n2 : (cz >= n2 ? cz - n2 : cz);
            const int c = cx + n0 * (cy + n1 * cz);
            const uint32_t b = cs[c];
            cnt = cs[c + 1] - b;
            S.b[j] = b;
            S.sh[j][0] = (int8_t)dx;
            S.sh[j][1] = (int8_t)dy;
            S.sh[j][2] = (int8_t)dz;
        }
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (j < nst) S.o[j] = carry + inc - cnt;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) S.o[nst] = carry;
    __syncwarp();
    return carry;
}

// The stencil of the staged path: as list_stencil, but the candidates of
// the cells that are not of lower colour (the home cell first) are numbered
// 0 .. n_other-1 and those of the lower-colour cells 0 .. n_low-1 in a second
// list (o[j] indexes the list of cell j's kind); n[j] holds the counts.
__device__ __forceinline__ void list_stencil_split(const RveDev *st, const uint32_t *cs, int hx, int hy, int hz,
                                                   int chi, StencilSmem &S, int &nst, uint32_t &n_other,
                                                   uint32_t &n_low)
{
    const int lane = threadIdx.x & 31;
    const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
    const int w0 = 2 * H0 + 1, w1 = 2 * H1 + 1, w2 = 2 * H2 + 1;
    nst = w0 * w1 * w2;
    const int center = H0 + w0 * (H1 + w1 * H2);
    const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
    uint32_t carry_o = 0, carry_l = 0;
    for (int base = 0; base < nst; base += 32) {
        const int j = base + lane;
        uint32_t co = 0, cl = 0;
        bool lo = false;
        if (j < nst) {
            const int jj = j == 0 ? center : (j == center ? 0 : j);
            const int dx = jj % w0 - H0, dy = (jj / w0) % w1 - H1, dz = jj / (w0 * w1) - H2;
            int cx = hx + dx, cy = hy + dy, cz = hz + dz;
            cx = cx < 0 ? cx + n0 : (cx >= n0 ? cx - n0 : cx);
            cy = cy < 0 ? cy + n1 : (cy >= n1 ? cy - n1 : cy);
            cz = cz < 0 ? cz + n2 : (cz >= n2 ? cz - n2 : cz);
            const int c = cx + n0 * (cy + n1 * cz);
            const uint32_t b = cs[c];
            const uint32_t cnt = cs[c + 1] - b;
            lo = cx % 3 + 3 * (cy % 3) + 9 * (cz % 3) < chi;
            S.b[j] = b;
            S.n[j] = cnt;
            S.cell[j] = c;
            S.low[j] = (uint8_t)lo;
            S.sh[j][0] = (int8_t)dx;
            S.sh[j][1] = (int8_t)dy;
            S.sh[j][2] = (int8_t)dz;
            (lo ? cl : co) = cnt;
        }
        uint32_t io = co, il = cl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yo = __shfl_up_sync(0xffffffffu, io, o), yl = __shfl_up_sync(0xffffffffu, il, o);
            if (lane >= o) {
                io += yo;
                il += yl;
            }
        }
        if (j < nst) S.o[j] = lo ? carry_l + il - cl : carry_o + io - co;
        carry_o += __shfl_sync(0xffffffffu, io, 31);
        carry_l += __shfl_sync(0xffffffffu, il, 31);
    }
    n_other = carry_o;
    n_low = carry_l;
    __syncwarp();
}

// Squared distance from a point (relative to the home corner) to the home box.
__device__ __forceinline__ float box_dist2(const float4 &t, const float w[3], int dim)
{
    const float ex = fmaxf(fmaxf(-t.x, t.x - w[0]), 0.f);
    const float ey = fmaxf(fmaxf(-t.y, t.y - w[1]), 0.f);
    const float ez = dim == 3 ? fmaxf(fmaxf(-t.z, t.z - w[2]), 0.f) : 0.f;
    return ex * ex + ey * ey + ez * ez;
}

// Stencil cell holding flattened candidate k (binary search over offsets).
__device__ __forceinline__ int find_cell(const StencilSmem &S, int nst, uint32_t k)
{
    int lo = 0, hi = nst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.o[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


}  // namespace srm
