// k_check.cu -- Algorithm 6 (collision check of the whole RVE) as a gather
// kernel, the colliding-pair list, the FP64 certification of the final state
// and the gather of P back to particle-id order.
//
// Every particle walks the cells within H of its home cell in a fixed order;
// per-particle results are flags and counts, reduced per warp with
// __reduce_add_sync and added to one 64-bit counter per RVE: integer sums,
// so the totals do not depend on scheduling.
#include "srm_dev.cuh"
#include "srm_launch.h"
#include "srm_stencil.cuh"

#include <type_traits>

namespace srm {

__device__ __forceinline__ void decode_cell(uint32_t c, const int32_t gn[3], int &x, int &y, int &z)
{
    x = (int)(c % (uint32_t)gn[0]);
    y = (int)((c / (uint32_t)gn[0]) % (uint32_t)gn[1]);
    z = (int)(c / ((uint32_t)gn[0] * (uint32_t)gn[1]));
}

__device__ __forceinline__ int wrapi(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// ---------------------------------------------------------------------------
// Algorithm 6 with a full count: one warp per cell stages the stencil's
// particles in shared memory, then for each particle of the cell the lanes
// test interleaved slices of the candidates and vote; the flag of every
// particle (sorted order) and the number of colliding particles result.
// ---------------------------------------------------------------------------
template <int DIM, bool F32>
__global__ void __launch_bounds__(SW_WARPS * 32) k_check(RveDev *st, int cap)
{
    extern __shared__ __align__(32) unsigned char smem[];
    if (!st->active || !st->do_check) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int cell = blockIdx.x * SW_WARPS + wib;
    int count = 0;
    unsigned examined = 0;
    if (cell < st->ncells) {
        const uint32_t *cs = st->cell_start;
        const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
        if (nh > 0) {
            using PT = typename std::conditional<F32, float4, double4_32a>::type;
            unsigned char *base = smem + (size_t)wib * warp_smem_bytes<PT>(cap);
            StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
            PT *cpos = reinterpret_cast<PT *>(base + ST_HDR);
            uint32_t *cidx = reinterpret_cast<uint32_t *>(cpos + cap);
            const Slot d = st->slot[st->dst_idx];
            const PT *pos = reinterpret_cast<const PT *>(d.pos);
            int hx, hy, hz;
            decode_cell((uint32_t)cell, st->gn, hx, hy, hz);
            int nst, center;
            const uint32_t T = list_stencil(st, cs, hx, hy, hz, S, nst, center);
            const float w0 = (float)st->gw[0], w1 = (float)st->gw[1], w2 = (float)st->gw[2];
            const bool staged = T <= (uint32_t)cap;
            auto fetch = [&](uint32_t k, uint32_t &g) -> PT {
                const int j = find_cell(S, nst, k);
                g = S.b[j] + (k - S.o[j]);
                PT c = pos[g];
                if (F32) {
                    c.x += (float)S.sh[j][0] * w0;
                    c.y += (float)S.sh[j][1] * w1;
                    c.z += (float)S.sh[j][2] * w2;
                }
                return c;
            };
            if (staged) {
                for (uint32_t k = lane; k < T; k += 32) {
                    uint32_t g;
                    cpos[k] = fetch(k, g);
                    cidx[k] = g;
                }
                __syncwarp();
            }
            const float g1 = 1.0f + st->guard;
            for (uint32_t m = 0; m < nh; m++) {
                const uint32_t gi = hb + m;
                const PT p = pos[gi];
                bool hit = false;
                for (uint32_t k = lane; k < T && !hit; k += 32) {
                    uint32_t g;
                    PT c;
                    if (staged) {
                        c = cpos[k];
                        g = cidx[k];
                    } else {
                        c = fetch(k, g);
                    }
                    if (g == gi) continue;
                    examined++;
                    if (F32) {
                        const float ex = (float)p.x - (float)c.x, ey = (float)p.y - (float)c.y;
                        float d2 = ex * ex + ey * ey;
                        if (DIM == 3) {
                            const float ez = (float)p.z - (float)c.z;
                            d2 += ez * ez;
                        }
                        const float rs = (float)p.w + (float)c.w;
                        hit = d2 <= rs * rs * g1;
                    } else {
                        const double q[3] = {(double)p.x, (double)p.y, (double)p.z};
                        hit = collide_exact<DIM>(q, (double)p.w, (double)c.x, (double)c.y, (double)c.z,
                                                 (double)c.w, st->L, st->halfL);
                    }
                }
                const bool any = __any_sync(0xffffffffu, hit);
                if (lane == 0) st->flags[gi] = (uint8_t)any;
                count += any;
            }
        }
    }
    if (lane == 0 && count) atomicAdd(&st->red[0], (unsigned long long)count);
    examined = __reduce_add_sync(0xffffffffu, examined);
    if (lane == 0 && examined) atomicAdd(&st->pairs_check, (unsigned long long)examined);
}

// ---------------------------------------------------------------------------
// Inspection of P in binary64: a fresh binning of P at its own scale into a
// scratch slot (absolute binary64 positions for either form), then pairs and
// certification on that slot.
// ---------------------------------------------------------------------------
__global__ void k_inspect_begin(RveDev *st)
{
    if (threadIdx.x || blockIdx.x) return;
    set_grid(st, st->lam_P);
    st->src_idx = st->p_idx;
    st->dst_idx = (st->p_idx + 1) % 3;
    st->lam_R = st->lam_P;
    st->active = 1;
    st->do_check = 0;
    st->red[1] = 0;
    st->red[2] = dkey(__longlong_as_double(0x7ff0000000000000LL));  // +inf
}

__global__ void k_inspect_end(RveDev *st)
{
    if (threadIdx.x || blockIdx.x) return;
    st->active = 0;
}

// Pairs i < j (by id) with the literal predicate of Algorithm 5; per-particle
// partner counts by id, the total, and the smallest gap S - (R_i + R_j).
template <int DIM>
__global__ void __launch_bounds__(256) k_pairs_count(RveDev *st, int want_gap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    double mg = __longlong_as_double(0x7ff0000000000000LL);
    if (i < st->n) {
        const Slot d = st->slot[st->dst_idx];
        const double4_32a *pos = reinterpret_cast<const double4_32a *>(d.pos);
        const uint32_t *cs = st->cell_start;
        const uint32_t me = d.pid[i];
        int hx, hy, hz;
        decode_cell(d.cell[i], st->gn, hx, hy, hz);
        const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
        const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
        const double4_32a p = pos[i];
        const double q[3] = {p.x, p.y, p.z};
        for (int dz = -H2; dz <= H2; dz++)
            for (int dy = -H1; dy <= H1; dy++) {
                const int row = n0 * (wrapi(hy + dy, n1) + n1 * wrapi(hz + dz, n2));
                for (int dx = -H0; dx <= H0; dx++) {
                    const int c = row + wrapi(hx + dx, n0);
                    for (uint32_t j = cs[c]; j < cs[c + 1]; j++) {
                        if (d.pid[j] <= me) continue;
                        const double4_32a t = pos[j];
                        const double tt[3] = {t.x, t.y, t.z};
                        double gap;
                        if (gap_exact<DIM>(q, p.w, tt, t.w, st->L, st->halfL, &gap)) cnt++;
                        if (gap < mg) mg = gap;
                    }
                }
            }
        st->pcount[me] = (uint32_t)cnt;
    }
    const int tot = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&st->red[1], (unsigned long long)tot);
    if (want_gap) {
        unsigned long long key = dkey(mg);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
            key = y < key ? y : key;
        }
        if ((threadIdx.x & 31) == 0) atomicMin(&st->red[2], key);
    }
}

// Partners of each particle at its offset, ascending partner id.
template <int DIM>
__global__ void __launch_bounds__(256) k_pairs_fill(RveDev *st, long long *ij)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st->n) return;
    const Slot d = st->slot[st->dst_idx];
    const double4_32a *pos = reinterpret_cast<const double4_32a *>(d.pos);
    const uint32_t *cs = st->cell_start;
    const uint32_t me = d.pid[i];
    const long long base = st->pcount[me];
    const long long cnt = (long long)st->pcount[me + 1] - base;
    if (cnt == 0) return;
    int hx, hy, hz;
    decode_cell(d.cell[i], st->gn, hx, hy, hz);
    const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
    const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
    const double4_32a p = pos[i];
    const double q[3] = {p.x, p.y, p.z};
    long long k = 0;
    for (int dz = -H2; dz <= H2; dz++)
        for (int dy = -H1; dy <= H1; dy++) {
            const int row = n0 * (wrapi(hy + dy, n1) + n1 * wrapi(hz + dz, n2));
            for (int dx = -H0; dx <= H0; dx++) {
                const int c = row + wrapi(hx + dx, n0);
                for (uint32_t j = cs[c]; j < cs[c + 1]; j++) {
                    const uint32_t other = d.pid[j];
                    if (other <= me) continue;
                    const double4_32a t = pos[j];
                    const double tt[3] = {t.x, t.y, t.z};
                    double gap;
                    if (gap_exact<DIM>(q, p.w, tt, t.w, st->L, st->halfL, &gap) && k < cnt) {
                        // insertion into the sorted run [base, base + k)
                        long long at = base + k;
                        while (at > base && ij[2 * (at - 1) + 1] > (long long)other) {
                            ij[2 * at] = ij[2 * (at - 1)];
                            ij[2 * at + 1] = ij[2 * (at - 1) + 1];
                            at--;
                        }
                        ij[2 * at] = (long long)me;
                        ij[2 * at + 1] = (long long)other;
                        k++;
                    }
                }
            }
        }
}

// P in particle-id order: positions (binary64, wrapped into [0, L)) and
// radii R_i = lambda_P r_i.
template <int DIM, bool F32>
__global__ void __launch_bounds__(256) k_gather(RveDev *st, double *xyz, double *rad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st->n) return;
    const Slot s = st->slot[st->p_idx];
    const uint32_t id = s.pid[i];
    double x[3];
    if (!F32) {
        const double4_32a p = reinterpret_cast<const double4_32a *>(s.pos)[i];
        x[0] = p.x;
        x[1] = p.y;
        x[2] = p.z;
    } else {
        const float4 p = reinterpret_cast<const float4 *>(s.pos)[i];
        int cx, cy, cz;
        decode_cell(s.cell[i], s.gn, cx, cy, cz);
        const int cc[3] = {cx, cy, cz};
        const float o[3] = {p.x, p.y, p.z};
        for (int a = 0; a < DIM; a++)
            x[a] = wrap_d(__dadd_rn(__dmul_rn((double)cc[a], s.gw[a]), (double)o[a]), st->L[a]);
    }
    for (int a = 0; a < DIM; a++) xyz[(size_t)id * DIM + a] = x[a];
    if (rad) rad[id] = __dmul_rn(st->lam_P, s.rb[i]);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

int check_cap_max(bool f32) { return f32 ? 1024 : 512; }

static size_t check_smem(bool f32, int cap)
{
    return SW_WARPS * (f32 ? warp_smem_bytes<float4>(cap) : warp_smem_bytes<double4_32a>(cap));
}

void launch_check(RveDev *d_st, const HostShape &sh, cudaStream_t s)
{
    const int nb = blocks_for(sh.ncells_cap, SW_WARPS);
    const int cap = sh.cap_check;
    const size_t smem = check_smem(sh.f32, cap);
    if (sh.dim == 2) {
        if (sh.f32) k_check<2, true><<<nb, SW_WARPS * 32, smem, s>>>(d_st, cap);
        else k_check<2, false><<<nb, SW_WARPS * 32, smem, s>>>(d_st, cap);
    } else {
        if (sh.f32) k_check<3, true><<<nb, SW_WARPS * 32, smem, s>>>(d_st, cap);
        else k_check<3, false><<<nb, SW_WARPS * 32, smem, s>>>(d_st, cap);
    }
}

void check_configure()
{
    const int s32 = (int)check_smem(true, check_cap_max(true));
    const int s64 = (int)check_smem(false, check_cap_max(false));
    cudaFuncSetAttribute(k_check<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_check<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_check<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(k_check<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
}

void launch_inspect_bin(RveDev *d_st, const HostShape &sh, cudaStream_t s)
{
    k_inspect_begin<<<1, 1, 0, s>>>(d_st);
    HostShape b = sh;
    b.out_f32 = false;
    launch_bin(d_st, b, s);
}

void launch_pairs_count(RveDev *d_st, const HostShape &sh, int want_gap, cudaStream_t s)
{
    const int nb = blocks_for(sh.n, 256);
    if (sh.dim == 2) k_pairs_count<2><<<nb, 256, 0, s>>>(d_st, want_gap);
    else k_pairs_count<3><<<nb, 256, 0, s>>>(d_st, want_gap);
}

void launch_pairs_fill(RveDev *d_st, const HostShape &sh, long long *ij, cudaStream_t s)
{
    const int nb = blocks_for(sh.n, 256);
    if (sh.dim == 2) k_pairs_fill<2><<<nb, 256, 0, s>>>(d_st, ij);
    else k_pairs_fill<3><<<nb, 256, 0, s>>>(d_st, ij);
}

void launch_inspect_end(RveDev *d_st, cudaStream_t s) { k_inspect_end<<<1, 1, 0, s>>>(d_st); }

void launch_gather(RveDev *d_st, const HostShape &sh, double *xyz, double *rad, cudaStream_t s)
{
    const int nb = blocks_for(sh.n, 256);
    if (sh.dim == 2) {
        if (sh.f32) k_gather<2, true><<<nb, 256, 0, s>>>(d_st, xyz, rad);
        else k_gather<2, false><<<nb, 256, 0, s>>>(d_st, xyz, rad);
    } else {
        if (sh.f32) k_gather<3, true><<<nb, 256, 0, s>>>(d_st, xyz, rad);
        else k_gather<3, false><<<nb, 256, 0, s>>>(d_st, xyz, rad);
    }
}

}  // namespace srm
