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
// Algorithm 6 with a full count, after a sweep (one thread per particle,
// walking the cells within H of its home cell).  Every particle moves at most
// once per sweep and a move is accepted only if the new position collides
// with no particle at that moment; every other particle is then either at
// its final position already or will itself move only to a position that
// collides with nothing.  Hence a pair in which at least one particle moved
// cannot collide at the end of the sweep, and the colliding particles of
// Algorithm 6 are exactly the non-moved particles that collide with another
// non-moved particle (the same predicate is evaluated on the same values, so
// the count equals the full check's).  Moved particles return at once, and
// the others test non-moved candidates only.
// ---------------------------------------------------------------------------
template <int DIM, bool F32>
__device__ __forceinline__ void check_one(RveDev *st, int i, int &hit, unsigned &examined)
{
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    {
        const Slot d = st->slot[st->dst_idx];
        const PT *pos = reinterpret_cast<const PT *>(d.pos);
        const uint32_t *cs = st->cell_start;
        int hx, hy, hz;
        decode_cell(d.cell[i], st->gn, hx, hy, hz);
        const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
        const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
        const float w0 = (float)st->gw[0], w1 = (float)st->gw[1], w2 = (float)st->gw[2];
        const float g1 = 1.0f + st->guard;
        const PT p = pos[i];
        for (int dz = -H2; dz <= H2 && !hit; dz++)
            for (int dy = -H1; dy <= H1 && !hit; dy++) {
                const int row = n0 * (wrapi(hy + dy, n1) + n1 * wrapi(hz + dz, n2));
                for (int dx = -H0; dx <= H0 && !hit; dx++) {
                    const int c = row + wrapi(hx + dx, n0);
                    for (uint32_t j = cs[c]; j < cs[c + 1]; j++) {
                        if ((int)j == i || st->flags[j]) continue;
                        examined++;
                        const PT t = pos[j];
                        bool h;
                        if constexpr (F32) {
                            // the sweep's arithmetic: shifted candidate, then
                            // the guarded predicate, with explicit roundings
                            const float ex = __fsub_rn(p.x, __fmaf_rn((float)dx, w0, t.x));
                            const float ey = __fsub_rn(p.y, __fmaf_rn((float)dy, w1, t.y));
                            float d2 = __fmaf_rn(ey, ey, __fmul_rn(ex, ex));
                            if (DIM == 3) {
                                const float ez = __fsub_rn(p.z, __fmaf_rn((float)dz, w2, t.z));
                                d2 = __fmaf_rn(ez, ez, d2);
                            }
                            const float rs = __fadd_rn(p.w, t.w);
                            h = d2 <= __fmul_rn(__fmul_rn(rs, rs), g1);
                        } else {
                            const double q[3] = {p.x, p.y, p.z};
                            h = collide64<DIM>(st->images, q, p.w, t.x, t.y, t.z, t.w, st->L, st->halfL);
                        }
                        if (h) {
                            hit = 1;
                            break;
                        }
                    }
                }
            }
    }
}

template <bool F32>
__global__ void __launch_bounds__(256) k_check(BatchDev *bd)
{
    int r;
    if (!plan_block(bd->actp, bd->B, r)) return;
    RveDev *st = bd->rv[r];
    if (!st->do_check) return;
    {
        const int i = (blockIdx.x - bd->actp[r]) * 256 + threadIdx.x;
        int hit = 0;
        unsigned examined = 0;
        if (i < st->n && !st->flags[i]) {
            if (st->dim == 3) check_one<3, F32>(st, i, hit, examined);
            else check_one<2, F32>(st, i, hit, examined);
        }
        const int tot = __reduce_add_sync(0xffffffffu, hit);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&st->red[0], (unsigned long long)tot);
        examined = __reduce_add_sync(0xffffffffu, examined);
        if ((threadIdx.x & 31) == 0 && examined) atomicAdd(&st->pairs_check, (unsigned long long)examined);
    }
}

// ---------------------------------------------------------------------------
// The same count, one warp per cell: the moved flags of the cell's particles
// decide whether it has work; if so, the non-moved particles of the cells
// within H are staged in shared memory (FP32 form: shifted into the home
// cell's frame), keeping those whose distance to the home cell box allows a
// contact with the largest non-moved home particle, and each non-moved home
// particle tests them with the lanes -- one load of each candidate per cell
// instead of one per home particle.  The predicate and its roundings are
// those of check_one, so the count is the same.  A cell whose staged set
// would exceed CK_CAP falls back to check_one per particle.
// ---------------------------------------------------------------------------
constexpr int CK_WARPS = 4;
constexpr int CK_CAP = 256;

template <bool F32>
struct CheckSmem {
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    static constexpr size_t off_gidx = ST_HDR + (size_t)CK_CAP * sizeof(PT);
    static constexpr size_t bytes = (off_gidx + (size_t)CK_CAP * 4 + 31) / 32 * 32;
};

template <int DIM, bool F32>
__device__ __forceinline__ void check_cell(RveDev *st, int cell, unsigned char *base, int &hits,
                                           unsigned &examined)
{
    using SM = CheckSmem<F32>;
    using PT = typename SM::PT;
    const int lane = threadIdx.x & 31;
    StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
    PT *cand = reinterpret_cast<PT *>(base + ST_HDR);
    uint32_t *gidx = reinterpret_cast<uint32_t *>(base + SM::off_gidx);
    const Slot d = st->slot[st->dst_idx];
    const PT *pos = reinterpret_cast<const PT *>(d.pos);
    const uint32_t *cs = st->cell_start;
    const uint8_t *flags = st->flags;
    const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
    if (nh == 0) return;
    // non-moved home particles and the largest radius among them
    bool any = false;
    float rh = 0.f;
    for (uint32_t m = lane; m < nh; m += 32)
        if (!flags[hb + m]) {
            any = true;
            rh = fmaxf(rh, (float)pos[hb + m].w);
        }
    if (!__any_sync(0xffffffffu, any)) return;
    for (int o = 16; o > 0; o >>= 1) rh = fmaxf(rh, __shfl_xor_sync(0xffffffffu, rh, o));
    int hx, hy, hz;
    decode_cell((uint32_t)cell, st->gn, hx, hy, hz);
    int nst, center;
    const uint32_t T = list_stencil(st, cs, hx, hy, hz, S, nst, center);
    const float w[3] = {(float)st->gw[0], (float)st->gw[1], (float)st->gw[2]};
    const double ox = hx * st->gw[0], oy = hy * st->gw[1], oz = hz * st->gw[2];
    auto approx = [&](const PT &c) -> float4 {
        if constexpr (F32) {
            return c;
        } else {
            double ex = c.x - ox, ey = c.y - oy, ez = DIM == 3 ? c.z - oz : 0.0;
            if (ex > st->halfL[0]) ex -= st->L[0];
            if (ex < -st->halfL[0]) ex += st->L[0];
            if (ey > st->halfL[1]) ey -= st->L[1];
            if (ey < -st->halfL[1]) ey += st->L[1];
            if (DIM == 3) {
                if (ez > st->halfL[2]) ez -= st->L[2];
                if (ez < -st->halfL[2]) ez += st->L[2];
            }
            return make_float4((float)ex, (float)ey, (float)ez, (float)c.w);
        }
    };
    // stage the non-moved candidates within reach of the home box; the flag
    // and the position of four chunks are loaded before any is used, so
    // that a cell costs few memory round trips
    constexpr int U = 4;
    uint32_t Tk = 0;
    bool overflow = false;
    for (uint32_t k0 = 0; k0 < T && !overflow; k0 += 32 * U) {
        PT c[U];
        uint8_t f[U];
        uint32_t g[U];
        int jj[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t k = k0 + 32 * u + (uint32_t)lane;
            f[u] = 1;
            g[u] = 0;
            jj[u] = 0;
            if (k < T) {
                jj[u] = find_cell(S, nst, k);
                g[u] = S.b[jj[u]] + (k - S.o[jj[u]]);
                f[u] = flags[g[u]];
                c[u] = pos[g[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            bool keep = false;
            if (!f[u]) {
                if constexpr (F32) {
                    // the shift of check_one: one fused multiply-add per axis
                    c[u].x = __fmaf_rn((float)S.sh[jj[u]][0], w[0], c[u].x);
                    c[u].y = __fmaf_rn((float)S.sh[jj[u]][1], w[1], c[u].y);
                    c[u].z = __fmaf_rn((float)S.sh[jj[u]][2], w[2], c[u].z);
                }
                const float4 ca = approx(c[u]);
                const float r = rh + ca.w;
                keep = box_dist2(ca, w, DIM) <= r * r * 1.0004f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (overflow || Tk + __popc(bal) > (uint32_t)CK_CAP) {
                overflow = true;
                continue;
            }
            if (keep) {
                const uint32_t at = Tk + __popc(bal & ((1u << lane) - 1u));
                cand[at] = c[u];
                gidx[at] = g[u];
            }
            Tk += __popc(bal);
        }
    }
    __syncwarp();
    if (overflow) {
        for (uint32_t m = lane; m < nh; m += 32) {
            int hit = 0;
            if (!flags[hb + m]) check_one<DIM, F32>(st, (int)(hb + m), hit, examined);
            hits += hit;
        }
        return;
    }
    const float g1 = 1.0f + st->guard;
    for (uint32_t m = 0; m < nh; m++) {
        const uint32_t gi = hb + m;
        if (flags[gi]) continue;  // the same value for every lane
        const PT p = pos[gi];
        bool hit = false;
        for (uint32_t kk = lane; kk < Tk && !hit; kk += 32) {
            if (gidx[kk] == gi) continue;
            const PT t = cand[kk];
            examined++;
            if constexpr (F32) {
                const float ex = __fsub_rn(p.x, t.x), ey = __fsub_rn(p.y, t.y);
                float d2 = __fmaf_rn(ey, ey, __fmul_rn(ex, ex));
                if (DIM == 3) {
                    const float ez = __fsub_rn(p.z, t.z);
                    d2 = __fmaf_rn(ez, ez, d2);
                }
                const float rs = __fadd_rn(p.w, t.w);
                hit = d2 <= __fmul_rn(__fmul_rn(rs, rs), g1);
            } else {
                const double q[3] = {p.x, p.y, p.z};
                hit = collide64<DIM>(st->images, q, p.w, t.x, t.y, t.z, t.w, st->L, st->halfL);
            }
        }
        if (__any_sync(0xffffffffu, hit) && lane == 0) hits++;
    }
}

// Cells of the RVEs at work (plan actc, 256-cell chunks), one warp per cell
// in a grid-stride loop.
template <bool F32>
__global__ void __launch_bounds__(CK_WARPS * 32) k_check_cells(BatchDev *bd)
{
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)wib * CheckSmem<F32>::bytes;
    const int B = bd->B;
    const int total = bd->actc[B] * 256;
    const int stride = gridDim.x * CK_WARPS;
    for (int gc = blockIdx.x * CK_WARPS + wib; gc < total; gc += stride) {
        const int chunk = gc >> 8;
        int r = 0;
        if (lane == 0) r = find_seg(bd->actc, B, chunk);
        r = __shfl_sync(0xffffffffu, r, 0);
        RveDev *st = bd->rv[r];
        const int cell = (chunk - bd->actc[r]) * 256 + (gc & 255);
        if (!st->do_check || cell >= st->ncells) continue;
        int hits = 0;
        unsigned examined = 0;
        if (st->dim == 3) check_cell<3, F32>(st, cell, base, hits, examined);
        else check_cell<2, F32>(st, cell, base, hits, examined);
        hits = __reduce_add_sync(0xffffffffu, hits);
        examined = __reduce_add_sync(0xffffffffu, examined);
        if (lane == 0) {
            if (hits) atomicAdd(&st->red[0], (unsigned long long)hits);
            if (examined) atomicAdd(&st->pairs_check, (unsigned long long)examined);
        }
    }
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
                        if (gap64<DIM>(st->images, q, p.w, tt, t.w, st->L, st->halfL, &gap)) cnt++;
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
                    if (gap64<DIM>(st->images, q, p.w, tt, t.w, st->L, st->halfL, &gap) && k < cnt) {
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

int check_cap_max(bool f32) { return f32 ? 512 : 256; }

static int g_ck_blocks[2] = {0, 0};

// Groups with dense stencils (whole-stencil estimate above 256 candidates, as
// the 1e6-sphere clustered RVE: 8% faster there) take the warp-per-cell
// check, a persistent grid of all the blocks that stay resident, at most one
// warp per cell; groups of small stencils (monodisperse RVEs, a cell or two
// of particles) keep one thread per particle, which measured faster there (a
// warp per cell of one or two particles leaves most lanes idle).
void launch_check(const BatchShape &b, cudaStream_t s)
{
    if (!b.check_cells) {
        if (b.f32) k_check<true><<<b.blocks_p, 256, 0, s>>>(b.d);
        else k_check<false><<<b.blocks_p, 256, 0, s>>>(b.d);
        return;
    }
    const int want = (b.blocks_c * 256 + CK_WARPS - 1) / CK_WARPS;
    const int res = g_ck_blocks[b.f32 ? 1 : 0];
    const int nb = want < res ? want : res;
    if (b.f32) k_check_cells<true><<<nb, CK_WARPS * 32, CK_WARPS * CheckSmem<true>::bytes, s>>>(b.d);
    else k_check_cells<false><<<nb, CK_WARPS * 32, CK_WARPS * CheckSmem<false>::bytes, s>>>(b.d);
}

void check_configure()
{
    if (g_ck_blocks[0]) return;
    int dev = 0, sms = 1, b32 = 0, b64 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_check_cells<true>, CK_WARPS * 32, CK_WARPS * CheckSmem<true>::bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_check_cells<false>, CK_WARPS * 32,
                                                  CK_WARPS * CheckSmem<false>::bytes);
    g_ck_blocks[1] = (b32 > 0 ? b32 : 1) * (sms > 0 ? sms : 1);
    g_ck_blocks[0] = (b64 > 0 ? b64 : 1) * (sms > 0 ? sms : 1);
}

// Binning of P into a scratch slot, in binary64, for the inspection of one
// RVE (its single-member batch).
void launch_inspect_bin(RveDev *d_st, const BatchShape &solo, cudaStream_t s)
{
    k_inspect_begin<<<1, 1, 0, s>>>(d_st);
    launch_plan(solo, s);
    launch_bin(solo, solo.f32, false, s);
}

void launch_pairs_count(RveDev *d_st, int dim, int64_t n, int want_gap, cudaStream_t s)
{
    const int nb = blocks_for(n, 256);
    if (dim == 2) k_pairs_count<2><<<nb, 256, 0, s>>>(d_st, want_gap);
    else k_pairs_count<3><<<nb, 256, 0, s>>>(d_st, want_gap);
}

void launch_pairs_fill(RveDev *d_st, int dim, int64_t n, long long *ij, cudaStream_t s)
{
    const int nb = blocks_for(n, 256);
    if (dim == 2) k_pairs_fill<2><<<nb, 256, 0, s>>>(d_st, ij);
    else k_pairs_fill<3><<<nb, 256, 0, s>>>(d_st, ij);
}

void launch_inspect_end(RveDev *d_st, cudaStream_t s) { k_inspect_end<<<1, 1, 0, s>>>(d_st); }

void launch_gather(RveDev *d_st, int dim, bool f32, int64_t n, double *xyz, double *rad, cudaStream_t s)
{
    const int nb = blocks_for(n, 256);
    if (dim == 2) {
        if (f32) k_gather<2, true><<<nb, 256, 0, s>>>(d_st, xyz, rad);
        else k_gather<2, false><<<nb, 256, 0, s>>>(d_st, xyz, rad);
    } else {
        if (f32) k_gather<3, true><<<nb, 256, 0, s>>>(d_st, xyz, rad);
        else k_gather<3, false><<<nb, 256, 0, s>>>(d_st, xyz, rad);
    }
}

}  // namespace srm
