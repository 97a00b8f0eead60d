// k_sweep.cu -- Algorithm 3 (random migration of every particle) as a
// coloured parallel sweep.
//
// Cells are coloured by (c_x mod 3, c_y mod 3[, c_z mod 3]); the sweep runs
// the 3^d colours in ascending order, one launch per colour.  Within a
// colour every cell is handled by one thread, which moves the particles of
// its cell one after the other in ascending id.  Two cells of one colour are
// at least three cells apart along some axis, while a particle reads only
// cells within H <= 2 of its home cell, so the cells of one colour never read
// each other's particles: the parallel sweep equals the serial sweep in
// colour -> cell -> id order, for any scheduling of the threads.
//
// A trial move (Algorithm 3 lines 4-10) is q = wrap(q_old + c_m u) with u
// the Philox-drawn direction; the collision test (Algorithm 5) scans the
// cells within H of the home cell, which contain every particle that can
// touch any trial position (cells are at least 2.5 R_max + c_m wide and the
// lists are at most one move stale).
#include "srm_dev.cuh"
#include "srm_launch.h"
#include "srm_stencil.cuh"

#include <type_traits>

namespace srm {

// ---------------------------------------------------------------------------
// Warp-per-cell sweep.  One warp owns one cell of the current colour:
//  1. the (2H+1)^d stencil cells around the home cell are listed (begin,
//     count, offset) and their particles staged in shared memory -- for the
//     FP32 form as positions relative to the home cell corner (the stencil
//     shift s*w is added once here), for the FP64 form as absolute binary64
//     positions;
//  2. the particles of the home cell are moved one after the other in
//     ascending id (Algorithm 3); lane l draws the direction of trial l in
//     parallel, and for each trial the 32 lanes test interleaved slices of
//     the staged candidates and vote with __any_sync (Algorithm 5);
//  3. an accepted move updates the staged copy (later particles of the cell
//     see it) and the slot in global memory.
// Candidate lists longer than the staging capacity are read from global
// memory instead (same arithmetic).
// ---------------------------------------------------------------------------
// ---- one kernel for both forms -----------------------------------------------
// Per-warp shared memory: stencil list | staged positions | (FP64 form: FP32
// copies relative to the home corner, for culling) | staged indices | near list.
constexpr int NEAR_CAP = 192;

template <bool F32>
struct SweepSmem {
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    static __host__ __device__ constexpr size_t bytes(int cap)
    {
        return (ST_HDR + (size_t)cap * sizeof(PT) + (F32 ? 0 : (size_t)cap * sizeof(float4)) +
                (size_t)cap * 4 + (size_t)NEAR_CAP * 2 + 31) / 32 * 32;
    }
};

// Cull test on FP32 positions relative to the home corner: t can touch a
// trial position of p (within c_m of p) only if |p - t| <= R_p + R_t + c_m;
// the relative slack 1e-4 covers the FP32 rounding of both positions, so the
// near list is a superset of every partner the exact test can find.
__device__ __forceinline__ bool near_f32(const float4 &p, const float4 &t, float cm, int dim)
{
    const float ex = p.x - t.x, ey = p.y - t.y, ez = dim == 3 ? p.z - t.z : 0.f;
    const float d2 = ex * ex + ey * ey + ez * ez;
    const float r = p.w + t.w + cm;
    return d2 <= r * r * 1.0002f;
}

template <int DIM, bool F32>
__global__ void __launch_bounds__(SW_WARPS * 32) k_sweep(RveDev *st, int chi, int cap)
{
    using PT = typename SweepSmem<F32>::PT;
    extern __shared__ __align__(32) unsigned char smem[];
    if (!st->active) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int t = blockIdx.x * SW_WARPS + wib;  // cell of this colour
    int moved = 0;
    unsigned long long examined = 0;
    if (t < st->nsub) {
        unsigned char *base = smem + (size_t)wib * SweepSmem<F32>::bytes(cap);
        StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
        PT *cpos = reinterpret_cast<PT *>(base + ST_HDR);
        float4 *capx = reinterpret_cast<float4 *>(cpos + cap);  // FP64 form only
        uint32_t *cidx = reinterpret_cast<uint32_t *>(F32 ? (void *)(cpos + cap) : (void *)(capx + cap));
        uint16_t *near = reinterpret_cast<uint16_t *>(cidx + cap);
        const int s0 = st->sub[0], s1 = st->sub[1];
        const int hx = 3 * (t % s0) + chi % 3;
        const int hy = 3 * ((t / s0) % s1) + (chi / 3) % 3;
        const int hz = DIM == 3 ? 3 * (t / (s0 * s1)) + chi / 9 : 0;
        const uint32_t *cs = st->cell_start;
        const int cell = hx + st->gn[0] * (hy + st->gn[1] * hz);
        const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
        if (nh > 0) {
            const Slot d = st->slot[st->dst_idx];
            PT *pos = reinterpret_cast<PT *>(d.pos);
            int nst, center;
            const uint32_t T = list_stencil(st, cs, hx, hy, hz, S, nst, center);
            const float w0 = (float)st->gw[0], w1 = (float)st->gw[1], w2 = (float)st->gw[2];
            // home corner (FP64 form: absolute; used for the FP32 culling copies)
            const double ox = hx * st->gw[0], oy = hy * st->gw[1], oz = hz * st->gw[2];
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
            // FP32 copy relative to the home corner (FP64 form), via the minimum image
            auto approx = [&](const double4_32a &c) -> float4 {
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
            };
            if (staged) {
                for (uint32_t k = lane; k < T; k += 32) {
                    uint32_t g;
                    const PT c = fetch(k, g);
                    cpos[k] = c;
                    if constexpr (!F32) capx[k] = approx(c);
                    cidx[k] = g;
                }
                __syncwarp();
            }
            const uint64_t seed = st->seed, sweep = st->sweep;
            const double c_m = st->c_m;
            const float cmf = (float)c_m;
            const float g1 = 1.0f + st->guard;
            const int N_l = st->N_l;
            const uint32_t ko = S.o[center];
            for (uint32_t m = 0; m < nh; m++) {
                const uint32_t gi = hb + m;
                const uint32_t kself = ko + m;
                const PT p = staged ? cpos[kself] : pos[gi];
                const uint64_t pid = d.pid[gi];
                // ---- near list of this particle (staged case)
                uint32_t nn = 0;
                bool use_near = false;
                if (staged) {
                    float4 pa;
                    if constexpr (F32) pa = p;
                    else pa = capx[kself];
                    for (uint32_t k0 = 0; k0 < T; k0 += 32) {
                        const uint32_t k = k0 + lane;
                        bool nb = false;
                        if (k < T && k != kself) {
                            float4 ca;
                            if constexpr (F32) ca = cpos[k];
                            else ca = capx[k];
                            nb = near_f32(pa, ca, cmf, DIM);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, nb);
                        const uint32_t at = nn + __popc(bal & ((1u << lane) - 1u));
                        if (nb && at < NEAR_CAP) near[at] = (uint16_t)k;
                        nn += __popc(bal);
                    }
                    use_near = nn <= NEAR_CAP;
                    __syncwarp();
                }
                const uint32_t L = use_near ? nn : T;
                bool done = false;
                // trials are drawn in batches, one per lane: 2 first (most
                // particles take the first trial), then 8 at a time
                for (int l0 = 0; l0 < N_l && !done;) {
                    const int bsz = l0 == 0 ? 2 : 8;
                    const int lmax = N_l - l0 < bsz ? N_l - l0 : bsz;
                    double qt[3] = {0.0, 0.0, 0.0};
                    float qs[3] = {0.f, 0.f, 0.f};
                    if constexpr (F32) {
                        qs[0] = p.x;
                        qs[1] = p.y;
                        qs[2] = p.z;
                    } else {
                        qt[0] = p.x;
                        qt[1] = p.y;
                        qt[2] = p.z;
                    }
                    if (lane < lmax) {
                        if constexpr (F32) {
                            float u[3];
                            unit_dir_f32<DIM>(seed, sweep, pid, (uint64_t)(l0 + lane), u);
                            qs[0] = p.x + cmf * u[0];
                            qs[1] = p.y + cmf * u[1];
                            if (DIM == 3) qs[2] = p.z + cmf * u[2];
                        } else {
                            double u[3];
                            unit_dir<DIM>(seed, sweep, pid, (uint64_t)(l0 + lane), u);
                            qt[0] = wrap_d(__dadd_rn((double)p.x, __dmul_rn(c_m, u[0])), st->L[0]);
                            qt[1] = wrap_d(__dadd_rn((double)p.y, __dmul_rn(c_m, u[1])), st->L[1]);
                            if (DIM == 3) qt[2] = wrap_d(__dadd_rn((double)p.z, __dmul_rn(c_m, u[2])), st->L[2]);
                        }
                    }
                    l0 += lmax;
                    for (int l = 0; l < lmax; l++) {
                        double q[3] = {0.0, 0.0, 0.0};
                        float qf[3] = {0.f, 0.f, 0.f};
                        if constexpr (F32) {
                            qf[0] = __shfl_sync(0xffffffffu, qs[0], l);
                            qf[1] = __shfl_sync(0xffffffffu, qs[1], l);
                            qf[2] = __shfl_sync(0xffffffffu, qs[2], l);
                        } else {
                            q[0] = __shfl_sync(0xffffffffu, qt[0], l);
                            q[1] = __shfl_sync(0xffffffffu, qt[1], l);
                            q[2] = __shfl_sync(0xffffffffu, qt[2], l);
                        }
                        bool hit = false;
                        for (uint32_t kk = lane; kk < L && !hit; kk += 32) {
                            PT c;
                            uint32_t g;
                            if (use_near) {
                                const uint32_t k = near[kk];
                                c = cpos[k];
                                g = gi + 1;  // never self: the near list excludes it
                            } else if (staged) {
                                c = cpos[kk];
                                g = cidx[kk];
                            } else {
                                c = fetch(kk, g);
                            }
                            if (g == gi) continue;
                            examined++;
                            if constexpr (F32) {
                                const float ex = qf[0] - c.x, ey = qf[1] - c.y;
                                float d2 = ex * ex + ey * ey;
                                if (DIM == 3) {
                                    const float ez = qf[2] - c.z;
                                    d2 += ez * ez;
                                }
                                const float rs = p.w + c.w;
                                hit = d2 <= rs * rs * g1;
                            } else {
                                hit = collide_exact<DIM>(q, (double)p.w, c.x, c.y, c.z, c.w, st->L, st->halfL);
                            }
                        }
                        if (!__any_sync(0xffffffffu, hit)) {
                            if (lane == 0) {
                                PT np;
                                if constexpr (F32) {
                                    np = make_float4(qf[0], qf[1], DIM == 3 ? qf[2] : p.z, p.w);
                                } else {
                                    np = make_double4_32a(q[0], q[1], DIM == 3 ? q[2] : p.z, p.w);
                                }
                                if (staged) {
                                    cpos[kself] = np;
                                    if constexpr (!F32) capx[kself] = approx(np);
                                }
                                pos[gi] = np;
                            }
                            moved++;
                            done = true;
                            __syncwarp();
                            break;
                        }
                    }
                }
            }
        }
    }
    if (lane == 0 && moved) atomicAdd(&st->red[3], (unsigned long long)moved);
    examined = __reduce_add_sync(0xffffffffu, (unsigned)examined);
    if (lane == 0 && examined) atomicAdd(&st->pairs_sweep, examined);
}

int sweep_cap_max(bool f32) { return f32 ? 1024 : 512; }

static size_t sweep_smem(bool f32, int cap)
{
    return SW_WARPS * (f32 ? SweepSmem<true>::bytes(cap) : SweepSmem<false>::bytes(cap));
}

void launch_sweep_colour(RveDev *d_st, const HostShape &sh, int chi, cudaStream_t s)
{
    const int nb = (int)((sh.nsub_cap + SW_WARPS - 1) / SW_WARPS);
    const int cap = sh.cap_sweep;
    const size_t smem = sweep_smem(sh.f32, cap);
    if (sh.f32) {
        if (sh.dim == 2) k_sweep<2, true><<<nb, SW_WARPS * 32, smem, s>>>(d_st, chi, cap);
        else k_sweep<3, true><<<nb, SW_WARPS * 32, smem, s>>>(d_st, chi, cap);
    } else {
        if (sh.dim == 2) k_sweep<2, false><<<nb, SW_WARPS * 32, smem, s>>>(d_st, chi, cap);
        else k_sweep<3, false><<<nb, SW_WARPS * 32, smem, s>>>(d_st, chi, cap);
    }
}

void launch_sweep(RveDev *d_st, const HostShape &sh, cudaStream_t s)
{
    const int ncol = sh.dim == 3 ? 27 : 9;
    for (int chi = 0; chi < ncol; chi++) launch_sweep_colour(d_st, sh, chi, s);
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel.
void sweep_configure()
{
    const int s32 = (int)sweep_smem(true, sweep_cap_max(true));
    const int s64 = (int)sweep_smem(false, sweep_cap_max(false));
    cudaFuncSetAttribute(k_sweep<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_sweep<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_sweep<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(k_sweep<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
}

}  // namespace srm
