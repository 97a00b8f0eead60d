// k_sweep.cu -- Algorithm 3 (random migration of every particle) as a
// coloured parallel sweep.
//
// Cells are coloured by (c_x mod 3, c_y mod 3[, c_z mod 3]); the sweep runs
// the 3^d colours in ascending order, one launch per colour.  Within a
// colour every cell is handled by one warp, which moves the particles of its
// cell one after the other in ascending id.  Two cells of one colour are at
// least three cells apart along some axis, while a particle reads only cells
// within H <= 2 of its home cell, so the cells of one colour never read each
// other's particles: the parallel sweep equals the serial sweep in
// colour -> cell -> id order, whatever the scheduling.
//
// A trial move (Algorithm 3) is q = wrap(q_old + c_m u) with u the
// Philox-drawn direction; the collision test (Algorithm 5) covers the cells
// within H of the home cell, which contain every particle that can touch any
// trial position (cells are at least 2.5 R_max + c_m wide and the lists are
// at most one move stale).
//
// Per cell, one warp:
//  1. lists the stencil cells (home cell first) and stages in shared memory
//     the candidates that can reach the home cell: distance to the home
//     cell box <= R_home,max + R_t + 2 c_m (a conservative bound: trials stay
//     within c_m of positions that stay within c_m of the box).  FP32 form:
//     positions relative to the home cell corner; FP64 form: absolute
//     binary64 positions plus binary32 copies relative to the corner;
//  2. for each particle of the cell, in ascending id: builds its near list,
//     the candidates within R_i + R_t + c_m of it (superset of everything a
//     trial can touch), as copies in shared memory; lane l draws trial l of a
//     batch; for each trial the lanes test the near list and vote;
//  3. an accepted move updates the staged copy (later particles of the cell
//     see it) and the slot in global memory, and marks the particle moved.
// If the culled candidates exceed the staging capacity, the near lists are
// built straight from global memory (same arithmetic, slower).
#include "srm_dev.cuh"
#include "srm_launch.h"
#include "srm_stencil.cuh"

#include <type_traits>

namespace srm {

constexpr int NEAR_CAP = 128;
constexpr int PRE_NH = 64;    // home particles whose first trials are drawn up front
constexpr int PRE_TRIALS = 2; // trials drawn up front per particle

template <bool F32>
struct SweepSmem {
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    using DT = typename std::conditional<F32, float, double>::type;
    static __host__ __device__ constexpr size_t bytes(int cap)
    {
        return (ST_HDR + (size_t)cap * sizeof(PT) + (F32 ? 0 : (size_t)cap * sizeof(float4)) +
                (size_t)NEAR_CAP * sizeof(PT) + (size_t)PRE_NH * PRE_TRIALS * 3 * sizeof(DT) + 31) /
               32 * 32;
    }
};

// |p - t|^2 against r^2 with relative slack 4e-4 (covers the binary32
// rounding of relative positions of magnitude up to a few cells).
__device__ __forceinline__ bool within_f32(const float4 &p, const float4 &t, float r, int dim)
{
    const float ex = p.x - t.x, ey = p.y - t.y, ez = dim == 3 ? p.z - t.z : 0.f;
    return ex * ex + ey * ey + ez * ez <= r * r * 1.0004f;
}

// Squared distance from a point (relative to the home corner) to the home box.
__device__ __forceinline__ float box_dist2(const float4 &t, const float w[3], int dim)
{
    const float ex = fmaxf(fmaxf(-t.x, t.x - w[0]), 0.f);
    const float ey = fmaxf(fmaxf(-t.y, t.y - w[1]), 0.f);
    const float ez = dim == 3 ? fmaxf(fmaxf(-t.z, t.z - w[2]), 0.f) : 0.f;
    return ex * ex + ey * ey + ez * ez;
}

// One-launch sweep: before a cell of colour chi is staged, every non-empty
// cell within reach (home +-H) whose colour is lower must have finished this
// sweep -- exactly the cells of lower colour whose moves the serial order
// lets it see; cells of higher colour wait for this one in turn, so they are
// still unmoved.  Cells are handed out in colour order, so every cell waited
// for is already held by a running warp.  A wait gives up after wait_limit
// polls and sets the RVE's status (the host reports SRM_E_DEVICE_TIMEOUT).
template <int DIM>
__device__ __forceinline__ void wait_lower_colours(RveDev *st, const uint32_t *cs, int hx, int hy, int hz, int chi,
                                                   uint32_t epoch)
{
    const int lane = threadIdx.x & 31;
    const int H0 = st->H[0], H1 = st->H[1], H2 = st->H[2];
    const int w0 = 2 * H0 + 1, w1 = 2 * H1 + 1, w2 = 2 * H2 + 1;
    const int nst = w0 * w1 * w2;
    const int n0 = st->gn[0], n1 = st->gn[1], n2 = st->gn[2];
    const int limit = st->wait_limit;
    for (int j = lane; j < nst; j += 32) {
        const int dx = j % w0 - H0, dy = (j / w0) % w1 - H1, dz = j / (w0 * w1) - H2;
        int cx = hx + dx, cy = hy + dy, cz = hz + dz;
        cx = cx < 0 ? cx + n0 : (cx >= n0 ? cx - n0 : cx);
        cy = cy < 0 ? cy + n1 : (cy >= n1 ? cy - n1 : cy);
        cz = cz < 0 ? cz + n2 : (cz >= n2 ? cz - n2 : cz);
        const int col = cx % 3 + 3 * (cy % 3) + (DIM == 3 ? 9 * (cz % 3) : 0);
        if (col >= chi) continue;
        const int c = cx + n0 * (cy + n1 * cz);
        if (cs[c + 1] == cs[c]) continue;
        if (limit < 0) {
            atomicExch(&st->status, STATUS_WAIT_TIMEOUT);
            continue;
        }
        for (int it = 0; ld_acquire(&st->done[c]) != epoch; it++) {
            if (it >= limit) {
                atomicExch(&st->status, STATUS_WAIT_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
    }
    __syncwarp();
    __threadfence();
}

// One cell of colour chi (work item t of its RVE), processed by one warp.
template <int DIM, bool F32>
__device__ __forceinline__ void sweep_cell(RveDev *st, int chi, int t, unsigned char *base, int cap,
                                           int &moved, unsigned &examined, bool dataflow)
{
    using PT = typename SweepSmem<F32>::PT;
    using DT = typename SweepSmem<F32>::DT;
    const int lane = threadIdx.x & 31;
    StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
    PT *cpos = reinterpret_cast<PT *>(base + ST_HDR);
    float4 *capx = reinterpret_cast<float4 *>(cpos + cap);  // FP64 form only
    PT *nbuf = reinterpret_cast<PT *>(F32 ? (void *)(cpos + cap) : (void *)(capx + cap));
    DT *pre = reinterpret_cast<DT *>(nbuf + NEAR_CAP);      // [PRE_NH][PRE_TRIALS][3]

    const Slot d = st->slot[st->dst_idx];
    PT *pos = reinterpret_cast<PT *>(d.pos);
    const uint32_t *cs = st->cell_start;
    const int s0 = st->sub[0], s1 = st->sub[1];
    const float w[3] = {(float)st->gw[0], (float)st->gw[1], (float)st->gw[2]};
    const uint64_t seed = st->seed, sweep = st->sweep;
    const double c_m = st->c_m;
    const float cmf = (float)c_m;
    const float g1 = 1.0f + st->guard;
    const int N_l = st->N_l;
    {
        const int hx = 3 * (t % s0) + chi % 3;
        const int hy = 3 * ((t / s0) % s1) + (chi / 3) % 3;
        const int hz = DIM == 3 ? 3 * (t / (s0 * s1)) + chi / 9 : 0;
        const int cell = hx + st->gn[0] * (hy + st->gn[1] * hz);
        const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
        if (nh == 0) return;  // nothing moves: nobody waits for an empty cell
        const uint32_t epoch = (uint32_t)(st->sweep + 1);
        if (dataflow) wait_lower_colours<DIM>(st, cs, hx, hy, hz, chi, epoch);
        int nst, center;
        const uint32_t T = list_stencil(st, cs, hx, hy, hz, S, nst, center);
        // home corner (FP64 form: the binary32 copies are relative to it)
        const double ox = hx * st->gw[0], oy = hy * st->gw[1], oz = hz * st->gw[2];
        auto fetch = [&](uint32_t k, uint32_t &g) -> PT {
            const int j = find_cell(S, nst, k);
            g = S.b[j] + (k - S.o[j]);
            PT c = pos[g];
            if constexpr (F32) {
                c.x += (float)S.sh[j][0] * w[0];
                c.y += (float)S.sh[j][1] * w[1];
                c.z += (float)S.sh[j][2] * w[2];
            }
            return c;
        };
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
        // largest radius among the particles of the home cell
        float rh = 0.f;
        for (uint32_t m = lane; m < nh; m += 32) rh = fmaxf(rh, (float)pos[hb + m].w);
        for (int o = 16; o > 0; o >>= 1) rh = fmaxf(rh, __shfl_xor_sync(0xffffffffu, rh, o));
        // 1. stage the candidates that can reach the home cell (home first)
        // Staging stops at the first 32-candidate chunk that would overflow
        // the capacity; candidates from kstop on are read from global memory
        // (culled the same way) when the near lists are built.
        uint32_t Tk = 0, kstop = T;
        for (uint32_t k0 = 0; k0 < T; k0 += 32) {
            const uint32_t k = k0 + lane;
            bool keep = false;
            PT c;
            float4 ca;
            if (k < T) {
                uint32_t g;
                c = fetch(k, g);
                ca = approx(c);
                const float r = rh + ca.w + 2.f * cmf;
                keep = k < nh || box_dist2(ca, w, DIM) <= r * r * 1.0004f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (Tk + __popc(bal) > (uint32_t)cap) {
                kstop = k0;
                break;
            }
            const uint32_t at = Tk + __popc(bal & ((1u << lane) - 1u));
            if (keep) {
                cpos[at] = c;
                if constexpr (!F32) capx[at] = ca;
            }
            Tk += __popc(bal);
        }
        const bool staged = kstop == T;
        if (!staged && lane == 0) atomicAdd(&st->stage_overflow, 1ull);
        // the first trial directions of every home particle, drawn in
        // parallel (they depend on the particle id and the counters only)
        const uint32_t npre = nh < (uint32_t)PRE_NH ? nh : (uint32_t)PRE_NH;
        for (uint32_t e = lane; e < npre * PRE_TRIALS; e += 32) {
            const uint32_t m = e / PRE_TRIALS, l = e % PRE_TRIALS;
            const uint64_t pid = d.pid[hb + m];
            DT *u = pre + 3 * e;
            if constexpr (F32) {
                float v[3];
                unit_dir_f32<DIM>(seed, sweep, pid, l, v);
                u[0] = v[0];
                u[1] = v[1];
                u[2] = v[2];
            } else {
                double v[3];
                unit_dir<DIM>(seed, sweep, pid, l, v);
                u[0] = v[0];
                u[1] = v[1];
                u[2] = v[2];
            }
        }
        __syncwarp();

        // 2. the particles of the home cell, ascending id
        for (uint32_t m = 0; m < nh; m++) {
            const uint32_t gi = hb + m;
            // home particles lead the candidate list and are always kept, so
            // the first ones are staged at their own index
            const PT p = m < Tk ? cpos[m] : pos[gi];
            const float4 pa = approx(p);
            const uint64_t pid = d.pid[gi];
            // near list: copies of every candidate within R_i + R_t + c_m
            // (staged candidates, then the unstaged remainder from global)
            uint32_t nn = 0;
            const uint32_t scan = Tk + (T - kstop);
            for (uint32_t k0 = 0; k0 < scan; k0 += 32) {
                const uint32_t k = k0 + lane;
                bool nb = false;
                PT c;
                if (k < scan) {
                    float4 ca;
                    bool self;
                    if (k < Tk) {
                        self = k == m;
                        c = cpos[k];
                        if constexpr (F32) ca = c;
                        else ca = capx[k];
                    } else {
                        uint32_t g;
                        c = fetch(kstop + (k - Tk), g);
                        self = g == gi;
                        ca = approx(c);
                    }
                    nb = !self && within_f32(pa, ca, pa.w + ca.w + cmf, DIM);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, nb);
                const uint32_t at = nn + __popc(bal & ((1u << lane) - 1u));
                if (nb && at < NEAR_CAP) nbuf[at] = c;
                nn += __popc(bal);
            }
            __syncwarp();
            const bool use_near = nn <= NEAR_CAP;
            bool done = false;
            // trials in batches, one per lane: 2 first (most particles take
            // the first trial), then 8 at a time
            for (int l0 = 0; l0 < N_l && !done;) {
                const int bsz = (l0 == 0 && m < (uint32_t)PRE_NH) ? PRE_TRIALS : 8;
                const int lmax = N_l - l0 < bsz ? N_l - l0 : bsz;
                double qt[3] = {0.0, 0.0, 0.0};
                float qs[3] = {0.f, 0.f, 0.f};
                if (l0 == 0 && m < (uint32_t)PRE_NH) {
                    // first trials: drawn up front for the whole cell
                    if (lane < lmax) {
                        const DT *up = pre + 3 * (m * PRE_TRIALS + lane);
                        if constexpr (F32) {
                            qs[0] = p.x + cmf * up[0];
                            qs[1] = p.y + cmf * up[1];
                            qs[2] = DIM == 3 ? p.z + cmf * up[2] : p.z;
                        } else {
                            qt[0] = wrap_d(__dadd_rn(p.x, __dmul_rn(c_m, up[0])), st->L[0]);
                            qt[1] = wrap_d(__dadd_rn(p.y, __dmul_rn(c_m, up[1])), st->L[1]);
                            qt[2] = DIM == 3 ? wrap_d(__dadd_rn(p.z, __dmul_rn(c_m, up[2])), st->L[2]) : p.z;
                        }
                    }
                } else {
                    // later trials: eight at a time, candidates drawn by all lanes
                    DT u[3];
                    draw8<DIM, F32>(seed, sweep, pid, l0, u);
                    if (lane < lmax) {
                        if constexpr (F32) {
                            qs[0] = p.x + cmf * u[0];
                            qs[1] = p.y + cmf * u[1];
                            qs[2] = DIM == 3 ? p.z + cmf * u[2] : p.z;
                        } else {
                            qt[0] = wrap_d(__dadd_rn(p.x, __dmul_rn(c_m, u[0])), st->L[0]);
                            qt[1] = wrap_d(__dadd_rn(p.y, __dmul_rn(c_m, u[1])), st->L[1]);
                            qt[2] = DIM == 3 ? wrap_d(__dadd_rn(p.z, __dmul_rn(c_m, u[2])), st->L[2]) : p.z;
                        }
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
                    const uint32_t L = use_near ? nn : scan;
                    for (uint32_t kk = lane; kk < L && !hit; kk += 32) {
                        PT c;
                        if (use_near) {
                            c = nbuf[kk];
                        } else if (kk < Tk) {
                            if (kk == m) continue;
                            c = cpos[kk];
                        } else {
                            uint32_t g;
                            c = fetch(kstop + (kk - Tk), g);
                            if (g == gi) continue;
                        }
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
                            hit = collide_exact<DIM>(q, p.w, c.x, c.y, c.z, c.w, st->L, st->halfL);
                        }
                    }
                    if (!__any_sync(0xffffffffu, hit)) {
                        if (lane == 0) {
                            PT np;
                            if constexpr (F32) np = make_float4(qf[0], qf[1], qf[2], p.w);
                            else np = make_double4_32a(q[0], q[1], q[2], p.w);
                            if (m < Tk) {
                                cpos[m] = np;
                                if constexpr (!F32) capx[m] = approx(np);
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
            if (lane == 0) st->flags[gi] = done ? 1 : 0;
            __syncwarp();
        }
        if (dataflow && lane == 0) {
            __threadfence();
            st_release(&st->done[cell], epoch);
        }
        __syncwarp();
    }
}

// One launch per colour over all RVEs of the batch: each warp takes the next
// (RVE, cell) work item from the colour's counter.  2D RVEs have 9 colours.
// Blocks per SM the register allocation must allow (a build-time knob).
#ifndef SRM_SWEEP_MIN_BLOCKS
#define SRM_SWEEP_MIN_BLOCKS 1
#endif

template <bool F32>
__global__ void __launch_bounds__(SW_WARPS * 32, SRM_SWEEP_MIN_BLOCKS) k_sweep(BatchDev *bd, int chi, int cap)
{
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)wib * SweepSmem<F32>::bytes(cap);
    const int B = bd->B;
    const int32_t *off = chi < 9 ? bd->act : bd->act3;  // RVEs at work with this colour
    const int total = off[B];
    for (;;) {
        int tg = 0, r = 0;
        if (lane == 0) {
            tg = (int)atomicAdd(&bd->wq[chi], 1u);
            if (tg < total) r = find_seg(off, B, tg);
        }
        tg = __shfl_sync(0xffffffffu, tg, 0);
        if (tg >= total) break;
        r = __shfl_sync(0xffffffffu, r, 0);
        RveDev *st = bd->rv[r];
        const int t = tg - off[r];
        if (!st->active || t >= st->nsub) continue;
        int moved = 0;
        unsigned examined = 0;
        if (st->dim == 3) {
            sweep_cell<3, F32>(st, chi, t, base, cap, moved, examined, false);
        } else {
            if (chi >= 9) continue;
            sweep_cell<2, F32>(st, chi, t, base, cap, moved, examined, false);
        }
        examined = __reduce_add_sync(0xffffffffu, examined);
        if (lane == 0) {
            if (moved) atomicAdd(&st->red[3], (unsigned long long)moved);
            if (examined) atomicAdd(&st->pairs_sweep, (unsigned long long)examined);
        }
    }
}

// All colours in one launch: work items are handed out in colour order from
// one counter; each cell waits for its lower-colour neighbours
// (wait_lower_colours) and stamps itself when done.
template <bool F32>
__global__ void __launch_bounds__(SW_WARPS * 32, SRM_SWEEP_MIN_BLOCKS) k_sweep_df(BatchDev *bd, int cap)
{
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)wib * SweepSmem<F32>::bytes(cap);
    const int B = bd->B;
    const int total = bd->coff[27];
    for (;;) {
        int tg = 0, chi = 0, r = 0, t = 0;
        if (lane == 0) {
            tg = (int)atomicAdd(&bd->wq[0], 1u);
            if (tg < total) {
                chi = find_seg(bd->coff, 27, tg);
                const int local = tg - bd->coff[chi];
                const int32_t *off = chi < 9 ? bd->act : bd->act3;
                r = find_seg(off, B, local);
                t = local - off[r];
            }
        }
        tg = __shfl_sync(0xffffffffu, tg, 0);
        if (tg >= total) break;
        chi = __shfl_sync(0xffffffffu, chi, 0);
        r = __shfl_sync(0xffffffffu, r, 0);
        t = __shfl_sync(0xffffffffu, t, 0);
        RveDev *st = bd->rv[r];
        if (!st->active || t >= st->nsub) continue;
        int moved = 0;
        unsigned examined = 0;
        if (st->dim == 3) sweep_cell<3, F32>(st, chi, t, base, cap, moved, examined, true);
        else sweep_cell<2, F32>(st, chi, t, base, cap, moved, examined, true);
        examined = __reduce_add_sync(0xffffffffu, examined);
        if (lane == 0) {
            if (moved) atomicAdd(&st->red[3], (unsigned long long)moved);
            if (examined) atomicAdd(&st->pairs_sweep, (unsigned long long)examined);
        }
    }
}

int sweep_cap_max(bool f32) { return f32 ? 512 : 256; }

static size_t sweep_smem(bool f32, int cap)
{
    return SW_WARPS * (f32 ? SweepSmem<true>::bytes(cap) : SweepSmem<false>::bytes(cap));
}

static int g_sms = 0;

// Blocks that stay resident on one SM at this shared memory size; a launch
// uses at most that many per SM and the warps pull work items.
template <typename K>
static int resident_blocks(K kern, size_t smem)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SW_WARPS * 32, smem);
    return nb > 0 ? nb : 1;
}

void launch_sweep_colour(const BatchShape &b, int chi, cudaStream_t s)
{
    const int cap = b.cap;
    const size_t smem = sweep_smem(b.f32, cap);
    const int64_t want64 = (b.sub_total + SW_WARPS - 1) / SW_WARPS;
    const int want = (int)(want64 > 0x7fffffff ? 0x7fffffff : want64);
    auto shape = [&](auto kern) {
        const int res = resident_blocks(kern, smem) * (g_sms > 0 ? g_sms : 1);
        return want < res ? want : res;
    };
    if (b.f32) k_sweep<true><<<shape(k_sweep<true>), SW_WARPS * 32, smem, s>>>(b.d, chi, cap);
    else k_sweep<false><<<shape(k_sweep<false>), SW_WARPS * 32, smem, s>>>(b.d, chi, cap);
}

void launch_sweep(const BatchShape &b, cudaStream_t s)
{
    const int cap = b.cap;
    const size_t smem = sweep_smem(b.f32, cap);
    const int64_t want64 = (b.sub_total * (b.has3d ? 27 : 9) + SW_WARPS - 1) / SW_WARPS;
    const int want = (int)(want64 > 0x7fffffff ? 0x7fffffff : want64);
    auto shape = [&](auto kern) {
        const int res = resident_blocks(kern, smem) * (g_sms > 0 ? g_sms : 1);
        return want < res ? want : res;
    };
    if (b.f32) k_sweep_df<true><<<shape(k_sweep_df<true>), SW_WARPS * 32, smem, s>>>(b.d, cap);
    else k_sweep_df<false><<<shape(k_sweep_df<false>), SW_WARPS * 32, smem, s>>>(b.d, cap);
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel.
void sweep_configure()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep_smem(true, sweep_cap_max(true)));
    cudaFuncSetAttribute(k_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep_smem(false, sweep_cap_max(false)));
    cudaFuncSetAttribute(k_sweep_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep_smem(true, sweep_cap_max(true)));
    cudaFuncSetAttribute(k_sweep_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep_smem(false, sweep_cap_max(false)));
}

}  // namespace srm
