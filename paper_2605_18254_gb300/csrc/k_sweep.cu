// k_sweep.cu -- Algorithm 3 (random migration of every particle) as one
// parallel sweep in the canonical colour order.
//
// Cells are coloured by (c_x mod 3, c_y mod 3[, c_z mod 3]); the canonical
// order visits the colours in ascending order, the cells of one colour in
// any order and the particles of a cell in ascending id.  Two cells of one
// colour are at least three cells apart along some axis, while a particle
// reads only cells within H <= 2 of its home cell, so the cells of one colour
// never read each other's particles.  The sweep of a group of RVEs is one
// launch per dimension: warps take (RVE, cell) work items from one counter,
// colour by colour, and a cell starts once every non-empty cell of lower
// colour within its reach has finished (per-cell epoch stamps).  The result
// equals the serial sweep in colour -> cell -> id order, whatever the
// scheduling.
//
// A trial move (Algorithm 3) is q = wrap(q_old + c_m u) with u the
// Philox-drawn direction; the collision test (Algorithm 5) covers the cells
// within H of the home cell, which contain every particle that can touch any
// trial position (cells are at least 2.5 R_max + c_m wide and the lists are
// at most one move stale).  The directions of trials 0 and 1 depend on the
// particle id and the counters only; k_draw draws them for every particle
// before the sweep, so that the sweep itself draws only the later trials of
// the few particles whose first two trials collide.
//
// Per cell, one warp (the general path; the staged path is described at
// sweep_cell_staged):
//  0. before waiting for the lower-colour neighbours, lists the stencil cells
//     (home cell first) and prefetches every candidate's line into L2;
//  1. stages in shared memory the candidates that can reach the home cell:
//     distance to the home cell box <= R_home,max + R_t + 2 c_m (a
//     conservative bound: trials stay within c_m of positions that stay
//     within c_m of the box).  FP32 form: positions relative to the home
//     cell corner, four 32-candidate chunks in flight (cp.async ring); FP64
//     form: absolute binary64 positions plus binary32 copies relative to the
//     corner, the next chunk's loads in flight while a chunk is culled;
//  2. for each particle of the cell, in ascending id: builds its near list,
//     the candidates within R_i + R_t + c_m of it (superset of everything a
//     trial can touch), as copies in shared memory; the two pre-drawn trials,
//     then batches of eight trials drawn by the lanes, are tested against
//     the near list and the first clean one is taken;
//  3. an accepted move updates the staged copy (later particles of the cell
//     see it) and the slot in global memory, and marks the particle moved.
// If the culled candidates exceed the staging capacity, the near lists are
// built straight from global memory (same arithmetic, slower).
#include "srm_dev.cuh"
#include "srm_launch.h"
#include "srm_stencil.cuh"

#include <type_traits>

namespace srm {

constexpr int NEAR_CAP = 64;
constexpr int PRE_NH = 32;    // home particles whose first trials are copied up front
constexpr int PRE_TRIALS = 2; // trials drawn ahead of the sweep per particle
constexpr int RING = 4;       // general path (FP32 form): 32-candidate chunks staged in flight
constexpr int NL_CAP = 256;   // staged path: entries of a particle's near index list

template <bool F32>
struct SweepSmem {
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    using DT = typename std::conditional<F32, float, double>::type;
    // general path: stencil, culled candidates (FP64 form: plus binary32
    // copies), near list, pre-drawn directions (FP32 form: plus the ring of
    // chunks in flight and their stencil cells)
    static __host__ __device__ constexpr size_t bytes_general(int cap)
    {
        return (ST_HDR + (size_t)cap * sizeof(PT) + (F32 ? 0 : (size_t)cap * sizeof(float4)) +
                (size_t)NEAR_CAP * sizeof(PT) + (size_t)PRE_NH * PRE_TRIALS * sizeof(PT) +
                (F32 ? (size_t)RING * 32 * (sizeof(PT) + 1) : 0) + 31) /
               32 * 32;
    }
    // staged path (FP32 form): stencil, every candidate, near bits (one word
    // per 32-candidate chunk and home particle of a group), stencil cell of
    // each candidate, a particle's near index list, the pre-tests of trials
    // 0 and 1 of a group's particles, pre-drawn directions
    static __host__ __device__ constexpr size_t off_bits(int cap) { return ST_HDR + (size_t)cap * sizeof(PT); }
    static __host__ __device__ constexpr size_t off_cid(int cap) { return off_bits(cap) + (size_t)cap * 4; }
    static __host__ __device__ constexpr size_t off_nl(int cap) { return (off_cid(cap) + (size_t)cap + 15) / 16 * 16; }
    static __host__ __device__ constexpr size_t off_shit(int cap) { return off_nl(cap) + NL_CAP * sizeof(uint16_t); }
    static __host__ __device__ constexpr size_t off_pre(int cap) { return (off_shit(cap) + 32 + 31) / 32 * 32; }
    static __host__ __device__ constexpr size_t bytes_staged(int cap)
    {
        return (off_pre(cap) + (size_t)PRE_NH * PRE_TRIALS * sizeof(PT) + 31) / 32 * 32;
    }
    static __host__ __device__ constexpr size_t bytes(int cap)
    {
        return bytes_general(cap) > bytes_staged(cap) ? bytes_general(cap) : bytes_staged(cap);
    }
};

// |p - t|^2 against r^2 with relative slack 4e-4 (covers the binary32
// rounding of relative positions of magnitude up to a few cells).
__device__ __forceinline__ bool within_f32(const float4 &p, const float4 &t, float r, int dim)
{
    const float ex = p.x - t.x, ey = p.y - t.y, ez = dim == 3 ? p.z - t.z : 0.f;
    return ex * ex + ey * ey + ez * ez <= r * r * 1.0004f;
}

// FP32 form of Algorithm 5 for one pair: trial q of a particle of radius Rq
// against candidate c (both relative to the same corner), with the guard g1.
// Explicit roundings (no contraction left to the compiler), so that the
// decision is the same wherever the test is inlined.
template <int DIM>
__device__ __forceinline__ bool hit_f32(const float q[3], float Rq, const float4 &c, float g1)
{
    const float ex = __fsub_rn(q[0], c.x), ey = __fsub_rn(q[1], c.y);
    float d2 = __fmaf_rn(ey, ey, __fmul_rn(ex, ex));
    if (DIM == 3) {
        const float ez = __fsub_rn(q[2], c.z);
        d2 = __fmaf_rn(ez, ez, d2);
    }
    const float rs = __fadd_rn(Rq, c.w);
    return d2 <= __fmul_rn(__fmul_rn(rs, rs), g1);
}

// Trial position of the FP32 form: p + c_m u per axis, one rounding.
__device__ __forceinline__ float trial_f32(float p, float cm, float u) { return __fmaf_rn(cm, u, p); }

// 16-byte asynchronous copy global -> shared (completes at cp_async_wait),
// through L2 only (no L1 line that another SM's writes could leave stale).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of the latest committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Position of the k-th (from 0) set bit of m; m has more than k set bits.
// It is the largest p with popc(m & (2^p - 1)) <= k: a binary search over p,
// five steps, the same for every lane.
__device__ __forceinline__ int nth_set(unsigned m, int k)
{
    int pos = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int p = pos + step;
        if (p <= 31 && __popc(m & ((1u << p) - 1u)) <= k) pos = p;
    }
    return pos;
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit j of lane i
// = entry (i, j)): lane j returns column j (bit i = entry (i, j)).  Five
// steps of the block recursion: at step s, lanes with bit s clear swap their
// upper s-blocks with the lower s-blocks of lane ^ s.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    const uint32_t lo[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int sft = 16 >> i;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
        x = (lane & sft) ? ((x & ~lo[i]) | ((y & ~lo[i]) >> sft)) : ((x & lo[i]) | ((y & lo[i]) << sft));
    }
    return x;
}

// ---------------------------------------------------------------------------
// Directions of trials 0 and 1 of particles g0 .. g0+31 of one RVE (slot
// order), drawn by one warp.  Trial t (0..63) is try t & 1 of particle
// g0 + (t >> 1); lane l owns trials l and 32 + l.  Each round every lane
// evaluates one candidate of a pending trial -- when fewer than 32 trials are
// pending, several lanes take consecutive candidates of one trial -- and a
// trial takes its first accepted candidate (the direction of the draw).
// ---------------------------------------------------------------------------
template <int DIM, bool F32>
__device__ __forceinline__ void draw_warp(const RveDev *st, const Slot &d, int64_t g0, int np_w)
{
    using PT = typename SweepSmem<F32>::PT;
    using DT = typename SweepSmem<F32>::DT;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const uint64_t seed = st->seed, sweep = st->sweep;
    const uint32_t pidv = lane < np_w ? d.pid[g0 + lane] : 0u;
    int nm[2] = {0, 0};
    bool pend[2] = {(lane >> 1) < np_w, ((32 + lane) >> 1) < np_w};
    DT res[2][3] = {{(DT)1, (DT)0, (DT)0}, {(DT)1, (DT)0, (DT)0}};
    for (;;) {
        const unsigned m0 = __ballot_sync(0xffffffffu, pend[0]), m1 = __ballot_sync(0xffffffffu, pend[1]);
        const int c0 = __popc(m0), np = c0 + __popc(m1);
        if (np == 0) break;
        // the trial this lane evaluates (rank k among the pending ones) and
        // its candidate index
        // lane = rep np + k; with np <= 31 the quotient of (lane + 1/2) / np
        // is never within 1/64 of an integer, so the binary32 value truncates
        // to it exactly
        int k = lane, rep = 0;
        if (np < 32) {
            rep = (int)(((float)lane + 0.5f) / (float)np);
            k = lane - rep * np;
        }
        const int tr = k < c0 ? nth_set(m0, k) : 32 + nth_set(m1, k - c0);
        const int nmA = __shfl_sync(0xffffffffu, nm[0], tr & 31), nmB = __shfl_sync(0xffffffffu, nm[1], tr & 31);
        const int mc = (tr < 32 ? nmA : nmB) + rep;
        const uint64_t pidt = __shfl_sync(0xffffffffu, pidv, tr >> 1);  // 32-bit id
        DT v[3] = {(DT)0, (DT)0, (DT)0}, s = (DT)0;
        bool ok = false;
        if (mc < MAX_CAND) {
            if constexpr (F32) ok = cand_f32<DIM>(seed, sweep, pidt, (uint64_t)(tr & 1), (uint64_t)mc, v, s);
            else ok = cand_f64<DIM>(seed, sweep, pidt, (uint64_t)(tr & 1), (uint64_t)mc, v, s);
        }
        DT w[3] = {(DT)0, (DT)0, (DT)0};
        if (ok) {
            if constexpr (F32) {
                const float inv = rsqrtf(s);
#pragma unroll
                for (int a = 0; a < DIM; a++) w[a] = v[a] * inv;
            } else {
                const double nrm = __dsqrt_rn(s);
#pragma unroll
                for (int a = 0; a < DIM; a++) w[a] = __ddiv_rn(v[a], nrm);
            }
        }
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            // lanes rank, rank + np, ... evaluated candidates nm, nm + 1, ...
            const int rank = h == 0 ? __popc(m0 & below) : c0 + __popc(m1 & below);
            const bool mine = pend[h] && rank < 32;
            int src = -1, nas = 0;
            if (mine) {
                for (int i = rank; i < 32; i += np) {
                    nas++;
                    if (src < 0 && ((okm >> i) & 1u)) src = i;
                }
            }
            DT x[3];
#pragma unroll
            for (int a = 0; a < 3; a++) x[a] = __shfl_sync(0xffffffffu, w[a], src < 0 ? lane : src);
            if (mine) {
                if (src >= 0) {
                    res[h][0] = x[0];
                    res[h][1] = x[1];
                    res[h][2] = DIM == 3 ? x[2] : (DT)0;
                    pend[h] = false;
                } else {
                    nm[h] += nas;
                    if (nm[h] >= MAX_CAND) pend[h] = false;  // no candidate accepted: e_0
                }
            }
        }
    }
    PT *out = reinterpret_cast<PT *>(st->dirs) + 2 * g0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int t = 32 * h + lane;
        if ((t >> 1) < np_w) {
            PT e;
            e.x = res[h][0];
            e.y = res[h][1];
            e.z = res[h][2];
            e.w = (DT)0;
            out[t] = e;
        }
    }
}

// Warps walk the 32-particle pieces of the RVEs at work (plan actp).
template <bool F32>
__global__ void __launch_bounds__(256) k_draw(BatchDev *bd)
{
    const int B = bd->B, stride = gridDim.x * (blockDim.x >> 5);
    int r, chunk, sub;
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); warp_piece(bd->actp, B, it, r, chunk, sub);
         it += stride) {
        const RveDev *st = bd->rv[r];
        const int64_t g0 = (int64_t)(chunk - bd->actp[r]) * 256 + sub * 32;
        const int n = st->n;
        if (g0 >= n) continue;
        const int np_w = n - g0 < 32 ? (int)(n - g0) : 32;
        const Slot d = st->slot[st->dst_idx];
        if (st->dim == 3) draw_warp<3, F32>(st, d, g0, np_w);
        else draw_warp<2, F32>(st, d, g0, np_w);
    }
}

// ---------------------------------------------------------------------------
// Dependencies of a cell in the one-launch sweep: before a cell of colour chi
// is staged, every non-empty cell within reach (home +-H) whose colour is
// lower must have finished this sweep -- exactly the cells of lower colour
// whose moves the serial order lets it see; cells of higher colour wait for
// this one in turn, so they are still unmoved.  Cells are handed out in
// colour order, so every cell waited for is already held by a running warp.
// A wait gives up after wait_limit polls and sets the RVE's status (the host
// reports SRM_E_DEVICE_TIMEOUT).
// ---------------------------------------------------------------------------
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
        for (int it = 0; ld_relaxed(&st->done[c]) != epoch; it++) {
            if (it >= limit) {
                atomicExch(&st->status, STATUS_WAIT_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
    }
    // the producer's writes happen before its release store; this lane's
    // relaxed loads that saw it, followed by the fence, synchronise with it;
    // the warp barrier orders the fence before every lane's later reads
    fence_acquire();
    __syncwarp();
}

// Work counters of one cell, reduced per warp after the cell.
struct CellCount {
    int moved = 0;
    unsigned examined = 0;          // pairs tested (this lane)
    unsigned long long trials = 0;  // trials evaluated (warp-uniform)
    unsigned long long alg5 = 0;    // trials x (3^d stencil population - 1)
};

// One cell of colour chi (work item t of its RVE), processed by one warp.
template <int DIM, bool F32>
__device__ __forceinline__ void sweep_cell(RveDev *st, int chi, int t, unsigned char *base, int cap, CellCount &cc)
{
    using PT = typename SweepSmem<F32>::PT;
    using DT = typename SweepSmem<F32>::DT;
    const int lane = threadIdx.x & 31;
    StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
    PT *cpos = reinterpret_cast<PT *>(base + ST_HDR);
    float4 *capx = reinterpret_cast<float4 *>(cpos + cap);  // FP64 form only
    PT *nbuf = reinterpret_cast<PT *>(F32 ? (void *)(cpos + cap) : (void *)(capx + cap));
    PT *pre = nbuf + NEAR_CAP;                               // [PRE_NH][PRE_TRIALS]

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

    const int hx = 3 * (t % s0) + chi % 3;
    const int hy = 3 * ((t / s0) % s1) + (chi / 3) % 3;
    const int hz = DIM == 3 ? 3 * (t / (s0 * s1)) + chi / 9 : 0;
    const int cell = hx + st->gn[0] * (hy + st->gn[1] * hz);
    const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
    if (nh == 0) return;  // nothing moves: nobody waits for an empty cell
    const uint32_t epoch = (uint32_t)(st->sweep + 1);
    // before the wait (none of this changes while the lower-colour cells
    // run): the pre-drawn directions of the cell's particles (slot order =
    // the cell's particles in ascending id), the stencil list, and an L2
    // prefetch of every candidate's line -- L2 is the point of coherence, so
    // lines of cells still moving are refreshed by their writes, and the
    // staging loads after the wait find them there
    const uint32_t npre = nh < (uint32_t)PRE_NH ? nh : (uint32_t)PRE_NH;
    {
        const PT *src = reinterpret_cast<const PT *>(st->dirs) + 2 * (size_t)hb;
        constexpr int PIECES = (int)(sizeof(PT) / 16);
        for (uint32_t e = lane; e < npre * PRE_TRIALS * PIECES; e += 32)
            cp_async16(reinterpret_cast<unsigned char *>(pre) + 16 * (size_t)e,
                       reinterpret_cast<const unsigned char *>(src) + 16 * (size_t)e);
        cp_async_commit();
    }
    int nst, center;
    const uint32_t T = list_stencil(st, cs, hx, hy, hz, S, nst, center);
    for (int j = lane; j < nst; j += 32) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(pos + S.b[j]);
        const uintptr_t e = a + (uintptr_t)(S.o[j + 1] - S.o[j]) * sizeof(PT);
        for (uintptr_t l = a & ~(uintptr_t)127; l < e; l += 128) prefetch_l2(reinterpret_cast<const void *>(l));
    }
    wait_lower_colours<DIM>(st, cs, hx, hy, hz, chi, epoch);
    // population of the 3^d cells around the home cell (Algorithm 5's own
    // candidate set; the listed stencil is larger when H = 2)
    uint32_t T3 = 0;
    for (int j = lane; j < nst; j += 32)
        if (S.sh[j][0] >= -1 && S.sh[j][0] <= 1 && S.sh[j][1] >= -1 && S.sh[j][1] <= 1 && S.sh[j][2] >= -1 &&
            S.sh[j][2] <= 1)
            T3 += S.o[j + 1] - S.o[j];
    T3 = __reduce_add_sync(0xffffffffu, T3);
    // home corner (FP64 form: the binary32 copies are relative to it)
    const double ox = hx * st->gw[0], oy = hy * st->gw[1], oz = hz * st->gw[2];
    auto locate = [&](uint32_t k, int &j) -> uint32_t {
        j = find_cell(S, nst, k);
        return S.b[j] + (k - S.o[j]);
    };
    auto shift = [&](PT c, int j) -> PT {
        if constexpr (F32) {
            c.x = __fmaf_rn((float)S.sh[j][0], w[0], c.x);
            c.y = __fmaf_rn((float)S.sh[j][1], w[1], c.y);
            c.z = __fmaf_rn((float)S.sh[j][2], w[2], c.z);
        }
        return c;
    };
    auto fetch = [&](uint32_t k, uint32_t &g) -> PT {
        int j;
        g = locate(k, j);
        return shift(pos[g], j);
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

    // 1. stage the candidates that can reach the home cell (home first).
    // FP32 form: RING - 1 chunks of 32 candidates ahead of the one being
    // culled are in flight (cp.async into a ring in shared memory); FP64
    // form: the load of the next chunk is issued before the current one is
    // culled.  Staging stops at the first chunk that would overflow the
    // capacity; candidates from kstop on are read from global memory (culled
    // the same way) when the near lists are built.
    float rh = 0.f;
    for (uint32_t m = lane; m < nh; m += 32) rh = fmaxf(rh, (float)pos[hb + m].w);
    for (int o = 16; o > 0; o >>= 1) rh = fmaxf(rh, __shfl_xor_sync(0xffffffffu, rh, o));
    uint32_t Tk = 0, kstop = T;
    bool stop = false;
    if constexpr (F32) {
        PT *ring = pre + PRE_NH * PRE_TRIALS;
        uint8_t *rj = reinterpret_cast<uint8_t *>(ring + RING * 32);  // stencil cell of each ring entry
        const uint32_t nq = (T + 31) / 32;
        // chunk q into ring slot q mod RING, one commit group per chunk
        auto issue = [&](uint32_t q) {
            const uint32_t k = q * 32 + (uint32_t)lane;
            if (q < nq && k < T) {
                int j;
                const uint32_t g = locate(k, j);
                cp_async16(ring + (q % RING) * 32 + lane, pos + g);
                rj[(q % RING) * 32 + lane] = (uint8_t)j;
            }
            cp_async_commit();
        };
        for (uint32_t q = 0; q + 1 < (uint32_t)RING; q++) issue(q);
        for (uint32_t q = 0; q < nq; q++) {
            issue(q + RING - 1);  // into the slot of chunk q - 1, culled in the last round
            cp_async_wait_group<RING - 1>();
            const uint32_t k0 = q * 32, k = k0 + lane;
            bool keep = false;
            PT c;
            if (k < T) {
                c = shift(ring[(q % RING) * 32 + lane], rj[(q % RING) * 32 + lane]);
                const float r = rh + c.w + 2.f * cmf;
                keep = k < nh || box_dist2(c, w, DIM) <= r * r * 1.0004f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (Tk + __popc(bal) > (uint32_t)cap) {
                kstop = k0;
                stop = true;
                break;
            }
            const uint32_t at = Tk + __popc(bal & ((1u << lane) - 1u));
            if (keep) cpos[at] = c;
            Tk += __popc(bal);
        }
    } else {
        PT cn;
        int jn = 0;
        if (lane < T) cn = pos[locate(lane, jn)];
        for (uint32_t k0 = 0; k0 < T; k0 += 32) {
            const uint32_t k = k0 + lane;
            const PT c = k < T ? shift(cn, jn) : cn;
            if (k + 32 < T) cn = pos[locate(k + 32, jn)];
            bool keep = false;
            float4 ca;
            if (k < T) {
                ca = approx(c);
                const float r = rh + ca.w + 2.f * cmf;
                keep = k < nh || box_dist2(ca, w, DIM) <= r * r * 1.0004f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (Tk + __popc(bal) > (uint32_t)cap) {
                kstop = k0;
                stop = true;
                break;
            }
            const uint32_t at = Tk + __popc(bal & ((1u << lane) - 1u));
            if (keep) {
                cpos[at] = c;
                if constexpr (!F32) capx[at] = ca;
            }
            Tk += __popc(bal);
        }
    }
    if (stop && lane == 0) atomicAdd(&st->stage_overflow, 1ull);
    cp_async_wait();
    __syncwarp();

    // 2. the particles of the home cell, ascending id
    const uint32_t scan = Tk + (T - kstop);
    for (uint32_t m = 0; m < nh; m++) {
        const uint32_t gi = hb + m;
        // home particles lead the candidate list and are always kept, so
        // the first ones are staged at their own index
        const PT p = m < Tk ? cpos[m] : pos[gi];
        const float4 pa = approx(p);
        const bool have_pre = m < (uint32_t)PRE_NH;
        // near list: copies of every candidate within R_i + R_t + c_m
        // (staged candidates, then the unstaged remainder from global)
        uint32_t nn = 0;
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
        if (!use_near && lane == 0) atomicAdd(&st->near_fallback, 1ull);
        bool done = false;
        int l0 = 0;
        PT np;
        // trials in batches, one trial per lane -- the two pre-drawn ones
        // first (most particles take the first trial), then eight at a time
        // drawn by all lanes -- each tested against the near list
        while (!done && l0 < N_l) {
            const bool first = l0 == 0 && have_pre;
            const int bsz = first ? PRE_TRIALS : 8;
            const int lmax = N_l - l0 < bsz ? N_l - l0 : bsz;
            double qt[3] = {0.0, 0.0, 0.0};
            float qs[3] = {0.f, 0.f, 0.f};
            DT u[3] = {(DT)0, (DT)0, (DT)0};
            if (first) {
                if (lane < lmax) {
                    const PT e = pre[PRE_TRIALS * m + lane];
                    u[0] = e.x;
                    u[1] = e.y;
                    u[2] = e.z;
                }
            } else {
                draw8<DIM, F32>(seed, sweep, (uint64_t)d.pid[gi], l0, u);
            }
            if (lane < lmax) {
                if constexpr (F32) {
                    qs[0] = trial_f32(p.x, cmf, u[0]);
                    qs[1] = trial_f32(p.y, cmf, u[1]);
                    qs[2] = DIM == 3 ? trial_f32(p.z, cmf, u[2]) : p.z;
                } else {
                    qt[0] = wrap_d(__dadd_rn(p.x, __dmul_rn(c_m, u[0])), st->L[0]);
                    qt[1] = wrap_d(__dadd_rn(p.y, __dmul_rn(c_m, u[1])), st->L[1]);
                    qt[2] = DIM == 3 ? wrap_d(__dadd_rn(p.z, __dmul_rn(c_m, u[2])), st->L[2]) : p.z;
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
                cc.trials++;
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
                    cc.examined++;
                    if constexpr (F32) hit = hit_f32<DIM>(qf, p.w, c, g1);
                    else hit = collide64<DIM>(st->images, q, p.w, c.x, c.y, c.z, c.w, st->L, st->halfL);
                }
                if (!__any_sync(0xffffffffu, hit)) {
                    if constexpr (F32) np = make_float4(qf[0], qf[1], qf[2], p.w);
                    else np = make_double4_32a(q[0], q[1], q[2], p.w);
                    done = true;
                    break;
                }
            }
        }
        if (done) {
            if (lane == 0) {
                if (m < Tk) {
                    cpos[m] = np;
                    if constexpr (!F32) capx[m] = approx(np);
                }
                pos[gi] = np;
            }
            cc.moved++;
        }
        if (lane == 0) st->flags[gi] = done ? 1 : 0;
        __syncwarp();
    }
    cc.alg5 += cc.trials * (unsigned long long)(T3 - 1);
    // lane 0 wrote every global update of this cell (positions, flags), so
    // its release store publishes them
    if (lane == 0) st_release(&st->done[cell], epoch);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// The staged path of one cell (FP32 form): every candidate of the stencil is
// copied to shared memory (cp.async, 16 bytes per copy), so that the cell's service
// time -- which lies on the chain of the colour order -- holds one memory
// round trip instead of a load per chunk, and the work that does not
// depend on lower-colour cells is done before waiting for them:
//  * the home cell and the cells of higher colour (which wait for this
//    one) cannot change before this cell finishes; they are copied, culled
//    (FP32 form: shifted into the home cell's frame) and compacted first;
//    the positions of trials 0 and 1 of the home particles (pre-drawn
//    directions, positions unchanged before each particle's turn) are
//    formed, and both the near bits and the pre-tests of these trials are
//    computed over these candidates -- all before the wait;
//  * each lower-colour cell is copied by the lane that polled it as soon as
//    its stamp is seen, into a list that starts on a 32-candidate chunk;
//    after the last one: cull, near bits and pre-tests over those chunks;
//  * near bits: per group of 32 home particles, lane i of a chunk marks
//    home particle m when candidate i is within R_m + R_t + c_m of it (plus
//    c_m for home candidates, which may move before m's turn) -- a superset
//    of everything a trial of m can touch -- and a 32 x 32 bit transpose
//    across the lanes gives each particle one word per chunk;
//  * pre-tests: trials 0 and 1 of every particle against its marked
//    candidates outside the home cell, which do not change while the cell
//    runs; at a particle's turn only its marked home candidates remain;
//  * later trials (drawn by the lanes) test every marked candidate, at
//    current positions (moves update the copies).
// The decisions are the predicate of Algorithm 5 on the same values as the
// general path, so the results are the same.  Returns false, having issued
// nothing, when the two lists do not fit cap candidates.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ bool sweep_cell_staged(RveDev *st, int chi, int t, unsigned char *base, int cap,
                                                  CellCount &cc)
{
    using SM = SweepSmem<true>;
    using PT = float4;
    const int lane = threadIdx.x & 31;
    StencilSmem &S = *reinterpret_cast<StencilSmem *>(base);
    PT *cpos = reinterpret_cast<PT *>(base + ST_HDR);
    uint32_t *wbits = reinterpret_cast<uint32_t *>(base + SM::off_bits(cap));
    uint8_t *cid = base + SM::off_cid(cap);
    // a particle's near list, as candidate indices
    uint16_t *nlist = reinterpret_cast<uint16_t *>(base + SM::off_nl(cap));
    uint32_t *shit = reinterpret_cast<uint32_t *>(base + SM::off_shit(cap));
    PT *pre = reinterpret_cast<PT *>(base + SM::off_pre(cap));
    uint8_t *const flags = st->flags;

    const Slot d = st->slot[st->dst_idx];
    PT *pos = reinterpret_cast<PT *>(d.pos);
    const uint32_t *cs = st->cell_start;
    const int s0 = st->sub[0], s1 = st->sub[1];
    const float w[3] = {(float)st->gw[0], (float)st->gw[1], (float)st->gw[2]};
    const uint64_t seed = st->seed, sweep = st->sweep;
    const float cmf = (float)st->c_m;
    const float g1 = 1.0f + st->guard;
    const int N_l = st->N_l;

    const int hx = 3 * (t % s0) + chi % 3;
    const int hy = 3 * ((t / s0) % s1) + (chi / 3) % 3;
    const int hz = DIM == 3 ? 3 * (t / (s0 * s1)) + chi / 9 : 0;
    const int cell = hx + st->gn[0] * (hy + st->gn[1] * hz);
    const uint32_t hb = cs[cell], nh = cs[cell + 1] - hb;
    if (nh == 0) return true;  // nothing moves: nobody waits for an empty cell
    int nst;
    uint32_t Tn, Tl;
    list_stencil_split(st, cs, hx, hy, hz, chi, S, nst, Tn, Tl);
    const uint32_t Rl = (Tn + 31) / 32 * 32;  // first index of the lower-colour list
    if (Rl + Tl > (uint32_t)cap) return false;
    const uint32_t epoch = (uint32_t)(st->sweep + 1);
    // the pre-drawn directions of the cell's first particles
    const uint32_t npre = nh < (uint32_t)PRE_NH ? nh : (uint32_t)PRE_NH;
    {
        const PT *src = reinterpret_cast<const PT *>(st->dirs) + 2 * (size_t)hb;
        for (uint32_t e = lane; e < npre * PRE_TRIALS; e += 32)
            cp_async16(reinterpret_cast<unsigned char *>(pre) + 16 * (size_t)e,
                       reinterpret_cast<const unsigned char *>(src) + 16 * (size_t)e);
    }
    // id of home particle `lane` (the draws of later trials)
    uint32_t my_pid = (uint32_t)lane < nh ? d.pid[hb + lane] : 0u;
    // copies of stencil cell j (by the lane that owns it) into a list
    auto copy_cell = [&](int j, uint32_t list0) {
        const uint32_t nj = S.n[j], o = list0 + S.o[j];
        const unsigned char *src = reinterpret_cast<const unsigned char *>(pos + S.b[j]);
        unsigned char *dst = reinterpret_cast<unsigned char *>(cpos + o);
        for (uint32_t e = 0; e < nj; e++) cp_async16(dst + 16 * (size_t)e, src + 16 * (size_t)e);
        for (uint32_t e = 0; e < nj; e++) cid[o + e] = (uint8_t)j;
    };
    for (int j = lane; j < nst; j += 32)
        if (!S.low[j]) copy_cell(j, 0);
    cp_async_wait();
    __syncwarp();

    // largest home radius
    float rh = 0.f;
    for (uint32_t m = lane; m < nh; m += 32) rh = fmaxf(rh, (float)cpos[m].w);
    for (int o = 16; o > 0; o >>= 1) rh = fmaxf(rh, __shfl_xor_sync(0xffffffffu, rh, o));
    // shift into the home cell's frame and keep the candidates of
    // [src, src + n) that can reach the home cell (the cull of the general
    // path), compacted to dst <= src -- a chunk's entries are
    // read before any is written, and writes land at or below the chunk's
    // first index.  The home particles (indices below nh of the first list)
    // are all kept, at their own index.
    auto cull = [&](uint32_t src, uint32_t n, uint32_t dst) -> uint32_t {
        uint32_t kept = 0;
        for (uint32_t k0 = 0; k0 < n; k0 += 32) {
            const uint32_t k = src + k0 + (uint32_t)lane;
            bool keep = false;
            PT c;
            if (k0 + lane < n) {
                c = cpos[k];
                const int j = cid[k];
                c.x = __fmaf_rn((float)S.sh[j][0], w[0], c.x);
                c.y = __fmaf_rn((float)S.sh[j][1], w[1], c.y);
                c.z = __fmaf_rn((float)S.sh[j][2], w[2], c.z);
                const float r = rh + c.w + 2.f * cmf;
                keep = (src == 0 && k < nh) || box_dist2(c, w, DIM) <= r * r * 1.0004f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) cpos[dst + kept + __popc(bal & ((1u << lane) - 1u))] = c;
            kept += __popc(bal);
            __syncwarp();
        }
        return kept;
    };
    // first list, padded to a whole chunk with candidates out of reach
    const uint32_t Tkn = cull(0, Tn, 0);
    const uint32_t Tkp = (Tkn + 31) / 32 * 32;
    if (Tkn + lane < Tkp) {
        cpos[Tkn + lane] = make_float4(1e30f, 1e30f, 1e30f, 0.0f);
    }
    // positions of trials 0 and 1 of the first home particles, in place of
    // their directions
    for (uint32_t pi = lane; pi < 2 * npre; pi += 32) {
        const uint32_t m = pi >> 1;
        if ((int)(pi & 1) >= N_l) continue;
        const PT p = cpos[m];
        const PT e = pre[pi];
        pre[pi] = make_float4(trial_f32(p.x, cmf, e.x), trial_f32(p.y, cmf, e.y),
                              DIM == 3 ? trial_f32(p.z, cmf, e.z) : p.z, 0.0f);
    }
    __syncwarp();
    // near bits of home particles g0 .. g0+gn-1 over chunks [c0, c1)
    auto mark = [&](uint32_t g0, uint32_t gn, uint32_t c0, uint32_t c1, uint32_t Tk) {
        for (uint32_t ch = c0; ch < c1; ch++) {
            const uint32_t k = ch * 32 + (uint32_t)lane;
            uint32_t bits = 0;
            if (k < Tk) {
                const float4 ca = cpos[k];
                const float base_r = ca.w + cmf + (k < nh ? cmf : 0.f);
                for (uint32_t mm = 0; mm < gn; mm += 4) {
                    float4 pm[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint32_t hq = mm + q < gn ? mm + q : gn - 1;
                        pm[q] = cpos[g0 + hq];
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint32_t hm = g0 + mm + q;
                        if (mm + q < gn && k != hm && within_f32(pm[q], ca, pm[q].w + base_r, DIM))
                            bits |= 1u << (mm + q);
                    }
                }
            }
            bits = transpose32(bits, lane);
            if ((uint32_t)lane < gn) wbits[ch * 32 + lane] = bits;
        }
        __syncwarp();
    };
    // pre-tests of trials 0 and 1 of the first home particles against their
    // marked candidates outside the home cell in chunks [c0, c1): lane pi of
    // round r takes particle 16 r + pi / 2, trial pi % 2; bit pi of shit[r]
    // = that trial hits (or-ed over the calls)
    auto pretest = [&](uint32_t c0, uint32_t c1) {
        for (uint32_t r0 = 0; r0 < 2 * npre; r0 += 32) {
            const uint32_t pi = r0 + (uint32_t)lane;
            const uint32_t mm = pi >> 1;
            bool hit = false;
            if (pi < 2 * npre && (int)(pi & 1) < N_l) {
                const float Rm = cpos[mm].w;
                const PT qq = pre[pi];
                const float qf[3] = {qq.x, qq.y, qq.z};
                for (uint32_t ch = c0; ch < c1 && !hit; ch++) {
                    uint32_t wd = wbits[ch * 32 + mm];
                    // drop the home candidates (indices below nh)
                    if (ch * 32 < nh) wd &= nh - ch * 32 >= 32 ? 0u : ~((1u << (nh - ch * 32)) - 1u);
                    while (wd && !hit) {
                        const int bt = __ffs(wd) - 1;
                        wd &= wd - 1;
                        const PT c = cpos[ch * 32 + bt];
                        cc.examined++;
                        hit = hit_f32<DIM>(qf, Rm, c, g1);
                    }
                }
            }
            const uint32_t hbits = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) shit[r0 >> 5] = (c0 == 0 ? 0u : shit[r0 >> 5]) | hbits;
        }
        __syncwarp();
    };
    const uint32_t gn0 = nh < 32u ? nh : 32u;
    mark(0, gn0, 0, Tkp / 32, Tkp);
    pretest(0, Tkp / 32);

    // lower-colour cells: wait for each (bounded), then copy it
    {
        const int limit = st->wait_limit;
        for (int j = lane; j < nst; j += 32) {
            if (!S.low[j] || S.n[j] == 0) continue;
            if (limit < 0) {
                atomicExch(&st->status, STATUS_WAIT_TIMEOUT);
            } else {
                const uint32_t *stamp = &st->done[S.cell[j]];
                for (int it = 0; ld_relaxed(stamp) != epoch; it++) {
                    if (it >= limit) {
                        atomicExch(&st->status, STATUS_WAIT_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            // the producer's writes happen before its release store; this
            // lane's relaxed load that saw it, followed by the fence,
            // synchronises with it before the copies below
            fence_acquire();
            copy_cell(j, Rl);
        }
    }
    cp_async_wait();
    __syncwarp();
    const uint32_t Tk = Tkp + cull(Rl, Tl, Tkp);
    const uint32_t nchunks = (Tk + 31) / 32;
    if (nchunks > Tkp / 32) {
        mark(0, gn0, Tkp / 32, nchunks, Tk);
        pretest(Tkp / 32, nchunks);
    }
    // population of the 3^d cells around the home cell (Algorithm 5's own
    // candidate set; the listed stencil is larger when H = 2)
    uint32_t T3 = 0;
    for (int j = lane; j < nst; j += 32)
        if (S.sh[j][0] >= -1 && S.sh[j][0] <= 1 && S.sh[j][1] >= -1 && S.sh[j][1] <= 1 && S.sh[j][2] >= -1 &&
            S.sh[j][2] <= 1)
            T3 += S.n[j];
    T3 = __reduce_add_sync(0xffffffffu, T3);
    // trials tested at once: lanes form `tpar` groups of G lanes, lane
    // (group t, position c) tests trial t against the marked candidates of
    // chunk c
    const int tpar = nchunks <= 4 ? 8 : (nchunks <= 8 ? 4 : (nchunks <= 16 ? 2 : 1));
    const int G = 32 / tpar, tsub = lane / G, csub = lane % G;
    // the word of chunk `lane` of home particle mm of the current group
    auto word_all = [&](uint32_t mm) -> uint32_t {
        return (uint32_t)lane < nchunks ? wbits[lane * 32 + mm] : 0u;
    };
    for (uint32_t g0 = 0; g0 < nh; g0 += 32) {
        const uint32_t gn = nh - g0 < 32u ? nh - g0 : 32u;
        if (g0 > 0) {
            my_pid = (uint32_t)lane < gn ? d.pid[hb + g0 + lane] : 0u;
            mark(g0, gn, 0, nchunks, Tk);
        }
        // the group's particles, ascending id
        for (uint32_t m = g0; m < g0 + gn; m++) {
            const uint32_t gi = hb + m;
            const uint32_t pid_m = __shfl_sync(0xffffffffu, my_pid, (int)(m - g0));
            const PT p = cpos[m];
            const uint32_t word = (uint32_t)csub < nchunks ? wbits[csub * 32 + (m - g0)] : 0u;
            const bool have_pre = m < (uint32_t)PRE_NH;
            bool done = false;
            int l0 = 0;
            PT np;
            if (have_pre && nh <= 32) {
                // trials 0 and 1, whose positions and pre-tests (candidates
                // outside the home cell) the pre-test pass left: lane h tests
                // both against home particle h at its current position when
                // h is marked near this particle
                const int lmax = N_l < PRE_TRIALS ? N_l : PRE_TRIALS;
                const uint32_t sb = (shit[(2 * (m - g0)) >> 5] >> ((2 * (m - g0)) & 31)) & 3u;
                const uint32_t hw = wbits[m - g0] & (nh == 32 ? 0xffffffffu : (1u << nh) - 1u);
                const PT q0 = pre[PRE_TRIALS * m], q1 = pre[PRE_TRIALS * m + 1];
                bool h0 = false, h1 = false;
                if ((hw >> lane) & 1u) {
                    const PT c = cpos[lane];
                    cc.examined += lmax;
                    const float a0[3] = {q0.x, q0.y, q0.z}, a1[3] = {q1.x, q1.y, q1.z};
                    h0 = hit_f32<DIM>(a0, p.w, c, g1);
                    h1 = lmax > 1 && hit_f32<DIM>(a1, p.w, c, g1);
                }
                const bool f0 = (sb & 1u) || __any_sync(0xffffffffu, h0);
                const bool f1 = lmax < 2 || (sb & 2u) || __any_sync(0xffffffffu, h1);
                if (!f0 || !f1) {
                    const PT qa = !f0 ? q0 : q1;
                    np = make_float4(qa.x, qa.y, qa.z, p.w);
                    done = true;
                    cc.trials += !f0 ? 1 : 2;
                } else {
                    cc.trials += lmax;
                }
                l0 = lmax;
            } else if (have_pre) {
                // the same with more than 32 home particles: lane t takes
                // trial t and walks the marked home candidates
                const int lmax = N_l < PRE_TRIALS ? N_l : PRE_TRIALS;
                const uint32_t sb = (shit[(2 * (m - g0)) >> 5] >> ((2 * (m - g0)) & 31)) & 3u;
                float qs[3] = {0.f, 0.f, 0.f};
                bool hit = false;
                if (lane < lmax) {
                    const PT e = pre[PRE_TRIALS * m + lane];  // the trial position
                    qs[0] = e.x;
                    qs[1] = e.y;
                    qs[2] = e.z;
                    hit = (sb >> lane) & 1u;
                    for (uint32_t ch = 0; ch * 32 < nh && !hit; ch++) {
                        uint32_t wd = wbits[ch * 32 + (m - g0)];
                        const uint32_t nin = nh - ch * 32;  // home candidates in this chunk
                        if (nin < 32) wd &= (1u << nin) - 1u;
                        while (wd && !hit) {
                            const int bt = __ffs(wd) - 1;
                            wd &= wd - 1;
                            const PT c = cpos[ch * 32 + bt];
                            cc.examined++;
                            hit = hit_f32<DIM>(qs, p.w, c, g1);
                        }
                    }
                }
                const unsigned clean = ~__ballot_sync(0xffffffffu, hit) & ((1u << lmax) - 1u);
                if (clean) {
                    const int sl = __ffs(clean) - 1;
                    np = make_float4(__shfl_sync(0xffffffffu, qs[0], sl), __shfl_sync(0xffffffffu, qs[1], sl),
                                     __shfl_sync(0xffffffffu, qs[2], sl), p.w);
                    done = true;
                    cc.trials += sl + 1;
                } else {
                    cc.trials += lmax;
                }
                l0 = lmax;
            }
            // later trials: the particle's marked candidates (every chunk,
            // home included) as one index list, so that lanes (t, j) test
            // trial t against list entries j, j + 4, ... -- eight trials at
            // once; lists longer than NL_CAP keep the chunk rounds below
            uint32_t nn = 0;
            if (!done && l0 < N_l) {
                const uint32_t cnt = __popc(word_all(m - g0));
                uint32_t inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                nn = __shfl_sync(0xffffffffu, inc, 31);
                if (nn <= (uint32_t)NL_CAP) {
                    uint32_t wd = word_all(m - g0), at = inc - cnt;
                    while (wd) {
                        const int bt = __ffs(wd) - 1;
                        wd &= wd - 1;
                        nlist[at++] = (uint16_t)(lane * 32 + bt);
                    }
                }
                __syncwarp();
            }
            while (!done && l0 < N_l) {
                // later trials eight at a time, drawn by the lanes
                const int lmax = N_l - l0 < 8 ? N_l - l0 : 8;
                float qs[3] = {0.f, 0.f, 0.f};
                float u[3] = {0.f, 0.f, 0.f};
                draw8<DIM, true>(seed, sweep, (uint64_t)pid_m, l0, u);
                if (lane < lmax) {
                    qs[0] = trial_f32(p.x, cmf, u[0]);
                    qs[1] = trial_f32(p.y, cmf, u[1]);
                    qs[2] = DIM == 3 ? trial_f32(p.z, cmf, u[2]) : p.z;
                }
                l0 += lmax;
                if (nn <= (uint32_t)NL_CAP) {
                    // lane (t, j): trial t = lane / 4 against entries j, j + 4, ...
                    const int tr = lane >> 2, j0 = lane & 3;
                    const int src = tr < lmax ? tr : 0;
                    const float qf[3] = {__shfl_sync(0xffffffffu, qs[0], src), __shfl_sync(0xffffffffu, qs[1], src),
                                         __shfl_sync(0xffffffffu, qs[2], src)};
                    bool hit = false;
                    if (tr < lmax) {
                        for (uint32_t jj = j0; jj < nn && !hit; jj += 4) {
                            const PT c = cpos[nlist[jj]];
                            cc.examined++;
                            hit = hit_f32<DIM>(qf, p.w, c, g1);
                        }
                    }
                    const unsigned hb_ = __ballot_sync(0xffffffffu, hit);
                    int acc = -1;
                    for (int tt = 0; tt < lmax; tt++)
                        if (!((hb_ >> (4 * tt)) & 15u)) {
                            acc = tt;
                            break;
                        }
                    cc.trials += acc >= 0 ? acc + 1 : lmax;
                    if (acc >= 0) {
                        np = make_float4(__shfl_sync(0xffffffffu, qs[0], acc), __shfl_sync(0xffffffffu, qs[1], acc),
                                         __shfl_sync(0xffffffffu, qs[2], acc), p.w);
                        done = true;
                    }
                    continue;
                }
                // rounds of tpar trials; the first clean trial of a round,
                // in trial order, is the move
                for (int lb = 0; lb < lmax && !done; lb += tpar) {
                    const int tr = lb + tsub;  // this lane's trial (valid if < lmax)
                    const int src = tr < lmax ? tr : 0;
                    const float qf[3] = {__shfl_sync(0xffffffffu, qs[0], src), __shfl_sync(0xffffffffu, qs[1], src),
                                         __shfl_sync(0xffffffffu, qs[2], src)};
                    bool hit = false;
                    if (tr < lmax) {
                        uint32_t wd = word;
                        while (wd && !hit) {
                            const int bt = __ffs(wd) - 1;
                            wd &= wd - 1;
                            const PT c = cpos[csub * 32 + bt];
                            cc.examined++;
                            hit = hit_f32<DIM>(qf, p.w, c, g1);
                        }
                    }
                    const unsigned hb_ = __ballot_sync(0xffffffffu, hit);
                    const int nr = lmax - lb < tpar ? lmax - lb : tpar;  // trials in this round
                    int acc = -1;
                    for (int tt = 0; tt < nr; tt++) {
                        const unsigned gm = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (tt * G);
                        if (!(hb_ & gm)) {
                            acc = tt;
                            break;
                        }
                    }
                    cc.trials += acc >= 0 ? acc + 1 : nr;
                    if (acc >= 0) {
                        const int sl = lb + acc;
                        np = make_float4(__shfl_sync(0xffffffffu, qs[0], sl), __shfl_sync(0xffffffffu, qs[1], sl),
                                         __shfl_sync(0xffffffffu, qs[2], sl), p.w);
                        done = true;
                    }
                }
            }
            if (done) {
                if (lane == 0) {
                    cpos[m] = np;
                    pos[gi] = np;
                }
                cc.moved++;
            }
            if (lane == 0) flags[gi] = done ? 1 : 0;
            __syncwarp();
        }
    }
    cc.alg5 += cc.trials * (unsigned long long)(T3 - 1);
    // lane 0 wrote every global update of this cell (positions, flags), so
    // its release store publishes them
    if (lane == 0) st_release(&st->done[cell], epoch);
    __syncwarp();
    return true;
}

// Blocks per SM the register allocation must allow (build-time knobs).  The
// FP32 form comes in two variants: with the staged path (128 registers, no
// spills) and general path only (96 registers, no spills: five blocks of
// four warps per SM where shared memory allows, the better choice for
// stencils of a few particles, where a cell's work is short and latency is
// hidden by more warps).  The FP64 form has the general path only.
#ifndef SRM_SWEEP_MIN_BLOCKS
#define SRM_SWEEP_MIN_BLOCKS 4
#endif
#ifndef SRM_SWEEP_MIN_BLOCKS_GENERAL
#define SRM_SWEEP_MIN_BLOCKS_GENERAL 5
#endif
#ifndef SRM_SWEEP_MIN_BLOCKS_F64
#define SRM_SWEEP_MIN_BLOCKS_F64 4
#endif

// The sweep of the DIM-dimensional RVEs of the group, all colours in one
// launch: work item tg is cell tg mod W of colour tg / W, W the colour cells
// of all DIM-dimensional RVEs at work (offsets act), so items are handed out
// in colour order.
template <int DIM, bool F32, bool STAGED>
__global__ void __launch_bounds__(SW_WARPS * 32, !F32 ? SRM_SWEEP_MIN_BLOCKS_F64
                                                 : (STAGED ? SRM_SWEEP_MIN_BLOCKS : SRM_SWEEP_MIN_BLOCKS_GENERAL))
    k_sweep_df(BatchDev *bd, int cap)
{
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base =
        smem + (size_t)wib * (STAGED ? SweepSmem<F32>::bytes(cap) : SweepSmem<F32>::bytes_general(cap));
    const int B = bd->B;
    const int32_t *off = DIM == 3 ? bd->act3 : bd->act2;
    uint32_t *wq = &bd->wq[DIM == 3 ? 0 : 1];
    const int W = off[B];
    const int total = W * (DIM == 3 ? 27 : 9);
    for (;;) {
        int tg = 0, r = 0;
        if (lane == 0) {
            tg = (int)atomicAdd(wq, 1u);
            if (tg < total) r = find_seg(off, B, tg % W);
        }
        tg = __shfl_sync(0xffffffffu, tg, 0);
        if (tg >= total) break;
        r = __shfl_sync(0xffffffffu, r, 0);
        const int chi = tg / W, t = tg % W - off[r];
        RveDev *st = bd->rv[r];
        if (!st->active || st->dim != DIM || t >= st->nsub) continue;
        CellCount cc;
        bool staged = false;
        if constexpr (STAGED && F32) staged = sweep_cell_staged<DIM>(st, chi, t, base, cap, cc);
        if (!staged) sweep_cell<DIM, F32>(st, chi, t, base, cap, cc);
        const unsigned examined = __reduce_add_sync(0xffffffffu, cc.examined);
        if (lane == 0) {
            if (cc.moved) atomicAdd(&st->red[3], (unsigned long long)cc.moved);
            if (examined) atomicAdd(&st->pairs_sweep, (unsigned long long)examined);
            if (cc.trials) {
                atomicAdd(&st->trials, cc.trials);
                atomicAdd(&st->pairs_alg5, cc.alg5);
            }
        }
    }
}

// The staged path keeps one near-bit word per 32-candidate chunk in a lane:
// at most 32 chunks.
int sweep_cap_max(bool f32) { return f32 ? 1024 : 384; }

static size_t sweep_smem(bool f32, int cap, bool staged)
{
    if (!staged) return SW_WARPS * (f32 ? SweepSmem<true>::bytes_general(cap) : SweepSmem<false>::bytes_general(cap));
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

template <int DIM, bool F32, bool STAGED>
static void launch_sweep_dim(const BatchShape &b, cudaStream_t s)
{
    const size_t smem = sweep_smem(F32, b.cap, STAGED);
    const int64_t want64 = (b.sub_total * (DIM == 3 ? 27 : 9) + SW_WARPS - 1) / SW_WARPS;
    const int want = (int)(want64 > 0x7fffffff ? 0x7fffffff : want64);
    int per_sm = resident_blocks(k_sweep_df<DIM, F32, STAGED>, smem);
    if (b.sweep_bps > 0 && b.sweep_bps < per_sm) per_sm = b.sweep_bps;
    const int res = per_sm * (g_sms > 0 ? g_sms : 1);
    k_sweep_df<DIM, F32, STAGED><<<want < res ? want : res, SW_WARPS * 32, smem, s>>>(b.d, b.cap);
}

// The FP64 form always takes the general path: measured, staging made it
// slower (1e5 monodisperse spheres: 29%; the clustered 1e6-sphere RVE: 11%),
// its binary64 arithmetic dominating what staging saves.
template <int DIM>
static void launch_sweep_form(const BatchShape &b, cudaStream_t s)
{
    if (!b.f32) launch_sweep_dim<DIM, false, false>(b, s);
    else if (b.staged) launch_sweep_dim<DIM, true, true>(b, s);
    else launch_sweep_dim<DIM, true, false>(b, s);
}

int sweep_blocks_per_sm(bool f32, int cap, bool staged)
{
    staged = staged && f32;
    const size_t smem = sweep_smem(f32, cap, staged);
    if (!f32) return resident_blocks(k_sweep_df<3, false, false>, smem);
    return staged ? resident_blocks(k_sweep_df<3, true, true>, smem) : resident_blocks(k_sweep_df<3, true, false>, smem);
}

// Trial directions (k_draw), then the sweep of the 3D and of the 2D RVEs
// (one launch per dimension present; measured faster than one launch over
// both, whose register budget is that of the larger 3D path).
void launch_sweep(const BatchShape &b, cudaStream_t s)
{
    const int nb = plan_blocks(b.blocks_p);
    if (b.f32) k_draw<true><<<nb, 256, 0, s>>>(b.d);
    else k_draw<false><<<nb, 256, 0, s>>>(b.d);
    if (b.has3d) launch_sweep_form<3>(b, s);
    if (b.has2d) launch_sweep_form<2>(b, s);
}

int sweep_launches(const BatchShape &b) { return 1 + (b.has3d ? 1 : 0) + (b.has2d ? 1 : 0); }

// Dynamic shared memory above 48 KB needs an opt-in per kernel.
void sweep_configure()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int s32 = (int)sweep_smem(true, sweep_cap_max(true), true);
    const int g32 = (int)sweep_smem(true, sweep_cap_max(true), false);
    const int s64 = (int)sweep_smem(false, sweep_cap_max(false), false);
    cudaFuncSetAttribute(k_sweep_df<3, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_sweep_df<2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(k_sweep_df<3, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g32);
    cudaFuncSetAttribute(k_sweep_df<2, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g32);
    cudaFuncSetAttribute(k_sweep_df<3, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(k_sweep_df<2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
}

}  // namespace srm
