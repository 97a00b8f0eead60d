// srm_dev.cuh -- device-side state of one RVE and the arithmetic shared by
// the kernels: Philox4x32-10, the unit-vector sampler, periodic wrap, cell
// coordinates, and the exact binary64 collision predicate.
//
// Every binary64 operation that decides a result is written with an explicit
// round-to-nearest intrinsic (__dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn) so
// that the compiler cannot fuse a multiply and an add: the FP64 form then
// evaluates exactly the IEEE-754 operations of Algorithms 3-5 in their
// written order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace srm {

// Modes of the per-RVE state machine of Algorithm 1.
enum Mode : int32_t {
    MODE_BEGIN = 0,  // next super-step starts an iteration (swell, new grid)
    MODE_KLOOP = 1,  // inside the N_k loop (Alg 1)
    MODE_SHAKE = 2,  // shake sweeps on P (Alg 1)
    MODE_DONE = 3,   // P at the target scale
    MODE_SWEEP = 4   // standalone sweep of P at its own scale
};

// One cell-sorted copy of a configuration.  FP64 form: pos = double4_32a
// {x, y, z, R}; FP32 form: pos = float4 {ox, oy, oz, R} with offsets relative
// to the corner of cell `cell` of the grid (gn, gw) the copy was binned on.
struct Slot {
    void *pos;
    double *rb;      // base radius r_i
    uint32_t *pid;   // particle id
    uint32_t *cell;  // linear cell index of the binning that wrote the slot
    int32_t gn[3];
    double gw[3];
};

struct RveDev {
    // ---- constants ----
    int32_t dim, prec, n, N_k, N_l, N_shake;
    double L[3], halfL[3];
    double rmax, c_w, c_m, lam_t;
    float guard;
    float Lf[3];
    uint64_t seed;
    int32_t ncells_cap;
    int64_t iter_cap;
    // ---- buffers ----
    Slot slot[3];
    uint32_t *counts;      // [ncells_cap], all zero between binnings
    uint32_t *cell_start;  // [ncells_cap + 1]
    uint32_t *scan_part;   // block partial sums
    uint32_t *src_cell;    // [n]
    uint32_t *src_rank;    // [n]
    uint8_t *flags;        // [n] 1 if the particle moved in the last sweep (sorted order)
    uint32_t *pcount;      // [n + 1] pair counts by particle id, then offsets
    unsigned long long *red;  // [0] colliding particles, [1] pairs, [2] min-gap key, [3] moves
    // ---- state ----
    int32_t mode, resume_mode, k, s;
    int32_t p_idx, src_idx, dst_idx;
    int32_t active, do_check;
    double lam_P, lam_Q, lam_R;
    uint64_t sweep;
    int32_t gn[3];
    double gw[3];
    int32_t ncells;
    int32_t H[3];
    int32_t sub[3];
    int32_t nsub;
    int64_t iters, accepted, shaken, sweeps;
    // last finished iteration
    int32_t it_result, it_k, it_shake;
    int64_t it_overlap;
    int64_t moved_last;
    int32_t status;
    // work counters: candidate pairs examined by the sweep and by the check
    unsigned long long pairs_sweep, pairs_check;
    unsigned long long stage_overflow;  // cells whose culled stencil exceeded the staging capacity
    unsigned long long trials;          // trial moves evaluated by the sweeps
    unsigned long long pairs_alg5;      // trials x (particles of the 3^d cells around the home cell - 1)
    unsigned long long near_fallback;   // particles whose near list exceeded its capacity (general path)
    uint32_t *done;       // [ncells_cap] epoch stamp of the last sweep that finished the cell
    int32_t wait_limit;   // polls of one dependency before the sweep gives up (< 0: none)
    int32_t images;       // FP64 form: periodicity by image particles instead of the minimum image
    // directions of trials 0 and 1 of every particle for the coming sweep,
    // in the cell-sorted order of the destination slot: [2 n] float4 (FP32
    // form) or double4_32a (FP64 form), entry 2 g + l for slot g, trial l
    void *dirs;
};

// Device status codes (RveDev::status), reported by the host as srm_status.
constexpr int32_t STATUS_WAIT_TIMEOUT = 5;

// A group of RVEs advanced by the same launches (one RVE for a single
// handle, many for a batch).  Kernels indexed by particles, cells or scan
// tiles run one grid over all RVEs: each RVE owns a contiguous range of
// blocks (offsets below, fixed by the RVE's capacities), so that a block
// serves one RVE.  The sweep hands out (RVE, cell) work items from one
// counter per dimension, colour by colour.
struct BatchDev {
    int32_t B;
    int32_t pad;
    RveDev **rv;      // [B]
    int32_t *blk_p;   // [B+1] first block of each RVE, particle-indexed launches
    int32_t *blk_c;   // [B+1] first block of each RVE, cell-indexed launches
    int32_t *tile_c;  // [B+1] first scan tile of each RVE over its cells
    int32_t *tile_n;  // [B+1] first scan tile of each RVE over its particles
    int32_t *sub;     // [B+1] first sweep work item of each RVE (cells of one colour)
    int32_t *act2;    // [B+1] first work item of each 2D RVE at work in this super-step
    int32_t *act3;    // [B+1] the same over the 3D RVEs at work
    int32_t *actp;    // [B+1] first 256-particle chunk of each RVE at work
    int32_t *actc;    // [B+1] first 256-cell chunk of each RVE at work (current grid)
    uint32_t wq[2];   // sweep work counters: [0] 3D RVEs, [1] 2D RVEs
};

// Acquire load / release store of a 32-bit word in global memory (the
// per-cell completion stamps of the one-launch sweep).
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polling without acquire semantics, and the fence that completes an
// acquire pattern once a relaxed load has seen the release store: a waiting
// warp then orders its later reads once per dependency instead of on every
// poll, so that the polls of waiting warps do not disturb the L1 contents
// of the warps at work on the same SM.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Hint: bring the global-memory line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Largest r with off[r] <= x (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int find_seg(const int32_t *off, int B, int x)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// RVE served by this block (all threads of the block must call it).
__device__ __forceinline__ int block_rve(const int32_t *off, int B)
{
    __shared__ int r_sh;
    if (threadIdx.x == 0) r_sh = find_seg(off, B, (int)blockIdx.x);
    __syncthreads();
    return r_sh;
}

// Warp-level walk of a plan of 256-wide chunks: warp w of the grid takes the
// 32-wide pieces w, w + (warps in the grid), ...; returns false when done.
// No block-wide synchronisation, so warps with uneven work do not wait for
// each other.
__device__ __forceinline__ bool warp_piece(const int32_t *off, int B, int it, int &r, int &chunk, int &sub)
{
    const int pieces = off[B] * 8;
    if (it >= pieces) return false;
    chunk = it >> 3;
    sub = it & 7;
    int rr = 0;
    if ((threadIdx.x & 31) == 0) rr = find_seg(off, B, chunk);
    r = __shfl_sync(0xffffffffu, rr, 0);
    return true;
}

// One block per chunk of a plan (offsets off[0..B], the RVEs at work in
// this super-step), in a grid sized for the group's capacity: block b serves
// chunk b; blocks past the plan return at once.  All threads of the block
// must call it; the result is the same for the whole block.
__device__ __forceinline__ bool plan_block(const int32_t *off, int B, int &r)
{
    if ((int)blockIdx.x >= off[B]) return false;
    r = block_rve(off, B);
    return true;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products (high halves xored with the other counter words
// and the key, low halves kept); the key is advanced by the Weyl constants
// between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

// COMPACT keeps the ten rounds as a loop: fewer registers, for the rare
// draws inside the sweep (whose register budget sets its occupancy).
template <bool COMPACT = false>
__device__ __forceinline__ void philox4x32(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    if constexpr (COMPACT) {
#pragma unroll 1
        for (int r = 0; r < 10; r++) {
            philox_round(c, k0, k1);
            k0 += W0;
            k1 += W1;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 10; r++) {
            philox_round(c, k0, k1);
            k0 += W0;
            k1 += W1;
        }
    }
}

// Counter of candidate m of try l of particle pid in sweep `sweep`, key = the
// 64-bit seed (l < 2^16, m < 2^16).
__device__ __forceinline__ void draw_block(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, uint64_t m,
                                           uint32_t c[4], uint32_t &k0, uint32_t &k1)
{
    c[0] = (uint32_t)pid;
    c[1] = (uint32_t)sweep;
    c[2] = (uint32_t)(l + (m << 16));
    c[3] = (uint32_t)(sweep >> 32);
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
}

constexpr int MAX_CAND = 32;

// Uniform direction in DIM dimensions for (seed, sweep, particle, try l):
// candidate m is the Philox block of draw_block, mapped to the lattice point
// (w_a - 2^31) 2^-31 of [-1, 1)^DIM; the first candidate with 0 < |v|^2 <= 1
// is divided by its norm, and after MAX_CAND rejected candidates the
// direction is e_0.  cand_f64 evaluates one candidate in binary64 (exact or
// correctly rounded operations only; the direction is v / sqrt(|v|^2),
// correctly rounded).  cand_f32 is the same draw for the FP32 form, without
// binary64 arithmetic in the common case (binary64 runs at 1/64 of the
// binary32 rate on this GPU): coordinate a is the top 24 bits of the Philox
// word, v_a = ((w_a >> 8) - 2^23) 2^-23, the binary64 lattice point truncated
// by less than 2^-23, so |v|^2 in binary32 is within 1e-6 of the binary64
// value and the acceptance test is decided in binary32 outside a band of
// +-2e-6 around 1 (and 0) and by the binary64 computation inside it -- the
// accepted candidate is always the one the binary64 draw accepts.  Its
// direction is v rsqrt(|v|^2) in binary32, with |v|^2 summed by explicit
// fused multiply-adds (the same rounding wherever the compiler inlines it).

template <int DIM, bool COMPACT = false>
__device__ __forceinline__ bool cand_f64(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, uint64_t m,
                                         double v[3], double &s)
{
    uint32_t c[4], k0, k1;
    draw_block(seed, sweep, pid, l, m, c, k0, k1);
    philox4x32<COMPACT>(c, k0, k1);
    v[2] = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) v[a] = __dmul_rn(__ll2double_rn((long long)c[a] - 2147483648LL), 0x1p-31);
    s = __dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1]));
    if (DIM == 3) s = __dadd_rn(s, __dmul_rn(v[2], v[2]));
    return s > 0.0 && s <= 1.0;
}

template <int DIM, bool COMPACT = false>
__device__ __forceinline__ bool cand_f32(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, uint64_t m,
                                         float v[3], float &s)
{
    uint32_t c[4], k0, k1;
    draw_block(seed, sweep, pid, l, m, c, k0, k1);
    philox4x32<COMPACT>(c, k0, k1);
    v[2] = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; a++) v[a] = (float)((int32_t)(c[a] >> 8) - (1 << 23)) * 0x1p-23f;
    s = __fmaf_rn(v[1], v[1], __fmul_rn(v[0], v[0]));
    if (DIM == 3) s = __fmaf_rn(v[2], v[2], s);
    if (s > 1.0f + 2e-6f) return false;
    if (s < 1.0f - 2e-6f && s > 2e-6f) return true;
    double vd[3];
#pragma unroll
    for (int a = 0; a < DIM; a++) vd[a] = __dmul_rn(__ll2double_rn((long long)c[a] - 2147483648LL), 0x1p-31);
    double sd = __dadd_rn(__dmul_rn(vd[0], vd[0]), __dmul_rn(vd[1], vd[1]));
    if (DIM == 3) sd = __dadd_rn(sd, __dmul_rn(vd[2], vd[2]));
    const bool ok = sd > 0.0 && sd <= 1.0;
    if (ok && !(s > 0.f)) s = (float)sd;
    return ok;
}

// Directions of trials l0 .. l0+7 of one particle, drawn by a whole warp:
// lane k evaluates candidate k % 4 of trial l0 + k / 4, a ballot picks for
// every trial its first accepted candidate (the draw's direction),
// and a trial whose four candidates are all rejected continues with
// candidates 4, 5, ... in its own lane.  Lane t (t < 8) returns the direction
// of trial l0 + t.  All lanes of the warp must call it.
template <int DIM, bool F32, typename DT>
__device__ __noinline__ void draw8(uint64_t seed, uint64_t sweep, uint64_t pid, int l0, DT u[3])
{
    const int lane = threadIdx.x & 31, t = lane >> 2, cidx = lane & 3;
    DT v[3], s;
    bool ok;
    if constexpr (F32) ok = cand_f32<DIM, true>(seed, sweep, pid, (uint64_t)(l0 + t), (uint64_t)cidx, v, s);
    else ok = cand_f64<DIM, true>(seed, sweep, pid, (uint64_t)(l0 + t), (uint64_t)cidx, v, s);
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    // normalise in the lane that holds the chosen candidate
    DT w[3] = {(DT)0, (DT)0, (DT)0};
    const unsigned mine = (bal >> (4 * t)) & 15u;
    const bool chosen = ok && (__ffs(mine) - 1) == cidx;
    if (chosen) {
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
    // lane t collects trial t from lane 4t + (first accepted candidate)
    const unsigned mt = lane < 8 ? (bal >> (4 * lane)) & 15u : 1u;
    const int src = 4 * (lane & 7) + (mt ? __ffs(mt) - 1 : 0);
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = __shfl_sync(0xffffffffu, w[a], src);
    if (lane < 8 && !mt) {
        // all four rejected (about 5% of 3D trials): continue in this lane
        u[0] = (DT)1;
        u[1] = (DT)0;
        u[2] = (DT)0;
        for (int m = 4; m < MAX_CAND; m++) {
            DT vv[3], ss;
            bool okk;
            if constexpr (F32) okk = cand_f32<DIM, true>(seed, sweep, pid, (uint64_t)(l0 + lane), (uint64_t)m, vv, ss);
            else okk = cand_f64<DIM, true>(seed, sweep, pid, (uint64_t)(l0 + lane), (uint64_t)m, vv, ss);
            if (okk) {
                if constexpr (F32) {
                    const float inv = rsqrtf(ss);
#pragma unroll
                    for (int a = 0; a < DIM; a++) u[a] = vv[a] * inv;
                } else {
                    const double nrm = __dsqrt_rn(ss);
#pragma unroll
                    for (int a = 0; a < DIM; a++) u[a] = __ddiv_rn(vv[a], nrm);
                }
                if (DIM == 2) u[2] = (DT)0;
                break;
            }
        }
    }
}

// Algorithm 4: "< 0" first, then ">= L".
__device__ __forceinline__ double wrap_d(double x, double L)
{
    if (x < 0.0) x = __dadd_rn(x, L);
    if (x >= L) x = __dsub_rn(x, L);
    return x;
}

// Algorithm 2: int(x / w), then ((c % n) + n) % n.
__device__ __forceinline__ int32_t cell_coord_d(double x, double w, int32_t n)
{
    long long c = __double2ll_rz(__ddiv_rn(x, w));
    long long nn = n;
    return (int32_t)(((c % nn) + nn) % nn);
}

// Algorithm 5 for one pair: minimum-image difference, then
// sqrt(dx^2 + dy^2 [+ dz^2]) <= Rq + Rt, in binary64.  Most pairs are decided
// from the squared distance against (Rq + Rt)^2 with a relative margin that
// covers every rounding of both sides; only pairs inside that band take the
// correctly rounded square root, so the outcome equals the literal test.
template <int DIM>
__device__ __forceinline__ bool collide_exact(const double q[3], double Rq, double tx, double ty,
                                              double tz, double Rt, const double L[3],
                                              const double halfL[3])
{
    double d0 = __dsub_rn(q[0], tx);
    if (d0 > halfL[0]) d0 = __dsub_rn(d0, L[0]);
    if (d0 < -halfL[0]) d0 = __dadd_rn(d0, L[0]);
    double d1 = __dsub_rn(q[1], ty);
    if (d1 > halfL[1]) d1 = __dsub_rn(d1, L[1]);
    if (d1 < -halfL[1]) d1 = __dadd_rn(d1, L[1]);
    double ss = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
    if (DIM == 3) {
        double d2 = __dsub_rn(q[2], tz);
        if (d2 > halfL[2]) d2 = __dsub_rn(d2, L[2]);
        if (d2 < -halfL[2]) d2 = __dadd_rn(d2, L[2]);
        ss = __dadd_rn(ss, __dmul_rn(d2, d2));
    }
    const double rs = __dadd_rn(Rq, Rt);
    const double b = __dmul_rn(rs, rs);
    // sqrt(ss) < rs for certain when ss <= b (1 - 2^-51); sqrt(ss) rounds
    // above rs for certain when ss >= b (1 + 2^-48).
    if (ss > __dmul_rn(b, 1.0 + 0x1p-48)) return false;
    if (ss <= __dmul_rn(b, 1.0 - 0x1p-51)) return true;
    return __dsqrt_rn(ss) <= rs;
}

// The same predicate with image particles instead of the minimum image
// (Section 2's other periodicity): per axis the image of t nearest to q,
// y = t + L or t - L (one rounding) when |q - t| exceeds half the box, then
// the plain difference q - y -- the arithmetic of the reference's image
// entries x_t + s L.
template <int DIM>
__device__ __forceinline__ bool collide_img(const double q[3], double Rq, double tx, double ty, double tz, double Rt,
                                            const double L[3], const double halfL[3])
{
    const double t[3] = {tx, ty, tz};
    double ss = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        double d = __dsub_rn(q[a], t[a]);
        if (d > halfL[a]) d = __dsub_rn(q[a], __dadd_rn(t[a], L[a]));
        else if (d < -halfL[a]) d = __dsub_rn(q[a], __dsub_rn(t[a], L[a]));
        ss = a == 0 ? __dmul_rn(d, d) : __dadd_rn(ss, __dmul_rn(d, d));
    }
    const double rs = __dadd_rn(Rq, Rt);
    const double b = __dmul_rn(rs, rs);
    if (ss > __dmul_rn(b, 1.0 + 0x1p-48)) return false;
    if (ss <= __dmul_rn(b, 1.0 - 0x1p-51)) return true;
    return __dsqrt_rn(ss) <= rs;
}

// Algorithm 5's pair test of the FP64 form under the RVE's periodicity.
template <int DIM>
__device__ __forceinline__ bool collide64(int images, const double q[3], double Rq, double tx, double ty, double tz,
                                          double Rt, const double L[3], const double halfL[3])
{
    return images ? collide_img<DIM>(q, Rq, tx, ty, tz, Rt, L, halfL)
                  : collide_exact<DIM>(q, Rq, tx, ty, tz, Rt, L, halfL);
}

// Gap S - (Rq + Rt) and the literal predicate, for certification.
template <int DIM>
__device__ __forceinline__ bool gap_exact(const double q[3], double Rq, const double t[3], double Rt,
                                          const double L[3], const double halfL[3], double *gap)
{
    double ss = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        double d = __dsub_rn(q[a], t[a]);
        if (d > halfL[a]) d = __dsub_rn(d, L[a]);
        if (d < -halfL[a]) d = __dadd_rn(d, L[a]);
        ss = a == 0 ? __dmul_rn(d, d) : __dadd_rn(ss, __dmul_rn(d, d));
    }
    const double S = __dsqrt_rn(ss);
    const double rs = __dadd_rn(Rq, Rt);
    *gap = __dsub_rn(S, rs);
    return S <= rs;
}

// gap_exact with image particles (the arithmetic of collide_img).
template <int DIM>
__device__ __forceinline__ bool gap_img(const double q[3], double Rq, const double t[3], double Rt, const double L[3],
                                        const double halfL[3], double *gap)
{
    double ss = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        double d = __dsub_rn(q[a], t[a]);
        if (d > halfL[a]) d = __dsub_rn(q[a], __dadd_rn(t[a], L[a]));
        else if (d < -halfL[a]) d = __dsub_rn(q[a], __dsub_rn(t[a], L[a]));
        ss = a == 0 ? __dmul_rn(d, d) : __dadd_rn(ss, __dmul_rn(d, d));
    }
    const double S = __dsqrt_rn(ss);
    const double rs = __dadd_rn(Rq, Rt);
    *gap = __dsub_rn(S, rs);
    return S <= rs;
}

template <int DIM>
__device__ __forceinline__ bool gap64(int images, const double q[3], double Rq, const double t[3], double Rt,
                                      const double L[3], const double halfL[3], double *gap)
{
    return images ? gap_img<DIM>(q, Rq, t, Rt, L, halfL, gap) : gap_exact<DIM>(q, Rq, t, Rt, L, halfL, gap);
}

// Grid of Algorithm 1 for scale lam: cellSize = 2.5 lam rmax + c_m,
// n = 3 max(1, int(L / (3 cellSize))), w = L / n.  Also the reach H of the
// neighbour search: cells within one of the home cell cover every possible
// partner of any trial move when 2 (lam rmax) + 2 c_m < w; otherwise two.
__device__ __forceinline__ void set_grid(RveDev *st, double lam)
{
    const double Rmax = __dmul_rn(lam, st->rmax);
    const double cs = __dadd_rn(__dmul_rn(2.5, Rmax), st->c_m);
    const double reach = __dadd_rn(__dmul_rn(2.0, Rmax), __dmul_rn(2.0, st->c_m));
    int32_t nc = 1, ns = 1;
    for (int a = 0; a < 3; a++) {
        if (a >= st->dim) {
            st->gn[a] = 1;
            st->gw[a] = st->L[a];
            st->H[a] = 0;
            st->sub[a] = 1;
            continue;
        }
        long long k = __double2ll_rz(__ddiv_rn(st->L[a], __dmul_rn(3.0, cs)));
        if (k < 1) k = 1;
        const int32_t n = (int32_t)(3 * k);
        const double w = __ddiv_rn(st->L[a], (double)n);
        st->gn[a] = n;
        st->gw[a] = w;
        int32_t H = reach < w * (1.0 - 1e-9) ? 1 : 2;
        if (H > (n - 1) / 2) H = (n - 1) / 2;
        st->H[a] = H;
        st->sub[a] = n / 3;
        nc *= n;
        ns *= n / 3;
    }
    st->ncells = nc;
    st->nsub = ns;
}

// Order-preserving map of a double onto an unsigned key (for atomicMin).
__device__ __forceinline__ unsigned long long dkey(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

}  // namespace srm
