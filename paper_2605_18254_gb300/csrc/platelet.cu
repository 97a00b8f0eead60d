// platelet.cu -- SRM for thin circular platelets (Section 3.3): spherodisk
// contact, the rotational migration move, and the binning, sweep and check
// kernels with the host control of Algorithm 1 for them.
//
// Centres, normals, draws and moves in binary64; the contact test in
// binary32 on the pair's relative geometry with a widened threshold (see
// collide).  This translation unit is compiled with --fmad=false: every
// multiply and add below is one IEEE operation in the order written
// (division and square root are correctly rounded), so the results equal
// the reference bit for bit.
//
// Layout in HBM: centres and normals as double4 (x, y, z, unused) in
// particle-id order, two copies each (P and the swollen copy Q of Algorithm
// 1); per sweep a cell list (cell of each platelet, cell starts, ids sorted
// by cell and by id inside a cell) and one completion stamp per cell.
//
// Sweep: one launch per sweep, cells from a work counter in canonical colour
// order, each waiting until the cells of lower colour within reach are
// stamped for this sweep (bounded polls), then moving its platelets one
// after the other in id order and releasing its stamp.  Two kernels with the
// same results: k_psweep_staged (a block per cell, the 27 cells around it in
// shared memory, eight trials decided at once; wherever that set holds every
// platelet a trial can touch) and k_psweep (a warp per cell: all lanes form
// the same trial, lanes 0..26 each scan one of the 27 cells around the
// trial's cell for platelets within bounding-sphere reach, all 32 lanes then
// decide the staged pairs, and a warp vote accepts the first trial without a
// collision).  The check (Algorithm 6) likewise: k_pcheck_staged or
// k_pcheck.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "runtime.h"
#include "srm_platelet.h"

namespace srm {
namespace plt {

constexpr int TOP = 3;                // first level evaluated: 8 intervals of the circle
constexpr int DEPTH = 20;             // finest level (binary32 still separates its midpoints)
constexpr int EVALS = 512;            // evaluations per level-3 arc (4096 per rim)
constexpr float SLACK = 0x1p-16f;     // threshold widening, in units of the disk radius
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ float dot3f(const float a[3], const float b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Orthonormal basis of the plane of the unit normal n: e1 = n x axis_k /
// |n x axis_k| with k the axis of smallest |n_k| (first on ties), e2 = n x e1.
__device__ __forceinline__ void basis(const float n[3], float e1[3], float e2[3])
{
    const float ax = fabsf(n[0]), ay = fabsf(n[1]), az = fabsf(n[2]);
    int k = 0;
    float m = ax;
    if (ay < m) {
        k = 1;
        m = ay;
    }
    if (az < m) k = 2;
    float c[3];
    if (k == 0) {
        c[0] = 0.0f;
        c[1] = n[2];
        c[2] = -n[1];
    } else if (k == 1) {
        c[0] = -n[2];
        c[1] = 0.0f;
        c[2] = n[0];
    } else {
        c[0] = n[1];
        c[1] = -n[0];
        c[2] = 0.0f;
    }
    const float r = sqrtf(dot3f(c, c));
    for (int a = 0; a < 3; a++) e1[a] = c[a] / r;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
}

// Height h of p above the disk's plane and excess e of its projected
// distance from the centre over the radius b (0 inside).
__device__ __forceinline__ void point_disk_he(const float p[3], const float cd[3], const float nd[3], float b,
                                              float &h, float &e)
{
    const float q[3] = {p[0] - cd[0], p[1] - cd[1], p[2] - cd[2]};
    const float hh = dot3f(q, nd);
    const float r[3] = {q[0] - hh * nd[0], q[1] - hh * nd[1], q[2] - hh * nd[2]};
    const float rr = dot3f(r, r);
    h = hh;
    e = rr <= b * b ? 0.0f : sqrtf(rr) - b;
}

// Is a point of the arc tau in [k0/2, (k0+1)/2) (one of the 8 arcs of level
// 3) of the circle (centre cc, basis e1 e2, radius a) within thr of the disk
// (cd, nd, b)?  sn: sine of the angle between the normals.  The circle is
// parametrised by tau in [0, 4): s = tau - 1 on the first half, ((1 - s^2)
// e1 + 2 s e2) / (1 + s^2), s = tau - 3 and the negated point on the second.
// Depth-first bisection, left half first: a midpoint with h^2 + e^2 <= thr^2
// is a collision; an interval whose lower bound max(0, |h| - V r sn)^2 +
// max(0, e - V r)^2 (V = a (2 - min s^2) >= 2 a / (1 + min s^2), the rim
// speed; r the half-width) exceeds thr^2 is dropped; an interval still open
// at level 20, or after 512 evaluations of the arc, counts as a collision.
// Binary32 throughout; the geometry is passed by value (registers).
__device__ __noinline__ bool arc_near_disk(const float3 cc3, const float3 e13, const float3 e23, float a,
                                           const float3 cd3, const float3 nd3, float b, float sn, float thr, int k0)
{
    const float cc[3] = {cc3.x, cc3.y, cc3.z}, e1[3] = {e13.x, e13.y, e13.z}, e2[3] = {e23.x, e23.y, e23.z};
    const float cd[3] = {cd3.x, cd3.y, cd3.z}, nd[3] = {nd3.x, nd3.y, nd3.z};
    int d = TOP, ne = 0;
    int k = k0;
    const float thr2 = thr * thr;
    for (;;) {
        const float w = __int_as_float((127 + 2 - d) << 23);  // 4 / 2^d
        const float lo = (float)k * w;
        const float tau = lo + 0.5f * w;
        const bool first = tau < 2.0f;
        const float s = first ? tau - 1.0f : tau - 3.0f;
        const float s2 = s * s;
        const float inv = 1.0f / (1.0f + s2);
        const float C = (1.0f - s2) * inv, S = (2.0f * s) * inv;
        const float sa = first ? a : -a;
        float p[3];
        for (int j = 0; j < 3; j++) p[j] = cc[j] + sa * (C * e1[j] + S * e2[j]);
        float h, e;
        point_disk_he(p, cd, nd, b, h, e);
        ne++;
        if (h * h + e * e <= thr2) return true;
        const float off = lo < 2.0f ? 1.0f : 3.0f;
        const float sl = lo - off, sr = (lo + w) - off;
        const float m2 = (sl <= 0.0f && sr >= 0.0f) ? 0.0f : (sl * sl < sr * sr ? sl * sl : sr * sr);
        const float r = (a * (2.0f - m2)) * (0.5f * w);
        float hl = fabsf(h) - r * sn, el = e - r;
        if (hl < 0.0f) hl = 0.0f;
        if (el < 0.0f) el = 0.0f;
        if (!(hl * hl + el * el > thr2)) {
            if (d == DEPTH || ne >= EVALS) return true;
            d++;
            k = 2 * k;
            continue;
        }
        while (d > TOP && (k & 1)) {
            k >>= 1;
            d--;
        }
        if (d == TOP) return false;
        k++;
    }
}

// The whole rim: its 8 arcs, stopping at the first that reports contact.
__device__ __forceinline__ bool rim_near_disk(const float3 cc, const float3 e1, const float3 e2, float a,
                                              const float3 cd, const float3 nd, float b, float sn, float thr)
{
    for (int k0 = 0; k0 < 8; k0++)
        if (arc_near_disk(cc, e1, e2, a, cd, nd, b, sn, thr, k0)) return true;
    return false;
}

// The binary32 part of a pair test up to the rims: rounded centre
// difference d and normals, widened threshold, bounding spheres and the two
// slabs.  Returns false if these separate the pair, else fills the inputs of
// the rim tests.
struct PairGeom {
    float3 d, u, v;
    float af, sn, thr;
};

__device__ __forceinline__ bool pair_pretest(const double dj[3], const double ni[3], const double nj[3], double a,
                                             double t, PairGeom &g)
{
    const float d[3] = {(float)dj[0], (float)dj[1], (float)dj[2]};
    const float u[3] = {(float)ni[0], (float)ni[1], (float)ni[2]};
    const float v[3] = {(float)nj[0], (float)nj[1], (float)nj[2]};
    const float af = (float)a, tf = (float)t;
    const float thr = (tf + tf) + af * SLACK;
    const float reach = (af + af) + thr;
    if (dot3f(d, d) > reach * reach) return false;
    const float c = dot3f(u, v);
    float s2 = 1.0f - c * c;
    if (s2 < 0.0f) s2 = 0.0f;
    const float sn = sqrtf(s2);
    const float ext = af * sn;
    if (fabsf(dot3f(d, u)) - ext > thr) return false;
    if (fabsf(dot3f(d, v)) - ext > thr) return false;
    g.d = make_float3(d[0], d[1], d[2]);
    g.u = make_float3(u[0], u[1], u[2]);
    g.v = make_float3(v[0], v[1], v[2]);
    g.af = af;
    g.sn = sn;
    g.thr = thr;
    return true;
}

// Arc k0 of rim `which` (0: the rim of i against the disk of j; 1: the rim
// of j against the disk of i) of a pair that passed the pre-tests.
__device__ __forceinline__ bool pair_arc(const PairGeom &g, int which, int k0)
{
    const float n[3] = {which ? g.v.x : g.u.x, which ? g.v.y : g.u.y, which ? g.v.z : g.u.z};
    float e1[3], e2[3];
    basis(n, e1, e2);
    const float3 zero = make_float3(0.0f, 0.0f, 0.0f);
    const float3 b1 = make_float3(e1[0], e1[1], e1[2]), b2 = make_float3(e2[0], e2[1], e2[2]);
    if (which == 0) return arc_near_disk(zero, b1, b2, g.af, g.d, g.v, g.af, g.sn, g.thr, k0);
    return arc_near_disk(g.d, b1, b2, g.af, zero, g.u, g.af, g.sn, g.thr, k0);
}

// Contact of two platelets with disk radius a and half-thickness t: dj =
// centre of j minus centre of i (minimum image, binary64).  Evaluated in
// binary32 on the rounded dj, normals and sizes against the threshold
// 2 t + 2^-16 a (the widening exceeds every binary32 rounding of the test,
// so a pair at distance <= 2 t is always found): bounding spheres, the two
// slabs along the normals, then the rim of i against the disk of j and the
// rim of j against the disk of i (the OR of their 16 arcs).
__device__ __forceinline__ bool collide(const double dj[3], const double ni[3], const double nj[3], double a, double t)
{
    PairGeom g;
    if (!pair_pretest(dj, ni, nj, a, t, g)) return false;
    for (int which = 0; which < 2; which++)
        for (int k0 = 0; k0 < 8; k0++)
            if (pair_arc(g, which, k0)) return true;
    return false;
}

// Uniform direction of try l from stream tag (0: translation, the draw of
// the spheres; 0x80000000: rotation): candidate m is the Philox4x32-10 block
// at counter (pid, sweep lo, l + 2^16 m, sweep hi | tag), key = the seed,
// coordinates (w - 2^31) 2^-31; first candidate with 0 < |v|^2 <= 1,
// divided by sqrt(|v|^2); after 32 rejections the first axis.
__device__ __noinline__ void unit_dir(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, uint32_t tag,
                                      double u[3])
{
    for (int m = 0; m < MAX_CAND; m++) {
        uint32_t c[4], k0, k1;
        draw_block(seed, sweep, pid, l, (uint64_t)m, c, k0, k1);
        c[3] |= tag;
        philox4x32<true>(c, k0, k1);
        double v[3];
        for (int j = 0; j < 3; j++) v[j] = (double)((long long)c[j] - 2147483648LL) * 0x1p-31;
        double s = v[0] * v[0] + v[1] * v[1];
        s = s + v[2] * v[2];
        if (s > 0.0 && s <= 1.0) {
            const double nrm = sqrt(s);
            for (int j = 0; j < 3; j++) u[j] = v[j] / nrm;
            return;
        }
    }
    u[0] = 1.0;
    u[1] = 0.0;
    u[2] = 0.0;
}

struct PltDev {
    double L[3], halfL[3], w[3];
    int32_t n[3], H[3];
    int32_t N, ncells, N_l, wait_limit;
    int32_t images;  // periodicity by image platelets instead of the minimum image
    double a, t, c_m, c_r;
    uint64_t seed, sweep;
    uint32_t epoch;
    double4_32a *X, *U;
    int32_t *cell_of, *count, *start, *members;
    uint32_t *stamp;
    uint32_t *ctr;  // [0] work counter, [1] status
    unsigned long long *acc;  // [0] accepted moves, [1] colliding platelets, [2] unstaged cells
};

__device__ __forceinline__ int32_t wrapc(int32_t c, int32_t n)
{
    c %= n;
    return c < 0 ? c + n : c;
}

__device__ __forceinline__ int32_t cell_of_point(const PltDev &d, const double q[3], int32_t c[3])
{
    for (int j = 0; j < 3; j++) c[j] = cell_coord_d(q[j], d.w[j], d.n[j]);
    return c[0] + d.n[0] * (c[1] + d.n[1] * c[2]);
}

// Centre of platelet t minus q under the handle's periodicity: the minimum
// image of the difference, or (images) the difference to t's periodic image
// nearest to q, (x_t +- L) - q, with the image formed first.
__device__ __forceinline__ void min_image(const PltDev &d, const double4_32a &xt, const double q[3], double dj[3])
{
    const double v[3] = {xt.x, xt.y, xt.z};
    for (int j = 0; j < 3; j++) {
        double x = v[j] - q[j];
        if (d.images) {
            if (x > d.halfL[j]) x = (v[j] - d.L[j]) - q[j];
            else if (x < -d.halfL[j]) x = (v[j] + d.L[j]) - q[j];
        } else {
            if (x > d.halfL[j]) x -= d.L[j];
            if (x < -d.halfL[j]) x += d.L[j];
        }
        dj[j] = x;
    }
}

// Algorithm 2 on centres: cell of each platelet and the cell counts.
__global__ void k_pbin_count(PltDev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const double4_32a p = d.X[i];
    const double q[3] = {p.x, p.y, p.z};
    int32_t c[3];
    const int32_t cell = cell_of_point(d, q, c);
    d.cell_of[i] = cell;
    atomicAdd(&d.count[cell], 1);
}

// Exclusive scan of the counts into the cell starts (one block of 1024
// threads walking the cells), counts reset for the scatter.
__global__ void __launch_bounds__(1024) k_pscan(PltDev d)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < d.ncells; base += 1024) {
        const int i = base + threadIdx.x;
        const int32_t v = i < d.ncells ? d.count[i] : 0;
        int32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const int32_t excl = carry + (warp ? wsum[warp - 1] : 0) + x - v;
        if (i < d.ncells) {
            d.start[i] = excl;
            d.count[i] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) d.start[d.ncells] = carry;
}

__global__ void k_pscatter(PltDev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int32_t c = d.cell_of[i];
    d.members[d.start[c] + atomicAdd(&d.count[c], 1)] = i;
}

// Ids of each cell in ascending order (insertion sort; cells hold a few
// tens of platelets).
__global__ void k_psort(PltDev d)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.ncells) return;
    const int32_t b = d.start[c], e = d.start[c + 1];
    for (int32_t i = b + 1; i < e; i++) {
        const int32_t v = d.members[i];
        int32_t j = i - 1;
        while (j >= b && d.members[j] > v) {
            d.members[j + 1] = d.members[j];
            j--;
        }
        d.members[j + 1] = v;
    }
}

// Trial l of platelet pid from (x0, u0): centre x0 + c_m u wrapped (Alg 4),
// normal (u0 + c_r v) / |u0 + c_r v| (unchanged when c_r = 0).
__device__ __forceinline__ void trial(const PltDev &d, uint64_t pid, uint64_t l, const double x0[3],
                                      const double u0[3], double q[3], double u[3])
{
    double dir[3];
    unit_dir(d.seed, d.sweep, pid, l, 0u, dir);
    for (int j = 0; j < 3; j++) q[j] = wrap_d(x0[j] + d.c_m * dir[j], d.L[j]);
    if (d.c_r > 0.0) {
        double v[3], m[3];
        unit_dir(d.seed, d.sweep, pid, l, 0x80000000u, v);
        for (int j = 0; j < 3; j++) m[j] = u0[j] + d.c_r * v[j];
        const double r = sqrt(dot3(m, m));
        for (int j = 0; j < 3; j++) u[j] = m[j] / r;
    } else {
        for (int j = 0; j < 3; j++) u[j] = u0[j];
    }
}

// Waits (lanes in parallel) until every cell of lower colour within H of
// (cx, cy, cz) carries this sweep's stamp.  False if a wait gave up (the
// status word is then set) or another warp already failed.
__device__ bool wait_lower(const PltDev &d, int cx, int cy, int cz, int chi, int lane)
{
    const int sx = 2 * d.H[0] + 1, sy = 2 * d.H[1] + 1, sz = 2 * d.H[2] + 1;
    const int total = sx * sy * sz;
    bool ok = true;
    for (int o = lane; o < total && ok; o += 32) {
        const int ox = o % sx - d.H[0], oy = (o / sx) % sy - d.H[1], oz = o / (sx * sy) - d.H[2];
        if (ox == 0 && oy == 0 && oz == 0) continue;
        const int nx = wrapc(cx + ox, d.n[0]), ny = wrapc(cy + oy, d.n[1]), nz = wrapc(cz + oz, d.n[2]);
        const int nchi = nx % 3 + 3 * (ny % 3) + 9 * (nz % 3);
        if (nchi >= chi) continue;
        const uint32_t *st = &d.stamp[nx + d.n[0] * (ny + d.n[1] * nz)];
        int polls = 0;
        while (ld_relaxed(st) != d.epoch) {
            if (d.wait_limit < 0 || ++polls > d.wait_limit) {
                atomicExch(&d.ctr[1], (uint32_t)STATUS_WAIT_TIMEOUT);
                ok = false;
                break;
            }
            if ((polls & 255) == 0 && ld_relaxed(&d.ctr[1]) != 0u) {
                ok = false;
                break;
            }
            __nanosleep(polls < 1024 ? 64 : 1000);
        }
    }
    // relaxed loads that saw the release stores, then the fence: the
    // cells' writes are visible to this lane, and after the vote to the warp
    fence_acquire();
    return __all_sync(FULL, ok);
}

constexpr int SLOT = 16;   // candidates a lane stages per trial (more are tested in place)
constexpr int PAIRS = 64;  // pairs per trial queued for the rim tests (more are tested in place)

struct WarpScratch {
    int32_t slot[27 * SLOT];
    int32_t flat[27 * SLOT];
    PairGeom pair[PAIRS];
    int npair;
};

// Is the trial (q, u) of platelet pid clear of every platelet listed in the
// 27 cells around q's cell?  Three phases, each spread over the lanes:
// lanes 0..26 scan one cell each and stage the platelets within
// bounding-sphere reach; the staged candidates get the binary32 pre-tests
// (bounding spheres, slabs) and those not separated are queued; the queued
// pairs' 16 arcs each (2 rims x 8 first-level arcs) are bisected one per
// lane, stopping at the first contact.  Overflowing stages and queues are
// tested in place by the lane that holds them.  The answer is the OR of the
// same pair decisions as the reference, on every lane.
__device__ bool trial_collides(const PltDev &d, int32_t pid, const double q[3], const double u[3], int lane,
                               WarpScratch &ws)
{
    int cnt = 0;
    bool hit = false;
    // a superset of the pairs that pass the first pre-test (its threshold
    // is widened by 2^-16 a and rounded to binary32)
    const double reach = ((d.a + d.a) + (d.t + d.t)) * 1.001;
    const double reach2 = reach * reach;
    if (lane == 0) ws.npair = 0;
    if (lane < 27) {
        int32_t qc[3];
        cell_of_point(d, q, qc);
        const int nx = wrapc(qc[0] + lane % 3 - 1, d.n[0]);
        const int ny = wrapc(qc[1] + (lane / 3) % 3 - 1, d.n[1]);
        const int nz = wrapc(qc[2] + lane / 9 - 1, d.n[2]);
        const int nc = nx + d.n[0] * (ny + d.n[1] * nz);
        const int32_t e0 = d.start[nc + 1];
        for (int32_t j = d.start[nc]; j < e0; j++) {
            const int32_t tj = d.members[j];
            if (tj == pid) continue;
            const double4_32a xt = d.X[tj];
            double dj[3];
            min_image(d, xt, q, dj);
            if (dot3(dj, dj) > reach2) continue;
            if (cnt < SLOT) {
                ws.slot[lane * SLOT + cnt] = tj;
                cnt++;
            } else if (!hit) {
                const double4_32a ut = d.U[tj];
                const double nt[3] = {ut.x, ut.y, ut.z};
                hit = collide(dj, u, nt, d.a, d.t);
            }
        }
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    for (int i = 0; i < cnt; i++) ws.flat[incl - cnt + i] = ws.slot[lane * SLOT + i];
    __syncwarp();
    if (__any_sync(FULL, hit)) return true;
    // pre-tests, queueing the pairs that need their rims
    for (int i = lane; i < total && !hit; i += 32) {
        const int32_t tj = ws.flat[i];
        const double4_32a xt = d.X[tj], ut = d.U[tj];
        double dj[3];
        min_image(d, xt, q, dj);
        const double nt[3] = {ut.x, ut.y, ut.z};
        PairGeom g;
        if (!pair_pretest(dj, u, nt, d.a, d.t, g)) continue;
        const int slot = atomicAdd(&ws.npair, 1);
        if (slot < PAIRS) {
            ws.pair[slot] = g;
        } else {
            for (int which = 0; which < 2 && !hit; which++)
                for (int k0 = 0; k0 < 8 && !hit; k0++) hit = pair_arc(g, which, k0);
        }
    }
    __syncwarp();
    if (__any_sync(FULL, hit)) return true;
    const int np = ws.npair < PAIRS ? ws.npair : PAIRS;
    const int tasks = 16 * np;
    bool found = false;
    for (int r0 = 0; r0 < tasks && !found; r0 += 32) {
        const int tsk = r0 + lane;
        bool h = false;
        if (tsk < tasks) h = pair_arc(ws.pair[tsk >> 4], (tsk >> 3) & 1, tsk & 7);
        found = __any_sync(FULL, h);
    }
    __syncwarp();
    return found;
}

// One sweep of Algorithm 3 over the cells in canonical colour order.
__global__ void __launch_bounds__(128) k_psweep(PltDev d)
{
    __shared__ WarpScratch s_ws[4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int S0 = d.n[0] / 3, S1 = d.n[1] / 3, S2 = d.n[2] / 3;
    const int per = S0 * S1 * S2;
    const int total = 27 * per;
    for (;;) {
        int w = 0;
        if (lane == 0) w = (int)atomicAdd(&d.ctr[0], 1u);
        w = __shfl_sync(FULL, w, 0);
        if (w >= total) return;
        const int chi = w / per, r = w - chi * per;
        const int cx = 3 * (r % S0) + chi % 3, cy = 3 * ((r / S0) % S1) + (chi / 3) % 3;
        const int cz = 3 * (r / (S0 * S1)) + chi / 9;
        const int cell = cx + d.n[0] * (cy + d.n[1] * cz);
        if (!wait_lower(d, cx, cy, cz, chi, lane)) return;
        unsigned long long acc = 0;
        const int32_t k1 = d.start[cell + 1];
        for (int32_t k = d.start[cell]; k < k1; k++) {
            const int32_t pid = d.members[k];
            const double4_32a xp = d.X[pid], up = d.U[pid];
            const double x0[3] = {xp.x, xp.y, xp.z}, u0[3] = {up.x, up.y, up.z};
            for (int l = 0; l < d.N_l; l++) {
                double q[3], u[3];
                trial(d, (uint64_t)pid, (uint64_t)l, x0, u0, q, u);
                if (!trial_collides(d, pid, q, u, lane, s_ws[wib])) {
                    if (lane == 0) {
                        double4_32a nx4, nu4;
                        nx4.x = q[0];
                        nx4.y = q[1];
                        nx4.z = q[2];
                        nx4.w = 0.0;
                        nu4.x = u[0];
                        nu4.y = u[1];
                        nu4.z = u[2];
                        nu4.w = 0.0;
                        d.X[pid] = nx4;
                        d.U[pid] = nu4;
                    }
                    acc++;
                    break;
                }
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (acc) atomicAdd(&d.acc[0], acc);
            st_release(&d.stamp[cell], d.epoch);
        }
    }
}

// ---------------------------------------------------------------------------
// Sweep with the cell's neighbourhood in shared memory (grids whose stencil
// half-width is 1 on every axis).  One block of CW warps per cell: after the
// waits the block copies the platelets listed in the 27 cells around the
// home cell (centres and normals in binary64, plus binary32 offsets from the
// home cell's centre) to shared memory.  These hold every platelet a trial of
// a home platelet can touch: a home platelet moves at most c_m, a listed
// platelet has moved at most c_m from where it was binned, and a contact
// needs centres within 2 (a + t) (plus the 2^-16 a widening), all below the
// cell width when the half-width is 1.  Platelets beyond reach are never in
// contact (the first pre-test), so the OR over the staged set equals the OR
// over the 27 cells around the trial's own cell.
//
// The home platelets go one after the other in id order.  Warp k forms and
// tests trial l0 + k, so CW trials are decided at once; the move is the
// first clean trial in trial order, and a warp stops early once a trial of
// lower index is known to be clean (its own answer no longer matters).  A
// trial test: a binary32 scan of the staged offsets keeps the platelets
// within the pre-test's reach (with a relative margin of 2^-10, far above
// the rounding of the offsets), then the binary64 minimum-image difference,
// the binary32 pre-tests and the rim bisections as in trial_collides.  The
// mover's new state goes to global memory and to the staged copy; its
// binary32 offset is recomputed.  Thread 0 makes every global write of the
// cell.
// ---------------------------------------------------------------------------
constexpr int CW = 8;          // warps of a cell block (trials decided at once)
constexpr int CCAP = 1024;     // platelets of the 27 cells a block stages
constexpr int CSURV = 128;     // prefilter survivors a warp lists per trial (more are tested in place)
constexpr int CPAIRS = 32;     // pairs per warp queued for the rim tests (more are tested in place)

struct CellStage {
    double4_32a X[CCAP], U[CCAP];
    float4 F[CCAP];  // offset from the home cell's centre (minimum image), binary32
    int32_t id[CCAP];
    int16_t surv[CW][CSURV];
    PairGeom pair[CW][CPAIRS];
    int npair[CW];
    int cstart[28];
    int ccell[27];
    int best[2];  // lowest clean trial of the current round (two rounds alternate)
    int item, ok;
};

__device__ __forceinline__ float4 stage_offset(const PltDev &d, const double4_32a &x, const double c[3])
{
    double v[3] = {x.x - c[0], x.y - c[1], x.z - c[2]};
    for (int j = 0; j < 3; j++) {
        if (v[j] > d.halfL[j]) v[j] -= d.L[j];
        if (v[j] < -d.halfL[j]) v[j] += d.L[j];
    }
    return make_float4((float)v[0], (float)v[1], (float)v[2], 0.0f);
}

// The full pair decision for staged platelet i against trial (q, u).
__device__ __forceinline__ bool staged_pair(const PltDev &d, const CellStage &S, int i, const double q[3],
                                            const double u[3])
{
    double dj[3];
    min_image(d, S.X[i], q, dj);
    const double nt[3] = {S.U[i].x, S.U[i].y, S.U[i].z};
    return collide(dj, u, nt, d.a, d.t);
}

// Does trial (q, u) of platelet pid (trial index l) touch a staged platelet?
// Warp-collective; may return early (true) once a trial below l is clean.
__device__ bool trial_collides_staged(const PltDev &d, CellStage &S, int nst, int32_t pid, int l, const int *best,
                                      const double q[3], const double u[3], const double c[3], int warp, int lane)
{
    float qf[3];
    {
        const float4 o = stage_offset(d, double4_32a{q[0], q[1], q[2], 0.0}, c);
        qf[0] = o.x;
        qf[1] = o.y;
        qf[2] = o.z;
    }
    const float Lf[3] = {(float)d.L[0], (float)d.L[1], (float)d.L[2]};
    const float hLf[3] = {0.5f * Lf[0], 0.5f * Lf[1], 0.5f * Lf[2]};
    const float af = (float)d.a, tf = (float)d.t;
    const float rf = ((af + af) + ((tf + tf) + af * SLACK)) * (1.0f + 0x1p-10f);
    const float rf2 = rf * rf;
    bool hit = false;
    int n = 0;
    for (int i0 = 0; i0 < nst; i0 += 32) {
        const int i = i0 + lane;
        bool keep = false;
        if (i < nst && S.id[i] != pid) {
            const float4 f = S.F[i];
            float v[3] = {f.x - qf[0], f.y - qf[1], f.z - qf[2]};
            for (int j = 0; j < 3; j++) {
                if (v[j] > hLf[j]) v[j] -= Lf[j];
                if (v[j] < -hLf[j]) v[j] += Lf[j];
            }
            keep = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] <= rf2;
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        const int at = n + __popc(bal & ((1u << lane) - 1u));
        if (keep) {
            if (at < CSURV) S.surv[warp][at] = (int16_t)i;
            else if (!hit) hit = staged_pair(d, S, i, q, u);
        }
        n += __popc(bal);
    }
    if (lane == 0) S.npair[warp] = 0;
    __syncwarp();
    if (__any_sync(FULL, hit)) return true;
    if (n > CSURV) n = CSURV;
    for (int k = lane; k < n && !hit; k += 32) {
        const int i = S.surv[warp][k];
        double dj[3];
        min_image(d, S.X[i], q, dj);
        const double nt[3] = {S.U[i].x, S.U[i].y, S.U[i].z};
        PairGeom g;
        if (!pair_pretest(dj, u, nt, d.a, d.t, g)) continue;
        const int slot = atomicAdd(&S.npair[warp], 1);
        if (slot < CPAIRS) {
            S.pair[warp][slot] = g;
        } else {
            for (int which = 0; which < 2 && !hit; which++)
                for (int k0 = 0; k0 < 8 && !hit; k0++) hit = pair_arc(g, which, k0);
        }
    }
    __syncwarp();
    if (__any_sync(FULL, hit)) return true;
    const int np = S.npair[warp] < CPAIRS ? S.npair[warp] : CPAIRS;
    const int tasks = 16 * np;
    for (int r0 = 0; r0 < tasks; r0 += 32) {
        // a lower trial is clean: this answer is unused (one vote, so that
        // the warp leaves together)
        if (__any_sync(FULL, *(volatile const int *)best < l)) return true;
        const int tsk = r0 + lane;
        bool h = false;
        if (tsk < tasks) h = pair_arc(S.pair[warp][tsk >> 4], (tsk >> 3) & 1, tsk & 7);
        if (__any_sync(FULL, h)) return true;
    }
    return false;
}

__global__ void __launch_bounds__(CW * 32, 1) k_psweep_staged(PltDev d)
{
    extern __shared__ __align__(32) unsigned char psm[];
    CellStage &S = *reinterpret_cast<CellStage *>(psm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S0 = d.n[0] / 3, S1 = d.n[1] / 3, S2 = d.n[2] / 3;
    const int per = S0 * S1 * S2;
    const int total = 27 * per;
    int round = 0;
    if (tid == 0) S.best[0] = S.best[1] = d.N_l;
    for (;;) {
        if (tid == 0) S.item = (int)atomicAdd(&d.ctr[0], 1u);
        __syncthreads();
        const int w = S.item;
        if (w >= total) return;
        const int chi = w / per, r = w - chi * per;
        const int cx = 3 * (r % S0) + chi % 3, cy = 3 * ((r / S0) % S1) + (chi / 3) % 3;
        const int cz = 3 * (r / (S0 * S1)) + chi / 9;
        const int cell = cx + d.n[0] * (cy + d.n[1] * cz);
        if (warp == 0) {
            const bool ok = wait_lower(d, cx, cy, cz, chi, lane);
            if (lane == 0) S.ok = ok;
        }
        __syncthreads();
        if (!S.ok) return;
        // warp 0 synchronised with the producers' release stores; every
        // thread orders its own reads after them
        fence_acquire();
        if (tid < 27) {
            const int nx = wrapc(cx + tid % 3 - 1, d.n[0]), ny = wrapc(cy + (tid / 3) % 3 - 1, d.n[1]);
            const int nz = wrapc(cz + tid / 9 - 1, d.n[2]);
            const int nc = nx + d.n[0] * (ny + d.n[1] * nz);
            S.ccell[tid] = nc;
            S.cstart[tid + 1] = d.start[nc + 1] - d.start[nc];
        }
        __syncthreads();
        if (tid == 0) {
            S.cstart[0] = 0;
            for (int k = 1; k <= 27; k++) S.cstart[k] += S.cstart[k - 1];
        }
        __syncthreads();
        const int nst = S.cstart[27];
        const double c[3] = {(cx + 0.5) * d.w[0], (cy + 0.5) * d.w[1], (cz + 0.5) * d.w[2]};
        unsigned long long acc = 0;
        if (nst > CCAP) {
            // too many to stage: warp 0 moves the cell's platelets as k_psweep
            // does (global memory), the other warps wait
            if (tid == 0) atomicAdd(&d.acc[2], 1ull);
            if (warp == 0) {
                WarpScratch &ws = *reinterpret_cast<WarpScratch *>(psm);  // over the unused stage
                const int32_t k1 = d.start[cell + 1];
                for (int32_t k = d.start[cell]; k < k1; k++) {
                    const int32_t pid = d.members[k];
                    const double4_32a xp = d.X[pid], up = d.U[pid];
                    const double x0[3] = {xp.x, xp.y, xp.z}, u0[3] = {up.x, up.y, up.z};
                    for (int l = 0; l < d.N_l; l++) {
                        double q[3], u[3];
                        trial(d, (uint64_t)pid, (uint64_t)l, x0, u0, q, u);
                        if (!trial_collides(d, pid, q, u, lane, ws)) {
                            if (lane == 0) {
                                d.X[pid] = double4_32a{q[0], q[1], q[2], 0.0};
                                d.U[pid] = double4_32a{u[0], u[1], u[2], 0.0};
                            }
                            acc++;
                            break;
                        }
                    }
                    __syncwarp();
                }
            }
        } else {
            for (int i = tid; i < nst; i += CW * 32) {
                int k = 0;
                while (S.cstart[k + 1] <= i) k++;
                const int32_t id = d.members[d.start[S.ccell[k]] + (i - S.cstart[k])];
                const double4_32a x = d.X[id];
                S.X[i] = x;
                S.U[i] = d.U[id];
                S.F[i] = stage_offset(d, x, c);
                S.id[i] = id;
            }
            __syncthreads();
            // the home cell is stencil cell 13 (offsets 0, 0, 0); its
            // platelets are listed in ascending id
            const int hs = S.cstart[13], he = S.cstart[14];
            for (int m = hs; m < he; m++) {
                const int32_t pid = S.id[m];
                const double4_32a xp = S.X[m], up = S.U[m];
                const double x0[3] = {xp.x, xp.y, xp.z}, u0[3] = {up.x, up.y, up.z};
                for (int l0 = 0; l0 < d.N_l; l0 += CW) {
                    const int l = l0 + warp;
                    int *best = &S.best[round & 1];
                    double q[3], u[3];
                    bool clean = false;
                    if (l < d.N_l) {
                        trial(d, (uint64_t)pid, (uint64_t)l, x0, u0, q, u);
                        clean = !trial_collides_staged(d, S, nst, pid, l, best, q, u, c, warp, lane);
                        if (clean && lane == 0) atomicMin(best, l);
                    }
                    __syncthreads();
                    const int lb = *best;  // N_l: no clean trial this round
                    if (lb < d.N_l && lb == l && lane == 0) {
                        const double4_32a nx4{q[0], q[1], q[2], 0.0}, nu4{u[0], u[1], u[2], 0.0};
                        S.X[m] = nx4;
                        S.U[m] = nu4;
                        S.F[m] = stage_offset(d, nx4, c);
                    }
                    if (tid == 0) S.best[(round + 1) & 1] = d.N_l;
                    round++;
                    __syncthreads();
                    if (lb < d.N_l) {
                        // thread 0 makes every global write of the cell, so
                        // that its release of the cell's stamp publishes them
                        if (tid == 0) {
                            d.X[pid] = S.X[m];
                            d.U[pid] = S.U[m];
                        }
                        acc++;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (acc) atomicAdd(&d.acc[0], acc);
            st_release(&d.stamp[cell], d.epoch);
        }
    }
}

// Algorithm 6: does platelet i collide with any other platelet listed in
// the 27 cells around its cell?
__global__ void __launch_bounds__(128) k_pcheck(PltDev d, uint8_t *flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const double4_32a xp = d.X[i], up = d.U[i];
    const double q[3] = {xp.x, xp.y, xp.z}, u[3] = {up.x, up.y, up.z};
    int32_t c[3];
    cell_of_point(d, q, c);
    bool hit = false;
    for (int o = 0; o < 27 && !hit; o++) {
        const int nx = wrapc(c[0] + o % 3 - 1, d.n[0]), ny = wrapc(c[1] + (o / 3) % 3 - 1, d.n[1]);
        const int nz = wrapc(c[2] + o / 9 - 1, d.n[2]);
        const int nc = nx + d.n[0] * (ny + d.n[1] * nz);
        const int32_t je = d.start[nc + 1];
        for (int32_t j = d.start[nc]; j < je && !hit; j++) {
            const int32_t tj = d.members[j];
            if (tj == i) continue;
            const double4_32a xt = d.X[tj], ut = d.U[tj];
            double dj[3];
            min_image(d, xt, q, dj);
            const double nt[3] = {ut.x, ut.y, ut.z};
            hit = collide(dj, u, nt, d.a, d.t);
        }
    }
    if (flags) flags[i] = hit ? 1 : 0;
    if (hit) atomicAdd(&d.acc[1], 1ull);
}

// Algorithm 6 with a cell's neighbourhood in shared memory (where the sweep's
// block kernel applies: the 27 cells around a cell hold every platelet
// within contact reach of its platelets): a block of CW warps per cell (a
// static stride over the cells), the warps taking the home platelets in
// turn, each decided as a trial at the platelet's own place and normal
// (trial_collides_staged, never stopped early).  Cells whose 27 neighbours
// hold more than CCAP platelets are checked by warp 0 one thread per
// platelet, as k_pcheck does.
__global__ void __launch_bounds__(CW * 32, 1) k_pcheck_staged(PltDev d, uint8_t *flags)
{
    extern __shared__ __align__(32) unsigned char psm[];
    CellStage &S = *reinterpret_cast<CellStage *>(psm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) S.best[0] = 1 << 30;  // no early stop
    for (int cell = blockIdx.x; cell < d.ncells; cell += gridDim.x) {
        __syncthreads();
        const int cx = cell % d.n[0], cy = (cell / d.n[0]) % d.n[1], cz = cell / (d.n[0] * d.n[1]);
        if (d.start[cell + 1] == d.start[cell]) continue;  // the same for every thread
        if (tid < 27) {
            const int nx = wrapc(cx + tid % 3 - 1, d.n[0]), ny = wrapc(cy + (tid / 3) % 3 - 1, d.n[1]);
            const int nz = wrapc(cz + tid / 9 - 1, d.n[2]);
            const int nc = nx + d.n[0] * (ny + d.n[1] * nz);
            S.ccell[tid] = nc;
            S.cstart[tid + 1] = d.start[nc + 1] - d.start[nc];
        }
        __syncthreads();
        if (tid == 0) {
            S.cstart[0] = 0;
            for (int k = 1; k <= 27; k++) S.cstart[k] += S.cstart[k - 1];
        }
        __syncthreads();
        const int nst = S.cstart[27];
        unsigned long long hits = 0;
        if (nst > CCAP) {
            if (warp == 0) {
                const int32_t k1 = d.start[cell + 1];
                for (int32_t k = d.start[cell] + lane; k < k1; k += 32) {
                    const int32_t i = d.members[k];
                    const double4_32a xp = d.X[i], up = d.U[i];
                    const double q[3] = {xp.x, xp.y, xp.z}, u[3] = {up.x, up.y, up.z};
                    bool hit = false;
                    for (int o = 0; o < 27 && !hit; o++) {
                        const int32_t je = d.start[S.ccell[o] + 1];
                        for (int32_t j = d.start[S.ccell[o]]; j < je && !hit; j++) {
                            const int32_t tj = d.members[j];
                            if (tj == i) continue;
                            const double4_32a xt = d.X[tj], ut = d.U[tj];
                            double dj[3];
                            min_image(d, xt, q, dj);
                            const double nt[3] = {ut.x, ut.y, ut.z};
                            hit = collide(dj, u, nt, d.a, d.t);
                        }
                    }
                    if (flags) flags[i] = hit ? 1 : 0;
                    hits += hit ? 1 : 0;
                }
            }
        } else {
            const double c[3] = {(cx + 0.5) * d.w[0], (cy + 0.5) * d.w[1], (cz + 0.5) * d.w[2]};
            for (int i = tid; i < nst; i += CW * 32) {
                int k = 0;
                while (S.cstart[k + 1] <= i) k++;
                const int32_t id = d.members[d.start[S.ccell[k]] + (i - S.cstart[k])];
                const double4_32a x = d.X[id];
                S.X[i] = x;
                S.U[i] = d.U[id];
                S.F[i] = stage_offset(d, x, c);
                S.id[i] = id;
            }
            __syncthreads();
            const int hs = S.cstart[13], he = S.cstart[14];
            for (int m = hs + warp; m < he; m += CW) {
                const double q[3] = {S.X[m].x, S.X[m].y, S.X[m].z}, u[3] = {S.U[m].x, S.U[m].y, S.U[m].z};
                const bool hit = trial_collides_staged(d, S, nst, S.id[m], 0, &S.best[0], q, u, c, warp, lane);
                if (lane == 0) {
                    if (flags) flags[S.id[m]] = hit ? 1 : 0;
                    hits += hit ? 1 : 0;
                }
            }
        }
        hits = __reduce_add_sync(0xffffffffu, (unsigned)hits);
        if (lane == 0 && hits) atomicAdd(&d.acc[1], hits);
    }
}

__global__ void k_ppairs(const double *dj, const double *ni, const double *nj, long long m, double a, double t,
                         uint8_t *out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const double d3[3] = {dj[3 * k], dj[3 * k + 1], dj[3 * k + 2]};
    const double a3[3] = {ni[3 * k], ni[3 * k + 1], ni[3 * k + 2]};
    const double b3[3] = {nj[3 * k], nj[3 * k + 1], nj[3 * k + 2]};
    out[k] = collide(d3, a3, b3, a, t) ? 1 : 0;
}

}  // namespace plt
}  // namespace srm

using srm::plt::PltDev;

struct srm_plt {
    cudaStream_t s = nullptr;
    int64_t n = 0;
    double L[3] = {1.0, 1.0, 1.0};
    double a0 = 0.0, t0 = 0.0, lam = 1.0, lam_t = 1.0;
    uint64_t seed = 0, sweep = 0;
    srm_plt_params p{};
    int cur = 0;                        // P = copy cur, Q = copy 1 - cur
    double4_32a *X[2] = {nullptr, nullptr}, *U[2] = {nullptr, nullptr};
    int32_t *cell_of = nullptr, *count = nullptr, *start = nullptr, *members = nullptr;
    uint32_t *stamp = nullptr, *ctr = nullptr;
    unsigned long long *acc = nullptr;
    uint8_t *flags = nullptr;
    unsigned long long *pin = nullptr;  // pinned: [0] moves, [1] colliding, [2] status
    int64_t ncells_cap = 0;
    uint32_t epoch = 0;
    int64_t iters = 0, accepted = 0, shaken = 0, sweeps = 0, moves = 0;
    int64_t staged_sweeps = 0, warp_sweeps = 0;  // sweeps by kernel
};

namespace {

constexpr int WAIT_DEFAULT = 1 << 23;  // polls; after the first 1024 each sleeps about 1 us

void grid_of(const srm_plt *h, double lam, int32_t n[3], double w[3], int32_t H[3])
{
    const double cs = 2.5 * (lam * (h->a0 + h->t0)) + h->p.c_m;
    const double reach = 2.0 * (lam * (h->a0 + h->t0)) + 2.0 * h->p.c_m;
    for (int a = 0; a < 3; a++) {
        int64_t k = (int64_t)(h->L[a] / (3.0 * cs));
        if (k < 1) k = 1;
        n[a] = (int32_t)(3 * k);
        w[a] = h->L[a] / (double)n[a];
        int32_t Ha = reach < w[a] * (1.0 - 1e-9) ? 1 : 2;
        if (Ha > (n[a] - 1) / 2) Ha = (n[a] - 1) / 2;
        H[a] = Ha;
    }
}

srm_status check_params(const srm_plt_params &p)
{
    if (!(p.c_m > 0.0)) return fail(SRM_E_ARG, "c_m must be > 0");
    if (!(p.c_w >= 0.0)) return fail(SRM_E_ARG, "c_w must be >= 0");
    if (!(p.c_r >= 0.0 && p.c_r < 1.0)) return fail(SRM_E_ARG, "c_r must be in [0, 1)");
    if (p.N_k < 1 || p.N_l < 1 || p.N_l > 65535 || p.N_shake < 0)
        return fail(SRM_E_ARG, "N_k >= 1, N_l in 1..65535, N_shake >= 0");
    if (p.sweep_kernel != 0 && p.sweep_kernel != 1) return fail(SRM_E_ARG, "sweep_kernel must be 0 or 1");
    return SRM_OK;
}

srm_status check_box(const srm_plt *h, const srm_plt_params &p, double lam_t)
{
    const double cs = 2.5 * (lam_t * (h->a0 + h->t0)) + p.c_m;
    for (int a = 0; a < 3; a++)
        if (h->L[a] < 3.0 * cs) return fail(SRM_E_ARG, "box narrower than three cells of the final cell size");
    return SRM_OK;
}

template <typename T>
srm_status dalloc(srm_plt *h, T **p, size_t count)
{
    if (cudaMallocAsync((void **)p, sizeof(T) * (count ? count : 1), h->s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SRM_E_NOMEM, "device allocation failed");
    }
    return SRM_OK;
}

void dfree(srm_plt *h, void *p)
{
    if (p) cudaFreeAsync(p, h->s);
}

srm_status ensure_cells(srm_plt *h, int64_t ncells)
{
    if (ncells <= h->ncells_cap) return SRM_OK;
    if (ncells > (1LL << 30)) return fail(SRM_E_ARG, "cell grid too fine (more than 2^30 cells)");
    dfree(h, h->count);
    dfree(h, h->start);
    dfree(h, h->stamp);
    h->count = nullptr;
    h->start = nullptr;
    h->stamp = nullptr;
    srm_status st;
    if ((st = dalloc(h, &h->count, (size_t)ncells)) != SRM_OK) return st;
    if ((st = dalloc(h, &h->start, (size_t)ncells + 1)) != SRM_OK) return st;
    if ((st = dalloc(h, &h->stamp, (size_t)ncells)) != SRM_OK) return st;
    CK(cudaMemsetAsync(h->stamp, 0, sizeof(uint32_t) * (size_t)ncells, h->s));
    h->ncells_cap = ncells;
    return SRM_OK;
}

// Binning of copy c on the grid of scale lam_grid (Algorithm 2), radii at
// scale lam; fills d for the following sweep or check.
srm_status bin(srm_plt *h, int c, double lam, double lam_grid, PltDev &d)
{
    std::memset(&d, 0, sizeof(d));
    grid_of(h, lam_grid, d.n, d.w, d.H);
    const int64_t ncells = (int64_t)d.n[0] * d.n[1] * d.n[2];
    srm_status st = ensure_cells(h, ncells);
    if (st != SRM_OK) return st;
    for (int a = 0; a < 3; a++) {
        d.L[a] = h->L[a];
        d.halfL[a] = 0.5 * h->L[a];
    }
    d.N = (int32_t)h->n;
    d.ncells = (int32_t)ncells;
    d.N_l = h->p.N_l;
    d.wait_limit = h->p.wait_limit == 0 ? WAIT_DEFAULT : h->p.wait_limit;
    d.images = h->p.images ? 1 : 0;
    d.a = lam * h->a0;
    d.t = lam * h->t0;
    d.c_m = h->p.c_m;
    d.c_r = h->p.c_r;
    d.seed = h->seed;
    d.sweep = h->sweep;
    d.X = h->X[c];
    d.U = h->U[c];
    d.cell_of = h->cell_of;
    d.count = h->count;
    d.start = h->start;
    d.members = h->members;
    d.stamp = h->stamp;
    d.ctr = h->ctr;
    d.acc = h->acc;
    const int nb = (int)((h->n + 255) / 256);
    CK(cudaMemsetAsync(h->count, 0, sizeof(int32_t) * (size_t)ncells, h->s));
    srm::plt::k_pbin_count<<<nb, 256, 0, h->s>>>(d);
    srm::plt::k_pscan<<<1, 1024, 0, h->s>>>(d);
    srm::plt::k_pscatter<<<nb, 256, 0, h->s>>>(d);
    srm::plt::k_psort<<<(int)((ncells + 255) / 256), 256, 0, h->s>>>(d);
    CK(cudaGetLastError());
    return SRM_OK;
}

// The staged sweep holds every platelet a trial can touch when a contact
// (centres within 2 (a + t) + 2^-16 a, the kernel's widened reach) plus the
// two moves of at most c_m stays below the cell width on every axis (taken
// with the widening doubled).
bool staged_fits(const PltDev &d)
{
    const double need = (2.0 * (d.a + d.t) + d.a * 0x1p-15) + 2.0 * d.c_m;
    for (int a = 0; a < 3; a++)
        if (d.H[a] != 1 || !(need < d.w[a])) return false;
    return true;
}

int staged_blocks_per_sm()
{
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(srm::plt::k_psweep_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(srm::plt::CellStage));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srm::plt::k_psweep_staged, srm::plt::CW * 32,
                                                      sizeof(srm::plt::CellStage));
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

int staged_check_blocks_per_sm()
{
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(srm::plt::k_pcheck_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(srm::plt::CellStage));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srm::plt::k_pcheck_staged, srm::plt::CW * 32,
                                                      sizeof(srm::plt::CellStage));
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

// One sweep of Algorithm 3 on copy c at scale lam, binned on the grid of
// lam_grid; advances the sweep counter.
srm_status sweep_once(srm_plt *h, int c, double lam, double lam_grid)
{
    PltDev d;
    srm_status st = bin(h, c, lam, lam_grid, d);
    if (st != SRM_OK) return st;
    d.epoch = ++h->epoch;
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(uint32_t), h->s));  // work counter (the status word stays)
    if (h->p.sweep_kernel == 0 && staged_fits(d)) {
        h->staged_sweeps++;
        // every block resident at once (a block may wait for any other)
        const int per_sm = staged_blocks_per_sm();
        int sms = 0, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int64_t blocks = (int64_t)per_sm * sms;
        if (blocks > d.ncells) blocks = d.ncells;
        srm::plt::k_psweep_staged<<<(int)blocks, srm::plt::CW * 32, sizeof(srm::plt::CellStage), h->s>>>(d);
    } else {
        h->warp_sweeps++;
        int64_t blocks = ((int64_t)d.ncells + 3) / 4;
        if (blocks > 152 * 8) blocks = 152 * 8;
        srm::plt::k_psweep<<<(int)blocks, 128, 0, h->s>>>(d);
    }
    CK(cudaGetLastError());
    h->sweep++;
    h->sweeps++;
    return SRM_OK;
}

// Reads the counters (synchronises the stream); SRM_E_DEVICE_TIMEOUT if a
// sweep gave up waiting.
srm_status read_counters(srm_plt *h, unsigned long long &moves, unsigned long long &colliding)
{
    CK(cudaMemcpyAsync(h->pin, h->acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->pin + 2, h->ctr + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    moves = h->pin[0];
    colliding = h->pin[1];
    const uint32_t status = (uint32_t)(h->pin[2] & 0xffffffffull);
    if (status != 0u) return fail(SRM_E_DEVICE_TIMEOUT, "a platelet sweep gave up waiting for a neighbouring cell");
    return SRM_OK;
}

srm_status zero_counters(srm_plt *h)
{
    CK(cudaMemsetAsync(h->acc, 0, 2 * sizeof(unsigned long long), h->s));
    return SRM_OK;
}

// Algorithm 6 on copy c at scale lam (grid of lam_grid): colliding count.
srm_status check_copy(srm_plt *h, int c, double lam, double lam_grid, uint8_t *flags_dev, int64_t &count,
                      unsigned long long &moves)
{
    PltDev d;
    srm_status st = bin(h, c, lam, lam_grid, d);
    if (st != SRM_OK) return st;
    CK(cudaMemsetAsync(h->acc + 1, 0, sizeof(unsigned long long), h->s));
    if (h->p.sweep_kernel == 0 && staged_fits(d)) {
        const int per_sm = staged_check_blocks_per_sm();
        int sms = 0, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int64_t blocks = (int64_t)per_sm * sms;
        if (blocks > d.ncells) blocks = d.ncells;
        srm::plt::k_pcheck_staged<<<(int)blocks, srm::plt::CW * 32, sizeof(srm::plt::CellStage), h->s>>>(d,
                                                                                                         flags_dev);
    } else {
        srm::plt::k_pcheck<<<(int)((h->n + 127) / 128), 128, 0, h->s>>>(d, flags_dev);
    }
    CK(cudaGetLastError());
    unsigned long long col = 0;
    if ((st = read_counters(h, moves, col)) != SRM_OK) return st;
    count = (int64_t)col;
    return SRM_OK;
}

double density(const srm_plt *h)
{
    const double D = 2.0 * (h->lam * (h->a0 + h->t0));
    return (double)h->n * (D * D * D) / (h->L[0] * h->L[1] * h->L[2]);
}

}  // namespace

extern "C" {

void srm_plt_params_default(srm_plt_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->c_w = 0.01;
    p->N_k = 10;
    p->N_l = 10;
    p->N_shake = 10;
}

srm_status srm_plt_lambda_for_density(const double box[3], int64_t n, double a0, double t0, double rho,
                                      double *lambda)
{
    if (!box || !lambda) return fail(SRM_E_ARG, "null argument");
    if (n < 1 || !(a0 > 0.0) || !(t0 > 0.0) || !(rho > 0.0)) return fail(SRM_E_ARG, "n, sizes and rho must be > 0");
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0.0)) return fail(SRM_E_ARG, "box lengths must be > 0");
    const double V = box[0] * box[1] * box[2];
    *lambda = std::cbrt(rho * V / (double)n) / (2.0 * (a0 + t0));
    return SRM_OK;
}

srm_status srm_plt_init(srm_plt **out, const double box[3], int64_t n, double a0, double t0, const double *x,
                        const double *u, double lambda0, double lambda_t, uint64_t seed, const srm_plt_params *pin,
                        void *cuda_stream)
{
    if (!out || !box || !x || !u) return fail(SRM_E_ARG, "null argument");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL - 1) return fail(SRM_E_ARG, "n must be in [1, 2^31 - 1)");
    if (!(a0 > 0.0) || !(t0 > 0.0)) return fail(SRM_E_ARG, "base sizes must be > 0");
    if (!(lambda0 > 0.0) || !(lambda_t >= lambda0)) return fail(SRM_E_ARG, "need 0 < lambda0 <= lambda_t");
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0.0)) return fail(SRM_E_ARG, "box lengths must be > 0");
    srm_plt_params p;
    if (pin) p = *pin;
    else srm_plt_params_default(&p);
    srm_status st = check_params(p);
    if (st != SRM_OK) return st;
    srm_plt *h = new (std::nothrow) srm_plt();
    if (!h) return fail(SRM_E_NOMEM, "host allocation failed");
    h->s = (cudaStream_t)cuda_stream;
    h->n = n;
    for (int a = 0; a < 3; a++) h->L[a] = box[a];
    h->a0 = a0;
    h->t0 = t0;
    h->lam = lambda0;
    h->lam_t = lambda_t;
    h->seed = seed;
    h->sweep = p.sweep0;
    h->p = p;
    if ((st = check_box(h, p, lambda_t)) != SRM_OK) {
        delete h;
        return st;
    }
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++)
            if (!(x[3 * i + a] >= 0.0 && x[3 * i + a] < box[a])) {
                delete h;
                return fail(SRM_E_ARG, "centres must lie in [0, L)");
            }
    const size_t nn = (size_t)n;
    if ((st = dalloc(h, &h->X[0], nn)) != SRM_OK || (st = dalloc(h, &h->X[1], nn)) != SRM_OK ||
        (st = dalloc(h, &h->U[0], nn)) != SRM_OK || (st = dalloc(h, &h->U[1], nn)) != SRM_OK ||
        (st = dalloc(h, &h->cell_of, nn)) != SRM_OK || (st = dalloc(h, &h->members, nn)) != SRM_OK ||
        (st = dalloc(h, &h->flags, nn)) != SRM_OK || (st = dalloc(h, &h->ctr, 2)) != SRM_OK ||
        (st = dalloc(h, &h->acc, 3)) != SRM_OK) {
        srm_plt_destroy(h);
        return st;
    }
    if (cudaMallocHost((void **)&h->pin, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        h->pin = nullptr;
        srm_plt_destroy(h);
        return fail(SRM_E_NOMEM, "pinned allocation failed");
    }
    std::memset(h->pin, 0, 4 * sizeof(unsigned long long));
    std::vector<double> hx(4 * nn), hu(4 * nn);
    for (size_t i = 0; i < nn; i++)
        for (int a = 0; a < 3; a++) {
            hx[4 * i + a] = x[3 * i + a];
            hu[4 * i + a] = u[3 * i + a];
        }
    cudaError_t e = cudaMemcpyAsync(h->X[0], hx.data(), sizeof(double) * 4 * nn, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->U[0], hu.data(), sizeof(double) * 4 * nn, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ctr, 0, 2 * sizeof(uint32_t), h->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, 3 * sizeof(unsigned long long), h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);  // host staging buffers go out of scope
    if (e != cudaSuccess) {
        srm_plt_destroy(h);
        return fail(SRM_E_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    *out = h;
    return SRM_OK;
}

srm_status srm_plt_set_params(srm_plt *h, const srm_plt_params *p)
{
    if (!h || !p) return fail(SRM_E_ARG, "null argument");
    srm_status st = check_params(*p);
    if (st != SRM_OK) return st;
    if ((st = check_box(h, *p, h->lam_t)) != SRM_OK) return st;
    const uint64_t keep = h->sweep;
    h->p = *p;
    h->p.sweep0 = keep;
    return SRM_OK;
}

srm_status srm_plt_step(srm_plt *h, srm_plt_step_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    srm_plt_step_info info;
    std::memset(&info, 0, sizeof(info));
    srm_status st;
    if (h->lam >= h->lam_t) {
        info.result = 2;
    } else {
        h->iters++;
        double lam_q = h->lam * (1.0 + h->p.c_w);
        if (lam_q > h->lam_t) lam_q = h->lam_t;
        const int P = h->cur, Q = 1 - h->cur;
        const size_t bytes = sizeof(double4_32a) * (size_t)h->n;
        CK(cudaMemcpyAsync(h->X[Q], h->X[P], bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->U[Q], h->U[P], bytes, cudaMemcpyDeviceToDevice, h->s));
        if ((st = zero_counters(h)) != SRM_OK) return st;
        int64_t cnt = -1;
        unsigned long long mv = 0;
        int k;
        for (k = 1; k <= h->p.N_k; k++) {
            if ((st = sweep_once(h, Q, lam_q, lam_q)) != SRM_OK) return st;
            if ((st = check_copy(h, Q, lam_q, lam_q, nullptr, cnt, mv)) != SRM_OK) return st;
            if (cnt == 0) break;
        }
        const bool acc = cnt == 0;
        info.k_sweeps = acc ? k : h->p.N_k;
        info.colliding = cnt;
        if (acc) {
            h->cur = Q;
            h->lam = lam_q;
            h->accepted++;
            info.result = 1;
        } else {
            for (int j = 0; j < h->p.N_shake; j++)
                if ((st = sweep_once(h, P, h->lam, lam_q)) != SRM_OK) return st;
            unsigned long long col = 0;
            if ((st = read_counters(h, mv, col)) != SRM_OK) return st;
            h->shaken++;
            info.result = 0;
            info.shake_sweeps = h->p.N_shake;
        }
        info.moves = (int64_t)mv;
        h->moves += (int64_t)mv;
    }
    info.lambda = h->lam;
    info.rho = density(h);
    info.sweep = h->sweep;
    if (out) *out = info;
    return SRM_OK;
}

srm_status srm_plt_run_to_target(srm_plt *h, int64_t max_iters, srm_plt_run_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    srm_plt_run_info r;
    std::memset(&r, 0, sizeof(r));
    const int64_t it0 = h->iters, acc0 = h->accepted, sh0 = h->shaken, sw0 = h->sweeps, mv0 = h->moves;
    int64_t it = 0;
    srm_status st = SRM_OK;
    while (h->lam < h->lam_t && (max_iters <= 0 || it < max_iters)) {
        if ((st = srm_plt_step(h, nullptr)) != SRM_OK) break;
        it++;
    }
    r.iterations = h->iters - it0;
    r.accepted = h->accepted - acc0;
    r.shaken = h->shaken - sh0;
    r.sweeps = h->sweeps - sw0;
    r.moves = h->moves - mv0;
    r.lambda = h->lam;
    r.rho = density(h);
    r.converged = h->lam >= h->lam_t ? 1 : 0;
    if (out) *out = r;
    if (st != SRM_OK) return st;
    return r.converged ? SRM_OK : fail(SRM_E_NOT_CONVERGED, "iteration cap reached before the target scale");
}

srm_status srm_plt_sweeps(srm_plt *h, int32_t count, int64_t *accepted)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    if (count < 0) return fail(SRM_E_ARG, "count must be >= 0");
    srm_status st = zero_counters(h);
    if (st != SRM_OK) return st;
    for (int32_t i = 0; i < count; i++)
        if ((st = sweep_once(h, h->cur, h->lam, h->lam)) != SRM_OK) return st;
    unsigned long long mv = 0, col = 0;
    if ((st = read_counters(h, mv, col)) != SRM_OK) return st;
    h->moves += (int64_t)mv;
    if (accepted) *accepted = (int64_t)mv;
    return SRM_OK;
}

srm_status srm_plt_check(srm_plt *h, int64_t *colliding, uint8_t *flags)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    int64_t cnt = 0;
    unsigned long long mv = 0;
    srm_status st = check_copy(h, h->cur, h->lam, h->lam, flags ? h->flags : nullptr, cnt, mv);
    if (st != SRM_OK) return st;
    if (flags) {
        CK(cudaMemcpyAsync(flags, h->flags, (size_t)h->n, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    if (colliding) *colliding = cnt;
    return SRM_OK;
}

srm_status srm_plt_state(srm_plt *h, double *x, double *u, double *lambda, double *rho, uint64_t *sweep)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    const size_t nn = (size_t)h->n;
    if (x || u) {
        std::vector<double> hx(4 * nn), hu(4 * nn);
        CK(cudaMemcpyAsync(hx.data(), h->X[h->cur], sizeof(double) * 4 * nn, cudaMemcpyDeviceToHost, h->s));
        CK(cudaMemcpyAsync(hu.data(), h->U[h->cur], sizeof(double) * 4 * nn, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        for (size_t i = 0; i < nn; i++)
            for (int a = 0; a < 3; a++) {
                if (x) x[3 * i + a] = hx[4 * i + a];
                if (u) u[3 * i + a] = hu[4 * i + a];
            }
    }
    if (lambda) *lambda = h->lam;
    if (rho) *rho = density(h);
    if (sweep) *sweep = h->sweep;
    return SRM_OK;
}

srm_status srm_plt_collide_pairs(const double *dj, const double *ni, const double *nj, int64_t m, double a,
                                 double t, uint8_t *out, void *cuda_stream)
{
    if (m < 0 || m > 0x7fffffffLL || !(a > 0.0) || !(t > 0.0))
        return fail(SRM_E_ARG, "0 <= m < 2^31, a > 0, t > 0");
    if (m == 0) return SRM_OK;
    if (!dj || !ni || !nj || !out) return fail(SRM_E_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t vb = sizeof(double) * 3 * (size_t)m;
    double *d = nullptr;
    uint8_t *o = nullptr;
    if (cudaMallocAsync((void **)&d, 3 * vb, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(SRM_E_NOMEM, "device allocation failed");
    }
    if (cudaMallocAsync((void **)&o, (size_t)m, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(d, s);
        return fail(SRM_E_NOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(d, dj, vb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 3 * m, ni, vb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 6 * m, nj, vb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        srm::plt::k_ppairs<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(d, d + 3 * m, d + 6 * m, (long long)m, a, t, o);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, o, (size_t)m, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    cudaFreeAsync(o, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SRM_E_CUDA, std::string("pair decisions: ") + cudaGetErrorString(e));
    return SRM_OK;
}

srm_status srm_plt_sweep_stats(srm_plt *h, int64_t out[3])
{
    if (!h || !out) return fail(SRM_E_ARG, "null argument");
    unsigned long long unstaged = 0;
    CK(cudaMemcpyAsync(&unstaged, h->acc + 2, sizeof(unstaged), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    out[0] = h->staged_sweeps;
    out[1] = h->warp_sweeps;
    out[2] = (int64_t)unstaged;
    return SRM_OK;
}

void srm_plt_destroy(srm_plt *h)
{
    if (!h) return;
    void *bufs[] = {h->X[0], h->X[1], h->U[0], h->U[1], h->cell_of, h->count, h->start,
                    h->members, h->stamp, h->ctr, h->acc, h->flags};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, h->s);
    cudaStreamSynchronize(h->s);
    if (h->pin) cudaFreeHost(h->pin);
    delete h;
}

}  // extern "C"
