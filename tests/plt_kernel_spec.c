/*
 * plt_kernel_spec.c -- kernel specification, TEST INFRASTRUCTURE ONLY.
 *
 * The platelet contact decision exactly as the CUDA kernel evaluates it, in
 * plain C, so that whole GPU sweeps can be compared bit for bit with the
 * reference's sweep run on this predicate.  It is not the reference: the
 * reference decides contact in binary64 (oracle/srm_platelet.c), and the
 * tests check this decision against it one-sidedly (every binary64 contact
 * is a contact here; a contact found only here is within the widening of
 * touching).
 *
 * What it computes (the collision routine of Section 3.3, the criterion
 * being disk-to-disk distance <= t_i + t_j): a binary32 evaluation on the
 * pair's relative geometry (centre difference formed in binary64 under the
 * minimum image, then rounded, like the normals and sizes), against the
 * threshold 2 t + 2^-16 a -- a widening larger than the binary32 rounding of
 * every quantity of the test, so that every true contact is found.  Exact
 * separations come first (bounding spheres, slabs along both normals); then
 * each rim is tested against the other disk by bisection over a rational
 * parametrisation of the circle, tau in [0, 4): s = tau - 1 gives the half
 * circle ((1 - s^2) e1 + 2 s e2) / (1 + s^2), s = tau - 3 the opposite half.
 * Over an interval of half-width r the rim point moves at most V r with
 * V = a (2 - s_min^2), so its height above the other plane changes at most
 * V r sin(theta) and its in-plane excess at most V r: a certified lower
 * bound.  Each of a rim's 8 first-level arcs is bisected on its own (the
 * kernel spreads them over lanes) and counts as contact when still
 * undecided at level 20 or after 512 evaluations (a near-contact the
 * bisection cannot resolve; spec_plt_collide32_reason tells those apart).
 * Built with
 * gcc -O2 -ffp-contract=off, like the kernel's --fmad=false.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define PLT_TOP 3        /* first level evaluated: 8 intervals of the circle */
#define PLT_DEPTH 20     /* finest level (binary32 still separates its midpoints) */
#define PLT_EVALS 512    /* evaluations per level-3 interval (4096 per rim) */
#define PLT_SLACK 0x1p-16f /* threshold widening, in units of the disk radius */

static float dot3f(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Orthonormal basis (e1, e2) of the plane of the unit normal n: e1 is n
 * crossed with the coordinate axis of smallest |n_k| (the first such axis),
 * normalised; e2 = n x e1. */
static void basis_f(const float n[3], float e1[3], float e2[3])
{
    float ax = fabsf(n[0]), ay = fabsf(n[1]), az = fabsf(n[2]);
    int k = 0;
    float m = ax;
    if (ay < m) {
        k = 1;
        m = ay;
    }
    if (az < m) k = 2;
    float c[3];
    if (k == 0) {
        c[0] = 0.0f; c[1] = n[2]; c[2] = -n[1];
    } else if (k == 1) {
        c[0] = -n[2]; c[1] = 0.0f; c[2] = n[0];
    } else {
        c[0] = n[1]; c[1] = -n[0]; c[2] = 0.0f;
    }
    float r = sqrtf(dot3f(c, c));
    for (int a = 0; a < 3; a++) e1[a] = c[a] / r;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
}

/* Point p against the disk of centre cd, unit normal nd, radius b: h =
 * height above the plane, e = distance of the projection from cd minus b,
 * or 0 when the projection lies in the disk. */
static void point_disk_he(const float p[3], const float cd[3], const float nd[3], float b, float *h, float *e)
{
    float q[3] = {p[0] - cd[0], p[1] - cd[1], p[2] - cd[2]};
    float hh = dot3f(q, nd);
    float r[3] = {q[0] - hh * nd[0], q[1] - hh * nd[1], q[2] - hh * nd[2]};
    float rr = dot3f(r, r);
    *h = hh;
    *e = rr <= b * b ? 0.0f : sqrtf(rr) - b;
}

/* Point of the circle (centre cc, basis e1 e2, radius a) at parameter tau in
 * [0, 4): tau < 2 gives s = tau - 1 and the half circle
 * ((1 - s^2) e1 + 2 s e2) / (1 + s^2), tau >= 2 gives s = tau - 3 and the
 * opposite half (the same point negated). */
static void rim_point(const float cc[3], const float e1[3], const float e2[3], float a, float tau, float p[3])
{
    int first = tau < 2.0f;
    float s = first ? tau - 1.0f : tau - 3.0f;
    float s2 = s * s;
    float inv = 1.0f / (1.0f + s2);
    float C = (1.0f - s2) * inv, S = (2.0f * s) * inv;
    float sa = first ? a : -a;
    for (int k = 0; k < 3; k++) p[k] = cc[k] + sa * (C * e1[k] + S * e2[k]);
}

/* Is some point of the arc tau in [k0/2, (k0+1)/2) (one of the 8 intervals
 * of level 3) of the circle (cc, e1, e2, a) within thr of the disk (cd, nd,
 * b)?  sn = sine of the angle between the two normals.  Depth-first
 * bisection, intervals [k w, (k+1) w) with w = 4 / 2^d, left half first.
 * Returns 1 (yes), 2 (undecided at level 20 or after 512 evaluations,
 * counted as contact) or 0;
 * *evals receives the number of midpoints evaluated.  The 8 intervals are
 * independent, so the answer for the whole rim is their OR in any order. */
static int arc_near_disk_f(const float cc[3], const float e1[3], const float e2[3], float a, const float cd[3],
                           const float nd[3], float b, float sn, float thr, int k0, int *evals)
{
    int d = PLT_TOP, ne = 0;
    int64_t k = k0;
    float thr2 = thr * thr;
    for (;;) {
        float w = ldexpf(4.0f, -d);
        float lo = (float)k * w;
        float p[3];
        rim_point(cc, e1, e2, a, lo + 0.5f * w, p);
        float h, e;
        point_disk_he(p, cd, nd, b, &h, &e);
        ne++;
        if (h * h + e * e <= thr2) {
            if (evals) *evals = ne;
            return 1;
        }
        float off = lo < 2.0f ? 1.0f : 3.0f;
        float sl = lo - off, sr = (lo + w) - off;
        float m2 = (sl <= 0.0f && sr >= 0.0f) ? 0.0f : (sl * sl < sr * sr ? sl * sl : sr * sr);
        float r = (a * (2.0f - m2)) * (0.5f * w);
        float hl = fabsf(h) - r * sn, el = e - r;
        if (hl < 0.0f) hl = 0.0f;
        if (el < 0.0f) el = 0.0f;
        if (!(hl * hl + el * el > thr2)) {
            if (d == PLT_DEPTH || ne >= PLT_EVALS) {
                if (evals) *evals = ne;
                return 2; /* undecided: counted as contact */
            }
            d++;
            k = 2 * k;
            continue;
        }
        while (d > PLT_TOP && (k & 1)) {
            k >>= 1;
            d--;
        }
        if (d == PLT_TOP) {
            if (evals) *evals = ne;
            return 0;
        }
        k++;
    }
}

/* The whole rim: the 8 level-3 arcs in order, stopping at the first that
 * reports contact; *evals receives the evaluations of the arcs visited. */
static int rim_near_disk_f(const float cc[3], const float e1[3], const float e2[3], float a, const float cd[3],
                           const float nd[3], float b, float sn, float thr, int *evals)
{
    int total = 0;
    for (int k0 = 0; k0 < 8; k0++) {
        int ne = 0;
        int r = arc_near_disk_f(cc, e1, e2, a, cd, nd, b, sn, thr, k0, &ne);
        total += ne;
        if (r) {
            if (evals) *evals = total;
            return 1;
        }
    }
    if (evals) *evals = total;
    return 0;
}

/* Do the spherodisks i and j (disk radius a, half-thickness t each) collide?
 * dj = centre of j minus centre of i (minimum image, binary64); ni, nj unit
 * normals.  The test runs in binary32 on dj, ni, nj, a and t rounded to
 * binary32, against the threshold 2 t + 2^-16 a (the widening exceeds every
 * binary32 rounding of the test, so a pair at distance <= 2 t is always
 * found).  Steps: bounding spheres (|dj| > 2 a + thr: no); slab along ni
 * (|dj.ni| - a sin > thr: no) and along nj, with sin the sine of the angle
 * between the normals; then the rim of i against the disk of j and the rim
 * of j against the disk of i. */
int spec_plt_collide32(const double dj[3], const double ni[3], const double nj[3], double a, double t)
{
    const float d[3] = {(float)dj[0], (float)dj[1], (float)dj[2]};
    const float u[3] = {(float)ni[0], (float)ni[1], (float)ni[2]};
    const float v[3] = {(float)nj[0], (float)nj[1], (float)nj[2]};
    const float af = (float)a, tf = (float)t;
    float thr = (tf + tf) + af * PLT_SLACK;
    float reach = (af + af) + thr;
    if (dot3f(d, d) > reach * reach) return 0;
    float c = dot3f(u, v);
    float s2 = 1.0f - c * c;
    if (s2 < 0.0f) s2 = 0.0f;
    float sn = sqrtf(s2);
    float ext = af * sn;
    if (fabsf(dot3f(d, u)) - ext > thr) return 0;
    if (fabsf(dot3f(d, v)) - ext > thr) return 0;
    float ei1[3], ei2[3], ej1[3], ej2[3];
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    basis_f(u, ei1, ei2);
    basis_f(v, ej1, ej2);
    if (rim_near_disk_f(zero, ei1, ei2, af, d, v, af, sn, thr, NULL)) return 1;
    if (rim_near_disk_f(d, ej1, ej2, af, zero, u, af, sn, thr, NULL)) return 1;
    return 0;
}

/* Why spec_plt_collide32 decides as it does: 0 separated, 1 some rim point
 * lies within the widened threshold, 2 contact only because some arc was
 * still undecided at level 20 or after 512 evaluations (a near-contact its
 * bisection could not resolve).  Evaluates all 16 arcs; nonzero exactly
 * when spec_plt_collide32 returns 1. */
int spec_plt_collide32_reason(const double dj[3], const double ni[3], const double nj[3], double a, double t)
{
    if (!spec_plt_collide32(dj, ni, nj, a, t)) return 0;
    const float d[3] = {(float)dj[0], (float)dj[1], (float)dj[2]};
    const float u[3] = {(float)ni[0], (float)ni[1], (float)ni[2]};
    const float v[3] = {(float)nj[0], (float)nj[1], (float)nj[2]};
    const float af = (float)a, tf = (float)t;
    float thr = (tf + tf) + af * PLT_SLACK;
    float c = dot3f(u, v);
    float s2 = 1.0f - c * c;
    if (s2 < 0.0f) s2 = 0.0f;
    float sn = sqrtf(s2);
    float ei1[3], ei2[3], ej1[3], ej2[3];
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    basis_f(u, ei1, ei2);
    basis_f(v, ej1, ej2);
    int why = 0;
    for (int k0 = 0; k0 < 8; k0++) {
        int r1 = arc_near_disk_f(zero, ei1, ei2, af, d, v, af, sn, thr, k0, NULL);
        int r2 = arc_near_disk_f(d, ej1, ej2, af, zero, u, af, sn, thr, k0, NULL);
        if (r1 == 1 || r2 == 1) return 1;
        if (r1 == 2 || r2 == 2) why = 2;
    }
    return why;
}
