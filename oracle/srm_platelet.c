/*
 * srm_platelet.c -- TEST INFRASTRUCTURE ONLY.
 *
 * FP64 reference of SRM for thin circular platelets (Section 3.3): the
 * method of Algorithms 1-6 with the geometry-dependent collision routine
 * replaced by a spherodisk test and the migration move extended by a small
 * rotation.  Only the tests, the smoke check and the CPU leg of the
 * benchmark load it; the product library never does, and it shares no code
 * with the CUDA path.  Built like srm_oracle.c (gcc -O2 -ffp-contract=off):
 * every operation is one IEEE binary64 operation in source order.
 *
 * Readings fixed here (the paper names the shape and the parameters only):
 *   - a spherodisk is the set of points within distance t of a flat circular
 *     disk of radius a (centre x, unit normal n); its diameter is
 *     D = 2 (a + t), its thickness 2 t, its aspect ratio D / (2 t);
 *   - every platelet has the same base sizes (a0, t0); swelling scales both,
 *     a = lambda a0, t = lambda t0 (Alg 1, the shape is kept);
 *   - the number density of Eq. 1 is rho = N D^3 / V with V the box volume;
 *   - two platelets collide when the distance between their disks is at
 *     most t_i + t_j (closed inequality, as for spheres), decided in
 *     binary32 with the widening described below;
 *   - try l of Alg 3 moves the centre by c_m u (u from stream 0, as for
 *     spheres) and turns the normal to (n + c_r v) / |n + c_r v| with v a
 *     second uniform direction (stream 1), 0 <= c_r < 1;
 *   - cells are sized from the bounding sphere, 2.5 lambda (a0 + t0) + c_m,
 *     since two platelets can touch only when their centres are within
 *     2 lambda (a0 + t0).
 *
 * Collision decision.  The distance between two disks is reached at a point
 * of one of the two rims (if the closest pair were interior to both disks,
 * the disks would be parallel and the overlap of their projections, bounded
 * by rim arcs, contains rim points at the same distance; if the disks cross,
 * an end of one disk's chord on the line where the planes meet lies inside
 * the other disk).  So the platelets collide exactly when some rim point of
 * one disk lies within t_i + t_j of the other disk.  The rim is walked by
 * bisection.  The rim point moves at most 2 a / (1 + s^2) <= a (2 - s^2)
 * =: V per unit of the rational parameter s (1 / (1 + x) <= 1 - x / 2 on
 * [0, 1]), and its distance to the other disk is
 * sqrt(h^2 + e^2) with h its height above that disk's plane and e the
 * excess of its projected distance from that disk's centre over the radius
 * (0 inside).  Along the rim h changes at most at V sin(theta) (the rim lies
 * in its own plane; theta is the angle between the normals) and e at most
 * at V, so over an interval of half-width r around its midpoint,
 * sqrt(max(0, |h| - V r sin)^2 + max(0, e - V r)^2) bounds the distance
 * from below.  Intervals whose bound is above the threshold are dropped, a
 * midpoint at or below it is a collision (both compared as squares: h^2 +
 * e^2 <= thr^2).  Each of the 8 first-level arcs of a rim is bisected on
 * its own; an arc still undecided at 2^-20 of the circle, or after 512
 * evaluations, counts as a collision (a near-contact the bisection cannot
 * resolve is reported as contact).  The arcs are independent, so the
 * decision is the OR of 16 arc results (2 rims x 8 arcs) in any order.  Cheap exact
 * separations come first: the bounding spheres, and the two slabs along the
 * normals.
 *
 * Precision.  The decision is evaluated in binary32 (the paper fixes no
 * precision for it) on the pair's relative geometry: the centre difference
 * is formed in binary64 under the minimum image and then rounded, like the
 * normals and sizes.  Its threshold is widened from t_i + t_j by 2^-16 a,
 * more than the binary32 rounding of every quantity in the test (a few
 * ulps of 3 a), so a pair whose true distance is at most t_i + t_j is
 * always reported (the widening only ever adds contacts).  Centres, normals,
 * draws and moves stay in binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_unit_dir_stream(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, int dim, int stream, double u[3]);
double orc_wrap(double x, double L);
void orc_grid(int dim, const double L[3], double lam, double rmax, double c_m, int64_t n[3], double w[3]);

#define PLT_TOP 3        /* first level evaluated: 8 intervals of the circle */
#define PLT_DEPTH 20     /* finest level (binary32 still separates its midpoints) */
#define PLT_EVALS 512    /* evaluations per level-3 interval (4096 per rim) */
#define PLT_SLACK 0x1p-16f /* threshold widening, in units of the disk radius */

static float dot3f(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

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

void orc_plt_basis(const double n[3], double e1[3], double e2[3])
{
    const float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
    float a[3], b[3];
    basis_f(nf, a, b);
    for (int k = 0; k < 3; k++) {
        e1[k] = a[k];
        e2[k] = b[k];
    }
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

/* Distance from point p to that disk: sqrt(h^2 + e^2) (binary32). */
double orc_plt_point_disk(const double p[3], const double cd[3], const double nd[3], double b)
{
    const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
    const float cf[3] = {(float)cd[0], (float)cd[1], (float)cd[2]};
    const float nf[3] = {(float)nd[0], (float)nd[1], (float)nd[2]};
    float h, e;
    point_disk_he(pf, cf, nf, (float)b, &h, &e);
    return sqrtf(h * h + e * e);
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
 * Returns 1 (yes, or undecided at level 20 or after 512 evaluations) or 0;
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
                return 1;
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

int orc_plt_rim_near_disk(const double cc[3], const double e1[3], const double e2[3], double a,
                          const double cd[3], const double nd[3], double b, double sn, double thr, int *evals)
{
    float c1[3], f1[3], f2[3], c2[3], n2[3];
    for (int k = 0; k < 3; k++) {
        c1[k] = (float)cc[k];
        f1[k] = (float)e1[k];
        f2[k] = (float)e2[k];
        c2[k] = (float)cd[k];
        n2[k] = (float)nd[k];
    }
    return rim_near_disk_f(c1, f1, f2, (float)a, c2, n2, (float)b, (float)sn, (float)thr, evals);
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
int orc_plt_collide(const double dj[3], const double ni[3], const double nj[3], double a, double t)
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

/* ---------------------------------------------------------------------------
 * Platelet system.  Centres X[3 pid + a] and unit normals U[3 pid + a] in id
 * order; sizes a = lambda a0, t = lambda t0.
 * ------------------------------------------------------------------------- */
typedef struct orc_plt {
    double L[3];
    int64_t N;
    double *X, *U;
    double a0, t0, lam, lam_t;
    double c_w, c_m, c_r;
    int N_k, N_l, N_shake;
    uint64_t seed, sweep;
    int64_t n[3];
    double w[3];
    int64_t ncells, cap_cells;
    int64_t *cell_start, *members;
    int64_t iters, accepted_iters, shake_iters, moves_accepted;
} orc_plt;

static int64_t pcell_coord(double x, double w, int64_t n)
{
    int64_t c = (int64_t)(x / w);
    return (c % n + n) % n;
}

/* Alg 2 on centres, grid of the bounding radius lambda (a0 + t0). */
static void pbin(orc_plt *s, const double *X, double lam_grid)
{
    orc_grid(3, s->L, lam_grid, s->a0 + s->t0, s->c_m, s->n, s->w);
    s->ncells = s->n[0] * s->n[1] * s->n[2];
    if (s->ncells + 1 > s->cap_cells) {
        free(s->cell_start);
        s->cap_cells = s->ncells + 1;
        s->cell_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)s->cap_cells);
    }
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->N > 0 ? s->N : 1));
    memset(s->cell_start, 0, sizeof(int64_t) * (size_t)(s->ncells + 1));
    for (int64_t i = 0; i < s->N; i++) {
        int64_t c[3];
        for (int a = 0; a < 3; a++) c[a] = pcell_coord(X[3 * i + a], s->w[a], s->n[a]);
        cell_of[i] = c[0] + s->n[0] * (c[1] + s->n[1] * c[2]);
        s->cell_start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < s->ncells; c++) s->cell_start[c + 1] += s->cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)s->ncells);
    memcpy(fill, s->cell_start, sizeof(int64_t) * (size_t)s->ncells);
    for (int64_t i = 0; i < s->N; i++) s->members[fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
}

/* Alg 5 for a platelet at centre q with normal u (id pid): any other
 * platelet listed in the 27 cells around q's cell that collides with it. */
static int pcollide(const orc_plt *s, const double *X, const double *U, double lam, const double q[3],
                    const double u[3], int64_t pid)
{
    int64_t c[3];
    for (int a = 0; a < 3; a++) c[a] = pcell_coord(q[a], s->w[a], s->n[a]);
    double a = lam * s->a0, t = lam * s->t0;
    for (int sx = -1; sx <= 1; sx++)
        for (int sy = -1; sy <= 1; sy++)
            for (int sz = -1; sz <= 1; sz++) {
                int64_t nx = (c[0] + sx + s->n[0]) % s->n[0];
                int64_t ny = (c[1] + sy + s->n[1]) % s->n[1];
                int64_t nz = (c[2] + sz + s->n[2]) % s->n[2];
                int64_t cell = nx + s->n[0] * (ny + s->n[1] * nz);
                for (int64_t k = s->cell_start[cell]; k < s->cell_start[cell + 1]; k++) {
                    int64_t j = s->members[k];
                    if (j == pid) continue;
                    double d[3];
                    for (int b = 0; b < 3; b++) {
                        double db = X[3 * j + b] - q[b];
                        if (db > 0.5 * s->L[b]) db -= s->L[b];
                        if (db < -0.5 * s->L[b]) db += s->L[b];
                        d[b] = db;
                    }
                    if (orc_plt_collide(d, u, &U[3 * j], a, t)) return 1;
                }
            }
    return 0;
}

/* Trial l of platelet pid from centre x0 and normal u0 (Alg 3 with the
 * rotation of Section 3.3). */
void orc_plt_trial(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, const double L[3], double c_m,
                   double c_r, const double x0[3], const double u0[3], double q[3], double u[3])
{
    double dir[3];
    orc_unit_dir_stream(seed, sweep, pid, l, 3, 0, dir);
    for (int a = 0; a < 3; a++) q[a] = orc_wrap(x0[a] + c_m * dir[a], L[a]);
    if (c_r > 0.0) {
        double v[3], m[3];
        orc_unit_dir_stream(seed, sweep, pid, l, 3, 1, v);
        for (int a = 0; a < 3; a++) m[a] = u0[a] + c_r * v[a];
        double r = sqrt(dot3(m, m));
        for (int a = 0; a < 3; a++) u[a] = m[a] / r;
    } else {
        for (int a = 0; a < 3; a++) u[a] = u0[a];
    }
}

static int pmove(orc_plt *s, double *X, double *U, double lam, int64_t pid)
{
    double x0[3], u0[3], q[3], u[3];
    for (int a = 0; a < 3; a++) {
        x0[a] = X[3 * pid + a];
        u0[a] = U[3 * pid + a];
    }
    for (int l = 0; l < s->N_l; l++) {
        orc_plt_trial(s->seed, s->sweep, (uint64_t)pid, (uint64_t)l, s->L, s->c_m, s->c_r, x0, u0, q, u);
        if (!pcollide(s, X, U, lam, q, u, pid)) {
            for (int a = 0; a < 3; a++) {
                X[3 * pid + a] = q[a];
                U[3 * pid + a] = u[a];
            }
            return 1;
        }
    }
    return 0;
}

/* One sweep of Alg 3 in the canonical coloured order (colour chi = sum_a
 * (c_a mod 3) 3^a ascending, cells of a colour in lexicographic order,
 * particles of a cell by ascending id).  Advances the sweep counter. */
static int64_t psweep(orc_plt *s, double *X, double *U, double lam, double lam_grid)
{
    pbin(s, X, lam_grid);
    int64_t acc = 0;
    for (int chi = 0; chi < 27; chi++) {
        int64_t a0 = chi % 3, a1 = (chi / 3) % 3, a2 = chi / 9;
        for (int64_t cz = a2; cz < s->n[2]; cz += 3)
            for (int64_t cy = a1; cy < s->n[1]; cy += 3)
                for (int64_t cx = a0; cx < s->n[0]; cx += 3) {
                    int64_t cell = cx + s->n[0] * (cy + s->n[1] * cz);
                    for (int64_t k = s->cell_start[cell]; k < s->cell_start[cell + 1]; k++)
                        acc += pmove(s, X, U, lam, s->members[k]);
                }
    }
    s->sweep++;
    s->moves_accepted += acc;
    return acc;
}

/* Alg 6 with a full count: platelets that collide with another. */
static int64_t pcheck(orc_plt *s, const double *X, const double *U, double lam, double lam_grid, uint8_t *flags)
{
    pbin(s, X, lam_grid);
    int64_t cnt = 0;
    for (int64_t i = 0; i < s->N; i++) {
        int hit = pcollide(s, X, U, lam, &X[3 * i], &U[3 * i], i);
        if (flags) flags[i] = (uint8_t)hit;
        cnt += hit;
    }
    return cnt;
}

orc_plt *orc_plt_create(const double L[3], int64_t N, const double *X, const double *U, double a0, double t0,
                        double lam, double lam_t, double c_w, double c_m, double c_r, int N_k, int N_l,
                        int N_shake, uint64_t seed, uint64_t sweep)
{
    orc_plt *s = (orc_plt *)calloc(1, sizeof(orc_plt));
    for (int a = 0; a < 3; a++) s->L[a] = L[a];
    s->N = N;
    size_t nn = (size_t)(N > 0 ? N : 1);
    s->X = (double *)malloc(sizeof(double) * 3 * nn);
    s->U = (double *)malloc(sizeof(double) * 3 * nn);
    s->members = (int64_t *)malloc(sizeof(int64_t) * nn);
    if (N > 0) {
        memcpy(s->X, X, sizeof(double) * 3 * (size_t)N);
        memcpy(s->U, U, sizeof(double) * 3 * (size_t)N);
    }
    s->a0 = a0;
    s->t0 = t0;
    s->lam = lam;
    s->lam_t = lam_t;
    s->c_w = c_w;
    s->c_m = c_m;
    s->c_r = c_r;
    s->N_k = N_k;
    s->N_l = N_l;
    s->N_shake = N_shake;
    s->seed = seed;
    s->sweep = sweep;
    return s;
}

void orc_plt_destroy(orc_plt *s)
{
    if (!s) return;
    free(s->X);
    free(s->U);
    free(s->members);
    free(s->cell_start);
    free(s);
}

void orc_plt_get(const orc_plt *s, double *X, double *U)
{
    memcpy(X, s->X, sizeof(double) * 3 * (size_t)s->N);
    memcpy(U, s->U, sizeof(double) * 3 * (size_t)s->N);
}
double orc_plt_lambda(const orc_plt *s) { return s->lam; }
uint64_t orc_plt_sweep_counter(const orc_plt *s) { return s->sweep; }

/* counters: iters, accepted iterations, shake iterations, accepted moves, sweeps */
void orc_plt_counters(const orc_plt *s, int64_t out[5])
{
    out[0] = s->iters;
    out[1] = s->accepted_iters;
    out[2] = s->shake_iters;
    out[3] = s->moves_accepted;
    out[4] = (int64_t)s->sweep;
}

/* One sweep of Alg 3 on P at its own scale (the relaxation move). */
int64_t orc_plt_sweep(orc_plt *s) { return psweep(s, s->X, s->U, s->lam, s->lam); }

/* Alg 6 on P at its own scale. */
int64_t orc_plt_check(orc_plt *s, uint8_t *flags) { return pcheck(s, s->X, s->U, s->lam, s->lam, flags); }

/* One iteration of Alg 1 (as orc_iterate: swell Q, up to N_k rounds of
 * sweep and check, accept, or discard and shake P with N_shake sweeps on
 * the grid of the iteration).  Returns 1 accepted, 0 discarded, 2 at the
 * target.  info: {k sweeps, colliding count of the last check, shake
 * sweeps}. */
int orc_plt_iterate(orc_plt *s, int64_t info[3])
{
    if (s->lam >= s->lam_t) return 2;
    s->iters++;
    double lam_q = s->lam * (1.0 + s->c_w);
    if (lam_q > s->lam_t) lam_q = s->lam_t;
    size_t bytes = sizeof(double) * 3 * (size_t)(s->N > 0 ? s->N : 1);
    double *QX = (double *)malloc(bytes), *QU = (double *)malloc(bytes);
    memcpy(QX, s->X, bytes);
    memcpy(QU, s->U, bytes);
    int64_t cnt = -1;
    int k;
    for (k = 1; k <= s->N_k; k++) {
        psweep(s, QX, QU, lam_q, lam_q);
        cnt = pcheck(s, QX, QU, lam_q, lam_q, NULL);
        if (cnt == 0) break;
    }
    int accepted = cnt == 0;
    if (accepted) {
        memcpy(s->X, QX, bytes);
        memcpy(s->U, QU, bytes);
        s->lam = lam_q;
        s->accepted_iters++;
    } else {
        for (int j = 0; j < s->N_shake; j++) psweep(s, s->X, s->U, s->lam, lam_q);
        s->shake_iters++;
    }
    free(QX);
    free(QU);
    if (info) {
        info[0] = accepted ? k : s->N_k;
        info[1] = cnt;
        info[2] = accepted ? 0 : s->N_shake;
    }
    return accepted;
}

int64_t orc_plt_run(orc_plt *s, int64_t max_iters)
{
    int64_t it = 0;
    while (s->lam < s->lam_t && it < max_iters) {
        orc_plt_iterate(s, NULL);
        it++;
    }
    return it;
}

/* All colliding pairs i < j by brute force over every pair (minimum image),
 * independent of the cell list: the certification of a final state.
 * Writes up to cap pairs, returns the count. */
int64_t orc_plt_pairs_brute(const double L[3], int64_t N, const double *X, const double *U, double a, double t,
                            int64_t *ij, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = i + 1; j < N; j++) {
            double d[3];
            for (int b = 0; b < 3; b++) {
                double db = X[3 * j + b] - X[3 * i + b];
                if (db > 0.5 * L[b]) db -= L[b];
                if (db < -0.5 * L[b]) db += L[b];
                d[b] = db;
            }
            if (orc_plt_collide(d, &U[3 * i], &U[3 * j], a, t)) {
                if (cnt < cap) {
                    ij[2 * cnt] = i;
                    ij[2 * cnt + 1] = j;
                }
                cnt++;
            }
        }
    return cnt;
}
