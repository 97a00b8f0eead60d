/*
 * srm_platelet.c -- TEST INFRASTRUCTURE ONLY.
 *
 * FP64 reference of SRM for thin circular platelets (Section 3.3): the
 * method of Algorithms 1-6 with the geometry-dependent collision routine
 * replaced by a spherodisk test and the migration move extended by a small
 * rotation.  Only the tests, the smoke check and the CPU leg of the
 * benchmark load it; the product library never does, and it shares no code
 * with the CUDA path.  Built like srm_oracle.c (gcc -O2 -ffp-contract=off):
 * every arithmetic operation is one IEEE binary64 operation in source order;
 * cos, sin and sqrt are the C library's binary64 functions.
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
 *     binary64 as described below;
 *   - try l of Alg 3 moves the centre by c_m u (u from stream 0, as for
 *     spheres) and turns the normal to (n + c_r v) / |n + c_r v| with v a
 *     second uniform direction (stream 1), 0 <= c_r < 1;
 *   - cells are sized from the bounding sphere, 2.5 lambda (a0 + t0) + c_m,
 *     since two platelets can touch only when their centres are within
 *     2 lambda (a0 + t0).
 *
 * Collision decision.  The distance between two disks is reached at a point
 * of one of the two rims: if the closest pair of points were interior to
 * both disks the disks would be parallel, and then the overlap of their
 * projections, which is bounded by rim arcs, contains rim points at the
 * same distance; if the disks cross, an end of one disk's chord on the line
 * where the planes meet lies inside the other disk.  So the platelets
 * collide exactly when some rim point of one disk lies within t_i + t_j of
 * the other disk.
 *
 * The distance from a point p to a disk (centre c, unit normal m, radius b)
 * is sqrt(h^2 + e^2), with h = (p - c).m its height above the disk's plane
 * and e the excess of its in-plane distance from c over b (0 inside).  On a
 * rim p(phi) = c_r + a (cos phi e1 + sin phi e2), the point moves at speed a
 * per radian along a tangent that lies in the rim's own plane, so h changes
 * at most at a sin(theta) (theta the angle between the two normals, sin
 * theta = |n_i x n_j|) and e at most at a.  Over an arc of half-width r
 * around phi_m the distance is therefore at least
 *     sqrt(max(0, |h(phi_m)| - a r sin theta)^2 + max(0, e(phi_m) - a r)^2),
 * a Lipschitz lower bound.  The rim is searched by branch and bound: an arc
 * whose midpoint is within the threshold decides "collision"; an arc whose
 * lower bound is above it is dropped; any other arc is halved (depth
 * first).  An arc still undecided at half-width 2^-40 rad counts as contact:
 * the distance there is within 2 a 2^-40 (2e-12 a) of the threshold.  As a
 * safety net a rim that needs more than 2^20 evaluations also counts as
 * contact; it only happens for pairs within rounding of touching.  Cheap
 * exact separations come first: the bounding spheres (every point of a disk
 * is within a of its centre), and the two slabs (disk j lies within
 * a sin(theta) of the plane through its centre parallel to disk i).  The
 * pair is evaluated in a frame centred between the two platelets, so that
 * swapping them gives the same operations and the same answer.
 *
 * Periodicity: the minimum image of the centre difference by default; in
 * the images mode (orc_plt_set_images) explicit image platelets as for the
 * spheres (orc_images.h): the difference is (x_j + s L) - x_i.
 *
 * Tests may substitute another contact predicate for the sweeps and checks
 * (orc_plt_set_contact) -- the binary32 decision of the CUDA kernel, kept as
 * a kernel specification beside the tests -- to compare whole sweeps with
 * the GPU bit for bit; the reference's own predicate, and the one of its
 * brute-force certification, is the binary64 decision above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_images.h"

int orc_unit_dir_stream(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, int dim, int stream, double u[3]);
double orc_wrap(double x, double L);
void orc_grid(int dim, const double L[3], double lam, double rmax, double c_m, int64_t n[3], double w[3]);

#define PLT_MIN_HALF_WIDTH 0x1p-40 /* radians: finest arc of the rim search */
#define PLT_MAX_EVALS (1 << 20)    /* evaluations per rim before counting as contact */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Orthonormal basis (e1, e2) of the plane of the unit normal n: e1 is n
 * crossed with the coordinate axis of smallest |n_k| (the first such axis),
 * normalised; e2 = n x e1. */
void orc_plt_basis(const double n[3], double e1[3], double e2[3])
{
    double ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
    int k = 0;
    double m = ax;
    if (ay < m) {
        k = 1;
        m = ay;
    }
    if (az < m) k = 2;
    double axis[3] = {0.0, 0.0, 0.0};
    axis[k] = 1.0;
    double c[3];
    cross3(n, axis, c);
    double r = sqrt(dot3(c, c));
    for (int a = 0; a < 3; a++) e1[a] = c[a] / r;
    cross3(n, e1, e2);
}

/* Point p against the disk of centre cd, unit normal nd, radius b: h =
 * height above the plane, e = distance of the projection from cd minus b,
 * or 0 when the projection lies in the disk. */
static void point_disk_he(const double p[3], const double cd[3], const double nd[3], double b, double *h, double *e)
{
    double q[3] = {p[0] - cd[0], p[1] - cd[1], p[2] - cd[2]};
    double hh = dot3(q, nd);
    double r[3] = {q[0] - hh * nd[0], q[1] - hh * nd[1], q[2] - hh * nd[2]};
    double rr = dot3(r, r);
    *h = hh;
    *e = rr <= b * b ? 0.0 : sqrt(rr) - b;
}

/* Distance from point p to that disk: sqrt(h^2 + e^2). */
double orc_plt_point_disk(const double p[3], const double cd[3], const double nd[3], double b)
{
    double h, e;
    point_disk_he(p, cd, nd, b, &h, &e);
    return sqrt(h * h + e * e);
}

/* Is some point of the rim of the disk (centre cc, in-plane basis e1 e2,
 * radius a) within thr of the disk (cd, nd, b)?  sn = sine of the angle
 * between the two normals.  Branch and bound over the rim angle (see the
 * header); *evals (may be NULL) receives the number of rim points
 * evaluated. */
static int rim_within(const double cc[3], const double e1[3], const double e2[3], double a, const double cd[3],
                      const double nd[3], double b, double sn, double thr, int *evals)
{
    const double pi = 3.14159265358979323846;
    const double thr2 = thr * thr;
    /* pending arcs (midpoint, half-width); depth first, so at most two per
     * halving level are pending: 2 x 42 levels fit */
    double mid[96], half[96];
    int top = 0, ne = 0, hit = 0;
    mid[0] = pi;
    half[0] = pi;
    top = 1;
    while (top > 0) {
        top--;
        double phi = mid[top], r = half[top];
        double p[3], h, e;
        double c = cos(phi), s = sin(phi);
        for (int k = 0; k < 3; k++) p[k] = cc[k] + a * (c * e1[k] + s * e2[k]);
        point_disk_he(p, cd, nd, b, &h, &e);
        ne++;
        if (h * h + e * e <= thr2) {
            hit = 1;
            break;
        }
        double hl = fabs(h) - a * r * sn, el = e - a * r;
        if (hl < 0.0) hl = 0.0;
        if (el < 0.0) el = 0.0;
        if (hl * hl + el * el > thr2) continue; /* the whole arc is farther than thr */
        if (r < PLT_MIN_HALF_WIDTH || ne >= PLT_MAX_EVALS) {
            hit = 1; /* undecided within 2 a r of the threshold: counted as contact */
            break;
        }
        /* left half on top, so that it is taken first */
        mid[top] = phi + 0.5 * r;
        half[top] = 0.5 * r;
        top++;
        mid[top] = phi - 0.5 * r;
        half[top] = 0.5 * r;
        top++;
    }
    if (evals) *evals = ne;
    return hit;
}

/* The rim of the disk (cc, normal n_c, radius a) against the disk (cd, nd,
 * b) at distance thr, with its own basis and angle (for the tests). */
int orc_plt_rim_near_disk(const double cc[3], const double n_c[3], double a, const double cd[3], const double nd[3],
                          double b, double thr, int *evals)
{
    double e1[3], e2[3], x[3];
    orc_plt_basis(n_c, e1, e2);
    cross3(n_c, nd, x);
    return rim_within(cc, e1, e2, a, cd, nd, b, sqrt(dot3(x, x)), thr, evals);
}

/* Do the spherodisks i and j (disk radius a, half-thickness t each) collide?
 * dj = centre of j minus centre of i (minimum image); ni, nj unit normals.
 * The distance between the disks is compared with thr = t_i + t_j = 2 t in
 * binary64, in the frame whose origin is the midpoint of the two centres
 * (i at -dj/2, j at +dj/2).  Steps: bounding spheres (|dj| > 2 a + thr: no);
 * slab along ni (|dj.ni| - a sin(theta) > thr: no) and along nj; the rim of
 * i against the disk of j; the rim of j against the disk of i. */
int orc_plt_collide(const double dj[3], const double ni[3], const double nj[3], double a, double t)
{
    double thr = t + t;
    double reach = (a + a) + thr;
    if (dot3(dj, dj) > reach * reach) return 0;
    double x[3];
    cross3(ni, nj, x);
    double sn = sqrt(dot3(x, x));
    double ext = a * sn;
    if (fabs(dot3(dj, ni)) - ext > thr) return 0;
    if (fabs(dot3(dj, nj)) - ext > thr) return 0;
    double ci[3], cj[3];
    for (int k = 0; k < 3; k++) {
        cj[k] = 0.5 * dj[k];
        ci[k] = -cj[k];
    }
    double ei1[3], ei2[3], ej1[3], ej2[3];
    orc_plt_basis(ni, ei1, ei2);
    orc_plt_basis(nj, ej1, ej2);
    if (rim_within(ci, ei1, ei2, a, cj, nj, a, sn, thr, NULL)) return 1;
    if (rim_within(cj, ej1, ej2, a, ci, ni, a, sn, thr, NULL)) return 1;
    return 0;
}

/* Contact predicate of the sweeps and checks (default orc_plt_collide). */
typedef int (*orc_plt_contact_fn)(const double dj[3], const double ni[3], const double nj[3], double a, double t);

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
    orc_plt_contact_fn contact;
    int images;      /* periodicity by image platelets instead of the minimum image */
    orc_imgtab img;
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
    if (s->images) orc_imgtab_build(&s->img, 3, s->n, s->w, X, s->N);
}

/* Alg 5 for a platelet at centre q with normal u (id pid): any other
 * platelet listed in the 27 cells around q's cell that collides with it. */
static int pcollide(const orc_plt *s, const double *X, const double *U, double lam, const double q[3],
                    const double u[3], int64_t pid)
{
    int64_t c[3];
    for (int a = 0; a < 3; a++) c[a] = pcell_coord(q[a], s->w[a], s->n[a]);
    double a = lam * s->a0, t = lam * s->t0;
    if (s->images) {
        /* image platelets: entries of the 27 padded cells around q's cell,
         * plain differences (x_j + s L) - q */
        const orc_imgtab *tb = &s->img;
        for (int sz = -1; sz <= 1; sz++)
            for (int sy = -1; sy <= 1; sy++)
                for (int sx = -1; sx <= 1; sx++) {
                    int64_t pc = orc_imgtab_near(tb, q, sx, sy, sz);
                    for (int64_t k = 0; k < tb->cnt[pc]; k++) {
                        int64_t j = tb->id[pc][k];
                        if (j == pid) continue;
                        const int8_t *sh = &tb->sh[pc][3 * k];
                        double d[3];
                        for (int b = 0; b < 3; b++) d[b] = (X[3 * j + b] + (double)sh[b] * s->L[b]) - q[b];
                        if (s->contact(d, u, &U[3 * j], a, t)) return 1;
                    }
                }
        return 0;
    }
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
                    if (s->contact(d, u, &U[3 * j], a, t)) return 1;
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
            if (s->images) orc_imgtab_move(&s->img, pid, x0, q);
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
    s->contact = orc_plt_collide;
    return s;
}

/* Substitutes the contact predicate of the sweeps and checks (NULL: the
 * reference's binary64 orc_plt_collide).  For tests only. */
void orc_plt_set_contact(orc_plt *s, orc_plt_contact_fn fn) { s->contact = fn ? fn : orc_plt_collide; }

/* Periodicity by image platelets (1) or by the minimum image (0). */
void orc_plt_set_images(orc_plt *s, int on) { s->images = on ? 1 : 0; }

/* Image entries kept move by move during the last sweep against a rebuild
 * from P (mismatching padded cells; -1 outside the images mode). */
int64_t orc_plt_images_verify(orc_plt *s)
{
    if (!s->images || !s->img.cnt) return -1;
    return orc_imgtab_verify(&s->img, s->X, s->N);
}

void orc_plt_destroy(orc_plt *s)
{
    if (!s) return;
    orc_imgtab_free(&s->img);
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
