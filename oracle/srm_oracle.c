/*
 * srm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 reference of the Swelling and Random
 * Migration (SRM) method (Tarasovs, "Efficient generation of large-scale
 * non-equilibrium distributions of particles", Section 2, Algorithms 1-6).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it; the product library never links, loads or calls it, and it shares
 * no code with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math): every
 * floating-point operation below is one IEEE-754 binary64 operation with
 * round-to-nearest, evaluated in source order, so the result is a function of
 * the inputs alone.
 *
 * Readings of the paper that this file fixes (the paper is silent or loose):
 *   - swelling is multiplicative, R_i = lambda * r_i, lambda <- lambda(1+c_w),
 *     capped at the target scale lambda_t (Alg 1, Section 2 step a,
 *     "minor adjustments" of the last iteration);
 *   - cell size uses the post-swell radius; the grid has n = 3*max(1,
 *     floor(L/(3*cellSize))) cells per axis of width w = L/n, so that cells
 *     can be coloured by (cell index mod 3) (Alg 1, Alg 2);
 *   - a particle never collides with itself (Alg 5 skips t == q);
 *   - touching counts as a collision: sqrt(dx^2+dy^2[+dz^2]) <= R_q + R_t
 *     (Alg 5);
 *   - "unit random vector" is a uniform direction: rejection sampling from
 *     the cube [-1,1)^d on a 2^-31 lattice, then division by the norm, with
 *     the draws taken from Philox4x32-10 keyed by the seed at counter
 *     (particle id, sweep index, try and candidate) (Alg 3);
 *   - the shake step runs N_shake sweeps of Alg 3 on the unswollen P, each
 *     preceded by a fresh binning, on the grid of the iteration (Alg 1,
 *     Section 2 step d);
 *   - the order of Alg 3's "for each particle" is the canonical coloured
 *     order: for colour chi = sum_a (c_a mod 3) 3^a ascending, for cells of
 *     that colour in lexicographic order, particles of the cell by ascending
 *     id.  A "literal" mode keeps plain id order (Alg 3 as printed);
 *   - periodicity: the minimum-image convention of Alg 5 by default; an
 *     "images" mode takes the other way Section 2 names, explicit image
 *     particles (see orc_set_images below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_images.h"

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11, Section 4.2): ten rounds of two 32x32->64 bit
 * multiplies (high halves xored with the other counter words and the key,
 * low halves kept), the key advanced by the two Weyl constants between
 * rounds.
 * ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

#define ORC_MAX_CAND 32

int orc_unit_dir_stream(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, int dim, int stream, double u[3]);

/* Uniform direction on the unit circle / sphere (Alg 3).  Candidate m of
 * try l takes one Philox block at counter (pid, sweep mod 2^32, l + 2^16 m,
 * sweep div 2^32) with key (seed mod 2^32, seed div 2^32); coordinate a is
 * (word_a - 2^31) * 2^-31, a point of the cube [-1,1) on a 2^-31 lattice,
 * exact in binary64.  The first candidate with 0 < |v|^2 <= 1 is normalised
 * by dividing each coordinate by sqrt(|v|^2).  After 32 rejected candidates
 * (probability < 1e-10) the direction is the first axis.  l < 2^16.
 * Returns the index of the accepted candidate. */
int orc_unit_dir(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, int dim, double u[3])
{
    return orc_unit_dir_stream(seed, sweep, pid, l, dim, 0, u);
}

/* The same draw from stream 0 or 1: stream 1 sets the top bit of the fourth
 * counter word (sweep < 2^63), giving a second independent direction per
 * try (the rotation of a platelet, Section 3.3). */
int orc_unit_dir_stream(uint64_t seed, uint64_t sweep, uint64_t pid, uint64_t l, int dim, int stream, double u[3])
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t hi = (uint32_t)(sweep >> 32) | (stream ? 0x80000000u : 0u);
    for (int m = 0; m < ORC_MAX_CAND; m++) {
        const uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)sweep, (uint32_t)(l + ((uint64_t)m << 16)), hi};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        double v[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; a++) v[a] = (double)((int64_t)w[a] - (int64_t)2147483648LL) * 0x1p-31;
        double s = v[0] * v[0] + v[1] * v[1];
        if (dim == 3) s = s + v[2] * v[2];
        if (s > 0.0 && s <= 1.0) {
            double nrm = sqrt(s);
            for (int a = 0; a < dim; a++) u[a] = v[a] / nrm;
            for (int a = dim; a < 3; a++) u[a] = 0.0;
            return m;
        }
    }
    u[0] = 1.0; u[1] = 0.0; u[2] = 0.0;
    return ORC_MAX_CAND;
}

/* Alg 4: periodic wrapping, "< 0" tested before ">= L". */
double orc_wrap(double x, double L)
{
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

/* Alg 1 with the coloured-grid reading: cellSize from the swollen
 * maximum radius, n a multiple of 3, w = L / n. */
void orc_grid(int dim, const double L[3], double lam, double rmax, double c_m,
              int64_t n[3], double w[3])
{
    double cell_size = 2.5 * (lam * rmax) + c_m;
    for (int a = 0; a < 3; a++) {
        if (a >= dim) { n[a] = 1; w[a] = L[a]; continue; }
        int64_t k = (int64_t)(L[a] / (3.0 * cell_size));
        if (k < 1) k = 1;
        n[a] = 3 * k;
        w[a] = L[a] / (double)n[a];
    }
}

/* Alg 2: cell coordinate of one position. */
static int64_t cell_coord(double x, double w, int64_t n)
{
    int64_t c = (int64_t)(x / w);
    return (c % n + n) % n;
}

/* ---------------------------------------------------------------------------
 * System state.  Positions X are kept in particle-id order, X[pid*dim + a].
 * ------------------------------------------------------------------------- */
typedef struct orc_sys {
    int dim;
    double L[3];
    int64_t N;
    double *X;      /* positions of P (accepted configuration) */
    double *r;      /* base radii; R_i = lambda * r_i */
    double rmax;
    double lam;     /* scale of P */
    double lam_t;   /* target scale */
    double c_w, c_m;
    int N_k, N_l, N_shake;
    uint64_t seed;
    uint64_t sweep;  /* sweeps done so far: the Philox sweep counter */
    int literal;     /* 1: Alg 3 in plain id order */
    /* bins (Alg 2): cell-sorted ids, ascending id inside each cell */
    int64_t n[3];
    double w[3];
    int64_t ncells;
    int64_t *cell_start; /* ncells + 1 */
    int64_t *members;    /* N */
    int64_t cap_cells;
    /* counters */
    int64_t iters, accepted_iters, shake_iters, moves_accepted;
    /* diagnostics for the FP32 tolerance tests (NULL when not wanted) */
    double *margin;
    /* periodicity by image particles (orc_images.h) instead of the
     * minimum image */
    int images;
    orc_imgtab img;
} orc_sys;

static void bin(orc_sys *s, const double *X, const double lam_grid)
{
    orc_grid(s->dim, s->L, lam_grid, s->rmax, s->c_m, s->n, s->w);
    s->ncells = s->n[0] * s->n[1] * s->n[2];
    if (s->ncells + 1 > s->cap_cells) {
        free(s->cell_start);
        s->cap_cells = s->ncells + 1;
        s->cell_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)s->cap_cells);
    }
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->N > 0 ? s->N : 1));
    memset(s->cell_start, 0, sizeof(int64_t) * (size_t)(s->ncells + 1));
    for (int64_t i = 0; i < s->N; i++) {
        int64_t c[3] = {0, 0, 0};
        for (int a = 0; a < s->dim; a++) c[a] = cell_coord(X[i * s->dim + a], s->w[a], s->n[a]);
        cell_of[i] = c[0] + s->n[0] * (c[1] + s->n[1] * c[2]);
        s->cell_start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < s->ncells; c++) s->cell_start[c + 1] += s->cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)s->ncells);
    memcpy(fill, s->cell_start, sizeof(int64_t) * (size_t)s->ncells);
    /* ascending id order makes each cell's list sorted by id */
    for (int64_t i = 0; i < s->N; i++) s->members[fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
}

/* ---------------------------------------------------------------------------
 * Image particles (Section 2: the alternative to the minimum image, "after
 * each particle translation, boundary crossings are detected, and the
 * corresponding periodic images are added or removed"): the table of
 * orc_images.h.  A move removes the mover's entries and inserts those of its
 * new position, so the entries are never stale; collision tests take the
 * 3^d padded cells around the tested position's cell and plain (not
 * minimum-image) differences q - (x_t + s L).  The sweep order still comes
 * from the binning of the sweep's start.
 * ------------------------------------------------------------------------- */
static void tab_cell_of(const orc_imgtab *t, const double *x, int64_t c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int a = 0; a < t->dim; a++) c[a] = cell_coord(x[a], t->w[a], t->n[a]);
}

static void tab_insert(orc_imgtab *t, int64_t id, const int8_t *sh, int64_t pc)
{
    if (t->cnt[pc] == t->cap[pc]) {
        t->cap[pc] = t->cap[pc] ? 2 * t->cap[pc] : 8;
        t->id[pc] = (int64_t *)realloc(t->id[pc], sizeof(int64_t) * (size_t)t->cap[pc]);
        t->sh[pc] = (int8_t *)realloc(t->sh[pc], 3 * (size_t)t->cap[pc]);
    }
    int64_t k = t->cnt[pc]++;
    t->id[pc][k] = id;
    memcpy(&t->sh[pc][3 * k], sh, 3);
}

static void tab_remove(orc_imgtab *t, int64_t id, const int8_t *sh, int64_t pc)
{
    for (int64_t k = 0; k < t->cnt[pc]; k++)
        if (t->id[pc][k] == id && memcmp(&t->sh[pc][3 * k], sh, 3) == 0) {
            int64_t last = --t->cnt[pc];
            t->id[pc][k] = t->id[pc][last];
            memcpy(&t->sh[pc][3 * k], &t->sh[pc][3 * last], 3);
            return;
        }
    abort(); /* an entry that should exist is missing: a bug of this file */
}

/* Calls fn for each entry (shift, padded cell) of particle id in cell c. */
static void tab_entries(orc_imgtab *t, const int64_t c[3], int64_t id,
                        void (*fn)(orc_imgtab *, int64_t, const int8_t *, int64_t))
{
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < t->dim; a++) {
        lo[a] = c[a] == t->n[a] - 1 ? -1 : 0;
        hi[a] = c[a] == 0 ? 1 : 0;
    }
    for (int sz = lo[2]; sz <= hi[2]; sz++)
        for (int sy = lo[1]; sy <= hi[1]; sy++)
            for (int sx = lo[0]; sx <= hi[0]; sx++) {
                const int8_t sh[3] = {(int8_t)sx, (int8_t)sy, (int8_t)sz};
                int64_t pc = 0, mul = 1;
                for (int a = 0; a < 3; a++) {
                    pc += (a < t->dim ? c[a] + sh[a] * t->n[a] + 1 : 0) * mul;
                    mul *= t->pn[a];
                }
                fn(t, id, sh, pc);
            }
}

void orc_imgtab_free(orc_imgtab *t)
{
    for (int64_t c = 0; c < t->pcells; c++) {
        free(t->id[c]);
        free(t->sh[c]);
    }
    free(t->id);
    free(t->sh);
    free(t->cnt);
    free(t->cap);
    t->id = NULL;
    t->sh = NULL;
    t->cnt = t->cap = NULL;
    t->pcells = 0;
}

void orc_imgtab_build(orc_imgtab *t, int dim, const int64_t n[3], const double w[3], const double *X, int64_t N)
{
    orc_imgtab_free(t);
    t->dim = dim;
    for (int a = 0; a < 3; a++) {
        t->n[a] = n[a];
        t->w[a] = w[a];
        t->pn[a] = a < dim ? n[a] + 2 : 1;
    }
    t->pcells = t->pn[0] * t->pn[1] * t->pn[2];
    t->cnt = (int64_t *)calloc((size_t)t->pcells, sizeof(int64_t));
    t->cap = (int64_t *)calloc((size_t)t->pcells, sizeof(int64_t));
    t->id = (int64_t **)calloc((size_t)t->pcells, sizeof(int64_t *));
    t->sh = (int8_t **)calloc((size_t)t->pcells, sizeof(int8_t *));
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3];
        tab_cell_of(t, &X[i * dim], c);
        tab_entries(t, c, i, tab_insert);
    }
}

void orc_imgtab_move(orc_imgtab *t, int64_t id, const double *old, const double *new_)
{
    int64_t c0[3], c1[3];
    tab_cell_of(t, old, c0);
    tab_cell_of(t, new_, c1);
    tab_entries(t, c0, id, tab_remove);
    tab_entries(t, c1, id, tab_insert);
}

int64_t orc_imgtab_near(const orc_imgtab *t, const double *x, int dx, int dy, int dz)
{
    int64_t c[3];
    tab_cell_of(t, x, c);
    const int dd[3] = {dx, dy, dz};
    int64_t pc = 0, mul = 1;
    for (int a = 0; a < 3; a++) {
        pc += (a < t->dim ? c[a] + dd[a] + 1 : 0) * mul;
        mul *= t->pn[a];
    }
    return pc;
}

int64_t orc_imgtab_verify(orc_imgtab *t, const double *X, int64_t N)
{
    orc_imgtab r = {0};
    orc_imgtab_build(&r, t->dim, t->n, t->w, X, N);
    int64_t bad = 0;
    for (int64_t c = 0; c < t->pcells; c++) {
        int ok = t->cnt[c] == r.cnt[c];
        for (int64_t k = 0; ok && k < t->cnt[c]; k++) {
            int found = 0;
            for (int64_t m = 0; m < r.cnt[c] && !found; m++)
                found = t->id[c][k] == r.id[c][m] && memcmp(&t->sh[c][3 * k], &r.sh[c][3 * m], 3) == 0;
            ok = found;
        }
        bad += !ok;
    }
    orc_imgtab_free(&r);
    return bad;
}

int64_t orc_imgtab_images(const orc_imgtab *t)
{
    int64_t n = 0;
    for (int64_t c = 0; c < t->pcells; c++)
        for (int64_t k = 0; k < t->cnt[c]; k++) n += t->sh[c][3 * k] || t->sh[c][3 * k + 1] || t->sh[c][3 * k + 2];
    return n;
}

/* Alg 5 with image particles: any entry other than pid's own in the 3^d
 * padded cells around q's cell within Rq + R_t of q (plain differences to
 * x_t + s L).  Margins as collide() below. */
static int collide_images(const orc_sys *s, const double *X, double lam, const double *q, double Rq, int64_t pid,
                          double *mg)
{
    const orc_imgtab *tb = &s->img;
    int zlo = s->dim == 3 ? -1 : 0, zhi = s->dim == 3 ? 1 : 0;
    int hit = 0;
    double best_hit = -1.0, best_miss = INFINITY;
    for (int sz = zlo; sz <= zhi; sz++)
        for (int sy = -1; sy <= 1; sy++)
            for (int sx = -1; sx <= 1; sx++) {
                int64_t pc = orc_imgtab_near(tb, q, sx, sy, sz);
                for (int64_t k = 0; k < tb->cnt[pc]; k++) {
                    int64_t t = tb->id[pc][k];
                    if (t == pid) continue;
                    const int8_t *sh = &tb->sh[pc][3 * k];
                    double d[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < s->dim; a++) {
                        double y = X[t * s->dim + a] + (double)sh[a] * s->L[a];
                        d[a] = q[a] - y;
                    }
                    double ss = d[0] * d[0] + d[1] * d[1];
                    if (s->dim == 3) ss = ss + d[2] * d[2];
                    double S = sqrt(ss);
                    double Rsum = Rq + lam * s->r[t];
                    if (S <= Rsum) {
                        if (!mg) return 1;
                        hit = 1;
                        double m = (Rsum - S) / Rsum;
                        if (m > best_hit) best_hit = m;
                    } else if (mg) {
                        double m = (S - Rsum) / Rsum;
                        if (m < best_miss) best_miss = m;
                    }
                }
            }
    if (mg) *mg = hit ? best_hit : best_miss;
    return hit;
}

/* Alg 5: does a particle of radius Rq at position q (id pid) collide with any
 * other particle listed in the 3^d cells around q's cell?  X holds current
 * positions; the lists may be stale by at most one migration step, which the
 * cell size (2.5 R_max + c_m) covers.  When margin tracking is on, every
 * candidate is visited and *mg receives the decision margin: for a collision
 * the largest (Rsum - S)/Rsum, otherwise the smallest (S - Rsum)/Rsum. */
static int collide(const orc_sys *s, const double *X, double lam, const double *q,
                   double Rq, int64_t pid, double *mg)
{
    if (s->images) return collide_images(s, X, lam, q, Rq, pid, mg);
    int64_t c[3] = {0, 0, 0};
    for (int a = 0; a < s->dim; a++) c[a] = cell_coord(q[a], s->w[a], s->n[a]);
    int zlo = s->dim == 3 ? -1 : 0, zhi = s->dim == 3 ? 1 : 0;
    int hit = 0;
    double best_hit = -1.0, best_miss = INFINITY;
    for (int sx = -1; sx <= 1; sx++)
        for (int sy = -1; sy <= 1; sy++)
            for (int sz = zlo; sz <= zhi; sz++) {
                int64_t nx = (c[0] + sx + s->n[0]) % s->n[0];
                int64_t ny = (c[1] + sy + s->n[1]) % s->n[1];
                int64_t nz = (c[2] + sz + s->n[2]) % s->n[2];
                int64_t cell = nx + s->n[0] * (ny + s->n[1] * nz);
                for (int64_t k = s->cell_start[cell]; k < s->cell_start[cell + 1]; k++) {
                    int64_t t = s->members[k];
                    if (t == pid) continue;
                    double d[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < s->dim; a++) {
                        double da = q[a] - X[t * s->dim + a];
                        if (da > 0.5 * s->L[a]) da -= s->L[a];
                        if (da < -0.5 * s->L[a]) da += s->L[a];
                        d[a] = da;
                    }
                    double ss = d[0] * d[0] + d[1] * d[1];
                    if (s->dim == 3) ss = ss + d[2] * d[2];
                    double S = sqrt(ss);
                    double Rsum = Rq + lam * s->r[t];
                    if (S <= Rsum) {
                        if (!mg) return 1;
                        hit = 1;
                        double m = (Rsum - S) / Rsum;
                        if (m > best_hit) best_hit = m;
                    } else if (mg) {
                        double m = (S - Rsum) / Rsum;
                        if (m < best_miss) best_miss = m;
                    }
                }
            }
    if (mg) *mg = hit ? best_hit : best_miss;
    return hit;
}

/* Alg 3 for one particle: up to N_l trial moves of length c_m from q_old;
 * the first collision-free trial is kept, otherwise q_old is restored. */
static int move_particle(orc_sys *s, double *X, double lam, int64_t pid)
{
    double q_old[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0}, u[3];
    for (int a = 0; a < s->dim; a++) q_old[a] = X[pid * s->dim + a];
    double Rq = lam * s->r[pid];
    double pmin = INFINITY;
    for (int l = 0; l < s->N_l; l++) {
        orc_unit_dir(s->seed, s->sweep, (uint64_t)pid, (uint64_t)l, s->dim, u);
        for (int a = 0; a < s->dim; a++) q[a] = orc_wrap(q_old[a] + s->c_m * u[a], s->L[a]);
        double mg = 0.0;
        int hit = collide(s, X, lam, q, Rq, pid, s->margin ? &mg : NULL);
        if (s->margin && mg < pmin) pmin = mg;
        if (!hit) {
            if (s->images) orc_imgtab_move(&s->img, pid, q_old, q);
            for (int a = 0; a < s->dim; a++) X[pid * s->dim + a] = q[a];
            if (s->margin) s->margin[pid] = pmin;
            return 1;
        }
    }
    if (s->margin) s->margin[pid] = pmin;
    return 0;
}

/* One sweep of Alg 3 over all particles of X at radii lam * r, on bins built
 * from X with the grid of lam_grid.  Advances the sweep counter. */
static int64_t sweep_once(orc_sys *s, double *X, double lam, double lam_grid)
{
    bin(s, X, lam_grid);
    if (s->images) orc_imgtab_build(&s->img, s->dim, s->n, s->w, X, s->N);
    int64_t acc = 0;
    if (s->literal) {
        for (int64_t pid = 0; pid < s->N; pid++) acc += move_particle(s, X, lam, pid);
    } else {
        int ncol = s->dim == 3 ? 27 : 9;
        for (int chi = 0; chi < ncol; chi++) {
            int64_t a0 = chi % 3, a1 = (chi / 3) % 3, a2 = chi / 9;
            for (int64_t cz = a2; cz < s->n[2]; cz += 3)
                for (int64_t cy = a1; cy < s->n[1]; cy += 3)
                    for (int64_t cx = a0; cx < s->n[0]; cx += 3) {
                        int64_t cell = cx + s->n[0] * (cy + s->n[1] * cz);
                        for (int64_t k = s->cell_start[cell]; k < s->cell_start[cell + 1]; k++)
                            acc += move_particle(s, X, lam, s->members[k]);
                    }
        }
    }
    s->sweep++;
    s->moves_accepted += acc;
    return acc;
}

/* Alg 6 with a full count: number of particles that collide with another. */
static int64_t check_count(orc_sys *s, const double *X, double lam, double lam_grid, uint8_t *flags)
{
    bin(s, X, lam_grid);
    if (s->images) orc_imgtab_build(&s->img, s->dim, s->n, s->w, X, s->N);
    int64_t cnt = 0;
    for (int64_t pid = 0; pid < s->N; pid++) {
        int hit = collide(s, X, lam, &X[pid * s->dim], lam * s->r[pid], pid, NULL);
        if (flags) flags[pid] = (uint8_t)hit;
        cnt += hit;
    }
    return cnt;
}

/* ---------------------------------------------------------------------------
 * Public entry points (ctypes).
 * ------------------------------------------------------------------------- */
orc_sys *orc_create(int dim, const double L[3], int64_t N, const double *X, const double *r,
                    double lam, double lam_t, double c_w, double c_m, int N_k, int N_l,
                    int N_shake, uint64_t seed, uint64_t sweep, int literal)
{
    orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
    s->dim = dim;
    for (int a = 0; a < 3; a++) s->L[a] = a < dim ? L[a] : 1.0;
    s->N = N;
    size_t nn = (size_t)(N > 0 ? N : 1);
    s->X = (double *)malloc(sizeof(double) * nn * (size_t)dim);
    s->r = (double *)malloc(sizeof(double) * nn);
    s->members = (int64_t *)malloc(sizeof(int64_t) * nn);
    if (N > 0) {
        memcpy(s->X, X, sizeof(double) * (size_t)N * (size_t)dim);
        memcpy(s->r, r, sizeof(double) * (size_t)N);
    }
    s->rmax = 0.0;
    for (int64_t i = 0; i < N; i++)
        if (r[i] > s->rmax) s->rmax = r[i];
    s->lam = lam;
    s->lam_t = lam_t;
    s->c_w = c_w;
    s->c_m = c_m;
    s->N_k = N_k;
    s->N_l = N_l;
    s->N_shake = N_shake;
    s->seed = seed;
    s->sweep = sweep;
    s->literal = literal;
    return s;
}

void orc_destroy(orc_sys *s)
{
    if (!s) return;
    orc_imgtab_free(&s->img);
    free(s->X);
    free(s->r);
    free(s->members);
    free(s->cell_start);
    free(s);
}

void orc_get_x(const orc_sys *s, double *X) { memcpy(X, s->X, sizeof(double) * (size_t)s->N * (size_t)s->dim); }
void orc_set_x(orc_sys *s, const double *X) { memcpy(s->X, X, sizeof(double) * (size_t)s->N * (size_t)s->dim); }
double orc_get_lambda(const orc_sys *s) { return s->lam; }
void orc_set_lambda(orc_sys *s, double lam) { s->lam = lam; }
uint64_t orc_get_sweep(const orc_sys *s) { return s->sweep; }
void orc_set_margin(orc_sys *s, double *margin) { s->margin = margin; }

/* Periodicity by image particles (1) or by the minimum image (0). */
void orc_set_images(orc_sys *s, int on) { s->images = on ? 1 : 0; }

/* Compares the image entries kept move by move during the last sweep with
 * a rebuild from X (the configuration swept last); the number of
 * mismatching padded cells (0 when consistent), -1 outside the images mode.
 * For the tests of the maintenance. */
int64_t orc_images_verify(orc_sys *s, const double *X)
{
    if (!s->images || !s->img.cnt) return -1;
    return orc_imgtab_verify(&s->img, X, s->N);
}

/* Image entries (shift != 0) currently held, or -1 outside the images mode. */
int64_t orc_images_count(const orc_sys *s)
{
    if (!s->images || !s->img.cnt) return -1;
    return orc_imgtab_images(&s->img);
}

/* counters: iters, accepted iterations, shake iterations, accepted moves, sweeps */
void orc_get_counters(const orc_sys *s, int64_t out[5])
{
    out[0] = s->iters;
    out[1] = s->accepted_iters;
    out[2] = s->shake_iters;
    out[3] = s->moves_accepted;
    out[4] = (int64_t)s->sweep;
}

/* Volume (area) fraction of P: lambda^d sum v(r_i) / prod L, with v the disk
 * area or sphere volume, summed in id order (Alg 1). */
double orc_phi(const orc_sys *s, double lam)
{
    double S0 = 0.0;
    for (int64_t i = 0; i < s->N; i++) {
        double ri = s->r[i];
        S0 += s->dim == 2 ? M_PI * ri * ri : (4.0 / 3.0) * M_PI * ri * ri * ri;
    }
    double V = s->L[0] * s->L[1];
    if (s->dim == 3) V = V * s->L[2];
    double ld = lam * lam;
    if (s->dim == 3) ld = ld * lam;
    return ld * S0 / V;
}

/* Scale at which P reaches volume fraction phi: (phi prod L / S0)^(1/d),
 * square root in 2D and cube root in 3D (Alg 1 with the
 * multiplicative swelling reading). */
double orc_lambda_for_phi(const orc_sys *s, double phi)
{
    double p1 = orc_phi(s, 1.0);
    double q = phi / p1;
    return s->dim == 2 ? sqrt(q) : cbrt(q);
}

/* One sweep of Alg 3 on P at its own scale, grid from that scale (the
 * relaxation move with c_w = 0).  Returns the number of accepted moves. */
int64_t orc_sweep(orc_sys *s) { return sweep_once(s, s->X, s->lam, s->lam); }

/* Alg 6 on P at its own scale: number of colliding particles, flags by id. */
int64_t orc_check(orc_sys *s, uint8_t *flags) { return check_count(s, s->X, s->lam, s->lam, flags); }

/* All colliding pairs (i < j) of P at its own scale, lexicographic order.
 * Writes at most cap pairs; returns the total number. */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_pairs(orc_sys *s, int64_t *ij, int64_t cap)
{
    bin(s, s->X, s->lam);
    if (s->images) orc_imgtab_build(&s->img, s->dim, s->n, s->w, s->X, s->N);
    int64_t cnt = 0;
    int64_t *part = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->N > 0 ? s->N : 1));
    int zlo = s->dim == 3 ? -1 : 0, zhi = s->dim == 3 ? 1 : 0;
    for (int64_t i = 0; i < s->N; i++) {
        const double *q = &s->X[i * s->dim];
        double Ri = s->lam * s->r[i];
        int64_t c[3] = {0, 0, 0};
        for (int a = 0; a < s->dim; a++) c[a] = cell_coord(q[a], s->w[a], s->n[a]);
        int64_t np = 0;
        if (s->images) {
            /* image particles: entries of the 3^d padded cells around i's
             * cell, plain differences to x_t + s L */
            const orc_imgtab *tb = &s->img;
            for (int sz = zlo; sz <= zhi; sz++)
                for (int sy = -1; sy <= 1; sy++)
                    for (int sx = -1; sx <= 1; sx++) {
                        int64_t pc = orc_imgtab_near(tb, q, sx, sy, sz);
                        for (int64_t k = 0; k < tb->cnt[pc]; k++) {
                            int64_t t = tb->id[pc][k];
                            if (t <= i) continue;
                            const int8_t *sh = &tb->sh[pc][3 * k];
                            double d[3] = {0.0, 0.0, 0.0};
                            for (int a = 0; a < s->dim; a++) d[a] = q[a] - (s->X[t * s->dim + a] + (double)sh[a] * s->L[a]);
                            double ss = d[0] * d[0] + d[1] * d[1];
                            if (s->dim == 3) ss = ss + d[2] * d[2];
                            if (sqrt(ss) <= Ri + s->lam * s->r[t]) part[np++] = t;
                        }
                    }
        }
        for (int sx = -1; sx <= 1 && !s->images; sx++)
            for (int sy = -1; sy <= 1; sy++)
                for (int sz = zlo; sz <= zhi; sz++) {
                    int64_t nx = (c[0] + sx + s->n[0]) % s->n[0];
                    int64_t ny = (c[1] + sy + s->n[1]) % s->n[1];
                    int64_t nz = (c[2] + sz + s->n[2]) % s->n[2];
                    int64_t cell = nx + s->n[0] * (ny + s->n[1] * nz);
                    for (int64_t k = s->cell_start[cell]; k < s->cell_start[cell + 1]; k++) {
                        int64_t t = s->members[k];
                        if (t <= i) continue;
                        double d[3] = {0.0, 0.0, 0.0};
                        for (int a = 0; a < s->dim; a++) {
                            double da = q[a] - s->X[t * s->dim + a];
                            if (da > 0.5 * s->L[a]) da -= s->L[a];
                            if (da < -0.5 * s->L[a]) da += s->L[a];
                            d[a] = da;
                        }
                        double ss = d[0] * d[0] + d[1] * d[1];
                        if (s->dim == 3) ss = ss + d[2] * d[2];
                        if (sqrt(ss) <= Ri + s->lam * s->r[t]) part[np++] = t;
                    }
                }
        qsort(part, (size_t)np, sizeof(int64_t), cmp_i64);
        for (int64_t k = 0; k < np; k++) {
            if (cnt < cap) {
                ij[2 * cnt] = i;
                ij[2 * cnt + 1] = part[k];
            }
            cnt++;
        }
    }
    free(part);
    return cnt;
}

/* One iteration of Alg 1.  Returns 1 if the swollen
 * configuration was accepted, 0 if it was discarded and P shaken, 2 if P was
 * already at the target scale (nothing to do).  info (may be NULL) receives
 * {k sweeps used, colliding count after the last check, shake sweeps}. */
int orc_iterate(orc_sys *s, int64_t info[3])
{
    if (s->lam >= s->lam_t) return 2;
    s->iters++;
    double lam_q = s->lam * (1.0 + s->c_w);
    if (lam_q > s->lam_t) lam_q = s->lam_t;
    size_t bytes = sizeof(double) * (size_t)s->N * (size_t)s->dim;
    double *Q = (double *)malloc(bytes > 0 ? bytes : sizeof(double));
    if (bytes) memcpy(Q, s->X, bytes);
    int64_t cnt = -1;
    int k;
    for (k = 1; k <= s->N_k; k++) {
        sweep_once(s, Q, lam_q, lam_q);
        cnt = check_count(s, Q, lam_q, lam_q, NULL);
        if (cnt == 0) break;
    }
    int accepted = cnt == 0;
    int ksw = accepted ? k : s->N_k;
    if (accepted) {
        if (bytes) memcpy(s->X, Q, bytes);
        s->lam = lam_q;
        s->accepted_iters++;
    } else {
        for (int j = 0; j < s->N_shake; j++) sweep_once(s, s->X, s->lam, lam_q);
        s->shake_iters++;
    }
    free(Q);
    if (info) {
        info[0] = ksw;
        info[1] = cnt;
        info[2] = accepted ? 0 : s->N_shake;
    }
    return accepted;
}

/* Alg 1: iterate until P reaches the target scale or max_iters iterations
 * were run.  Returns the number of iterations run. */
int64_t orc_run(orc_sys *s, int64_t max_iters)
{
    int64_t it = 0;
    while (s->lam < s->lam_t && it < max_iters) {
        orc_iterate(s, NULL);
        it++;
    }
    return it;
}

/* ---------------------------------------------------------------------------
 * Brute force O(N^2) overlap pairs and minimum gap: the certification of the
 * final state (termination, Section 2 step e), independent of any cell list.
 * Pairs i < j with sqrt(|d|^2) <= R_i + R_j under the minimum image; returns
 * the count, writes up to cap pairs, and the smallest S - (R_i + R_j).
 * ------------------------------------------------------------------------- */
int64_t orc_pairs_brute(int dim, const double L[3], int64_t N, const double *X, const double *R,
                        int64_t *ij, int64_t cap, double *min_gap)
{
    int64_t cnt = 0;
    double mg = INFINITY;
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = i + 1; j < N; j++) {
            double d[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < dim; a++) {
                double da = X[i * dim + a] - X[j * dim + a];
                if (da > 0.5 * L[a]) da -= L[a];
                if (da < -0.5 * L[a]) da += L[a];
                d[a] = da;
            }
            double ss = d[0] * d[0] + d[1] * d[1];
            if (dim == 3) ss = ss + d[2] * d[2];
            double S = sqrt(ss);
            double Rsum = R[i] + R[j];
            if (S - Rsum < mg) mg = S - Rsum;
            if (S <= Rsum) {
                if (cnt < cap) {
                    ij[2 * cnt] = i;
                    ij[2 * cnt + 1] = j;
                }
                cnt++;
            }
        }
    if (min_gap) *min_gap = mg;
    return cnt;
}

/* Cell-list certification for sizes where O(N^2) is too slow: colliding pair
 * count and minimum gap S - (R_i + R_j) over pairs within one cell of each
 * other, on a grid with cells at least 2 R_max wide (3 per axis at least). */
int64_t orc_certify(int dim, const double L[3], int64_t N, const double *X, const double *R,
                    double *min_gap)
{
    double Rmax = 0.0;
    for (int64_t i = 0; i < N; i++)
        if (R[i] > Rmax) Rmax = R[i];
    int64_t n[3] = {1, 1, 1};
    double w[3] = {L[0], L[1], dim == 3 ? L[2] : 1.0};
    /* at most about 4 N cells in total */
    int64_t kcap = (int64_t)pow(4.0 * (double)(N > 0 ? N : 1), 1.0 / (double)dim) + 3;
    for (int a = 0; a < dim; a++) {
        int64_t k = (int64_t)(L[a] / (2.0 * Rmax * 1.000001));
        if (k > kcap) k = kcap;
        if (k < 3) k = 3;
        n[a] = k;
        w[a] = L[a] / (double)k;
    }
    int64_t nc = n[0] * n[1] * n[2];
    int64_t *start = (int64_t *)calloc((size_t)(nc + 1), sizeof(int64_t));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3] = {0, 0, 0};
        for (int a = 0; a < dim; a++) c[a] = cell_coord(X[i * dim + a], w[a], n[a]);
        cell_of[i] = c[0] + n[0] * (c[1] + n[1] * c[2]);
        start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) start[c + 1] += start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    memcpy(fill, start, sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < N; i++) mem[fill[cell_of[i]]++] = i;
    free(fill);
    int64_t cnt = 0;
    double mg = INFINITY;
    int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3];
        c[0] = cell_of[i] % n[0];
        c[1] = (cell_of[i] / n[0]) % n[1];
        c[2] = cell_of[i] / (n[0] * n[1]);
        for (int sx = -1; sx <= 1; sx++)
            for (int sy = -1; sy <= 1; sy++)
                for (int sz = zlo; sz <= zhi; sz++) {
                    int64_t cell = (c[0] + sx + n[0]) % n[0] +
                                   n[0] * ((c[1] + sy + n[1]) % n[1] + n[1] * ((c[2] + sz + n[2]) % n[2]));
                    for (int64_t k = start[cell]; k < start[cell + 1]; k++) {
                        int64_t j = mem[k];
                        if (j <= i) continue;
                        double d[3] = {0.0, 0.0, 0.0};
                        for (int a = 0; a < dim; a++) {
                            double da = X[i * dim + a] - X[j * dim + a];
                            if (da > 0.5 * L[a]) da -= L[a];
                            if (da < -0.5 * L[a]) da += L[a];
                            d[a] = da;
                        }
                        double ss = d[0] * d[0] + d[1] * d[1];
                        if (dim == 3) ss = ss + d[2] * d[2];
                        double S = sqrt(ss);
                        double Rsum = R[i] + R[j];
                        if (S - Rsum < mg) mg = S - Rsum;
                        if (S <= Rsum) cnt++;
                    }
                }
    }
    free(start);
    free(cell_of);
    free(mem);
    if (min_gap) *min_gap = mg;
    return cnt;
}
