/*
 * gen.c -- seeded synthetic inputs for SRM runs: particle radii and a
 * non-overlapping starting configuration by random sequential addition (RSA),
 * the initialisation the paper assumes before its main loop (Section 2: "the
 * procedure begins by placing the required number of inclusions at a low
 * initial volume fraction ... using the classical RSA algorithm").
 *
 * This file holds no step of the SRM method itself.  Both the FP64 reference
 * used by the tests and the product library's srm_init use it to build a
 * starting state, so that the two sides can be given identical inputs.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), a stream of its own, not the
 * generator that drives the migration moves.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } inp_rng;

static uint64_t sm64_next(inp_rng *g)
{
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in [0, 1) on a 2^-53 lattice */
static double uni(inp_rng *g) { return (double)(sm64_next(g) >> 11) * 0x1p-53; }

/* standard normal by the Box-Muller transform */
static double gauss(inp_rng *g)
{
    double u1;
    do { u1 = uni(g); } while (u1 <= 0.0);
    double u2 = uni(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static void rng_init(inp_rng *g, uint64_t seed, uint64_t tag)
{
    g->s = seed * 0xD1342543DE82EF95ULL + tag;
    sm64_next(g);
}

/* Radii drawn from a log-normal law with the given mean and standard
 * deviation of the radius itself, re-drawn until inside [lo, hi]. */
int inp_radii_lognormal(int64_t n, double mean, double sd, double lo, double hi,
                        uint64_t seed, double *out)
{
    inp_rng g;
    rng_init(&g, seed, 0x52414449ULL); /* "RADI" */
    double s2 = log(1.0 + (sd * sd) / (mean * mean));
    double mu = log(mean) - 0.5 * s2;
    double sg = sqrt(s2);
    for (int64_t i = 0; i < n; i++) {
        double r;
        int tries = 0;
        do {
            r = exp(mu + sg * gauss(&g));
            if (++tries > 1000000) return -1;
        } while (r < lo || r > hi);
        out[i] = r;
    }
    return 0;
}

static double wrap_into(double x, double L)
{
    x = fmod(x, L);
    if (x < 0.0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

/* Random sequential addition of n particles with radii R[i] into the
 * periodic box L (placed in index order).  mode 0: proposals uniform in the
 * box.  mode 1: n_clusters centres uniform in the box; particle i belongs to
 * a cluster drawn uniformly; its first proposal is the centre plus a Gaussian
 * offset g of standard deviation sigma per axis, and each rejected proposal
 * is retried one largest diameter further out along g (so that a particle
 * whose cluster core is already saturated settles on the edge of the core
 * after a bounded number of tries instead of waiting for a rare far draw).
 * A proposal is rejected when |d|^2 <= (R_i + R_j)^2 (1 + 1e-9) under the
 * minimum image for some placed j.  Returns 0, or -1 when a particle found
 * no place in max_attempts proposals. */
int inp_rsa(int dim, const double L[3], int64_t n, const double *R, uint64_t seed, int mode,
            int64_t n_clusters, double sigma, int64_t max_attempts, double *X)
{
    inp_rng g;
    rng_init(&g, seed, 0x52534121ULL); /* "RSA!" */
    double Rmax = 0.0;
    for (int64_t i = 0; i < n; i++)
        if (R[i] > Rmax) Rmax = R[i];
    int64_t nc[3] = {1, 1, 1};
    double w[3] = {1.0, 1.0, 1.0};
    int64_t kcap = (int64_t)pow(4.0 * (double)(n > 0 ? n : 1), 1.0 / (double)dim) + 3;
    for (int a = 0; a < dim; a++) {
        int64_t k = (int64_t)(L[a] / (2.0 * Rmax * 1.000001));
        if (k > kcap) k = kcap;
        if (k < 3) k = 3;
        nc[a] = k;
        w[a] = L[a] / (double)k;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; c++) head[c] = -1;
    double *cen = NULL;
    if (mode == 1) {
        if (n_clusters < 1) n_clusters = 1;
        cen = (double *)malloc(sizeof(double) * (size_t)n_clusters * 3);
        for (int64_t c = 0; c < n_clusters; c++)
            for (int a = 0; a < 3; a++) cen[c * 3 + a] = a < dim ? uni(&g) * L[a] : 0.0;
    }
    int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; i++) {
        int64_t cl = mode == 1 ? (int64_t)(uni(&g) * (double)n_clusters) : 0;
        if (cl >= n_clusters) cl = n_clusters - 1;
        int64_t att = 0;
        double off[3] = {0.0, 0.0, 0.0}, dir[3] = {0.0, 0.0, 0.0};
        if (mode == 1) {
            double nrm = 0.0;
            for (int a = 0; a < dim; a++) {
                off[a] = sigma * gauss(&g);
                nrm += off[a] * off[a];
            }
            nrm = sqrt(nrm);
            for (int a = 0; a < dim; a++) dir[a] = nrm > 0.0 ? off[a] / nrm : (a == 0 ? 1.0 : 0.0);
        }
        for (;;) {
            if (++att > max_attempts) { rc = -1; break; }
            double p[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < dim; a++) {
                if (mode == 1) p[a] = wrap_into(cen[cl * 3 + a] + off[a], L[a]);
                else p[a] = uni(&g) * L[a];
            }
            int64_t c[3] = {0, 0, 0};
            for (int a = 0; a < dim; a++) {
                c[a] = (int64_t)(p[a] / w[a]);
                if (c[a] >= nc[a]) c[a] = nc[a] - 1;
            }
            int ok = 1;
            for (int sx = -1; sx <= 1 && ok; sx++)
                for (int sy = -1; sy <= 1 && ok; sy++)
                    for (int sz = zlo; sz <= zhi && ok; sz++) {
                        int64_t cell = (c[0] + sx + nc[0]) % nc[0] +
                                       nc[0] * ((c[1] + sy + nc[1]) % nc[1] +
                                                nc[1] * ((c[2] + sz + nc[2]) % nc[2]));
                        for (int64_t j = head[cell]; j >= 0 && ok; j = next[j]) {
                            double d2 = 0.0;
                            for (int a = 0; a < dim; a++) {
                                double da = p[a] - X[j * dim + a];
                                if (da > 0.5 * L[a]) da -= L[a];
                                if (da < -0.5 * L[a]) da += L[a];
                                d2 += da * da;
                            }
                            double rs = R[i] + R[j];
                            if (d2 <= rs * rs * (1.0 + 1e-9)) ok = 0;
                        }
                    }
            if (!ok) {
                if (mode == 1)
                    for (int a = 0; a < dim; a++) off[a] += 2.0 * Rmax * dir[a];
                continue;
            }
            for (int a = 0; a < dim; a++) X[i * dim + a] = p[a];
            int64_t cell = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
            next[i] = head[cell];
            head[cell] = i;
            break;
        }
    }
    free(head);
    free(next);
    free(cen);
    return rc;
}

/* 64-bit words of the input stream for (seed, tag): used by the batched
 * ensemble recipe to draw per-RVE sizes and targets. */
void inp_uniforms(uint64_t seed, uint64_t tag, int64_t n, double *out)
{
    inp_rng g;
    rng_init(&g, seed, tag);
    for (int64_t i = 0; i < n; i++) out[i] = uni(&g);
}
