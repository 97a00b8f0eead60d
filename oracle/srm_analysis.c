/*
 * srm_analysis.c -- FP64 reference of the structure descriptors used to
 * assess generated microstructures (Section 3.2: nearest-neighbour distance
 * distributions, Fig. 4d; local volume fraction = particle area or volume
 * over the area or volume of its Voronoi cell, Figs. 5 and 7) and the radial
 * distribution function of the centres.  TEST INFRASTRUCTURE ONLY: plain
 * brute-force loops over all pairs (or all voxels x particles), usable for
 * a few thousand particles.
 *
 * Conventions shared with the definitions of the method (srm_oracle.c):
 * periodic box [0, L_a), minimum-image difference per axis (d > L/2 then
 * d -= L, d < -L/2 then d += L, with L/2 = 0.5 L), squared distance summed
 * in axis order, distance = correctly rounded square root; gcc -O2
 * -ffp-contract=off, so every operation is one IEEE binary64 operation.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static double mi(double d, double L, double hL)
{
    if (d > hL) d -= L;
    if (d < -hL) d += L;
    return d;
}

static double dist2(int dim, const double *L, const double *hL, const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < dim; k++) {
        const double d = mi(a[k] - b[k], L[k], hL[k]);
        s = k == 0 ? d * d : s + d * d;
    }
    return s;
}

/* Nearest neighbours of every particle: the smallest centre distance S_ij
 * over j != i (nn_dist, partner nn_id; ties to the smaller j) and the
 * smallest surface gap S_ij - (R_i + R_j) over j != i (gap). */
void orc_nn(int dim, const double L[3], int64_t N, const double *X, const double *R, double *nn_dist,
            int64_t *nn_id, double *gap)
{
    double hL[3];
    for (int k = 0; k < 3; k++) hL[k] = 0.5 * L[k];
    for (int64_t i = 0; i < N; i++) {
        double best = INFINITY, bestgap = INFINITY;
        int64_t bj = -1;
        for (int64_t j = 0; j < N; j++) {
            if (j == i) continue;
            const double S = sqrt(dist2(dim, L, hL, X + i * dim, X + j * dim));
            if (S < best) {
                best = S;
                bj = j;
            }
            const double g = S - (R[i] + R[j]);
            if (g < bestgap) bestgap = g;
        }
        nn_dist[i] = best;
        if (nn_id) nn_id[i] = bj;
        gap[i] = bestgap;
    }
}

/* Radial distribution of the centres: counts[k] = number of ordered pairs
 * (i, j), i != j, with S_ij in [k dr, (k+1) dr), dr = r_max / bins, bin
 * k = floor(S / dr); g[k] = counts[k] V / (N (N - 1) V_k) with V_k the
 * volume (area) of shell k.  Returns the number of pairs below r_max. */
int64_t orc_rdf(int dim, const double L[3], int64_t N, const double *X, double r_max, int bins, int64_t *counts,
                double *g)
{
    double hL[3];
    for (int k = 0; k < 3; k++) hL[k] = 0.5 * L[k];
    const double dr = r_max / (double)bins;
    memset(counts, 0, sizeof(int64_t) * (size_t)bins);
    int64_t tot = 0;
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = i + 1; j < N; j++) {
            const double S = sqrt(dist2(dim, L, hL, X + i * dim, X + j * dim));
            if (!(S < r_max)) continue;
            const int64_t b = (int64_t)floor(S / dr);
            if (b >= bins) continue;
            counts[b] += 2;
            tot += 2;
        }
    double V = 1.0;
    for (int k = 0; k < dim; k++) V *= L[k];
    const double pi = 3.14159265358979323846;
    for (int b = 0; b < bins; b++) {
        const double r0 = b * dr, r1 = (b + 1) * dr;
        const double shell = dim == 2 ? pi * (r1 * r1 - r0 * r0) : 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
        g[b] = (double)counts[b] * V / ((double)N * (double)(N - 1) * shell);
    }
    return tot;
}

/* Discrete periodic Voronoi tessellation on M[0] x M[1] (x M[2]) voxels:
 * voxel centre c_a = (i_a + 0.5) h_a with h_a = L_a / M_a belongs to the
 * particle with the smallest squared minimum-image distance (ties to the
 * smaller id).  count[j] = voxels of particle j; lvf[j] = v_j / (count[j]
 * prod h_a) with v_j = pi R_j^2 (2D) or 4/3 pi R_j^3 (3D), +inf if the cell
 * is empty.  Voxel order: x fastest. */
void orc_voronoi_lvf(int dim, const double L[3], int64_t N, const double *X, const double *R, const int32_t M[3],
                     int64_t *count, double *lvf)
{
    double hL[3], h[3];
    for (int k = 0; k < 3; k++) {
        hL[k] = 0.5 * L[k];
        h[k] = L[k] / (double)(k < dim ? M[k] : 1);
    }
    memset(count, 0, sizeof(int64_t) * (size_t)N);
    const int64_t mz = dim == 3 ? M[2] : 1;
    for (int64_t iz = 0; iz < mz; iz++)
        for (int64_t iy = 0; iy < M[1]; iy++)
            for (int64_t ix = 0; ix < M[0]; ix++) {
                const double c[3] = {((double)ix + 0.5) * h[0], ((double)iy + 0.5) * h[1],
                                     ((double)iz + 0.5) * h[2]};
                double best = INFINITY;
                int64_t bj = -1;
                for (int64_t j = 0; j < N; j++) {
                    const double s = dist2(dim, L, hL, c, X + j * dim);
                    if (s < best) {
                        best = s;
                        bj = j;
                    }
                }
                if (bj >= 0) count[bj]++;
            }
    double hv = 1.0;
    for (int k = 0; k < dim; k++) hv *= h[k];
    const double pi = 3.14159265358979323846;
    for (int64_t j = 0; j < N; j++) {
        const double v = dim == 2 ? pi * R[j] * R[j] : 4.0 / 3.0 * pi * R[j] * R[j] * R[j];
        lvf[j] = count[j] ? v / ((double)count[j] * hv) : INFINITY;
    }
}
