/*
 * srm_platelet.h -- C interface of SRM for thin circular platelets
 * (Tarasovs, Section 3.3 "Application example"): the method of Algorithms
 * 1-6 with the geometry-dependent collision routine replaced by a test for
 * spherodisks and the migration move extended by a small rotation.
 *
 * Geometry.  A spherodisk is the set of points within distance t of a flat
 * circular disk of radius a (centre x, unit normal u).  Its diameter is
 * D = 2 (a + t), its thickness 2 t, its aspect ratio D / (2 t).  All platelets
 * of a handle share the base sizes (a0, t0); the scale lambda of Algorithm 1
 * multiplies both (a = lambda a0, t = lambda t0), so swelling keeps the
 * shape.  The non-dimensional number density of Eq. 1 is rho = N D^3 / V,
 * V the box volume.
 *
 * Contact.  Two platelets collide when the distance between their disks is
 * at most t_i + t_j.  The library decides this on the rims of the two disks
 * (the distance between two disks is reached at a rim point of one of them)
 * by bisection with a certified lower bound, each of a rim's 8 first-level
 * arcs on its own; a near-contact that the bisection cannot resolve within
 * 2^-20 of the circle or 512 evaluations of an arc counts as contact.  Cheap exact separations come first (bounding
 * spheres, slabs along the two normals).  The test runs in binary32 on the
 * pair's relative geometry (centre difference formed in binary64 under the
 * minimum image, then rounded) against the threshold t_i + t_j + 2^-16 a:
 * the widening exceeds the binary32 rounding of the test, so every pair
 * closer than t_i + t_j is found; pairs within the widening count as
 * touching.  Centres, normals, draws and moves are binary64.
 *
 * Move.  Try l of Algorithm 3 moves the centre by c_m u (u a uniform
 * direction, the same draw as for spheres) and turns the normal to
 * (n + c_r v) / |n + c_r v| with v a second uniform direction (the same
 * Philox4x32-10 counter with the top bit of its fourth word set).  c_r = 0
 * keeps orientations fixed.
 *
 * Order and cells.  Cells are sized from the bounding sphere,
 * 2.5 lambda (a0 + t0) + c_m, n = 3 max(1, floor(L / (3 cellSize))) per axis;
 * each sweep visits the platelets in the canonical coloured order (colour
 * sum_a (c_a mod 3) 3^a ascending, cells of a colour, platelets of a cell by
 * ascending id).  Results are bit-identical to the FP64 reference for the
 * same inputs.
 *
 * Conventions are those of srm.h: status codes (srm_status), messages from
 * srm_last_error(), caller-owned host arrays copied in and out, all device
 * work ordered on the handle's CUDA stream, functions that return host
 * results synchronise that stream, one thread per handle at a time.  Arrays
 * of centres and normals are n x 3 doubles in particle-id order.
 */
#ifndef SRM_PLATELET_H
#define SRM_PLATELET_H

#include <stdint.h>

#include "srm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srm_plt srm_plt;

typedef struct srm_plt_params {
    double c_w;          /* swelling rate: lambda <- lambda (1 + c_w)          */
    double c_m;          /* migration step length (absolute), > 0              */
    double c_r;          /* rotation rate in [0, 1): n <- (n + c_r v)/|.|      */
    int32_t N_k;         /* sweeps tried per iteration before the shake        */
    int32_t N_l;         /* trial moves per platelet and sweep, 1..65535       */
    int32_t N_shake;     /* sweeps of the shake step                           */
    int32_t wait_limit;  /* polls of one cell-to-cell dependency in a sweep    */
                         /* before SRM_E_DEVICE_TIMEOUT (0: 2^22; < 0: give    */
                         /* up at the first dependency -- for tests)           */
    uint64_t sweep0;     /* first value of the sweep counter                   */
    int32_t images;      /* periodicity (Section 2): 0 the minimum image of    */
                         /* the centre difference; 1 image platelets: the      */
                         /* difference to a platelet near a face is taken to   */
                         /* its periodic image, (x_j + s L) - x_i, one         */
                         /* rounding per axis                                  */
    int32_t sweep_kernel; /* 0: sweeps and checks with a block per cell and   */
                         /* the 27 cells around it in shared memory wherever   */
                         /* that set holds every platelet a trial can touch    */
                         /* (stencil half-width 1 and 2 (a + t) + 2^-15 a +    */
                         /* 2 c_m below the cell width), else a warp per cell  */
                         /* (sweep) and a thread per platelet (check) reading  */
                         /* global memory; 1: always the latter.  Same results */
} srm_plt_params;

/* Defaults: c_w = 0.01, c_m = 0 (must be set), c_r = 0, N_k = N_l =
 * N_shake = 10, wait_limit 0, sweep0 0. */
void srm_plt_params_default(srm_plt_params *p);

/* Scale lambda at which n platelets of base sizes (a0, t0) in the box reach
 * the number density rho of Eq. 1: (rho V / n)^(1/3) / (2 (a0 + t0)).
 * SRM_E_ARG for n < 1, sizes or box <= 0, rho <= 0.  Host only. */
srm_status srm_plt_lambda_for_density(const double box[3], int64_t n, double a0, double t0, double rho,
                                      double *lambda);

/* Creates a platelet RVE in the periodic box [0, L_0) x [0, L_1) x [0, L_2):
 * n platelets with centres x (in the box) and normals u (unit vectors,
 * used as given), base sizes a0 > 0, t0 > 0, starting scale lambda0 > 0
 * (the starting state must be free of collisions at that scale), target
 * scale lambda_t >= lambda0, seed of the draws, parameters p (NULL:
 * defaults, which leave c_m = 0 and fail), CUDA stream (NULL: the legacy
 * default stream).  Rejects (SRM_E_ARG): n < 1 or
 * >= 2^31, non-positive sizes or box, c_m <= 0, c_w < 0, c_r outside [0, 1),
 * N_k, N_l outside 1..65535, N_shake < 0, and boxes narrower than three
 * cells of the final cell size 2.5 lambda_t (a0 + t0) + c_m on some axis. */
srm_status srm_plt_init(srm_plt **out, const double box[3], int64_t n, double a0, double t0, const double *x,
                        const double *u, double lambda0, double lambda_t, uint64_t seed, const srm_plt_params *p,
                        void *cuda_stream);

/* Replaces the migration and control parameters between phases (for
 * example the relaxation with c_w = 0 and a larger c_m of Section 3.3).
 * p->sweep0 is ignored (the sweep counter continues).  Same checks as
 * srm_plt_init. */
srm_status srm_plt_set_params(srm_plt *h, const srm_plt_params *p);

typedef struct srm_plt_step_info {
    int32_t result;        /* 1 swollen state accepted, 0 discarded and shaken, 2 at target */
    int32_t k_sweeps;      /* sweeps of the N_k loop                                        */
    int32_t shake_sweeps;  /* sweeps of the shake step                                      */
    int32_t reserved;
    int64_t colliding;     /* colliding platelets after the last check of the N_k loop      */
    int64_t moves;         /* accepted moves in this iteration                              */
    double lambda;         /* scale of P after the iteration                                */
    double rho;            /* number density of P (Eq. 1)                                   */
    uint64_t sweep;        /* sweep counter after the iteration                             */
} srm_plt_step_info;

/* One iteration of Algorithm 1 on the platelets: swell the copy Q to
 * min(lambda (1 + c_w), lambda_t), up to N_k rounds of (bin, sweep, check);
 * accept Q if a check finds no colliding pair, else discard it and run
 * N_shake sweeps on P (binned before each, on the grid of the swollen
 * scale).  out may be NULL. */
srm_status srm_plt_step(srm_plt *h, srm_plt_step_info *out);

typedef struct srm_plt_run_info {
    int64_t iterations, accepted, shaken, sweeps, moves;
    double lambda, rho;
    int32_t converged;  /* 1 if lambda reached lambda_t */
    int32_t reserved;
} srm_plt_run_info;

/* Iterates until lambda_t or max_iters iterations (<= 0: no cap).  Returns
 * SRM_E_NOT_CONVERGED when the cap stops it first. */
srm_status srm_plt_run_to_target(srm_plt *h, int64_t max_iters, srm_plt_run_info *out);

/* count sweeps of Algorithm 3 on P at its own scale (binned before each):
 * the relaxation with zero swelling.  accepted (may be NULL) receives the
 * number of accepted moves. */
srm_status srm_plt_sweeps(srm_plt *h, int32_t count, int64_t *accepted);

/* Algorithm 6 on P at its own scale: number of colliding platelets and, if
 * flags is not NULL, one byte per platelet (1 = collides), id order. */
srm_status srm_plt_check(srm_plt *h, int64_t *colliding, uint8_t *flags);

/* Current state: centres and normals (n x 3, may be NULL), scale, number
 * density (Eq. 1) and sweep counter (each may be NULL). */
srm_status srm_plt_state(srm_plt *h, double *x, double *u, double *lambda, double *rho, uint64_t *sweep);

/* The contact decision alone, for m pairs: pair k has centre difference
 * dj[3k..3k+2] (minimum image already taken), unit normals ni and nj, disk
 * radius a and half-thickness t for both.  out[k] = 1 if they collide.
 * Host arrays; runs on the given stream with its own temporary buffers.
 * SRM_E_ARG for m outside [0, 2^31), a <= 0 or t <= 0. */
srm_status srm_plt_collide_pairs(const double *dj, const double *ni, const double *nj, int64_t m, double a,
                                 double t, uint8_t *out, void *cuda_stream);

/* Sweep kernels used so far: out[0] sweeps run by the block-per-cell kernel
 * with the staged neighbourhood, out[1] sweeps run by the warp-per-cell
 * kernel, out[2] cells the block-per-cell kernel moved from global memory
 * because their 27 cells held more than 1024 platelets.  Synchronises the
 * stream. */
srm_status srm_plt_sweep_stats(srm_plt *h, int64_t out[3]);

void srm_plt_destroy(srm_plt *h);

#ifdef __cplusplus
}
#endif

#endif
