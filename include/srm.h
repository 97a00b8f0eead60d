/*
 * srm.h -- C interface of the GB300 implementation of Swelling and Random
 * Migration (SRM): generation of periodic representative volume elements
 * (RVEs) of non-overlapping disks (2D) or spheres (3D) at a target volume
 * fraction (Tarasovs, "Efficient generation of large-scale non-equilibrium
 * distributions of particles", Section 2, Algorithms 1-6).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an srm_status; no C++ exception crosses this
 *     interface.  On failure srm_last_error() returns a message for the
 *     calling thread.
 *   - Host pointers are caller-owned; the library copies what it needs and
 *     never keeps them.  Device memory of a handle is owned by the handle and
 *     released by srm_destroy (through the allocator given to srm_init, if
 *     any).
 *   - All device work of a handle is ordered on the CUDA stream given at
 *     creation.  Functions that return host results synchronise that stream.
 *   - A handle must not be used by two threads at once.
 *   - Positions are in [0, L) per axis, particle-id order, dim values per
 *     particle (x, y[, z]), double precision.
 *   - Radii: each particle has a base radius r_i; its radius is R_i =
 *     lambda * r_i with one scale factor lambda per RVE (the swelling of
 *     Algorithm 1, read as a multiplicative factor (1 + c_w) per
 *     iteration).
 */
#ifndef SRM_H
#define SRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum srm_status {
    SRM_OK = 0,
    SRM_E_ARG = 1,            /* invalid argument (message says which)          */
    SRM_E_NOMEM = 2,          /* device or host allocation failed                */
    SRM_E_CUDA = 3,           /* a CUDA call failed (message has the CUDA error) */
    SRM_E_NOT_CONVERGED = 4,  /* iteration cap reached before the target        */
    SRM_E_DEVICE_TIMEOUT = 5, /* a bounded device-side wait gave up              */
    SRM_E_CERTIFY_FAILED = 6, /* FP64 certification found overlapping pairs     */
    SRM_E_STATE = 7,          /* call not valid in the handle's current state   */
    SRM_E_INIT = 8            /* random sequential addition could not place all */
} srm_status;

/* Base radii.  SRM_RADII_EXPLICIT: r[0..n) given.  SRM_RADII_MONO: every
 * r_i = mean.  SRM_RADII_LOGNORMAL: log-normal with the given mean and
 * standard deviation of the radius itself, truncated to [lo, hi] by redrawing
 * (drawn from the handle's seed). */
typedef enum { SRM_RADII_EXPLICIT = 0, SRM_RADII_MONO = 1, SRM_RADII_LOGNORMAL = 2 } srm_radii_kind;

typedef struct srm_radii {
    int32_t kind;
    int64_t n;
    const double *r;
    double mean, sd, lo, hi;
} srm_radii;

/* Starting configuration (Algorithm 1).  RSA: random sequential
 * addition at volume fraction f0, proposals uniform in the box or Gaussian
 * around n_clusters uniform centres (standard deviation cluster_sigma).
 * EXPLICIT: init_pos holds non-overlapping positions at scale lambda0. */
typedef enum { SRM_INIT_RSA_UNIFORM = 0, SRM_INIT_RSA_CLUSTERED = 1, SRM_INIT_EXPLICIT = 2 } srm_init_kind;

/* Arithmetic of the path: SRM_PREC_F64 keeps absolute positions in binary64
 * and reproduces the FP64 reference bit for bit; SRM_PREC_F32 keeps binary32
 * offsets relative to the particle's cell and decides collisions with a
 * conservative guard band, with the scale, phi and the final certification in
 * binary64. */
typedef enum { SRM_PREC_F64 = 64, SRM_PREC_F32 = 32 } srm_precision;

typedef struct srm_params {
    double c_w;              /* swelling rate: lambda <- lambda (1 + c_w)        */
    double c_m;              /* migration step length (absolute)                 */
    int32_t N_k;             /* sweeps tried per iteration before the shake      */
    int32_t N_l;             /* trial moves per particle and sweep, 1..65535     */
    int32_t N_shake;         /* sweeps of the shake step                          */
    int32_t precision;       /* srm_precision                                    */
    int32_t init;            /* srm_init_kind                                    */
    int32_t n_clusters;      /* SRM_INIT_RSA_CLUSTERED                           */
    double cluster_sigma;    /* SRM_INIT_RSA_CLUSTERED                           */
    double f0;               /* RSA: starting volume fraction                    */
    const double *init_pos;  /* SRM_INIT_EXPLICIT: host, n*dim                   */
    double lambda0;          /* > 0: starting scale (EXPLICIT); else 1            */
    double lambda_t;         /* > 0: target scale instead of the one of phi      */
    double guard;            /* SRM_PREC_F32: relative guard on squared distance */
    uint64_t sweep0;         /* first value of the sweep counter (resume)        */
    int32_t wait_limit;      /* polls of one cell-to-cell dependency inside a    */
                             /* sweep before the run fails with                  */
                             /* SRM_E_DEVICE_TIMEOUT (0: 2^22; < 0: give up at   */
                             /* the first dependency -- for tests of the path)   */
    int32_t images;          /* periodicity (Section 2): 0 the minimum image of  */
                             /* Alg 5; 1 image particles, the other way the      */
                             /* paper names: a candidate near a face is tested   */
                             /* at its periodic image x + s L (one rounding per  */
                             /* axis), then by the plain difference.  Decides    */
                             /* the FP64 form's arithmetic, certification        */
                             /* included; the FP32 form's cell-relative offsets  */
                             /* already place every candidate at its image       */
                             /* beside the home cell, so it is the same there    */
} srm_params;

/* Fills p with the defaults: c_w = 0.01, c_m = 0 (must be set), N_k = N_l =
 * N_shake = 10, FP64, RSA uniform, f0 = 0.1, guard = 4e-6. */
void srm_params_default(srm_params *p);

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer of at least bytes, usable on stream, or NULL.
 * NULL allocator: the library uses cudaMallocAsync/cudaFreeAsync on the
 * handle's stream. */
typedef struct srm_allocator {
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
    void *ctx;
} srm_allocator;

typedef struct srm_rve srm_rve;

/* Creates an RVE: periodic box L[0..dim), dimension 2 or 3, base radii,
 * target volume fraction phi_t in (0, 1), seed of the migration draws,
 * parameters (NULL: defaults, which leaves c_m = 0 and fails), CUDA stream
 * (NULL: the legacy default stream), allocator (NULL: cudaMallocAsync).
 * The target scale is lambda_t = (phi_t prod L / S0)^(1/d), S0 = sum of the
 * base disk areas or sphere volumes (Algorithm 1).
 * Rejects (SRM_E_ARG): dim not 2 or 3, n < 1, L <= 0, phi_t outside (0, 1),
 * c_m <= 0, N_k, N_l outside 1..65535, N_shake < 0, and boxes narrower than three cells of
 * the final cell size 2.5 lambda_t max r + c_m on some axis (the minimum-image
 * search of Algorithm 5 needs them).  The starting positions are uploaded;
 * device state is created.  Returns SRM_E_INIT if RSA fails. */
srm_status srm_init(srm_rve **out, int32_t dim, const double box[3], const srm_radii *radii,
                    double phi_t, uint64_t seed, const srm_params *p, void *cuda_stream,
                    const srm_allocator *alloc);

typedef struct srm_step_info {
    int32_t result;        /* 1 swollen state accepted, 0 discarded and shaken, 2 at target */
    int32_t k_sweeps;      /* sweeps of the N_k loop in this iteration                      */
    int32_t shake_sweeps;  /* sweeps of the shake step                                       */
    int64_t overlapping;   /* colliding particles after the last check of the N_k loop       */
    double phi;            /* volume fraction of P after the iteration (binary64)            */
    double lambda;         /* scale of P after the iteration                                 */
    uint64_t sweep;        /* sweep counter after the iteration                              */
} srm_step_info;

/* One iteration of Algorithm 1: swell the copy Q, up to N_k
 * rounds of (bin, sweep of Algorithm 3, check of Algorithm 6); accept Q if it
 * is collision-free, else discard it and shake P with N_shake sweeps. */
srm_status srm_step(srm_rve *h, srm_step_info *out);

typedef struct srm_run_info {
    int64_t iterations, accepted, shaken, sweeps;
    double phi, lambda;
    uint64_t sweep;
} srm_run_info;

/* Iterates Algorithm 1 until P reaches the target scale (volume fraction
 * phi_t, Section 2 step e) or max_iters iterations were run
 * (SRM_E_NOT_CONVERGED).  Runs on the device without a host round trip per
 * iteration; the host polls a completion word every few dozen sweeps. */
srm_status srm_run_to_target(srm_rve *h, int64_t max_iters, srm_run_info *out);

/* FP64 certification of P (termination, Section 2 step e): number of pairs
 * i < j with sqrt(|x_i - x_j|^2) <= R_i + R_j under the minimum image,
 * smallest gap S - (R_i + R_j) over pairs of neighbouring cells, and phi.
 * Any pointer may be NULL.  Returns SRM_E_CERTIFY_FAILED if pairs > 0. */
srm_status srm_certify(srm_rve *h, int64_t *overlap_pairs, double *min_gap, double *phi);

/* Copies P to the host in particle-id order: xyz[n*dim], radii[n] (R_i =
 * lambda r_i; may be NULL).  Synchronises the stream. */
srm_status srm_positions(srm_rve *h, double *xyz, double *radii);

/* Colliding pairs of P at its current scale (Algorithm 6 over all pairs),
 * i < j by particle id, lexicographic order, as int64 pairs ij[2k], ij[2k+1];
 * writes min(cap, *n) pairs and sets *n to the total. */
srm_status srm_overlap_pairs(srm_rve *h, int64_t *ij, int64_t cap, int64_t *n);

/* ---- structure descriptors of P (Section 3.2) ---------------------------
 * The statistics the paper uses to tell clustered from equilibrium-like
 * configurations: nearest-neighbour distances (Fig. 4d), the local volume
 * fraction of every particle -- its area (volume) over the area (volume) of
 * its Voronoi cell (Figs. 5 and 7) -- and the radial distribution of the
 * centres.  They read P at its current scale in binary64 (periodic minimum
 * image; distance = correctly rounded root of the squared differences summed
 * in axis order).  Outputs are caller-owned host arrays in particle-id order;
 * each call synchronises the handle's stream.  SRM_E_STATE inside an
 * iteration (as srm_certify). */

/* Nearest neighbour of every particle: nn_dist[i] = min over j != i of the
 * centre distance S_ij, nn_id[i] = that j (ties to the smaller id; may be
 * NULL), gap[i] = min over j != i of S_ij - (R_i + R_j) (the smallest
 * surface gap; negative for overlaps).  Arrays of n. */
srm_status srm_nearest(srm_rve *h, double *nn_dist, int64_t *nn_id, double *gap);

/* Radial distribution of the centres: counts[k] = ordered pairs (i, j),
 * i != j, with S_ij in [k dr, (k+1) dr), dr = r_max / bins (bin floor(S /
 * dr)); gr[k] (may be NULL) = counts[k] V / (N (N - 1) V_k), V_k the volume
 * (area) of shell k.  0 < r_max <= half the smallest box length (else
 * SRM_E_ARG), 1 <= bins <= 4096. */
srm_status srm_rdf(srm_rve *h, double r_max, int32_t bins, int64_t *counts, double *gr);

/* Local volume fraction from a discrete periodic Voronoi tessellation on
 * voxels[0] x voxels[1] (x voxels[2]) voxels (voxels[2] ignored in 2D; each
 * in [1, 65536], at most 2^34 in total): the voxel centre ((i_a + 0.5) h_a,
 * h_a = L_a / voxels[a]) belongs to the nearest particle centre (ties to the
 * smaller id); count[j] = voxels of particle j, lvf[j] (may be NULL) = v_j /
 * (count[j] prod h_a) with v_j = pi R_j^2 (2D) or 4/3 pi R_j^3 (3D), +inf for
 * an empty cell.  The discrete cell volumes converge to the Voronoi volumes
 * as the voxels shrink; their sum is the box volume exactly. */
srm_status srm_voronoi_lvf(srm_rve *h, const int32_t voxels[3], int64_t *count, double *lvf);

/* Runs count sweeps of Algorithm 3 on P at its current scale (each preceded
 * by a fresh binning, grid of the current scale): the relaxation move with
 * no swelling (Section 3.3, zero swelling rate).  Advances the sweep counter.
 * *moved (may be NULL) receives the number of accepted moves of the last
 * sweep. */
srm_status srm_sweep(srm_rve *h, int32_t count, int64_t *moved);

/* Sets the scale of P (no moves; may create overlaps). */
srm_status srm_set_scale(srm_rve *h, double lambda);

typedef struct srm_state_info {
    int32_t dim, precision;
    int64_t n;
    double lambda, lambda_t, phi, phi_t;
    uint64_t sweep;
    int64_t iterations, accepted, shaken, sweeps;
    int32_t done;
    int32_t grid[3];            /* cells per axis of the current iteration           */
    int64_t kernel_launches;    /* kernels this handle has launched since creation   */
    uint64_t pairs_sweep;       /* candidate pairs tested by the sweeps (Alg 3/5)    */
    uint64_t pairs_check;       /* candidate pairs tested by the checks (Alg 6)      */
    uint64_t stage_overflow;    /* sweep cells whose candidates exceeded the staging */
    int32_t stage_capacity;     /* candidates a sweep warp stages in shared memory   */
    int32_t check_kernel;       /* Alg 6 kernel: 0 a thread per particle, 1 a warp per
                                   cell (whole-stencil estimate above 256)          */
    uint64_t trials;            /* trial moves evaluated by the sweeps (Alg 3)       */
    uint64_t pairs_alg5;        /* pairs Alg 5 examines for those trials: for each,
                                   the particles of the 3^d cells around the home
                                   cell other than the mover (the method's own
                                   candidate set, before any culling)               */
    uint64_t near_fallback;     /* particles of sweep cells on the general path whose
                                   near list exceeded its capacity and were tested
                                   against every staged candidate instead         */
} srm_state_info;

srm_status srm_get_state(srm_rve *h, srm_state_info *out);

/* Launch shape of the sweep (not in the paper: a property of this GPU
 * implementation).  Results do not depend on it -- the sweep's order is
 * fixed by the cells' colours, and cells whose stencil exceeds the staging
 * capacity read the rest from global memory -- only the speed does. */
typedef struct srm_tuning {
    int32_t sweep_blocks_per_sm;   /* blocks per SM of the persistent sweep grid; 0 = all that fit */
    int32_t stage_capacity;        /* candidates a sweep warp stages in shared memory (rounded up to a
                                      multiple of 32, clamped to [64, 1024] FP32 / [64, 384] FP64;
                                      <= 0 keeps the current one) */
    int32_t candidates;            /* autotune output: shapes tried */
    int32_t sweep_path;            /* FP32 sweep kernel: 1 = general path only (fewer registers, more
                                      resident warps), 2 = with the staged path (a cell's whole stencil
                                      copied to shared memory); 0 keeps the current one.  The FP64
                                      sweep has the general path only (2 is SRM_E_ARG there).  Default
                                      at creation: 1, with the staging capacity at most 256 */
    double ns_per_particle_sweep;  /* autotune output: best device time per particle sweep */
} srm_tuning;

/* Autotuner: runs the RVE (or batch) for `supersteps` super-steps (>= 1,
 * rounded up to whole recorded graphs of 8) with each candidate shape --
 * blocks per SM from 2 to the resident maximum, staging capacity at the
 * current value and twice (never below: stencils grow as the particles
 * swell); the sweep kernel (sweep_path) stays as set -- in two
 * interleaved rounds, scores each
 * by device time per particle sweep (CUDA events) and keeps the fastest.
 * The super-steps are real work: the RVEs advance (and may finish).  *best
 * (may be NULL) receives the chosen shape.  Synchronises the stream. */
srm_status srm_autotune(srm_rve *h, int32_t supersteps, srm_tuning *best);
srm_status srm_set_tuning(srm_rve *h, const srm_tuning *t);   /* re-records the graphs */
srm_status srm_get_tuning(srm_rve *h, srm_tuning *t);

/* Per-stage device time of the super-steps run while timing is on, from CUDA
 * events recorded between the launches of each super-step (one host
 * synchronisation per super-step while on, so use it for measurement only).
 * Stages: begin + binning (Algorithm 2), the sweep (Algorithm 3, one launch
 * for all colours), the check (Algorithm 6), the control step. */
typedef struct srm_timings {
    double ms_bin, ms_sweep, ms_check, ms_control;
    int64_t supersteps;       /* super-steps that did work while timing was on */
    int64_t sweep_launches;   /* launches of the sweep kernel                   */
    int64_t check_launches;   /* launches of the check kernel that did work     */
} srm_timings;

/* on != 0: later srm_step / srm_run_to_target / srm_sweep calls record
 * per-stage times (and the accumulated times are reset); on == 0: back to
 * plain graph replay. */
srm_status srm_set_timing(srm_rve *h, int32_t on);
srm_status srm_get_timings(srm_rve *h, srm_timings *out);

/* ---------------------------------------------------------------------------
 * Checkpoints.  The state of an RVE between iterations (accepted positions
 * exactly as stored, radii, scale, sweep counter, counters, parameters) is
 * serialised into a caller buffer; a handle loaded from it continues bit for
 * bit as the saved one would have (the migration draws are counter-based).
 * srm_save: buf == NULL sets *len to the size needed; otherwise *len is the
 * buffer size (SRM_E_ARG if too small) and receives the bytes written.
 * --------------------------------------------------------------------------- */
srm_status srm_save(srm_rve *h, void *buf, size_t *len);
srm_status srm_load(srm_rve **out, const void *buf, size_t len, void *cuda_stream,
                    const srm_allocator *alloc);

/* ---------------------------------------------------------------------------
 * Batches: many independent RVEs advanced by the same kernel launches (sizes,
 * dimensions and targets may differ; one precision per batch).  Each RVE
 * keeps its own state, grid, buffers and Philox counters, so its result does
 * not depend on which other RVEs share the batch.
 * --------------------------------------------------------------------------- */
typedef struct srm_job {
    int32_t dim;
    double box[3];
    srm_radii radii;
    double phi_t;
    uint64_t seed;
    srm_params params;
} srm_job;

typedef struct srm_batch srm_batch;

/* A batch holding the given jobs, each loaded into a slot sized for it. */
srm_status srm_batch_create(srm_batch **out, const srm_job *jobs, int32_t n_jobs, void *cuda_stream,
                            const srm_allocator *alloc);

/* A batch of n_slots empty slots for continuous serving: each slot takes a
 * job of at most max_particles particles and max_cells cells on the finest
 * grid of its run (srm_job_footprint), of dimension dim (2 or 3; 0: either
 * -- every super-step then runs the sweeps of both dimensions, one after
 * the other).  stage_capacity: candidates a sweep warp stages in shared
 * memory (0: 256). */
srm_status srm_batch_create_slots(srm_batch **out, int32_t n_slots, int64_t max_particles,
                                  int64_t max_cells, int32_t dim, int32_t precision, int32_t stage_capacity,
                                  void *cuda_stream, const srm_allocator *alloc);

/* Particles and finest-grid cells a job needs (for admission decisions). */
srm_status srm_job_footprint(const srm_job *job, int64_t *particles, int64_t *cells);

/* Loads a job into a slot that is empty or finished and polled (SRM_E_STATE
 * if the slot is busy, SRM_E_ARG if the job does not fit). */
srm_status srm_batch_admit(srm_batch *b, int32_t slot, const srm_job *job);

/* Enqueues `supersteps` super-steps (one sweep each, with binning, check and
 * control) for every running slot; returns without waiting. */
srm_status srm_batch_advance(srm_batch *b, int32_t supersteps);

/* Runs every RVE of the batch to its target (at most max_iters iterations
 * each; SRM_E_NOT_CONVERGED otherwise). */
srm_status srm_batch_run(srm_batch *b, int64_t max_iters);

/* The autotuner and launch shape of a batch (as srm_autotune). */
srm_status srm_batch_autotune(srm_batch *b, int32_t supersteps, srm_tuning *best);
srm_status srm_batch_set_tuning(srm_batch *b, const srm_tuning *t);
srm_status srm_batch_get_tuning(srm_batch *b, srm_tuning *t);

/* Slots that reached their target since the last poll, each reported once. */
srm_status srm_batch_poll(srm_batch *b, int32_t *done_slots, int32_t cap, int32_t *n_done);

/* Marks a finished slot free for the next admission. */
srm_status srm_batch_release(srm_batch *b, int32_t slot);

int32_t srm_batch_size(const srm_batch *b);
srm_status srm_batch_state(srm_batch *b, int32_t slot, srm_state_info *out);
srm_status srm_batch_positions(srm_batch *b, int32_t slot, double *xyz, double *radii);
srm_status srm_batch_certify(srm_batch *b, int32_t slot, int64_t *overlap_pairs, double *min_gap,
                             double *phi);
srm_status srm_batch_set_timing(srm_batch *b, int32_t on);
srm_status srm_batch_get_timings(srm_batch *b, srm_timings *out);
void srm_batch_destroy(srm_batch *b);

/* ---------------------------------------------------------------------------
 * Certification without device allocation.
 *
 * The paper has no counterpart to this call: it exists for callers that may
 * not allocate device memory at all -- plug-ins of a host application that
 * owns every device allocation (its own pool or a fixed arena, so a
 * cudaMalloc from a library would bypass its accounting), code that runs
 * under a fixed device-memory budget where a new allocation could fail,
 * and latency-bound paths where an allocation could block.  Such a caller
 * keeps the configuration in its own device buffers and passes them in; the
 * call computes the same binary64 certification as srm_certify (colliding
 * pairs i < j by index, and the smallest gap S - (R_i + R_j) over pairs in
 * neighbouring cells of a grid with cells at least 2 R_max wide), with all
 * working memory in one static device array of the library (1,966,592
 * bytes = 1.97 MB = 1.88 MiB, held by every GPU that loads the library until
 * the process exits).  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * dim: 2 or 3; box: L[0..dim); n: particles, 1 <= n <= 32768
 * (SRM_NOALLOC_MAX_PARTICLES, larger n is rejected with SRM_E_ARG); xyz:
 * device pointer to n*dim binary64 positions in [0, L), particle order;
 * radii: device pointer to n binary64 radii; overlap_pairs, min_gap: host
 * pointers receiving the results; cuda_stream: stream to run on (NULL: the
 * legacy default stream), synchronised before returning.  Boxes narrower
 * than 4 R_max on some axis, and radii that are negative, infinite or NaN,
 * are rejected (SRM_E_ARG).  A CUDA error already pending on the calling
 * thread when the call starts is reported (SRM_E_CUDA) and left pending.
 *
 * The first call on a device looks up the device address of the static
 * array (cudaGetSymbolAddress) with that device current.  All calls share
 * the one array, whose contents are whatever the last call left (each call
 * clears what it needs zeroed): calls that overlap on the GPU -- from two
 * threads, or on two streams without ordering between them -- race and give
 * wrong results. */
#define SRM_NOALLOC_MAX_PARTICLES 32768
#define SRM_NOALLOC_MAX_CELLS 65536
srm_status srm_certify_noalloc(int32_t dim, const double box[3], int64_t n, const double *xyz,
                               const double *radii, int64_t *overlap_pairs, double *min_gap,
                               void *cuda_stream);

/* Releases the handle and its device memory (stream-ordered). */
void srm_destroy(srm_rve *h);

/* Message of the last failure on this thread ("" if none). */
const char *srm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SRM_H */
