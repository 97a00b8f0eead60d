// srm_launch.h -- host-side launchers of the SRM kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace srm {

struct RveDev;
struct BatchDev;

// Launch shape of a group of RVEs (one RVE, or a batch).  The kernels read
// everything that changes between iterations (grid, scale, buffer roles)
// from the device state, so a captured sequence of launches stays valid for
// the whole run.
struct BatchShape {
    BatchDev *d;        // device descriptor
    int B;              // RVEs
    int blocks_p;       // blocks of particle-indexed launches (256 threads)
    int blocks_c;       // blocks of cell-indexed launches (256 threads)
    int tiles_c;        // scan tiles over cells
    int tiles_n;        // scan tiles over particles
    int64_t sub_total;  // sweep work items per colour (sum of colour-cell capacities)
    bool f32;           // arithmetic of the working copies
    bool has3d;         // some RVE is (or a slot may hold) a 3D RVE
    bool has2d;         // some RVE is (or a slot may hold) a 2D RVE
    int cap;            // candidates a sweep warp stages in shared memory
    int sweep_bps;      // blocks per SM of the persistent sweep grid (0: all that fit)
    bool staged;        // FP32 sweep: the variant with the staged path
    bool check_cells;   // check: a warp per cell (dense stencils) instead of a thread per particle
};

void launch_begin(const BatchShape &b, cudaStream_t s);
void launch_plan(const BatchShape &b, cudaStream_t s);
int plan_blocks(int64_t capacity_chunks);
void launch_control(const BatchShape &b, cudaStream_t s);
void launch_bin(const BatchShape &b, bool in32, bool out32, cudaStream_t s);
void launch_scan(const BatchShape &b, int which, cudaStream_t s);
int64_t scan_part_len(int64_t max_len);
int scan_tile();
void launch_sweep(const BatchShape &b, cudaStream_t s);
int sweep_launches(const BatchShape &b);
void sweep_configure();
int sweep_cap_max(bool f32);
int sweep_blocks_per_sm(bool f32, int cap, bool staged);  // resident sweep blocks per SM (3D kernel)
int check_cap_max(bool f32);
void launch_check(const BatchShape &b, cudaStream_t s);
void check_configure();

// single RVE
void launch_inspect_bin(RveDev *d_st, const BatchShape &solo, cudaStream_t s);
void launch_inspect_end(RveDev *d_st, cudaStream_t s);
void launch_pairs_count(RveDev *d_st, int dim, int64_t n, int want_gap, cudaStream_t s);
void launch_pairs_fill(RveDev *d_st, int dim, int64_t n, long long *ij, cudaStream_t s);
void launch_gather(RveDev *d_st, int dim, bool f32, int64_t n, double *xyz, double *rad, cudaStream_t s);

// structure descriptors (k_analysis.cu), on the binning of launch_inspect_bin
void launch_nearest(RveDev *d_st, int dim, int64_t n, double *nn_dist, long long *nn_id, double *gap, cudaStream_t s);
void launch_rdf(RveDev *d_st, int dim, int64_t n, double r_max, int bins, const int lo[3], const int hi[3],
                unsigned long long *counts, cudaStream_t s);
void launch_voronoi(RveDev *d_st, int dim, const int32_t M[3], const double h[3], unsigned long long *count,
                    cudaStream_t s);
void launch_import(RveDev *d_st, int dim, bool f32, int64_t n, const double *xyz, const double *rb,
                   cudaStream_t s);

}  // namespace srm
