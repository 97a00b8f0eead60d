// srm_launch.h -- host-side launchers of the SRM kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace srm {

struct RveDev;

// Sizes fixed at creation; the kernels read everything that changes between
// iterations (grid, scale, buffer roles) from the device state, so that a
// captured sequence of launches stays valid for the whole run.
struct HostShape {
    int dim;
    int64_t n;
    int64_t ncells_cap;  // largest number of cells of any iteration
    int64_t nsub_cap;    // largest number of cells of one colour
    bool f32;            // arithmetic of the working copies (input format of binning)
    bool out_f32;        // format written by binning (false: absolute binary64)
    int cap_sweep;       // candidates a warp stages in shared memory (sweep)
    int cap_check;       // same for the check kernel
};

void launch_begin(RveDev *d_st, cudaStream_t s);
void launch_control(RveDev *d_st, cudaStream_t s);
void launch_bin(RveDev *d_st, const HostShape &sh, cudaStream_t s);
void launch_scan(RveDev *d_st, int which, int64_t max_len, cudaStream_t s);
int64_t scan_part_len(int64_t max_len);
void launch_sweep(RveDev *d_st, const HostShape &sh, cudaStream_t s);
void sweep_configure();
int sweep_cap_max(bool f32);
int check_cap_max(bool f32);
void launch_sweep_colour(RveDev *d_st, const HostShape &sh, int chi, cudaStream_t s);
void launch_check(RveDev *d_st, const HostShape &sh, cudaStream_t s);
void check_configure();
void launch_inspect_bin(RveDev *d_st, const HostShape &sh, cudaStream_t s);
void launch_inspect_end(RveDev *d_st, cudaStream_t s);
void launch_pairs_count(RveDev *d_st, const HostShape &sh, int want_gap, cudaStream_t s);
void launch_pairs_fill(RveDev *d_st, const HostShape &sh, long long *ij, cudaStream_t s);
void launch_gather(RveDev *d_st, const HostShape &sh, double *xyz, double *rad, cudaStream_t s);
void launch_import(RveDev *d_st, const HostShape &sh, const double *xyz, const double *rb,
                   cudaStream_t s);

}  // namespace srm
