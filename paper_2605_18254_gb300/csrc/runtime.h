// runtime.h -- host-side structures shared by the C interface files
// (internal; not installed).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "srm.h"
#include "srm_dev.cuh"
#include "srm_launch.h"

using srm::BatchDev;
using srm::BatchShape;
using srm::RveDev;

srm_status fail(srm_status st, const std::string &msg);

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(SRM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Host-side preparation of one job: radii, starting positions, scales and
// the capacities it needs.
struct Prep {
    int dim = 3;
    int64_t n = 0;
    double L[3] = {1.0, 1.0, 1.0};
    std::vector<double> r, x;
    double rmax = 0.0, S0 = 0.0, V = 1.0, phi_t = 0.5, lam0 = 1.0, lam_t = 1.0, lam_min = 1.0;
    srm_params p{};
    uint64_t seed = 0;
    int64_t ncells_need = 0, nsub_need = 0;
    int cap_est = 64;
};

// One RVE: its device state and buffers (sized by capacities, so that a
// slot of a batch can take successive jobs up to those sizes).
struct Member {
    RveDev h{};           // host copy: constants and buffer pointers
    RveDev *d = nullptr;  // device state
    int64_t n_cap = 0, ncells_cap = 0, nsub_cap = 0;
    bool loaded = false, harvested = false, any_dim = false;  // any_dim: a slot for 2D or 3D jobs
    int slot_dim = 0;  // dimension a serving slot accepts (0: either)
    int dim = 3;
    int64_t n = 0;
    double S0 = 0.0, V = 1.0, phi_t = 0.0, lam_min = 0.0;
    double *stage_x = nullptr, *stage_r = nullptr;  // upload buffers of a starting state
    BatchDev *solo_d = nullptr;                     // the member as a group of one
    BatchShape solo{};
    double *d_xyz = nullptr, *d_rad = nullptr;
    long long *d_ij = nullptr;
    int64_t d_ij_cap = 0;
    void *d_an = nullptr;  // scratch of the structure descriptors (grows)
    size_t an_bytes = 0;
};

// RVEs advanced by the same launches.
struct Group {
    std::vector<Member *> m;
    bool f32 = false;
    int cap = 64;
    int sweep_bps = 0;  // blocks per SM of the sweep grid (0: all that fit)
    int sweep_path = 1;  // FP32 sweep variant: 1 general path only, 2 with the staged path
    int stencil_est = 0;  // particle-weighted mean whole-stencil estimate of the members (the check's kernel choice)
    BatchDev *d = nullptr;
    BatchShape sh{};
    cudaStream_t stream = nullptr;      // the caller's stream: all work runs here
    cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
    srm_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> owned;
    RveDev *pin = nullptr;  // pinned mirror of every member's state
    unsigned long long *pin_red = nullptr;
    cudaGraphExec_t g1 = nullptr, gN = nullptr, gT = nullptr;
    int gN_steps = 8;
    int64_t launches = 0, launches_per_step = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    srm_timings tm{};
};

struct srm_rve {
    Group g;
};

struct srm_batch {
    Group g;
};

inline void group_setup(Group &g, void *stream, const srm_allocator *alloc)
{
    g.stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        g.alloc = *alloc;
        g.has_alloc = true;
    }
}

double phi_of(int dim, double S0, double V, double lam);
int64_t cells_for(int dim, const double L[3], double rmax, double c_m, double lam, int64_t per_axis[3]);
srm_status prepare(int32_t dim, const double box[3], const srm_radii *radii, double phi_t, uint64_t seed,
                   const srm_params *pin, Prep &q, bool place = true);
void *dev_alloc(Group &g, size_t bytes);
void group_free(Group &g);
srm_status member_alloc(Group &g, Member &mb, int64_t n_cap, int64_t ncells_cap, int64_t nsub_cap);
bool member_fits(const Member &mb, const Prep &q);
srm_status member_load(Group &g, Member &mb, const Prep &q);
srm_status group_finalize(Group &g);
srm_status pull_states(Group &g);
srm_status pull_state(Group &g, size_t r);
srm_status run_graph(Group &g, int steps);
srm_status run_group(Group &g, int64_t max_iters);
void launch_set_cap(Group &g, size_t r, int64_t cap);
bool idle_mode(int32_t m);
srm_status member_idle(Group &g, size_t r);
srm_status group_set_tuning(Group &g, int sweep_bps, int cap, int path);
// Sweep kernel when none is chosen: the general path only (measured on GB300,
// FP32: faster than the staged kernel on the clustered 1e6-sphere RVE (7%),
// on the ensemble of small RVEs (25%) and, with its L2 prefetch and staging
// ring, on 1e5 monodisperse spheres (3%)).
constexpr int DEFAULT_SWEEP_PATH = 1;
int default_capacity(int estimate, bool f32);
srm_status group_autotune(Group &g, int32_t supersteps, srm_tuning *best);
srm_status member_certify(Group &g, size_t r, int64_t *overlap_pairs, double *min_gap, double *phi);
srm_status member_positions(Group &g, size_t r, double *xyz, double *radii);
void fill_state(const Group &g, size_t r, srm_state_info *o);
