// runtime.cu -- host side of the C interface declared in include/srm.h:
// handle creation and device memory, starting configurations, the captured
// super-step graph and its replay, inspection and read-back.
//
// A "super-step" is one sweep of Algorithm 3 with everything around it:
//   k_begin (state machine: swell and new grid at the start of an
//   iteration, buffer roles) -> binning (Algorithm 2) -> 3^d colour launches
//   of the sweep -> Algorithm 6 check (N_k loop only) -> k_control
//   (accept / next round / shake / done).
// Every launch reads what changes from the device state, so one captured
// CUDA graph of a few super-steps is replayed for the whole run and the host
// only polls the state word every few dozen sweeps.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "srm.h"
#include "srm_dev.cuh"
#include "srm_launch.h"

extern "C" int inp_radii_lognormal(int64_t n, double mean, double sd, double lo, double hi,
                                   uint64_t seed, double *out);
extern "C" int inp_rsa(int dim, const double L[3], int64_t n, const double *R, uint64_t seed,
                       int mode, int64_t n_clusters, double sigma, int64_t max_attempts, double *X);

using srm::RveDev;

static thread_local std::string g_err;

static srm_status fail(srm_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

namespace srm {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace srm

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(SRM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct srm_rve {
    RveDev h{};               // host copy: constants and buffer pointers
    RveDev *d = nullptr;      // device state
    RveDev *pin = nullptr;    // pinned host mirror for read-back
    srm::HostShape sh{};
    cudaStream_t stream = nullptr;      // the caller's stream: all work runs here
    cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
    unsigned long long *pin_red = nullptr;
    srm_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> owned;
    cudaGraphExec_t g1 = nullptr, gN = nullptr;
    int gN_steps = 8;
    double S0 = 0.0, V = 0.0, phi_t = 0.0, lam_min = 0.0;
    double *d_xyz = nullptr, *d_rad = nullptr;
    long long *d_ij = nullptr;
    int64_t d_ij_cap = 0;
    int64_t launches = 0;          // kernels launched (graph nodes counted per replay)
    int64_t launches_per_step = 0; // kernels in one super-step
    // timing mode
    bool timing = false;
    cudaGraphExec_t gT = nullptr;
    std::vector<cudaEvent_t> ev;   // events of one timed super-step
    srm_timings tm{};
};

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
static void *dev_alloc(srm_rve *h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(h->alloc.ctx, bytes, (void *)h->stream);
    } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
        p = nullptr;
    }
    if (p) h->owned.push_back(p);
    return p;
}

static void dev_free_all(srm_rve *h)
{
    for (void *p : h->owned) {
        if (h->has_alloc) h->alloc.free(h->alloc.ctx, p, (void *)h->stream);
        else cudaFreeAsync(p, h->stream);
    }
    h->owned.clear();
}

// ---------------------------------------------------------------------------
// closed forms of the bookkeeping (binary64)
// ---------------------------------------------------------------------------
static double base_measure(int dim, const double *r, int64_t n)
{
    // sum of base disk areas / sphere volumes in id order
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double ri = r[i];
        s += dim == 2 ? M_PI * ri * ri : (4.0 / 3.0) * M_PI * ri * ri * ri;
    }
    return s;
}

static double phi_of(const srm_rve *h, double lam)
{
    double ld = lam * lam;
    if (h->h.dim == 3) ld = ld * lam;
    return ld * h->S0 / h->V;
}

static double lam_of(int dim, double S0, double V, double phi)
{
    const double q = phi / (1.0 * S0 / V);
    return dim == 2 ? std::sqrt(q) : std::cbrt(q);
}

// cells per axis of the grid for scale lam (same rule as the device)
static int64_t cells_for(const srm_rve *h, double lam, int64_t per_axis[3])
{
    const double cs = 2.5 * (lam * h->h.rmax) + h->h.c_m;
    int64_t tot = 1;
    for (int a = 0; a < 3; a++) {
        per_axis[a] = 1;
        if (a >= h->h.dim) continue;
        int64_t k = (int64_t)(h->h.L[a] / (3.0 * cs));
        if (k < 1) k = 1;
        per_axis[a] = 3 * k;
        tot *= per_axis[a];
    }
    return tot;
}

// ---------------------------------------------------------------------------
// device state read-back and small writes
// ---------------------------------------------------------------------------
static srm_status pull_state(srm_rve *h)
{
    CK(cudaMemcpyAsync(h->pin, h->d, sizeof(RveDev), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->pin->status != 0) return fail(SRM_E_STATE, "device state reports an error");
    return SRM_OK;
}

__global__ void k_set_mode(RveDev *st, int32_t mode, int32_t resume)
{
    st->mode = mode;
    st->resume_mode = resume;
}

__global__ void k_set_scale(RveDev *st, double lam)
{
    st->lam_P = lam;
    st->mode = lam >= st->lam_t ? srm::MODE_DONE : srm::MODE_BEGIN;
}

__global__ void k_set_cap(RveDev *st, int64_t cap) { st->iter_cap = cap; }

// ---------------------------------------------------------------------------
// super-step graphs
// ---------------------------------------------------------------------------
// kernels of one super-step: begin, binning (count, 3 scan passes, scatter,
// stamp, in-cell sort), 3^d sweep colours, check, control
static int64_t kernels_per_superstep(int dim) { return 1 + 7 + (dim == 3 ? 27 : 9) + 1 + 1; }

static void enqueue_superstep(srm_rve *h, cudaStream_t s, const std::vector<cudaEvent_t> *ev = nullptr)
{
    srm::HostShape sh = h->sh;
    sh.out_f32 = sh.f32;
    if (ev) cudaEventRecordWithFlags((*ev)[0], s, cudaEventRecordExternal);
    srm::launch_begin(h->d, s);
    srm::launch_bin(h->d, sh, s);
    if (ev) {
        const int ncol = sh.dim == 3 ? 27 : 9;
        for (int chi = 0; chi < ncol; chi++) {
            cudaEventRecordWithFlags((*ev)[1 + chi], s, cudaEventRecordExternal);
            srm::launch_sweep_colour(h->d, sh, chi, s);
        }
        cudaEventRecordWithFlags((*ev)[1 + ncol], s, cudaEventRecordExternal);
        srm::launch_check(h->d, sh, s);
        cudaEventRecordWithFlags((*ev)[2 + ncol], s, cudaEventRecordExternal);
        srm::launch_control(h->d, s);
        cudaEventRecordWithFlags((*ev)[3 + ncol], s, cudaEventRecordExternal);
    } else {
        srm::launch_sweep(h->d, sh, s);
        srm::launch_check(h->d, sh, s);
        srm::launch_control(h->d, s);
    }
}

// The graph is recorded on a private stream (recording runs nothing) and
// launched on the caller's stream, which may be the legacy default stream.
static srm_status capture(srm_rve *h, int steps, cudaGraphExec_t *out, bool timed = false)
{
    cudaGraph_t g = nullptr;
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < steps; i++) enqueue_superstep(h, h->cap_stream, timed ? &h->ev : nullptr);
    CK(cudaStreamEndCapture(h->cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SRM_E_CUDA, std::string("graph: ") + cudaGetErrorString(e));
    return SRM_OK;
}

static srm_status pull_state(srm_rve *h);

// Timing mode: one super-step per replay, with events between the stages;
// the host waits for each replay and adds up the stage times.
static srm_status run_timed(srm_rve *h, int steps)
{
    const int ncol = h->sh.dim == 3 ? 27 : 9;
    if (h->ev.empty()) {
        h->ev.resize((size_t)ncol + 4);
        for (auto &e : h->ev) CK(cudaEventCreate(&e));
    }
    if (!h->gT) {
        srm_status s = capture(h, 1, &h->gT, true);
        if (s != SRM_OK) return s;
    }
    for (int i = 0; i < steps; i++) {
        const int64_t sw0 = h->pin->sweeps;
        CK(cudaGraphLaunch(h->gT, h->stream));
        h->launches += h->launches_per_step;
        srm_status s = pull_state(h);
        if (s != SRM_OK) return s;
        if (h->pin->sweeps == sw0) continue;  // nothing ran (target reached or capped)
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        h->tm.ms_bin += ms;
        for (int c = 0; c < ncol; c++) {
            CK(cudaEventElapsedTime(&ms, h->ev[1 + c], h->ev[2 + c]));
            h->tm.ms_sweep += ms;
        }
        h->tm.sweep_launches += ncol;
        CK(cudaEventElapsedTime(&ms, h->ev[1 + ncol], h->ev[2 + ncol]));
        h->tm.ms_check += ms;
        if (h->pin->do_check) h->tm.check_launches += 1;
        CK(cudaEventElapsedTime(&ms, h->ev[2 + ncol], h->ev[3 + ncol]));
        h->tm.ms_control += ms;
        h->tm.supersteps += 1;
    }
    return SRM_OK;
}

static srm_status run_graph(srm_rve *h, int steps)
{
    if (h->timing) return run_timed(h, steps == 1 ? 1 : h->gN_steps);
    cudaGraphExec_t *g = steps == 1 ? &h->g1 : &h->gN;
    if (!*g) {
        srm_status s = capture(h, steps == 1 ? 1 : h->gN_steps, g);
        if (s != SRM_OK) return s;
    }
    CK(cudaGraphLaunch(*g, h->stream));
    h->launches += h->launches_per_step * (steps == 1 ? 1 : h->gN_steps);
    return SRM_OK;
}

// ---------------------------------------------------------------------------
// C interface
// ---------------------------------------------------------------------------
extern "C" {

void srm_params_default(srm_params *p)
{
    std::memset(p, 0, sizeof(*p));
    p->c_w = 0.01;
    p->c_m = 0.0;
    p->N_k = 10;
    p->N_l = 10;
    p->N_shake = 10;
    p->precision = SRM_PREC_F64;
    p->init = SRM_INIT_RSA_UNIFORM;
    p->n_clusters = 0;
    p->cluster_sigma = 0.0;
    p->f0 = 0.1;
    p->init_pos = nullptr;
    p->lambda0 = 0.0;
    p->lambda_t = 0.0;
    p->guard = 4e-6;
    p->sweep0 = 0;
}

const char *srm_last_error(void) { return g_err.c_str(); }

srm_status srm_init(srm_rve **out, int32_t dim, const double box[3], const srm_radii *radii,
                    double phi_t, uint64_t seed, const srm_params *pin, void *cuda_stream,
                    const srm_allocator *alloc)
{
    g_err.clear();
    if (!out || !box || !radii) return fail(SRM_E_ARG, "null argument");
    *out = nullptr;
    srm_params p;
    if (pin) p = *pin;
    else srm_params_default(&p);
    if (dim != 2 && dim != 3) return fail(SRM_E_ARG, "dim must be 2 or 3");
    const int64_t n = radii->n;
    if (n < 1) return fail(SRM_E_ARG, "n must be >= 1");
    if (n > 0x7fffffffLL) return fail(SRM_E_ARG, "n must be < 2^31");
    for (int a = 0; a < dim; a++)
        if (!(box[a] > 0.0)) return fail(SRM_E_ARG, "box lengths must be > 0");
    if (!(phi_t > 0.0 && phi_t < 1.0)) return fail(SRM_E_ARG, "target phi must be in (0, 1)");
    if (!(p.c_m > 0.0)) return fail(SRM_E_ARG, "c_m must be > 0");
    if (!(p.c_w >= 0.0)) return fail(SRM_E_ARG, "c_w must be >= 0");
    if (p.N_k < 1 || p.N_l < 1 || p.N_shake < 0) return fail(SRM_E_ARG, "N_k, N_l >= 1, N_shake >= 0");
    if (p.precision != SRM_PREC_F64 && p.precision != SRM_PREC_F32)
        return fail(SRM_E_ARG, "precision must be 32 or 64");
    if (p.precision == SRM_PREC_F32 && !(p.guard > 0.0 && p.guard < 1e-2))
        return fail(SRM_E_ARG, "FP32 guard must be in (0, 1e-2)");

    // base radii
    std::vector<double> r((size_t)n);
    if (radii->kind == SRM_RADII_EXPLICIT) {
        if (!radii->r) return fail(SRM_E_ARG, "explicit radii need r");
        std::memcpy(r.data(), radii->r, sizeof(double) * (size_t)n);
    } else if (radii->kind == SRM_RADII_MONO) {
        for (auto &v : r) v = radii->mean;
    } else if (radii->kind == SRM_RADII_LOGNORMAL) {
        if (!(radii->mean > 0 && radii->sd >= 0 && radii->lo <= radii->hi))
            return fail(SRM_E_ARG, "bad log-normal parameters");
        if (inp_radii_lognormal(n, radii->mean, radii->sd, radii->lo, radii->hi, seed, r.data()))
            return fail(SRM_E_ARG, "log-normal truncation window too narrow");
    } else {
        return fail(SRM_E_ARG, "unknown radii kind");
    }
    double rmax = 0.0;
    for (double v : r) {
        if (!(v > 0.0)) return fail(SRM_E_ARG, "radii must be > 0");
        rmax = v > rmax ? v : rmax;
    }

    srm_rve *h = new srm_rve();
    h->stream = (cudaStream_t)cuda_stream;
    if (alloc && alloc->alloc && alloc->free) {
        h->alloc = *alloc;
        h->has_alloc = true;
    }
    RveDev &s = h->h;
    s.dim = dim;
    s.prec = p.precision;
    s.n = (int32_t)n;
    s.N_k = p.N_k;
    s.N_l = p.N_l;
    s.N_shake = p.N_shake;
    for (int a = 0; a < 3; a++) {
        s.L[a] = a < dim ? box[a] : 1.0;
        s.halfL[a] = 0.5 * s.L[a];
        s.Lf[a] = (float)s.L[a];
    }
    s.rmax = rmax;
    s.c_w = p.c_w;
    s.c_m = p.c_m;
    s.guard = (float)p.guard;
    s.seed = seed;
    s.iter_cap = INT64_MAX;
    h->V = s.L[0] * s.L[1];
    if (dim == 3) h->V = h->V * s.L[2];
    h->S0 = base_measure(dim, r.data(), n);
    h->phi_t = phi_t;
    s.lam_t = p.lambda_t > 0.0 ? p.lambda_t : lam_of(dim, h->S0, h->V, phi_t);

    // starting configuration
    std::vector<double> x((size_t)n * dim);
    double lam0 = 1.0;
    if (p.init == SRM_INIT_EXPLICIT) {
        if (!p.init_pos) {
            delete h;
            return fail(SRM_E_ARG, "explicit start needs init_pos");
        }
        std::memcpy(x.data(), p.init_pos, sizeof(double) * x.size());
        for (size_t i = 0; i < x.size(); i++) {
            const int a = (int)(i % dim);
            if (!(x[i] >= 0.0 && x[i] < s.L[a])) {
                delete h;
                return fail(SRM_E_ARG, "start positions must lie in [0, L)");
            }
        }
        lam0 = p.lambda0 > 0.0 ? p.lambda0 : 1.0;
    } else if (p.init == SRM_INIT_RSA_UNIFORM || p.init == SRM_INIT_RSA_CLUSTERED) {
        if (!(p.f0 > 0.0 && p.f0 <= phi_t)) {
            delete h;
            return fail(SRM_E_ARG, "f0 must be in (0, phi_t]");
        }
        lam0 = lam_of(dim, h->S0, h->V, p.f0);
        std::vector<double> R0((size_t)n);
        for (int64_t i = 0; i < n; i++) R0[(size_t)i] = lam0 * r[(size_t)i];
        const int clustered = p.init == SRM_INIT_RSA_CLUSTERED;
        if (inp_rsa(dim, s.L, n, R0.data(), seed, clustered, p.n_clusters, p.cluster_sigma,
                    100000000LL, x.data())) {
            delete h;
            return fail(SRM_E_INIT, "random sequential addition could not place every particle");
        }
    } else {
        delete h;
        return fail(SRM_E_ARG, "unknown init kind");
    }
    s.lam_P = lam0;
    s.lam_Q = lam0;

    // the minimum-image search needs at least three cells of the final size
    {
        const double cs_t = 2.5 * (s.lam_t * rmax) + p.c_m;
        for (int a = 0; a < dim; a++)
            if (s.L[a] < 3.0 * cs_t) {
                delete h;
                return fail(SRM_E_ARG, "box narrower than three cells of size 2.5 R_max + c_m");
            }
    }

    // capacities: the grid is finest at the smallest scale
    h->lam_min = (lam0 < s.lam_t ? lam0 : s.lam_t) * (1.0 - 1e-9);
    int64_t per[3];
    const int64_t ncap = cells_for(h, h->lam_min, per);
    if (ncap > 0x7ffffff0LL) {
        delete h;
        return fail(SRM_E_ARG, "too many cells (radii too small for the box)");
    }
    int64_t nsub = 1;
    for (int a = 0; a < dim; a++) nsub *= per[a] / 3;
    s.ncells_cap = (int32_t)ncap;
    h->sh.dim = dim;
    h->sh.n = n;
    h->sh.ncells_cap = ncap;
    h->sh.nsub_cap = nsub;
    h->sh.f32 = p.precision == SRM_PREC_F32;
    h->sh.out_f32 = h->sh.f32;
    h->launches_per_step = kernels_per_superstep(dim);

    // Staging capacity of the warp-per-cell sweep: the 95th percentile of
    // the stencil population of the starting positions on the grid of the
    // target scale (the coarsest grid of the run), times the part of the
    // stencil volume within reach of the home cell, with slack.  Denser
    // cells stage what fits and read the rest from global memory.
    {
        int64_t pa[3];
        const int64_t nc = cells_for(h, s.lam_t, pa);
        std::vector<uint32_t> occ((size_t)nc, 0u);
        for (int64_t i = 0; i < n; i++) {
            int64_t lin = 0, mul = 1;
            for (int a = 0; a < dim; a++) {
                const double wa = s.L[a] / (double)pa[a];
                int64_t c = (int64_t)(x[(size_t)i * dim + a] / wa);
                c = ((c % pa[a]) + pa[a]) % pa[a];
                lin += c * mul;
                mul *= pa[a];
            }
            occ[(size_t)lin]++;
        }
        std::vector<uint32_t> tpop;
        tpop.reserve((size_t)n);
        const int zr = dim == 3 ? 1 : 0;
        for (int64_t c = 0; c < nc; c++) {
            if (!occ[(size_t)c]) continue;
            const int64_t cx = c % pa[0], cy = (c / pa[0]) % pa[1], cz = c / (pa[0] * pa[1]);
            uint32_t t = 0;
            for (int dz = -zr; dz <= zr; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        const int64_t ex = (cx + dx + pa[0]) % pa[0], ey = (cy + dy + pa[1]) % pa[1],
                                      ez = (cz + dz + pa[2]) % pa[2];
                        t += occ[(size_t)(ex + pa[0] * (ey + pa[1] * ez))];
                    }
            for (uint32_t k = 0; k < occ[(size_t)c]; k++) tpop.push_back(t);  // per particle
        }
        uint32_t t95 = 0;
        if (!tpop.empty()) {
            const size_t q = tpop.size() * 95 / 100;
            std::nth_element(tpop.begin(), tpop.begin() + (ptrdiff_t)q, tpop.end());
            t95 = tpop[q];
        }
        const double wt = s.L[0] / (double)pa[0];
        const double reach = 2.0 * (2.0 * s.lam_t * rmax + 2.0 * p.c_m);
        double frac = (wt + reach) / (3.0 * wt);
        frac = frac > 1.0 ? 1.0 : frac;
        frac = dim == 3 ? frac * frac * frac : frac * frac;
        const bool f32 = p.precision == SRM_PREC_F32;
        int64_t cap = (int64_t)(1.25 * frac * (double)t95) + 16;
        cap = (cap + 31) / 32 * 32;
        if (cap < 64) cap = 64;
        h->sh.cap_sweep = (int)(cap < srm::sweep_cap_max(f32) ? cap : srm::sweep_cap_max(f32));
        h->sh.cap_check = h->sh.cap_sweep;
    }

    // device buffers
    bool ok = true;
    auto A = [&](size_t bytes) -> void * {
        void *q = dev_alloc(h, bytes);
        if (!q) ok = false;
        return q;
    };
    for (int k = 0; k < 3; k++) {
        s.slot[k].pos = A(sizeof(double4_32a) * (size_t)n);
        s.slot[k].rb = (double *)A(sizeof(double) * (size_t)n);
        s.slot[k].pid = (uint32_t *)A(sizeof(uint32_t) * (size_t)n);
        s.slot[k].cell = (uint32_t *)A(sizeof(uint32_t) * (size_t)n);
    }
    s.counts = (uint32_t *)A(sizeof(uint32_t) * (size_t)ncap);
    s.cell_start = (uint32_t *)A(sizeof(uint32_t) * (size_t)(ncap + 1));
    const int64_t parts = srm::scan_part_len((ncap > n + 1 ? ncap : n + 1));
    s.scan_part = (uint32_t *)A(sizeof(uint32_t) * (size_t)(parts + 1));
    s.src_cell = (uint32_t *)A(sizeof(uint32_t) * (size_t)n);
    s.src_rank = (uint32_t *)A(sizeof(uint32_t) * (size_t)n);
    s.flags = (uint8_t *)A((size_t)n);
    s.pcount = (uint32_t *)A(sizeof(uint32_t) * (size_t)(n + 1));
    s.red = (unsigned long long *)A(sizeof(unsigned long long) * 8);
    h->d = (RveDev *)A(sizeof(RveDev));
    double *d_x = (double *)A(sizeof(double) * x.size());
    double *d_r = (double *)A(sizeof(double) * (size_t)n);
    if (!ok) {
        dev_free_all(h);
        cudaStreamSynchronize(h->stream);
        delete h;
        return fail(SRM_E_NOMEM, "device allocation failed");
    }
    if (cudaMallocHost((void **)&h->pin, sizeof(RveDev)) != cudaSuccess ||
        cudaMallocHost((void **)&h->pin_red, sizeof(unsigned long long) * 8) != cudaSuccess) {
        dev_free_all(h);
        delete h;
        return fail(SRM_E_NOMEM, "pinned host allocation failed");
    }
    s.mode = s.lam_P >= s.lam_t ? srm::MODE_DONE : srm::MODE_BEGIN;
    s.p_idx = 0;
    s.dst_idx = 1;
    s.sweep = p.sweep0;

    srm::sweep_configure();
    srm::check_configure();
    srm_status st = SRM_OK;
    auto chk = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == SRM_OK) st = fail(SRM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    chk(cudaMemsetAsync(s.counts, 0, sizeof(uint32_t) * (size_t)ncap, h->stream), "memset");
    chk(cudaMemsetAsync(s.red, 0, sizeof(unsigned long long) * 8, h->stream), "memset");
    chk(cudaMemsetAsync(s.flags, 0, (size_t)n, h->stream), "memset");
    *h->pin = s;
    chk(cudaMemcpyAsync(h->d, h->pin, sizeof(RveDev), cudaMemcpyHostToDevice, h->stream), "state");
    chk(cudaMemcpyAsync(d_x, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice, h->stream), "x");
    chk(cudaMemcpyAsync(d_r, r.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream), "r");
    srm::launch_import(h->d, h->sh, d_x, d_r, h->stream);
    h->launches += 2;
    chk(cudaGetLastError(), "import");
    chk(cudaStreamSynchronize(h->stream), "sync");
    // record the replayed graphs now, so that no later call pays for it
    if (st == SRM_OK) st = capture(h, 1, &h->g1);
    if (st == SRM_OK) st = capture(h, h->gN_steps, &h->gN);
    if (st != SRM_OK) {
        srm_destroy(h);
        return st;
    }
    *out = h;
    return SRM_OK;
}

void srm_destroy(srm_rve *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->gN) cudaGraphExecDestroy(h->gN);
    if (h->gT) cudaGraphExecDestroy(h->gT);
    for (auto e : h->ev) cudaEventDestroy(e);
    dev_free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->pin) cudaFreeHost(h->pin);
    if (h->pin_red) cudaFreeHost(h->pin_red);
    delete h;
}

static void fill_step(srm_rve *h, srm_step_info *o, int32_t result)
{
    const RveDev &s = *h->pin;
    o->result = result;
    o->k_sweeps = s.it_k;
    o->shake_sweeps = s.it_shake;
    o->overlapping = s.it_overlap;
    o->phi = phi_of(h, s.lam_P);
    o->lambda = s.lam_P;
    o->sweep = s.sweep;
}

srm_status srm_step(srm_rve *h, srm_step_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    srm_status st = pull_state(h);
    if (st != SRM_OK) return st;
    if (h->pin->mode == srm::MODE_DONE) {
        if (out) fill_step(h, out, 2);
        return SRM_OK;
    }
    if (h->pin->mode != srm::MODE_BEGIN) return fail(SRM_E_STATE, "handle is inside an iteration");
    const int64_t it0 = h->pin->iters;
    for (;;) {
        if ((st = run_graph(h, 1)) != SRM_OK) return st;
        if ((st = pull_state(h)) != SRM_OK) return st;
        const int32_t m = h->pin->mode;
        if ((m == srm::MODE_BEGIN || m == srm::MODE_DONE) && h->pin->iters > it0) break;
        if (!h->pin->active && h->pin->iters == it0)
            return fail(SRM_E_STATE, "no iteration could start");
    }
    if (out) fill_step(h, out, h->pin->it_result);
    return SRM_OK;
}

srm_status srm_run_to_target(srm_rve *h, int64_t max_iters, srm_run_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    if (max_iters < 0) return fail(SRM_E_ARG, "max_iters must be >= 0");
    srm_status st = pull_state(h);
    if (st != SRM_OK) return st;
    const int32_t m0 = h->pin->mode;
    if (m0 != srm::MODE_BEGIN && m0 != srm::MODE_DONE) return fail(SRM_E_STATE, "handle is inside an iteration");
    const int64_t it0 = h->pin->iters;
    const int64_t cap = max_iters > INT64_MAX - it0 ? INT64_MAX : it0 + max_iters;
    k_set_cap<<<1, 1, 0, h->stream>>>(h->d, cap);
    h->launches++;
    CK(cudaGetLastError());
    int64_t last_sweeps = -1;
    const int launches_per_poll = 4;
    while (h->pin->mode != srm::MODE_DONE) {
        for (int i = 0; i < launches_per_poll; i++)
            if ((st = run_graph(h, h->gN_steps)) != SRM_OK) return st;
        if ((st = pull_state(h)) != SRM_OK) return st;
        if (h->pin->mode == srm::MODE_BEGIN && h->pin->iters >= cap && h->pin->sweeps == last_sweeps) break;
        last_sweeps = h->pin->sweeps;
    }
    k_set_cap<<<1, 1, 0, h->stream>>>(h->d, INT64_MAX);
    h->launches++;
    CK(cudaGetLastError());
    if ((st = pull_state(h)) != SRM_OK) return st;
    if (out) {
        const RveDev &s = *h->pin;
        out->iterations = s.iters;
        out->accepted = s.accepted;
        out->shaken = s.shaken;
        out->sweeps = s.sweeps;
        out->phi = phi_of(h, s.lam_P);
        out->lambda = s.lam_P;
        out->sweep = s.sweep;
    }
    if (h->pin->mode != srm::MODE_DONE)
        return fail(SRM_E_NOT_CONVERGED, "iteration cap reached before the target volume fraction");
    return SRM_OK;
}

static srm_status check_idle(srm_rve *h)
{
    srm_status st = pull_state(h);
    if (st != SRM_OK) return st;
    if (h->pin->mode != srm::MODE_BEGIN && h->pin->mode != srm::MODE_DONE)
        return fail(SRM_E_STATE, "handle is inside an iteration");
    return SRM_OK;
}

srm_status srm_certify(srm_rve *h, int64_t *overlap_pairs, double *min_gap, double *phi)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    srm_status st = check_idle(h);
    if (st != SRM_OK) return st;
    srm::launch_inspect_bin(h->d, h->sh, h->stream);
    srm::launch_pairs_count(h->d, h->sh, 1, h->stream);
    srm::launch_inspect_end(h->d, h->stream);
    h->launches += 1 + 7 + 1 + 1;
    CK(cudaGetLastError());
    if ((st = pull_state(h)) != SRM_OK) return st;
    CK(cudaMemcpyAsync(h->pin_red, h->h.red, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int64_t pairs = (int64_t)h->pin_red[1];
    unsigned long long key = h->pin_red[2];
    const unsigned long long b = (key >> 63) ? (key & 0x7fffffffffffffffULL) : ~key;
    double gap;
    std::memcpy(&gap, &b, sizeof(gap));
    if (overlap_pairs) *overlap_pairs = pairs;
    if (min_gap) *min_gap = gap;
    if (phi) *phi = phi_of(h, h->pin->lam_P);
    if (pairs > 0) return fail(SRM_E_CERTIFY_FAILED, "overlapping pairs in the final state");
    return SRM_OK;
}

srm_status srm_overlap_pairs(srm_rve *h, int64_t *ij, int64_t cap, int64_t *n)
{
    if (!h || !n || (cap > 0 && !ij)) return fail(SRM_E_ARG, "null argument");
    srm_status st = check_idle(h);
    if (st != SRM_OK) return st;
    srm::launch_inspect_bin(h->d, h->sh, h->stream);
    srm::launch_pairs_count(h->d, h->sh, 0, h->stream);
    srm::launch_scan(h->d, 1, h->sh.n, h->stream);
    h->launches += 1 + 7 + 1 + 3 + 2;
    CK(cudaGetLastError());
    uint32_t total = 0;
    CK(cudaMemcpyAsync(h->pin_red, h->h.pcount + h->sh.n, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(&total, h->pin_red, sizeof(uint32_t));
    if ((int64_t)total > h->d_ij_cap) {
        void *q = dev_alloc(h, sizeof(long long) * 2 * (size_t)total);
        if (!q) return fail(SRM_E_NOMEM, "pair buffer");
        h->d_ij = (long long *)q;
        h->d_ij_cap = total;
    }
    if (total > 0) srm::launch_pairs_fill(h->d, h->sh, h->d_ij, h->stream);
    srm::launch_inspect_end(h->d, h->stream);
    CK(cudaGetLastError());
    const int64_t m = (int64_t)total < cap ? (int64_t)total : cap;
    if (m > 0)
        CK(cudaMemcpyAsync(ij, h->d_ij, sizeof(long long) * 2 * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *n = total;
    return SRM_OK;
}

srm_status srm_positions(srm_rve *h, double *xyz, double *radii)
{
    if (!h || !xyz) return fail(SRM_E_ARG, "null argument");
    srm_status st = check_idle(h);
    if (st != SRM_OK) return st;
    const size_t n = (size_t)h->sh.n, dim = (size_t)h->sh.dim;
    if (!h->d_xyz) {
        h->d_xyz = (double *)dev_alloc(h, sizeof(double) * n * dim);
        h->d_rad = (double *)dev_alloc(h, sizeof(double) * n);
        if (!h->d_xyz || !h->d_rad) return fail(SRM_E_NOMEM, "read-back buffers");
    }
    srm::launch_gather(h->d, h->sh, h->d_xyz, h->d_rad, h->stream);
    h->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(xyz, h->d_xyz, sizeof(double) * n * dim, cudaMemcpyDeviceToHost, h->stream));
    if (radii) CK(cudaMemcpyAsync(radii, h->d_rad, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SRM_OK;
}

srm_status srm_sweep(srm_rve *h, int32_t count, int64_t *moved)
{
    if (!h || count < 0) return fail(SRM_E_ARG, "bad argument");
    srm_status st = check_idle(h);
    if (st != SRM_OK) return st;
    if (h->pin->lam_P < h->lam_min) return fail(SRM_E_ARG, "scale below the grid capacity");
    const int32_t resume = h->pin->mode;
    for (int32_t c = 0; c < count; c++) {
        k_set_mode<<<1, 1, 0, h->stream>>>(h->d, srm::MODE_SWEEP, resume);
        h->launches++;
        CK(cudaGetLastError());
        if ((st = run_graph(h, 1)) != SRM_OK) return st;
    }
    if ((st = pull_state(h)) != SRM_OK) return st;
    if (moved) *moved = h->pin->moved_last;
    return SRM_OK;
}

srm_status srm_set_scale(srm_rve *h, double lambda)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    if (!(lambda >= h->lam_min)) return fail(SRM_E_ARG, "scale below the grid capacity of this handle");
    srm_status st = check_idle(h);
    if (st != SRM_OK) return st;
    k_set_scale<<<1, 1, 0, h->stream>>>(h->d, lambda);
    h->launches++;
    CK(cudaGetLastError());
    return pull_state(h);
}

srm_status srm_get_state(srm_rve *h, srm_state_info *o)
{
    if (!h || !o) return fail(SRM_E_ARG, "null argument");
    srm_status st = pull_state(h);
    if (st != SRM_OK) return st;
    const RveDev &s = *h->pin;
    o->dim = s.dim;
    o->precision = s.prec;
    o->n = s.n;
    o->lambda = s.lam_P;
    o->lambda_t = s.lam_t;
    o->phi = phi_of(h, s.lam_P);
    o->phi_t = h->phi_t;
    o->sweep = s.sweep;
    o->iterations = s.iters;
    o->accepted = s.accepted;
    o->shaken = s.shaken;
    o->sweeps = s.sweeps;
    o->done = s.mode == srm::MODE_DONE;
    for (int a = 0; a < 3; a++) o->grid[a] = s.gn[a];
    o->kernel_launches = h->launches;
    o->pairs_sweep = s.pairs_sweep;
    o->pairs_check = s.pairs_check;
    o->stage_overflow = s.stage_overflow;
    o->stage_capacity = h->sh.cap_sweep;
    return SRM_OK;
}

srm_status srm_set_timing(srm_rve *h, int32_t on)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    h->timing = on != 0;
    std::memset(&h->tm, 0, sizeof(h->tm));
    return SRM_OK;
}

srm_status srm_get_timings(srm_rve *h, srm_timings *out)
{
    if (!h || !out) return fail(SRM_E_ARG, "null argument");
    *out = h->tm;
    return SRM_OK;
}

}  // extern "C"
