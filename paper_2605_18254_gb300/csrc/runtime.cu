// runtime.cu -- host side of the C interface declared in include/srm.h:
// RVE creation and device memory, starting configurations, the captured
// super-step graphs and their replay, batches of RVEs, inspection and
// read-back.
//
// A "super-step" is one sweep of Algorithm 3 with everything around it, for
// every RVE of a group at once:
//   k_begin (state machine: swell and new grid at the start of an
//   iteration, buffer roles) -> binning (Algorithm 2) -> 3^d colour launches
//   of the sweep -> Algorithm 6 check (N_k loop only) -> k_control
//   (accept / next round / shake / done).
// Every launch reads what changes from the device state, so one captured
// CUDA graph of a few super-steps is replayed for the whole run and the host
// only polls the state every few dozen sweeps.  A single handle is a group
// of one RVE; a batch is a group of many (uneven sizes, 2D and 3D mixed),
// advanced by the same launches.
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>

extern "C" int inp_radii_lognormal(int64_t n, double mean, double sd, double lo, double hi,
                                   uint64_t seed, double *out);
extern "C" int inp_rsa(int dim, const double L[3], int64_t n, const double *R, uint64_t seed,
                       int mode, int64_t n_clusters, double sigma, int64_t max_attempts, double *X);

static thread_local std::string g_err;

srm_status fail(srm_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

namespace srm {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace srm

// ---------------------------------------------------------------------------
// host-side preparation of one job: radii, starting positions, scales,
// capacities
// ---------------------------------------------------------------------------

// sum of base disk areas / sphere volumes in id order
static double base_measure(int dim, const double *r, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double ri = r[i];
        s += dim == 2 ? M_PI * ri * ri : (4.0 / 3.0) * M_PI * ri * ri * ri;
    }
    return s;
}

double phi_of(int dim, double S0, double V, double lam)
{
    double ld = lam * lam;
    if (dim == 3) ld = ld * lam;
    return ld * S0 / V;
}

static double lam_of(int dim, double S0, double V, double phi)
{
    const double q = phi / (1.0 * S0 / V);
    return dim == 2 ? std::sqrt(q) : std::cbrt(q);
}

// cells per axis of the grid for scale lam (the device rule of set_grid)
int64_t cells_for(int dim, const double L[3], double rmax, double c_m, double lam, int64_t per_axis[3])
{
    const double cs = 2.5 * (lam * rmax) + c_m;
    int64_t tot = 1;
    for (int a = 0; a < 3; a++) {
        per_axis[a] = 1;
        if (a >= dim) continue;
        int64_t k = (int64_t)(L[a] / (3.0 * cs));
        if (k < 1) k = 1;
        per_axis[a] = 3 * k;
        tot *= per_axis[a];
    }
    return tot;
}

// Whole-stencil staging estimate: the staged path copies a cell's whole
// stencil (3^d cells) to shared memory when it fits, so this is sized from
// the mean stencil population on the grid of the target scale (the coarsest
// grid of the run, whose cells hold the most particles), 3^d N / cells, with
// room for 1.8 times the mean (measured at the end of the 1e6-sphere
// clustered run: median 1.07, maximum 1.76 times the mean).  The general
// path culls while it stages and needs less (default_capacity); denser
// cells read what does not fit from global memory (same results).
static int staging_estimate(const Prep &q)
{
    int64_t pa[3];
    const int64_t nc = cells_for(q.dim, q.L, q.rmax, q.p.c_m, q.lam_t, pa);
    const double mean = (q.dim == 3 ? 27.0 : 9.0) * (double)q.n / (double)(nc > 0 ? nc : 1);
    int64_t cap = (int64_t)(1.8 * mean) + 32;
    cap = (cap + 31) / 32 * 32;
    return (int)(cap < 64 ? 64 : cap);
}

srm_status prepare(int32_t dim, const double box[3], const srm_radii *radii, double phi_t, uint64_t seed,
                   const srm_params *pin, Prep &q, bool place)
{
    if (!box || !radii) return fail(SRM_E_ARG, "null argument");
    if (pin) q.p = *pin;
    else srm_params_default(&q.p);
    const srm_params &p = q.p;
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
    if (p.N_l > 65535) return fail(SRM_E_ARG, "N_l must be <= 65535 (the try index takes 16 counter bits)");
    if (p.precision != SRM_PREC_F64 && p.precision != SRM_PREC_F32)
        return fail(SRM_E_ARG, "precision must be 32 or 64");
    if (p.precision == SRM_PREC_F32 && !(p.guard > 0.0 && p.guard < 1e-2))
        return fail(SRM_E_ARG, "FP32 guard must be in (0, 1e-2)");
    q.dim = dim;
    q.n = n;
    q.seed = seed;
    q.phi_t = phi_t;
    for (int a = 0; a < 3; a++) q.L[a] = a < dim ? box[a] : 1.0;

    // base radii
    q.r.assign((size_t)n, 0.0);
    if (radii->kind == SRM_RADII_EXPLICIT) {
        if (!radii->r) return fail(SRM_E_ARG, "explicit radii need r");
        std::memcpy(q.r.data(), radii->r, sizeof(double) * (size_t)n);
    } else if (radii->kind == SRM_RADII_MONO) {
        for (auto &v : q.r) v = radii->mean;
    } else if (radii->kind == SRM_RADII_LOGNORMAL) {
        if (!(radii->mean > 0 && radii->sd >= 0 && radii->lo <= radii->hi))
            return fail(SRM_E_ARG, "bad log-normal parameters");
        if (inp_radii_lognormal(n, radii->mean, radii->sd, radii->lo, radii->hi, seed, q.r.data()))
            return fail(SRM_E_ARG, "log-normal truncation window too narrow");
    } else {
        return fail(SRM_E_ARG, "unknown radii kind");
    }
    q.rmax = 0.0;
    for (double v : q.r) {
        if (!(v > 0.0)) return fail(SRM_E_ARG, "radii must be > 0");
        q.rmax = v > q.rmax ? v : q.rmax;
    }
    q.V = q.L[0] * q.L[1];
    if (dim == 3) q.V = q.V * q.L[2];
    q.S0 = base_measure(dim, q.r.data(), n);
    q.lam_t = p.lambda_t > 0.0 ? p.lambda_t : lam_of(dim, q.S0, q.V, phi_t);

    // starting configuration (Algorithm 1); without `place` only the
    // scales and capacities are computed
    q.x.assign(place ? (size_t)n * dim : 0, 0.0);
    if (p.init == SRM_INIT_EXPLICIT && !place) {
        q.lam0 = p.lambda0 > 0.0 ? p.lambda0 : 1.0;
    } else if ((p.init == SRM_INIT_RSA_UNIFORM || p.init == SRM_INIT_RSA_CLUSTERED) && !place) {
        if (!(p.f0 > 0.0 && p.f0 <= phi_t)) return fail(SRM_E_ARG, "f0 must be in (0, phi_t]");
        q.lam0 = lam_of(dim, q.S0, q.V, p.f0);
    } else if (p.init == SRM_INIT_EXPLICIT) {
        if (!p.init_pos) return fail(SRM_E_ARG, "explicit start needs init_pos");
        std::memcpy(q.x.data(), p.init_pos, sizeof(double) * q.x.size());
        for (size_t i = 0; i < q.x.size(); i++) {
            const int a = (int)(i % dim);
            if (!(q.x[i] >= 0.0 && q.x[i] < q.L[a])) return fail(SRM_E_ARG, "start positions must lie in [0, L)");
        }
        q.lam0 = p.lambda0 > 0.0 ? p.lambda0 : 1.0;
    } else if (p.init == SRM_INIT_RSA_UNIFORM || p.init == SRM_INIT_RSA_CLUSTERED) {
        if (!(p.f0 > 0.0 && p.f0 <= phi_t)) return fail(SRM_E_ARG, "f0 must be in (0, phi_t]");
        q.lam0 = lam_of(dim, q.S0, q.V, p.f0);
        std::vector<double> R0((size_t)n);
        for (int64_t i = 0; i < n; i++) R0[(size_t)i] = q.lam0 * q.r[(size_t)i];
        const int clustered = p.init == SRM_INIT_RSA_CLUSTERED;
        if (inp_rsa(dim, q.L, n, R0.data(), seed, clustered, p.n_clusters, p.cluster_sigma, 100000000LL,
                    q.x.data()))
            return fail(SRM_E_INIT, "random sequential addition could not place every particle");
    } else {
        return fail(SRM_E_ARG, "unknown init kind");
    }

    // the minimum-image search needs at least three cells of the final size
    const double cs_t = 2.5 * (q.lam_t * q.rmax) + p.c_m;
    for (int a = 0; a < dim; a++)
        if (q.L[a] < 3.0 * cs_t) return fail(SRM_E_ARG, "box narrower than three cells of size 2.5 R_max + c_m");

    // capacities: the grid is finest at the smallest scale
    q.lam_min = (q.lam0 < q.lam_t ? q.lam0 : q.lam_t) * (1.0 - 1e-9);
    int64_t per[3];
    q.ncells_need = cells_for(dim, q.L, q.rmax, p.c_m, q.lam_min, per);
    if (q.ncells_need > 0x7ffffff0LL) return fail(SRM_E_ARG, "too many cells (radii too small for the box)");
    q.nsub_need = 1;
    for (int a = 0; a < dim; a++) q.nsub_need *= per[a] / 3;
    q.cap_est = staging_estimate(q);
    return SRM_OK;
}

// ---------------------------------------------------------------------------
// members (one RVE each) and groups (RVEs advanced together)
// ---------------------------------------------------------------------------
void *dev_alloc(Group &g, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g.has_alloc) {
        p = g.alloc.alloc(g.alloc.ctx, bytes, (void *)g.stream);
    } else if (cudaMallocAsync(&p, bytes, g.stream) != cudaSuccess) {
        p = nullptr;
    }
    if (p) g.owned.push_back(p);
    return p;
}

void group_free(Group &g)
{
    cudaStreamSynchronize(g.stream);
    if (g.g1) cudaGraphExecDestroy(g.g1);
    if (g.gN) cudaGraphExecDestroy(g.gN);
    if (g.gT) cudaGraphExecDestroy(g.gT);
    g.g1 = g.gN = g.gT = nullptr;
    for (auto e : g.ev) cudaEventDestroy(e);
    g.ev.clear();
    for (void *p : g.owned) {
        if (g.has_alloc) g.alloc.free(g.alloc.ctx, p, (void *)g.stream);
        else cudaFreeAsync(p, g.stream);
    }
    g.owned.clear();
    cudaStreamSynchronize(g.stream);
    if (g.cap_stream) cudaStreamDestroy(g.cap_stream);
    g.cap_stream = nullptr;

    if (g.pin) cudaFreeHost(g.pin);
    if (g.pin_red) cudaFreeHost(g.pin_red);
    g.pin = nullptr;
    g.pin_red = nullptr;
    for (Member *mm : g.m) delete mm;
    g.m.clear();
}

// Device buffers of a member with room for n_cap particles and ncells_cap
// cells (any dimension).
srm_status member_alloc(Group &g, Member &mb, int64_t n_cap, int64_t ncells_cap, int64_t nsub_cap)
{
    bool ok = true;
    auto A = [&](size_t bytes) -> void * {
        void *q = dev_alloc(g, bytes);
        if (!q) ok = false;
        return q;
    };
    RveDev &s = mb.h;
    const size_t n = (size_t)n_cap;
    for (int k = 0; k < 3; k++) {
        s.slot[k].pos = A(sizeof(double4_32a) * n);
        s.slot[k].rb = (double *)A(sizeof(double) * n);
        s.slot[k].pid = (uint32_t *)A(sizeof(uint32_t) * n);
        s.slot[k].cell = (uint32_t *)A(sizeof(uint32_t) * n);
    }
    s.counts = (uint32_t *)A(sizeof(uint32_t) * (size_t)ncells_cap);
    s.cell_start = (uint32_t *)A(sizeof(uint32_t) * (size_t)(ncells_cap + 1));
    const int64_t parts = srm::scan_part_len(ncells_cap > n_cap + 1 ? ncells_cap : n_cap + 1);
    s.scan_part = (uint32_t *)A(sizeof(uint32_t) * (size_t)(parts + 1));
    s.src_cell = (uint32_t *)A(sizeof(uint32_t) * n);
    s.src_rank = (uint32_t *)A(sizeof(uint32_t) * n);
    s.flags = (uint8_t *)A(n);
    s.pcount = (uint32_t *)A(sizeof(uint32_t) * (n + 1));
    s.red = (unsigned long long *)A(sizeof(unsigned long long) * 8);
    s.done = (uint32_t *)A(sizeof(uint32_t) * (size_t)ncells_cap);
    s.dirs = A((g.f32 ? sizeof(float4) : sizeof(double4_32a)) * 2 * n);
    mb.d = (RveDev *)A(sizeof(RveDev));
    mb.stage_x = (double *)A(sizeof(double) * 3 * n);
    mb.stage_r = (double *)A(sizeof(double) * n);
    if (!ok) return fail(SRM_E_NOMEM, "device allocation failed");
    mb.n_cap = n_cap;
    mb.ncells_cap = ncells_cap;
    mb.nsub_cap = nsub_cap;
    CK(cudaMemsetAsync(s.counts, 0, sizeof(uint32_t) * (size_t)ncells_cap, g.stream));
    CK(cudaMemsetAsync(s.red, 0, sizeof(unsigned long long) * 8, g.stream));
    CK(cudaMemsetAsync(s.flags, 0, n, g.stream));
    // an empty member takes no part in the super-steps
    s.mode = srm::MODE_DONE;
    s.n = 0;
    s.dim = 3;
    s.ncells_cap = (int32_t)ncells_cap;
    s.iter_cap = INT64_MAX;
    CK(cudaMemcpyAsync(mb.d, &s, sizeof(RveDev), cudaMemcpyHostToDevice, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    return SRM_OK;
}

bool member_fits(const Member &mb, const Prep &q)
{
    return q.n <= mb.n_cap && q.ncells_need <= mb.ncells_cap && q.nsub_need <= mb.nsub_cap;
}

// Loads a prepared job into a member: constants, fresh state, starting
// positions (uploaded and binned on the grid of the starting scale).
srm_status member_load(Group &g, Member &mb, const Prep &q)
{
    if (!member_fits(mb, q)) return fail(SRM_E_ARG, "job exceeds the capacity of the slot");
    if ((q.p.precision == SRM_PREC_F32) != g.f32) return fail(SRM_E_ARG, "job precision differs from the batch");
    RveDev &s = mb.h;
    s.dim = q.dim;
    s.prec = q.p.precision;
    s.n = (int32_t)q.n;
    s.N_k = q.p.N_k;
    s.N_l = q.p.N_l;
    s.N_shake = q.p.N_shake;
    for (int a = 0; a < 3; a++) {
        s.L[a] = q.L[a];
        s.halfL[a] = 0.5 * q.L[a];
        s.Lf[a] = (float)q.L[a];
    }
    s.rmax = q.rmax;
    s.c_w = q.p.c_w;
    s.c_m = q.p.c_m;
    s.guard = (float)q.p.guard;
    s.seed = q.seed;
    s.lam_t = q.lam_t;
    s.ncells_cap = (int32_t)mb.ncells_cap;
    s.iter_cap = INT64_MAX;
    s.lam_P = q.lam0;
    s.lam_Q = q.lam0;
    s.mode = q.lam0 >= q.lam_t ? srm::MODE_DONE : srm::MODE_BEGIN;
    s.resume_mode = s.mode;
    s.k = s.s = 0;
    s.p_idx = 0;
    s.src_idx = 0;
    s.dst_idx = 1;
    s.active = s.do_check = 0;
    s.sweep = q.p.sweep0;
    s.iters = s.accepted = s.shaken = s.sweeps = 0;
    s.it_result = s.it_k = s.it_shake = 0;
    s.it_overlap = s.moved_last = 0;
    s.status = 0;
    s.pairs_sweep = s.pairs_check = s.stage_overflow = s.trials = s.pairs_alg5 = s.near_fallback = 0;
    s.wait_limit = q.p.wait_limit == 0 ? (1 << 22) : q.p.wait_limit;
    s.images = q.p.images ? 1 : 0;
    mb.dim = q.dim;
    mb.n = q.n;
    mb.S0 = q.S0;
    mb.V = q.V;
    mb.phi_t = q.phi_t;
    mb.lam_min = q.lam_min;
    // completion stamps of an earlier job in this slot must not match
    CK(cudaMemsetAsync(s.done, 0, sizeof(uint32_t) * (size_t)mb.ncells_cap, g.stream));
    CK(cudaMemcpyAsync(mb.d, &s, sizeof(RveDev), cudaMemcpyHostToDevice, g.stream));
    CK(cudaMemcpyAsync(mb.stage_x, q.x.data(), sizeof(double) * q.x.size(), cudaMemcpyHostToDevice, g.stream));
    CK(cudaMemcpyAsync(mb.stage_r, q.r.data(), sizeof(double) * (size_t)q.n, cudaMemcpyHostToDevice, g.stream));
    srm::launch_import(mb.d, q.dim, g.f32, q.n, mb.stage_x, mb.stage_r, g.stream);
    g.launches += 2;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(g.stream));
    mb.loaded = true;
    mb.harvested = false;
    return SRM_OK;
}

static int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Device descriptor of a set of members, with the block offsets of each.
static srm_status make_batchdev(Group &g, const std::vector<Member *> &ms, BatchDev **d_out, BatchShape &sh)
{
    const int B = (int)ms.size();
    std::vector<int32_t> off(5 * (size_t)(B + 1), 0);
    int32_t *bp = off.data(), *bc = bp + B + 1, *tc = bc + B + 1, *tn = tc + B + 1, *sb = tn + B + 1;
    bool has3d = false, has2d = false;
    for (int r = 0; r < B; r++) {
        const Member &mb = *ms[(size_t)r];
        bp[r + 1] = bp[r] + blocks(mb.n_cap, 256);
        bc[r + 1] = bc[r] + blocks(mb.ncells_cap, 256);
        tc[r + 1] = tc[r] + blocks(mb.ncells_cap, srm::scan_tile());
        tn[r + 1] = tn[r] + blocks(mb.n_cap, srm::scan_tile());
        sb[r + 1] = sb[r] + (int32_t)mb.nsub_cap;
        has3d = has3d || mb.dim == 3 || mb.any_dim;
        has2d = has2d || mb.dim == 2 || mb.any_dim;
    }
    BatchDev *d = (BatchDev *)dev_alloc(g, sizeof(BatchDev));
    int32_t *d_off = (int32_t *)dev_alloc(g, sizeof(int32_t) * (off.size() + 4 * (size_t)(B + 1)));
    RveDev **d_rv = (RveDev **)dev_alloc(g, sizeof(RveDev *) * (size_t)B);
    if (!d || !d_off || !d_rv) return fail(SRM_E_NOMEM, "device allocation failed");
    std::vector<RveDev *> rv((size_t)B);
    for (int r = 0; r < B; r++) rv[(size_t)r] = ms[(size_t)r]->d;
    BatchDev hb{};
    hb.B = B;
    hb.rv = d_rv;
    hb.blk_p = d_off;
    hb.blk_c = d_off + (B + 1);
    hb.tile_c = d_off + 2 * (B + 1);
    hb.tile_n = d_off + 3 * (B + 1);
    hb.sub = d_off + 4 * (B + 1);
    hb.act2 = d_off + 5 * (B + 1);
    hb.act3 = d_off + 6 * (B + 1);
    hb.actp = d_off + 7 * (B + 1);
    hb.actc = d_off + 8 * (B + 1);
    CK(cudaMemsetAsync(hb.act2, 0, sizeof(int32_t) * 4 * (size_t)(B + 1), g.stream));
    CK(cudaMemcpyAsync(d_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, g.stream));
    CK(cudaMemcpyAsync(d_rv, rv.data(), sizeof(RveDev *) * (size_t)B, cudaMemcpyHostToDevice, g.stream));
    CK(cudaMemcpyAsync(d, &hb, sizeof(BatchDev), cudaMemcpyHostToDevice, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    *d_out = d;
    sh.d = d;
    sh.B = B;
    sh.blocks_p = bp[B];
    sh.blocks_c = bc[B];
    sh.tiles_c = tc[B];
    sh.tiles_n = tn[B];
    sh.sub_total = sb[B];
    sh.f32 = g.f32;
    sh.has3d = has3d;
    sh.has2d = has2d;
    sh.cap = g.cap;
    sh.sweep_bps = g.sweep_bps;
    sh.staged = g.sweep_path == 2;
    sh.check_cells = g.stencil_est > 256;
    return SRM_OK;
}

// kernels of one super-step: begin and plan, binning (count, 3 scan passes,
// scatter, stamp, in-cell sort), the trial draws and the sweep, check,
// control
static int64_t kernels_per_superstep(const BatchShape &sh) { return 2 + 7 + srm::sweep_launches(sh) + 1 + 1; }

static void enqueue_superstep(Group &g, cudaStream_t s, const std::vector<cudaEvent_t> *ev = nullptr)
{
    const BatchShape &sh = g.sh;
    auto mark = [&](int k) {
        if (ev) cudaEventRecordWithFlags((*ev)[(size_t)k], s, cudaEventRecordExternal);
    };
    mark(0);
    srm::launch_begin(sh, s);
    srm::launch_bin(sh, sh.f32, sh.f32, s);
    mark(1);
    srm::launch_sweep(sh, s);
    mark(2);
    srm::launch_check(sh, s);
    mark(3);
    srm::launch_control(sh, s);
    mark(4);
}

// The graph is recorded on a private stream (recording runs nothing) and
// launched on the caller's stream, which may be the legacy default stream.
static srm_status capture(Group &g, int steps, cudaGraphExec_t *out, bool timed = false)
{
    cudaGraph_t gr = nullptr;
    if (!g.cap_stream) CK(cudaStreamCreateWithFlags(&g.cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(g.cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < steps; i++) enqueue_superstep(g, g.cap_stream, timed ? &g.ev : nullptr);
    CK(cudaStreamEndCapture(g.cap_stream, &gr));
    cudaError_t e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(SRM_E_CUDA, std::string("graph: ") + cudaGetErrorString(e));
    return SRM_OK;
}

// Builds the group descriptors and records the graphs (after the members
// exist).
srm_status group_finalize(Group &g)
{
    srm::sweep_configure();
    srm::check_configure();
    srm_status st = make_batchdev(g, g.m, &g.d, g.sh);
    if (st != SRM_OK) return st;
    for (Member *mb : g.m) {
        std::vector<Member *> one{mb};
        if ((st = make_batchdev(g, one, &mb->solo_d, mb->solo)) != SRM_OK) return st;
    }
    g.launches_per_step = kernels_per_superstep(g.sh);
    const size_t B = g.m.size();
    if (cudaMallocHost((void **)&g.pin, sizeof(RveDev) * B) != cudaSuccess ||
        cudaMallocHost((void **)&g.pin_red, sizeof(unsigned long long) * 8) != cudaSuccess)
        return fail(SRM_E_NOMEM, "pinned host allocation failed");
    if ((st = capture(g, 1, &g.g1)) != SRM_OK) return st;
    return capture(g, g.gN_steps, &g.gN);
}

bool idle_mode(int32_t m);

// Launch shape of the sweep: blocks per SM of its persistent grid and the
// staging capacity.  The graphs are recorded again; results do not depend
// on either (the dataflow order is that of the cells' colours, and cells
// that do not fit the staging read the rest from global memory).
// Staging capacity when none is chosen: at most 256 culled candidates per
// warp.  Measured (GB300, FP32): on the clustered 1e6-sphere RVE the general
// kernel at capacity 256 swept 5% faster than at the whole-stencil estimate
// 704 (20 resident warps per SM instead of 12, no staging overflow).
int default_capacity(int estimate, bool f32) { return std::min(std::min(estimate, 256), srm::sweep_cap_max(f32)); }

srm_status group_set_tuning(Group &g, int sweep_bps, int cap, int path)
{
    const int cmax = srm::sweep_cap_max(g.f32);
    cap = cap <= 0 ? g.cap : (cap + 31) / 32 * 32;
    if (cap < 64) cap = 64;
    if (cap > cmax) cap = cmax;
    if (sweep_bps < 0) return fail(SRM_E_ARG, "blocks per SM must be >= 0");
    if (path < 0 || path > 2) return fail(SRM_E_ARG, "sweep path must be 0, 1 or 2");
    if (path == 2 && !g.f32) return fail(SRM_E_ARG, "the FP64 sweep has no staged variant");
    if (path == 0) path = g.sweep_path;
    CK(cudaStreamSynchronize(g.stream));
    if (g.g1) cudaGraphExecDestroy(g.g1);
    if (g.gN) cudaGraphExecDestroy(g.gN);
    if (g.gT) cudaGraphExecDestroy(g.gT);
    g.g1 = g.gN = g.gT = nullptr;
    g.cap = cap;
    g.sweep_bps = sweep_bps;
    g.sh.cap = cap;
    g.sh.sweep_bps = sweep_bps;
    g.sweep_path = path;
    g.sh.staged = path == 2;
    srm_status st = capture(g, 1, &g.g1);
    if (st != SRM_OK) return st;
    return capture(g, g.gN_steps, &g.gN);
}

// Particle sweeps done so far, summed over the group's RVEs (N x sweeps).
static double group_work(const Group &g)
{
    double w = 0.0;
    for (size_t r = 0; r < g.m.size(); r++) w += (double)g.pin[r].n * (double)g.pin[r].sweeps;
    return w;
}

// Tries each candidate launch shape on the running group, in interleaved
// rounds of `supersteps` super-steps (real work: the RVEs advance), scores
// it by device time per particle sweep, and keeps the best.
srm_status group_autotune(Group &g, int32_t supersteps, srm_tuning *best)
{
    if (supersteps < 1) return fail(SRM_E_ARG, "supersteps must be >= 1");
    // capacities at the current value and twice: never below it, since the
    // tuning runs early in a run, where stencils are sparsest, and a smaller
    // capacity measured there overflows later as the particles swell (seen on
    // the ensemble: 128 picked at the start, 8% slower over the run than 224)
    const int cap0 = g.cap, cmax = srm::sweep_cap_max(g.f32);
    std::vector<int> caps{cap0};
    for (int c : {2 * cap0}) {
        c = std::max(64, std::min(cmax, (c + 31) / 32 * 32));
        if (std::find(caps.begin(), caps.end(), c) == caps.end()) caps.push_back(c);
    }
    struct Cand {
        int bps, cap, path;
    };
    // the sweep kernel stays the current one: measured early in a run (the
    // only place the tuner can), the staged kernel looked faster on the
    // ensemble of small RVEs and was 25% slower over the whole run
    std::vector<Cand> cand;
    for (int path = g.sweep_path; path <= g.sweep_path; path++)
        for (int c : caps) {
            const int mx = srm::sweep_blocks_per_sm(g.f32, c, path == 2);
            for (int b = 2; b < mx; b++) cand.push_back({b, c, path});
            cand.push_back({0, c, path});
        }
    const int path0 = g.sweep_path;
    std::vector<double> score(cand.size(), 0.0);
    std::vector<int> seen(cand.size(), 0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int graphs = (supersteps + g.gN_steps - 1) / g.gN_steps;
    srm_status st = SRM_OK;
    for (int round = 0; round < 2 && st == SRM_OK; round++) {
        for (size_t k = 0; k < cand.size() && st == SRM_OK; k++) {
            if ((st = group_set_tuning(g, cand[k].bps, cand[k].cap, cand[k].path)) != SRM_OK) break;
            if ((st = pull_states(g)) != SRM_OK) break;
            const double w0 = group_work(g);
            CK(cudaEventRecord(e0, g.stream));
            for (int i = 0; i < graphs; i++) CK(cudaGraphLaunch(g.gN, g.stream));
            CK(cudaEventRecord(e1, g.stream));
            g.launches += g.launches_per_step * g.gN_steps * graphs;
            if ((st = pull_states(g)) != SRM_OK) break;
            const double dw = group_work(g) - w0;
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (dw > 0.0) {
                score[k] += ms / dw;
                seen[k]++;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SRM_OK) return st;
    size_t bi = 0;
    double bs = 1e300;
    for (size_t k = 0; k < cand.size(); k++)
        if (seen[k] && score[k] / seen[k] < bs) {
            bs = score[k] / seen[k];
            bi = k;
        }
    const bool any = bs < 1e300;
    const int bps = any ? cand[bi].bps : 0, cap = any ? cand[bi].cap : cap0, path = any ? cand[bi].path : path0;
    if ((st = group_set_tuning(g, bps, cap, path)) != SRM_OK) return st;
    // leave every RVE between iterations, as the other calls expect (an
    // iteration takes at most N_k + N_shake + 1 super-steps)
    for (int k = 0; k < 4096; k++) {
        if ((st = pull_states(g)) != SRM_OK) return st;
        bool idle = true;
        for (size_t r = 0; r < g.m.size(); r++) idle = idle && idle_mode(g.pin[r].mode);
        if (idle) break;
        CK(cudaGraphLaunch(g.g1, g.stream));
        g.launches += g.launches_per_step;
    }
    if (best) {
        best->sweep_blocks_per_sm = bps;
        best->stage_capacity = cap;
        best->candidates = (int32_t)cand.size();
        best->sweep_path = path;
        best->ns_per_particle_sweep = any ? 1e6 * bs : 0.0;
    }
    return SRM_OK;
}

static srm_status device_status(int32_t code)
{
    if (code == srm::STATUS_WAIT_TIMEOUT)
        return fail(SRM_E_DEVICE_TIMEOUT, "a sweep gave up waiting for a neighbouring cell (wait_limit polls)");
    return fail(SRM_E_STATE, "device state reports an error");
}

srm_status pull_states(Group &g)
{
    CK(cudaStreamSynchronize(g.stream));
    for (size_t r = 0; r < g.m.size(); r++)
        CK(cudaMemcpyAsync(&g.pin[r], g.m[r]->d, sizeof(RveDev), cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    for (size_t r = 0; r < g.m.size(); r++)
        if (g.pin[r].status != 0) return device_status(g.pin[r].status);
    return SRM_OK;
}

srm_status pull_state(Group &g, size_t r)
{
    CK(cudaMemcpyAsync(&g.pin[r], g.m[r]->d, sizeof(RveDev), cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    if (g.pin[r].status != 0) return device_status(g.pin[r].status);
    return SRM_OK;
}

static int64_t total_sweeps(const Group &g)
{
    int64_t s = 0;
    for (size_t r = 0; r < g.m.size(); r++) s += g.pin[r].sweeps;
    return s;
}

// Timing mode: one super-step per replay, with events between the stages;
// the host waits for each replay and adds up the stage times.
static srm_status run_timed(Group &g, int steps)
{
    if (g.ev.empty()) {
        g.ev.resize(5);
        for (auto &e : g.ev) CK(cudaEventCreate(&e));
    }
    if (!g.gT) {
        srm_status s = capture(g, 1, &g.gT, true);
        if (s != SRM_OK) return s;
    }
    for (int i = 0; i < steps; i++) {
        srm_status s = pull_states(g);
        if (s != SRM_OK) return s;
        const int64_t sw0 = total_sweeps(g);
        CK(cudaGraphLaunch(g.gT, g.stream));
        g.launches += g.launches_per_step;
        if ((s = pull_states(g)) != SRM_OK) return s;
        if (total_sweeps(g) == sw0) continue;  // nothing ran (targets reached or capped)
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]));
        g.tm.ms_bin += ms;
        CK(cudaEventElapsedTime(&ms, g.ev[1], g.ev[2]));
        g.tm.ms_sweep += ms;
        g.tm.sweep_launches += 1;
        CK(cudaEventElapsedTime(&ms, g.ev[2], g.ev[3]));
        g.tm.ms_check += ms;
        bool checked = false;
        for (size_t r = 0; r < g.m.size(); r++) checked = checked || g.pin[r].do_check;
        if (checked) g.tm.check_launches += 1;
        CK(cudaEventElapsedTime(&ms, g.ev[3], g.ev[4]));
        g.tm.ms_control += ms;
        g.tm.supersteps += 1;
    }
    return SRM_OK;
}

srm_status run_graph(Group &g, int steps)
{
    if (g.timing) return run_timed(g, steps == 1 ? 1 : g.gN_steps);
    cudaGraphExec_t ge = steps == 1 ? g.g1 : g.gN;
    CK(cudaGraphLaunch(ge, g.stream));
    g.launches += g.launches_per_step * (steps == 1 ? 1 : g.gN_steps);
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

void launch_set_cap(Group &g, size_t r, int64_t cap)
{
    k_set_cap<<<1, 1, 0, g.stream>>>(g.m[r]->d, cap);
    g.launches++;
}

bool idle_mode(int32_t m) { return m == srm::MODE_BEGIN || m == srm::MODE_DONE; }

// Replays super-steps until every member is done, or until no member can
// start a new iteration (iteration caps) -- then SRM_E_NOT_CONVERGED.
srm_status run_group(Group &g, int64_t max_iters)
{
    srm_status st = pull_states(g);
    if (st != SRM_OK) return st;
    for (size_t r = 0; r < g.m.size(); r++)
        if (!idle_mode(g.pin[r].mode)) return fail(SRM_E_STATE, "an RVE is inside an iteration");
    for (size_t r = 0; r < g.m.size(); r++) {
        const int64_t it0 = g.pin[r].iters;
        launch_set_cap(g, r, max_iters > INT64_MAX - it0 ? INT64_MAX : it0 + max_iters);
    }
    CK(cudaGetLastError());
    int64_t last = -1;
    const int launches_per_poll = 4;
    for (;;) {
        if ((st = pull_states(g)) != SRM_OK) return st;
        bool all_done = true;
        for (size_t r = 0; r < g.m.size(); r++) all_done = all_done && g.pin[r].mode == srm::MODE_DONE;
        if (all_done) break;
        const int64_t sw = total_sweeps(g);
        if (sw == last) break;  // nothing moves: capped
        last = sw;
        for (int i = 0; i < launches_per_poll; i++)
            if ((st = run_graph(g, g.gN_steps)) != SRM_OK) return st;
    }
    for (size_t r = 0; r < g.m.size(); r++) launch_set_cap(g, r, INT64_MAX);
    CK(cudaGetLastError());
    if ((st = pull_states(g)) != SRM_OK) return st;
    for (size_t r = 0; r < g.m.size(); r++)
        if (g.pin[r].mode != srm::MODE_DONE)
            return fail(SRM_E_NOT_CONVERGED, "iteration cap reached before the target volume fraction");
    return SRM_OK;
}

// ---------------------------------------------------------------------------
// per-member operations (inspection and read-back)
// ---------------------------------------------------------------------------
srm_status member_idle(Group &g, size_t r)
{
    srm_status st = pull_state(g, r);
    if (st != SRM_OK) return st;
    if (!idle_mode(g.pin[r].mode)) return fail(SRM_E_STATE, "RVE is inside an iteration");
    return SRM_OK;
}

srm_status member_certify(Group &g, size_t r, int64_t *overlap_pairs, double *min_gap, double *phi)
{
    Member &mb = *g.m[r];
    srm_status st = member_idle(g, r);
    if (st != SRM_OK) return st;
    if (!mb.loaded) return fail(SRM_E_STATE, "empty slot");
    srm::launch_inspect_bin(mb.d, mb.solo, g.stream);
    srm::launch_pairs_count(mb.d, mb.dim, mb.n, 1, g.stream);
    srm::launch_inspect_end(mb.d, g.stream);
    g.launches += 1 + 1 + 7 + 1 + 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(g.pin_red, mb.h.red, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    const int64_t pairs = (int64_t)g.pin_red[1];
    const unsigned long long key = g.pin_red[2];
    const unsigned long long b = (key >> 63) ? (key & 0x7fffffffffffffffULL) : ~key;
    double gap;
    std::memcpy(&gap, &b, sizeof(gap));
    if (overlap_pairs) *overlap_pairs = pairs;
    if (min_gap) *min_gap = gap;
    if (phi) *phi = phi_of(mb.dim, mb.S0, mb.V, g.pin[r].lam_P);
    if (pairs > 0) return fail(SRM_E_CERTIFY_FAILED, "overlapping pairs in the final state");
    return SRM_OK;
}

srm_status member_positions(Group &g, size_t r, double *xyz, double *radii)
{
    Member &mb = *g.m[r];
    srm_status st = member_idle(g, r);
    if (st != SRM_OK) return st;
    if (!mb.loaded) return fail(SRM_E_STATE, "empty slot");
    const size_t n = (size_t)mb.n, dim = (size_t)mb.dim;
    if (!mb.d_xyz) {
        mb.d_xyz = (double *)dev_alloc(g, sizeof(double) * (size_t)mb.n_cap * 3);
        mb.d_rad = (double *)dev_alloc(g, sizeof(double) * (size_t)mb.n_cap);
        if (!mb.d_xyz || !mb.d_rad) return fail(SRM_E_NOMEM, "read-back buffers");
    }
    srm::launch_gather(mb.d, mb.dim, g.f32, mb.n, mb.d_xyz, mb.d_rad, g.stream);
    g.launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(xyz, mb.d_xyz, sizeof(double) * n * dim, cudaMemcpyDeviceToHost, g.stream));
    if (radii) CK(cudaMemcpyAsync(radii, mb.d_rad, sizeof(double) * n, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    return SRM_OK;
}

void fill_state(const Group &g, size_t r, srm_state_info *o)
{
    const RveDev &s = g.pin[r];
    const Member &mb = *g.m[r];
    o->dim = mb.dim;
    o->precision = g.f32 ? SRM_PREC_F32 : SRM_PREC_F64;
    o->n = mb.n;
    o->lambda = s.lam_P;
    o->lambda_t = s.lam_t;
    o->phi = mb.loaded ? phi_of(mb.dim, mb.S0, mb.V, s.lam_P) : 0.0;
    o->phi_t = mb.phi_t;
    o->sweep = s.sweep;
    o->iterations = s.iters;
    o->accepted = s.accepted;
    o->shaken = s.shaken;
    o->sweeps = s.sweeps;
    o->done = s.mode == srm::MODE_DONE;
    for (int a = 0; a < 3; a++) o->grid[a] = s.gn[a];
    o->kernel_launches = g.launches;
    o->pairs_sweep = s.pairs_sweep;
    o->pairs_check = s.pairs_check;
    o->stage_overflow = s.stage_overflow;
    o->trials = s.trials;
    o->pairs_alg5 = s.pairs_alg5;
    o->near_fallback = s.near_fallback;
    o->stage_capacity = g.cap;
    o->check_kernel = g.sh.check_cells ? 1 : 0;
}

// ---------------------------------------------------------------------------
// C interface: single RVE
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

srm_status srm_init(srm_rve **out, int32_t dim, const double box[3], const srm_radii *radii, double phi_t,
                    uint64_t seed, const srm_params *p, void *cuda_stream, const srm_allocator *alloc)
{
    g_err.clear();
    if (!out) return fail(SRM_E_ARG, "null argument");
    *out = nullptr;
    Prep q;
    srm_status st = prepare(dim, box, radii, phi_t, seed, p, q);
    if (st != SRM_OK) return st;
    srm_rve *h = new srm_rve();
    Group &g = h->g;
    group_setup(g, cuda_stream, alloc);
    g.f32 = q.p.precision == SRM_PREC_F32;
    g.cap = default_capacity(q.cap_est, g.f32);
    g.sweep_path = DEFAULT_SWEEP_PATH;
    g.stencil_est = q.cap_est;
    Member *mb = new Member();
    mb->dim = q.dim;
    g.m.push_back(mb);
    if ((st = member_alloc(g, *mb, q.n, q.ncells_need, q.nsub_need)) == SRM_OK &&
        (st = member_load(g, *mb, q)) == SRM_OK)
        st = group_finalize(g);
    if (st != SRM_OK) {
        const std::string msg = g_err;
        group_free(g);
        delete h;
        g_err = msg;
        return st;
    }
    *out = h;
    return SRM_OK;
}

void srm_destroy(srm_rve *h)
{
    if (!h) return;
    group_free(h->g);
    delete h;
}

srm_status srm_step(srm_rve *h, srm_step_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    Group &g = h->g;
    srm_status st = pull_state(g, 0);
    if (st != SRM_OK) return st;
    const Member &mb = *g.m[0];
    auto fill = [&](int32_t result) {
        if (!out) return;
        const RveDev &s = g.pin[0];
        out->result = result;
        out->k_sweeps = s.it_k;
        out->shake_sweeps = s.it_shake;
        out->overlapping = s.it_overlap;
        out->phi = phi_of(mb.dim, mb.S0, mb.V, s.lam_P);
        out->lambda = s.lam_P;
        out->sweep = s.sweep;
    };
    if (g.pin[0].mode == srm::MODE_DONE) {
        fill(2);
        return SRM_OK;
    }
    if (g.pin[0].mode != srm::MODE_BEGIN) return fail(SRM_E_STATE, "handle is inside an iteration");
    const int64_t it0 = g.pin[0].iters;
    for (;;) {
        if ((st = run_graph(g, 1)) != SRM_OK) return st;
        if ((st = pull_state(g, 0)) != SRM_OK) return st;
        if (idle_mode(g.pin[0].mode) && g.pin[0].iters > it0) break;
        if (!g.pin[0].active && g.pin[0].iters == it0) return fail(SRM_E_STATE, "no iteration could start");
    }
    fill(g.pin[0].it_result);
    return SRM_OK;
}

srm_status srm_run_to_target(srm_rve *h, int64_t max_iters, srm_run_info *out)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    if (max_iters < 0) return fail(SRM_E_ARG, "max_iters must be >= 0");
    Group &g = h->g;
    const srm_status st = run_group(g, max_iters);
    if (st != SRM_OK && st != SRM_E_NOT_CONVERGED) return st;
    if (out) {
        const RveDev &s = g.pin[0];
        const Member &mb = *g.m[0];
        out->iterations = s.iters;
        out->accepted = s.accepted;
        out->shaken = s.shaken;
        out->sweeps = s.sweeps;
        out->phi = phi_of(mb.dim, mb.S0, mb.V, s.lam_P);
        out->lambda = s.lam_P;
        out->sweep = s.sweep;
    }
    return st;
}

srm_status srm_certify(srm_rve *h, int64_t *overlap_pairs, double *min_gap, double *phi)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    return member_certify(h->g, 0, overlap_pairs, min_gap, phi);
}

// ---------------------------------------------------------------------------
// Structure descriptors of P (Section 3.2), on its binary64 binning at its
// own scale (as the certification).
// ---------------------------------------------------------------------------
static void *analysis_scratch(Group &g, Member &mb, size_t bytes)
{
    if (bytes > mb.an_bytes) {
        void *q = dev_alloc(g, bytes);
        if (!q) return nullptr;
        mb.d_an = q;
        mb.an_bytes = bytes;
    }
    return mb.d_an;
}

srm_status srm_nearest(srm_rve *h, double *nn_dist, int64_t *nn_id, double *gap)
{
    if (!h || !nn_dist || !gap) return fail(SRM_E_ARG, "null argument");
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    const size_t n = (size_t)mb.n;
    unsigned char *buf = (unsigned char *)analysis_scratch(g, mb, 24 * n);
    if (!buf) return fail(SRM_E_NOMEM, "analysis scratch");
    double *d_dist = (double *)buf, *d_gap = (double *)(buf + 8 * n);
    long long *d_id = (long long *)(buf + 16 * n);
    srm::launch_inspect_bin(mb.d, mb.solo, g.stream);
    srm::launch_nearest(mb.d, mb.dim, mb.n, d_dist, d_id, d_gap, g.stream);
    srm::launch_inspect_end(mb.d, g.stream);
    g.launches += 1 + 1 + 7 + 1 + 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(nn_dist, d_dist, 8 * n, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaMemcpyAsync(gap, d_gap, 8 * n, cudaMemcpyDeviceToHost, g.stream));
    if (nn_id) CK(cudaMemcpyAsync(nn_id, d_id, 8 * n, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    return SRM_OK;
}

srm_status srm_rdf(srm_rve *h, double r_max, int32_t bins, int64_t *counts, double *gr)
{
    if (!h || !counts) return fail(SRM_E_ARG, "null argument");
    if (!(r_max > 0.0) || bins < 1 || bins > 4096) return fail(SRM_E_ARG, "need r_max > 0 and 1 <= bins <= 4096");
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    const RveDev &s0 = mb.h;
    for (int a = 0; a < mb.dim; a++)
        if (r_max > 0.5 * s0.L[a]) return fail(SRM_E_ARG, "r_max exceeds half the box (minimum image)");
    unsigned long long *d_c = (unsigned long long *)analysis_scratch(g, mb, sizeof(unsigned long long) * (size_t)bins);
    if (!d_c) return fail(SRM_E_NOMEM, "analysis scratch");
    CK(cudaMemsetAsync(d_c, 0, sizeof(unsigned long long) * (size_t)bins, g.stream));
    srm::launch_inspect_bin(mb.d, mb.solo, g.stream);
    if ((st = pull_state(g, 0)) != SRM_OK) return st;  // the grid of the inspection binning
    const RveDev &sv = g.pin[0];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < mb.dim; a++) {
        const int H = (int)std::ceil(r_max / sv.gw[a]);
        if (2 * H + 1 >= sv.gn[a]) {
            lo[a] = 0;
            hi[a] = sv.gn[a] - 1;
        } else {
            lo[a] = -H;
            hi[a] = H;
        }
    }
    srm::launch_rdf(mb.d, mb.dim, mb.n, r_max, bins, lo, hi, d_c, g.stream);
    srm::launch_inspect_end(mb.d, g.stream);
    g.launches += 1 + 1 + 7 + 1 + 1;
    CK(cudaGetLastError());
    std::vector<unsigned long long> hc((size_t)bins);
    CK(cudaMemcpyAsync(hc.data(), d_c, sizeof(unsigned long long) * (size_t)bins, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    double V = 1.0;
    for (int a = 0; a < mb.dim; a++) V *= s0.L[a];
    const double pi = 3.14159265358979323846, dr = r_max / (double)bins, N = (double)mb.n;
    for (int b = 0; b < bins; b++) {
        counts[b] = (int64_t)hc[(size_t)b];
        if (gr) {
            const double r0 = b * dr, r1 = (b + 1) * dr;
            const double shell =
                mb.dim == 2 ? pi * (r1 * r1 - r0 * r0) : 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
            gr[b] = (double)counts[b] * V / (N * (N - 1.0) * shell);
        }
    }
    return SRM_OK;
}

srm_status srm_voronoi_lvf(srm_rve *h, const int32_t voxels[3], int64_t *count, double *lvf)
{
    if (!h || !voxels || !count) return fail(SRM_E_ARG, "null argument");
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    int32_t M[3] = {1, 1, 1};
    double hv[3] = {1.0, 1.0, 1.0};
    long long total = 1;
    for (int a = 0; a < mb.dim; a++) {
        if (voxels[a] < 1 || voxels[a] > 65536) return fail(SRM_E_ARG, "voxels per axis must be in [1, 65536]");
        M[a] = voxels[a];
        hv[a] = mb.h.L[a] / (double)M[a];
        total *= M[a];
    }
    if (total > (1LL << 34)) return fail(SRM_E_ARG, "more than 2^34 voxels");
    const size_t n = (size_t)mb.n;
    unsigned long long *d_c = (unsigned long long *)analysis_scratch(g, mb, 8 * n);
    if (!d_c) return fail(SRM_E_NOMEM, "analysis scratch");
    CK(cudaMemsetAsync(d_c, 0, 8 * n, g.stream));
    srm::launch_inspect_bin(mb.d, mb.solo, g.stream);
    srm::launch_voronoi(mb.d, mb.dim, M, hv, d_c, g.stream);
    srm::launch_inspect_end(mb.d, g.stream);
    g.launches += 1 + 1 + 7 + 1 + 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(count, d_c, 8 * n, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    if (lvf) {
        std::vector<double> xyz(n * (size_t)mb.dim), rad(n);
        if ((st = member_positions(g, 0, xyz.data(), rad.data())) != SRM_OK) return st;
        double cell = 1.0;
        for (int a = 0; a < mb.dim; a++) cell *= hv[a];
        const double pi = 3.14159265358979323846;
        for (size_t j = 0; j < n; j++) {
            const double R = rad[j];
            const double v = mb.dim == 2 ? pi * R * R : 4.0 / 3.0 * pi * R * R * R;
            lvf[j] = count[j] ? v / ((double)count[j] * cell) : HUGE_VAL;
        }
    }
    return SRM_OK;
}

srm_status srm_autotune(srm_rve *h, int32_t supersteps, srm_tuning *best)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    return group_autotune(h->g, supersteps, best);
}

srm_status srm_set_tuning(srm_rve *h, const srm_tuning *t)
{
    if (!h || !t) return fail(SRM_E_ARG, "null argument");
    return group_set_tuning(h->g, t->sweep_blocks_per_sm, t->stage_capacity, t->sweep_path);
}

srm_status srm_get_tuning(srm_rve *h, srm_tuning *t)
{
    if (!h || !t) return fail(SRM_E_ARG, "null argument");
    *t = srm_tuning{};
    t->sweep_blocks_per_sm = h->g.sweep_bps;
    t->stage_capacity = h->g.cap;
    t->sweep_path = h->g.sweep_path;
    return SRM_OK;
}

srm_status srm_overlap_pairs(srm_rve *h, int64_t *ij, int64_t cap, int64_t *n)
{
    if (!h || !n || (cap > 0 && !ij)) return fail(SRM_E_ARG, "null argument");
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    srm::launch_inspect_bin(mb.d, mb.solo, g.stream);
    srm::launch_pairs_count(mb.d, mb.dim, mb.n, 0, g.stream);
    srm::launch_scan(mb.solo, 1, g.stream);
    g.launches += 1 + 1 + 7 + 1 + 3;
    CK(cudaGetLastError());
    uint32_t total = 0;
    CK(cudaMemcpyAsync(g.pin_red, mb.h.pcount + mb.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    std::memcpy(&total, g.pin_red, sizeof(uint32_t));
    if ((int64_t)total > mb.d_ij_cap) {
        void *q = dev_alloc(g, sizeof(long long) * 2 * (size_t)total);
        if (!q) return fail(SRM_E_NOMEM, "pair buffer");
        mb.d_ij = (long long *)q;
        mb.d_ij_cap = total;
    }
    if (total > 0) {
        srm::launch_pairs_fill(mb.d, mb.dim, mb.n, mb.d_ij, g.stream);
        g.launches++;
    }
    srm::launch_inspect_end(mb.d, g.stream);
    g.launches++;
    CK(cudaGetLastError());
    const int64_t m = (int64_t)total < cap ? (int64_t)total : cap;
    if (m > 0) CK(cudaMemcpyAsync(ij, mb.d_ij, sizeof(long long) * 2 * (size_t)m, cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    *n = total;
    return SRM_OK;
}

srm_status srm_positions(srm_rve *h, double *xyz, double *radii)
{
    if (!h || !xyz) return fail(SRM_E_ARG, "null argument");
    return member_positions(h->g, 0, xyz, radii);
}

srm_status srm_sweep(srm_rve *h, int32_t count, int64_t *moved)
{
    if (!h || count < 0) return fail(SRM_E_ARG, "bad argument");
    Group &g = h->g;
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    if (g.pin[0].lam_P < g.m[0]->lam_min) return fail(SRM_E_ARG, "scale below the grid capacity");
    const int32_t resume = g.pin[0].mode;
    for (int32_t c = 0; c < count; c++) {
        k_set_mode<<<1, 1, 0, g.stream>>>(g.m[0]->d, srm::MODE_SWEEP, resume);
        g.launches++;
        CK(cudaGetLastError());
        if ((st = run_graph(g, 1)) != SRM_OK) return st;
    }
    if ((st = pull_state(g, 0)) != SRM_OK) return st;
    if (moved) *moved = g.pin[0].moved_last;
    return SRM_OK;
}

srm_status srm_set_scale(srm_rve *h, double lambda)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    Group &g = h->g;
    if (!(lambda >= g.m[0]->lam_min)) return fail(SRM_E_ARG, "scale below the grid capacity of this handle");
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    k_set_scale<<<1, 1, 0, g.stream>>>(g.m[0]->d, lambda);
    g.launches++;
    CK(cudaGetLastError());
    return pull_state(g, 0);
}

srm_status srm_get_state(srm_rve *h, srm_state_info *o)
{
    if (!h || !o) return fail(SRM_E_ARG, "null argument");
    srm_status st = pull_state(h->g, 0);
    if (st != SRM_OK) return st;
    fill_state(h->g, 0, o);
    return SRM_OK;
}

srm_status srm_set_timing(srm_rve *h, int32_t on)
{
    if (!h) return fail(SRM_E_ARG, "null handle");
    h->g.timing = on != 0;
    std::memset(&h->g.tm, 0, sizeof(h->g.tm));
    return SRM_OK;
}

srm_status srm_get_timings(srm_rve *h, srm_timings *out)
{
    if (!h || !out) return fail(SRM_E_ARG, "null argument");
    *out = h->g.tm;
    return SRM_OK;
}

}  // extern "C"
