// batch.cu -- the C interface for groups of RVEs (batches and serving slots)
// and for checkpoints of a single RVE.
//
// A batch advances all its RVEs with the same launches: every kernel of a
// super-step serves every RVE (blocks are assigned to RVEs by fixed offsets,
// sweep cells are pulled from one work counter per colour), so many small
// RVEs of uneven sizes and mixed dimension fill the GPU together, and one
// captured graph replays the whole batch.  Each RVE keeps its own state
// machine, grid, Philox counters and buffers: its arithmetic does not
// depend on the other RVEs of the batch, so its result is the same alone or
// in any mix.
#include "runtime.h"

#include <algorithm>
#include <cstring>

namespace {

srm_status job_prepare(const srm_job *job, Prep &q, bool place = true)
{
    if (!job) return fail(SRM_E_ARG, "null job");
    return prepare(job->dim, job->box, &job->radii, job->phi_t, job->seed, &job->params, q, place);
}

bool valid_slot(const srm_batch *b, int32_t slot) { return b && slot >= 0 && (size_t)slot < b->g.m.size(); }

}  // namespace

extern "C" {

srm_status srm_batch_create(srm_batch **out, const srm_job *jobs, int32_t n_jobs, void *cuda_stream,
                            const srm_allocator *alloc)
{
    if (!out || !jobs || n_jobs < 1) return fail(SRM_E_ARG, "bad argument");
    *out = nullptr;
    std::vector<Prep> qs((size_t)n_jobs);
    for (int32_t i = 0; i < n_jobs; i++) {
        srm_status st = job_prepare(&jobs[i], qs[(size_t)i]);
        if (st != SRM_OK) return st;
        if (qs[(size_t)i].p.precision != qs[0].p.precision) return fail(SRM_E_ARG, "jobs of one batch share the precision");
    }
    srm_batch *b = new srm_batch();
    Group &g = b->g;
    group_setup(g, cuda_stream, alloc);
    g.f32 = qs[0].p.precision == SRM_PREC_F32;
    int cap = 64;
    double wsum = 0.0, nsum = 0.0;
    for (const Prep &q : qs) {
        cap = std::max(cap, q.cap_est);
        wsum += (double)q.n * q.cap_est;
        nsum += (double)q.n;
    }
    g.cap = default_capacity(cap, g.f32);
    g.sweep_path = DEFAULT_SWEEP_PATH;
    // the check's kernel follows the typical member (particle-weighted mean
    // estimate), not the densest one: on the ensemble of small RVEs (largest
    // estimate 448) the thread-per-particle check made the run 8% faster
    g.stencil_est = nsum > 0.0 ? (int)(wsum / nsum) : cap;
    srm_status st = SRM_OK;
    for (int32_t i = 0; i < n_jobs && st == SRM_OK; i++) {
        const Prep &q = qs[(size_t)i];
        Member *mb = new Member();
        mb->dim = q.dim;
        g.m.push_back(mb);
        if ((st = member_alloc(g, *mb, q.n, q.ncells_need, q.nsub_need)) == SRM_OK) st = member_load(g, *mb, q);
    }
    if (st == SRM_OK) st = group_finalize(g);
    if (st != SRM_OK) {
        group_free(g);
        delete b;
        return st;
    }
    *out = b;
    return SRM_OK;
}

srm_status srm_batch_create_slots(srm_batch **out, int32_t n_slots, int64_t max_particles, int64_t max_cells,
                                  int32_t dim, int32_t precision, int32_t stage_capacity, void *cuda_stream,
                                  const srm_allocator *alloc)
{
    if (!out || n_slots < 1 || max_particles < 1 || max_cells < 27) return fail(SRM_E_ARG, "bad argument");
    if (dim != 0 && dim != 2 && dim != 3) return fail(SRM_E_ARG, "dim must be 0, 2 or 3");
    if (precision != SRM_PREC_F32 && precision != SRM_PREC_F64) return fail(SRM_E_ARG, "precision must be 32 or 64");
    if (max_particles > 0x7fffffffLL || max_cells > 0x7ffffff0LL) return fail(SRM_E_ARG, "capacity too large");
    *out = nullptr;
    srm_batch *b = new srm_batch();
    Group &g = b->g;
    group_setup(g, cuda_stream, alloc);
    g.f32 = precision == SRM_PREC_F32;
    const int cap = stage_capacity > 0 ? stage_capacity : 256;
    g.cap = std::max(64, std::min((cap + 31) / 32 * 32, srm::sweep_cap_max(g.f32)));
    g.sweep_path = DEFAULT_SWEEP_PATH;
    srm_status st = SRM_OK;
    for (int32_t i = 0; i < n_slots && st == SRM_OK; i++) {
        Member *mb = new Member();
        mb->any_dim = dim == 0;  // a slot for either dimension: both sweeps are launched
        mb->dim = dim == 0 ? 3 : dim;
        mb->slot_dim = dim;
        g.m.push_back(mb);
        st = member_alloc(g, *mb, max_particles, max_cells, max_cells / 9);
    }
    if (st == SRM_OK) st = group_finalize(g);
    if (st != SRM_OK) {
        group_free(g);
        delete b;
        return st;
    }
    *out = b;
    return SRM_OK;
}

srm_status srm_job_footprint(const srm_job *job, int64_t *particles, int64_t *cells)
{
    Prep q;
    srm_status st = job_prepare(job, q, false);
    if (st != SRM_OK) return st;
    if (particles) *particles = q.n;
    if (cells) *cells = q.ncells_need;
    return SRM_OK;
}

srm_status srm_batch_admit(srm_batch *b, int32_t slot, const srm_job *job)
{
    if (!valid_slot(b, slot)) return fail(SRM_E_ARG, "bad slot");
    Group &g = b->g;
    Member &mb = *g.m[(size_t)slot];
    srm_status st = pull_state(g, (size_t)slot);
    if (st != SRM_OK) return st;
    if (mb.loaded && !mb.harvested) return fail(SRM_E_STATE, "slot is busy");
    if (mb.loaded && g.pin[slot].mode != srm::MODE_DONE) return fail(SRM_E_STATE, "slot is busy");
    Prep q;
    if ((st = job_prepare(job, q)) != SRM_OK) return st;
    if (!member_fits(mb, q)) return fail(SRM_E_ARG, "job exceeds the capacity of the slot");
    if (mb.slot_dim != 0 && q.dim != mb.slot_dim) return fail(SRM_E_ARG, "job dimension differs from the slot's");
    return member_load(g, mb, q);
}

srm_status srm_batch_advance(srm_batch *b, int32_t supersteps)
{
    if (!b || supersteps < 0) return fail(SRM_E_ARG, "bad argument");
    Group &g = b->g;
    int32_t left = supersteps;
    while (left >= g.gN_steps) {
        srm_status st = run_graph(g, g.gN_steps);
        if (st != SRM_OK) return st;
        left -= g.gN_steps;
    }
    while (left-- > 0) {
        srm_status st = run_graph(g, 1);
        if (st != SRM_OK) return st;
    }
    return SRM_OK;
}

srm_status srm_batch_autotune(srm_batch *b, int32_t supersteps, srm_tuning *best)
{
    if (!b) return fail(SRM_E_ARG, "null handle");
    return group_autotune(b->g, supersteps, best);
}

srm_status srm_batch_set_tuning(srm_batch *b, const srm_tuning *t)
{
    if (!b || !t) return fail(SRM_E_ARG, "null argument");
    return group_set_tuning(b->g, t->sweep_blocks_per_sm, t->stage_capacity, t->sweep_path);
}

srm_status srm_batch_get_tuning(srm_batch *b, srm_tuning *t)
{
    if (!b || !t) return fail(SRM_E_ARG, "null argument");
    *t = srm_tuning{};
    t->sweep_blocks_per_sm = b->g.sweep_bps;
    t->stage_capacity = b->g.cap;
    t->sweep_path = b->g.sweep_path;
    return SRM_OK;
}

srm_status srm_batch_run(srm_batch *b, int64_t max_iters)
{
    if (!b || max_iters < 0) return fail(SRM_E_ARG, "bad argument");
    return run_group(b->g, max_iters);
}

srm_status srm_batch_poll(srm_batch *b, int32_t *done_slots, int32_t cap, int32_t *n_done)
{
    if (!b || !n_done || (cap > 0 && !done_slots)) return fail(SRM_E_ARG, "bad argument");
    Group &g = b->g;
    srm_status st = pull_states(g);
    if (st != SRM_OK) return st;
    int32_t k = 0;
    for (size_t r = 0; r < g.m.size() && k < cap; r++) {
        Member &mb = *g.m[r];
        if (mb.loaded && !mb.harvested && g.pin[r].mode == srm::MODE_DONE) {
            done_slots[k++] = (int32_t)r;
            mb.harvested = true;
        }
    }
    *n_done = k;
    return SRM_OK;
}

srm_status srm_batch_release(srm_batch *b, int32_t slot)
{
    if (!valid_slot(b, slot)) return fail(SRM_E_ARG, "bad slot");
    Group &g = b->g;
    srm_status st = pull_state(g, (size_t)slot);
    if (st != SRM_OK) return st;
    if (g.pin[slot].mode != srm::MODE_DONE) return fail(SRM_E_STATE, "slot is still running");
    g.m[(size_t)slot]->harvested = true;
    return SRM_OK;
}

int32_t srm_batch_size(const srm_batch *b) { return b ? (int32_t)b->g.m.size() : 0; }

srm_status srm_batch_state(srm_batch *b, int32_t slot, srm_state_info *out)
{
    if (!valid_slot(b, slot) || !out) return fail(SRM_E_ARG, "bad argument");
    srm_status st = pull_state(b->g, (size_t)slot);
    if (st != SRM_OK) return st;
    fill_state(b->g, (size_t)slot, out);
    return SRM_OK;
}

srm_status srm_batch_positions(srm_batch *b, int32_t slot, double *xyz, double *radii)
{
    if (!valid_slot(b, slot) || !xyz) return fail(SRM_E_ARG, "bad argument");
    return member_positions(b->g, (size_t)slot, xyz, radii);
}

srm_status srm_batch_certify(srm_batch *b, int32_t slot, int64_t *overlap_pairs, double *min_gap, double *phi)
{
    if (!valid_slot(b, slot)) return fail(SRM_E_ARG, "bad slot");
    return member_certify(b->g, (size_t)slot, overlap_pairs, min_gap, phi);
}

srm_status srm_batch_set_timing(srm_batch *b, int32_t on)
{
    if (!b) return fail(SRM_E_ARG, "null batch");
    b->g.timing = on != 0;
    std::memset(&b->g.tm, 0, sizeof(b->g.tm));
    return SRM_OK;
}

srm_status srm_batch_get_timings(srm_batch *b, srm_timings *out)
{
    if (!b || !out) return fail(SRM_E_ARG, "null argument");
    *out = b->g.tm;
    return SRM_OK;
}

void srm_batch_destroy(srm_batch *b)
{
    if (!b) return;
    group_free(b->g);
    delete b;
}

// ---------------------------------------------------------------------------
// checkpoints of a single RVE
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, dim, prec, pad;
    int64_t n;
    double L[3];
    double phi_t;
    uint64_t seed;
    srm_params p;
    double rmax_unused;
    double lam_P, lam_t;
    uint64_t sweep;
    int64_t iters, accepted, shaken, sweeps;
    int32_t gn[3], mode;
    double gw[3];
};
const char kMagic[8] = {'S', 'R', 'M', 'C', 'K', 'P', 'T', '1'};
}  // namespace

srm_status srm_save(srm_rve *h, void *buf, size_t *len)
{
    if (!h || !len) return fail(SRM_E_ARG, "null argument");
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm_status st = member_idle(g, 0);
    if (st != SRM_OK) return st;
    const size_t n = (size_t)mb.n;
    const size_t pos_b = (g.f32 ? sizeof(float4) : sizeof(double4_32a)) * n;
    const size_t need = sizeof(CkptHeader) + pos_b + n * (sizeof(double) + 2 * sizeof(uint32_t)) + n * sizeof(double);
    if (!buf) {
        *len = need;
        return SRM_OK;
    }
    if (*len < need) return fail(SRM_E_ARG, "checkpoint buffer too small");
    const RveDev &s = g.pin[0];
    const srm::Slot &P = s.slot[s.p_idx];
    CkptHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.dim = mb.dim;
    hd.prec = g.f32 ? SRM_PREC_F32 : SRM_PREC_F64;
    hd.n = mb.n;
    for (int a = 0; a < 3; a++) hd.L[a] = s.L[a];
    hd.phi_t = mb.phi_t;
    hd.seed = s.seed;
    srm_params_default(&hd.p);
    hd.p.c_w = s.c_w;
    hd.p.c_m = s.c_m;
    hd.p.N_k = s.N_k;
    hd.p.N_l = s.N_l;
    hd.p.N_shake = s.N_shake;
    hd.p.precision = hd.prec;
    hd.p.guard = s.guard;
    hd.p.images = s.images;
    hd.lam_P = s.lam_P;
    hd.lam_t = s.lam_t;
    hd.sweep = s.sweep;
    hd.iters = s.iters;
    hd.accepted = s.accepted;
    hd.shaken = s.shaken;
    hd.sweeps = s.sweeps;
    hd.mode = s.mode;
    for (int a = 0; a < 3; a++) {
        hd.gn[a] = P.gn[a];
        hd.gw[a] = P.gw[a];
    }
    unsigned char *o = static_cast<unsigned char *>(buf);
    std::memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    CK(cudaMemcpyAsync(o, P.pos, pos_b, cudaMemcpyDeviceToHost, g.stream));
    o += pos_b;
    CK(cudaMemcpyAsync(o, P.rb, n * sizeof(double), cudaMemcpyDeviceToHost, g.stream));
    o += n * sizeof(double);
    CK(cudaMemcpyAsync(o, P.pid, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, g.stream));
    o += n * sizeof(uint32_t);
    CK(cudaMemcpyAsync(o, P.cell, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, g.stream));
    o += n * sizeof(uint32_t);
    // base radii in id order (to rebuild the job)
    double *rb_id = reinterpret_cast<double *>(o);
    CK(cudaStreamSynchronize(g.stream));
    const double *rb = reinterpret_cast<const double *>(static_cast<unsigned char *>(buf) + sizeof(hd) + pos_b);
    const uint32_t *pid = reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(rb) + n * sizeof(double));
    for (size_t i = 0; i < n; i++) rb_id[pid[i]] = rb[i];
    *len = need;
    return SRM_OK;
}

__global__ void k_restore(RveDev *st, srm::Slot P, int32_t p_idx, uint64_t sweep, int64_t iters, int64_t acc,
                          int64_t shaken, int64_t sweeps, int32_t mode)
{
    st->slot[p_idx] = P;
    st->p_idx = p_idx;
    st->sweep = sweep;
    st->iters = iters;
    st->accepted = acc;
    st->shaken = shaken;
    st->sweeps = sweeps;
    st->mode = mode;
}

srm_status srm_load(srm_rve **out, const void *buf, size_t len, void *cuda_stream, const srm_allocator *alloc)
{
    if (!out || !buf || len < sizeof(CkptHeader)) return fail(SRM_E_ARG, "bad checkpoint");
    *out = nullptr;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1) return fail(SRM_E_ARG, "not an SRM checkpoint");
    const size_t n = (size_t)hd.n;
    const bool f32 = hd.prec == SRM_PREC_F32;
    const size_t pos_b = (f32 ? sizeof(float4) : sizeof(double4_32a)) * n;
    const size_t need = sizeof(CkptHeader) + pos_b + n * (sizeof(double) + 2 * sizeof(uint32_t)) + n * sizeof(double);
    if (len < need) return fail(SRM_E_ARG, "truncated checkpoint");
    const unsigned char *base = static_cast<const unsigned char *>(buf) + sizeof(hd);
    const unsigned char *pos = base;
    const double *rb = reinterpret_cast<const double *>(base + pos_b);
    const uint32_t *pid = reinterpret_cast<const uint32_t *>(base + pos_b + n * sizeof(double));
    const uint32_t *cell = pid + n;
    const double *rb_id = reinterpret_cast<const double *>(cell + n);
    // absolute positions in id order: the job is rebuilt as an explicit start
    std::vector<double> x(n * (size_t)hd.dim);
    for (size_t i = 0; i < n; i++) {
        for (int a = 0; a < hd.dim; a++) {
            double v;
            if (f32) {
                const float *p4 = reinterpret_cast<const float *>(pos) + 4 * i;
                uint32_t c = cell[i], ca;
                if (a == 0) ca = c % (uint32_t)hd.gn[0];
                else if (a == 1) ca = (c / (uint32_t)hd.gn[0]) % (uint32_t)hd.gn[1];
                else ca = c / ((uint32_t)hd.gn[0] * (uint32_t)hd.gn[1]);
                v = (double)ca * hd.gw[a] + (double)p4[a];
                if (v < 0.0) v += hd.L[a];
                if (v >= hd.L[a]) v -= hd.L[a];
            } else {
                v = reinterpret_cast<const double *>(pos)[4 * i + a];
            }
            x[(size_t)pid[i] * hd.dim + a] = v;
        }
    }
    srm_radii R{};
    R.kind = SRM_RADII_EXPLICIT;
    R.n = hd.n;
    R.r = rb_id;
    srm_params p = hd.p;
    p.init = SRM_INIT_EXPLICIT;
    p.init_pos = x.data();
    p.lambda0 = hd.lam_P;
    p.lambda_t = hd.lam_t;
    p.sweep0 = hd.sweep;
    srm_rve *h = nullptr;
    srm_status st = srm_init(&h, hd.dim, hd.L, &R, hd.phi_t, hd.seed, &p, cuda_stream, alloc);
    if (st != SRM_OK) return st;
    // the accepted configuration exactly as saved (cell-sorted, offsets of
    // the FP32 form relative to the saved grid)
    Group &g = h->g;
    Member &mb = *g.m[0];
    srm::Slot P = mb.h.slot[0];
    for (int a = 0; a < 3; a++) {
        P.gn[a] = hd.gn[a];
        P.gw[a] = hd.gw[a];
    }
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        fail(SRM_E_CUDA, std::string("restore: ") + cudaGetErrorString(e));
        return true;
    };
    if (bad(cudaMemcpyAsync(P.pos, pos, pos_b, cudaMemcpyHostToDevice, g.stream)) ||
        bad(cudaMemcpyAsync(P.rb, rb, n * sizeof(double), cudaMemcpyHostToDevice, g.stream)) ||
        bad(cudaMemcpyAsync(P.pid, pid, n * sizeof(uint32_t), cudaMemcpyHostToDevice, g.stream)) ||
        bad(cudaMemcpyAsync(P.cell, cell, n * sizeof(uint32_t), cudaMemcpyHostToDevice, g.stream))) {
        srm_destroy(h);
        return SRM_E_CUDA;
    }
    k_restore<<<1, 1, 0, g.stream>>>(mb.d, P, 0, hd.sweep, hd.iters, hd.accepted, hd.shaken, hd.sweeps, hd.mode);
    g.launches++;
    if (bad(cudaGetLastError()) || bad(cudaStreamSynchronize(g.stream))) {
        srm_destroy(h);
        return SRM_E_CUDA;
    }
    *out = h;
    return SRM_OK;
}

}  // extern "C"
