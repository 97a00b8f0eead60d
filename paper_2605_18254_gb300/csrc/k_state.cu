// k_state.cu -- the per-RVE state machine of Algorithm 1 (one thread per
// RVE) and the binning of Algorithm 2 as a counting sort into cell-sorted
// structure-of-arrays copies: cell ids with an atomic histogram, an
// exclusive scan over cells, a scatter, and an in-cell sort by particle id
// that makes the order of every cell canonical.
#include "srm_dev.cuh"
#include "srm_launch.h"

#include <type_traits>

namespace srm {

__global__ void k_begin(BatchDev *bd)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        bd->wq[0] = 0u;
        bd->wq[1] = 0u;
    }
    if (r >= bd->B) return;
    RveDev *st = bd->rv[r];
    st->active = 0;
    st->do_check = 0;
    const int32_t mode = st->mode;
    if (mode == MODE_DONE) return;
    if (mode == MODE_BEGIN) {
        if (st->lam_P >= st->lam_t) {
            st->mode = MODE_DONE;
            return;
        }
        if (st->iters >= st->iter_cap) return;
        st->iters++;
        double lq = __dmul_rn(st->lam_P, __dadd_rn(1.0, st->c_w));
        if (lq > st->lam_t) lq = st->lam_t;
        st->lam_Q = lq;
        set_grid(st, lq);
        st->k = 0;
        st->s = 0;
        st->mode = MODE_KLOOP;
        st->src_idx = st->p_idx;
    } else if (mode == MODE_KLOOP) {
        st->src_idx = st->dst_idx;
    } else if (mode == MODE_SHAKE) {
        st->src_idx = st->p_idx;
    } else if (mode == MODE_SWEEP) {
        set_grid(st, st->lam_P);
        st->src_idx = st->p_idx;
    }
    const int32_t src = st->src_idx, p = st->p_idx;
    st->dst_idx = src == p ? (p + 1) % 3 : 3 - p - src;
    st->lam_R = st->mode == MODE_KLOOP ? st->lam_Q : st->lam_P;
    st->do_check = st->mode == MODE_KLOOP;
    st->active = 1;
    st->red[0] = 0;
    st->red[3] = 0;
}

__global__ void k_control(BatchDev *bd)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= bd->B) return;
    RveDev *st = bd->rv[r];
    if (!st->active) return;
    st->sweep++;
    st->sweeps++;
    st->moved_last = (int64_t)st->red[3];
    const int32_t mode = st->mode;
    if (mode == MODE_KLOOP) {
        st->k++;
        const int64_t cnt = (int64_t)st->red[0];
        if (cnt == 0) {
            st->p_idx = st->dst_idx;
            st->lam_P = st->lam_Q;
            st->accepted++;
            st->it_result = 1;
            st->it_k = st->k;
            st->it_shake = 0;
            st->it_overlap = 0;
            st->mode = st->lam_P >= st->lam_t ? MODE_DONE : MODE_BEGIN;
        } else if (st->k >= st->N_k) {
            st->it_k = st->k;
            st->it_overlap = cnt;
            if (st->N_shake > 0) {
                st->mode = MODE_SHAKE;
                st->s = 0;
            } else {
                st->shaken++;
                st->it_result = 0;
                st->it_shake = 0;
                st->mode = MODE_BEGIN;
            }
        }
    } else if (mode == MODE_SHAKE) {
        st->s++;
        st->p_idx = st->dst_idx;
        if (st->s >= st->N_shake) {
            st->shaken++;
            st->it_result = 0;
            st->it_shake = st->s;
            st->mode = MODE_BEGIN;
        }
    } else if (mode == MODE_SWEEP) {
        st->p_idx = st->dst_idx;
        st->mode = st->resume_mode;
    }
}

// Work plans of this super-step, over the RVEs at work only (finished or
// empty members of a batch cost nothing): the colour cells of the 2D and of
// the 3D RVEs (sweep work items), and the 256-wide particle and cell chunks
// (particle- and cell-indexed kernels).  One block: block-wide exclusive
// scans of the four per-RVE counts.
__global__ void __launch_bounds__(1024) k_plan(BatchDev *bd)
{
    constexpr int Q = 4;
    const int B = bd->B;
    __shared__ int32_t carry[Q];
    __shared__ int32_t ws[Q][32];
    int32_t *const out[Q] = {bd->act2, bd->act3, bd->actp, bd->actc};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x < Q) carry[threadIdx.x] = 0;
    __syncthreads();
    for (int base = 0; base < B; base += blockDim.x) {
        const int r = base + threadIdx.x;
        int32_t v[Q] = {0, 0, 0, 0};
        if (r < B) {
            const RveDev *st = bd->rv[r];
            if (st->active) {
                v[0] = st->dim == 2 ? st->nsub : 0;
                v[1] = st->dim == 3 ? st->nsub : 0;
                v[2] = (st->n + 255) / 256;
                v[3] = (st->ncells + 255) / 256;
            }
        }
        int32_t x[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            x[q] = v[q];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, x[q], o);
                if (lane >= o) x[q] += y;
            }
            if (lane == 31) ws[q][wid] = x[q];
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int q = 0; q < Q; q++) {
                int32_t t = lane < nw ? ws[q][lane] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                ws[q][lane] = t;
            }
        }
        __syncthreads();
        int32_t before[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            before[q] = wid ? ws[q][wid - 1] : 0;
            if (r < B) out[q][r] = carry[q] + before[q] + x[q] - v[q];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            for (int q = 0; q < Q; q++) carry[q] += before[q] + x[q];
        __syncthreads();
    }
    if (threadIdx.x < Q) out[threadIdx.x][B] = carry[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Binning.  The source slot (P or the previous working copy) is read in its
// stored order; each particle gets its cell and a rank from an atomic
// histogram; the scan turns counts into cell starts (and clears the counts);
// the scatter writes the destination slot; the in-cell sort restores
// ascending particle id inside each cell.
// ---------------------------------------------------------------------------
template <int DIM, bool F32>
__device__ __forceinline__ void src_abs(const RveDev *st, const Slot &s, int i, double x[3])
{
    if (!F32) {
        const double4_32a p = reinterpret_cast<const double4_32a *>(s.pos)[i];
        x[0] = p.x;
        x[1] = p.y;
        x[2] = p.z;
    } else {
        const float4 p = reinterpret_cast<const float4 *>(s.pos)[i];
        const uint32_t c = s.cell[i];
        const int32_t cx = (int32_t)(c % (uint32_t)s.gn[0]);
        const int32_t cy = (int32_t)((c / (uint32_t)s.gn[0]) % (uint32_t)s.gn[1]);
        const int32_t cz = (int32_t)(c / ((uint32_t)s.gn[0] * (uint32_t)s.gn[1]));
        const float o[3] = {p.x, p.y, p.z};
        const int32_t cc[3] = {cx, cy, cz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (a < DIM)
                x[a] = wrap_d(__dadd_rn(__dmul_rn((double)cc[a], s.gw[a]), (double)o[a]), st->L[a]);
            else
                x[a] = 0.0;
        }
    }
}

// FP32 form on an unchanged grid: a particle has moved less than one cell
// since it was binned, so its new cell is the old one shifted by
// floor(offset / w) per axis (wrapped) and its offset is re-expressed in
// binary32; no binary64 arithmetic.  Count and scatter evaluate the same
// expressions, so they agree on the cell.
template <int DIM>
__device__ __forceinline__ uint32_t shift_cell_f32(const RveDev *st, const Slot &s, int i, float o[3])
{
    const float4 p = reinterpret_cast<const float4 *>(s.pos)[i];
    const uint32_t c = s.cell[i];
    int32_t cc[3];
    cc[0] = (int32_t)(c % (uint32_t)s.gn[0]);
    cc[1] = (int32_t)((c / (uint32_t)s.gn[0]) % (uint32_t)s.gn[1]);
    cc[2] = (int32_t)(c / ((uint32_t)s.gn[0] * (uint32_t)s.gn[1]));
    o[0] = p.x;
    o[1] = p.y;
    o[2] = p.z;
    uint32_t lin = 0, mul = 1;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const float w = (float)st->gw[a];
        const int32_t n = st->gn[a];
        const int32_t sh = (int32_t)floorf(o[a] / w);
        o[a] = __fmaf_rn(-(float)sh, w, o[a]);  // one rounding, wherever inlined
        int32_t ca = (cc[a] + sh) % n;
        ca += ca < 0 ? n : 0;
        lin += (uint32_t)ca * mul;
        mul *= (uint32_t)n;
    }
    return lin;
}

__device__ __forceinline__ bool same_grid(const RveDev *st, const Slot &s)
{
    return s.gn[0] == st->gn[0] && s.gn[1] == st->gn[1] && s.gn[2] == st->gn[2];
}

template <int DIM, bool F32, bool FAST>
__device__ __forceinline__ void bin_count_one(RveDev *st, int i)
{
    const Slot s = st->slot[st->src_idx];
    uint32_t lin = 0;
    if (FAST && same_grid(st, s)) {
        float o[3];
        lin = shift_cell_f32<DIM>(st, s, i, o);
    } else {
        double x[3];
        src_abs<DIM, F32>(st, s, i, x);
        uint32_t mul = 1;
#pragma unroll
        for (int a = 0; a < DIM; a++) {
            lin += (uint32_t)cell_coord_d(x[a], st->gw[a], st->gn[a]) * mul;
            mul *= (uint32_t)st->gn[a];
        }
    }
    st->src_cell[i] = lin;
    st->src_rank[i] = atomicAdd(&st->counts[lin], 1u);
}

template <bool F32, bool FAST>
__global__ void __launch_bounds__(256) k_bin_count(BatchDev *bd)
{
    int r;
    if (!plan_block(bd->actp, bd->B, r)) return;
    RveDev *st = bd->rv[r];
    const int i = (blockIdx.x - bd->actp[r]) * 256 + threadIdx.x;
    if (i >= st->n) return;
    if (st->dim == 3) bin_count_one<3, F32, FAST>(st, i);
    else bin_count_one<2, F32, FAST>(st, i);
}

template <int DIM, bool IN32, bool OUT32>
__device__ __forceinline__ void bin_scatter_one(RveDev *st, int i)
{
    const Slot s = st->slot[st->src_idx];
    const Slot d = st->slot[st->dst_idx];
    const uint32_t lin = st->src_cell[i];
    const uint32_t j = st->cell_start[lin] + st->src_rank[i];
    const double rb = s.rb[i];
    const double R = __dmul_rn(st->lam_R, rb);
    if (IN32 && OUT32 && same_grid(st, s)) {
        float o[3];
        shift_cell_f32<DIM>(st, s, i, o);
        reinterpret_cast<float4 *>(d.pos)[j] = make_float4(o[0], o[1], o[2], (float)R);
        d.rb[j] = rb;
        d.pid[j] = s.pid[i];
        d.cell[j] = lin;
        return;
    }
    double x[3];
    src_abs<DIM, IN32>(st, s, i, x);
    if (!OUT32) {
        reinterpret_cast<double4_32a *>(d.pos)[j] = make_double4_32a(x[0], x[1], x[2], R);
    } else {
        const int32_t cx = (int32_t)(lin % (uint32_t)st->gn[0]);
        const int32_t cy = (int32_t)((lin / (uint32_t)st->gn[0]) % (uint32_t)st->gn[1]);
        const int32_t cz = (int32_t)(lin / ((uint32_t)st->gn[0] * (uint32_t)st->gn[1]));
        const int32_t cc[3] = {cx, cy, cz};
        float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < DIM; a++) o[a] = (float)__dsub_rn(x[a], __dmul_rn((double)cc[a], st->gw[a]));
        reinterpret_cast<float4 *>(d.pos)[j] = make_float4(o[0], o[1], o[2], (float)R);
    }
    d.rb[j] = rb;
    d.pid[j] = s.pid[i];
    d.cell[j] = lin;
}

template <bool IN32, bool OUT32>
__global__ void __launch_bounds__(256) k_bin_scatter(BatchDev *bd)
{
    int r;
    if (!plan_block(bd->actp, bd->B, r)) return;
    RveDev *st = bd->rv[r];
    const int i = (blockIdx.x - bd->actp[r]) * 256 + threadIdx.x;
    if (i >= st->n) return;
    if (st->dim == 3) bin_scatter_one<3, IN32, OUT32>(st, i);
    else bin_scatter_one<2, IN32, OUT32>(st, i);
}

// The destination slot records the grid its offsets refer to.
__global__ void k_bin_stamp(BatchDev *bd)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= bd->B) return;
    RveDev *st = bd->rv[r];
    if (!st->active) return;
    Slot &d = st->slot[st->dst_idx];
    for (int a = 0; a < 3; a++) {
        d.gn[a] = st->gn[a];
        d.gw[a] = st->gw[a];
    }
}

template <bool F32>
__device__ __forceinline__ void cell_sort_one(RveDev *st, int c)
{
    const uint32_t b = st->cell_start[c], e = st->cell_start[c + 1];
    if (e - b < 2) return;
    const Slot d = st->slot[st->dst_idx];
    for (uint32_t i = b + 1; i < e; i++) {
        const uint32_t key = d.pid[i];
        const double rb = d.rb[i];
        uint32_t j = i;
        if (!F32) {
            double4_32a *pos = reinterpret_cast<double4_32a *>(d.pos);
            const double4_32a v = pos[i];
            while (j > b && d.pid[j - 1] > key) {
                pos[j] = pos[j - 1];
                d.rb[j] = d.rb[j - 1];
                d.pid[j] = d.pid[j - 1];
                j--;
            }
            pos[j] = v;
        } else {
            float4 *pos = reinterpret_cast<float4 *>(d.pos);
            const float4 v = pos[i];
            while (j > b && d.pid[j - 1] > key) {
                pos[j] = pos[j - 1];
                d.rb[j] = d.rb[j - 1];
                d.pid[j] = d.pid[j - 1];
                j--;
            }
            pos[j] = v;
        }
        d.rb[j] = rb;
        d.pid[j] = key;
    }
}

// In-cell sort by particle id.  Each warp of a block takes 32 consecutive
// cells: a cell of 2..32 particles is sorted by the whole warp (lane i loads
// element i, its rank is the number of smaller ids, every element is written
// once to its rank); a larger cell is insertion-sorted by its own lane.
template <bool F32>
__global__ void __launch_bounds__(256) k_cell_sort(BatchDev *bd)
{
    using PT = typename std::conditional<F32, float4, double4_32a>::type;
    int r;
    if (!plan_block(bd->actc, bd->B, r)) return;
    RveDev *st = bd->rv[r];
    const int lane = threadIdx.x & 31;
    const int cl = (blockIdx.x - bd->actc[r]) * 256 + threadIdx.x;
    uint32_t cb = 0, ce = 0;
    if (cl < st->ncells) {
        cb = st->cell_start[cl];
        ce = st->cell_start[cl + 1];
    }
    if (ce - cb > 32) cell_sort_one<F32>(st, cl);
    const Slot d = st->slot[st->dst_idx];
    PT *pos = reinterpret_cast<PT *>(d.pos);
    unsigned todo = __ballot_sync(0xffffffffu, ce - cb >= 2 && ce - cb <= 32);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t b = __shfl_sync(0xffffffffu, cb, src);
        const uint32_t n = __shfl_sync(0xffffffffu, ce, src) - b;
        uint32_t key = 0xffffffffu;
        PT v;
        double rb = 0.0;
        if (lane < (int)n) {
            key = d.pid[b + lane];
            v = pos[b + lane];
            rb = d.rb[b + lane];
        }
        uint32_t rank = 0;
        for (uint32_t j = 0; j < n; j++) rank += __shfl_sync(0xffffffffu, key, (int)j) < key ? 1u : 0u;
        __syncwarp();
        if (lane < (int)n) {
            pos[b + rank] = v;
            d.rb[b + rank] = rb;
            d.pid[b + rank] = key;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 counts (3 passes: block sums, scan of the block
// sums, block scans with offsets).  The number of elements is read from the
// device (the grid of the current iteration); blocks past it do nothing.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_V = 4, SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
        uint32_t z = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        warp_tot[lane] = z - t;
        if (lane == 31 && total) *total = z;
    }
    __syncthreads();
    const uint32_t r = warp_tot[wid] + x - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int scan_len(const RveDev *st, int which)
{
    return which == 0 ? st->ncells : st->n;
}

__device__ __forceinline__ uint32_t *scan_in(const RveDev *st, int which)
{
    return which == 0 ? st->counts : st->pcount;
}

// which == 0: the cell counts of each RVE (only RVEs at work in this
// super-step); which == 1: the pair counts by particle of each RVE.
__global__ void __launch_bounds__(SCAN_T) k_scan_part(BatchDev *bd, int which)
{
    const int32_t *tiles = which == 0 ? bd->tile_c : bd->tile_n;
    const int r = block_rve(tiles, bd->B);
    RveDev *st = bd->rv[r];
    if (which == 0 && !st->active) return;
    const int m = scan_len(st, which);
    const int tile = blockIdx.x - tiles[r];
    const int base = tile * SCAN_TILE;
    if (base >= m) return;
    const uint32_t *in = scan_in(st, which);
    uint32_t s = 0;
#pragma unroll
    for (int v = 0; v < SCAN_V; v++) {
        const int i = base + threadIdx.x * SCAN_V + v;
        if (i < m) s += in[i];
    }
    __shared__ uint32_t tot;
    block_excl_scan(s, &tot);
    __syncthreads();
    if (threadIdx.x == 0) st->scan_part[tile] = tot;
}

// one block per RVE
__global__ void __launch_bounds__(SCAN_T) k_scan_top(BatchDev *bd, int which)
{
    RveDev *st = bd->rv[blockIdx.x];
    if (which == 0 && !st->active) return;
    const int m = scan_len(st, which);
    const int nb = (m + SCAN_TILE - 1) / SCAN_TILE;
    const int per = (nb + SCAN_T - 1) / SCAN_T;
    uint32_t s = 0;
    for (int k = 0; k < per; k++) {
        const int b = threadIdx.x * per + k;
        if (b < nb) s += st->scan_part[b];
    }
    __shared__ uint32_t tot;
    uint32_t off = block_excl_scan(s, &tot);
    for (int k = 0; k < per; k++) {
        const int b = threadIdx.x * per + k;
        if (b < nb) {
            const uint32_t v = st->scan_part[b];
            st->scan_part[b] = off;
            off += v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t *out = which == 0 ? st->cell_start : st->pcount;
        out[m] = tot;
    }
}

// which == 0: counts -> cell_start, counts cleared.  which == 1: pcount in
// place (pcount has n + 1 entries).
__global__ void __launch_bounds__(SCAN_T) k_scan_down(BatchDev *bd, int which)
{
    const int32_t *tiles = which == 0 ? bd->tile_c : bd->tile_n;
    const int r = block_rve(tiles, bd->B);
    RveDev *st = bd->rv[r];
    if (which == 0 && !st->active) return;
    const int m = scan_len(st, which);
    const int tile = blockIdx.x - tiles[r];
    const int base = tile * SCAN_TILE;
    if (base >= m) return;
    uint32_t *in = scan_in(st, which);
    uint32_t *out = which == 0 ? st->cell_start : st->pcount;
    uint32_t v[SCAN_V];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; k++) {
        const int i = base + threadIdx.x * SCAN_V + k;
        v[k] = i < m ? in[i] : 0u;
        s += v[k];
    }
    uint32_t off = block_excl_scan(s, nullptr) + st->scan_part[tile];
#pragma unroll
    for (int k = 0; k < SCAN_V; k++) {
        const int i = base + threadIdx.x * SCAN_V + k;
        if (i < m) {
            out[i] = off;
            if (which == 0) in[i] = 0u;
            off += v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_begin(const BatchShape &b, cudaStream_t s)
{
    k_begin<<<blocks_for(b.B, 128), 128, 0, s>>>(b.d);
    launch_plan(b, s);
}
void launch_control(const BatchShape &b, cudaStream_t s) { k_control<<<blocks_for(b.B, 128), 128, 0, s>>>(b.d); }

void launch_scan(const BatchShape &b, int which, cudaStream_t s)
{
    const int nt = which == 0 ? b.tiles_c : b.tiles_n;
    k_scan_part<<<nt, SCAN_T, 0, s>>>(b.d, which);
    k_scan_top<<<b.B, SCAN_T, 0, s>>>(b.d, which);
    k_scan_down<<<nt, SCAN_T, 0, s>>>(b.d, which);
}

int64_t scan_part_len(int64_t max_len) { return blocks_for(max_len, SCAN_TILE); }
int scan_tile() { return SCAN_TILE; }

// Blocks of a launch whose blocks walk a plan (k_draw): at most eight
// 256-thread blocks per SM (full residency), at most the chunks of the
// group's capacity.
int plan_blocks(int64_t capacity_chunks)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t cap = (int64_t)sms * 8;
    return (int)(capacity_chunks < cap ? (capacity_chunks > 0 ? capacity_chunks : 1) : cap);
}

void launch_plan(const BatchShape &b, cudaStream_t s) { k_plan<<<1, 1024, 0, s>>>(b.d); }

void launch_bin(const BatchShape &b, bool in32, bool out32, cudaStream_t s)
{
    const int T = 256, np = b.blocks_p, nc = b.blocks_c;
    // the binary32 shift path only where the scatter also writes binary32
    if (in32 && out32) k_bin_count<true, true><<<np, T, 0, s>>>(b.d);
    else if (in32) k_bin_count<true, false><<<np, T, 0, s>>>(b.d);
    else k_bin_count<false, false><<<np, T, 0, s>>>(b.d);
    launch_scan(b, 0, s);
    if (in32 && out32) k_bin_scatter<true, true><<<np, T, 0, s>>>(b.d);
    else if (in32) k_bin_scatter<true, false><<<np, T, 0, s>>>(b.d);
    else k_bin_scatter<false, false><<<np, T, 0, s>>>(b.d);
    k_bin_stamp<<<blocks_for(b.B, 128), 128, 0, s>>>(b.d);
    if (out32) k_cell_sort<true><<<nc, T, 0, s>>>(b.d);
    else k_cell_sort<false><<<nc, T, 0, s>>>(b.d);
}

// ---------------------------------------------------------------------------
// Import of a starting configuration (absolute binary64 positions in id
// order) into slot P, binned on the grid of the starting scale.
// ---------------------------------------------------------------------------
__global__ void k_import_begin(RveDev *st)
{
    if (threadIdx.x || blockIdx.x) return;
    set_grid(st, st->lam_P);
    Slot &p = st->slot[st->p_idx];
    for (int a = 0; a < 3; a++) {
        p.gn[a] = st->gn[a];
        p.gw[a] = st->gw[a];
    }
}

template <int DIM, bool F32>
__global__ void k_import(RveDev *st, const double *xyz, const double *rb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st->n) return;
    const Slot p = st->slot[st->p_idx];
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < DIM; a++) x[a] = xyz[(size_t)i * DIM + a];
    uint32_t lin = 0, mul = 1;
    int32_t cc[3] = {0, 0, 0};
    for (int a = 0; a < DIM; a++) {
        cc[a] = cell_coord_d(x[a], p.gw[a], p.gn[a]);
        lin += (uint32_t)cc[a] * mul;
        mul *= (uint32_t)p.gn[a];
    }
    const double R = __dmul_rn(st->lam_P, rb[i]);
    if (!F32) {
        reinterpret_cast<double4_32a *>(p.pos)[i] = make_double4_32a(x[0], x[1], x[2], R);
    } else {
        float o[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < DIM; a++) o[a] = (float)__dsub_rn(x[a], __dmul_rn((double)cc[a], p.gw[a]));
        reinterpret_cast<float4 *>(p.pos)[i] = make_float4(o[0], o[1], o[2], (float)R);
    }
    p.rb[i] = rb[i];
    p.pid[i] = (uint32_t)i;
    p.cell[i] = lin;
}

void launch_import(RveDev *d_st, int dim, bool f32, int64_t n, const double *xyz, const double *rb,
                   cudaStream_t s)
{
    k_import_begin<<<1, 1, 0, s>>>(d_st);
    const int nb = blocks_for(n, 256);
    if (dim == 2) {
        if (f32) k_import<2, true><<<nb, 256, 0, s>>>(d_st, xyz, rb);
        else k_import<2, false><<<nb, 256, 0, s>>>(d_st, xyz, rb);
    } else {
        if (f32) k_import<3, true><<<nb, 256, 0, s>>>(d_st, xyz, rb);
        else k_import<3, false><<<nb, 256, 0, s>>>(d_st, xyz, rb);
    }
}

}  // namespace srm
