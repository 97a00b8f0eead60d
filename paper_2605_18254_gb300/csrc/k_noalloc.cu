// k_noalloc.cu -- srm_certify_noalloc: the FP64 overlap certification of a
// configuration held in caller-owned device buffers, for callers that cannot
// allocate device memory.  Its working memory (cell counts, cell starts, the
// cell-sorted copy of the particles and the two result words) lives in one
// file-scope static device array of fixed size, so the call allocates
// nothing; see include/srm.h for the limits and the rules of use.
#include <cstring>
#include <mutex>
#include <string>

#include "srm.h"
#include "srm_dev.cuh"

namespace {

constexpr int NA_MAXN = SRM_NOALLOC_MAX_PARTICLES;
constexpr int NA_MAXC = SRM_NOALLOC_MAX_CELLS;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// layout of the scratch array (byte offsets, each 256-byte aligned)
struct NaLayout {
    static constexpr size_t hdr = 0;  // NaHeader
    static constexpr size_t counts = align256(hdr + 256);
    static constexpr size_t start = align256(counts + sizeof(uint32_t) * NA_MAXC);
    static constexpr size_t cellof = align256(start + sizeof(uint32_t) * (NA_MAXC + 1));
    static constexpr size_t rank = align256(cellof + sizeof(uint32_t) * NA_MAXN);
    static constexpr size_t order = align256(rank + sizeof(uint32_t) * NA_MAXN);
    static constexpr size_t sorted = align256(order + sizeof(uint32_t) * NA_MAXN);
    static constexpr size_t total = align256(sorted + sizeof(double4_32a) * NA_MAXN);
};

struct NaHeader {
    unsigned long long pairs;    // colliding pairs i < j
    unsigned long long gap_key;  // order-preserving key of the smallest gap
    int32_t n[3];
    int32_t ncells;
    int32_t error;               // 1: box narrower than 4 R_max on some axis;
                                 // 2: a radius that is negative, infinite or NaN
    int32_t pad;
    double w[3];
};

// The working memory of every call on this device: 1,966,592 bytes (1.97 MB,
// 1.88 MiB), the figure include/srm.h states.
static_assert(NaLayout::total == 1966592, "scratch size changed: update the figure in include/srm.h");
static __device__ __align__(256) unsigned char g_na_scratch[NaLayout::total];

struct NaView {
    NaHeader *h;
    uint32_t *counts, *start, *cellof, *rank, *order;
    double4_32a *sorted;
};

__host__ __device__ inline NaView na_view(unsigned char *base)
{
    NaView v;
    v.h = reinterpret_cast<NaHeader *>(base + NaLayout::hdr);
    v.counts = reinterpret_cast<uint32_t *>(base + NaLayout::counts);
    v.start = reinterpret_cast<uint32_t *>(base + NaLayout::start);
    v.cellof = reinterpret_cast<uint32_t *>(base + NaLayout::cellof);
    v.rank = reinterpret_cast<uint32_t *>(base + NaLayout::rank);
    v.order = reinterpret_cast<uint32_t *>(base + NaLayout::order);
    v.sorted = reinterpret_cast<double4_32a *>(base + NaLayout::sorted);
    return v;
}

// One block: largest radius, grid with cells at least 2 R_max wide (3 per
// axis at least, NA_MAXC in total at most), cleared counts and results.
__global__ void __launch_bounds__(1024) k_na_setup(unsigned char *base, int dim, double L0, double L1,
                                                   double L2, int n, const double *R)
{
    NaView v = na_view(base);
    __shared__ double smax[32];
    __shared__ int bad_sh;
    if (threadIdx.x == 0) bad_sh = 0;
    __syncthreads();
    double m = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = R[i];
        // fmax would skip a NaN and leave R_max too small for the grid
        if (!(r >= 0.0) || isinf(r)) bad = 1;
        else m = fmax(m, r);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) bad_sh = 1;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    __shared__ int nc_sh;
    if (threadIdx.x == 0) {
        double rmax = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) rmax = fmax(rmax, smax[k]);
        const double L[3] = {L0, L1, L2};
        const int kcap = dim == 3 ? 40 : 256;  // kcap^dim <= NA_MAXC
        int nc = 1, err = 0;
        for (int a = 0; a < 3; a++) {
            if (a >= dim) {
                v.h->n[a] = 1;
                v.h->w[a] = L[a];
                continue;
            }
            if (L[a] < 4.0 * rmax) err = 1;
            long long k = rmax > 0.0 ? (long long)(L[a] / (2.0 * rmax * 1.000001)) : kcap;
            if (k > kcap) k = kcap;
            if (k < 3) k = 3;
            v.h->n[a] = (int)k;
            v.h->w[a] = L[a] / (double)k;
            nc *= (int)k;
        }
        v.h->ncells = nc;
        v.h->error = bad_sh ? 2 : err;
        v.h->pairs = 0ull;
        v.h->gap_key = srm::dkey(__longlong_as_double(0x7ff0000000000000LL));
        nc_sh = nc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc_sh; c += blockDim.x) v.counts[c] = 0u;
}

__global__ void k_na_count(unsigned char *base, int dim, int n, const double *xyz)
{
    NaView v = na_view(base);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t lin = 0, mul = 1;
    for (int a = 0; a < dim; a++) {
        lin += (uint32_t)srm::cell_coord_d(xyz[(size_t)i * dim + a], v.h->w[a], v.h->n[a]) * mul;
        mul *= (uint32_t)v.h->n[a];
    }
    v.cellof[i] = lin;
    v.rank[i] = atomicAdd(&v.counts[lin], 1u);
}

// Exclusive scan of up to NA_MAXC counts in one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_na_scan(unsigned char *base)
{
    NaView v = na_view(base);
    const int nc = v.h->ncells;
    constexpr int PER = NA_MAXC / 1024;
    const int b0 = threadIdx.x * PER;
    uint32_t loc[PER];
    uint32_t s = 0;
    for (int k = 0; k < PER; k++) {
        loc[k] = b0 + k < nc ? v.counts[b0 + k] : 0u;
        s += loc[k];
    }
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const uint32_t t = wsum[lane];
        uint32_t z = t;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z - t;
    }
    __syncthreads();
    uint32_t off = wsum[wid] + x - s;
    for (int k = 0; k < PER; k++) {
        if (b0 + k < nc) v.start[b0 + k] = off;
        off += loc[k];
    }
    if (threadIdx.x == 1023) v.start[nc] = off;
}

__global__ void k_na_scatter(unsigned char *base, int dim, int n, const double *xyz, const double *R)
{
    NaView v = na_view(base);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = v.start[v.cellof[i]] + v.rank[i];
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; a++) x[a] = xyz[(size_t)i * dim + a];
    v.sorted[j] = make_double4_32a(x[0], x[1], x[2], R[i]);
    v.order[j] = (uint32_t)i;
}

// Pairs i < j (by index) with sqrt(|d|^2) <= R_i + R_j under the minimum
// image, and the smallest gap, over the cells within one of each particle's.
template <int DIM>
__global__ void k_na_pairs(unsigned char *base, int n, double L0, double L1, double L2)
{
    NaView v = na_view(base);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double L[3] = {L0, L1, L2};
    const double halfL[3] = {0.5 * L0, 0.5 * L1, 0.5 * L2};
    int cnt = 0;
    double mg = __longlong_as_double(0x7ff0000000000000LL);
    if (s < n) {
        const double4_32a p = v.sorted[s];
        const uint32_t me = v.order[s];
        const double q[3] = {p.x, p.y, p.z};
        int c[3] = {0, 0, 0};
        for (int a = 0; a < DIM; a++) c[a] = srm::cell_coord_d(q[a], v.h->w[a], v.h->n[a]);
        const int n0 = v.h->n[0], n1 = v.h->n[1], n2 = v.h->n[2];
        const int zr = DIM == 3 ? 1 : 0;
        for (int dz = -zr; dz <= zr; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int cx = (c[0] + dx + n0) % n0, cy = (c[1] + dy + n1) % n1, cz = (c[2] + dz + n2) % n2;
                    const int cell = cx + n0 * (cy + n1 * cz);
                    for (uint32_t k = v.start[cell]; k < v.start[cell + 1]; k++) {
                        if (v.order[k] <= me) continue;
                        const double4_32a t = v.sorted[k];
                        const double tt[3] = {t.x, t.y, t.z};
                        double gap;
                        if (srm::gap_exact<DIM>(q, p.w, tt, t.w, L, halfL, &gap)) cnt++;
                        if (gap < mg) mg = gap;
                    }
                }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    unsigned long long key = srm::dkey(mg);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
        key = y < key ? y : key;
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(&v.h->pairs, (unsigned long long)cnt);
        atomicMin(&v.h->gap_key, key);
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mu;
void *g_na_ptr[64];

}  // namespace

namespace srm {
// the thread-local message returned by srm_last_error (runtime.cu)
void set_last_error(const std::string &msg);
}  // namespace srm

extern "C" srm_status srm_certify_noalloc(int32_t dim, const double box[3], int64_t n, const double *xyz,
                                          const double *radii, int64_t *overlap_pairs, double *min_gap,
                                          void *cuda_stream)
{
    auto fail = [](srm_status s, const std::string &m) {
        srm::set_last_error(m);
        return s;
    };
    if (dim != 2 && dim != 3) return fail(SRM_E_ARG, "dim must be 2 or 3");
    if (!box || !xyz || !radii || !overlap_pairs || !min_gap) return fail(SRM_E_ARG, "null argument");
    if (n < 1) return fail(SRM_E_ARG, "n must be >= 1");
    if (n > NA_MAXN) return fail(SRM_E_ARG, "n exceeds SRM_NOALLOC_MAX_PARTICLES");
    for (int a = 0; a < dim; a++)
        if (!(box[a] > 0.0)) return fail(SRM_E_ARG, "box lengths must be > 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(SRM_E_CUDA, "no current device");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p) return fail(SRM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_na_ptr[dev]);
    }
    // An error left by earlier work on this thread is reported as such and
    // left pending for its owner (cudaPeekAtLastError does not clear it);
    // the checks after each launch below then see this call's own errors.
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return fail(SRM_E_CUDA, std::string("a CUDA error from earlier work on this thread is pending: ") +
                                    cudaGetErrorString(pending));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double L[3] = {box[0], box[1], dim == 3 ? box[2] : 1.0};
    const int nn = (int)n, nb = (nn + 255) / 256;
    cudaError_t e = cudaSuccess;
    auto launched = [&e](const char *name) {
        if (e != cudaSuccess) return;
        const cudaError_t x = cudaGetLastError();
        if (x != cudaSuccess) {
            e = x;
            srm::set_last_error(std::string("launch of ") + name + ": " + cudaGetErrorString(x));
        }
    };
    k_na_setup<<<1, 1024, 0, s>>>(base, dim, L[0], L[1], L[2], nn, radii);
    launched("k_na_setup");
    if (e == cudaSuccess) {
        k_na_count<<<nb, 256, 0, s>>>(base, dim, nn, xyz);
        launched("k_na_count");
    }
    if (e == cudaSuccess) {
        k_na_scan<<<1, 1024, 0, s>>>(base);
        launched("k_na_scan");
    }
    if (e == cudaSuccess) {
        k_na_scatter<<<nb, 256, 0, s>>>(base, dim, nn, xyz, radii);
        launched("k_na_scatter");
    }
    if (e == cudaSuccess) {
        if (dim == 2) k_na_pairs<2><<<nb, 256, 0, s>>>(base, nn, L[0], L[1], L[2]);
        else k_na_pairs<3><<<nb, 256, 0, s>>>(base, nn, L[0], L[1], L[2]);
        launched("k_na_pairs");
    }
    if (e != cudaSuccess) return SRM_E_CUDA;  // message set by `launched`
    NaHeader hdr;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdr, base + NaLayout::hdr, sizeof(hdr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SRM_E_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    if (hdr.error == 2) return fail(SRM_E_ARG, "radii must be finite and non-negative");
    if (hdr.error) return fail(SRM_E_ARG, "box narrower than 4 R_max on some axis");
    const unsigned long long key = hdr.gap_key;
    const unsigned long long b = (key >> 63) ? (key & 0x7fffffffffffffffULL) : ~key;
    std::memcpy(min_gap, &b, sizeof(double));
    *overlap_pairs = (int64_t)hdr.pairs;
    return SRM_OK;
}
