// Evaluation without any allocation: rbf_eval_noalloc.
//
// Some callers cannot allocate device memory at the point where they need the surface:
// code running inside a region where cudaMalloc is not allowed or would stall (e.g. while
// a caller's own allocator or memory pool is locked, or under a strict memory budget that
// must not grow), or plain C/Fortran hosts that own all device buffers themselves and do
// not want a library context. This entry point evaluates
// f(q) = sum_j c_j phi(||q - xi_j|| / R) for caller-owned inputs and output, binning the
// centres into a scratch area that is a file-scope static device array of fixed size,
// reserved once when the library is loaded (every GPU that loads the library holds it
// until the process exits).
//
// Limits: M <= kNaMaxCentres centres and a cell grid of at most kNaMaxCells cells of side R
// over bbox; larger inputs are rejected with RBF_ERR_LIMIT before any work is queued.
// The scratch is shared by every call on a device: two calls whose work overlaps on the
// GPU (different streams, or different host threads on the same device) race on it.
// Calls on one stream are ordered and safe. The cell counters are cleared by each call.
//
// The host needs the scratch's device address, which belongs to the CUDA context that is
// current. It is looked up with cudaGetSymbolAddress the first time a context is seen and
// cached under that context's unique id (cuCtxGetId, never reused within a process), so a
// context created after a device reset gets its own lookup instead of a stale address.
//
// Within a cell the centres are in the order their atomic counters handed out, which can
// change from call to call: the sums of one query are then added in a different order and
// two identical calls can differ in the last bits (the value agrees with rbf_eval to
// rounding, not bit for bit).
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "rbf_internal.h"

namespace rbf {
namespace {

constexpr int kNaMaxCentres = 65536;
constexpr int kNaMaxCells = 65536;
constexpr int kNaThreads = 1024;

// scratch layout (bytes): counts int[kNaMaxCells] | cstart int[kNaMaxCells + 4] |
// key int[kNaMaxCentres] | rank int[kNaMaxCentres] | sx, sy, sc double[kNaMaxCentres] each
constexpr size_t kNaCounts = 0;
constexpr size_t kNaStart = kNaCounts + sizeof(int) * kNaMaxCells;
constexpr size_t kNaKey = kNaStart + sizeof(int) * (kNaMaxCells + 4);
constexpr size_t kNaRank = kNaKey + sizeof(int) * kNaMaxCentres;
constexpr size_t kNaSx = kNaRank + sizeof(int) * kNaMaxCentres;
constexpr size_t kNaSy = kNaSx + sizeof(double) * kNaMaxCentres;
constexpr size_t kNaSc = kNaSy + sizeof(double) * kNaMaxCentres;
constexpr size_t kNaBytes = kNaSc + sizeof(double) * kNaMaxCentres;   // 2.6 MB

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct NaView {
    int* counts;
    int* cstart;
    int* key;
    int* rank;
    double* sx;
    double* sy;
    double* sc;
};

__host__ __device__ inline NaView na_view(unsigned char* base) {
    NaView v;
    v.counts = reinterpret_cast<int*>(base + kNaCounts);
    v.cstart = reinterpret_cast<int*>(base + kNaStart);
    v.key = reinterpret_cast<int*>(base + kNaKey);
    v.rank = reinterpret_cast<int*>(base + kNaRank);
    v.sx = reinterpret_cast<double*>(base + kNaSx);
    v.sy = reinterpret_cast<double*>(base + kNaSy);
    v.sc = reinterpret_cast<double*>(base + kNaSc);
    return v;
}

__global__ void k_na_zero(unsigned char* base, int ncell) {
    const NaView v = na_view(base);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x)
        v.counts[i] = 0;
}

__global__ void k_na_count(unsigned char* base, Grid g, const double* __restrict__ cx,
                           const double* __restrict__ cy, int M) {
    const NaView v = na_view(base);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const int k = cell_iy(g, cy[i]) * g.gx + cell_ix(g, cx[i]);
        v.key[i] = k;
        v.rank[i] = atomicAdd(&v.counts[k], 1);
    }
}

// Exclusive scan of the cell counts into cstart[0..ncell] (one block).
__global__ void __launch_bounds__(kNaThreads) k_na_scan(unsigned char* base, int ncell) {
    const NaView v = na_view(base);
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t0 = 0; t0 < ncell; t0 += kNaThreads) {
        const int i = t0 + threadIdx.x;
        const int val = i < ncell ? v.counts[i] : 0;
        int x = val;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_tot[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - val;
        if (i < ncell) v.cstart[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) v.cstart[ncell] = carry;
}

__global__ void k_na_scatter(unsigned char* base, const double* __restrict__ cx,
                             const double* __restrict__ cy, const double* __restrict__ c, int M) {
    const NaView v = na_view(base);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const int d = v.cstart[v.key[i]] + v.rank[i];
        v.sx[d] = cx[i];
        v.sy[d] = cy[i];
        v.sc[d] = c[i];
    }
}

template <int KIND>
__global__ void k_na_eval(unsigned char* base, Grid g, const double* __restrict__ qx,
                          const double* __restrict__ qy, int64_t Q, double* __restrict__ f) {
    const NaView v = na_view(base);
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < Q;
         q += int64_t(gridDim.x) * blockDim.x) {
        const double x = qx[q], y = qy[q];
        const int ix = cell_ix(g, x), iy = cell_iy(g, y);
        const int xa = max(ix - 1, 0), xb = min(ix + 1, g.gx - 1);
        double acc = 0.0;
        for (int row = max(iy - 1, 0); row <= min(iy + 1, g.gy - 1); ++row) {
            const int s0 = v.cstart[row * g.gx + xa], s1 = v.cstart[row * g.gx + xb + 1];
            for (int s = s0; s < s1; ++s) {
                const double dx = x - v.sx[s], dy = y - v.sy[s];
                if (inside_exact(dx, dy, g.R, g.R2)) {
                    const double r = sqrt_nr(fma(dx, dx, dy * dy)) * g.invR;
                    acc = fma(v.sc[s], wendland<KIND, double>(r), acc);
                }
            }
        }
        f[q] = acc;
    }
}

// Device address of g_na_scratch per CUDA context. The driver's context functions are
// reached through the runtime's entry-point query, so the library does not link libcuda.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
constexpr int kNaCache = 64;
struct NaEntry {
    unsigned long long ctx_id;
    void* ptr;
};
std::mutex g_na_mutex;
NaEntry g_na_cache[kNaCache] = {};
int g_na_used = 0, g_na_next = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

rbf_status na_driver_fns() {
    if (g_get_current && g_get_id) return RBF_OK;
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
            cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b) {
        cudaGetLastError();
        return RBF_ERR_CUDA;
    }
    g_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_get_id = reinterpret_cast<CtxGetIdFn>(b);
    return RBF_OK;
}

// The scratch address in the context current on device `dev` (made current first if the
// runtime has not yet set one up on this thread).
rbf_status na_scratch(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    rbf_status s = na_driver_fns();
    if (s != RBF_OK) return s;
    CUcontext cu = nullptr;
    if (g_get_current(&cu) != CUDA_SUCCESS) return RBF_ERR_CUDA;
    if (!cu) {
        // no context on this thread yet: make the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess || g_get_current(&cu) != CUDA_SUCCESS || !cu) {
            cudaGetLastError();
            return RBF_ERR_CUDA;
        }
    }
    unsigned long long id = 0;
    if (g_get_id(cu, &id) != CUDA_SUCCESS) return RBF_ERR_CUDA;
    for (int k = 0; k < g_na_used; ++k)
        if (g_na_cache[k].ctx_id == id) {
            *out = static_cast<unsigned char*>(g_na_cache[k].ptr);
            return RBF_OK;
        }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return RBF_ERR_CUDA;
    }
    const int slot = g_na_used < kNaCache ? g_na_used++ : (g_na_next++ % kNaCache);
    g_na_cache[slot] = NaEntry{id, p};
    *out = static_cast<unsigned char*>(p);
    return RBF_OK;
}

}  // namespace
}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_eval_noalloc(const double* cx, const double* cy, const double* c,
                                       int64_t M, double R, const double* bbox, rbf_kernel kernel,
                                       const double* qx, const double* qy, int64_t Q, double* f,
                                       void* stream) {
    if (M < 1 || Q < 0 || !cx || !cy || !c || !bbox || (Q > 0 && (!qx || !qy || !f)))
        return RBF_ERR_ARG;
    if (!(R > 0.0) || !isfinite(R) || kernel < RBF_W30 || kernel > RBF_W33) return RBF_ERR_ARG;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(bbox[k])) return RBF_ERR_ARG;
    if (!(bbox[2] >= bbox[0]) || !(bbox[3] >= bbox[1])) return RBF_ERR_ARG;
    if (M > kNaMaxCentres) return RBF_ERR_LIMIT;
    Grid g;
    g.x0 = bbox[0];
    g.y0 = bbox[1];
    g.R = R;
    g.invR = 1.0 / R;
    g.R2 = R * R;
    g.h = R * kCellMargin;
    g.invh = 1.0 / g.h;
    const double nxf = std::max(1.0, ceil((bbox[2] - bbox[0]) * g.invh));
    const double nyf = std::max(1.0, ceil((bbox[3] - bbox[1]) * g.invh));
    if (nxf * nyf > double(kNaMaxCells)) return RBF_ERR_LIMIT;
    g.gx = int(nxf);
    g.gy = int(nyf);
    g.ncell = g.gx * g.gy;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RBF_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    rbf_status s = na_scratch(dev, &base);
    if (s != RBF_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int m = int(M);
    const int gm = std::min(div_up(m, 256), 1024);
    k_na_zero<<<std::min(div_up(g.ncell, 256), 256), 256, 0, st>>>(base, g.ncell);
    k_na_count<<<gm, 256, 0, st>>>(base, g, cx, cy, m);
    k_na_scan<<<1, kNaThreads, 0, st>>>(base, g.ncell);
    k_na_scatter<<<gm, 256, 0, st>>>(base, cx, cy, c, m);
    if (Q > 0) {
        const int gq = int(std::min<int64_t>((Q + 255) / 256, 152 * 32));
        switch (kernel) {
            case RBF_W30: k_na_eval<0><<<gq, 256, 0, st>>>(base, g, qx, qy, Q, f); break;
            case RBF_W31: k_na_eval<1><<<gq, 256, 0, st>>>(base, g, qx, qy, Q, f); break;
            case RBF_W32: k_na_eval<2><<<gq, 256, 0, st>>>(base, g, qx, qy, Q, f); break;
            default: k_na_eval<3><<<gq, 256, 0, st>>>(base, g, qx, qy, Q, f); break;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return RBF_ERR_CUDA;
    return RBF_OK;
}
