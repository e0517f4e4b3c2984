// Step (e): evaluate the approximant f(x) = sum_j c_j phi(||x - xi_j|| / R) (Eq. 3) at
// query points or on a node-centred grid, a warp per 32 queries. Only the centres of the 3x3
// cells around the query's cell can contribute (compact support, Eq. 18); they are three
// contiguous ranges of the cell-sorted centre order. Also: export of the assembled B for
// diagnostics.
#include <algorithm>

#include "rbf_internal.h"
#include "rbf_evalpairs.cuh"

namespace rbf {
namespace {

__global__ void k_diag_sqrt(const double* __restrict__ a, double* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        out[3 * i] = sqrt_nr(a[i]);
        out[3 * i + 1] = sqrt_fast(a[i]);
        out[3 * i + 2] = sqrt(a[i]);
    }
}

// The linear polynomial of Section 3 (Eq. 6-7), coefficients (a_x, a_y, a_0) in the caller's
// coordinates; 0 without one.
__device__ __forceinline__ double poly_at(const double* __restrict__ k, double x, double y) {
    return k ? fma(k[0], x, fma(k[1], y, k[2])) : 0.0;
}

constexpr int kEvalWarps = 8;

// f at 32 queries (lane l owning query l) in the single system's frame.
template <int KIND>
__device__ __forceinline__ double eval_warp32(const Binned& bd, const double* __restrict__ c,
                                              double x, double y, bool valid, int lane,
                                              EvalWarpSmem& sm) {
    const Grid& g = bd.g;
    EvalQuery q;
    q.valid = valid;
    q.x = valid ? x : 0.0;
    q.y = valid ? y : 0.0;
    q.ix = q.iy = 0;
    q.uq = q.vq = 0.0f;
    if (valid) {
        q.ix = cell_ix(g, x);
        q.iy = cell_iy(g, y);
        q.uq = float((x - (g.x0 + q.ix * g.h)) * g.invR);
        q.vq = float((y - (g.y0 + q.iy * g.h)) * g.invR);
    }
    const EvalFrame fr{g.R, g.R2, g.invR, 0, g.gx - 1, 0, g.gy - 1};
    return eval_pairs32<KIND>(bd, c, q, fr, lane, sm);
}

// Persistent warps over groups of 32 query points.
template <int KIND>
__global__ void __launch_bounds__(kEvalWarps * 32)
    k_eval_points(Binned bd, const double* __restrict__ c, const double* __restrict__ qx,
                  const double* __restrict__ qy, int64_t Q, double* __restrict__ f,
                  const double* __restrict__ k) {
    __shared__ EvalWarpSmem sm[kEvalWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t groups = (Q + 31) / 32;
    for (int64_t gi = blockIdx.x * int64_t(kEvalWarps) + w; gi < groups;
         gi += int64_t(gridDim.x) * kEvalWarps) {
        const int64_t i = gi * 32 + lane;
        const bool valid = i < Q;
        const double x = valid ? qx[i] : 0.0, y = valid ? qy[i] : 0.0;
        const double v = eval_warp32<KIND>(bd, c, x, y, valid, lane, sm[w]);
        if (valid) f[i] = v + poly_at(k, x, y);
    }
}

// Grid node coordinates follow an inclusive linspace: start + j * step (separately
// rounded), the last node exactly at the end of the box. Persistent warps over segments of
// 32 consecutive nodes of a row (consecutive warps on neighbouring segments, so that their
// candidates stay in L1).
template <int KIND>
__global__ void __launch_bounds__(kEvalWarps * 32)
    k_eval_grid(Binned bd, const double* __restrict__ c, int nx, int ny, double x0, double y0,
                double x1, double y1, double sx, double sy, double* __restrict__ f,
                const double* __restrict__ k) {
    __shared__ EvalWarpSmem sm[kEvalWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int segs = (nx + 31) / 32;
    const int64_t groups = int64_t(segs) * ny;
    for (int64_t gi = blockIdx.x * int64_t(kEvalWarps) + w; gi < groups;
         gi += int64_t(gridDim.x) * kEvalWarps) {
        const int i = int(gi / segs), j = int(gi % segs) * 32 + lane;
        const bool valid = j < nx;
        const double x = (j == nx - 1 && nx > 1) ? x1 : __dadd_rn(__dmul_rn(double(j), sx), x0);
        const double y = (i == ny - 1 && ny > 1) ? y1 : __dadd_rn(__dmul_rn(double(i), sy), y0);
        const double v = eval_warp32<KIND>(bd, c, x, y, valid, lane, sm[w]);
        if (valid) f[int64_t(i) * nx + j] = v + poly_at(k, x, y);
    }
}

// One thread per stored row s: its nonzero values B[s][t], t >= s, as COO triplets in the
// caller's centre order (the halved diagonal doubled), and b and the support counts.
template <typename T>
__global__ void k_export(Binned bd, const T* __restrict__ B, const double* __restrict__ bvec,
                         const int* __restrict__ support, int64_t cap, int32_t* __restrict__ row,
                         int32_t* __restrict__ col, double* __restrict__ val,
                         double* __restrict__ bout, int32_t* __restrict__ sout,
                         unsigned long long* __restrict__ counter) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bd.M) return;
    const RowMeta rm = bd.rmeta[s];
    const int lo[3] = {s & ~3, rm.lo1, rm.lo2};
    long long o = 4LL * rm.off;
    for (int k = 0; k < 3; ++k) {
        const int len = 4 * seg_quads(rm.len, k);
        for (int j = 0; j < len; ++j) {
            const int t = lo[k] + j;
            double v = double(B[o + j]);
            if (t < s || v == 0.0) continue;   // widening slots of the row hold zeros
            if (t == s) v *= 2.0;
            const unsigned long long pos = atomicAdd(counter, 1ull);
            if (pos < (unsigned long long)cap) {
                row[pos] = bd.cperm[s];
                col[pos] = bd.cperm[t];
                val[pos] = v;
            }
        }
        o += len;
    }
    if (bout) bout[bd.cperm[s]] = bvec[s];
    if (sout) sout[bd.cperm[s]] = support[s];
}

// Number of stored values that are not exactly zero (one warp-level ballot per 32 values).
template <typename T>
__global__ void k_count_nonzero(const T* __restrict__ B, int64_t n,
                                unsigned long long* __restrict__ counter) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        c += B[i] != T(0) ? 1ull : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counter, c);
}

int eval_grid_size(int64_t Q) { return int(std::min<int64_t>((Q + 255) / 256, 152 * 32)); }
// warps of kEvalWarps per block, one query each, persistent over the queries
// Blocks for Q queries: a warp per 32 of them, persistent beyond 8 blocks per SM.
int eval_warp_grid(int64_t Q) {
    const int64_t groups = (Q + 31) / 32;
    return int(std::max<int64_t>(1, std::min<int64_t>((groups + kEvalWarps - 1) / kEvalWarps, 152 * 8)));
}

}  // namespace

rbf_status diag_sqrt_run(const double* a, double* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return RBF_OK;
    k_diag_sqrt<<<eval_grid_size(n), 256, 0, st>>>(a, out, n);
    return cudaGetLastError() == cudaSuccess ? RBF_OK : RBF_ERR_CUDA;
}

rbf_status eval_points_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                           int64_t Q, double* f, cudaStream_t st) {
    return eval_points_poly_run(ctx, c, nullptr, qx, qy, Q, f, st);
}

rbf_status eval_points_poly_run(rbf_ctx* ctx, const double* c, const double* k, const double* qx,
                                const double* qy, int64_t Q, double* f, cudaStream_t st) {
    rbf_status s = ensure(ctx, ctx->csort, sizeof(double) * ctx->M, st);
    if (s != RBF_OK) return s;
    const Binned bd = view(ctx);
    launch_gather_sorted(c, bd.cperm, ctx->csort.as<double>(), ctx->M, st);
    ctx->launches += 1;
    if (Q <= 0) return RBF_OK;
    const double* cs = ctx->csort.as<double>();
    const int gb = eval_warp_grid(Q);
    constexpr int T = kEvalWarps * 32;
    switch (ctx->kernel) {
        case RBF_W30: k_eval_points<0><<<gb, T, 0, st>>>(bd, cs, qx, qy, Q, f, k); break;
        case RBF_W31: k_eval_points<1><<<gb, T, 0, st>>>(bd, cs, qx, qy, Q, f, k); break;
        case RBF_W32: k_eval_points<2><<<gb, T, 0, st>>>(bd, cs, qx, qy, Q, f, k); break;
        default: k_eval_points<3><<<gb, T, 0, st>>>(bd, cs, qx, qy, Q, f, k); break;
    }
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    return RBF_OK;
}

rbf_status eval_grid_run(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                         double* f, cudaStream_t st, const double* k) {
    rbf_status s = ensure(ctx, ctx->csort, sizeof(double) * ctx->M, st);
    if (s != RBF_OK) return s;
    const Binned bd = view(ctx);
    launch_gather_sorted(c, bd.cperm, ctx->csort.as<double>(), ctx->M, st);
    const double* cs = ctx->csort.as<double>();
    const double x0 = box[0], y0 = box[1], x1 = box[2], y1 = box[3];
    const double sx = nx > 1 ? (x1 - x0) / double(nx - 1) : 0.0;
    const double sy = ny > 1 ? (y1 - y0) / double(ny - 1) : 0.0;
    const int gb = eval_warp_grid(int64_t(nx) * ny);
    constexpr int T = kEvalWarps * 32;
    switch (ctx->kernel) {
        case RBF_W30: k_eval_grid<0><<<gb, T, 0, st>>>(bd, cs, nx, ny, x0, y0, x1, y1, sx, sy, f, k); break;
        case RBF_W31: k_eval_grid<1><<<gb, T, 0, st>>>(bd, cs, nx, ny, x0, y0, x1, y1, sx, sy, f, k); break;
        case RBF_W32: k_eval_grid<2><<<gb, T, 0, st>>>(bd, cs, nx, ny, x0, y0, x1, y1, sx, sy, f, k); break;
        default: k_eval_grid<3><<<gb, T, 0, st>>>(bd, cs, nx, ny, x0, y0, x1, y1, sx, sy, f, k); break;
    }
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 2;
    return RBF_OK;
}

rbf_status export_upper_run(rbf_ctx* ctx, int64_t cap, int32_t* row, int32_t* col, double* val,
                            double* bvec, int32_t* support, int64_t* nnz, cudaStream_t st) {
    const Binned bd = view(ctx);
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(ctx->stats.as<char>() + 32);
    RBF_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    const int nb = div_up(ctx->M, 128);
    if (ctx->prec == RBF_FP64)
        k_export<double><<<nb, 128, 0, st>>>(bd, bvals_dev<double>(ctx), ctx->bvec.as<double>(),
                                             ctx->support.as<int>(), cap, row, col, val, bvec,
                                             support, counter);
    else
        k_export<float><<<nb, 128, 0, st>>>(bd, bvals_dev<float>(ctx), ctx->bvec.as<double>(),
                                            ctx->support.as<int>(), cap, row, col, val, bvec,
                                            support, counter);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    unsigned long long* h = static_cast<unsigned long long*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(h, counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    *nnz = int64_t(*h);
    if (*nnz > cap) return set_err(ctx, RBF_ERR_ARG, "export capacity too small");
    return RBF_OK;
}

rbf_status layout_stats_run(rbf_ctx* ctx, rbf_layout_stats* out, cudaStream_t st) {
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(ctx->stats.as<char>() + 40);
    RBF_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    const int nb = int(std::min<int64_t>((ctx->nvals + 255) / 256, 152 * 16));
    if (ctx->nvals > 0) {
        if (ctx->prec == RBF_FP64)
            k_count_nonzero<double><<<nb, 256, 0, st>>>(bvals_dev<double>(ctx), ctx->nvals, counter);
        else
            k_count_nonzero<float><<<nb, 256, 0, st>>>(bvals_dev<float>(ctx), ctx->nvals, counter);
        RBF_CUDA_TRY(cudaGetLastError());
        ctx->launches += 1;
    }
    unsigned long long* h = static_cast<unsigned long long*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(h, counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(h + 1, ctx->stats.as<int>() + 12, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    out->stored_values = ctx->nvals;
    out->nonzeros = int64_t(h[0]);
    out->row_groups = ctx->ngroup;
    out->dropped = *reinterpret_cast<const int*>(h + 1);
    out->host_blocks = ctx->b_in_host ? ctx->bblocks : 0;
    return RBF_OK;
}

}  // namespace rbf
