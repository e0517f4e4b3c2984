// Step (d): solve the normal equations B c = b (Section 2) by Jacobi-preconditioned
// conjugate gradients on the stored upper triangle of B.
//
// SpMV y = B x over the cell-blocked upper storage (one warp per output cell c):
//   part A: the rows of cell c -- a dense m_c x L_c row-major block (own upper part,
//           three contiguous column ranges), streamed with coalesced loads and
//           reduced per row with warp shuffles;
//   part B: the transposed contributions of the 12 lower neighbour cells c', whose
//           row blocks hold the entries B[c', c] as an m_c' x m_c sub-block; lane j
//           reads column j of it (consecutive lanes read consecutive addresses).
//   The sub-blocks of part B were streamed by their owner cell shortly before (cells
//   run in key order), so the second read is served from L2: HBM sees each stored
//   value about once per SpMV, half the traffic of storing both triangles.
//
// CG runs as a chain of three kernels per iteration (SpMV + p.q, vector update +
// r.z / r.r, direction update); the scalars live in device memory and grid-wide sums
// use a last-block-done ticket (no spin waits). A chunk of iterations is captured into
// a CUDA graph once and replayed; every kernel checks a device-side state word first,
// so replays past convergence cost only empty launches.
//
// Precision RBF_FP32_REFINE: B is FP32 and the inner CG runs in FP32 on the correction
// equation B d = r; the residual r = A^T (h - A c) is recomputed matrix-free in FP64
// from the points (so the refinement converges to the FP64 least-squares solution, not
// to that of the rounded B), and c += d is applied in FP64.
#include <math.h>

#include <algorithm>

#include "rbf_internal.h"

namespace rbf {

struct CgScalars {
    double rz, pq, alpha, beta, rr, bb, tol2, rr0;
    int it, maxit, state, pad;
    unsigned int ticket, pad2;
};

enum { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxIt = 3 };

namespace {

constexpr int kVecThreads = 256;
constexpr int kSpmvWarps = 8;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV doubles; the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        v[k] = warp_sum_d(v[k]);
        if (lane == 0) red[k][w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? red[k][lane] : 0.0;
            v[k] = warp_sum_d(s);
        }
    }
}

// Stores this block's NV partial sums; returns true in the (single) last block to finish,
// which then holds the totals, summed in block order, in tot[] (thread 0 only).
template <int NV>
__device__ bool last_block_total(double (&v)[NV], double* partial, unsigned int* ticket,
                                 double (&tot)[NV]) {
    __shared__ bool amlast;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[NV * blockIdx.x + k] = v[k];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        amlast = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!amlast) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partial[NV * b + k]);
    // fixed-order reduction of the per-thread sums
    block_sum<NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = acc[k];
        *ticket = 0;
    }
    return true;
}

__device__ __forceinline__ int colmap(const RowSeg& sg, int k) {
    return k < sg.l0 ? sg.s0 + k : (k < sg.l0 + sg.l1 ? sg.s1 + (k - sg.l0) : sg.s2 + (k - sg.l0 - sg.l1));
}

// y = B x (rows with dinv == 0 -- pinned centres -- give 0). With sc != nullptr the kernel
// is a CG step: it returns at once unless the solve is running, and accumulates p.q.
template <typename T>
__global__ void __launch_bounds__(kSpmvWarps * 32)
    k_spmv(Binned bd, const T* __restrict__ B, const T* __restrict__ x, T* __restrict__ y,
           const T* __restrict__ dinv, CgScalars* __restrict__ sc, double* __restrict__ partial) {
    if (sc && sc->state != kRunning) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kSpmvWarps + warp;
    const Grid& g = bd.g;
    double dsum = 0.0;
    if (c < g.ncell) {
        const int cs = bd.cstart[c];
        const int m = bd.cstart[c + 1] - cs;
        if (m > 0) {
            const RowSeg sg = bd.seg[c];
            const int L = sg.l0 + sg.l1 + sg.l2;
            const T* Bc = B + bd.rboff[c];
            const int ix = c % g.gx, iy = c / g.gx;
            for (int j0 = 0; j0 < m; j0 += 32) {
                T acc = T(0);
                const int jend = min(m, j0 + 32);
                // part A: own upper rows
                for (int i = j0; i < jend; ++i) {
                    const T* row = Bc + int64_t(i) * L;
                    T s = T(0);
                    for (int k = lane; k < L; k += 32) s = fma(row[k], x[colmap(sg, k)], s);
                    s = warp_sum(s);
                    if (lane == i - j0) acc += s;
                }
                // part B: transposed blocks of the 12 lower neighbours
                const bool jv = j0 + lane < m;
#pragma unroll 1
                for (int nbr = 0; nbr < 12; ++nbr) {
                    int dx, dy;
                    if (nbr < 2) {
                        dx = -1 - nbr;
                        dy = 0;
                    } else {
                        dx = (nbr - 2) % 5 - 2;
                        dy = (nbr - 2) / 5 + 1;
                    }
                    const int nx = ix + dx, ny = iy - dy;
                    if (nx < 0 || nx >= g.gx || ny < 0) continue;
                    const int cp = ny * g.gx + nx;
                    const int csp = bd.cstart[cp];
                    const int mp = bd.cstart[cp + 1] - csp;
                    if (mp == 0) continue;
                    const RowSeg sp = bd.seg[cp];
                    const int Lp = sp.l0 + sp.l1 + sp.l2;
                    int koff;
                    if (dy == 0) koff = cs - sp.s0;
                    else if (dy == 1) koff = sp.l0 + (cs - sp.s1);
                    else koff = sp.l0 + sp.l1 + (cs - sp.s2);
                    const T* blk = B + bd.rboff[cp] + koff + j0 + lane;
                    if (jv) {
                        T a2 = T(0);
                        for (int i = 0; i < mp; ++i) a2 = fma(blk[int64_t(i) * Lp], x[csp + i], a2);
                        acc += a2;
                    }
                }
                if (jv) {
                    const int s = cs + j0 + lane;
                    const T out = (dinv && dinv[s] == T(0)) ? T(0) : acc;
                    y[s] = out;
                    if (sc) dsum += double(x[s]) * double(out);
                }
            }
        }
    }
    if (!sc) return;
    double v[1] = {dsum}, tot[1];
    if (last_block_total<1>(v, partial, &sc->ticket, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
            sc->state = kBreakdown;
        } else {
            sc->pq = pq;
            sc->alpha = sc->rz / pq;
        }
    }
}

// x += alpha p; r -= alpha q; z = dinv r; then rz, rr, convergence test and beta.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_update(int M, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                const T* __restrict__ p, const T* __restrict__ q, const T* __restrict__ dinv,
                CgScalars* __restrict__ sc, double* __restrict__ partial) {
    if (sc->state != kRunning) return;
    const T alpha = T(sc->alpha);
    double rz = 0.0, rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const T pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        const T zi = dinv[i] * ri;
        z[i] = zi;
        rz += double(ri) * double(zi);
        rr += double(ri) * double(ri);
    }
    double v[2] = {rz, rr}, tot[2];
    if (last_block_total<2>(v, partial, &sc->ticket, tot) && threadIdx.x == 0) {
        sc->it += 1;
        sc->rr = tot[1];
        if (!isfinite(tot[0]) || !isfinite(tot[1])) {
            sc->state = kBreakdown;
        } else if (tot[1] <= sc->tol2 * sc->bb) {
            sc->state = kConverged;
        } else if (sc->it >= sc->maxit) {
            sc->state = kMaxIt;
        } else {
            sc->beta = tot[0] / sc->rz;
            sc->rz = tot[0];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_p(int M, const T* __restrict__ z, T* __restrict__ p, const CgScalars* __restrict__ sc) {
    if (sc->state != kRunning) return;
    const T beta = T(sc->beta);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// r = b - y (or b when y == nullptr), masked; z = dinv r; p = z; sums rz, rr, bb.
template <typename T, typename TB>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_init(int M, const TB* __restrict__ b, double bscale, const T* __restrict__ y,
              T* __restrict__ r, T* __restrict__ z, T* __restrict__ p, const T* __restrict__ dinv,
              CgScalars* __restrict__ sc, double* __restrict__ partial) {
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const T di = dinv[i];
        const T bi = di == T(0) ? T(0) : T(double(b[i]) * bscale);
        const T ri = y ? bi - y[i] : bi;
        const T ri2 = di == T(0) ? T(0) : ri;
        const T zi = di * ri2;
        r[i] = ri2;
        z[i] = zi;
        p[i] = zi;
        rz += double(ri2) * double(zi);
        rr += double(ri2) * double(ri2);
        bb += double(bi) * double(bi);
    }
    double v[3] = {rz, rr, bb}, tot[3];
    if (last_block_total<3>(v, partial, &sc->ticket, tot) && threadIdx.x == 0) {
        sc->rz = tot[0];
        sc->rr = tot[1];
        sc->rr0 = tot[1];
        sc->bb = tot[2];
        sc->it = 0;
        if (tot[1] <= sc->tol2 * tot[2] || tot[2] == 0.0) sc->state = kConverged;
        else if (sc->maxit <= 0) sc->state = kMaxIt;
        else sc->state = kRunning;
    }
}

// dinv[s] = 1 / B_ss for centres with at least min_support points inside their support,
// else 0 (pinned: the row and column are removed from the system).
template <typename T>
__global__ void k_dinv(Binned bd, const T* __restrict__ B, const int* __restrict__ support,
                       int min_support, T* __restrict__ dinv, int* __restrict__ npinned) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= bd.g.ncell) return;
    const int cs = bd.cstart[c], m = bd.cstart[c + 1] - cs;
    if (m == 0) return;
    const RowSeg sg = bd.seg[c];
    const int L = sg.l0 + sg.l1 + sg.l2;
    const T* Bc = B + bd.rboff[c];
    int np = 0;
    for (int i = 0; i < m; ++i) {
        const T d = Bc[int64_t(i) * L + i];
        const bool pin = support[cs + i] < min_support || !(d > T(0));
        dinv[cs + i] = pin ? T(0) : T(1) / d;
        np += pin;
    }
    if (np) atomicAdd(npinned, np);
}

__global__ void k_gather(const double* __restrict__ src, const int* __restrict__ perm,
                         double* __restrict__ dst, int M) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) dst[s] = src[perm[s]];
}
__global__ void k_scatter(const double* __restrict__ src, const int* __restrict__ perm,
                          double* __restrict__ dst, int M) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) dst[perm[s]] = src[s];
}

// x64 = (x64 + scale * d32) on unpinned rows; x64 pinned rows forced to 0.
__global__ void k_axpy_mixed(int M, double* __restrict__ x, const float* __restrict__ d,
                             double scale, const float* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) x[i] = dinv[i] == 0.0f ? 0.0 : fma(scale, double(d[i]), x[i]);
}

__global__ void k_mask_zero(int M, double* __restrict__ x, const float* __restrict__ dinv32,
                            const double* __restrict__ dinv64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) {
        const bool pin = dinv32 ? dinv32[i] == 0.0f : dinv64[i] == 0.0;
        if (pin) x[i] = 0.0;
    }
}

// ||v||^2 over unpinned rows into out[0] (single block, fixed order).
__global__ void k_norm2(int M, const double* __restrict__ v, const float* __restrict__ dinv32,
                        double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        if (dinv32 && dinv32[i] == 0.0f) continue;
        s += v[i] * v[i];
    }
    double a[1] = {s};
    block_sum<1>(a);
    if (threadIdx.x == 0) out[0] = a[0];
}

template <typename T>
struct CgVecs {
    T *x, *r, *z, *p, *q, *dinv;
};

template <typename T>
CgVecs<T> vecs(rbf_ctx* ctx);
template <>
CgVecs<double> vecs<double>(rbf_ctx* ctx) {
    return {ctx->x.as<double>(), ctx->r.as<double>(), ctx->z.as<double>(), ctx->p.as<double>(),
            ctx->q.as<double>(), ctx->dinv.as<double>()};
}
template <>
CgVecs<float> vecs<float>(rbf_ctx* ctx) {
    return {ctx->x32.as<float>(), ctx->r32.as<float>(), ctx->z32.as<float>(), ctx->p32.as<float>(),
            ctx->q32.as<float>(), ctx->dinv32.as<float>()};
}

int spmv_grid(const rbf_ctx* ctx) { return div_up(ctx->g.ncell, kSpmvWarps); }
int vec_grid(const rbf_ctx* ctx) { return std::min(div_up(ctx->M, kVecThreads), 152 * 8); }

// CUDA graph holding `chunk` CG iterations for precision T (cached per context).
// Graph chunk sizes are powers of two from 8 to 256.
int chunk_of(const rbf_ctx*, int chunk) {
    int ck = 0;
    while ((8 << ck) < chunk && ck < 5) ++ck;
    return 8 << ck;
}

template <typename T>
rbf_status cg_graph(rbf_ctx* ctx, int chunk, cudaGraphExec_t* out) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    int ck = 0;
    while ((8 << ck) < chunk && ck < 5) ++ck;
    chunk = 8 << ck;
    rbf_ctx::GraphCache& gc = ctx->graphs[slot][ck];
    const Binned bd = view(ctx);
    const CgVecs<T> v = vecs<T>(ctx);
    const void* key[8] = {ctx->bvals.p, v.x, v.p, v.q, ctx->scal.p, ctx->partial.p, bd.cstart,
                          bd.seg};
    bool hit = gc.exec && gc.M == ctx->M && gc.ncell == ctx->g.ncell && gc.gx == ctx->g.gx;
    for (int k = 0; k < 8 && hit; ++k) hit = gc.key[k] == key[k];
    if (hit) {
        *out = gc.exec;
        return RBF_OK;
    }
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    cudaStream_t cs = ctx->capture_stream;
    RBF_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    CgScalars* sc = ctx->scal.as<CgScalars>();
    double* part = ctx->partial.as<double>();
    const T* B = ctx->bvals.as<T>();
    for (int k = 0; k < chunk; ++k) {
        k_spmv<T><<<spmv_grid(ctx), kSpmvWarps * 32, 0, cs>>>(bd, B, v.p, v.q, v.dinv, sc, part);
        k_cg_update<T><<<vec_grid(ctx), kVecThreads, 0, cs>>>(ctx->M, v.x, v.r, v.z, v.p, v.q,
                                                              v.dinv, sc, part);
        k_cg_p<T><<<vec_grid(ctx), kVecThreads, 0, cs>>>(ctx->M, v.z, v.p, sc);
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate", __FILE__, __LINE__);
    gc.M = ctx->M;
    gc.ncell = ctx->g.ncell;
    gc.gx = ctx->g.gx;
    for (int k = 0; k < 8; ++k) gc.key[k] = key[k];
    *out = gc.exec;
    return RBF_OK;
}

// Jacobi-PCG on the assembled B (precision T) for B x = bscale * b. x holds the start
// vector when use_x0 (sorted order, pinned rows zero). Returns the final state.
template <typename T, typename TB>
rbf_status run_cg(rbf_ctx* ctx, const TB* b, double bscale, bool use_x0, double tol, int maxit,
                  int* iters, double* relres, int* state, cudaStream_t st) {
    const Binned bd = view(ctx);
    const CgVecs<T> v = vecs<T>(ctx);
    const int M = ctx->M;
    CgScalars* sc = ctx->scal.as<CgScalars>();
    double* part = ctx->partial.as<double>();
    CgScalars h{};
    h.tol2 = tol * tol;
    h.maxit = maxit;
    h.state = kRunning;
    RBF_CUDA_TRY(cudaMemcpyAsync(sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, st));
    if (use_x0) {
        k_spmv<T><<<spmv_grid(ctx), kSpmvWarps * 32, 0, st>>>(bd, ctx->bvals.as<T>(), v.x, v.q,
                                                              v.dinv, nullptr, nullptr);
    } else {
        RBF_CUDA_TRY(cudaMemsetAsync(v.x, 0, sizeof(T) * M, st));
    }
    k_cg_init<T, TB><<<vec_grid(ctx), kVecThreads, 0, st>>>(M, b, bscale, use_x0 ? v.q : nullptr,
                                                            v.r, v.z, v.p, v.dinv, sc, part);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += use_x0 ? 2 : 1;
    CgScalars* hs = static_cast<CgScalars*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    // replay graph chunks; the chunk length follows the observed convergence rate
    int chunk = 16;
    double log_rr_prev = log(std::max(hs->rr, 1e-300));
    int it_prev = 0;
    while (hs->state == kRunning) {
        cudaGraphExec_t ex;
        rbf_status s = cg_graph<T>(ctx, chunk, &ex);
        if (s != RBF_OK) return s;
        RBF_CUDA_TRY(cudaGraphLaunch(ex, st));
        ctx->launches += 3 * chunk_of(ctx, chunk);
        RBF_CUDA_TRY(cudaMemcpyAsync(hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs->state != kRunning) break;
        // predict the iterations left from the decrease of log ||r||^2 per iteration
        const double lr = log(std::max(hs->rr, 1e-300));
        const double target = log(std::max(hs->tol2 * hs->bb, 1e-300));
        const double rate = (log_rr_prev - lr) / std::max(1, hs->it - it_prev);
        int want = rate > 0 ? int((lr - target) / rate) + 1 : 64;
        want = std::min(std::max(want, 8), std::min(256, std::max(8, hs->maxit - hs->it)));
        // keep a small set of graph sizes so that the cache stays warm
        int c2 = 8;
        while (c2 < want) c2 *= 2;
        chunk = c2;
        log_rr_prev = lr;
        it_prev = hs->it;
    }
    *iters = hs->it;
    *relres = hs->bb > 0 ? sqrt(hs->rr / hs->bb) : 0.0;
    *state = hs->state;
    return RBF_OK;
}

}  // namespace

void launch_gather_sorted(const double* c_orig, const int* cperm, double* c_sorted, int M,
                          cudaStream_t st) {
    k_gather<<<div_up(M, 256), 256, 0, st>>>(c_orig, cperm, c_sorted, M);
}
void launch_scatter_orig(const double* c_sorted, const int* cperm, double* c_orig, int M,
                         cudaStream_t st) {
    k_scatter<<<div_up(M, 256), 256, 0, st>>>(c_sorted, cperm, c_orig, M);
}

size_t cg_scalars_bytes() { return sizeof(CgScalars); }

rbf_status bench_spmv_run(rbf_ctx* ctx, int reps, cudaStream_t st) {
    const Binned bd = view(ctx);
    for (int k = 0; k < reps; ++k) {
        if (ctx->prec == RBF_FP64)
            k_spmv<double><<<spmv_grid(ctx), kSpmvWarps * 32, 0, st>>>(
                bd, ctx->bvals.as<double>(), ctx->p.as<double>(), ctx->q.as<double>(),
                ctx->dinv.as<double>(), nullptr, nullptr);
        else
            k_spmv<float><<<spmv_grid(ctx), kSpmvWarps * 32, 0, st>>>(
                bd, ctx->bvals.as<float>(), ctx->p32.as<float>(), ctx->q32.as<float>(),
                ctx->dinv32.as<float>(), nullptr, nullptr);
    }
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += reps;
    return RBF_OK;
}

static rbf_status finish_status(rbf_ctx* ctx, int state) {
    if (state == kConverged) return RBF_OK;
    if (state == kBreakdown) return set_err(ctx, RBF_ERR_BREAKDOWN, "CG breakdown (p^T B p <= 0 or non-finite)");
    return set_err(ctx, RBF_ERR_NOT_CONVERGED, "CG reached maxit before tol");
}

rbf_status solve_run(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit, int min_support,
                     rbf_solve_info* info, cudaStream_t st) {
    const int M = ctx->M;
    const Binned bd = view(ctx);
    rbf_status s;
#define ENS(buf, bytes) \
    if ((s = ensure(ctx, ctx->buf, (bytes), st)) != RBF_OK) return s;
    ENS(x, sizeof(double) * M);
    ENS(r, sizeof(double) * M);
    ENS(scal, sizeof(CgScalars) + 64);
    ENS(partial, sizeof(double) * 3 * std::max(spmv_grid(ctx), vec_grid(ctx)));
    int64_t* npin_h = static_cast<int64_t*>(ctx->hpinned) + 64;
    int* npin_d = reinterpret_cast<int*>(ctx->scal.as<char>() + sizeof(CgScalars));
    RBF_CUDA_TRY(cudaMemsetAsync(npin_d, 0, sizeof(int), st));
    rbf_solve_info inf{};
    int state = kConverged;

    if (ctx->prec == RBF_FP64) {
        ENS(z, sizeof(double) * M);
        ENS(p, sizeof(double) * M);
        ENS(q, sizeof(double) * M);
        ENS(dinv, sizeof(double) * M);
        k_dinv<double><<<div_up(ctx->g.ncell, 128), 128, 0, st>>>(
            bd, ctx->bvals.as<double>(), ctx->support.as<int>(), min_support,
            ctx->dinv.as<double>(), npin_d);
        ctx->launches += 1;
        if (use_c0) {
            launch_gather_sorted(c, bd.cperm, ctx->x.as<double>(), M, st);
            k_mask_zero<<<div_up(M, 256), 256, 0, st>>>(M, ctx->x.as<double>(), nullptr,
                                                        ctx->dinv.as<double>());
            ctx->launches += 2;
        }
        RBF_CUDA_TRY(cudaGetLastError());
        int it = 0;
        double rel = 0.0;
        s = run_cg<double, double>(ctx, ctx->bvec.as<double>(), 1.0, use_c0 != 0, tol, maxit, &it,
                                   &rel, &state, st);
        if (s != RBF_OK) return s;
        inf.iterations = it;
        inf.rel_residual = rel;
    } else {
        ENS(x32, sizeof(float) * M);
        ENS(r32, sizeof(float) * M);
        ENS(z32, sizeof(float) * M);
        ENS(p32, sizeof(float) * M);
        ENS(q32, sizeof(float) * M);
        ENS(dinv32, sizeof(float) * M);
        k_dinv<float><<<div_up(ctx->g.ncell, 128), 128, 0, st>>>(
            bd, ctx->bvals.as<float>(), ctx->support.as<int>(), min_support,
            ctx->dinv32.as<float>(), npin_d);
        ctx->launches += 1;
        double* x64 = ctx->x.as<double>();
        double* r64 = ctx->r.as<double>();
        double* nrm_d = reinterpret_cast<double*>(ctx->scal.as<char>() + sizeof(CgScalars) + 8);
        double* nrm_h = reinterpret_cast<double*>(static_cast<char*>(ctx->hpinned) + 1024);
        const float* dinv32 = ctx->dinv32.as<float>();
        // ||b|| over unpinned rows
        k_norm2<<<1, 1024, 0, st>>>(M, ctx->bvec.as<double>(), dinv32, nrm_d);
        ctx->launches += 1;
        RBF_CUDA_TRY(cudaMemcpyAsync(nrm_h, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, st));
        if (use_c0) {
            launch_gather_sorted(c, bd.cperm, x64, M, st);
            k_mask_zero<<<div_up(M, 256), 256, 0, st>>>(M, x64, dinv32, nullptr);
            ctx->launches += 2;
            RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
            if ((s = residual_run(ctx, x64, r64, false, st)) != RBF_OK) return s;
        } else {
            RBF_CUDA_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * M, st));
            RBF_CUDA_TRY(cudaMemcpyAsync(r64, ctx->bvec.p, sizeof(double) * M,
                                         cudaMemcpyDeviceToDevice, st));
        }
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        const double bnorm = sqrt(nrm_h[0]);
        int total_it = 0, outer = 0;
        double rel = 0.0;
        state = kMaxIt;
        // Inner tolerance: each refinement step should gain about 4 digits; FP32 rounding of
        // B (relative 6e-8 per entry) limits the gain per step, not the final accuracy.
        const double inner_tol = 1e-4;
        for (outer = 0; outer <= 30; ++outer) {
            k_norm2<<<1, 1024, 0, st>>>(M, r64, dinv32, nrm_d);
            ctx->launches += 1;
            RBF_CUDA_TRY(cudaMemcpyAsync(nrm_h, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, st));
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            const double rn = sqrt(nrm_h[0]);
            rel = bnorm > 0 ? rn / bnorm : 0.0;
            if (rel <= tol || rn == 0.0) {
                state = kConverged;
                break;
            }
            if (outer == 30) break;
            int it = 0, ist = 0;
            double irel = 0.0;
            s = run_cg<float, double>(ctx, r64, 1.0 / rn, false, std::max(inner_tol, 0.5 * tol / rel),
                                      maxit, &it, &irel, &ist, st);
            if (s != RBF_OK) return s;
            total_it += it;
            if (ist == kBreakdown) {
                state = kBreakdown;
                break;
            }
            k_axpy_mixed<<<div_up(M, 256), 256, 0, st>>>(M, x64, ctx->x32.as<float>(), rn, dinv32);
            ctx->launches += 2;   // with the mask below
            RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
            if ((s = residual_run(ctx, x64, r64, false, st)) != RBF_OK) return s;
            k_mask_zero<<<div_up(M, 256), 256, 0, st>>>(M, r64, dinv32, nullptr);
        }
        inf.iterations = total_it;
        inf.refinements = outer;
        inf.rel_residual = rel;
    }
    launch_scatter_orig(ctx->x.as<double>(), bd.cperm, c, M, st);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    ctx->solved = true;
    RBF_CUDA_TRY(cudaMemcpyAsync(npin_h, npin_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    inf.pinned = *reinterpret_cast<int*>(npin_h);
    if (info) *info = inf;
#undef ENS
    return finish_status(ctx, state);
}

}  // namespace rbf
