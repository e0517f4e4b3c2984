// C-ABI entry points of librbf (declared in include/rbf.h): argument checks, context
// and workspace management; the work itself is done by the kernels of the other units.
#include <stdint.h>
#include <math.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <new>

#include "rbf_internal.h"

namespace rbf {

rbf_status set_err(rbf_ctx* ctx, rbf_status s, const char* msg) {
    if (ctx) ctx->err = msg;
    return s;
}

rbf_status cuda_fail(rbf_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
             cudaGetErrorString(e), what, file, line);
    if (ctx) ctx->err = buf;
    return RBF_ERR_CUDA;
}

void release(rbf_ctx* ctx, rbf_buf& b) {
    if (!b.p) return;
    if (ctx->free_fn)
        ctx->free_fn(b.p, b.bytes, nullptr, ctx->user);
    else
        cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

rbf_status ensure(rbf_ctx* ctx, rbf_buf& b, size_t bytes, cudaStream_t st) {
    bytes = std::max<size_t>(bytes, 256);
    if (b.p && b.bytes >= bytes) return RBF_OK;
    if (b.p) {
        // the old buffer may still be read by queued work on this stream
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize", __FILE__, __LINE__);
        release(ctx, b);
    }
    // round up to limit reallocations when sizes grow slowly
    const size_t want = bytes + bytes / 8;
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(want, st, ctx->user);
    } else if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) return set_err(ctx, RBF_ERR_ALLOC, "workspace allocation failed");
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
        // the kernels read the workspace in 16-byte vectors from offsets that assume it
        if (ctx->free_fn) ctx->free_fn(p, want, nullptr, ctx->user);
        return set_err(ctx, RBF_ERR_ALLOC, "the allocator returned memory not aligned to 256 bytes");
    }
    b.p = p;
    b.bytes = want;
    return RBF_OK;
}

Binned view(const rbf_ctx* ctx) {
    Binned v;
    v.g = ctx->g;
    v.M = ctx->M;
    v.N = ctx->N;
    v.cstart = ctx->cstart.as<int>();
    v.pstart = ctx->pstart.as<int>();
    v.cx = ctx->cx.as<double>();
    v.cy = ctx->cy.as<double>();
    v.cu = ctx->cu.as<float>();
    v.cv = ctx->cv.as<float>();
    v.px = ctx->px.as<double>();
    v.py = ctx->py.as<double>();
    v.ph = ctx->ph.as<double>();
    v.pu = ctx->pu.as<float>();
    v.pv = ctx->pv.as<float>();
    v.cperm = ctx->cperm.as<int>();
    v.rmeta = ctx->rmeta.as<RowMeta>();
    v.gdesc = ctx->gdesc.as<GroupRec>();
    v.ngroup = ctx->ngroup;
    v.bjoff = ctx->bjoff.as<int64_t>();
    v.crow = ctx->crow.as<int4>();
    return v;
}

}  // namespace rbf

using namespace rbf;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

rbf_status rbf_create(rbf_ctx** out, int device, rbf_alloc_fn alloc, rbf_free_fn free_fn,
                      void* user) {
    if (!out) return RBF_ERR_ARG;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return RBF_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return RBF_ERR_CUDA;
    }
    rbf_ctx* ctx = new (std::nothrow) rbf_ctx();
    if (!ctx) return RBF_ERR_ALLOC;
    ctx->device = device;
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    DeviceGuard dg(device);
    if (cudaMallocHost(&ctx->hpinned, 4096) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->hpinned) cudaFreeHost(ctx->hpinned);
        delete ctx;
        return RBF_ERR_CUDA;
    }
    *out = ctx;
    return RBF_OK;
}

rbf_status rbf_destroy(rbf_ctx* ctx) {
    if (!ctx) return RBF_ERR_ARG;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    for (auto& sg : ctx->cg_graph)
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
    tiles_release(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    rbf_buf* bufs[] = {&ctx->ccount, &ctx->pcount, &ctx->cstart, &ctx->pstart, &ctx->ckey,
                       &ctx->crank, &ctx->pkey, &ctx->prank, &ctx->cx, &ctx->cy, &ctx->cu,
                       &ctx->cv, &ctx->cperm, &ctx->px, &ctx->py, &ctx->ph, &ctx->pu, &ctx->pv,
                       &ctx->rmeta, &ctx->rsize, &ctx->roff, &ctx->gcount, &ctx->gstart, &ctx->gdesc, &ctx->wcount, &ctx->wstart, &ctx->bjsize, &ctx->bjoff,
                       &ctx->work, &ctx->scan_tmp, &ctx->stats, &ctx->bvals, &ctx->bvec,
                       &ctx->support, &ctx->x, &ctx->r, &ctx->cgv[0], &ctx->cgv[1],
                       &ctx->dinv, &ctx->dinv32, &ctx->bjinv, &ctx->bjinv32, &ctx->crow,
                       &ctx->partial, &ctx->scal, &ctx->csort, &ctx->sigma, &ctx->feat,
                       &ctx->mlp_part, &ctx->astore, &ctx->amask, &ctx->woff, &ctx->wsize,
                       &ctx->pE, &ctx->pE32, &ctx->pdev, &ctx->pepart, &ctx->bblock, &ctx->bandtab,
                       &ctx->win_eval, &ctx->win_edges, &ctx->win_count, &ctx->win_off, &ctx->win_c, &ctx->win_cidx, &ctx->win_p};
    for (rbf_buf* b : bufs) release(ctx, *b);
    if (ctx->hpinned) cudaFreeHost(ctx->hpinned);
    if (ctx->bhost) cudaFreeHost(ctx->bhost);
    delete ctx;
    return RBF_OK;
}

const char* rbf_last_error(const rbf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rbf_max_candidates(void) { return kMaxCand; }

rbf_status rbf_bin(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M, const double* px,
                   const double* py, const double* h, int64_t N, double R, const double* bbox,
                   void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    ctx->win_on = false;
    ctx->binned = false;
    ctx->assembled = false;
    ctx->solved = false;
    if (!cx || !cy || !px || !py || !h || !bbox)
        return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    if (M < 1 || N < 1 || M > (int64_t(1) << 30) || N > (int64_t(1) << 30))
        return set_err(ctx, RBF_ERR_ARG, "need 1 <= M, N <= 2^30");
    if (!(R > 0.0) || !isfinite(R)) return set_err(ctx, RBF_ERR_ARG, "R must be finite and > 0");
    for (int k = 0; k < 4; ++k)
        if (!isfinite(bbox[k])) return set_err(ctx, RBF_ERR_ARG, "non-finite bbox");
    if (!(bbox[2] >= bbox[0]) || !(bbox[3] >= bbox[1]))
        return set_err(ctx, RBF_ERR_ARG, "bbox must be {x0, y0, x1, y1} with x1 >= x0, y1 >= y0");
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
    if (nxf * nyf > double(1 << 24))
        return set_err(ctx, RBF_ERR_LIMIT, "cell grid larger than 2^24 cells (R too small for bbox)");
    g.gx = int(nxf);
    g.gy = int(nyf);
    g.ncell = g.gx * g.gy;
    ctx->g = g;
    ctx->M = int(M);
    ctx->N = int(N);
    ctx->T = 0;
    ctx->astore_ok = false;
    DeviceGuard dg(ctx->device);
    rbf_status s = bin_run(ctx, cx, cy, px, py, h, as_stream(stream));
    if (s == RBF_OK) ctx->binned = true;
    return s;
}

rbf_status rbf_assemble(rbf_ctx* ctx, rbf_kernel kernel, rbf_prec prec, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned) return set_err(ctx, RBF_ERR_ARG, "rbf_assemble before rbf_bin");
    if (kernel < RBF_W30 || kernel > RBF_W33) return set_err(ctx, RBF_ERR_ARG, "unknown kernel");
    if (prec != RBF_FP64 && prec != RBF_FP32_REFINE) return set_err(ctx, RBF_ERR_ARG, "unknown precision");
    DeviceGuard dg(ctx->device);
    ctx->kernel = kernel;
    ctx->prec = prec;
    ctx->solved = false;
    rbf_status s = assemble_run(ctx, kernel, prec, as_stream(stream));
    ctx->assembled = s == RBF_OK;
    return s;
}

rbf_status rbf_solve(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit, int min_support,
                     rbf_solve_info* info, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_solve before rbf_assemble");
    if (!c) return set_err(ctx, RBF_ERR_ARG, "null c");
    if (!(tol >= 0.0) || maxit < 0) return set_err(ctx, RBF_ERR_ARG, "need tol >= 0, maxit >= 0");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "batched context: use rbf_solve_tiles");
    DeviceGuard dg(ctx->device);
    return solve_run(ctx, c, use_c0, tol, maxit, min_support, info, as_stream(stream));
}

rbf_status rbf_assemble_poly(rbf_ctx* ctx, rbf_kernel kernel, rbf_prec prec, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned) return set_err(ctx, RBF_ERR_ARG, "rbf_assemble_poly before rbf_bin");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_assemble_poly on a batched context");
    if (kernel < RBF_W30 || kernel > RBF_W33) return set_err(ctx, RBF_ERR_ARG, "unknown kernel");
    if (prec != RBF_FP64 && prec != RBF_FP32_REFINE) return set_err(ctx, RBF_ERR_ARG, "unknown precision");
    DeviceGuard dg(ctx->device);
    ctx->kernel = kernel;
    ctx->prec = prec;
    ctx->solved = false;
    rbf_status s = assemble_run(ctx, kernel, prec, as_stream(stream), true);
    ctx->assembled = s == RBF_OK;
    return s;
}

rbf_status rbf_solve_poly(rbf_ctx* ctx, double* c, double* k, double tol, int maxit,
                          int min_support, rbf_solve_info* info, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled || !ctx->poly)
        return set_err(ctx, RBF_ERR_ARG, "rbf_solve_poly before rbf_assemble_poly");
    if (!c || !k) return set_err(ctx, RBF_ERR_ARG, "null c or k");
    if (!(tol >= 0.0) || maxit < 0) return set_err(ctx, RBF_ERR_ARG, "need tol >= 0, maxit >= 0");
    DeviceGuard dg(ctx->device);
    return solve_poly_run(ctx, c, k, tol, maxit, min_support, info, as_stream(stream));
}

rbf_status rbf_eval_poly(rbf_ctx* ctx, const double* c, const double* k, const double* qx,
                         const double* qy, int64_t Q, double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned || ctx->kernel < 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval_poly before rbf_assemble");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval_poly on a batched context");
    if (Q < 0 || (Q > 0 && (!c || !k || !qx || !qy || !f)))
        return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    DeviceGuard dg(ctx->device);
    return eval_points_poly_run(ctx, c, k, qx, qy, Q, f, as_stream(stream));
}

rbf_status rbf_eval_grid_poly(rbf_ctx* ctx, const double* c, const double* k, int nx, int ny,
                              const double* box, double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned || ctx->kernel < 0)
        return set_err(ctx, RBF_ERR_ARG, "rbf_eval_grid_poly before rbf_assemble");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval_grid_poly on a batched context");
    if (nx < 1 || ny < 1 || !c || !k || !box || !f) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    for (int j = 0; j < 4; ++j)
        if (!isfinite(box[j])) return set_err(ctx, RBF_ERR_ARG, "non-finite box");
    DeviceGuard dg(ctx->device);
    return eval_grid_run(ctx, c, nx, ny, box, f, as_stream(stream), k);
}

rbf_status rbf_bin_tiles(rbf_ctx* ctx, const rbf_tile* tiles, int T, const double* cx,
                         const double* cy, int64_t Mtot, const double* px, const double* py,
                         const double* h, int64_t Ntot, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    ctx->binned = false;
    ctx->assembled = false;
    ctx->solved = false;
    ctx->win_on = false;
    if (!tiles || T < 1) return set_err(ctx, RBF_ERR_ARG, "need T >= 1 tiles");
    if (!cx || !cy || (Ntot > 0 && (!px || !py || !h)))
        return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    if (Mtot < 1 || Ntot < 0 || Mtot > (int64_t(1) << 30) || Ntot > (int64_t(1) << 30))
        return set_err(ctx, RBF_ERR_ARG, "need 1 <= Mtot <= 2^30, 0 <= Ntot <= 2^30");
    DeviceGuard dg(ctx->device);
    rbf_status s = bin_tiles_run(ctx, tiles, T, cx, cy, Mtot, px, py, h, Ntot, as_stream(stream));
    if (s == RBF_OK) ctx->binned = true;
    return s;
}

rbf_status rbf_bin_windows(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M,
                           const double* px, const double* py, const double* h, int64_t N,
                           double R, const double* bbox, int wx, int wy, double overlap,
                           double margin, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    ctx->binned = false;
    ctx->assembled = false;
    ctx->solved = false;
    ctx->win_on = false;
    if (!cx || !cy || !px || !py || !h || !bbox) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    if (M < 1 || N < 1 || M > (int64_t(1) << 30) || N > (int64_t(1) << 30))
        return set_err(ctx, RBF_ERR_ARG, "need 1 <= M, N <= 2^30");
    if (!(R > 0.0) || !isfinite(R)) return set_err(ctx, RBF_ERR_ARG, "R must be finite and > 0");
    for (int k = 0; k < 4; ++k)
        if (!isfinite(bbox[k])) return set_err(ctx, RBF_ERR_ARG, "non-finite bbox");
    if (!(bbox[2] > bbox[0]) || !(bbox[3] > bbox[1]))
        return set_err(ctx, RBF_ERR_ARG, "bbox must be {x0, y0, x1, y1} with x1 > x0, y1 > y0");
    if (wx < 1 || wy < 1 || int64_t(wx) * wy > 65536)
        return set_err(ctx, RBF_ERR_ARG, "need wx, wy >= 1 and wx * wy <= 65536 windows");
    if (!(double(wx) / (bbox[2] - bbox[0]) < 1e30) || !(double(wy) / (bbox[3] - bbox[1]) < 1e30))
        return set_err(ctx, RBF_ERR_ARG, "windows narrower than 1e-30");
    if (!(overlap >= 0.0) || !isfinite(overlap)) return set_err(ctx, RBF_ERR_ARG, "overlap must be finite and >= 0");
    if (!(margin >= 0.0) || !isfinite(margin)) return set_err(ctx, RBF_ERR_ARG, "margin must be finite and >= 0");
    DeviceGuard dg(ctx->device);
    rbf_status s = window_bin_run(ctx, cx, cy, M, px, py, h, N, R, bbox, wx, wy, overlap, margin,
                                  as_stream(stream));
    if (s == RBF_OK) ctx->binned = true;
    return s;
}

rbf_status rbf_window_sizes(const rbf_ctx* ctx, int64_t* Mtot, int64_t* Ntot) {
    if (!ctx || !Mtot || !Ntot || !ctx->win_on) return RBF_ERR_ARG;
    *Mtot = ctx->win_M;
    *Ntot = ctx->win_N;
    return RBF_OK;
}

rbf_status rbf_window_centres(rbf_ctx* ctx, int64_t* idx, int64_t cap, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->win_on) return set_err(ctx, RBF_ERR_ARG, "rbf_window_centres before rbf_bin_windows");
    if (!idx || cap < ctx->win_M) return set_err(ctx, RBF_ERR_ARG, "idx must hold rbf_window_sizes' Mtot values");
    DeviceGuard dg(ctx->device);
    RBF_CUDA_TRY(cudaMemcpyAsync(idx, ctx->win_cidx.p, sizeof(int64_t) * size_t(ctx->win_M),
                                 cudaMemcpyDeviceToDevice, as_stream(stream)));
    return RBF_OK;
}

rbf_status rbf_eval_windows(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                            int64_t Q, double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->win_on || !ctx->assembled)
        return set_err(ctx, RBF_ERR_ARG, "rbf_eval_windows before rbf_bin_windows + rbf_assemble");
    if (Q < 0 || (Q > 0 && (!c || !qx || !qy || !f))) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    DeviceGuard dg(ctx->device);
    return window_eval_run(ctx, c, qx, qy, Q, 0, 0, nullptr, f, as_stream(stream));
}

rbf_status rbf_eval_windows_grid(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                                 double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->win_on || !ctx->assembled)
        return set_err(ctx, RBF_ERR_ARG, "rbf_eval_windows_grid before rbf_bin_windows + rbf_assemble");
    if (!c || !box || !f || nx < 1 || ny < 1) return set_err(ctx, RBF_ERR_ARG, "bad grid arguments");
    for (int k = 0; k < 4; ++k)
        if (!isfinite(box[k])) return set_err(ctx, RBF_ERR_ARG, "non-finite box");
    DeviceGuard dg(ctx->device);
    return window_eval_run(ctx, c, nullptr, nullptr, 0, nx, ny, box, f, as_stream(stream));
}

rbf_status rbf_solve_tiles(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                           int min_support, rbf_tile_info* tile_info, rbf_solve_info* info,
                           void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled || ctx->T < 1)
        return set_err(ctx, RBF_ERR_ARG, "rbf_solve_tiles before rbf_bin_tiles + rbf_assemble");
    if (!c) return set_err(ctx, RBF_ERR_ARG, "null c");
    if (!(tol >= 0.0) || maxit < 0) return set_err(ctx, RBF_ERR_ARG, "need tol >= 0, maxit >= 0");
    DeviceGuard dg(ctx->device);
    return solve_tiles_run(ctx, c, use_c0, tol, maxit, min_support, tile_info, info,
                           as_stream(stream));
}

rbf_status rbf_eval_tiles(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                          const int64_t* qoff, double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled || ctx->T < 1)
        return set_err(ctx, RBF_ERR_ARG, "rbf_eval_tiles before rbf_bin_tiles + rbf_assemble");
    if (!c || !qoff) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    if (qoff[0] != 0) return set_err(ctx, RBF_ERR_ARG, "qoff[0] must be 0");
    for (int t = 0; t < ctx->T; ++t)
        if (qoff[t + 1] < qoff[t]) return set_err(ctx, RBF_ERR_ARG, "qoff must be non-decreasing");
    if (qoff[ctx->T] > 0 && (!qx || !qy || !f)) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    DeviceGuard dg(ctx->device);
    return eval_tiles_run(ctx, c, qx, qy, qoff, 0, 0, f, as_stream(stream));
}

rbf_status rbf_eval_tiles_grid(rbf_ctx* ctx, const double* c, int nx, int ny, double* f,
                               void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled || ctx->T < 1)
        return set_err(ctx, RBF_ERR_ARG, "rbf_eval_tiles_grid before rbf_bin_tiles + rbf_assemble");
    if (nx < 1 || ny < 1 || !c || !f) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    DeviceGuard dg(ctx->device);
    return eval_tiles_run(ctx, c, nullptr, nullptr, nullptr, nx, ny, f, as_stream(stream));
}

rbf_status rbf_features(rbf_ctx* ctx, float* feat, double* sigma, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned) return set_err(ctx, RBF_ERR_ARG, "rbf_features before rbf_bin / rbf_bin_tiles");
    if (!feat) return set_err(ctx, RBF_ERR_ARG, "null feat");
    DeviceGuard dg(ctx->device);
    return features_run(ctx, feat, sigma, as_stream(stream));
}

rbf_status rbf_mlp_forward(rbf_ctx* ctx, const float* params, const float* feat, int64_t n,
                           float* y, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (n < 0 || (n > 0 && (!params || !feat || !y))) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    if (reinterpret_cast<uintptr_t>(feat) % 16) return set_err(ctx, RBF_ERR_ARG, "feat must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    return mlp_forward_run(ctx, params, feat, n, y, as_stream(stream));
}

rbf_status rbf_mlp_train_step(rbf_ctx* ctx, float* params, float* m, float* v, int step, double lr,
                              const float* feat, const float* target, const int32_t* idx,
                              int64_t n, float* grad, double* loss, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (n < 1 || !params || !feat || !target) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    if (step < 0 || (step > 0 && (!m || !v || !(lr > 0.0))))
        return set_err(ctx, RBF_ERR_ARG, "an Adam step needs m, v and lr > 0");
    DeviceGuard dg(ctx->device);
    return mlp_step_run(ctx, params, m, v, step, lr, feat, target, idx, n, grad, loss,
                        as_stream(stream));
}

rbf_status rbf_warm_start(rbf_ctx* ctx, const float* params, double* c0, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned) return set_err(ctx, RBF_ERR_ARG, "rbf_warm_start before rbf_bin / rbf_bin_tiles");
    if (!params || !c0) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    DeviceGuard dg(ctx->device);
    return warm_start_run(ctx, params, c0, as_stream(stream));
}

rbf_status rbf_mlp_targets(rbf_ctx* ctx, const double* c, float* target, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned) return set_err(ctx, RBF_ERR_ARG, "rbf_mlp_targets before rbf_bin / rbf_bin_tiles");
    if (!c || !target) return set_err(ctx, RBF_ERR_ARG, "null pointer argument");
    DeviceGuard dg(ctx->device);
    return mlp_targets_run(ctx, c, target, as_stream(stream));
}

rbf_status rbf_autotune(rbf_ctx* ctx, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled || ctx->T < 1)
        return set_err(ctx, RBF_ERR_ARG, "rbf_autotune before rbf_bin_tiles + rbf_assemble");
    DeviceGuard dg(ctx->device);
    rbf_status s = autotune_run(ctx, as_stream(stream));
    ctx->solved = false;
    return s;
}

rbf_status rbf_get_tuning(const rbf_ctx* ctx, int* spmv_blocks_per_sm, int* spmv_chunk,
                          int* update_threads, double* us_per_iteration) {
    if (!ctx) return RBF_ERR_ARG;
    const rbf_ctx::TileTuning& tu = ctx->tune[ctx->prec == RBF_FP64 ? 0 : 1];
    if (spmv_blocks_per_sm) *spmv_blocks_per_sm = tu.spmv_bps;
    if (spmv_chunk) *spmv_chunk = tu.chunk;
    if (update_threads) *update_threads = tu.nt;
    if (us_per_iteration) *us_per_iteration = tu.us_per_iter;
    return RBF_OK;
}

rbf_status rbf_eval(rbf_ctx* ctx, const double* c, const double* qx, const double* qy, int64_t Q,
                    double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned || ctx->kernel < 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval before rbf_assemble");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval on a batched context");
    if (Q < 0 || (Q > 0 && (!c || !qx || !qy || !f))) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    DeviceGuard dg(ctx->device);
    return eval_points_run(ctx, c, qx, qy, Q, f, as_stream(stream));
}

rbf_status rbf_eval_grid(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                         double* f, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->binned || ctx->kernel < 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval_grid before rbf_assemble");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_eval_grid on a batched context");
    if (nx < 1 || ny < 1 || !c || !box || !f) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    for (int k = 0; k < 4; ++k)
        if (!isfinite(box[k])) return set_err(ctx, RBF_ERR_ARG, "non-finite box");
    DeviceGuard dg(ctx->device);
    return eval_grid_run(ctx, c, nx, ny, box, f, as_stream(stream));
}

rbf_status rbf_get_layout(const rbf_ctx* ctx, int64_t* nvals, int* value_bytes, int* gx, int* gy) {
    if (!ctx) return RBF_ERR_ARG;
    if (nvals) *nvals = ctx->nvals;
    if (value_bytes) *value_bytes = ctx->prec == RBF_FP32_REFINE ? 4 : 8;
    if (gx) *gx = ctx->g.gx;
    if (gy) *gy = ctx->g.gy;
    return RBF_OK;
}

rbf_status rbf_get_layout_stats(rbf_ctx* ctx, rbf_layout_stats* out, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!out) return set_err(ctx, RBF_ERR_ARG, "null out");
    if (!ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_get_layout_stats before rbf_assemble");
    DeviceGuard dg(ctx->device);
    return layout_stats_run(ctx, out, as_stream(stream));
}

rbf_status rbf_export_upper(rbf_ctx* ctx, int64_t cap, int32_t* row, int32_t* col, double* val,
                            double* bvec, int32_t* support, int64_t* nnz, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_export_upper before rbf_assemble");
    if (!nnz || cap < 0 || (cap > 0 && (!row || !col || !val))) return set_err(ctx, RBF_ERR_ARG, "bad arguments");
    DeviceGuard dg(ctx->device);
    return export_upper_run(ctx, cap, row, col, val, bvec, support, nnz, as_stream(stream));
}

rbf_status rbf_selftest_sqrt(const double* a, double* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!a || !out))) return RBF_ERR_ARG;
    return diag_sqrt_run(a, out, n, as_stream(stream));
}

rbf_status rbf_set_param(rbf_ctx* ctx, const char* name, double value) {
    if (!ctx || !name) return RBF_ERR_ARG;
    if (!strcmp(name, "inner_tol")) {
        if (!(value > 0.0 && value < 1.0)) return set_err(ctx, RBF_ERR_ARG, "inner_tol must be in (0, 1)");
        ctx->inner_tol = value;
        return RBF_OK;
    }
    if (!strcmp(name, "max_refinements")) {
        if (!(value >= 0.0 && value <= 1000.0)) return set_err(ctx, RBF_ERR_ARG, "max_refinements must be in [0, 1000]");
        ctx->max_refine = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "store_a")) {
        if (!(value == 0.0 || value == 1.0)) return set_err(ctx, RBF_ERR_ARG, "store_a must be 0 or 1");
        ctx->store_a = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "autotune")) {
        if (!(value == 0.0 || value == 1.0)) return set_err(ctx, RBF_ERR_ARG, "autotune must be 0 or 1");
        ctx->autotune = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "spmv_blocks_per_sm")) {
        if (!(value >= 0.0 && value <= 8.0 && value == floor(value)))
            return set_err(ctx, RBF_ERR_ARG, "spmv_blocks_per_sm must be an integer in [0, 8]");
        ctx->force_bps = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "spmv_chunk")) {
        if (!(value >= 0.0 && value <= 64.0 && value == floor(value)))
            return set_err(ctx, RBF_ERR_ARG, "spmv_chunk must be an integer in [0, 64]");
        ctx->force_chunk = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "update_threads")) {
        if (!(value == 0.0 || value == 128.0 || value == 256.0 || value == 512.0))
            return set_err(ctx, RBF_ERR_ARG, "update_threads must be 0, 128, 256 or 512");
        ctx->force_nt = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "cg_persistent")) {
        if (!(value == 0.0 || value == 1.0 || value == -1.0))
            return set_err(ctx, RBF_ERR_ARG, "cg_persistent must be -1, 0 or 1");
        ctx->cg_persistent = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "cg_barrier_test")) {
        if (!(value == 0.0 || value == 1.0)) return set_err(ctx, RBF_ERR_ARG, "cg_barrier_test must be 0 or 1");
        ctx->cg_barrier_extra = int(value);
        return RBF_OK;
    }
    if (!strcmp(name, "b_device_mb")) {
        if (!(value >= 0.0 && value <= 1e9))
            return set_err(ctx, RBF_ERR_ARG, "b_device_mb must be in [0, 1e9]");
        ctx->b_device_mb = value;
        return RBF_OK;
    }
    return set_err(ctx, RBF_ERR_ARG, "unknown parameter");
}

rbf_status rbf_get_launch_count(const rbf_ctx* ctx, int64_t* launches) {
    if (!ctx || !launches) return RBF_ERR_ARG;
    *launches = ctx->launches;
    return RBF_OK;
}

rbf_status rbf_bench_spmv(rbf_ctx* ctx, int reps, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_spmv before rbf_assemble");
    if (reps < 0) return set_err(ctx, RBF_ERR_ARG, "reps < 0");
    DeviceGuard dg(ctx->device);
    if (ctx->T > 0) {
        if (!ctx->solved) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_spmv on a batch before rbf_solve_tiles");
        return bench_tiles_run(ctx, reps, true, as_stream(stream));
    }
    return bench_spmv_run(ctx, reps, as_stream(stream));
}

rbf_status rbf_bench_cg(rbf_ctx* ctx, int reps, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->solved || !ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_cg before rbf_solve");
    if (reps < 0) return set_err(ctx, RBF_ERR_ARG, "reps < 0");
    DeviceGuard dg(ctx->device);
    if (ctx->T > 0) return bench_tiles_run(ctx, reps, false, as_stream(stream));
    return bench_cg_run(ctx, reps, as_stream(stream));
}

rbf_status rbf_bench_fma(rbf_ctx* ctx, int prec, int64_t reps, double* flops, void* stream) {
    if (!ctx || !flops) return RBF_ERR_ARG;
    if (prec != RBF_FP64 && prec != RBF_FP32_REFINE) return set_err(ctx, RBF_ERR_ARG, "unknown precision");
    if (reps < 1 || reps > (int64_t(1) << 32)) return set_err(ctx, RBF_ERR_ARG, "reps must be in [1, 2^32]");
    DeviceGuard dg(ctx->device);
    return bench_fma_run(ctx, prec, (long long)reps, flops, as_stream(stream));
}

rbf_status rbf_bench_residual(rbf_ctx* ctx, int reps, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->solved || !ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_residual before rbf_solve");
    if (reps < 0) return set_err(ctx, RBF_ERR_ARG, "reps < 0");
    if (ctx->T > 0 || ctx->poly) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_residual on a batched or polynomial context");
    DeviceGuard dg(ctx->device);
    return bench_residual_run(ctx, reps, as_stream(stream));
}

rbf_status rbf_bench_cg_loop(rbf_ctx* ctx, int reps, void* stream) {
    if (!ctx) return RBF_ERR_ARG;
    if (!ctx->solved || !ctx->assembled) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_cg_loop before rbf_solve");
    if (reps < 1) return set_err(ctx, RBF_ERR_ARG, "reps < 1");
    if (ctx->T > 0) return set_err(ctx, RBF_ERR_ARG, "rbf_bench_cg_loop on a batched context");
    DeviceGuard dg(ctx->device);
    return bench_cg_loop_run(ctx, reps, as_stream(stream));
}

}  // extern "C"
