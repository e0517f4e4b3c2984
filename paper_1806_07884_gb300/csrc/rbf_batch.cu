// Batched tiles: many independent fitting problems of uneven size, each kernel launched once
// for all of them.
//
// Packing. Tile t is moved to its own frame u = (x - x0_t) / R_t, where its support radius
// is 1, and its cells (side kCellMargin in that frame) become one band of rows of a single
// cell grid: band t holds cell rows oy_t .. oy_t + gy_t - 1 and columns 0 .. gx_t - 1, and two
// empty rows separate consecutive bands. Items of different tiles are then never in
// neighbouring cells (3x3 for the rows of A, 5x5 for the blocks of B), so the packed normal
// matrix is block diagonal with one block per tile, each tile's centres are contiguous in
// the cell-sorted order, and the binning, assembly and FP64 residual kernels of the
// single-system path run unchanged over every tile in one launch each. The FP64 coordinates
// kept for those kernels are tile-local, so their rounding is that of one tile whatever the
// packing.
//
// Solve. The CG iteration is the Chronopoulos-Gear iteration of the single-system solver
// with its scalars held per tile: alpha_t, beta_t, the stopping test and the iteration count
// of tile t depend only on tile t's own reductions, so every tile follows the iterates of its
// own CG and stops at its own tolerance. The iteration loop is one CUDA graph (conditional
// WHILE node) that runs until every tile has stopped; each pass of its body first lists the
// work of the tiles still running (SpMV items of consecutive row groups of one tile, update
// items of consecutive rows of one tile), so stopped tiles cost nothing, and the SpMV and update
// kernels are persistent loops over those lists. Per-tile sums: one atomic per item and value
// (the start kernel's segmented sums by tile: warp segmented sums, shared-memory atomics per
// tile, one global atomic per tile and block). FP32 refinement works per tile: own scale, own
// inner tolerance, own FP64 residual norm, stopping test and promotion to FP64.
//
// Launch configuration. The SpMV's blocks per SM, the number of row groups per SpMV item and the
// update kernel's block size are picked by timing candidate configurations on the assembled
// system and cached per system shape (rbf_autotune).
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rbf_cg.cuh"
#include "rbf_evalpairs.cuh"

namespace rbf {
namespace {

// Placement of one tile in the packed grid (device copy of the host descriptor).
struct TileDev {
    long long c0, m, p0, n;    // centre and point ranges of the concatenated inputs
    double x0, y0, R;          // frame: u = (x - x0) / R
    double x1, y1;             // upper corner of the tile's box
    int gx, gy, oy, pad;       // cells per axis, first cell row of the band
};

// Per-tile CG state, double-buffered by iteration parity like the single-system CgSlot.
struct TSlot {
    double gamma_prev, alpha_prev;
    int it, state;
};
struct BatchScal {
    unsigned int ndone;        // tiles that have stopped (or take no part in this solve)
    int T, maxit;
    int passes;                // loop passes of the solve graph so far
    int n_spmv, n_upd;         // items in the current work lists
    unsigned int ndone_built;  // ndone when the work lists were built
    int built;                 // the work lists belong to this solve
};

// Device view of the per-tile arrays (one allocation, layout in TileLayout).
struct TileCg {
    BatchScal* bs;
    TSlot* sl[2];
    double *g[2], *rr[2], *dl[2];   // gamma = (r, u), (r, r) and delta = u^T B u per tile
    double *bb, *tol2, *bscale;     // (b, b) of the scaled right-hand side, tol^2, scale of b
    double* out_rr;                 // (r, r) when the tile stopped
    int *out_it, *out_state;
};

// Byte offsets of the per-tile arrays for T tiles; [0, init_end) is written by the host
// before each solve, [init_end, total) read back after it.
struct TileLayout {
    size_t bs, sl0, sl1, g0, g1, rr0, rr1, dl0, dl1, bb, tol2, bscale, init_end;
    size_t out_rr, out_it, out_state, total;
    explicit TileLayout(int T) {
        size_t o = 0;
        auto take = [&](size_t n) {
            const size_t r = o;
            o += (n + 15) / 16 * 16;
            return r;
        };
        const size_t t = size_t(T);
        bs = take(sizeof(BatchScal));
        sl0 = take(sizeof(TSlot) * t);
        sl1 = take(sizeof(TSlot) * t);
        g0 = take(8 * t);
        g1 = take(8 * t);
        rr0 = take(8 * t);
        rr1 = take(8 * t);
        dl0 = take(8 * t);
        dl1 = take(8 * t);
        bb = take(8 * t);
        tol2 = take(8 * t);
        bscale = take(8 * t);
        init_end = o;
        out_rr = take(8 * t);
        out_it = take(4 * t);
        out_state = take(4 * t);
        total = o;
    }
    TileCg view(char* b) const {
        TileCg v;
        v.bs = reinterpret_cast<BatchScal*>(b + bs);
        v.sl[0] = reinterpret_cast<TSlot*>(b + sl0);
        v.sl[1] = reinterpret_cast<TSlot*>(b + sl1);
        v.g[0] = reinterpret_cast<double*>(b + g0);
        v.g[1] = reinterpret_cast<double*>(b + g1);
        v.rr[0] = reinterpret_cast<double*>(b + rr0);
        v.rr[1] = reinterpret_cast<double*>(b + rr1);
        v.dl[0] = reinterpret_cast<double*>(b + dl0);
        v.dl[1] = reinterpret_cast<double*>(b + dl1);
        v.bb = reinterpret_cast<double*>(b + bb);
        v.tol2 = reinterpret_cast<double*>(b + tol2);
        v.bscale = reinterpret_cast<double*>(b + bscale);
        v.out_rr = reinterpret_cast<double*>(b + out_rr);
        v.out_it = reinterpret_cast<int*>(b + out_it);
        v.out_state = reinterpret_cast<int*>(b + out_state);
        return v;
    }
};

// Per-tile ranges and the CG work lists (twork). A tile's row groups are consecutive in the
// group list and its centres consecutive in the sorted order (bands follow tile order).
// Work items cover one tile each: SpMV items {first, end} of `chunk` row groups, update items
// {first, end} of `nt` rows; .z the tile, .w = 1 on a tile's first update item (the tile's
// owner).
struct TileWork {
    int *clb, *cle;            // [T] tile t's row groups clb[t] .. cle[t]-1
    int *rb, *re;              // [T] tile t's rows (sorted centres) rb[t] .. re[t]-1
    int4* items_s;             // [cap_s] SpMV items
    int4* items_u;             // [cap_u] update items
};
struct WorkLayout {
    size_t clb, cle, rb, re, items_s, items_u, ranges_end, total;
    int cap_s, cap_u;
    // capacities for chunk >= 1 row groups and nt >= 128 rows per item
    WorkLayout(int T, int ngroup, int M) {
        cap_s = ngroup + T;
        cap_u = div_up(M, 128) + T;
        size_t o = 0;
        auto take = [&](size_t n) {
            const size_t r = o;
            o += (n + 15) / 16 * 16;
            return r;
        };
        clb = take(4 * size_t(T));
        cle = take(4 * size_t(T));
        rb = take(4 * size_t(T));
        re = take(4 * size_t(T));
        ranges_end = o;
        items_s = take(sizeof(int4) * size_t(cap_s));
        items_u = take(sizeof(int4) * size_t(cap_u));
        total = o;
    }
    TileWork view(char* b) const {
        TileWork w;
        w.clb = reinterpret_cast<int*>(b + clb);
        w.cle = reinterpret_cast<int*>(b + cle);
        w.rb = reinterpret_cast<int*>(b + rb);
        w.re = reinterpret_cast<int*>(b + re);
        w.items_s = reinterpret_cast<int4*>(b + items_s);
        w.items_u = reinterpret_cast<int4*>(b + items_u);
        return w;
    }
};

// Per-tile reduction area (tred): norms [T] double, a second norm [T], pinned counts [T]
// double, scale [T] double.
struct RedLayout {
    size_t n0, n1, pin, scale, total;
    explicit RedLayout(int T) {
        const size_t t = (size_t(T) * 8 + 15) / 16 * 16;
        n0 = 0;
        n1 = t;
        pin = 2 * t;
        scale = 3 * t;
        total = 4 * t;
    }
};

// ---------------------------------------------------------------------------
// binning of a batch
// ---------------------------------------------------------------------------

__device__ __forceinline__ int tile_cell(double l, double invh, int n) {
    double f = floor(l * invh);
    f = fmin(fmax(f, 0.0), double(n - 1));
    return int(f);
}

// Cell key of every centre (which == 0) or point (which == 1) of tile blockIdx.y, in the
// packed grid: key = (oy_t + iy) * gx + ix with (ix, iy) the cell of (x - x0_t) / R_t.
__global__ void k_tile_count(const TileDev* __restrict__ td, int which, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ h, Grid g,
                             int* __restrict__ count, int* __restrict__ key,
                             int* __restrict__ rank, int* __restrict__ stats) {
    const TileDev t = td[blockIdx.y];
    const long long b = which ? t.p0 : t.c0, n = which ? t.n : t.m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = b + i;
        const double xi = x[k], yi = y[k];
        bool bad = !isfinite(xi) || !isfinite(yi);
        if (h) bad = bad || !isfinite(h[k]);
        if (bad) atomicOr(&stats[2], 1);
        int kk = t.oy * g.gx;
        if (!bad) {
            const double xl = (xi - t.x0) / t.R, yl = (yi - t.y0) / t.R;
            kk = (t.oy + tile_cell(yl, g.invh, t.gy)) * g.gx + tile_cell(xl, g.invh, t.gx);
        }
        key[k] = kk;
        rank[k] = atomicAdd(&count[kk], 1);
    }
}

// Scatter into cell-sorted order with tile-local FP64 coordinates and FP32 coordinates
// local to the item's cell (units of R_t).
__global__ void k_tile_scatter(const TileDev* __restrict__ td, int which,
                               const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ h, Grid g, const int* __restrict__ key,
                               const int* __restrict__ rank, const int* __restrict__ start,
                               double* __restrict__ sx, double* __restrict__ sy,
                               double* __restrict__ sh, float* __restrict__ su,
                               float* __restrict__ sv, int* __restrict__ perm) {
    const TileDev t = td[blockIdx.y];
    const long long b = which ? t.p0 : t.c0, n = which ? t.n : t.m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = b + i;
        const int kk = key[k];
        const int d = start[kk] + rank[k];
        const double xl = (x[k] - t.x0) / t.R, yl = (y[k] - t.y0) / t.R;
        sx[d] = xl;
        sy[d] = yl;
        if (sh) sh[d] = h[k];
        if (perm) perm[d] = int(k);
        const int ix = kk % g.gx, iy = kk / g.gx - t.oy;
        su[d] = float(xl - ix * g.h);
        sv[d] = float(yl - iy * g.h);
    }
}

// Each tile's range in the group list and in the sorted rows, from the ends of its runs.
__global__ void k_tile_ranges(const GroupRec* __restrict__ gdesc, int ngroup,
                              const int4* __restrict__ crow, int M, TileWork tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ngroup) {
        const int t = crow[gdesc[i].d.r0].w;
        if (i == 0 || crow[gdesc[i - 1].d.r0].w != t) tw.clb[t] = i;
        if (i == ngroup - 1 || crow[gdesc[i + 1].d.r0].w != t) tw.cle[t] = i + 1;
    }
    if (i < M) {
        const int t = crow[i].w;
        if (i == 0 || crow[i - 1].w != t) tw.rb[t] = i;
        if (i == M - 1 || crow[i + 1].w != t) tw.re[t] = i + 1;
    }
}

// ---------------------------------------------------------------------------
// segmented (per-tile) reductions
// ---------------------------------------------------------------------------

// Warp segmented sum of NV values keyed by tile: keys are equal over contiguous runs of lanes
// (rows are in tile order). Afterwards the first lane of each run holds the run's sums;
// returns true in those lanes.
template <int NV, typename TV>
__device__ __forceinline__ bool warp_segsum(int key, TV (&v)[NV]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ok = __shfl_down_sync(kFull, key, o);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const TV ov = __shfl_down_sync(kFull, v[k], o);
            if (lane + o < 32 && ok == key) v[k] += ov;
        }
    }
    const int up = __shfl_up_sync(kFull, key, 1);
    return lane == 0 || up != key;
}

// Rows i0 .. i1-1 of one block belong to tiles t0 .. t0+span-1. Adds each thread's NV values
// (key = its row's tile, INT_MAX for none) into dst[k][tile]: warp segmented sums, shared
// atomics per tile, then one global atomic per tile and value. sred: [NV][NT] shared doubles
// zeroed for j < span before the call (with a barrier in between).
template <int NV, int NT, typename TV>
__device__ __forceinline__ void tile_reduce(int key, TV (&v)[NV], int t0, int span,
                                            double (*sred)[NT], double* const (&dst)[NV]) {
    // warp sums in the values' own type (FP32 for the FP32 solver), totals in FP64
    if (warp_segsum<NV, TV>(key, v) && key != INT_MAX) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (v[k] != TV(0)) atomicAdd(&sred[k][key - t0], double(v[k]));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < span; j += NT) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (sred[k][j] != 0.0) atomicAdd(dst[k] + t0 + j, sred[k][j]);
    }
}

// Tiles of the rows of block `blk` (NT rows each): t0 and span.
__device__ __forceinline__ void block_tiles(const Binned& bd, int i0, int i1, int& t0, int& span) {
    t0 = bd.crow[i0].w;
    span = bd.crow[i1 - 1].w - t0 + 1;
}

// Per-tile sum of v_i^2 (v may be null) over rows whose mask is nonzero, and per-tile count
// of rows whose mask is zero (pinned centres), one block per 256 rows.
template <typename TM>
__global__ void __launch_bounds__(256)
    k_tile_norm2(Binned bd, const double* __restrict__ v, const TM* __restrict__ mask,
                 double* __restrict__ out2, double* __restrict__ npin) {
    constexpr int NT = 256;
    __shared__ double sred[2][NT];
    const int i0 = blockIdx.x * NT;
    if (i0 >= bd.M) return;
    const int i1 = min(i0 + NT, bd.M);
    int t0, span;
    block_tiles(bd, i0, i1, t0, span);
    for (int j = threadIdx.x; j < span; j += NT) sred[0][j] = sred[1][j] = 0.0;
    __syncthreads();
    const int i = i0 + threadIdx.x;
    int key = INT_MAX;
    double a[2] = {0.0, 0.0};
    if (i < i1) {
        key = bd.crow[i].w;
        const bool pinned = mask[i] == TM(0);
        if (v && !pinned) a[0] = v[i] * v[i];
        a[1] = pinned ? 1.0 : 0.0;
    }
    double* const dst[2] = {out2, npin};
    tile_reduce<2, NT, double>(key, a, t0, span, sred, dst);
}

// x = x + scale_t d on unpinned rows, x = 0 on pinned rows.
__global__ void k_tile_axpy(Binned bd, double* __restrict__ x, const float* __restrict__ d,
                            const double* __restrict__ scale, const float* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < bd.M) x[i] = dinv[i] == 0.0f ? 0.0 : fma(scale[bd.crow[i].w], double(d[i]), x[i]);
}

__global__ void k_zero_masked(int M, double* __restrict__ x, const float* __restrict__ dinv32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && dinv32[i] == 0.0f) x[i] = 0.0;
}

template <typename T>
__global__ void k_tile_from_sorted(const T* __restrict__ src, const int* __restrict__ perm,
                                   double* __restrict__ dst, int M) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) dst[perm[s]] = double(src[s]);
}
template <typename T>
__global__ void k_copy_masked(int M, const double* __restrict__ src, const T* __restrict__ dinv,
                              T* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) dst[i] = dinv[i] == T(0) ? T(0) : T(src[i]);
}

// f(x) = sum_j c_j phi(||x - xi_j|| / R_t) for a query x of tile t: the centres of the 3x3
// cells around the query's cell in the tile's band, FP32 prefilter on cell-local
// coordinates, exact support test and FP64 evaluation on tile-local coordinates.
template <int KIND>
__device__ __forceinline__ double eval_tile_at(const Binned& bd, const TileDev& t,
                                               const double* __restrict__ c, double x, double y) {
    const Grid& g = bd.g;
    const double xl = (x - t.x0) / t.R, yl = (y - t.y0) / t.R;
    const int ix = tile_cell(xl, g.invh, t.gx), iy = tile_cell(yl, g.invh, t.gy);
    const float uq = float(xl - ix * g.h), vq = float(yl - iy * g.h);
    double f = 0.0;
    for (int r = max(iy - 1, 0); r <= min(iy + 1, t.gy - 1); ++r) {
        const float oy = float(r - iy);
        for (int cx = max(ix - 1, 0); cx <= min(ix + 1, t.gx - 1); ++cx) {
            const float ox = float(cx - ix);
            const int cell = (t.oy + r) * g.gx + cx;
            const int s0 = bd.cstart[cell], s1 = bd.cstart[cell + 1];
            for (int s = s0; s < s1; ++s) {
                const float du = uq - (bd.cu[s] + ox), dv = vq - (bd.cv[s] + oy);
                if (du * du + dv * dv >= kPrefilterR2) continue;
                const double dx = xl - bd.cx[s], dy = yl - bd.cy[s];
                double d2;
                if (inside_exact_d2(dx, dy, 1.0, 1.0, d2)) {
                    const double rr = sqrt_fast(d2);
                    f = fma(c[s], wendland<KIND, double>(rr), f);
                }
            }
        }
    }
    return f;
}

// A query at (x, y) located in tile t's frame for the pair-stream evaluation engine: the frame
// coordinates (x - x0_t) / R_t, the packed cell and the FP32 cell-frame coordinates.
__device__ __forceinline__ EvalQuery tile_query(const Binned& bd, const TileDev& t, double x,
                                                double y, bool valid) {
    EvalQuery q;
    q.valid = valid;
    q.x = q.y = 0.0;
    q.ix = q.iy = 0;
    q.uq = q.vq = 0.0f;
    if (valid) {
        const double xl = (x - t.x0) / t.R, yl = (y - t.y0) / t.R;
        const int cx = tile_cell(xl, bd.g.invh, t.gx), cy = tile_cell(yl, bd.g.invh, t.gy);
        q.x = xl;
        q.y = yl;
        q.ix = cx;
        q.iy = t.oy + cy;
        q.uq = float(xl - cx * bd.g.h);
        q.vq = float(yl - cy * bd.g.h);
    }
    return q;
}
// Tile t's frame: R = 1 in its coordinates, the cells of its band of the packed grid.
__device__ __forceinline__ EvalFrame tile_frame(const TileDev& t) {
    return EvalFrame{1.0, 1.0, 1.0, 0, t.gx - 1, t.oy, t.oy + t.gy - 1};
}

constexpr int kTileEvalWarps = 8;

// Queries of tile blockIdx.y: [qoff[t], qoff[t+1]) of qx, qy, f; a warp per 32 of them.
template <int KIND>
__global__ void __launch_bounds__(kTileEvalWarps * 32)
k_eval_tiles(Binned bd, const TileDev* __restrict__ td, const double* __restrict__ c,
             const double* __restrict__ qx, const double* __restrict__ qy,
             const long long* __restrict__ qoff, double* __restrict__ f) {
    __shared__ EvalWarpSmem sm[kTileEvalWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const TileDev t = td[blockIdx.y];
    const EvalFrame fr = tile_frame(t);
    const long long q0 = qoff[blockIdx.y], q1 = qoff[blockIdx.y + 1];
    for (long long g0 = q0 + (blockIdx.x * (long long)kTileEvalWarps + wp) * 32; g0 < q1;
         g0 += (long long)gridDim.x * kTileEvalWarps * 32) {
        const long long q = g0 + lane;
        const bool valid = q < q1;
        const EvalQuery e = tile_query(bd, t, valid ? qx[q] : 0.0, valid ? qy[q] : 0.0, valid);
        const double v = eval_pairs32<KIND>(bd, c, e, fr, lane, sm[wp]);
        if (valid) f[q] = v;
    }
}

// The nx x ny node grid over each tile's own box (inclusive linspace, last node exactly at the
// box's end), tile t's values at f[t nx ny + i nx + j]; a warp per 32 nodes.
template <int KIND>
__global__ void __launch_bounds__(kTileEvalWarps * 32)
k_eval_tiles_grid(Binned bd, const TileDev* __restrict__ td, const double* __restrict__ c,
                  int nx, int ny, double* __restrict__ f) {
    __shared__ EvalWarpSmem sm[kTileEvalWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const TileDev t = td[blockIdx.y];
    const EvalFrame fr = tile_frame(t);
    const long long Q = (long long)nx * ny;
    const double sx = nx > 1 ? (t.x1 - t.x0) / (nx - 1) : 0.0;
    const double sy = ny > 1 ? (t.y1 - t.y0) / (ny - 1) : 0.0;
    double* ft = f + (long long)blockIdx.y * Q;
    for (long long g0 = (blockIdx.x * (long long)kTileEvalWarps + wp) * 32; g0 < Q;
         g0 += (long long)gridDim.x * kTileEvalWarps * 32) {
        const long long q = g0 + lane;
        const bool valid = q < Q;
        double x = 0.0, y = 0.0;
        if (valid) {
            const int i = int(q / nx), j = int(q % nx);
            x = (j == nx - 1 && nx > 1) ? t.x1 : __dadd_rn(__dmul_rn(double(j), sx), t.x0);
            y = (i == ny - 1 && ny > 1) ? t.y1 : __dadd_rn(__dmul_rn(double(i), sy), t.y0);
        }
        const double v = eval_pairs32<KIND>(bd, c, tile_query(bd, t, x, y, valid), fr, lane, sm[wp]);
        if (valid) ft[q] = v;
    }
}

// ---------------------------------------------------------------------------
// batched CG kernels
// ---------------------------------------------------------------------------

// Work lists for the tiles running at the start of a solve-graph body (slot 0, on which every
// body starts): tile order, each tile's SpMV items then its update items at offsets from
// block-wide scans over the tiles, written by whole warps. Kept when no tile has stopped
// since the last build. One block; tiles in rounds of kWlThreads.
constexpr int kWlThreads = 1024;
__global__ void __launch_bounds__(kWlThreads)
    k_bcg_worklist(TileCg tc, TileWork tw, int ntile, int chunk, int nt) {
    __shared__ int s_skip, s_base_s, s_base_u, s_tot_s, s_tot_u;
    __shared__ int s_ws[kWlThreads / 32], s_wu[kWlThreads / 32];
    BatchScal* bs = tc.bs;
    const unsigned int nd = bs->ndone;
    if (threadIdx.x == 0) {
        s_skip = bs->built && bs->ndone_built == nd;
        s_base_s = 0;
        s_base_u = 0;
    }
    __syncthreads();
    if (s_skip) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int base = 0; base < ntile; base += kWlThreads) {
        const int t = base + threadIdx.x;
        int ns = 0, nu = 0, c0 = 0, c1 = 0, r0 = 0, r1 = 0;
        if (t < ntile && tc.sl[0][t].state == kRunning) {
            c0 = tw.clb[t];
            c1 = tw.cle[t];
            r0 = tw.rb[t];
            r1 = tw.re[t];
            ns = (c1 - c0 + chunk - 1) / chunk;
            nu = (r1 - r0 + nt - 1) / nt;
        }
        int is = ns, iu = nu;   // inclusive scans within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int xs = __shfl_up_sync(kFull, is, o), xu = __shfl_up_sync(kFull, iu, o);
            if (lane >= o) {
                is += xs;
                iu += xu;
            }
        }
        if (lane == 31) {
            s_ws[wp] = is;
            s_wu[wp] = iu;
        }
        __syncthreads();
        if (wp == 0) {
            const int a0 = s_ws[lane], b0 = s_wu[lane];
            int a = a0, b = b0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int xa = __shfl_up_sync(kFull, a, o), xb = __shfl_up_sync(kFull, b, o);
                if (lane >= o) {
                    a += xa;
                    b += xb;
                }
            }
            s_ws[lane] = a - a0;
            s_wu[lane] = b - b0;
            if (lane == 31) {
                s_tot_s = a;
                s_tot_u = b;
            }
        }
        __syncthreads();
        const int os = s_base_s + s_ws[wp] + is - ns, ou = s_base_u + s_wu[wp] + iu - nu;
        // the warp writes its 32 tiles' items one tile at a time, lanes over the items
        for (int l = 0; l < 32; ++l) {
            const int tl = __shfl_sync(kFull, t, l);
            const int nsl = __shfl_sync(kFull, ns, l), osl = __shfl_sync(kFull, os, l);
            const int nul = __shfl_sync(kFull, nu, l), oul = __shfl_sync(kFull, ou, l);
            const int c0l = __shfl_sync(kFull, c0, l), c1l = __shfl_sync(kFull, c1, l);
            const int r0l = __shfl_sync(kFull, r0, l), r1l = __shfl_sync(kFull, r1, l);
            for (int j = lane; j < nsl; j += 32) {
                const int a = c0l + j * chunk;
                tw.items_s[osl + j] = make_int4(a, min(a + chunk, c1l), tl, 0);
            }
            for (int j = lane; j < nul; j += 32) {
                const int a = r0l + j * nt;
                tw.items_u[oul + j] = make_int4(a, min(a + nt, r1l), tl, j == 0 ? 1 : 0);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base_s += s_tot_s;
            s_base_u += s_tot_u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bs->n_spmv = s_base_s;
        bs->n_upd = s_base_u;
        bs->ndone_built = nd;
        bs->built = 1;
    }
}

// w += B u over the SpMV items of the running tiles; delta_t = u^T B u per tile (one atomic
// per item). Persistent warps stride over the items (runs of row groups of one tile), the next
// group's descriptor moving into L1 while the current group streams. A tile that stops inside
// a graph body keeps its items until the next body (at most kItersPerBody - 1 SpMVs whose w
// and delta its stopped state leaves unused). Also zeroes the per-tile sums the next update
// kernel accumulates (parity P ^ 1).
template <typename T>
__global__ void __launch_bounds__(kSpmvWarps * 32, sizeof(T) == 4 ? 3 : 2)
    k_bcg_spmv(Binned bd, const int4* __restrict__ items, const T* __restrict__ B,
               const T* __restrict__ u, T* __restrict__ w, int P, int ntile, TileCg tc) {
    __shared__ GroupSmem gsm[kSpmvWarps];
    // parity selection by value (indexing the parameter's arrays with P would copy them to
    // local memory)
    double* __restrict__ gQ = P ? tc.g[0] : tc.g[1];
    double* __restrict__ rrQ = P ? tc.rr[0] : tc.rr[1];
    double* __restrict__ dlP = P ? tc.dl[1] : tc.dl[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntile; t += gridDim.x * blockDim.x) {
        gQ[t] = 0.0;
        rrQ[t] = 0.0;
    }
    const int n = tc.bs->n_spmv;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = gridDim.x * kSpmvWarps;
    int q = blockIdx.x * kSpmvWarps + wid;
    if (q >= n) return;
    int4 it = items[q];
    // the next group's record is loaded while this group's rows stream: this item's next
    // group, else the next item's first
    stage_group(bd.gdesc, it.x, gsm[wid], 0, lane);
    int b = 0;
    for (; q < n; q += nw) {
        const int4 next = q + nw < n ? items[q + nw] : make_int4(0, 0, 0, 0);
        T acc = T(0);   // this lane's share of the item's delta (warp sum in T)
        for (int g = it.x; g < it.y; ++g, b ^= 1) {
            const int gn = g + 1 < it.y ? g + 1 : (q + nw < n ? next.x : -1);
            if (gn >= 0) {
                stage_group(bd.gdesc, gn, gsm[wid], b ^ 1, lane);
                group_wait<1>();
            } else {
                group_wait<0>();
            }
            acc += spmv_group<T>(b, B, u, w, bd.M, lane, gsm[wid]);
        }
        const T sum = warp_sum<T>(acc);
        if (lane == 0 && sum != T(0)) atomicAdd(&dlP[it.z], double(sum));
        it = next;
    }
}

// Persistent blocks stride over the update items (NT rows of one tile each). Per item:
// the row values are loaded first, then thread 0 takes tile t's step (alpha_t, beta_t and
// the stopping test from the tile's sums, in the solver's precision T; the same values in
// every item of the tile); the owner item also writes the tile's next slot, clears its delta
// sum of the other parity and, when the tile stops, records its result, counts it done and
// marks the stop in both slots (another item reading the slot meanwhile takes the same
// decision from the same sums). Body as the single-system update; per-tile sums of gamma and
// (r, r) for the next iteration, one atomic per item.
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
    k_bcg_update(Binned bd, CgVec<T> v, const int4* __restrict__ items, int P, TileCg tc) {
    __shared__ T s_ab[2];
    __shared__ int s_go;
    // new residuals of the item's rows, for the block-Jacobi step (rows of a cell outside the
    // item are recomputed with the same operations)
    __shared__ T rsm[NT];
    TSlot* slP = P ? tc.sl[1] : tc.sl[0];
    TSlot* slQ = P ? tc.sl[0] : tc.sl[1];
    const double* __restrict__ gP = P ? tc.g[1] : tc.g[0];
    const double* __restrict__ rrP = P ? tc.rr[1] : tc.rr[0];
    const double* __restrict__ dlP = P ? tc.dl[1] : tc.dl[0];
    double* __restrict__ gQ = P ? tc.g[0] : tc.g[1];
    double* __restrict__ rrQ = P ? tc.rr[0] : tc.rr[1];
    double* __restrict__ dlQ = P ? tc.dl[0] : tc.dl[1];
    const T* __restrict__ rP = P ? v.r[1] : v.r[0];
    const T* __restrict__ sP = P ? v.s[1] : v.s[0];
    const T* __restrict__ wP = P ? v.w[1] : v.w[0];
    T* __restrict__ rQ = P ? v.r[0] : v.r[1];
    T* __restrict__ sQ = P ? v.s[0] : v.s[1];
    T* __restrict__ wQ = P ? v.w[0] : v.w[1];
    const int n = tc.bs->n_upd;
    const int maxit = tc.bs->maxit;
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        const int4 item = items[b];
        const int r0 = item.x, r1 = item.y, t = item.z;
        const int i = r0 + threadIdx.x;
        const bool valid = i < r1;
        // the row's values, loaded before the tile's step so that their latency overlaps it
        int4 cm = make_int4(0, 0, 0, 0);
        T f_d = T(0), f_w = T(0), f_s = T(0), f_p = T(0), f_u = T(0), f_r = T(0), f_x = T(0);
        if (valid) {
            cm = bd.crow[i];
            f_d = v.dinv[i];
            f_w = wP[i];
            f_s = sP[i];
            f_p = v.p[i];
            f_u = v.u[i];
            f_r = rP[i];
            f_x = v.x[i];
        }
        if (threadIdx.x == 0) {
            const TSlot sl = slP[t];
            const T g = T(__ldcg(gP + t)), rr = T(__ldcg(rrP + t)), d = T(__ldcg(dlP + t));
            const T tol2 = T(tc.tol2[t]), bb = T(__ldcg(tc.bb + t));
            int state = sl.state;
            T alpha = T(0), beta = T(0);
            if (state == kRunning) {
                if (!isfinite(g) || !isfinite(rr)) {
                    state = kBreakdown;
                } else if (rr <= tol2 * bb) {
                    state = kConverged;
                } else if (sl.it >= maxit) {
                    state = kMaxIt;
                } else {
                    beta = sl.it == 0 ? T(0) : g / T(sl.gamma_prev);
                    const T den = sl.it == 0 ? d : d - beta * g / T(sl.alpha_prev);
                    alpha = g / den;
                    if (!(den > T(0)) || !isfinite(alpha)) state = kBreakdown;
                }
            }
            if (item.w) {
                TSlot nx = sl;
                nx.state = state;
                if (state == kRunning) {
                    nx.gamma_prev = double(g);
                    nx.alpha_prev = double(alpha);
                    nx.it = sl.it + 1;
                }
                slQ[t] = nx;
                dlQ[t] = 0.0;
                if (sl.state == kRunning && state != kRunning) {
                    slP[t] = nx;
                    tc.out_rr[t] = double(rr);
                    tc.out_it[t] = sl.it;
                    tc.out_state[t] = state;
                    atomicAdd(&tc.bs->ndone, 1u);
                }
            }
            s_ab[0] = alpha;
            s_ab[1] = beta;
            s_go = state == kRunning;
        }
        __syncthreads();
        if (s_go) {   // uniform over the block
            const T ta = s_ab[0], tb = s_ab[1];
            T di = T(0), ri = T(0);
            if (valid) {
                di = f_d;
                const T wi = di == T(0) ? T(0) : f_w;
                const T si = fma(tb, f_s, wi);
                const T pi = fma(tb, f_p, f_u);
                ri = di == T(0) ? T(0) : fma(-ta, si, f_r);
                sQ[i] = si;
                v.p[i] = pi;
                v.x[i] = fma(ta, pi, f_x);
                rQ[i] = ri;
                wQ[i] = T(0);
            }
            rsm[threadIdx.x] = ri;
            __syncthreads();
            T acc[2] = {T(0), T(0)};
            if (valid) {
                const T ui = apply_prec<T>(bd, v.bjinv, cm, i, di, ri, [&](int jj) {
                    const int o = jj - r0;
                    return o >= 0 && o < NT ? rsm[o] : next_r(rP[jj], sP[jj], wP[jj], ta, tb);
                });
                v.u[i] = ui;
                acc[0] = ri * ui;
                acc[1] = ri * ri;
            }
            double tot[2];
            block_sum_t<2, T>(acc, tot);
            if (threadIdx.x == 0) {
                if (tot[0] != 0.0) atomicAdd(gQ + t, tot[0]);
                if (tot[1] != 0.0) atomicAdd(rrQ + t, tot[1]);
            }
        }
        __syncthreads();   // s_ab, s_go and rsm are the next item's
    }
}

// Start of a batched solve of B x = bscale_t b per tile (tiles with bscale_t = 0 take no
// part: their rows get r = u = 0 and keep x when use_x0, else x = 0):
// r = bscale_t b - B x0 (B x0 in w[1] when use_x0), u = D^-1 r, p = s[0] = w[0] = 0;
// per-tile gamma_0, (r_0, r_0) and (b, b).
template <typename T, typename TB>
__global__ void __launch_bounds__(256)
    k_bcg_init(Binned bd, CgVec<T> v, const TB* __restrict__ b, int use_x0, TileCg tc) {
    constexpr int NT = 256;
    __shared__ double sred[3][NT];
    const int i0 = blockIdx.x * NT;
    if (i0 >= bd.M) return;
    const int i1 = min(i0 + NT, bd.M);
    int t0, span;
    block_tiles(bd, i0, i1, t0, span);
    for (int j = threadIdx.x; j < span; j += NT) sred[0][j] = sred[1][j] = sred[2][j] = 0.0;
    __syncthreads();
    const int i = i0 + threadIdx.x;
    int key = INT_MAX;
    double acc[3] = {0.0, 0.0, 0.0};
    if (i < i1) {
        const int4 cm = bd.crow[i];
        key = cm.w;
        const double bs = tc.bscale[cm.w];
        const T* __restrict__ w1 = v.w[1];
        auto r0 = [&](int j) -> T {
            const T bj = T(double(b[j]) * bs);
            return use_x0 ? bj - w1[j] : bj;
        };
        const T di = v.dinv[i];
        const bool act = bs != 0.0;
        const T bi = act && di != T(0) ? T(double(b[i]) * bs) : T(0);
        const T ri = act && di != T(0) ? r0(i) : T(0);
        const T ui = act ? apply_prec<T>(bd, v.bjinv, cm, i, di, ri, r0) : T(0);
        if (!use_x0) v.x[i] = T(0);
        v.r[0][i] = ri;
        v.u[i] = ui;
        v.p[i] = T(0);
        v.s[0][i] = T(0);
        v.w[0][i] = T(0);
        acc[0] = double(ri) * double(ui);
        acc[1] = double(ri) * double(ri);
        acc[2] = double(bi) * double(bi);
    }
    double* const dst[3] = {tc.g[0], tc.rr[0], tc.bb};
    tile_reduce<3, NT, double>(key, acc, t0, span, sred, dst);
}

__global__ void k_bcg_cond(BatchScal* __restrict__ bs, cudaGraphConditionalHandle h) {
    // every running tile stops by maxit; the pass bound ends the loop whatever the states
    const int passes = ++bs->passes;
    const bool more = bs->ndone < unsigned(bs->T) && passes <= bs->maxit / kItersPerBody + 2;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct Cfg {
    int bps, chunk, nt;
};

template <typename T>
int spmv_occupancy() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bcg_spmv<T>, kSpmvWarps * 32, 0);
    return std::max(1, a);
}

int sm_count(const rbf_ctx* ctx) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    return std::max(1, sms);
}

TileCg tile_view(rbf_ctx* ctx) { return TileLayout(ctx->T).view(ctx->tcg.as<char>()); }
WorkLayout work_layout(const rbf_ctx* ctx) { return WorkLayout(ctx->T, ctx->ngroup, ctx->M); }
TileWork work_view(rbf_ctx* ctx) { return work_layout(ctx).view(ctx->twork.as<char>()); }

// Persistent update grid: as many blocks of NT threads as can be resident, at most one per
// item of the longest list.
template <typename T>
int update_grid(rbf_ctx* ctx, int nt) {
    int a = 0;
    switch (nt) {
        case 128: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bcg_update<T, 128>, 128, 0); break;
        case 512: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bcg_update<T, 512>, 512, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bcg_update<T, 256>, 256, 0); break;
    }
    const WorkLayout L = work_layout(ctx);
    return std::max(1, std::min(std::max(a, 1) * sm_count(ctx), L.cap_u));
}

void launch_worklist(rbf_ctx* ctx, const TileCg& tc, const Cfg& cf, cudaStream_t cs) {
    k_bcg_worklist<<<1, kWlThreads, 0, cs>>>(tc, work_view(ctx), ctx->T, cf.chunk, cf.nt);
}

// One batched CG iteration (two kernels) reading the buffers of parity P.
template <typename T>
void launch_bcg_iteration(rbf_ctx* ctx, const CgVec<T>& v, const TileCg& tc, const Cfg& cf,
                          int P, cudaStream_t cs) {
    const Binned bd = view(ctx);
    const TileWork tw = work_view(ctx);
    const int items = div_up(ctx->ngroup, cf.chunk) + ctx->T;   // most SpMV items
    const int grid = std::max(1, std::min(cf.bps * sm_count(ctx), div_up(items, kSpmvWarps)));
    k_bcg_spmv<T><<<grid, kSpmvWarps * 32, 0, cs>>>(bd, tw.items_s, bvals_dev<T>(ctx), v.u,
                                                    v.w[P], P, ctx->T, tc);
    const int nb = update_grid<T>(ctx, cf.nt);
    switch (cf.nt) {
        case 128: k_bcg_update<T, 128><<<nb, 128, 0, cs>>>(bd, v, tw.items_u, P, tc); break;
        case 512: k_bcg_update<T, 512><<<nb, 512, 0, cs>>>(bd, v, tw.items_u, P, tc); break;
        default: k_bcg_update<T, 256><<<nb, 256, 0, cs>>>(bd, v, tw.items_u, P, tc); break;
    }
}

// Write the per-tile start state: tiles with active[t] run with scale bscale[t] and
// tolerance tol[t]; the others are counted done.
rbf_status write_tile_state(rbf_ctx* ctx, const std::vector<char>& active,
                            const std::vector<double>& bscale, const std::vector<double>& tol,
                            int maxit, cudaStream_t st) {
    const int T = ctx->T;
    const TileLayout L(T);
    char* h = static_cast<char*>(ctx->hbt);
    memset(h, 0, L.total);
    TileCg hv = L.view(h);
    unsigned int inactive = 0;
    for (int t = 0; t < T; ++t) {
        TSlot s;
        s.gamma_prev = 1.0;
        s.alpha_prev = 1.0;
        s.it = 0;
        s.state = active[t] ? kRunning : kInactive;
        hv.sl[0][t] = s;
        hv.sl[1][t] = s;
        hv.tol2[t] = tol[t] * tol[t];
        hv.bscale[t] = active[t] ? bscale[t] : 0.0;
        hv.out_state[t] = s.state;
        inactive += active[t] ? 0u : 1u;
    }
    hv.bs->ndone = inactive;
    hv.bs->T = T;
    hv.bs->maxit = maxit;
    RBF_CUDA_TRY(cudaMemcpyAsync(ctx->tcg.p, h, L.total, cudaMemcpyHostToDevice, st));
    return RBF_OK;
}

template <typename T, typename TB>
rbf_status bcg_start(rbf_ctx* ctx, const TB* b, bool use_x0, const Cfg& cf, cudaStream_t st) {
    const Binned bd = view(ctx);
    const CgVec<T> v = cg_vectors<T>(ctx);
    if (use_x0) {
        RBF_CUDA_TRY(cudaMemsetAsync(v.w[1], 0, sizeof(T) * ctx->M, st));
        launch_spmv(ctx, sizeof(T) == 8 ? RBF_FP64 : RBF_FP32_REFINE, v.x, v.w[1], st);
    }
    k_bcg_init<T, TB><<<std::max(1, div_up(ctx->M, 256)), 256, 0, st>>>(bd, v, b, use_x0 ? 1 : 0,
                                                                       tile_view(ctx));
    launch_worklist(ctx, tile_view(ctx), cf, st);   // for iterations launched one by one
    ctx->launches += 2;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

Cfg default_cfg(rbf_ctx* ctx, int slot) {
    Cfg c;
    c.bps = ctx->force_bps ? ctx->force_bps
                           : (slot == 0 ? spmv_occupancy<double>() : spmv_occupancy<float>());
    c.chunk = ctx->force_chunk ? ctx->force_chunk : 4;
    c.nt = ctx->force_nt ? ctx->force_nt : 256;
    return c;
}

// Time `iters` batched iterations in configuration cf from a fresh start (all tiles running,
// never converging), after two warm-up iterations.
template <typename T>
rbf_status time_cfg(rbf_ctx* ctx, const Cfg& cf, int iters, cudaEvent_t e0, cudaEvent_t e1,
                    double* us, cudaStream_t st) {
    const int T_ = ctx->T;
    std::vector<char> act(T_, 1);
    std::vector<double> one(T_, 1.0), zero(T_, 0.0);
    rbf_status s = write_tile_state(ctx, act, one, zero, 1 << 30, st);
    if (s != RBF_OK) return s;
    if ((s = bcg_start<T, double>(ctx, ctx->bvec.as<double>(), false, cf, st)) != RBF_OK) return s;
    const CgVec<T> v = cg_vectors<T>(ctx);
    const TileCg tc = tile_view(ctx);
    launch_bcg_iteration<T>(ctx, v, tc, cf, 0, st);
    launch_bcg_iteration<T>(ctx, v, tc, cf, 1, st);
    RBF_CUDA_TRY(cudaEventRecord(e0, st));
    for (int k = 0; k < iters; ++k) launch_bcg_iteration<T>(ctx, v, tc, cf, k & 1, st);
    RBF_CUDA_TRY(cudaEventRecord(e1, st));
    RBF_CUDA_TRY(cudaEventSynchronize(e1));
    RBF_CUDA_TRY(cudaGetLastError());
    float ms = 0.0f;
    RBF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *us = 1000.0 * ms / iters;
    ctx->launches += 2 * int64_t(iters + 2);
    return RBF_OK;
}

// The autotuner: SpMV blocks per SM x cells per SpMV item (update block size 256), then the
// update block size for the best SpMV choice; 8 timed iterations per candidate.
template <typename T>
rbf_status autotune_impl(rbf_ctx* ctx, cudaStream_t st) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RBF_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    const int occ = spmv_occupancy<T>();
    const int chunks[] = {1, 2, 4, 8, 16};
    const int nts[] = {128, 256, 512};
    Cfg best{occ, 4, 256};
    double best_us = 1e300;
    rbf_status s = RBF_OK;
    for (int bps = 1; bps <= occ && s == RBF_OK; ++bps)
        for (int ch : chunks) {
            const Cfg cf{bps, ch, 256};
            double us = 0.0;
            if ((s = time_cfg<T>(ctx, cf, 8, e0, e1, &us, st)) != RBF_OK) break;
            if (us < best_us) {
                best_us = us;
                best = cf;
            }
        }
    for (int nt : nts) {
        if (s != RBF_OK || nt == 256) continue;
        const Cfg cf{best.bps, best.chunk, nt};
        double us = 0.0;
        if ((s = time_cfg<T>(ctx, cf, 8, e0, e1, &us, st)) != RBF_OK) break;
        if (us < best_us) {
            best_us = us;
            best = cf;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != RBF_OK) return s;
    rbf_ctx::TileTuning& tu = ctx->tune[slot];
    tu.spmv_bps = best.bps;
    tu.chunk = best.chunk;
    tu.nt = best.nt;
    tu.us_per_iter = best_us;
    tu.ngroup = ctx->ngroup;
    tu.M = ctx->M;
    tu.nvals = ctx->nvals;
    return RBF_OK;
}

// Configuration for this system: forced values, else the tuned one for this shape (tuning
// now when enabled), else the default.
template <typename T>
rbf_status pick_cfg(rbf_ctx* ctx, Cfg* out, cudaStream_t st) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    const rbf_ctx::TileTuning& tu = ctx->tune[slot];
    const bool fresh = tu.nt != 0 && tu.ngroup == ctx->ngroup && tu.M == ctx->M && tu.nvals == ctx->nvals;
    if (!fresh && ctx->autotune && !ctx->no_tune_now &&
        !(ctx->force_bps || ctx->force_chunk || ctx->force_nt)) {
        rbf_status s = autotune_impl<T>(ctx, st);
        if (s != RBF_OK) return s;
    }
    Cfg c = default_cfg(ctx, slot);
    if (ctx->tune[slot].nt != 0 && ctx->tune[slot].ngroup == ctx->ngroup && ctx->tune[slot].M == ctx->M &&
        ctx->tune[slot].nvals == ctx->nvals) {
        if (!ctx->force_bps) c.bps = ctx->tune[slot].spmv_bps;
        if (!ctx->force_chunk) c.chunk = ctx->tune[slot].chunk;
        if (!ctx->force_nt) c.nt = ctx->tune[slot].nt;
    }
    *out = c;
    return RBF_OK;
}

// The batched solve graph: a conditional WHILE node whose body runs kItersPerBody
// iterations and then continues while some tile is still running.
template <typename T>
rbf_status bcg_graph(rbf_ctx* ctx, const Cfg& cf, cudaGraphExec_t* out) {
    rbf_ctx::TileGraph& sg = ctx->bt_graph[sizeof(T) == 8 ? 0 : 1];
    const CgVec<T> v = cg_vectors<T>(ctx);
    const void* key[13] = {ctx->twork.p, bvals_dev<void>(ctx), v.x, v.dinv, v.bjinv, ctx->tcg.p, ctx->gdesc.p,
                           ctx->rmeta.p, ctx->crow.p, ctx->bjoff.p, ctx->cstart.p, nullptr,
                           nullptr};
    bool hit = sg.exec && sg.T == ctx->T && sg.M == ctx->M && sg.ngroup == ctx->ngroup &&
               sg.bps == cf.bps && sg.chunk == cf.chunk && sg.nt == cf.nt;
    for (int k = 0; k < 13 && hit; ++k) hit = sg.key[k] == key[k];
    if (hit) {
        *out = sg.exec;
        return RBF_OK;
    }
    if (sg.exec) {
        cudaGraphExecDestroy(sg.exec);
        sg.exec = nullptr;
    }
    if (!ctx->capture_stream)
        RBF_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    RBF_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
    cudaStream_t cs = ctx->capture_stream;
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const TileCg tc = tile_view(ctx);
        launch_worklist(ctx, tc, cf, cs);   // kept unless some tile stopped
        for (int k = 0; k < kItersPerBody; ++k) launch_bcg_iteration<T>(ctx, v, tc, cf, k & 1, cs);
        k_bcg_cond<<<1, 1, 0, cs>>>(tc.bs, handle);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cs, &captured);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        sg.exec = nullptr;
        return cuda_fail(ctx, e, "building the batched CG solve graph", __FILE__, __LINE__);
    }
    sg.T = ctx->T;
    sg.M = ctx->M;
    sg.ngroup = ctx->ngroup;
    sg.bps = cf.bps;
    sg.chunk = cf.chunk;
    sg.nt = cf.nt;
    for (int k = 0; k < 13; ++k) sg.key[k] = key[k];
    *out = sg.exec;
    return RBF_OK;
}

// Results of one batched CG run, per tile.
struct BcgOut {
    std::vector<int> it, state;
    std::vector<double> rel;
};

// Batched CG on B (precision T) for B x_t = bscale_t b_t on the active tiles, from x0
// (sorted order, FP64; null for x = 0). Every row of x0 is copied in, so tiles that take no
// part keep the iterate x0 gives them. The copy follows the configuration choice: the
// autotuner times its iterations on the solver's own vectors.
template <typename T, typename TB>
rbf_status run_bcg(rbf_ctx* ctx, const TB* b, const double* x0, const std::vector<char>& active,
                   const std::vector<double>& bscale, const std::vector<double>& tol, int maxit,
                   BcgOut* out, cudaStream_t st) {
    rbf_status s;
    Cfg cf;
    if ((s = pick_cfg<T>(ctx, &cf, st)) != RBF_OK) return s;
    cudaGraphExec_t ex;
    if ((s = bcg_graph<T>(ctx, cf, &ex)) != RBF_OK) return s;
    if ((s = write_tile_state(ctx, active, bscale, tol, maxit, st)) != RBF_OK) return s;
    if (x0) {
        const CgVec<T> v = cg_vectors<T>(ctx);
        k_copy_masked<T><<<std::max(1, div_up(ctx->M, 256)), 256, 0, st>>>(ctx->M, x0, v.dinv, v.x);
        ctx->launches += 1;
    }
    if ((s = bcg_start<T, TB>(ctx, b, x0 != nullptr, cf, st)) != RBF_OK) return s;
    RBF_CUDA_TRY(cudaGraphLaunch(ex, st));
    const TileLayout L(ctx->T);
    char* h = static_cast<char*>(ctx->hbt);
    RBF_CUDA_TRY(cudaMemcpyAsync(h, ctx->tcg.p, L.total, cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    const TileCg hv = L.view(h);
    const int T_ = ctx->T;
    out->it.assign(T_, 0);
    out->state.assign(T_, kInactive);
    out->rel.assign(T_, 0.0);
    int max_it = 0;
    for (int t = 0; t < T_; ++t) {
        if (!active[t]) continue;
        out->it[t] = hv.out_it[t];
        out->state[t] = hv.out_state[t];
        out->rel[t] = hv.bb[t] > 0.0 ? sqrt(hv.out_rr[t] / hv.bb[t]) : 0.0;
        max_it = std::max(max_it, hv.out_it[t]);
    }
    ctx->launches += int64_t(max_it / kItersPerBody + 1) * (2 * kItersPerBody + 2);
    return RBF_OK;
}

// Per-tile ||v||^2 over unpinned rows (mask = FP32 or FP64 dinv) into host vector n2, and,
// when npin is not null, per-tile pinned counts.
template <typename TM>
rbf_status tile_norms(rbf_ctx* ctx, const double* v, const TM* mask, std::vector<double>* n2,
                      std::vector<int64_t>* npin, cudaStream_t st) {
    const int T = ctx->T;
    const RedLayout R(T);
    char* d = ctx->tred.as<char>();
    RBF_CUDA_TRY(cudaMemsetAsync(d, 0, R.scale, st));
    k_tile_norm2<TM><<<std::max(1, div_up(ctx->M, 256)), 256, 0, st>>>(
        view(ctx), v, mask, reinterpret_cast<double*>(d + R.n0), reinterpret_cast<double*>(d + R.pin));
    ctx->launches += 1;
    char* h = static_cast<char*>(ctx->hbt);
    RBF_CUDA_TRY(cudaMemcpyAsync(h, d, R.scale, cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    const double* hn = reinterpret_cast<const double*>(h + R.n0);
    const double* hp = reinterpret_cast<const double*>(h + R.pin);
    if (n2) n2->assign(hn, hn + T);
    if (npin) {
        npin->resize(T);
        for (int t = 0; t < T; ++t) (*npin)[t] = int64_t(llround(hp[t]));
    }
    return RBF_OK;
}

rbf_status status_of(int state) {
    if (state == kConverged) return RBF_OK;
    if (state == kBreakdown) return RBF_ERR_BREAKDOWN;
    return RBF_ERR_NOT_CONVERGED;
}

}  // namespace

// ---- binning hooks called by bin_run ----

rbf_status tiles_count(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                       const double* py, const double* h, cudaStream_t st) {
    const dim3 grid(8, ctx->T);
    const TileDev* td = ctx->tdesc.as<TileDev>();
    int* stats = ctx->stats.as<int>();
    k_tile_count<<<grid, 256, 0, st>>>(td, 0, cx, cy, nullptr, ctx->g, ctx->ccount.as<int>(),
                                       ctx->ckey.as<int>(), ctx->crank.as<int>(), stats);
    k_tile_count<<<grid, 256, 0, st>>>(td, 1, px, py, h, ctx->g, ctx->pcount.as<int>(),
                                       ctx->pkey.as<int>(), ctx->prank.as<int>(), stats);
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status tiles_scatter(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                         const double* py, const double* h, cudaStream_t st) {
    const dim3 grid(8, ctx->T);
    const TileDev* td = ctx->tdesc.as<TileDev>();
    k_tile_scatter<<<grid, 256, 0, st>>>(td, 0, cx, cy, nullptr, ctx->g, ctx->ckey.as<int>(),
                                         ctx->crank.as<int>(), ctx->cstart.as<int>(),
                                         ctx->cx.as<double>(), ctx->cy.as<double>(), nullptr,
                                         ctx->cu.as<float>(), ctx->cv.as<float>(),
                                         ctx->cperm.as<int>());
    k_tile_scatter<<<grid, 256, 0, st>>>(td, 1, px, py, h, ctx->g, ctx->pkey.as<int>(),
                                         ctx->prank.as<int>(), ctx->pstart.as<int>(),
                                         ctx->px.as<double>(), ctx->py.as<double>(),
                                         ctx->ph.as<double>(), ctx->pu.as<float>(),
                                         ctx->pv.as<float>(), nullptr);
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

// Centres scattered again after their rank within the cell has changed (x order).
rbf_status tiles_scatter_centres(rbf_ctx* ctx, const double* cx, const double* cy, cudaStream_t st) {
    const dim3 grid(8, ctx->T);
    k_tile_scatter<<<grid, 256, 0, st>>>(ctx->tdesc.as<TileDev>(), 0, cx, cy, nullptr, ctx->g,
                                         ctx->ckey.as<int>(), ctx->crank.as<int>(),
                                         ctx->cstart.as<int>(), ctx->cx.as<double>(),
                                         ctx->cy.as<double>(), nullptr, ctx->cu.as<float>(),
                                         ctx->cv.as<float>(), ctx->cperm.as<int>());
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

// Each tile's range of row groups (the batched SpMV's work) and of sorted rows, and room for
// the work lists; the row groups must be described (gdesc) first.
rbf_status tiles_group_ranges(rbf_ctx* ctx, cudaStream_t st) {
    rbf_status s;
    const WorkLayout L = work_layout(ctx);
    if ((s = ensure(ctx, ctx->twork, L.total, st)) != RBF_OK) return s;
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->twork.p, 0, L.ranges_end, st));
    k_tile_ranges<<<std::max(1, div_up(std::max(ctx->ngroup, ctx->M), 256)), 256, 0, st>>>(
        ctx->gdesc.as<GroupRec>(), ctx->ngroup, ctx->crow.as<int4>(), ctx->M, work_view(ctx));
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

void tiles_release(rbf_ctx* ctx) {
    for (auto& sg : ctx->bt_graph)
        if (sg.exec) {
            cudaGraphExecDestroy(sg.exec);
            sg.exec = nullptr;
        }
    rbf_buf* bufs[] = {&ctx->tdesc, &ctx->rowtile, &ctx->tcg, &ctx->twork,
                       &ctx->tred, &ctx->qoff};
    for (rbf_buf* b : bufs) release(ctx, *b);
    if (ctx->hbt) cudaFreeHost(ctx->hbt);
    ctx->hbt = nullptr;
    ctx->hbt_bytes = 0;
}

// Packing of the tiles (host) and the binning of the packed system.
rbf_status bin_tiles_run(rbf_ctx* ctx, const rbf_tile* tiles, int T, const double* cx,
                         const double* cy, int64_t Mtot, const double* px, const double* py,
                         const double* h, int64_t Ntot, cudaStream_t st) {
    // ranges must partition [0, Mtot) and [0, Ntot)
    std::vector<std::pair<int64_t, int64_t>> cr, pr;
    for (int t = 0; t < T; ++t) {
        const rbf_tile& q = tiles[t];
        if (q.M < 1 || q.N < 0 || q.c0 < 0 || q.p0 < 0 || q.c0 + q.M > Mtot || q.p0 + q.N > Ntot)
            return set_err(ctx, RBF_ERR_ARG, "tile range outside the concatenated arrays");
        if (!(q.R > 0.0) || !isfinite(q.R)) return set_err(ctx, RBF_ERR_ARG, "tile R must be finite and > 0");
        for (int k = 0; k < 4; ++k)
            if (!isfinite(q.bbox[k])) return set_err(ctx, RBF_ERR_ARG, "non-finite tile bbox");
        if (!(q.bbox[2] >= q.bbox[0]) || !(q.bbox[3] >= q.bbox[1]))
            return set_err(ctx, RBF_ERR_ARG, "tile bbox must be {x0, y0, x1, y1} with x1 >= x0, y1 >= y0");
        cr.push_back({q.c0, q.M});
        if (q.N > 0) pr.push_back({q.p0, q.N});
    }
    auto partitions = [](std::vector<std::pair<int64_t, int64_t>>& r, int64_t total) {
        std::sort(r.begin(), r.end());
        int64_t at = 0;
        for (auto& x : r) {
            if (x.first != at) return false;
            at += x.second;
        }
        return at == total;
    };
    if (!partitions(cr, Mtot)) return set_err(ctx, RBF_ERR_ARG, "tile centre ranges must partition [0, Mtot)");
    if (!partitions(pr, Ntot)) return set_err(ctx, RBF_ERR_ARG, "tile point ranges must partition [0, Ntot)");

    // bands of cell rows, two empty rows apart
    const double hcell = kCellMargin, invh = 1.0 / kCellMargin;
    std::vector<TileDev> td(T);
    int64_t W = 1, GY = 0;
    for (int t = 0; t < T; ++t) {
        const rbf_tile& q = tiles[t];
        const double nx = std::max(1.0, ceil((q.bbox[2] - q.bbox[0]) / q.R * invh));
        const double ny = std::max(1.0, ceil((q.bbox[3] - q.bbox[1]) / q.R * invh));
        if (nx * ny > double(1 << 24))
            return set_err(ctx, RBF_ERR_LIMIT, "tile cell grid larger than 2^24 cells");
        TileDev d;
        d.c0 = q.c0;
        d.m = q.M;
        d.p0 = q.p0;
        d.n = q.N;
        d.x0 = q.bbox[0];
        d.y0 = q.bbox[1];
        d.x1 = q.bbox[2];
        d.y1 = q.bbox[3];
        d.R = q.R;
        d.gx = int(nx);
        d.gy = int(ny);
        d.oy = int(GY);
        d.pad = 0;
        td[t] = d;
        W = std::max<int64_t>(W, d.gx);
        GY += d.gy + (t + 1 < T ? 2 : 0);
        if (GY > (int64_t(1) << 24)) break;
    }
    if (double(W) * double(GY) > double(1 << 24))
        return set_err(ctx, RBF_ERR_LIMIT, "packed cell grid of the tiles larger than 2^24 cells");
    Grid g;
    g.x0 = 0.0;
    g.y0 = 0.0;
    g.R = 1.0;
    g.invR = 1.0;
    g.R2 = 1.0;
    g.h = hcell;
    g.invh = invh;
    g.gx = int(W);
    g.gy = int(GY);
    g.ncell = g.gx * g.gy;
    std::vector<int> rowtile(GY, -1);
    for (int t = 0; t < T; ++t)
        for (int r = 0; r < td[t].gy; ++r) rowtile[td[t].oy + r] = t;

    tiles_release(ctx);
    ctx->astore_ok = false;
    ctx->T = T;
    ctx->tiles.assign(tiles, tiles + T);
    ctx->g = g;
    ctx->M = int(Mtot);
    ctx->N = int(Ntot);
    rbf_status s;
    if ((s = ensure(ctx, ctx->tdesc, sizeof(TileDev) * T, st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->rowtile, sizeof(int) * GY, st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->tcg, TileLayout(T).total, st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->tred, RedLayout(T).total, st)) != RBF_OK) return s;
    const size_t hb = std::max(TileLayout(T).total, RedLayout(T).total);
    if (cudaMallocHost(&ctx->hbt, hb) != cudaSuccess) {
        cudaGetLastError();
        ctx->hbt = nullptr;
        return set_err(ctx, RBF_ERR_ALLOC, "pinned host buffer for the tile scalars");
    }
    ctx->hbt_bytes = hb;
    RBF_CUDA_TRY(cudaMemcpyAsync(ctx->tdesc.p, td.data(), sizeof(TileDev) * T,
                                 cudaMemcpyHostToDevice, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(ctx->rowtile.p, rowtile.data(), sizeof(int) * GY,
                                 cudaMemcpyHostToDevice, st));
    // the host vectors are pageable: the copies above complete before returning
    return bin_run(ctx, cx, cy, px, py, h, st);
}

rbf_status solve_tiles_run(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                           int min_support, rbf_tile_info* tinfo, rbf_solve_info* info,
                           cudaStream_t st) {
    const int M = ctx->M, T = ctx->T;
    const Binned bd = view(ctx);
    rbf_status s;
#define ENS(buf, bytes) \
    if ((s = ensure(ctx, ctx->buf, (bytes), st)) != RBF_OK) return s;
    ENS(x, sizeof(double) * M);
    ENS(r, sizeof(double) * M);
    ENS(scal, 256);
    int* npin_d = ctx->scal.as<int>();
    RBF_CUDA_TRY(cudaMemsetAsync(npin_d, 0, sizeof(int), st));
    std::vector<int> iters(T, 0), refs(T, 0), state(T, kConverged);
    std::vector<double> rel(T, 0.0);
    std::vector<int64_t> npin(T, 0);
    std::vector<char> tpro(T, 0);   // tiles finished in FP64 after their FP32 refinement
    int promoted = 0;
    const int nb = div_up(M, 256);

    auto fp64_solve = [&](const std::vector<char>& active, const double* x0) -> rbf_status {
        // FP64 batched CG from x0 (sorted order), else from the caller's c0, else from 0
        ENS(cgv[0], sizeof(double) * kCgVecs * cg_stride(M));
        const CgVec<double> v = cg_vectors<double>(ctx);
        if (!x0 && use_c0) {
            double* c0s = ctx->r.as<double>();   // free in the FP64 path
            launch_gather_sorted(c, bd.cperm, c0s, M, st);
            ctx->launches += 1;
            x0 = c0s;
        }
        std::vector<double> one(T, 1.0), tl(T, tol);
        BcgOut o;
        rbf_status s2 = run_bcg<double, double>(ctx, ctx->bvec.as<double>(), x0, active, one, tl,
                                                maxit, &o, st);
        if (s2 != RBF_OK) return s2;
        for (int t = 0; t < T; ++t) {
            if (!active[t]) continue;
            iters[t] += o.it[t];
            state[t] = o.state[t];
            rel[t] = o.rel[t];
        }
        k_tile_from_sorted<double><<<nb, 256, 0, st>>>(v.x, bd.cperm, c, M);
        ctx->launches += 1;
        RBF_CUDA_TRY(cudaGetLastError());
        return RBF_OK;
    };

    if (ctx->prec == RBF_FP64) {
        ENS(dinv, sizeof(double) * M);
        ENS(bjinv, sizeof(double) * std::max<int64_t>(ctx->nbj, 1));
        if ((s = prec_setup_run(ctx, RBF_FP64, min_support, npin_d, st)) != RBF_OK) return s;
        if ((s = tile_norms<double>(ctx, nullptr, ctx->dinv.as<double>(), nullptr, &npin, st)) != RBF_OK)
            return s;
        std::vector<char> all(T, 1);
        if ((s = fp64_solve(all, nullptr)) != RBF_OK) return s;
    } else {
        ENS(cgv[1], sizeof(float) * kCgVecs * cg_stride(M));
        ENS(dinv32, sizeof(float) * M);
        ENS(bjinv32, sizeof(float) * std::max<int64_t>(ctx->nbj, 1));
        if ((s = prec_setup_run(ctx, RBF_FP32_REFINE, min_support, npin_d, st)) != RBF_OK) return s;
        const float* dinv32 = ctx->dinv32.as<float>();
        const CgVec<float> v = cg_vectors<float>(ctx);
        double* x64 = ctx->x.as<double>();
        double* r64 = ctx->r.as<double>();
        std::vector<double> bn2, rn2;
        if ((s = tile_norms<float>(ctx, ctx->bvec.as<double>(), dinv32, &bn2, &npin, st)) != RBF_OK)
            return s;
        // a start vector's first residual from the FP32 matrix (as in the single-system
        // solver: accurate far below the inner tolerance, replaced by the FP64 residual of
        // the next refinement step, never used to declare convergence)
        bool approx_r = false;
        if (use_c0) {
            launch_gather_sorted(c, bd.cperm, x64, M, st);
            k_zero_masked<<<nb, 256, 0, st>>>(M, x64, dinv32);
            ctx->launches += 2;
            launch_resid32(ctx, x64, r64, st);
            approx_r = true;
        } else {
            RBF_CUDA_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * M, st));
            RBF_CUDA_TRY(cudaMemcpyAsync(r64, ctx->bvec.p, sizeof(double) * M,
                                         cudaMemcpyDeviceToDevice, st));
            k_zero_masked<<<nb, 256, 0, st>>>(M, r64, dinv32);
            ctx->launches += 1;
        }
        if ((s = tile_norms<float>(ctx, r64, dinv32, &rn2, nullptr, st)) != RBF_OK) return s;
        std::vector<double> bn(T), rn(T);
        for (int t = 0; t < T; ++t) {
            bn[t] = sqrt(bn2[t]);
            rn[t] = sqrt(rn2[t]);
        }
        // stall[t]: tile t's refinement stopped helping (or its FP32 CG broke down before a
        // step); it leaves the FP32 loop and is finished in FP64, the other tiles go on
        std::vector<char> conv(T, 0), active(T, 0), stall(T, 0), weak(T, 0);
        double* dscale = reinterpret_cast<double*>(ctx->tred.as<char>() + RedLayout(T).scale);
        std::vector<double> hscale(T);
        for (int outer = 0;; ++outer) {
            int nact = 0;
            for (int t = 0; t < T; ++t) {
                const double rl = bn[t] > 0.0 ? rn[t] / bn[t] : 0.0;
                rel[t] = rl;
                if (!conv[t] && ((rl <= tol && !approx_r) || rn[t] == 0.0)) conv[t] = 1;
                active[t] = !conv[t] && !stall[t];
                nact += active[t];
            }
            if (nact == 0 || outer == ctx->max_refine) break;
            std::vector<double> bsc(T, 0.0), itol(T, 1.0);
            for (int t = 0; t < T; ++t) {
                if (!active[t]) continue;
                bsc[t] = 1.0 / rn[t];
                itol[t] = std::max(ctx->inner_tol, 0.5 * tol / rel[t]);
            }
            BcgOut o;
            if ((s = run_bcg<float, double>(ctx, r64, nullptr, active, bsc, itol, maxit, &o, st)) != RBF_OK)
                return s;
            for (int t = 0; t < T; ++t) {
                hscale[t] = active[t] ? rn[t] : 0.0;
                if (!active[t]) continue;
                iters[t] += o.it[t];
                refs[t] += 1;
                // an inner breakdown before any step (FP32 rounding can make B32 indefinite on
                // a very ill-conditioned tile) leaves nothing to apply: hand over to FP64
                if (o.state[t] == kBreakdown && o.it[t] == 0) stall[t] = 1;
            }
            RBF_CUDA_TRY(cudaMemcpyAsync(dscale, hscale.data(), sizeof(double) * T,
                                         cudaMemcpyHostToDevice, st));
            k_tile_axpy<<<nb, 256, 0, st>>>(bd, x64, v.x, dscale, dinv32);
            RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
            if ((s = residual_run(ctx, x64, r64, false, st)) != RBF_OK) return s;
            k_zero_masked<<<nb, 256, 0, st>>>(M, r64, dinv32);
            ctx->launches += 2;
            if ((s = tile_norms<float>(ctx, r64, dinv32, &rn2, nullptr, st)) != RBF_OK) return s;
            approx_r = false;
            for (int t = 0; t < T; ++t) {
                if (!active[t]) continue;   // other tiles keep their iterate and residual
                const double rnew = sqrt(rn2[t]);
                // stalled: two steps in a row each gained less than half of what the inner
                // solve was asked for (and at most a halving), short of the tolerance; one weak
                // step alone is retried (the FP32 iterates vary from run to run, and a retry
                // costs a few hundred iterations of one tile against an FP64 finish)
                if (!(rnew <= tol * bn[t]) && !(rnew < std::max(0.5, 2.0 * itol[t]) * rn[t])) {
                    if (++weak[t] >= 2) stall[t] = 1;
                } else {
                    weak[t] = 0;
                }
                rn[t] = rnew;
            }
        }
        for (int t = 0; t < T; ++t) {
            rel[t] = bn[t] > 0.0 ? rn[t] / bn[t] : 0.0;
            if (!conv[t] && ((rel[t] <= tol && !approx_r) || rn[t] == 0.0)) conv[t] = 1;
            state[t] = conv[t] ? kConverged : kMaxIt;
        }
        bool all = true;
        for (int t = 0; t < T; ++t) all = all && conv[t];
        if (all) {
            launch_scatter_orig(x64, bd.cperm, c, M, st);
            ctx->launches += 1;
        } else {
            // Promote: assemble B in FP64 and finish the unconverged tiles with FP64 CG
            // started from their refined iterates; converged tiles keep theirs.
            if ((s = assemble_run(ctx, ctx->kernel, RBF_FP64, st)) != RBF_OK) return s;
            ctx->prec = RBF_FP64;
            promoted = 1;
            ENS(dinv, sizeof(double) * M);
            ENS(bjinv, sizeof(double) * std::max<int64_t>(ctx->nbj, 1));
            RBF_CUDA_TRY(cudaMemsetAsync(npin_d, 0, sizeof(int), st));
            if ((s = prec_setup_run(ctx, RBF_FP64, min_support, npin_d, st)) != RBF_OK) return s;
            for (int t = 0; t < T; ++t) tpro[t] = !conv[t];
            // a few tiles, typically: not worth tuning the FP64 loop for the whole batch
            ctx->no_tune_now = true;
            s = fp64_solve(tpro, x64);
            ctx->no_tune_now = false;
            if (s != RBF_OK) return s;
        }
    }
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->solved = true;
    rbf_solve_info tot{};
    rbf_status worst = RBF_OK;
    for (int t = 0; t < T; ++t) {
        const rbf_status ts = status_of(state[t]);
        if (ts == RBF_ERR_BREAKDOWN) worst = RBF_ERR_BREAKDOWN;
        else if (ts != RBF_OK && worst == RBF_OK) worst = ts;
        tot.iterations = std::max(tot.iterations, iters[t]);
        tot.refinements = std::max(tot.refinements, refs[t]);
        tot.rel_residual = std::max(tot.rel_residual, rel[t]);
        tot.pinned += npin[t];
        if (tinfo) {
            tinfo[t].iterations = iters[t];
            tinfo[t].refinements = refs[t];
            tinfo[t].rel_residual = rel[t];
            tinfo[t].pinned = npin[t];
            tinfo[t].status = ts;
            tinfo[t].promoted = tpro[t];
        }
    }
    tot.promoted = promoted;
    if (info) *info = tot;
#undef ENS
    if (worst == RBF_ERR_BREAKDOWN) return set_err(ctx, worst, "CG breakdown in some tile");
    if (worst != RBF_OK) return set_err(ctx, worst, "some tile did not reach tol");
    return RBF_OK;
}

template <typename T>
__global__ void k_tile_fill(T* __restrict__ v, int n, T value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = value;
}

// Timing hooks on a batched system (after rbf_solve_tiles): `reps` launches of the batched
// SpMV alone with every tile running and u = 1, or `reps` batched CG iterations from a cold
// start, in the configuration the solver uses.
template <typename T>
rbf_status bench_tiles_impl(rbf_ctx* ctx, int reps, bool spmv_only, cudaStream_t st) {
    Cfg cf;
    rbf_status s = pick_cfg<T>(ctx, &cf, st);
    if (s != RBF_OK) return s;
    const int T_ = ctx->T;
    std::vector<char> act(T_, 1);
    std::vector<double> one(T_, 1.0), zero(T_, 0.0);
    if ((s = write_tile_state(ctx, act, one, zero, 1 << 30, st)) != RBF_OK) return s;
    const CgVec<T> v = cg_vectors<T>(ctx);
    const TileCg tc = tile_view(ctx);
    if (spmv_only) {
        k_tile_fill<T><<<div_up(ctx->M, 256), 256, 0, st>>>(v.u, ctx->M, T(1));
        RBF_CUDA_TRY(cudaMemsetAsync(v.w[0], 0, sizeof(T) * ctx->M, st));
        launch_worklist(ctx, tc, cf, st);
        const Binned bd = view(ctx);
        const int items = div_up(ctx->ngroup, cf.chunk) + ctx->T;
        const int grid = std::max(1, std::min(cf.bps * sm_count(ctx), div_up(items, kSpmvWarps)));
        for (int k = 0; k < reps; ++k)
            k_bcg_spmv<T><<<grid, kSpmvWarps * 32, 0, st>>>(bd, work_view(ctx).items_s,
                                                            bvals_dev<T>(ctx), v.u, v.w[0], 0,
                                                            ctx->T, tc);
        ctx->launches += reps + 2;
    } else {
        if ((s = bcg_start<T, double>(ctx, ctx->bvec.as<double>(), false, cf, st)) != RBF_OK) return s;
        for (int k = 0; k < reps; ++k) launch_bcg_iteration<T>(ctx, v, tc, cf, k & 1, st);
        ctx->launches += 2 * int64_t(reps);
    }
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status bench_tiles_run(rbf_ctx* ctx, int reps, bool spmv_only, cudaStream_t st) {
    return ctx->prec == RBF_FP64 ? bench_tiles_impl<double>(ctx, reps, spmv_only, st)
                                 : bench_tiles_impl<float>(ctx, reps, spmv_only, st);
}

// Batched step (e): queries grouped by tile (qoff: HOST, T+1 offsets), or each tile's own
// nx x ny grid when qx is null.
rbf_status eval_tiles_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                          const int64_t* qoff, int nx, int ny, double* f, cudaStream_t st) {
    const int T = ctx->T;
    rbf_status s = ensure(ctx, ctx->csort, sizeof(double) * ctx->M, st);
    if (s != RBF_OK) return s;
    const Binned bd = view(ctx);
    launch_gather_sorted(c, bd.cperm, ctx->csort.as<double>(), ctx->M, st);
    ctx->launches += 1;
    const TileDev* td = ctx->tdesc.as<TileDev>();
    const double* cs = ctx->csort.as<double>();
    int64_t most = 0;
    if (qx) {
        for (int t = 0; t < T; ++t) most = std::max<int64_t>(most, qoff[t + 1] - qoff[t]);
        if ((s = ensure(ctx, ctx->qoff, sizeof(long long) * (T + 1), st)) != RBF_OK) return s;
        RBF_CUDA_TRY(cudaMemcpyAsync(ctx->qoff.p, qoff, sizeof(long long) * (T + 1),
                                     cudaMemcpyHostToDevice, st));
    } else {
        most = int64_t(nx) * ny;
    }
    if (most == 0) return RBF_OK;
    const dim3 grid(std::max(1, std::min(div_up(most, 256), 64)), T);
    const long long* qo = ctx->qoff.as<long long>();
#define EVAL_TILES(K)                                                                       \
    if (qx) k_eval_tiles<K><<<grid, 256, 0, st>>>(bd, td, cs, qx, qy, qo, f);               \
    else k_eval_tiles_grid<K><<<grid, 256, 0, st>>>(bd, td, cs, nx, ny, f);
    switch (ctx->kernel) {
        case RBF_W30: EVAL_TILES(0) break;
        case RBF_W31: EVAL_TILES(1) break;
        case RBF_W32: EVAL_TILES(2) break;
        default: EVAL_TILES(3) break;
    }
#undef EVAL_TILES
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    if (qx) RBF_CUDA_TRY(cudaStreamSynchronize(st));   // qoff's host array is pageable
    return RBF_OK;
}

rbf_status autotune_run(rbf_ctx* ctx, cudaStream_t st) {
    const int M = ctx->M;
    rbf_status s;
    if ((s = ensure(ctx, ctx->scal, 256, st)) != RBF_OK) return s;
    int* npin_d = ctx->scal.as<int>();
    if (ctx->prec == RBF_FP64) {
        if ((s = ensure(ctx, ctx->cgv[0], sizeof(double) * kCgVecs * cg_stride(M), st)) != RBF_OK) return s;
        if ((s = ensure(ctx, ctx->dinv, sizeof(double) * M, st)) != RBF_OK) return s;
        if ((s = ensure(ctx, ctx->bjinv, sizeof(double) * std::max<int64_t>(ctx->nbj, 1), st)) != RBF_OK)
            return s;
        if ((s = prec_setup_run(ctx, RBF_FP64, 3, npin_d, st)) != RBF_OK) return s;
        return autotune_impl<double>(ctx, st);
    }
    if ((s = ensure(ctx, ctx->cgv[1], sizeof(float) * kCgVecs * cg_stride(M), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->dinv32, sizeof(float) * M, st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->bjinv32, sizeof(float) * std::max<int64_t>(ctx->nbj, 1), st)) != RBF_OK)
        return s;
    if ((s = prec_setup_run(ctx, RBF_FP32_REFINE, 3, npin_d, st)) != RBF_OK) return s;
    return autotune_impl<float>(ctx, st);
}

// ---------------------------------------------------------------------------------------
// Moving window (the "moving window" technique of the paper's future work, Section 7): the
// domain is cut into wx x wy overlapping windows; each is one tile of the batched fit over its
// own points and the centres whose support reaches them, and the surface blends the windows'
// local surfaces with a smooth-step partition of unity. Window geometry:
//   core edges  a_i = x0 + (x1 - x0) i / wx  (likewise along y)
//   extended    [a_i - d, a_{i+1} + d], closed; a side on the domain's boundary is open to
//               infinity (items outside the box belong to the edge windows)
//   data box    the extended box grown by the margin m on its inner sides; the window's
//               points and centres are those in it (a centre at its edge keeps about half of
//               its support's points, so the window's system stays well conditioned)
//   weight      product over the inner sides of s((q - (a_i - d)) / 2d), s(((a_{i+1} + d) - q)
//               / 2d), s(t) = t^2 (3 - 2t) clamped to [0, 1]; with d = 0 the steps q >= a_i,
//               q < a_{i+1}
// ---------------------------------------------------------------------------------------
namespace {

// The layout's bounds, computed once on the host in the operation order of the definition
// (membership decisions are exact comparisons against these values), DEVICE table:
//   x: data_lo[wx], data_hi[wx], ext_lo[wx], ext_hi[wx]; then y likewise (wy each)
// data = extended box grown by the margin; sides on the domain's boundary are -inf / +inf.
struct WinGeom {
    double x0, y0, d;
    float inv_cx, inv_cy;        // wx / (x1 - x0), wy / (y1 - y0): candidate lookup only
    float reach_data, reach_ext; // d + margin, d
    const double* tx;            // x bounds (4 wx values)
    const double* ty;            // y bounds (4 wy values)
    int wx, wy;
};

// Core edge i of n over [lo, hi] (host).
inline double win_edge(double lo, double hi, int i, int n) {
    return lo + (hi - lo) * double(i) / double(n);
}

// Is v inside window i's interval along one axis? t: that axis' bounds, data or extended.
__device__ __forceinline__ bool win_member(double v, const double* __restrict__ t, int i, int n,
                                           bool data) {
    const double* b = t + (data ? 0 : 2 * n);
    return v >= b[i] && v <= b[n + i];
}

// The windows along one axis that may hold v: a superset (one window of slack on each side
// absorbs the FP32 rounding); callers test each exactly. v - lo is taken in FP64 so that the
// rounding is relative to the offset into the domain, not to the coordinates.
__device__ __forceinline__ int2 win_range(double v, double lo, float inv_c, int n, float reach) {
    const float dv = float(v - lo);
    const float a = floorf((dv - reach) * inv_c) - 1.0f, b = floorf((dv + reach) * inv_c) + 1.0f;
    const int i0 = int(fminf(fmaxf(a, 0.0f), float(n - 1)));
    const int i1 = int(fminf(fmaxf(b, 0.0f), float(n - 1)));
    return make_int2(i0, i1);
}

__device__ __forceinline__ double smooth_step01(double t) {
    t = fmin(fmax(t, 0.0), 1.0);
    return t * t * (3.0 - 2.0 * t);
}

// Window i's partition-of-unity factor along one axis (t: that axis' bounds).
__device__ __forceinline__ double win_axis_weight(double v, const double* __restrict__ t, int i,
                                                  int n, double d) {
    const double lo = t[2 * n + i], hi = t[3 * n + i];
    double w = 1.0;
    if (d > 0.0) {
        if (i > 0) w *= smooth_step01((v - lo) / (2.0 * d));
        if (i < n - 1) w *= smooth_step01((hi - v) / (2.0 * d));
    } else {
        if (i > 0 && !(v >= lo)) w = 0.0;
        if (i < n - 1 && !(v < hi)) w = 0.0;
    }
    return w;
}

// Calls f(w) for every window w whose data box holds (xv, yv).
template <class F>
__device__ __forceinline__ void for_each_window(double xv, double yv, const WinGeom& g, F&& f) {
    const int2 rx = win_range(xv, g.x0, g.inv_cx, g.wx, g.reach_data);
    const int2 ry = win_range(yv, g.y0, g.inv_cy, g.wy, g.reach_data);
    for (int j = ry.x; j <= ry.y; ++j) {
        if (!win_member(yv, g.ty, j, g.wy, true)) continue;
        for (int i = rx.x; i <= rx.y; ++i)
            if (win_member(xv, g.tx, i, g.wx, true)) f(j * g.wx + i);
    }
}

// Count (cursor == nullptr) or scatter the items into the windows that hold them: each item
// of window w goes to off[w] + (a slot taken with an atomic), with its input index. One
// global atomic per (item, window): for many windows, where few items share a counter.
__global__ void k_win_items(const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ h, int64_t n, WinGeom g,
                            int* __restrict__ count, const long long* __restrict__ off,
                            int* __restrict__ cursor, double* __restrict__ ox,
                            double* __restrict__ oy, double* __restrict__ oh,
                            long long* __restrict__ oidx) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n;
         k += int64_t(gridDim.x) * blockDim.x) {
        const double xv = x[k], yv = y[k];
        for_each_window(xv, yv, g, [&](int w) {
            if (!cursor) {
                atomicAdd(&count[w], 1);
                return;
            }
            const long long slot = off[w] + atomicAdd(&cursor[w], 1);
            ox[slot] = xv;
            oy[slot] = yv;
            if (oh) oh[slot] = h[k];
            if (oidx) oidx[slot] = k;
        });
    }
}

// The same for few windows (T <= kWinBlockMax), where every item of a window would hit one
// counter: per chunk of kWinItems items the block counts its items per window in shared
// memory, takes one range per window with one global atomic, then scatters into its ranges.
constexpr int kWinBlockMax = 4096;
constexpr int kWinThreads = 512;
constexpr int kWinPerThread = 4;

__global__ void __launch_bounds__(kWinThreads)
k_win_items_block(const double* __restrict__ x, const double* __restrict__ y,
                  const double* __restrict__ h, int64_t n, WinGeom g,
                  int* __restrict__ count, const long long* __restrict__ off,
                  int* __restrict__ cursor, double* __restrict__ ox, double* __restrict__ oy,
                  double* __restrict__ oh, long long* __restrict__ oidx) {
    extern __shared__ int win_sm[];
    const int T = g.wx * g.wy;
    int* scnt = win_sm;          // per window: this chunk's items, then the scatter cursor
    int* sbase = win_sm + T;     // per window: the chunk's first slot in the window's range
    constexpr int64_t kChunk = int64_t(kWinThreads) * kWinPerThread;
    for (int64_t k0 = blockIdx.x * kChunk; k0 < n; k0 += int64_t(gridDim.x) * kChunk) {
        for (int w = threadIdx.x; w < T; w += kWinThreads) scnt[w] = 0;
        __syncthreads();
        for (int r = 0; r < kWinPerThread; ++r) {
            const int64_t k = k0 + r * kWinThreads + threadIdx.x;
            if (k < n) for_each_window(x[k], y[k], g, [&](int w) { atomicAdd(&scnt[w], 1); });
        }
        __syncthreads();
        for (int w = threadIdx.x; w < T; w += kWinThreads) {
            const int c = scnt[w];
            if (c > 0) {
                if (!cursor) atomicAdd(&count[w], c);
                else sbase[w] = atomicAdd(&cursor[w], c);
            }
            scnt[w] = 0;
        }
        __syncthreads();
        if (cursor) {
            for (int r = 0; r < kWinPerThread; ++r) {
                const int64_t k = k0 + r * kWinThreads + threadIdx.x;
                if (k >= n) continue;
                const double xv = x[k], yv = y[k];
                for_each_window(xv, yv, g, [&](int w) {
                    const long long slot = off[w] + sbase[w] + atomicAdd(&scnt[w], 1);
                    ox[slot] = xv;
                    oy[slot] = yv;
                    if (oh) oh[slot] = h[k];
                    if (oidx) oidx[slot] = k;
                });
            }
        }
        __syncthreads();
    }
}

// Counts or scatters the items into their windows (the block kernel for few windows).
void launch_win_items(const double* x, const double* y, const double* h, int64_t n,
                      const WinGeom& g, int* count, const long long* off,
                      int* cursor, double* ox, double* oy, double* oh, long long* oidx,
                      cudaStream_t st) {
    if (n <= 0) return;
    const int T = g.wx * g.wy;
    if (T <= kWinBlockMax) {
        const int64_t chunks = div_up(n, int64_t(kWinThreads) * kWinPerThread);
        const int grid = int(std::min<int64_t>(chunks, 152 * 4));
        k_win_items_block<<<grid, kWinThreads, sizeof(int) * 2 * size_t(T), st>>>(
            x, y, h, n, g, count, off, cursor, ox, oy, oh, oidx);
    } else {
        k_win_items<<<152 * 8, 256, 0, st>>>(x, y, h, n, g, count, off, cursor, ox, oy, oh, oidx);
    }
}

// The blended surface at (x, y): sum_w weight_w f_w / sum_w weight_w over the windows whose
// extended box holds the query (f_w: the window's own surface, as the batched evaluation).
template <int KIND>
__device__ __forceinline__ double eval_windows_at(const Binned& bd, const TileDev* __restrict__ td,
                                                  const double* __restrict__ c, const WinGeom& g,
                                                  double x, double y) {
    const int2 rx = win_range(x, g.x0, g.inv_cx, g.wx, g.reach_ext);
    const int2 ry = win_range(y, g.y0, g.inv_cy, g.wy, g.reach_ext);
    double num = 0.0, den = 0.0;
    for (int j = ry.x; j <= ry.y; ++j) {
        if (!win_member(y, g.ty, j, g.wy, false)) continue;
        const double wy = win_axis_weight(y, g.ty, j, g.wy, g.d);
        if (wy == 0.0) continue;
        for (int i = rx.x; i <= rx.y; ++i) {
            if (!win_member(x, g.tx, i, g.wx, false)) continue;
            const double wt = wy * win_axis_weight(x, g.tx, i, g.wx, g.d);
            if (wt == 0.0) continue;
            num = fma(wt, eval_tile_at<KIND>(bd, td[j * g.wx + i], c, x, y), num);
            den += wt;
        }
    }
    return den > 0.0 ? num / den : 0.0;
}

template <int KIND>
__global__ void k_eval_windows(Binned bd, const TileDev* __restrict__ td, const double* __restrict__ c,
                               WinGeom g, const double* __restrict__ qx, const double* __restrict__ qy,
                               int64_t Q, double* __restrict__ f) {
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < Q;
         q += int64_t(gridDim.x) * blockDim.x)
        f[q] = eval_windows_at<KIND>(bd, td, c, g, qx[q], qy[q]);
}

// The node-centred nx x ny grid over box (inclusive linspace, the last node exactly at the
// box's end), f[i nx + j], window by window: a work item is a segment of 32 consecutive nodes
// of one grid row inside one window's node range (host-computed, one node of slack; each lane
// tests its node against the window's extended box exactly), evaluated by the pair-stream
// engine in the window's tile frame; the weighted values are added into f with FP64 atomics
// (f zeroed first) and k_eval_windows_finish divides by the sum of the weights.
struct WinNodes {
    int j0, j1, i0, i1;          // node columns [j0, j1] and rows [i0, i1] of the window
};
constexpr int kWinEvalWarps = 8;

__device__ __forceinline__ double grid_node(int j, int n, double lo, double hi, double step) {
    return (j == n - 1 && n > 1) ? hi : __dadd_rn(__dmul_rn(double(j), step), lo);
}

template <int KIND>
__global__ void __launch_bounds__(kWinEvalWarps * 32)
k_eval_windows_grid(Binned bd, const TileDev* __restrict__ td, const double* __restrict__ c,
                    WinGeom g, const WinNodes* __restrict__ wn, const long long* __restrict__ woff,
                    int T, int nx, int ny, double bx0, double by0, double bx1, double by1,
                    double sx, double sy, double* __restrict__ f) {
    __shared__ EvalWarpSmem sm[kWinEvalWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long total = woff[T];
    for (long long gi = blockIdx.x * (long long)kWinEvalWarps + wp; gi < total;
         gi += (long long)gridDim.x * kWinEvalWarps) {
        int lo = 0, hi = T - 1;      // the window: the last with woff[win] <= gi
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (woff[mid] <= gi) lo = mid;
            else hi = mid - 1;
        }
        const int win = lo;
        const WinNodes r = wn[win];
        const int spr = (r.j1 - r.j0 + 32) / 32;
        const long long loc = gi - woff[win];
        const int i = r.i0 + int(loc / spr);
        const int j = r.j0 + int(loc % spr) * 32 + lane;
        const int wi = win % g.wx, wj = win / g.wx;
        bool valid = j <= r.j1;
        double x = 0.0, y = 0.0, wt = 0.0;
        if (valid) {
            x = grid_node(j, nx, bx0, bx1, sx);
            y = grid_node(i, ny, by0, by1, sy);
            valid = win_member(x, g.tx, wi, g.wx, false) && win_member(y, g.ty, wj, g.wy, false);
            if (valid) {
                wt = win_axis_weight(y, g.ty, wj, g.wy, g.d) * win_axis_weight(x, g.tx, wi, g.wx, g.d);
                valid = wt != 0.0;
            }
        }
        const TileDev t = td[win];
        const double fw = eval_pairs32<KIND>(bd, c, tile_query(bd, t, x, y, valid), tile_frame(t),
                                             lane, sm[wp]);
        if (valid) atomicAdd(&f[(long long)i * nx + j], wt * fw);
    }
}

// f[q] /= the sum of the weights of the windows whose extended box holds node q (0 where none
// does).
__global__ void k_eval_windows_finish(WinGeom g, int nx, int ny, double bx0, double by0,
                                      double bx1, double by1, double sx, double sy,
                                      double* __restrict__ f) {
    const int64_t Q = int64_t(nx) * ny;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < Q;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(q / nx), j = int(q % nx);
        const double x = grid_node(j, nx, bx0, bx1, sx), y = grid_node(i, ny, by0, by1, sy);
        const int2 rx = win_range(x, g.x0, g.inv_cx, g.wx, g.reach_ext);
        const int2 ry = win_range(y, g.y0, g.inv_cy, g.wy, g.reach_ext);
        double den = 0.0;
        for (int jj = ry.x; jj <= ry.y; ++jj) {
            if (!win_member(y, g.ty, jj, g.wy, false)) continue;
            const double wy = win_axis_weight(y, g.ty, jj, g.wy, g.d);
            if (wy == 0.0) continue;
            for (int ii = rx.x; ii <= rx.y; ++ii) {
                if (!win_member(x, g.tx, ii, g.wx, false)) continue;
                const double wt = wy * win_axis_weight(x, g.tx, ii, g.wx, g.d);
                if (wt == 0.0) continue;
                den += wt;
            }
        }
        f[q] = den > 0.0 ? f[q] / den : 0.0;
    }
}

// Node range [j0, j1] of an n-node linspace from lo (step) that may lie in [a, b] (either
// side possibly infinite), with one node of slack; j0 > j1 when none can.
inline void node_range(double a, double b, int n, double lo, double step, int& j0, int& j1) {
    if (n == 1 || !(step > 0.0)) {   // one node, or a degenerate or reversed box: every node
        j0 = 0;
        j1 = n - 1;
        return;
    }
    const double u0 = std::isfinite(a) ? floor((a - lo) / step) - 1.0 : 0.0;
    const double u1 = std::isfinite(b) ? ceil((b - lo) / step) + 1.0 : double(n - 1);
    j0 = int(std::min(std::max(u0, 0.0), double(n - 1)));
    j1 = int(std::min(std::max(u1, 0.0), double(n - 1)));
    if (u1 < 0.0 || u0 > double(n - 1)) j1 = j0 - 1;
}

// The layout's geometry over its bounds table (DEVICE, 4 (wx + wy) values).
WinGeom make_win_geom(const double* bbox, int wx, int wy, double overlap, double margin,
                      const double* table) {
    WinGeom g;
    g.x0 = bbox[0];
    g.y0 = bbox[1];
    g.d = overlap;
    g.inv_cx = float(double(wx) / (bbox[2] - bbox[0]));
    g.inv_cy = float(double(wy) / (bbox[3] - bbox[1]));
    g.reach_data = float(overlap + margin);
    g.reach_ext = float(overlap);
    g.tx = table;
    g.ty = table + 4 * size_t(wx);
    g.wx = wx;
    g.wy = wy;
    return g;
}

// The bounds table on the host: per axis data_lo, data_hi, ext_lo, ext_hi (n values each).
std::vector<double> win_table(const double* bbox, int wx, int wy, double d, double m) {
    std::vector<double> t(4 * (size_t(wx) + wy));
    auto axis = [&](double* b, double lo, double hi, int n) {
        for (int i = 0; i < n; ++i) {
            const double elo = win_edge(lo, hi, i, n) - d, ehi = win_edge(lo, hi, i + 1, n) + d;
            b[i] = i == 0 ? -INFINITY : elo - m;
            b[n + i] = i == n - 1 ? INFINITY : ehi + m;
            b[2 * n + i] = i == 0 ? -INFINITY : elo;
            b[3 * n + i] = i == n - 1 ? INFINITY : ehi;
        }
    };
    axis(t.data(), bbox[0], bbox[2], wx);
    axis(t.data() + 4 * size_t(wx), bbox[1], bbox[3], wy);
    return t;
}

WinGeom win_geom(const rbf_ctx* ctx) {
    return make_win_geom(ctx->win_bbox, ctx->win_wx, ctx->win_wy, ctx->win_overlap,
                         ctx->win_margin, ctx->win_edges.as<double>());
}

}  // namespace

rbf_status window_bin_run(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M,
                          const double* px, const double* py, const double* h, int64_t N,
                          double R, const double* bbox, int wx, int wy, double overlap,
                          double margin, cudaStream_t st) {
    ctx->win_on = false;
    const int T = wx * wy;
    rbf_status s;
    const std::vector<double> tab = win_table(bbox, wx, wy, overlap, margin);
    if ((s = ensure(ctx, ctx->win_edges, sizeof(double) * tab.size(), st)) != RBF_OK) return s;
    // `tab` is pageable host memory: the copy has read it when cudaMemcpyAsync returns
    RBF_CUDA_TRY(cudaMemcpyAsync(ctx->win_edges.p, tab.data(), sizeof(double) * tab.size(),
                                 cudaMemcpyHostToDevice, st));
    const WinGeom g = make_win_geom(bbox, wx, wy, overlap, margin, ctx->win_edges.as<double>());
    if ((s = ensure(ctx, ctx->win_count, sizeof(int) * 4 * size_t(T), st)) != RBF_OK) return s;
    int* ccount = ctx->win_count.as<int>();
    int* pcount = ccount + T;
    int* ccur = ccount + 2 * T;
    int* pcur = ccount + 3 * T;
    RBF_CUDA_TRY(cudaMemsetAsync(ccount, 0, sizeof(int) * 4 * size_t(T), st));
    launch_win_items(cx, cy, nullptr, M, g, ccount, nullptr, nullptr, nullptr, nullptr, nullptr,
                     nullptr, st);
    launch_win_items(px, py, nullptr, N, g, pcount, nullptr, nullptr, nullptr, nullptr, nullptr,
                     nullptr, st);
    ctx->launches += 2;
    RBF_CUDA_TRY(cudaGetLastError());
    std::vector<int> cnt(2 * size_t(T));
    RBF_CUDA_TRY(cudaMemcpyAsync(cnt.data(), ccount, sizeof(int) * 2 * size_t(T),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    // each window's range of the concatenated centres and points, and its tile
    std::vector<long long> off(2 * (size_t(T) + 1), 0);
    std::vector<rbf_tile> tiles(T);
    long long Mtot = 0, Ntot = 0;
    for (int w = 0; w < T; ++w) {
        if (cnt[w] < 1)
            return set_err(ctx, RBF_ERR_ARG, "a window holds no centre: use fewer windows or more overlap");
        off[w] = Mtot;
        off[T + 1 + w] = Ntot;
        const int i = w % wx, j = w / wx;
        rbf_tile& t = tiles[w];
        t.c0 = Mtot;
        t.M = cnt[w];
        t.p0 = Ntot;
        t.N = cnt[T + w];
        t.R = R;
        // the tile's box: the window's data box (the domain's box on its sides; items beyond
        // it go to the edge cells)
        const double* bx = tab.data();
        const double* by = tab.data() + 4 * size_t(wx);
        t.bbox[0] = i == 0 ? bbox[0] : bx[i];
        t.bbox[2] = i == wx - 1 ? bbox[2] : bx[wx + i];
        t.bbox[1] = j == 0 ? bbox[1] : by[j];
        t.bbox[3] = j == wy - 1 ? bbox[3] : by[wy + j];
        Mtot += cnt[w];
        Ntot += cnt[T + w];
    }
    off[T] = Mtot;
    off[2 * size_t(T) + 1] = Ntot;
    if (Mtot > (int64_t(1) << 30) || Ntot > (int64_t(1) << 30))
        return set_err(ctx, RBF_ERR_LIMIT, "the windows hold more than 2^30 centres or points");
    if ((s = ensure(ctx, ctx->win_off, sizeof(long long) * off.size(), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->win_c, sizeof(double) * 2 * size_t(std::max(Mtot, 1LL)), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->win_cidx, sizeof(long long) * size_t(std::max(Mtot, 1LL)), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->win_p, sizeof(double) * 3 * size_t(std::max(Ntot, 1LL)), st)) != RBF_OK) return s;
    RBF_CUDA_TRY(cudaMemcpyAsync(ctx->win_off.p, off.data(), sizeof(long long) * off.size(),
                                 cudaMemcpyHostToDevice, st));
    double* wc = ctx->win_c.as<double>();
    double* wp = ctx->win_p.as<double>();
    const long long* doff = ctx->win_off.as<long long>();
    launch_win_items(cx, cy, nullptr, M, g, nullptr, doff, ccur, wc, wc + Mtot, nullptr,
                     ctx->win_cidx.as<long long>(), st);
    launch_win_items(px, py, h, N, g, nullptr, doff + T + 1, pcur, wp, wp + Ntot, wp + 2 * Ntot,
                     nullptr, st);
    ctx->launches += N > 0 ? 2 : 1;
    RBF_CUDA_TRY(cudaGetLastError());
    // `off` is pageable host memory: the copy has read it by the time cudaMemcpyAsync returns
    if ((s = bin_tiles_run(ctx, tiles.data(), T, wc, wc + Mtot, Mtot, wp, wp + Ntot, wp + 2 * Ntot,
                           Ntot, st)) != RBF_OK)
        return s;
    ctx->win_on = true;
    ctx->win_wx = wx;
    ctx->win_wy = wy;
    ctx->win_overlap = overlap;
    ctx->win_margin = margin;
    for (int k = 0; k < 4; ++k) ctx->win_bbox[k] = bbox[k];
    ctx->win_M = Mtot;
    ctx->win_N = Ntot;
    return RBF_OK;
}

// The blended surface: at queries (qx non-null) or on the nx x ny grid over box.
rbf_status window_eval_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                           int64_t Q, int nx, int ny, const double* box, double* f, cudaStream_t st) {
    rbf_status s = ensure(ctx, ctx->csort, sizeof(double) * ctx->M, st);
    if (s != RBF_OK) return s;
    const Binned bd = view(ctx);
    launch_gather_sorted(c, bd.cperm, ctx->csort.as<double>(), ctx->M, st);
    ctx->launches += 1;
    const TileDev* td = ctx->tdesc.as<TileDev>();
    const double* cs = ctx->csort.as<double>();
    const WinGeom g = win_geom(ctx);
    const int64_t n = qx ? Q : int64_t(nx) * ny;
    if (n == 0) return RBF_OK;
    const int grid = int(std::min<int64_t>(div_up(n, 256), 152 * 16));
    if (qx) {
#define EVAL_WIN(K) k_eval_windows<K><<<grid, 256, 0, st>>>(bd, td, cs, g, qx, qy, Q, f);
        switch (ctx->kernel) {
            case RBF_W30: EVAL_WIN(0) break;
            case RBF_W31: EVAL_WIN(1) break;
            case RBF_W32: EVAL_WIN(2) break;
            default: EVAL_WIN(3) break;
        }
#undef EVAL_WIN
        ctx->launches += 1;
        RBF_CUDA_TRY(cudaGetLastError());
        return RBF_OK;
    }
    // the grid: per window its node ranges and first work item (host), then the windows'
    // weighted values added into f, then the division by the weights
    const int wx = ctx->win_wx, wy = ctx->win_wy, T = wx * wy;
    const std::vector<double> tab = win_table(ctx->win_bbox, wx, wy, ctx->win_overlap, ctx->win_margin);
    const double* tx = tab.data();
    const double* ty = tab.data() + 4 * size_t(wx);
    const double x0 = box[0], y0 = box[1], x1 = box[2], y1 = box[3];
    const double sx = nx > 1 ? (x1 - x0) / double(nx - 1) : 0.0;
    const double sy = ny > 1 ? (y1 - y0) / double(ny - 1) : 0.0;
    std::vector<WinNodes> wn(T);
    std::vector<long long> woff(size_t(T) + 1, 0);
    for (int w = 0; w < T; ++w) {
        const int i = w % wx, j = w / wx;
        WinNodes& r = wn[w];
        node_range(tx[2 * wx + i], tx[3 * wx + i], nx, x0, sx, r.j0, r.j1);
        node_range(ty[2 * wy + j], ty[3 * wy + j], ny, y0, sy, r.i0, r.i1);
        long long items = 0;
        if (r.j1 >= r.j0 && r.i1 >= r.i0) items = (long long)(r.i1 - r.i0 + 1) * ((r.j1 - r.j0 + 32) / 32);
        woff[w + 1] = woff[w] + items;
    }
    const size_t wn_bytes = (sizeof(WinNodes) * size_t(T) + 15) & ~size_t(15);
    if ((s = ensure(ctx, ctx->win_eval, wn_bytes + sizeof(long long) * woff.size(), st)) != RBF_OK) return s;
    WinNodes* dwn = reinterpret_cast<WinNodes*>(ctx->win_eval.p);
    long long* dwoff = reinterpret_cast<long long*>(ctx->win_eval.as<char>() + wn_bytes);
    // the host vectors are pageable: each copy has read its source when cudaMemcpyAsync returns
    RBF_CUDA_TRY(cudaMemcpyAsync(dwn, wn.data(), sizeof(WinNodes) * size_t(T), cudaMemcpyHostToDevice, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(dwoff, woff.data(), sizeof(long long) * woff.size(),
                                 cudaMemcpyHostToDevice, st));
    RBF_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(double) * size_t(n), st));
    const long long items = woff[T];
    if (items > 0) {
        const int eg = int(std::min<long long>((items + kWinEvalWarps - 1) / kWinEvalWarps, 152 * 8));
#define EVAL_WG(K)                                                                               \
    k_eval_windows_grid<K><<<eg, kWinEvalWarps * 32, 0, st>>>(bd, td, cs, g, dwn, dwoff, T, nx, ny, \
                                                            x0, y0, x1, y1, sx, sy, f);
        switch (ctx->kernel) {
            case RBF_W30: EVAL_WG(0) break;
            case RBF_W31: EVAL_WG(1) break;
            case RBF_W32: EVAL_WG(2) break;
            default: EVAL_WG(3) break;
        }
#undef EVAL_WG
        ctx->launches += 1;
    }
    k_eval_windows_finish<<<grid, 256, 0, st>>>(g, nx, ny, x0, y0, x1, y1, sx, sy, f);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

}  // namespace rbf
