// Step (a): bin centres and points into a uniform grid of cell side R.
//
// This replaces the kd-tree range query of Algorithm 1: every point within R of a
// centre lies in the 3x3 cells around the centre's cell, and every centre pair with a
// nonzero entry of B = A^T A (Eq. 11-12) lies within 2R, i.e. in the 5x5 cells around
// either one. The binning is a counting sort (histogram with atomics, device-wide
// exclusive scan, scatter); afterwards each cell's items are contiguous, so any 1 x k
// row of cells is one contiguous range of the sorted order. The centres of each cell are
// then ordered by x (ties by input index), so the centres of a cell row are ordered by x.
//
// The same pass lays out the stored upper triangle of B (Section 5 keeps only the upper
// triangle): for every centre s, the three column ranges of the sorted order its row keeps
// (see RowMeta: the centres of its own and the next two cell rows that lie within 2R in x of
// the chord of the 2R disc), found by binary search in x, the row's offset in the value array
// (a scan of the row lengths), and the row groups the SpMV sweeps (up to kGroupRows
// consecutive rows of one cell row with the union of their ranges).
#include <limits.h>

#include "rbf_internal.h"

namespace rbf {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan across a block of kScanThreads threads. Returns the thread's exclusive
// prefix; *total receives the block sum.
template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const T excl = x - v + (w > 0 ? wsum[w - 1] : T(0));
    *total = wsum[31];
    __syncthreads();
    return excl;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const TI* in, int n, TO* bsum) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    TO s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += TO(in[base + k]);
    TO tot;
    block_exclusive_scan<TO>(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan in place of nb <= kScanTile block sums (one block).
template <typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_bsum(TO* bsum, int nb) {
    const int base = threadIdx.x * kScanItems;
    TO v[kScanItems];
    TO s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < nb) ? bsum[base + k] : TO(0);
        s += v[k];
    }
    TO tot;
    TO e = block_exclusive_scan<TO>(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < nb) bsum[base + k] = e;
        e += v[k];
    }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const TI* in, int n, const TO* bsum,
                                                              TO* out) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    TO v[kScanItems];
    TO s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? TO(in[base + k]) : TO(0);
        s += v[k];
    }
    TO tot;
    TO e = block_exclusive_scan<TO>(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = e;
        if (base + k == n - 1) out[n] = e + v[k];
        e += v[k];
    }
}

template <typename TI, typename TO>
rbf_status scan_impl(rbf_ctx* ctx, const TI* in, TO* out, int n, cudaStream_t st) {
    if (n <= 0) {
        RBF_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(TO), st));
        return RBF_OK;
    }
    const int nb = div_up(n, kScanTile);
    if (nb > kScanTile) return set_err(ctx, RBF_ERR_LIMIT, "scan longer than 2^24 items");
    rbf_status s = ensure(ctx, ctx->scan_tmp, sizeof(int64_t) * (nb + 1), st);
    if (s != RBF_OK) return s;
    TO* bsum = ctx->scan_tmp.as<TO>();
    k_scan_reduce<TI, TO><<<nb, kScanThreads, 0, st>>>(in, n, bsum);
    k_scan_bsum<TO><<<1, kScanThreads, 0, st>>>(bsum, nb);
    k_scan_apply<TI, TO><<<nb, kScanThreads, 0, st>>>(in, n, bsum, out);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 3;
    return RBF_OK;
}

// ---------------------------------------------------------------------------
// counting sort
// ---------------------------------------------------------------------------

// stats[0]: max 3x3 candidates, stats[1]: max points per cell, stats[2]: non-finite input
__global__ void k_bin_count(const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ h, int n, Grid g, int* __restrict__ count,
                            int* __restrict__ key, int* __restrict__ rank, int* __restrict__ stats) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double xi = x[i], yi = y[i];
        bool bad = !isfinite(xi) || !isfinite(yi);
        if (h) bad = bad || !isfinite(h[i]);
        if (bad) atomicOr(&stats[2], 1);
        const int k = bad ? 0 : cell_iy(g, yi) * g.gx + cell_ix(g, xi);
        key[i] = k;
        rank[i] = atomicAdd(&count[k], 1);
    }
}

__global__ void k_scatter_centres(const double* __restrict__ x, const double* __restrict__ y, int n,
                                  Grid g, const int* __restrict__ key, const int* __restrict__ rank,
                                  const int* __restrict__ start, double* __restrict__ sx,
                                  double* __restrict__ sy, float* __restrict__ su,
                                  float* __restrict__ sv, int* __restrict__ perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = key[i];
        const int d = start[k] + rank[i];
        const double xi = x[i], yi = y[i];
        sx[d] = xi;
        sy[d] = yi;
        perm[d] = i;
        const int ix = k % g.gx, iy = k / g.gx;
        su[d] = float((xi - (g.x0 + ix * g.h)) * g.invR);
        sv[d] = float((yi - (g.y0 + iy * g.h)) * g.invR);
    }
}

__global__ void k_scatter_points(const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ h, int n, Grid g,
                                 const int* __restrict__ key, const int* __restrict__ rank,
                                 const int* __restrict__ start, double* __restrict__ sx,
                                 double* __restrict__ sy, double* __restrict__ sh,
                                 float* __restrict__ su, float* __restrict__ sv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = key[i];
        const int d = start[k] + rank[i];
        const double xi = x[i], yi = y[i];
        sx[d] = xi;
        sy[d] = yi;
        sh[d] = h[i];
        const int ix = k % g.gx, iy = k / g.gx;
        su[d] = float((xi - (g.x0 + ix * g.h)) * g.invR);
        sv[d] = float((yi - (g.y0 + iy * g.h)) * g.invR);
    }
}

// Rank of every centre within its cell in (x, input index) order, written to rank[] at the
// centre's input index (the counting sort's scatter then places the cell's centres in that
// order). One warp per cell, the cell's keys compared 32 at a time through shuffles. Cells of
// more than kMaxCellCentres centres are not ranked and raise stats[3].
constexpr int kMaxCellCentres = 16384;
__global__ void k_cell_xrank(int ncell, const int* __restrict__ cstart, const double* __restrict__ sx,
                             const int* __restrict__ perm, int* __restrict__ rank,
                             int* __restrict__ stats) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const int cs = cstart[c], m = cstart[c + 1] - cs;
    if (m <= 1) {
        if (m == 1 && lane == 0) rank[perm[cs]] = 0;
        return;
    }
    if (m > kMaxCellCentres) {
        if (lane == 0) atomicOr(&stats[3], 1);
        return;
    }
    for (int d0 = 0; d0 < m; d0 += 32) {
        const int d = d0 + lane;
        const double xd = d < m ? sx[cs + d] : 0.0;
        const int pd = d < m ? perm[cs + d] : 0;
        int r = 0;
        for (int e0 = 0; e0 < m; e0 += 32) {
            const int e = e0 + lane;
            const double xe = e < m ? sx[cs + e] : 0.0;
            const int pe = e < m ? perm[cs + e] : 0;
            const int ne = min(32, m - e0);
            for (int j = 0; j < ne; ++j) {
                const double xj = __shfl_sync(0xffffffffu, xe, j);
                const int pj = __shfl_sync(0xffffffffu, pe, j);
                r += (xj < xd || (xj == xd && pj < pd)) ? 1 : 0;
            }
        }
        if (d < m) rank[pd] = r;
    }
}

// Contiguous sorted-centre range of the cells (xa..xb, row), clipped to the grid.
__device__ __forceinline__ void cell_row_range(const Grid& g, const int* cstart, int row, int xa,
                                               int xb, int& s, int& e) {
    xa = max(xa, 0);
    xb = min(xb, g.gx - 1);
    if (row < 0 || row >= g.gy || xa > xb) {
        s = e = 0;
        return;
    }
    s = cstart[row * g.gx + xa];
    e = cstart[row * g.gx + xb + 1];
}

// Per cell: the centres' cell records, the size of the cell's inverse diagonal block, the
// assembly work items of its points, and the largest 3x3 candidate count of a point cell.
__global__ void k_rows(Grid g, const int* __restrict__ cstart, const int* __restrict__ pstart,
                       const int* __restrict__ rowtile, int64_t* __restrict__ bjsize,
                       int* __restrict__ wcount, int4* __restrict__ crow, int* __restrict__ stats) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int ix = c % g.gx, iy = c / g.gx;
    const int cs = cstart[c];
    const int m = cstart[c + 1] - cs;
    const int tile = rowtile ? rowtile[iy] : 0;
    for (int i = 0; i < m; ++i) crow[cs + i] = make_int4(cs, m, c, tile);
    bjsize[c] = m <= kMaxBlock ? int64_t(m) * m : 0;
    const int np = pstart[c + 1] - pstart[c];
    wcount[c] = (np + kWorkPoints - 1) / kWorkPoints;
    if (np > 0) {
        int ncand = 0;
        for (int d = -1; d <= 1; ++d) {
            int s, e;
            cell_row_range(g, cstart, iy + d, ix - 1, ix + 1, s, e);
            ncand += e - s;
        }
        atomicMax(&stats[0], ncand);
        atomicMax(&stats[1], np);
    }
}

// First index t in [a, b) with x[t] > v (strict) or >= v, over x ordered ascending.
__device__ __forceinline__ int upper_index(const double* x, int a, int b, double v, bool strict) {
    while (a < b) {
        const int mid = (a + b) >> 1;
        const bool right = strict ? (x[mid] > v) : (x[mid] >= v);
        if (right) b = mid;
        else a = mid + 1;
    }
    return a;
}

// Column ranges of row s (RowMeta without its offset) and the row's stored length in pairs.
// Coordinates are those of the sorted copies: the grid's frame for one system, the tile's
// frame (units of R_t, R = 1) for a batch; the lower edge of the row's own cell row is taken
// from the cell-local FP32 coordinate (error ~1e-7 R, far inside the disc margin).
__global__ void k_row_ranges(Grid g, int M, const int* __restrict__ cstart,
                             const double* __restrict__ sx, const double* __restrict__ sy,
                             const float* __restrict__ sv, const int4* __restrict__ crow,
                             RowMeta* __restrict__ rmeta, int64_t* __restrict__ rsize,
                             int* __restrict__ stats) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int c = crow[s].z;
    const int ix = c % g.gx, iy = c / g.gx;
    const double xs = sx[s], ys = sy[s];
    const double W = 2.0 * g.R * kDiscMargin;
    const double ybot = ys - double(sv[s]) * g.R;      // lower edge of the row's cell row
    int lo[3], hi[3];
    {   // own cell row: t >= s with x_t < x_s + W, within cells ix .. ix+2
        int a, e;
        cell_row_range(g, cstart, iy, ix, ix + 2, a, e);
        lo[0] = s;
        hi[0] = max(s + 1, upper_index(sx, s, e, xs + W, false));
    }
#pragma unroll
    for (int k = 1; k <= 2; ++k) {
        lo[k] = hi[k] = 0;
        const double dy = fmax(0.0, ybot + k * g.h - ys);
        if (iy + k >= g.gy || dy >= W) continue;
        const double w = sqrt(W * W - dy * dy);
        int a, e;
        cell_row_range(g, cstart, iy + k, ix - 2, ix + 2, a, e);
        lo[k] = upper_index(sx, a, e, xs - w, true);
        hi[k] = upper_index(sx, lo[k], e, xs + w, false);
    }
    RowMeta rm;
    unsigned int len = 0;
    int tot = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int l = lo[k] & ~3, h = (hi[k] + 3) & ~3;
        if (hi[k] <= lo[k]) l = h = lo[k] & ~3;
        const int q = (h - l) >> 2;
        if (q > kMaxSegQuads) atomicOr(&stats[4], 1);
        len |= unsigned(min(q, kMaxSegQuads)) << (kLenBits * k);
        tot += q;
        if (k == 1) rm.lo1 = l;
        if (k == 2) rm.lo2 = l;
    }
    rm.off = 0;
    rm.len = len;
    rmeta[s] = rm;
    rsize[s] = tot;      // in quads of values
}

// Offsets of the rows in the value array (in quads), from the scan of the row lengths.
__global__ void k_row_off(int M, const int64_t* __restrict__ roff, RowMeta* __restrict__ rmeta,
                          int* __restrict__ stats) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int64_t o = roff[s];
    if (o + (1 << (3 * kLenBits)) > (int64_t(1) << 32)) atomicOr(&stats[5], 1);
    rmeta[s].off = unsigned(o);
}

// Row groups per cell row: ceil(rows / kGroupRows) of the centres of cell row b.
__global__ void k_group_count(Grid g, const int* __restrict__ cstart, int* __restrict__ gcount) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.gy) return;
    const int n = cstart[(b + 1) * g.gx] - cstart[b * g.gx];
    gcount[b] = (n + kGroupRows - 1) / kGroupRows;
}

// One thread per row group: its rows and the union of their column ranges per segment.
__global__ void k_groups(Grid g, int ngroup, const int* __restrict__ cstart,
                         const int* __restrict__ gstart, const RowMeta* __restrict__ rmeta,
                         GroupRec* __restrict__ gdesc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ngroup) return;
    int a = 0, b = g.gy;            // cell row of the group: last b with gstart[b] <= q
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (gstart[mid] <= q) a = mid;
        else b = mid;
    }
    const int band = a;
    const int r0 = cstart[band * g.gx] + (q - gstart[band]) * kGroupRows;
    const int n = min(kGroupRows, cstart[(band + 1) * g.gx] - r0);
    int lo[3] = {r0 & ~3, INT_MAX, INT_MAX}, hi[3] = {r0 & ~3, INT_MIN, INT_MIN};
    for (int i = 0; i < n; ++i) {
        const RowMeta rm = rmeta[r0 + i];
        const int l[3] = {(r0 + i) & ~3, rm.lo1, rm.lo2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int p = seg_quads(rm.len, k);
            if (p == 0) continue;
            lo[k] = min(lo[k], l[k]);
            hi[k] = max(hi[k], l[k] + 4 * p);
        }
    }
    GroupDesc d;
    d.r0 = r0;
    d.n = n;
    d.lo0 = lo[0];
    d.q0 = (hi[0] - lo[0]) >> 2;
    d.lo1 = hi[1] > lo[1] ? lo[1] : 0;
    d.q1 = hi[1] > lo[1] ? (hi[1] - lo[1]) >> 2 : 0;
    d.lo2 = hi[2] > lo[2] ? lo[2] : 0;
    d.q2 = hi[2] > lo[2] ? (hi[2] - lo[2]) >> 2 : 0;
    GroupRec& rec = gdesc[q];
    rec.d = d;
    for (int i = 0; i < kGroupRows; ++i) rec.rows[i] = i < n ? rmeta[r0 + i] : RowMeta{0, 0, 0, 0};
}

__global__ void k_work_fill(int ncell, const int* __restrict__ pstart,
                            const int* __restrict__ wstart, int4* __restrict__ work) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int p0 = pstart[c], p1 = pstart[c + 1];
    int w = wstart[c];
    for (int q = p0; q < p1; q += kWorkPoints, ++w) work[w] = make_int4(c, q, min(q + kWorkPoints, p1), 0);
}

}  // namespace

rbf_status scan_i32(rbf_ctx* ctx, const int* in, int* out, int n, cudaStream_t st) {
    return scan_impl<int, int>(ctx, in, out, n, st);
}
rbf_status scan_i64(rbf_ctx* ctx, const int64_t* in, int64_t* out, int n, cudaStream_t st) {
    return scan_impl<int64_t, int64_t>(ctx, in, out, n, st);
}

rbf_status bin_run(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                   const double* py, const double* h, cudaStream_t st) {
    const Grid& g = ctx->g;
    const int M = ctx->M, N = ctx->N, nc = g.ncell;
    rbf_status s;
#define ENS(buf, bytes)                                   \
    if ((s = ensure(ctx, ctx->buf, (bytes), st)) != RBF_OK) return s;
    ENS(ccount, sizeof(int) * nc);
    ENS(pcount, sizeof(int) * nc);
    ENS(cstart, sizeof(int) * (nc + 1));
    ENS(pstart, sizeof(int) * (nc + 1));
    ENS(ckey, sizeof(int) * M);
    ENS(crank, sizeof(int) * M);
    ENS(pkey, sizeof(int) * N);
    ENS(prank, sizeof(int) * N);
    ENS(cx, sizeof(double) * M);
    ENS(cy, sizeof(double) * M);
    ENS(cu, sizeof(float) * M);
    ENS(cv, sizeof(float) * M);
    ENS(cperm, sizeof(int) * M);
    ENS(px, sizeof(double) * N);
    ENS(py, sizeof(double) * N);
    ENS(ph, sizeof(double) * N);
    ENS(pu, sizeof(float) * N);
    ENS(pv, sizeof(float) * N);
    ENS(rmeta, sizeof(RowMeta) * M);
    ENS(rsize, sizeof(int64_t) * M);
    ENS(roff, sizeof(int64_t) * (M + 1));
    ENS(gcount, sizeof(int) * g.gy);
    ENS(gstart, sizeof(int) * (g.gy + 1));
    ENS(wcount, sizeof(int) * nc);
    ENS(bjsize, sizeof(int64_t) * nc);
    ENS(crow, sizeof(int4) * M);
    ENS(bjoff, sizeof(int64_t) * (nc + 1));
    ENS(wstart, sizeof(int) * (nc + 1));
    ENS(stats, sizeof(int64_t) * 8);
    int* stats = ctx->stats.as<int>();
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->ccount.p, 0, sizeof(int) * nc, st));
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->pcount.p, 0, sizeof(int) * nc, st));
    RBF_CUDA_TRY(cudaMemsetAsync(stats, 0, sizeof(int64_t) * 8, st));

    const int T = 256;
    const int gbM = std::min(div_up(M, T), 152 * 16), gbN = std::min(div_up(N, T), 152 * 16);
    if (ctx->T > 0) {
        if ((s = tiles_count(ctx, cx, cy, px, py, h, st)) != RBF_OK) return s;
    } else {
        k_bin_count<<<gbM, T, 0, st>>>(cx, cy, nullptr, M, g, ctx->ccount.as<int>(),
                                       ctx->ckey.as<int>(), ctx->crank.as<int>(), stats);
        k_bin_count<<<gbN, T, 0, st>>>(px, py, h, N, g, ctx->pcount.as<int>(), ctx->pkey.as<int>(),
                                       ctx->prank.as<int>(), stats);
    }
    RBF_CUDA_TRY(cudaGetLastError());
    if ((s = scan_i32(ctx, ctx->ccount.as<int>(), ctx->cstart.as<int>(), nc, st)) != RBF_OK) return s;
    if ((s = scan_i32(ctx, ctx->pcount.as<int>(), ctx->pstart.as<int>(), nc, st)) != RBF_OK) return s;
    if (ctx->T > 0) {
        if ((s = tiles_scatter(ctx, cx, cy, px, py, h, st)) != RBF_OK) return s;
    } else {
        k_scatter_centres<<<gbM, T, 0, st>>>(cx, cy, M, g, ctx->ckey.as<int>(),
                                             ctx->crank.as<int>(), ctx->cstart.as<int>(),
                                             ctx->cx.as<double>(), ctx->cy.as<double>(),
                                             ctx->cu.as<float>(), ctx->cv.as<float>(),
                                             ctx->cperm.as<int>());
        k_scatter_points<<<gbN, T, 0, st>>>(px, py, h, N, g, ctx->pkey.as<int>(),
                                            ctx->prank.as<int>(), ctx->pstart.as<int>(),
                                            ctx->px.as<double>(), ctx->py.as<double>(),
                                            ctx->ph.as<double>(), ctx->pu.as<float>(),
                                            ctx->pv.as<float>());
    }
    // order each cell's centres by x, then scatter them again in that order
    k_cell_xrank<<<div_up(nc, 8), 256, 0, st>>>(nc, ctx->cstart.as<int>(), ctx->cx.as<double>(),
                                                ctx->cperm.as<int>(), ctx->crank.as<int>(), stats);
    if (ctx->T > 0) {
        if ((s = tiles_scatter_centres(ctx, cx, cy, st)) != RBF_OK) return s;
    } else {
        k_scatter_centres<<<gbM, T, 0, st>>>(cx, cy, M, g, ctx->ckey.as<int>(),
                                             ctx->crank.as<int>(), ctx->cstart.as<int>(),
                                             ctx->cx.as<double>(), ctx->cy.as<double>(),
                                             ctx->cu.as<float>(), ctx->cv.as<float>(),
                                             ctx->cperm.as<int>());
    }
    k_rows<<<div_up(nc, T), T, 0, st>>>(g, ctx->cstart.as<int>(), ctx->pstart.as<int>(),
                                        ctx->T > 0 ? ctx->rowtile.as<int>() : nullptr,
                                        ctx->bjsize.as<int64_t>(), ctx->wcount.as<int>(),
                                        ctx->crow.as<int4>(), stats);
    // the stored rows of B: column ranges, offsets, row groups
    k_row_ranges<<<div_up(M, T), T, 0, st>>>(g, M, ctx->cstart.as<int>(), ctx->cx.as<double>(),
                                             ctx->cy.as<double>(), ctx->cv.as<float>(),
                                             ctx->crow.as<int4>(), ctx->rmeta.as<RowMeta>(),
                                             ctx->rsize.as<int64_t>(), stats);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 7;
    if ((s = scan_i64(ctx, ctx->rsize.as<int64_t>(), ctx->roff.as<int64_t>(), M, st)) != RBF_OK)
        return s;
    k_row_off<<<div_up(M, T), T, 0, st>>>(M, ctx->roff.as<int64_t>(), ctx->rmeta.as<RowMeta>(), stats);
    k_group_count<<<div_up(g.gy, T), T, 0, st>>>(g, ctx->cstart.as<int>(), ctx->gcount.as<int>());
    ctx->launches += 2;
    if ((s = scan_i32(ctx, ctx->gcount.as<int>(), ctx->gstart.as<int>(), g.gy, st)) != RBF_OK) return s;
    if ((s = scan_i32(ctx, ctx->wcount.as<int>(), ctx->wstart.as<int>(), nc, st)) != RBF_OK) return s;
    if ((s = scan_i64(ctx, ctx->bjsize.as<int64_t>(), ctx->bjoff.as<int64_t>(), nc, st)) != RBF_OK)
        return s;

    // read back the sizes the host needs to allocate B and launch the assembly
    int64_t* hp = static_cast<int64_t*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[0], ctx->roff.as<int64_t>() + M, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[1], ctx->wstart.as<int>() + nc, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[2], stats, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[6], ctx->bjoff.as<int64_t>() + nc, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[7], ctx->gstart.as<int>() + g.gy, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    const int* hs = reinterpret_cast<const int*>(&hp[2]);
    ctx->nvals = 4 * hp[0];
    ctx->nbj = hp[6];
    ctx->nwork = *reinterpret_cast<const int*>(&hp[1]);
    ctx->ngroup = *reinterpret_cast<const int*>(&hp[7]);
    ctx->max_cand = hs[0];
    ctx->max_cell_pts = hs[1];
    if (hs[2]) return set_err(ctx, RBF_ERR_ARG, "non-finite coordinate or height");
    if (ctx->max_cand > kMaxCand)
        return set_err(ctx, RBF_ERR_LIMIT,
                       "more than rbf_max_candidates() centres in one 3x3 cell neighbourhood");
    if (hs[3]) return set_err(ctx, RBF_ERR_LIMIT, "more than 16384 centres in one cell");
    if (hs[4])
        return set_err(ctx, RBF_ERR_LIMIT, "more than 4092 centres within 2R of a centre in one cell row");
    if (hs[5]) return set_err(ctx, RBF_ERR_LIMIT, "stored B larger than 2^34 values");
    ENS(gdesc, sizeof(GroupRec) * std::max(ctx->ngroup, 1));
    k_groups<<<div_up(std::max(ctx->ngroup, 1), T), T, 0, st>>>(
        g, ctx->ngroup, ctx->cstart.as<int>(), ctx->gstart.as<int>(), ctx->rmeta.as<RowMeta>(),
        ctx->gdesc.as<GroupRec>());
    ctx->launches += 1;
    if (ctx->T > 0 && (s = tiles_group_ranges(ctx, st)) != RBF_OK) return s;
    ENS(work, sizeof(int4) * std::max(ctx->nwork, 1));
    k_work_fill<<<div_up(nc, T), T, 0, st>>>(nc, ctx->pstart.as<int>(), ctx->wstart.as<int>(),
                                             ctx->work.as<int4>());
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
#undef ENS
    return RBF_OK;
}

}  // namespace rbf
