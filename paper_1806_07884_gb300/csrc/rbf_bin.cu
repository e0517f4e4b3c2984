// Step (a): bin centres and points into a uniform grid of cell side R.
//
// This replaces the kd-tree range query of Algorithm 1: every point within R of a
// centre lies in the 3x3 cells around the centre's cell, and every centre pair with a
// nonzero entry of B = A^T A (Eq. 11-12) lies within 2R, i.e. in the 5x5 cells around
// either one. The binning is a counting sort (histogram with atomics, device-wide
// exclusive scan, scatter); afterwards each cell's items are contiguous, so any 1 x k
// row of cells is one contiguous range of the sorted order.
//
// The same pass sizes the stored upper triangle of B (Section 5 keeps only the
// upper triangle): the rows of the centres of cell c form a dense m_c x L_c block
// whose columns are the three contiguous ranges of RowSeg.
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

// Contiguous sorted-centre range of the cells (xa..xb, row), clipped to the grid.
__device__ __forceinline__ void cell_row_range(const Grid& g, const int* cstart, int row, int xa,
                                               int xb, int& s, int& l) {
    xa = max(xa, 0);
    xb = min(xb, g.gx - 1);
    if (row < 0 || row >= g.gy || xa > xb) {
        s = 0;
        l = 0;
        return;
    }
    s = cstart[row * g.gx + xa];
    l = cstart[row * g.gx + xb + 1] - s;
}

__global__ void k_rows(Grid g, const int* __restrict__ cstart, const int* __restrict__ pstart,
                       const int* __restrict__ rowtile, RowSeg* __restrict__ seg,
                       int64_t* __restrict__ rbsize, int64_t* __restrict__ bjsize,
                       int* __restrict__ wcount, int4* __restrict__ crow, int* __restrict__ stats) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int ix = c % g.gx, iy = c / g.gx;
    RowSeg sg;
    cell_row_range(g, cstart, iy, ix, ix + 2, sg.s0, sg.l0);
    cell_row_range(g, cstart, iy + 1, ix - 2, ix + 2, sg.s1, sg.l1);
    cell_row_range(g, cstart, iy + 2, ix - 2, ix + 2, sg.s2, sg.l2);
    sg.lp = (sg.l0 + sg.l1 + sg.l2 + kRowPad - 1) / kRowPad * kRowPad;
    seg[c] = sg;
    const int cs = cstart[c];
    const int m = cstart[c + 1] - cs;
    rbsize[c] = int64_t(m) * int64_t(sg.lp);
    const int tile = rowtile ? rowtile[iy] : 0;
    for (int i = 0; i < m; ++i) crow[cs + i] = make_int4(cs, m, c, tile);
    bjsize[c] = m <= kMaxBlock ? int64_t(m) * m : 0;
    const int np = pstart[c + 1] - pstart[c];
    wcount[c] = (np + kWorkPoints - 1) / kWorkPoints;
    if (np > 0) {
        int ncand = 0;
        for (int d = -1; d <= 1; ++d) {
            int s, l;
            cell_row_range(g, cstart, iy + d, ix - 1, ix + 1, s, l);
            ncand += l;
        }
        atomicMax(&stats[0], ncand);
        atomicMax(&stats[1], np);
    }
}

__global__ void k_work_fill(int ncell, const int* __restrict__ pstart,
                            const int* __restrict__ wstart, int4* __restrict__ work) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int p0 = pstart[c], p1 = pstart[c + 1];
    int w = wstart[c];
    for (int q = p0; q < p1; q += kWorkPoints, ++w) work[w] = make_int4(c, q, min(q + kWorkPoints, p1), 0);
}

__global__ void k_cell_desc(int ncell, int gx, const int* __restrict__ cstart,
                            const RowSeg* __restrict__ seg, const int64_t* __restrict__ rboff,
                            const int* __restrict__ rowtile, CellDesc* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const RowSeg sg = seg[c];
    CellDesc d;
    d.cs = cstart[c];
    d.m = cstart[c + 1] - d.cs;
    d.lp = sg.lp;
    d.pad = rowtile ? rowtile[c / gx] : 0;   // tile of the cell (batched systems)
    d.rboff = rboff[c];
    d.s0 = sg.s0;
    d.l0 = sg.l0;
    d.s1 = sg.s1;
    d.l1 = sg.l1;
    d.s2 = sg.s2;
    d.l2 = sg.l2;
    out[c] = d;
}

}  // namespace

void launch_cell_desc(rbf_ctx* ctx, cudaStream_t st) {
    k_cell_desc<<<div_up(ctx->g.ncell, 256), 256, 0, st>>>(
        ctx->g.ncell, ctx->g.gx, ctx->cstart.as<int>(), ctx->seg.as<RowSeg>(),
        ctx->rboff.as<int64_t>(), ctx->T > 0 ? ctx->rowtile.as<int>() : nullptr,
        ctx->cdesc.as<CellDesc>());
    ctx->launches += 1;
}

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
    ENS(seg, sizeof(RowSeg) * nc);
    ENS(rbsize, sizeof(int64_t) * nc);
    ENS(rboff, sizeof(int64_t) * (nc + 1));
    ENS(wcount, sizeof(int) * nc);
    ENS(bjsize, sizeof(int64_t) * nc);
    ENS(crow, sizeof(int4) * M);
    ENS(cdesc, sizeof(CellDesc) * nc);
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
    k_rows<<<div_up(nc, T), T, 0, st>>>(g, ctx->cstart.as<int>(), ctx->pstart.as<int>(),
                                        ctx->T > 0 ? ctx->rowtile.as<int>() : nullptr,
                                        ctx->seg.as<RowSeg>(), ctx->rbsize.as<int64_t>(),
                                        ctx->bjsize.as<int64_t>(), ctx->wcount.as<int>(),
                                        ctx->crow.as<int4>(), stats);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 5;
    if ((s = scan_i64(ctx, ctx->rbsize.as<int64_t>(), ctx->rboff.as<int64_t>(), nc, st)) != RBF_OK)
        return s;
    launch_cell_desc(ctx, st);
    if ((s = scan_i32(ctx, ctx->wcount.as<int>(), ctx->wstart.as<int>(), nc, st)) != RBF_OK) return s;
    if ((s = scan_i64(ctx, ctx->bjsize.as<int64_t>(), ctx->bjoff.as<int64_t>(), nc, st)) != RBF_OK)
        return s;

    // read back the sizes the host needs to allocate B and launch the assembly
    int64_t* hp = static_cast<int64_t*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[0], ctx->rboff.as<int64_t>() + nc, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[1], ctx->wstart.as<int>() + nc, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[2], stats, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(&hp[4], ctx->bjoff.as<int64_t>() + nc, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    const int* hs = reinterpret_cast<const int*>(&hp[2]);
    ctx->nvals = hp[0];
    ctx->nbj = hp[4];
    ctx->nwork = *reinterpret_cast<const int*>(&hp[1]);
    ctx->max_cand = hs[0];
    ctx->max_cell_pts = hs[1];
    if (hs[2]) return set_err(ctx, RBF_ERR_ARG, "non-finite coordinate or height");
    if (ctx->max_cand > kMaxCand)
        return set_err(ctx, RBF_ERR_LIMIT,
                       "more than rbf_max_candidates() centres in one 3x3 cell neighbourhood");
    if (ctx->T > 0 && (s = tiles_cell_list(ctx, st)) != RBF_OK) return s;
    ENS(work, sizeof(int4) * std::max(ctx->nwork, 1));
    k_work_fill<<<div_up(nc, T), T, 0, st>>>(nc, ctx->pstart.as<int>(), ctx->wstart.as<int>(),
                                             ctx->work.as<int4>());
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
#undef ENS
    return RBF_OK;
}

}  // namespace rbf
