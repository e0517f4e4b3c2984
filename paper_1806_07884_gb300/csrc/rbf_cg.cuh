// Device building blocks of the conjugate-gradient solvers (single system and batched
// tiles): warp and block reductions, the symmetric SpMV of one row group of the stored upper
// triangle, and the block-Jacobi preconditioner application.
#pragma once

#include <type_traits>
#include "rbf_internal.h"

namespace rbf {

// CG state of one system (or one tile of a batch).
enum { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxIt = 3, kInactive = 4 };

constexpr int kSpmvWarps = 8;
constexpr unsigned kFull = 0xffffffffu;
// CG iterations per pass of the solve graph's loop body (even: the buffers alternate).
constexpr int kItersPerBody = 4;
// Vectors of the CG workspace: x, u, p, r0, r1, s0, s1, w0, w1.
constexpr int kCgVecs = 9;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
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
        for (int k = 0; k < NV; ++k) v[k] = warp_sum_d(lane < nw ? red[k][lane] : 0.0);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide sums of NV values of type T: each warp sums in T (FP32 for the FP32 solver,
// keeping the slow FP64 pipe out of the per-row work), the warp totals are added in FP64.
// The result is valid in thread 0.
template <int NV, typename T>
__device__ __forceinline__ void block_sum_t(const T (&v)[NV], double (&out)[NV]) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const T s = warp_sum<T>(v[k]);
        if (lane == 0) red[k][w] = double(s);
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = warp_sum_d(lane < nw ? red[k][lane] : 0.0);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// Sum v[0..15] over the 32 lanes of a warp so that lane l ends up holding the total of
// row (l >> 1) & 15: four exchange-and-halve steps (xor 16, 8, 4, 2) and a final xor 1.
template <typename T>
__device__ __forceinline__ T butterfly16(T (&v)[16], int lane) {
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const T send = hi ? v[j] : v[j + 8];
            const T keep = hi ? v[j + 8] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T send = hi ? v[j] : v[j + 4];
            const T keep = hi ? v[j + 4] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const T send = hi ? v[j] : v[j + 2];
            const T keep = hi ? v[j + 2] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, 4);
        }
    }
    {
        const bool hi = lane & 2;
        const T send = hi ? v[0] : v[1];
        const T keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 2);
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

static_assert(kGroupRows == 16, "the row reduction is a 16-row butterfly");

// Per row of a group and segment, what a lane needs to find the value of its column t:
// lo <= t < lo + len, value at B[base + t].
struct __align__(16) SegSlot {
    int lo, len;
    long long base;
};
// Shared memory of one warp for spmv_group.
struct GroupSmem {
    SegSlot seg[kGroupRows][3];
};

__device__ __forceinline__ GroupDesc load_group(const GroupDesc* d) {
    GroupDesc v;
    const int4* p = reinterpret_cast<const int4*>(d);
    int4* q = reinterpret_cast<int4*>(&v);
    q[0] = __ldg(p);
    q[1] = __ldg(p + 1);
    return v;
}

// y += B x over the stored rows of one row group (warp-cooperative; all 32 lanes; see
// RowMeta and GroupDesc). The warp sweeps the union of the rows' column ranges in column
// pairs, lane l taking pair 32 q + l of the union in pass q; for each of the group's rows the
// lane loads the row's two values at its columns (one aligned 2-vector load, skipped where
// the columns are outside the row's own range), and every value B[s][t] feeds both products:
//   row sums    y[s] += sum_t B[s][t] x[t]   (16 rows in registers, butterfly reduction)
//   column sums y[t] += sum_s B[s][t] x[s]   (the lane's two columns, summed over the rows)
// The halved diagonal makes the two sums count it once. Both are added with atomics.
// Returns this lane's share (in T) of x^T B x: sum_s x[s] rowsum[s] + sum_t colsum[t] x[t].
template <typename T>
__device__ T spmv_group(const GroupDesc& gd, const RowMeta* __restrict__ rmeta,
                        const T* __restrict__ B, const T* x, T* y, int M, int lane,
                        GroupSmem& sm) {
    using T2 = typename Pair<T>::type;
    const int n = gd.n, r0 = gd.r0;
    __syncwarp();
    if (lane < kGroupRows) {
        SegSlot e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) e[k] = SegSlot{0, 0, 0};
        if (lane < n) {
            const int s = r0 + lane;
            const int4 q = __ldg(reinterpret_cast<const int4*>(rmeta + s));
            const unsigned int len = unsigned(q.w);
            const long long off = 2LL * unsigned(q.x);
            const int l0 = 2 * seg_pairs(len, 0), l1 = 2 * seg_pairs(len, 1);
            const int l2 = 2 * seg_pairs(len, 2);
            e[0] = SegSlot{s & ~1, l0, off - (s & ~1)};
            e[1] = SegSlot{q.y, l1, off + l0 - q.y};
            e[2] = SegSlot{q.z, l2, off + l0 + l1 - q.z};
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) sm.seg[lane][k] = e[k];
    }
    const T xrow = lane < n ? ldcg(x + r0 + lane) : T(0);
    T xg[kGroupRows];
#pragma unroll
    for (int i = 0; i < kGroupRows; ++i) xg[i] = __shfl_sync(kFull, xrow, i);
    __syncwarp();
    const int P0 = gd.p0, P1 = gd.p1, PT = gd.p0 + gd.p1 + gd.p2;
    T rp[kGroupRows];
#pragma unroll
    for (int i = 0; i < kGroupRows; ++i) rp[i] = T(0);
    T dot = T(0);
    for (int q0 = 0; q0 < PT; q0 += 32) {
        const int q = q0 + lane;
        const bool act = q < PT;
        const int k = q < P0 ? 0 : (q < P0 + P1 ? 1 : 2);
        const int col = k == 0 ? gd.lo0 + 2 * q
                               : (k == 1 ? gd.lo1 + 2 * (q - P0) : gd.lo2 + 2 * (q - P0 - P1));
        const T xt0 = act && col < M ? ldcg(x + col) : T(0);
        const T xt1 = act && col + 1 < M ? ldcg(x + col + 1) : T(0);
        // every row's two values first (kGroupRows loads in flight), then the products
        T2 v[kGroupRows];
#pragma unroll
        for (int i = 0; i < kGroupRows; ++i) {
            const SegSlot e = sm.seg[i][k];
            const bool ok = act && unsigned(col - e.lo) < unsigned(e.len);
            v[i] = ok ? __ldg(reinterpret_cast<const T2*>(B + e.base + col)) : T2{T(0), T(0)};
        }
        T ca0 = T(0), ca1 = T(0);
#pragma unroll
        for (int i = 0; i < kGroupRows; ++i) {
            rp[i] = fma(v[i].x, xt0, fma(v[i].y, xt1, rp[i]));
            ca0 = fma(v[i].x, xg[i], ca0);
            ca1 = fma(v[i].y, xg[i], ca1);
        }
        // (a widening slot past the last column holds a zero, but 0 * x can be NaN when x
        // is not finite: the bounds are tested, not inferred from the sums)
        if (act && col < M && ca0 != T(0)) {
            atomicAdd(y + col, ca0);
            dot = fma(ca0, xt0, dot);
        }
        if (act && col + 1 < M && ca1 != T(0)) {
            atomicAdd(y + col + 1, ca1);
            dot = fma(ca1, xt1, dot);
        }
    }
    const T tot = butterfly16(rp, lane);       // lanes 2r, 2r+1 hold row r
    const int r = (lane >> 1) & 15;
    const T xr = __shfl_sync(kFull, xrow, r);
    if ((lane & 1) == 0 && r < n) {
        atomicAdd(y + r0 + r, tot);
        dot = fma(tot, xr, dot);
    }
    return dot;
}

// Start moving a group descriptor (32 bytes) into L1 without holding registers for it; a
// later load_group of it then hits L1.
__device__ __forceinline__ void prefetch_group(const GroupDesc* d) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(d)));
}

// Value of B[s][t] (s, t in the same cell; the preconditioner's diagonal blocks) from the
// stored upper rows; the diagonal is stored halved.
template <typename T>
__device__ __forceinline__ T b_same_cell(const RowMeta* __restrict__ rmeta, const T* __restrict__ B,
                                         int s, int t) {
    const int a = min(s, t), b = max(s, t);
    const long long o = 2LL * rmeta[a].off + (b - (a & ~1));
    const T v = B[o];
    return a == b ? T(2) * v : v;
}

template <typename T>
struct CgVec {
    T *x, *u, *p;
    T *r[2], *s[2], *w[2];
    const T* dinv;     // 1 / B_ss, 0 for pinned centres (the mask)
    const T* bjinv;    // inverse diagonal cell blocks (cells with m <= kMaxBlock)
};

// The residual of a row after this iteration's update, r - alpha (w + beta s), evaluated
// with the same operations by every thread that needs it.
template <typename T>
__device__ __forceinline__ T next_r(T r, T s, T w, T ta, T tb) {
    return fma(-ta, fma(tb, s, w), r);
}

// u_i = sum_j Dinv[i][j] r_j over the rows j of row i's cell (row a of the cell's inverse
// block), r_j produced by rj(j) for the cell's rows; or dinv_i r_i for large cells.
template <typename T, typename F>
__device__ __forceinline__ T apply_prec(const Binned& bd, const T* __restrict__ bjinv, int4 cm,
                                        int i, T di, T ri, F rj) {
    if (cm.y > kMaxBlock) return di * ri;
    const int a = i - cm.x;
    const T* drow = bjinv + bd.bjoff[cm.z] + (long long)a * cm.y;
    T ui = T(0);
#pragma unroll 4
    for (int j = 0; j < cm.y; ++j) ui = fma(__ldg(drow + j), rj(cm.x + j), ui);
    return ui;
}

template <typename T>
CgVec<T> cg_vectors(rbf_ctx* ctx) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    T* base = ctx->cgv[slot].as<T>();
    const size_t M = size_t(ctx->M);
    CgVec<T> v;
    v.x = base;
    v.u = base + M;
    v.p = base + 2 * M;
    v.r[0] = base + 3 * M;
    v.r[1] = base + 4 * M;
    v.s[0] = base + 5 * M;
    v.s[1] = base + 6 * M;
    v.w[0] = base + 7 * M;
    v.w[1] = base + 8 * M;
    v.dinv = slot == 0 ? reinterpret_cast<const T*>(ctx->dinv.p)
                       : reinterpret_cast<const T*>(ctx->dinv32.p);
    v.bjinv = slot == 0 ? reinterpret_cast<const T*>(ctx->bjinv.p)
                        : reinterpret_cast<const T*>(ctx->bjinv32.p);
    return v;
}


}  // namespace rbf
