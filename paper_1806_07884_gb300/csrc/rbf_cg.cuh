// Device building blocks of the conjugate-gradient solvers (single system and batched
// tiles): warp and block reductions, the cell-blocked symmetric SpMV of one cell, and the
// block-Jacobi preconditioner application.
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
// Rows of a cell's block whose values one SpMV lane loads together (16-byte loads in flight):
// 4 suits a B that stays in L2 at three CTAs per SM, 8 an HBM-resident B at two CTAs per SM
// (measured).
constexpr int kSpmvGroupL2 = 4;
constexpr int kSpmvGroupHbm = 8;

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

__device__ __forceinline__ int colmap(const RowSeg& sg, int k) {
    return k < sg.l0 ? sg.s0 + k : (k < sg.l0 + sg.l1 ? sg.s1 + (k - sg.l0) : sg.s2 + (k - sg.l0 - sg.l1));
}

// Four consecutive values of a row (16-byte aligned: rows are padded to kRowPad values).
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

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

// y += B x restricted to the stored upper row block of cell c (warp-cooperative; all 32
// lanes). Lane l streams columns 4l .. 4l+3 of each row with vector loads; every loaded
// value B[s][t] feeds both products:
//   row sums    y[s] += sum_t B[s][t] x[t]   (16 rows in registers, butterfly reduction)
//   column sums y[t] += sum_s B[s][t] x[s]   for t outside the diagonal block c x c
//   (the diagonal block is stored in full, so its transposed half is already in the rows)
// and are added with atomics. Returns this lane's share (in T) of x^T B x over the cell's entries:
// sum_s x[s] rowsum[s] + sum_t colsum[t] x[t].
template <typename T, int G>
__device__ T spmv_cell(const CellDesc& cd, const T* __restrict__ B, const T* x, T* y, int lane) {
    const int cs = cd.cs, m = cd.m;
    if (m == 0) return T(0);
    RowSeg sg;
    sg.s0 = cd.s0;
    sg.l0 = cd.l0;
    sg.s1 = cd.s1;
    sg.l1 = cd.l1;
    sg.s2 = cd.s2;
    sg.l2 = cd.l2;
    const int L = sg.l0 + sg.l1 + sg.l2, lp = cd.lp;
    const T* Bc = B + cd.rboff;
    T dot = T(0);
    for (int j0 = 0; j0 < m; j0 += 16) {
        const int mm = min(16, m - j0);
        const T xs_lane = lane < mm ? ldcg(x + cs + j0 + lane) : T(0);
        T rp[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) rp[i] = T(0);
        for (int k0 = 0; k0 < L; k0 += 128) {
            const int kb = k0 + 4 * lane;
            const bool active = kb < L;
            int t[4];
            T xt[4], ca[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                t[q] = kb + q < L ? colmap(sg, kb + q) : -1;
                xt[q] = t[q] >= 0 ? ldcg(x + t[q]) : T(0);
                ca[q] = T(0);
            }
            // Rows are streamed in groups of G whose loads are all issued before any of them
            // is used, so each lane keeps G 16-byte loads in flight. Loads are unconditional:
            // rows past the block's last (i >= mm) re-read row mm-1 and lanes past the row's
            // end (not active) read the row's start -- both valid addresses -- and contribute
            // nothing (x_i = 0 for i >= mm, x_t = 0 and no column update when not active).
            const T* rb = Bc + (long long)j0 * lp + (active ? kb : 0);
            // With 8-row groups, a last group with at most 4 rows left loads only 4 rows (at
            // about 9 rows per cell this saves a quarter of the loads; measured on the batched
            // SpMV, while the 4-row shape is faster without the second code path).
            auto rows = [&](int g0, auto ng) {
                constexpr int NG = decltype(ng)::value;
                T v[NG][4];
#pragma unroll
                for (int i = 0; i < NG; ++i)
                    load4(rb + (long long)min(g0 + i, mm - 1) * lp, v[i]);
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    const T xi = __shfl_sync(kFull, xs_lane, g0 + i);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        rp[g0 + i] = fma(v[i][q], xt[q], rp[g0 + i]);
                        ca[q] = fma(v[i][q], xi, ca[q]);
                    }
                }
            };
#pragma unroll
            for (int g0 = 0; g0 < 16; g0 += G) {
                if (g0 < mm) {                // warp-uniform
                    if constexpr (G == 8) {
                        if (mm - g0 <= 4)
                            rows(g0, std::integral_constant<int, 4>());
                        else
                            rows(g0, std::integral_constant<int, 8>());
                    } else {
                        rows(g0, std::integral_constant<int, G>());
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (kb + q >= m && t[q] >= 0 && ca[q] != T(0)) {
                    atomicAdd(y + t[q], ca[q]);
                    dot = fma(ca[q], xt[q], dot);
                }
            }
        }
        const T tot = butterfly16(rp, lane);       // lanes 2r, 2r+1 hold row r
        const int r = (lane >> 1) & 15;
        const T xr = __shfl_sync(kFull, xs_lane, r);
        if ((lane & 1) == 0 && r < mm) {
            atomicAdd(y + cs + j0 + r, tot);
            dot = fma(tot, xr, dot);
        }
    }
    return dot;
}

// Start moving a cell descriptor (48 bytes, at most two cache lines) into L1 without holding
// registers for it; a later load_desc of it then hits L1.
__device__ __forceinline__ void prefetch_desc(const CellDesc* d) {
    const char* p = reinterpret_cast<const char*>(d);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p + sizeof(CellDesc) - 1));
}

__device__ __forceinline__ CellDesc load_desc(const CellDesc* d) {
    CellDesc v;
    const int4* p = reinterpret_cast<const int4*>(d);
    int4* q = reinterpret_cast<int4*>(&v);
    q[0] = __ldg(p);
    q[1] = __ldg(p + 1);
    q[2] = __ldg(p + 2);
    return v;
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
