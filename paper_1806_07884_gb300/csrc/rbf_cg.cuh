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
// Stride of the CG workspace vectors: M rounded up to a multiple of 4, so every vector starts
// on a 16-byte boundary (the SpMV reads x and adds into y four values at a time).
inline size_t cg_stride(int M) { return (size_t(M) + 3) & ~size_t(3); }

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

// Block-wide sums of NV values of type T, entirely in T (FP32 for the FP32 solver: FP64 on
// this GPU issues at a small fraction of the FP32 rate with a long latency, and the sums of
// the block's few dozen warp totals need no more than the precision of their terms). The
// result, in thread 0, is handed out as double.
template <int NV, typename T>
__device__ __forceinline__ void block_sum_t(const T (&v)[NV], double (&out)[NV]) {
    __shared__ T red[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const T s = warp_sum<T>(v[k]);
        if (lane == 0) red[k][w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = double(warp_sum<T>(lane < nw ? red[k][lane] : T(0)));
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Sum v[0..7] over the 32 lanes of a warp so that lane l ends up holding the total of
// row (l >> 2) & 7: three exchange-and-halve steps (xor 16, 8, 4), then xor 2 and xor 1.
template <typename T>
__device__ __forceinline__ T butterfly8(T (&v)[8], int lane) {
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T send = hi ? v[j] : v[j + 4];
            const T keep = hi ? v[j + 4] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const T send = hi ? v[j] : v[j + 2];
            const T keep = hi ? v[j + 2] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
        const T send = hi ? v[0] : v[1];
        const T keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    v[0] += __shfl_xor_sync(kFull, v[0], 2);
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

static_assert(kGroupRows == 8, "the row reduction is an 8-row butterfly");

// Four consecutive values (16-byte aligned for FP32, 32-byte for FP64).
struct V4f { float x, y, z, w; };
struct V4d { double x, y, z, w; };
template <typename T> struct V4;
template <> struct V4<float> { using type = V4f; };
template <> struct V4<double> { using type = V4d; };
// Values of B, through the read-only data path.
__device__ __forceinline__ V4f ld4(const float* p) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    return V4f{q.x, q.y, q.z, q.w};
}
__device__ __forceinline__ V4d ld4(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    return V4d{a.x, a.y, b.x, b.y};
}
// x[t..t+3] (t a multiple of 4; the vector is 16-byte aligned), zero past M
template <typename T>
__device__ __forceinline__ typename V4<T>::type ldx4(const T* x, int t, int M) {
    using R = typename V4<T>::type;
    if (t + 3 < M) {
        if constexpr (sizeof(T) == 4) {
            const float4 q = __ldcg(reinterpret_cast<const float4*>(x + t));
            return R{q.x, q.y, q.z, q.w};
        } else {
            const double2 a = __ldcg(reinterpret_cast<const double2*>(x + t));
            const double2 b = __ldcg(reinterpret_cast<const double2*>(x + t + 2));
            return R{a.x, a.y, b.x, b.y};
        }
    }
    return R{t < M ? ldcg(x + t) : T(0), t + 1 < M ? ldcg(x + t + 1) : T(0),
             t + 2 < M ? ldcg(x + t + 2) : T(0), t + 3 < M ? ldcg(x + t + 3) : T(0)};
}
// y[t..t+3] += v (t a multiple of 4), nothing past M or for zero parts
template <typename T>
__device__ __forceinline__ void atomic_add4(T* y, int t, int M, const typename V4<T>::type& v) {
    if constexpr (sizeof(T) == 4) {
        if (t + 3 < M) {
            if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f)
                atomicAdd(reinterpret_cast<float4*>(y + t), make_float4(v.x, v.y, v.z, v.w));
            return;
        }
    }
    if (t < M && v.x != T(0)) atomicAdd(y + t, v.x);
    if (t + 1 < M && v.y != T(0)) atomicAdd(y + t + 1, v.y);
    if (t + 2 < M && v.z != T(0)) atomicAdd(y + t + 2, v.z);
    if (t + 3 < M && v.w != T(0)) atomicAdd(y + t + 3, v.w);
}

// Per row of a group and segment, what a lane needs to find the value of its column t:
// lo <= t < lo + len, value at Bg[rel + t] with Bg the group's first stored value.
struct SegSlot {
    int lo, len, rel, pad;
};
// Shared memory of one warp for spmv_group: two record slots (the current group's, and the
// next group's arriving) and the current group's segment slots.
struct GroupSmem {
    int4 rec[2][kGroupRecInt4];
    SegSlot seg[kGroupRows][3];
};

// Start copying group g's record (GroupRec: description and the rows' RowMeta) into record
// slot b of the warp's shared memory, one 16-byte asynchronous copy per lane for lanes <
// kGroupRecInt4, as one commit group of every lane; group_wait makes it visible.
__device__ __forceinline__ void stage_group(const GroupRec* __restrict__ gdesc, int g,
                                            GroupSmem& sm, int b, int lane) {
    if (lane < kGroupRecInt4) {
        const unsigned dst = unsigned(__cvta_generic_to_shared(&sm.rec[b][lane]));
        const int4* src = reinterpret_cast<const int4*>(gdesc + g) + lane;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// Wait for all but the `pending` most recent commit groups of this lane, then make the warp's
// copies visible to every lane.
template <int pending>
__device__ __forceinline__ void group_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(pending) : "memory");
    __syncwarp();
}

// y += B x over the stored rows of one row group (warp-cooperative; all 32 lanes; see
// RowMeta and GroupDesc), given its record staged by stage_group. The warp sweeps the union of
// the rows' column ranges in column quads, lane l taking quad 32 q + l of the union in pass q
// (one pass for unions up to 128 columns); for each of the group's rows the lane loads the
// row's four values at its columns (one aligned 4-vector load, skipped where the columns are
// outside the row's own range), and every value B[s][t] feeds both products:
//   row sums    y[s] += sum_t B[s][t] x[t]   (8 rows in registers, butterfly reduction)
//   column sums y[t] += sum_s B[s][t] x[s]   (the lane's four columns, summed over the rows,
//                                             added with one 4-vector atomic)
// The halved diagonal makes the two sums count it once.
// Returns this lane's share (in T) of x^T B x: sum_s x[s] rowsum[s] + sum_t colsum[t] x[t].
template <typename T>
__device__ T spmv_group(int b, const T* __restrict__ B, const T* x, T* y, int M, int lane,
                        GroupSmem& sm) {
    using R4 = typename V4<T>::type;
    const int4 h0 = sm.rec[b][0], h1 = sm.rec[b][1];
    const int r0 = h0.x, n = h0.y;
    const int lo0 = h0.z, Q0 = h0.w, lo1 = h1.x, Q1 = h1.y, lo2 = h1.z, QT = h0.w + h1.y + h1.w;
    // the group's first stored value (row r0, column r0 & ~3)
    const long long gbase = 4LL * unsigned(sm.rec[b][2].x);
    // x of row lane, in flight with the values below
    const T xrow = lane < n ? ldcg(x + r0 + lane) : T(0);
    if (lane < kGroupRows) {
        SegSlot e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) e[k] = SegSlot{0, 0, 0, 0};
        if (lane < n) {
            const int4 meta = sm.rec[b][2 + lane];
            const int s = r0 + lane;
            const unsigned int len = unsigned(meta.w);
            const int rel = int(4LL * unsigned(meta.x) - gbase);
            const int l0 = 4 * seg_quads(len, 0), l1 = 4 * seg_quads(len, 1);
            const int l2 = 4 * seg_quads(len, 2);
            e[0] = SegSlot{s & ~3, l0, rel - (s & ~3), 0};
            e[1] = SegSlot{meta.y, l1, rel + l0 - meta.y, 0};
            e[2] = SegSlot{meta.z, l2, rel + l0 + l1 - meta.z, 0};
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) sm.seg[lane][k] = e[k];
    }
    __syncwarp();
    const T* Bg = B + gbase;
    T rp[kGroupRows];
#pragma unroll
    for (int i = 0; i < kGroupRows; ++i) rp[i] = T(0);
    T dot = T(0);
    for (int qq = 0; qq < QT; qq += 32) {
        const int q = qq + lane;
        const bool act = q < QT;
        const int k = q < Q0 ? 0 : (q < Q0 + Q1 ? 1 : 2);
        const int col = k == 0 ? lo0 + 4 * q : (k == 1 ? lo1 + 4 * (q - Q0) : lo2 + 4 * (q - Q0 - Q1));
        const R4 xt = act ? ldx4<T>(x, col, M) : R4{T(0), T(0), T(0), T(0)};
        // every row's four values first (kGroupRows loads in flight), then the products
        R4 v[kGroupRows];
#pragma unroll
        for (int i = 0; i < kGroupRows; ++i) {
            const SegSlot e = sm.seg[i][k];
            const bool ok = act && unsigned(col - e.lo) < unsigned(e.len);
            v[i] = ok ? ld4(Bg + (e.rel + col)) : R4{T(0), T(0), T(0), T(0)};
        }
        R4 ca{T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < kGroupRows; ++i) {
            const T xi = __shfl_sync(kFull, xrow, i);   // x of row i
            rp[i] = fma(v[i].x, xt.x, fma(v[i].y, xt.y, fma(v[i].z, xt.z, fma(v[i].w, xt.w, rp[i]))));
            ca.x = fma(v[i].x, xi, ca.x);
            ca.y = fma(v[i].y, xi, ca.y);
            ca.z = fma(v[i].z, xi, ca.z);
            ca.w = fma(v[i].w, xi, ca.w);
        }
        if (act) {
            // (a widening slot past the last column holds a zero, but 0 * x can be NaN when x
            // is not finite: atomic_add4 tests the bounds itself)
            atomic_add4<T>(y, col, M, ca);
            dot = fma(ca.x, xt.x, fma(ca.y, xt.y, fma(ca.z, xt.z, fma(ca.w, xt.w, dot))));
        }
    }
    const T tot = butterfly8(rp, lane);        // lanes 4r .. 4r+3 hold row r
    const int r = (lane >> 2) & 7;
    const T xr = __shfl_sync(kFull, xrow, r);
    if ((lane & 3) == 0 && r < n) {
        atomicAdd(y + r0 + r, tot);
        dot = fma(tot, xr, dot);
    }
    __syncwarp();   // the segment slots and this record slot are free for the next group
    return dot;
}

// Value of B[s][t] (s, t in the same cell; the preconditioner's diagonal blocks) from the
// stored upper rows; the diagonal is stored halved.
template <typename T>
__device__ __forceinline__ T b_same_cell(const RowMeta* __restrict__ rmeta, const T* __restrict__ B,
                                         int s, int t) {
    const int a = min(s, t), b = max(s, t);
    const long long o = 4LL * rmeta[a].off + (b - (a & ~3));
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
// block), r_j produced by rj(j) for the cell's rows; or dinv_i r_i for large cells. kB columns
// at a time: every load of a batch is in flight before its products, which are then summed in
// column order (zeros past the block add nothing), so every kB gives the same bits.
template <typename T, int kB = 4, typename F>
__device__ __forceinline__ T apply_prec(const Binned& bd, const T* __restrict__ bjinv, int4 cm,
                                        int i, T di, T ri, F rj) {
    if (cm.y > kMaxBlock) return di * ri;
    const int a = i - cm.x;
    // the inverse block is stored exactly symmetric: row a is read as column a, so that the
    // cell's threads (consecutive a) read consecutive words
    const T* dcol = bjinv + bd.bjoff[cm.z] + a;
    T ui = T(0);
    for (int j0 = 0; j0 < cm.y; j0 += kB) {
        T dv[kB], rv[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) dv[k] = j0 + k < cm.y ? __ldg(dcol + (long long)(j0 + k) * cm.y) : T(0);
#pragma unroll
        for (int k = 0; k < kB; ++k) rv[k] = j0 + k < cm.y ? rj(cm.x + j0 + k) : T(0);
#pragma unroll
        for (int k = 0; k < kB; ++k) ui = fma(dv[k], rv[k], ui);
    }
    return ui;
}

template <typename T>
CgVec<T> cg_vectors(rbf_ctx* ctx) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    T* base = ctx->cgv[slot].as<T>();
    const size_t M = cg_stride(ctx->M);
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
