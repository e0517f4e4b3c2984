// Step (d): solve the normal equations B c = b (Section 2) by preconditioned conjugate
// gradients on the stored upper triangle of B. The preconditioner is block-Jacobi over the
// cells of the grid: the inverse of each cell's diagonal block B[c, c] (the centres of one
// cell share most of their support and are the strongest couplings of B).
//
// SpMV y = B x over the stored upper triangle (Section 5 keeps only the upper triangle), one
// warp per row group (persistent warps striding over the groups): the rows of a group are up
// to 16 consecutive centres of one cell row, each storing the three column ranges of the
// sorted order that can hold its nonzeros (about 1.3 times the true nonzeros, against about
// twice for dense cell-pair blocks); the warp sweeps the union of the rows' ranges in column
// pairs with aligned 2-vector loads, and each value feeds both the row product (16 rows held in
// registers, summed across lanes by a butterfly transpose-reduction) and the transposed
// product of the lower triangle (column sums over the group's rows, added to y with atomics).
// HBM and L2 see each stored value once per SpMV and no transposed reads are needed. The same
// pass yields x^T B x locally.
//
// The CG iteration uses the Chronopoulos-Gear recurrences: one SpMV and one fused pair of
// reductions per iteration, as two kernels. The SpMV kernel accumulates delta = u^T B u
// with warp atomics spread over 64 slots; the update kernel derives alpha and beta from
// them at its start, updates the vectors one thread per row (each thread recomputes the new
// residual of its cell's rows to apply its row of the block inverse, so r, s and w are
// double-buffered by iteration parity), and its last block to finish reduces gamma and
// (r, r) and advances the scalar state in device memory. The iteration loop is a CUDA graph
// with a conditional WHILE node: the host launches the solve once and reads the state once.
//
// Precision RBF_FP32_REFINE: B is FP32 and the inner CG runs in FP32 on the correction
// equation B d = r; the residual r = A^T (h - A c) is recomputed matrix-free in FP64
// from the points (so the refinement converges to the FP64 least-squares solution, not
// to that of the rounded B), and c += d is applied in FP64.
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "rbf_cg.cuh"

namespace rbf {

constexpr int kAccSlots = 64;

// Scalars carried between iterations, double-buffered by iteration parity: iteration k
// reads slot k & 1 and block 0 of its update kernel writes slot (k + 1) & 1.
struct CgSlot {
    double gamma_prev, alpha_prev;
    int it, state;
};
struct CgScalars {
    double bb, tol2, bscale;     // (b, b); parameters written by the host before each solve
    int maxit, passes;           // passes: loop passes of the solve graph so far
    unsigned int ticket, pad2;   // last-block-done counter of the start kernel
    CgSlot sl[2];
    double out_rr, out_gamma;    // result, written when the solve stops
    int out_it, out_state;
    double acc_delta[2][kAccSlots];   // u^T B u of the SpMV of each parity, spread over slots
    // grid barrier of the persistent solve kernel: arrivals so far (never reset within a
    // solve: barrier n completes at n times the grid's blocks), timed-out flag
    unsigned long long bar_count;
    int bar_err, bar_pad;
};


namespace {

// Threads per block of the CG vector kernels: 512, so a solve of 100 k rows runs ~200 blocks,
// whose per-block partial sums every update block's prologue adds in one batch of loads.
constexpr int kVecThreads = 512;

// Stores this block's NV partial sums; returns true in the single last block to finish,
// whose thread 0 then holds the totals, summed in block order, in tot[].
template <int NV>
__device__ bool last_block_total(double (&v)[NV], double* partial, unsigned int* ticket,
                                 double (&tot)[NV]) {
    __shared__ bool amlast;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[NV * blockIdx.x + k] = v[k];
        __threadfence();
        amlast = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!amlast) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partial[NV * b + k]);
    block_sum<NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = acc[k];
        *ticket = 0;
    }
    return true;
}

// Standalone SpMV y += B x (persistent warps striding over the row groups; y zeroed by the
// caller).
template <typename T>
__global__ void __launch_bounds__(kSpmvWarps * 32, sizeof(T) == 4 ? 3 : 2)
    k_spmv(Binned bd, const T* __restrict__ B, const T* __restrict__ x, T* __restrict__ y) {
    __shared__ GroupSmem gsm[kSpmvWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = gridDim.x * kSpmvWarps;
    int q = blockIdx.x * kSpmvWarps + wid;
    if (q >= bd.ngroup) return;
    // the next group's record is copied while this group's rows stream
    stage_group(bd.gdesc, q, gsm[wid], 0, lane);
    for (int b = 0; q < bd.ngroup; q += nw, b ^= 1) {
        if (q + nw < bd.ngroup) {
            stage_group(bd.gdesc, q + nw, gsm[wid], b ^ 1, lane);
            group_wait<1>();
        } else {
            group_wait<0>();
        }
        spmv_group<T>(b, B, x, y, bd.M, lane, gsm[wid]);
    }
}


// Preconditioned CG in the Chronopoulos-Gear form (one SpMV and two reductions per
// iteration), for B x = bscale * b:
//   r = b - B x, u = D^-1 r, w = B u, gamma = (r, u), delta = (w, u) = u^T B u
//   beta = gamma / gamma_prev (0 at the start), alpha = gamma / (delta - beta gamma / alpha_prev)
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r
// It stops when (r, r) <= tol^2 (b, b).

// w += B u (w zero on entry); delta = u^T B u into the slots of sc->acc_delta. It does not
// wait for the solver's state: after the solve stops (at most kItersPerBody - 1 SpMVs before
// the loop condition is read) its w and delta go unused, and the next start resets the slots.
template <typename T>
__global__ void __launch_bounds__(kSpmvWarps * 32, sizeof(T) == 4 ? 3 : 2)
    k_cg_spmv(Binned bd, const T* __restrict__ B, const T* __restrict__ u, T* __restrict__ w,
              int P, CgScalars* __restrict__ sc) {
    __shared__ GroupSmem gsm[kSpmvWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kSpmvWarps + wid;
    const int nw = gridDim.x * kSpmvWarps;
    T d = T(0);
    if (gw < bd.ngroup) {
        // the next group's record is copied while this group's rows stream
        stage_group(bd.gdesc, gw, gsm[wid], 0, lane);
        int b = 0;
        for (int q = gw; q < bd.ngroup; q += nw, b ^= 1) {
            if (q + nw < bd.ngroup) {
                stage_group(bd.gdesc, q + nw, gsm[wid], b ^ 1, lane);
                group_wait<1>();
            } else {
                group_wait<0>();
            }
            d += spmv_group<T>(b, B, u, w, bd.M, lane, gsm[wid]);
        }
    }
    d = warp_sum<T>(d);
    if (lane == 0 && d != T(0)) atomicAdd(&sc->acc_delta[P][gw & (kAccSlots - 1)], double(d));
}

// One thread per row i. Prologue (warp 0 of every block, identical results in all blocks):
// gamma_k and (r_k, r_k) from the previous kernel's per-block partials, delta_k from the
// SpMV's slots, the stopping test, then beta_k and alpha_k; block 0 writes the next slot.
// Body: s, p, x, r updated; u = D^-1 r with the cell's new residuals from shared memory (rows
// of the cell outside the block's chunk recomputed with the same operations); w of the other
// parity zeroed for the next SpMV; per-block partials of gamma_{k+1} and (r_{k+1}, r_{k+1}).
// P is the parity k & 1.
// The scalar step is taken in the solver's precision T (FP32 for the FP32 inner solver, whose
// iterates the FP64 refinement corrects): every block repeats it, and FP64 issues at 1/64
// of the FP32 rate on this GPU.
constexpr int kPartBatch = 8;   // per-block partials loaded per lane before they are summed
// With the linear polynomial of Eq. 10 (pd non-null) the system is bordered by the three
// polynomial rows: the w of row i gains E_i . u_k (E = A^T P in the solver's precision, u_k the
// polynomial part of u), the polynomial rows' w_k = E^T u + G u_k (G = P^T P; E^T u from the
// previous kernel's per-block partials pe), and delta gains 2 (E^T u) . u_k + u_k^T G u_k.
// Block 0's thread 0 advances the three rows' recurrences (FP64) with u_k = G^-1 r_k.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_update(Binned bd, CgVec<T> v, int P, CgScalars* __restrict__ sc,
                T* __restrict__ pbuf, const T* __restrict__ E, T* __restrict__ pe,
                PolyDev* __restrict__ pd) {
    __shared__ T s_ab[2];
    __shared__ int s_go;
    __shared__ T s_uk[3];
    __shared__ double s_pg[2];   // block 0: the polynomial rows' share of gamma and (r, r)
    static_assert(kAccSlots == 64, "two slots per lane");
    const int nblk = gridDim.x;
    const int M = bd.M;
    const T* __restrict__ rP = P ? v.r[1] : v.r[0];
    const T* __restrict__ sP = P ? v.s[1] : v.s[0];
    const T* __restrict__ wP = P ? v.w[1] : v.w[0];
    // the first chunk's row values, loaded before the prologue so that their latency overlaps it
    const int i_first = blockIdx.x * kVecThreads + threadIdx.x;
    T f_d = T(0), f_w = T(0), f_s = T(0), f_p = T(0), f_u = T(0), f_r = T(0), f_x = T(0);
    int4 f_cm = make_int4(0, 0, 0, 0);
    if (i_first < M) {
        f_d = v.dinv[i_first];
        f_w = wP[i_first];
        f_s = sP[i_first];
        f_p = v.p[i_first];
        f_u = v.u[i_first];
        f_r = rP[i_first];
        f_x = v.x[i_first];
        f_cm = bd.crow[i_first];
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const CgSlot sl = sc->sl[P];
        // The partials (gamma, (r, r)) of block b are adjacent: one vector load each, up to
        // kPartBatch per lane in flight before the first add (the sums keep block order).
        using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        const T2* pb = reinterpret_cast<const T2*>(pbuf + size_t(P) * 2 * nblk);
        T g = T(0), rr = T(0);
        T d = T(__ldcg(&sc->acc_delta[P][lane])) + T(__ldcg(&sc->acc_delta[P][lane + 32]));
        for (int b0 = lane; b0 < nblk; b0 += 32 * kPartBatch) {
            T2 pv[kPartBatch];
#pragma unroll
            for (int k = 0; k < kPartBatch; ++k) {
                const int b = b0 + 32 * k;
                pv[k] = b < nblk ? __ldcg(pb + b) : T2{T(0), T(0)};
            }
#pragma unroll
            for (int k = 0; k < kPartBatch; ++k) {
                g += pv[k].x;
                rr += pv[k].y;
            }
        }
        T et[3] = {T(0), T(0), T(0)};
        if (pd) {
            const T* pp = pe + size_t(P) * 4 * nblk;
            for (int b = lane; b < nblk; b += 32)
#pragma unroll
                for (int j = 0; j < 3; ++j) et[j] += __ldcg(pp + 4 * b + j);
#pragma unroll
            for (int j = 0; j < 3; ++j) et[j] = warp_sum<T>(et[j]);
        }
        int state = sl.state;
        if (state != kRunning) g = rr = d = T(0);
        g = warp_sum<T>(g);
        rr = warp_sum<T>(rr);
        d = warp_sum<T>(d);
        double wk[3] = {0.0, 0.0, 0.0};
        if (pd && lane == 0) {
            // w_k = E^T u + G u_k; delta += 2 (E^T u) . u_k + u_k^T G u_k
            double dp = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double ui = __ldcg(&pd->uk[P][i]);
                double gu = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j) gu = fma(pd->gp[3 * i + j], __ldcg(&pd->uk[P][j]), gu);
                wk[i] = double(et[i]) + gu;
                dp += ui * (2.0 * double(et[i]) + gu);
                s_uk[i] = T(ui);
            }
            if (state == kRunning) d += T(dp);
        }
        if (lane == 0) {
            T alpha = T(0), beta = T(0);
            const int was = state;
            if (state == kRunning) {
                if (!isfinite(g) || !isfinite(rr)) {
                    state = kBreakdown;
                } else if (rr <= T(sc->tol2) * T(sc->bb)) {
                    state = kConverged;
                } else if (sl.it >= sc->maxit) {
                    state = kMaxIt;
                } else {
                    beta = sl.it == 0 ? T(0) : g / T(sl.gamma_prev);
                    const T den = sl.it == 0 ? d : d - beta * g / T(sl.alpha_prev);
                    alpha = g / den;
                    if (!(den > T(0)) || !isfinite(alpha)) state = kBreakdown;
                }
            }
            s_ab[0] = alpha;
            s_ab[1] = beta;
            s_go = state == kRunning;
            if (pd && blockIdx.x == 0 && state == kRunning) {
                // the three polynomial rows: s = w + beta s, p = u + beta p, x += alpha p,
                // r -= alpha s, u = G^-1 r (FP64)
                double rn[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double sk = fma(double(beta), pd->sk[i], wk[i]);
                    const double pk = fma(double(beta), pd->pk[i], __ldcg(&pd->uk[P][i]));
                    pd->sk[i] = sk;
                    pd->pk[i] = pk;
                    pd->xk[i] = fma(double(alpha), pk, pd->xk[i]);
                    rn[i] = fma(-double(alpha), sk, pd->rkc[i]);
                    pd->rkc[i] = rn[i];
                }
                double pg = 0.0, prr = 0.0;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    double un = 0.0;
#pragma unroll
                    for (int j = 0; j < 3; ++j) un = fma(pd->ginv[3 * i + j], rn[j], un);
                    pd->uk[P ^ 1][i] = un;
                    pg = fma(rn[i], un, pg);
                    prr = fma(rn[i], rn[i], prr);
                }
                s_pg[0] = pg;
                s_pg[1] = prr;
            }
            if (blockIdx.x == 0) {
                CgSlot nx = sl;
                nx.state = state;
                if (state == kRunning) {
                    nx.gamma_prev = double(g);
                    nx.alpha_prev = double(alpha);
                    nx.it = sl.it + 1;
                }
                sc->sl[P ^ 1] = nx;
                if (was == kRunning && state != kRunning) {
                    sc->out_rr = double(rr);
                    sc->out_gamma = double(g);
                    sc->out_it = sl.it;
                    sc->out_state = state;
                }
            }
        }
        if (blockIdx.x == 0) {
            sc->acc_delta[P ^ 1][lane] = 0.0;
            sc->acc_delta[P ^ 1][lane + 32] = 0.0;
        }
    }
    __syncthreads();
    if (!s_go) return;
    const T ta = s_ab[0], tb = s_ab[1];
    T* __restrict__ rQ = P ? v.r[0] : v.r[1];
    T* __restrict__ sQ = P ? v.s[0] : v.s[1];
    T* __restrict__ wQ = P ? v.w[0] : v.w[1];
    T acc[2] = {T(0), T(0)};
    T eacc[3] = {T(0), T(0), T(0)};
    const T uk0 = pd ? s_uk[0] : T(0), uk1 = pd ? s_uk[1] : T(0), uk2 = pd ? s_uk[2] : T(0);
    // w_j of the bordered system: B u + E_j . u_k
    auto wfull = [&](int j, T wj) -> T {
        return pd ? fma(E[j], uk0, fma(E[M + j], uk1, fma(E[2 * M + j], uk2, wj))) : wj;
    };
    // The new residual of each row of the chunk is kept in shared memory for the block-Jacobi
    // step; rows of a cell outside the chunk are recomputed with the same operations.
    __shared__ T rsm[kVecThreads];
    // The row values of the block's next chunk are loaded at the start of the current one, so
    // that their latency overlaps this chunk's work (with M far beyond the grid, each block
    // takes several chunks and the update is bound by these round trips).
    T c_d = f_d, c_w = f_w, c_s = f_s, c_p = f_p, c_u = f_u, c_r = f_r, c_x = f_x;
    int4 c_cm = f_cm;
    const int stride = gridDim.x * kVecThreads;
    for (int base = blockIdx.x * kVecThreads; base < M; base += stride) {
        const int i = base + threadIdx.x;
        const bool valid = i < M;
        const int in = i + stride;
        T n_d = T(0), n_w = T(0), n_s = T(0), n_p = T(0), n_u = T(0), n_r = T(0), n_x = T(0);
        int4 n_cm = make_int4(0, 0, 0, 0);
        if (in < M) {
            n_d = v.dinv[in];
            n_w = wP[in];
            n_s = sP[in];
            n_p = v.p[in];
            n_u = v.u[in];
            n_r = rP[in];
            n_x = v.x[in];
            n_cm = bd.crow[in];
        }
        T di = T(0), ri = T(0);
        if (valid) {
            di = c_d;
            const T wi = di == T(0) ? T(0) : wfull(i, c_w);
            const T si = fma(tb, c_s, wi);
            const T pi = fma(tb, c_p, c_u);
            ri = di == T(0) ? T(0) : fma(-ta, si, c_r);
            sQ[i] = si;
            v.p[i] = pi;
            v.x[i] = fma(ta, pi, c_x);
            rQ[i] = ri;
            wQ[i] = T(0);
        }
        rsm[threadIdx.x] = ri;
        __syncthreads();
        if (valid) {
            // rows of pinned centres carry zeros in the inverse block, so r_j need no mask
            const T ui = apply_prec<T>(bd, v.bjinv, c_cm, i, di, ri, [&](int j) {
                const int o = j - base;
                return o >= 0 && o < kVecThreads ? rsm[o]
                                                 : next_r(rP[j], sP[j], wfull(j, wP[j]), ta, tb);
            });
            v.u[i] = ui;
            acc[0] = fma(ri, ui, acc[0]);
            acc[1] = fma(ri, ri, acc[1]);
            if (pd) {
                eacc[0] = fma(E[i], ui, eacc[0]);
                eacc[1] = fma(E[M + i], ui, eacc[1]);
                eacc[2] = fma(E[2 * M + i], ui, eacc[2]);
            }
        }
        c_d = n_d;
        c_w = n_w;
        c_s = n_s;
        c_p = n_p;
        c_u = n_u;
        c_r = n_r;
        c_x = n_x;
        c_cm = n_cm;
        __syncthreads();
    }
    double tot[2];
    block_sum_t<2, T>(acc, tot);
    if (threadIdx.x == 0) {
        if (pd && blockIdx.x == 0) {
            tot[0] += s_pg[0];
            tot[1] += s_pg[1];
        }
        T* pb = pbuf + size_t(P ^ 1) * 2 * nblk;
        pb[2 * blockIdx.x] = T(tot[0]);
        pb[2 * blockIdx.x + 1] = T(tot[1]);
    }
    if (pd) {
        double et[3];
        block_sum_t<3, T>(eacc, et);
        if (threadIdx.x == 0) {
            T* pp = pe + size_t(P ^ 1) * 4 * nblk + 4 * blockIdx.x;
#pragma unroll
            for (int j = 0; j < 3; ++j) pp[j] = T(et[j]);
        }
    }
}

// Start: r = bscale b - B x0 (B x0 in w[1] when use_x0), u = D^-1 r, p = s[0] = w[0] = 0
// (x = 0 without a start vector); per-block partials of gamma_0 and (r_0, r_0) for the first
// update, and (b, b) reduced by the last block, which also sets the parity-0 slot.
// With the polynomial (pd): its three rows start from r_k = bscale * pd->bk (x_k = 0, no start
// vector), u_k = G^-1 r_k; block 0 adds their shares of gamma, (r, r) and (b, b); the
// per-block partials of E^T u of parity 0 are written for the first update.
template <typename T, typename TB>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_init(Binned bd, CgVec<T> v, const TB* __restrict__ b, int use_x0,
              CgScalars* __restrict__ sc, T* __restrict__ pbuf, double* __restrict__ partial,
              const T* __restrict__ E, T* __restrict__ pe, PolyDev* __restrict__ pd) {
    const double bscale = sc->bscale;
    const T* __restrict__ w1 = v.w[1];
    auto r0 = [&](int j) -> T {
        const T bj = T(double(b[j]) * bscale);
        return use_x0 ? bj - w1[j] : bj;
    };
    T acc[2] = {T(0), T(0)};
    T eacc[3] = {T(0), T(0), T(0)};
    double bb[1] = {0.0}, tot[1];
    const int M = bd.M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const T di = v.dinv[i];
        const T bi = di == T(0) ? T(0) : T(double(b[i]) * bscale);
        const T ri = di == T(0) ? T(0) : r0(i);
        const T ui = apply_prec<T>(bd, v.bjinv, bd.crow[i], i, di, ri, r0);
        if (!use_x0) v.x[i] = T(0);
        v.r[0][i] = ri;
        v.u[i] = ui;
        v.p[i] = T(0);
        v.s[0][i] = T(0);
        v.w[0][i] = T(0);
        acc[0] = fma(ri, ui, acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
        bb[0] += double(bi) * double(bi);
        if (pd) {
            eacc[0] = fma(E[i], ui, eacc[0]);
            eacc[1] = fma(E[M + i], ui, eacc[1]);
            eacc[2] = fma(E[2 * M + i], ui, eacc[2]);
        }
    }
    if (pd && blockIdx.x == 0 && threadIdx.x == 0) {
        double rk[3];
        for (int i = 0; i < 3; ++i) {
            rk[i] = pd->bk[i] * bscale;
            pd->rkc[i] = rk[i];
            pd->xk[i] = pd->pk[i] = pd->sk[i] = 0.0;
            bb[0] += rk[i] * rk[i];
        }
        for (int i = 0; i < 3; ++i) {
            double un = 0.0;
            for (int j = 0; j < 3; ++j) un = fma(pd->ginv[3 * i + j], rk[j], un);
            pd->uk[0][i] = un;
            pd->uk[1][i] = 0.0;
            acc[0] += T(rk[i] * un);
            acc[1] += T(rk[i] * rk[i]);
        }
    }
    double at[2];
    block_sum_t<2, T>(acc, at);
    if (threadIdx.x == 0) {
        pbuf[2 * blockIdx.x] = T(at[0]);
        pbuf[2 * blockIdx.x + 1] = T(at[1]);
    }
    if (pd) {
        double et[3];
        block_sum_t<3, T>(eacc, et);
        if (threadIdx.x == 0)
            for (int j = 0; j < 3; ++j) pe[4 * blockIdx.x + j] = T(et[j]);
    }
    if (last_block_total<1>(bb, partial, &sc->ticket, tot) && threadIdx.x == 0) {
        sc->bb = tot[0];
        CgSlot s0;
        s0.gamma_prev = 1.0;
        s0.alpha_prev = 1.0;
        s0.it = 0;
        s0.state = kRunning;
        sc->sl[0] = s0;
        sc->sl[1] = s0;
        sc->out_state = kRunning;
    }
}

// Loop condition of the solve graph (after an even number of iterations the next slot is
// slot 0): keep iterating while the state is running.
__global__ void k_cg_cond(CgScalars* __restrict__ sc, cudaGraphConditionalHandle h) {
    // every running pass advances the iteration count, which stops at maxit; the pass bound
    // ends the loop even if the state were never to leave "running"
    const int passes = ++sc->passes;
    const bool more = sc->sl[0].state == kRunning && passes <= sc->maxit / kItersPerBody + 2;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------------------
// Persistent solve: the whole CG loop of one system in a single cooperative launch (one block
// per SM, every block resident), the SpMV and the update of each iteration separated by grid
// barriers instead of kernel boundaries. Per iteration k (parity P = k & 1):
//   SpMV phase   w_P += B u over the block's contiguous range of row groups (each warp's
//                first group fixed and staged during the previous barrier, the rest taken
//                from a shared-memory counter, so the warps of a block finish together);
//                the block's share of delta_k = u^T B u summed warp by warp into one
//                per-block partial; each thread then loads its first row's vectors
//   barrier
//   scalar step  every block sums the per-block delta partials, and has gamma_k, (r_k, r_k)
//                from the previous update's partials, both in block order: identical alpha,
//                beta and stop decision in every block
//   update phase the rows (as k_cg_update), per-block partials of gamma_{k+1}, (r_{k+1},
//                r_{k+1}); w of the other parity zeroed
//   barrier
// Vectors written inside the kernel are read through L2 (ld.global.cg), never from a stale L1
// line. The barrier is one 64-bit arrival counter in device memory: thread 0 of each block adds
// 1 with release semantics (the block's writes, ordered before it by __syncthreads, become
// visible with it) and polls with acquire loads until the count reaches the barrier's target.
// Every wait is bounded (kBarrierTimeoutNs by the global timer); a waiter that runs out raises
// bar_err, on which every other waiter gives up too, and all blocks leave the loop (the host
// reports RBF_ERR_TIMEOUT). Cooperative launch rejects a grid that cannot be resident at once,
// so no block waits for one that has not started.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

template <typename T>
struct PersistCfg {
    // FP32: 24 warps per SM at <= 85 registers; FP64: 16 warps at <= 128
    static constexpr int threads = sizeof(T) == 4 ? 768 : 512;
    static constexpr int warps = threads / 32;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// All blocks of the grid; `target` = the arrivals that complete this barrier. False (in every
// thread of the block) if the wait ran out or another block's did.
__device__ bool grid_barrier(CgScalars* sc, unsigned long long target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add_u64(&sc->bar_count, 1ull);
        if (ld_acquire_u64(&sc->bar_count) < target) {
            const unsigned long long t0 = global_ns();
            unsigned n = 0;
            while (ld_acquire_u64(&sc->bar_count) < target) {
                if ((++n & 15u) == 0 &&
                    (*reinterpret_cast<volatile int*>(&sc->bar_err) != 0 ||
                     global_ns() - t0 > kBarrierTimeoutNs)) {
                    atomicExch(&sc->bar_err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(PersistCfg<T>::threads, 1)
    k_cg_persist(Binned bd, CgVec<T> v, const T* __restrict__ B, CgScalars* __restrict__ sc,
                 const T* __restrict__ pinit, int ninit, T* __restrict__ pbuf, int bar_extra) {
    constexpr int NT = PersistCfg<T>::threads, NW = PersistCfg<T>::warps;
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    __shared__ GroupSmem gsm[NW];
    __shared__ T s_dw[NW];    // per-warp delta partials
    __shared__ int s_next[2]; // next group of the block's range to take, per parity
    __shared__ T s_ab[2];     // alpha_k, beta_k
    __shared__ int s_go;
    __shared__ T rsm[NT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nblk = int(gridDim.x);
    // arrivals per barrier: the grid, plus a test hook's blocks that never come
    const unsigned long long narrive = unsigned(nblk) + unsigned(bar_extra);
    unsigned long long target = 0;
    const int M = bd.M, ngroup = bd.ngroup;

    // This block's row groups [g0, g1), equal shares by count (a group's time is mostly its
    // fixed latency, not its bytes); warp wid starts at g0 + wid, the others are taken from a
    // shared-memory counter. Its rows [rb0, rb1): equal shares moved back to the start of
    // their cell, so that every cell's rows (the preconditioner's blocks) lie in one block and
    // one chunk of it.
    const int g0 = int((long long)ngroup * blockIdx.x / nblk);
    const int g1 = int((long long)ngroup * (blockIdx.x + 1) / nblk);
    auto cell_start = [&](int r) -> int {
        if (r >= M) return M;
        const int4 cm = __ldg(bd.crow + r);
        return cm.y <= kMaxBlock ? cm.x : r;   // rows of larger cells need no neighbours
    };
    const int rb0 = blockIdx.x == 0 ? 0 : cell_start(int((long long)M * blockIdx.x / nblk));
    const int rb1 = cell_start(int((long long)M * (blockIdx.x + 1) / nblk));
    // end of the chunk of at most NT rows that starts at row c
    auto chunk_end = [&](int c) -> int {
        const int e = min(c + NT, rb1);
        return e < rb1 ? cell_start(e) : e;
    };
    const int ce_first = chunk_end(rb0);
    const int gfirst = g0 + wid;
    const int i_first = rb0 + threadIdx.x < ce_first ? rb0 + threadIdx.x : M;
    T* __restrict__ pgr = pbuf;              // [2 parities][nblk] x (gamma, (r, r))
    T* __restrict__ pdl = pbuf + 4 * nblk;   // [nblk] delta
    // scalar state (thread 0 of every block, identical in all blocks)
    T gprev = T(1), aprev = T(1);
    int it = 0, state = kRunning;
    const T tol2bb = T(sc->tol2) * T(sc->bb);
    const int maxit = sc->maxit;
    if (threadIdx.x == 0) {
        s_next[0] = g0 + NW;
        s_next[1] = g0 + NW;
    }
    if (gfirst < g1) stage_group(bd.gdesc, gfirst, gsm[wid], 0, lane);
    __syncthreads();
    bool timed_out = false;
    for (int P = 0;; P ^= 1) {
        const T* __restrict__ rP = P ? v.r[1] : v.r[0];
        const T* __restrict__ sP = P ? v.s[1] : v.s[0];
        T* __restrict__ wP = P ? v.w[1] : v.w[0];
        // ---- SpMV phase
        T d = T(0);
        if (gfirst < g1) {
            int b = 0;
            for (;;) {
                int qn = 0;
                if (lane == 0) qn = atomicAdd(&s_next[P], 1);
                qn = __shfl_sync(kFull, qn, 0);
                if (qn < g1) {
                    stage_group(bd.gdesc, qn, gsm[wid], b ^ 1, lane);
                    group_wait<1>();
                } else {
                    group_wait<0>();
                }
                d += spmv_group<T>(b, B, v.u, wP, M, lane, gsm[wid]);
                if (qn >= g1) break;
                b ^= 1;
            }
            // the records are fixed: the next iteration's first one travels during the barrier
            stage_group(bd.gdesc, gfirst, gsm[wid], 0, lane);
            d = warp_sum<T>(d);
        }
        if (lane == 0) s_dw[wid] = d;
        // this thread's first row, loaded before the barrier (none of it changes in the SpMV)
        T f_d = T(0), f_s = T(0), f_p = T(0), f_u = T(0), f_r = T(0), f_x = T(0);
        int4 f_cm = make_int4(0, 0, 0, 0);
        if (i_first < M) {
            f_d = __ldg(v.dinv + i_first);
            f_s = __ldcg(sP + i_first);
            f_p = __ldcg(v.p + i_first);
            f_u = __ldcg(v.u + i_first);
            f_r = __ldcg(rP + i_first);
            f_x = __ldcg(v.x + i_first);
            f_cm = __ldg(bd.crow + i_first);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T db = T(0);
            for (int w = 0; w < NW; ++w) db += s_dw[w];
            pdl[blockIdx.x] = db;
        }
        target += narrive;
        if (!grid_barrier(sc, target)) {
            timed_out = true;
            break;
        }
        // ---- scalar step
        const T f_w = i_first < M ? __ldcg(wP + i_first) : T(0);
        if (wid == 0) {
            // delta_k from this iteration's per-block partials; gamma_k and (r_k, r_k) from the
            // previous update's (the start kernel's at k = 0), all loads in one batch, each sum
            // in block order
            const T2* pp = reinterpret_cast<const T2*>(it == 0 ? pinit : pgr + size_t(P ^ 1) * 2 * nblk);
            const int npp = it == 0 ? ninit : nblk;
            T dd = T(0), g = T(0), rr = T(0);
            for (int b0 = lane; b0 < max(nblk, npp); b0 += 32 * kPartBatch) {
                T pv[kPartBatch];
                T2 qv[kPartBatch];
#pragma unroll
                for (int k = 0; k < kPartBatch; ++k) {
                    const int b = b0 + 32 * k;
                    pv[k] = b < nblk ? __ldcg(pdl + b) : T(0);
                    qv[k] = b < npp ? __ldcg(pp + b) : T2{T(0), T(0)};
                }
#pragma unroll
                for (int k = 0; k < kPartBatch; ++k) {
                    dd += pv[k];
                    g += qv[k].x;
                    rr += qv[k].y;
                }
            }
            dd = warp_sum<T>(dd);
            g = warp_sum<T>(g);
            rr = warp_sum<T>(rr);
            if (lane == 0) {
                T alpha = T(0), beta = T(0);
                if (!isfinite(g) || !isfinite(rr)) {
                    state = kBreakdown;
                } else if (rr <= tol2bb) {
                    state = kConverged;
                } else if (it >= maxit) {
                    state = kMaxIt;
                } else {
                    beta = it == 0 ? T(0) : g / gprev;
                    const T den = it == 0 ? dd : dd - beta * g / aprev;
                    alpha = g / den;
                    if (!(den > T(0)) || !isfinite(alpha)) state = kBreakdown;
                }
                s_ab[0] = alpha;
                s_ab[1] = beta;
                s_go = state == kRunning;
                if (state == kRunning) {
                    gprev = g;
                    aprev = alpha;
                } else if (blockIdx.x == 0) {
                    sc->out_rr = double(rr);
                    sc->out_gamma = double(g);
                    sc->out_it = it;
                    sc->out_state = state;
                }
                // the other parity's counter, next used after the coming barrier
                s_next[P ^ 1] = g0 + NW;
            }
        }
        __syncthreads();
        if (!s_go) break;
        ++it;
        // ---- update phase
        const T ta = s_ab[0], tb = s_ab[1];
        T* __restrict__ rQ = P ? v.r[0] : v.r[1];
        T* __restrict__ sQ = P ? v.s[0] : v.s[1];
        T* __restrict__ wQ = P ? v.w[0] : v.w[1];
        T acc[2] = {T(0), T(0)};
        // With several chunks per block (large systems), row cend + tid of the next chunk is
        // loaded at the start of the current one (and the next chunk's end with it), so that
        // those round trips overlap this chunk's work; a row the chunk's cut moves to a later
        // chunk is simply loaded again there.
        T c_d = f_d, c_w = f_w, c_s = f_s, c_p = f_p, c_u = f_u, c_r = f_r, c_x = f_x;
        int4 c_cm = f_cm;
        int i_c = i_first;
        for (int base = rb0, cend = ce_first; base < rb1;) {
            const int nend = cend < rb1 ? chunk_end(cend) : rb1;
            const int in = cend + threadIdx.x;
            T n_d = T(0), n_w = T(0), n_s = T(0), n_p = T(0), n_u = T(0), n_r = T(0), n_x = T(0);
            int4 n_cm = make_int4(0, 0, 0, 0);
            if (in < rb1) {
                n_d = __ldg(v.dinv + in);
                n_w = __ldcg(wP + in);
                n_s = __ldcg(sP + in);
                n_p = __ldcg(v.p + in);
                n_u = __ldcg(v.u + in);
                n_r = __ldcg(rP + in);
                n_x = __ldcg(v.x + in);
                n_cm = __ldg(bd.crow + in);
            }
            const int i = base + threadIdx.x;
            const bool valid = i < cend;
            const bool have = i == i_c;
            T di = T(0), ri = T(0);
            if (valid) {
                di = have ? c_d : __ldg(v.dinv + i);
                const T wi = di == T(0) ? T(0) : (have ? c_w : __ldcg(wP + i));
                const T si = fma(tb, have ? c_s : __ldcg(sP + i), wi);
                const T pi = fma(tb, have ? c_p : __ldcg(v.p + i), have ? c_u : __ldcg(v.u + i));
                ri = di == T(0) ? T(0) : fma(-ta, si, have ? c_r : __ldcg(rP + i));
                sQ[i] = si;
                v.p[i] = pi;
                v.x[i] = fma(ta, pi, have ? c_x : __ldcg(v.x + i));
                rQ[i] = ri;
                wQ[i] = T(0);
            }
            rsm[threadIdx.x] = ri;
            __syncthreads();
            if (valid) {
                const int4 cm = have ? c_cm : __ldg(bd.crow + i);
                // the cell's rows are all in this chunk
                const T ui = apply_prec<T, 16>(bd, v.bjinv, cm, i, di, ri, [&](int j) { return rsm[j - base]; });
                v.u[i] = ui;
                acc[0] = fma(ri, ui, acc[0]);
                acc[1] = fma(ri, ri, acc[1]);
            }
            __syncthreads();
            c_d = n_d;
            c_w = n_w;
            c_s = n_s;
            c_p = n_p;
            c_u = n_u;
            c_r = n_r;
            c_x = n_x;
            c_cm = n_cm;
            i_c = in;
            base = cend;
            cend = nend;
        }
        double tot[2];
        block_sum_t<2, T>(acc, tot);
        if (threadIdx.x == 0) {
            T* pq = pgr + size_t(P) * 2 * nblk;
            pq[2 * blockIdx.x] = T(tot[0]);
            pq[2 * blockIdx.x + 1] = T(tot[1]);
        }
        target += narrive;
        if (!grid_barrier(sc, target)) {
            timed_out = true;
            break;
        }
    }
    // no copy of this thread may still be in flight when the block ends
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (timed_out && blockIdx.x == 0 && threadIdx.x == 0) sc->out_state = kBreakdown;
}

// Preconditioner set-up, one warp per cell: dinv[s] = 1 / B_ss for centres with at least
// min_support points inside their support, else 0 (pinned: row and column removed from the
// system); and, for cells with m <= kMaxBlock, the inverse of the cell's diagonal block
// B[c, c] (pinned rows and columns replaced by the identity before, and zeroed after, the
// inversion), by Gauss-Jordan elimination in FP64 without pivoting (the block is SPD),
// symmetrised and stored row-major in the precision of B.
constexpr int kBjWarps = 4;
template <typename T>
__global__ void __launch_bounds__(kBjWarps * 32)
    k_prec_setup(Binned bd, const T* __restrict__ B, const int* __restrict__ support,
                 int min_support, T* __restrict__ dinv, T* __restrict__ bjinv,
                 int* __restrict__ npinned) {
    __shared__ double A[kBjWarps][kMaxBlock][kMaxBlock + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kBjWarps + warp;
    if (c >= bd.g.ncell) return;
    const int cs = bd.cstart[c], m = bd.cstart[c + 1] - cs;
    if (m == 0) return;
    int np = 0;
    for (int i = lane; i < m; i += 32) {
        const T d = b_same_cell<T>(bd.rmeta, B, cs + i, cs + i);
        const bool pin = support[cs + i] < min_support || !(d > T(0));
        dinv[cs + i] = pin ? T(0) : T(1) / d;
        np += pin;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(kFull, np, o);
    if (lane == 0 && np) atomicAdd(npinned, np);
    if (m > kMaxBlock) return;
    __syncwarp();
    double (*a)[kMaxBlock + 1] = A[warp];
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - (e / m) * m;
        const bool pin = dinv[cs + i] == T(0) || dinv[cs + j] == T(0);
        a[i][j] = pin ? (i == j ? 1.0 : 0.0) : double(b_same_cell<T>(bd.rmeta, B, cs + i, cs + j));
    }
    __syncwarp();
    for (int k = 0; k < m; ++k) {
        const double piv = a[k][k];
        __syncwarp();
        if (lane < m) a[k][lane] = (lane == k ? 1.0 : a[k][lane]) / piv;
        __syncwarp();
        for (int i = 0; i < m; ++i) {
            if (i == k) continue;
            const double f = a[i][k];
            __syncwarp();
            if (lane < m) a[i][lane] = (lane == k ? 0.0 : a[i][lane]) - f * a[k][lane];
            __syncwarp();
        }
    }
    T* out = bjinv + bd.bjoff[c];
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - (e / m) * m;
        const bool pin = dinv[cs + i] == T(0) || dinv[cs + j] == T(0);
        out[e] = pin ? T(0) : T(0.5 * (a[i][j] + a[j][i]));
    }
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
// dst (sorted, precision T) = src (caller order, FP64), pinned rows zero.
template <typename T>
__global__ void k_to_sorted_T(const double* __restrict__ src, const int* __restrict__ perm,
                              const T* __restrict__ dinv, T* __restrict__ dst, int M) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) dst[s] = dinv[s] == T(0) ? T(0) : T(src[perm[s]]);
}
template <typename T>
__global__ void k_from_sorted_T(const T* __restrict__ src, const int* __restrict__ perm,
                                double* __restrict__ dst, int M) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) dst[perm[s]] = double(src[s]);
}

// x64 = (x64 + scale * d) on unpinned rows; x64 pinned rows forced to 0.
template <typename T>
__global__ void k_axpy_mixed(int M, double* __restrict__ x, const T* __restrict__ d,
                             double scale, const T* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) x[i] = dinv[i] == T(0) ? 0.0 : fma(scale, double(d[i]), x[i]);
}

// ---- the three polynomial rows of Eq. 10 (one thread each) ----

// G^-1 = adj(G) / det(G) for the SPD 3 x 3 block G = P^T P (FP64); tmp[0] = 1 when G is
// numerically singular (the points are collinear: a linear polynomial is not determined).
// Also clears the FP64 iterate of the polynomial unknowns.
__global__ void k_poly_setup(PolyDev* pd) {
    const double* g = pd->gp;
    const double c00 = g[4] * g[8] - g[5] * g[7], c01 = g[5] * g[6] - g[3] * g[8],
                 c02 = g[3] * g[7] - g[4] * g[6];
    const double det = g[0] * c00 + g[1] * c01 + g[2] * c02;
    const double tr = (g[0] + g[4] + g[8]) / 3.0;
    const bool bad = !(det > 1e-12 * tr * tr * tr) || !isfinite(det);
    const double id = bad ? 0.0 : 1.0 / det;
    double a[9] = {c00, g[2] * g[7] - g[1] * g[8], g[1] * g[5] - g[2] * g[4],
                   c01, g[0] * g[8] - g[2] * g[6], g[2] * g[3] - g[0] * g[5],
                   c02, g[1] * g[6] - g[0] * g[7], g[0] * g[4] - g[1] * g[3]};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) pd->ginv[3 * i + j] = 0.5 * (a[3 * i + j] + a[3 * j + i]) * id;
    for (int i = 0; i < 3; ++i) pd->k64[i] = 0.0;
    pd->tmp[0] = bad ? 1.0 : 0.0;
}

// k64 += scale * x_k (the correction of the last CG solve)
__global__ void k_poly_axpy(PolyDev* pd, double scale) {
    for (int i = 0; i < 3; ++i) pd->k64[i] = fma(scale, pd->xk[i], pd->k64[i]);
}

// out[0] += ||v||^2 (three values)
__global__ void k_poly_norm_add(const double* __restrict__ v, double* __restrict__ out) {
    out[0] += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
}

// The coefficients in the caller's coordinates: u = (x - xc) sx, v = (y - yc) sy, so
// k0 u + k1 v + k2 = (k0 sx) x + (k1 sy) y + (k2 - k0 sx xc - k1 sy yc).
__global__ void k_poly_export(const PolyDev* __restrict__ pd, double xc, double yc, double sx,
                              double sy, double* __restrict__ out) {
    const double ax = pd->k64[0] * sx, ay = pd->k64[1] * sy;
    out[0] = ax;
    out[1] = ay;
    out[2] = pd->k64[2] - ax * xc - ay * yc;
}

template <typename TM>
__global__ void k_mask_zero(int M, double* __restrict__ x, const TM* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && dinv[i] == TM(0)) x[i] = 0.0;
}

__global__ void k_to_f32(int M, const double* __restrict__ x, float* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) u[i] = float(x[i]);
}
// r = b - w on unpinned rows, 0 on pinned rows (w = B32 x from the FP32 SpMV).
__global__ void k_resid32(int M, const double* __restrict__ b, const float* __restrict__ w,
                          const float* __restrict__ dinv32, double* __restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) r[i] = dinv32[i] == 0.0f ? 0.0 : b[i] - double(w[i]);
}

// ||v||^2 over unpinned rows into out[0], in a fixed order: per-block partial sums (blocks of
// kVecThreads rows strided over the vector) into part[], then one block adds them in block
// order.
constexpr int kNormBlocks = 304;
__global__ void __launch_bounds__(kVecThreads)
    k_norm2_part(int M, const double* __restrict__ v, const float* __restrict__ dinv32,
                 double* __restrict__ part) {
    double s = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < M; i += gridDim.x * kVecThreads) {
        if (dinv32 && dinv32[i] == 0.0f) continue;
        s = fma(v[i], v[i], s);
    }
    double a[1] = {s};
    block_sum<1>(a);
    if (threadIdx.x == 0) part[blockIdx.x] = a[0];
}
__global__ void __launch_bounds__(kVecThreads)
    k_norm2_total(int nb, const double* __restrict__ part, double* __restrict__ out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += kVecThreads) s += part[b];
    double a[1] = {s};
    block_sum<1>(a);
    if (threadIdx.x == 0) out[0] = a[0];
}

// ||v||^2 (unpinned rows when dinv32 is given) into out (device), two launches.
void launch_norm2(rbf_ctx* ctx, const double* v, const float* dinv32, double* out, cudaStream_t st) {
    const int nb = std::max(1, std::min(kNormBlocks, div_up(ctx->M, kVecThreads)));
    double* part = ctx->partial.as<double>();   // free between CG solves
    k_norm2_part<<<nb, kVecThreads, 0, st>>>(ctx->M, v, dinv32, part);
    k_norm2_total<<<1, kVecThreads, 0, st>>>(nb, part, out);
    ctx->launches += 2;
}

// Persistent SpMV grid: as many blocks as can be resident (never more than the cells need).
template <typename T>
int spmv_grid_T(rbf_ctx* ctx) {
    int& per_sm = ctx->spmv_blocks_per_sm[sizeof(T) == 8 ? 0 : 1];
    if (per_sm == 0) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_spmv<T>, kSpmvWarps * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmv<T>, kSpmvWarps * 32, 0);
        per_sm = std::max(1, std::min(a, b));
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    return std::max(1, std::min(per_sm * std::max(sms, 1), div_up(ctx->ngroup, kSpmvWarps)));
}
// Vector-kernel grid: one block per kVecThreads rows, at most the two blocks per SM of
// 512 threads that stay resident (152 SMs): no second wave, and the blocks of a large system
// take several chunks each, whose row loads the update kernel overlaps (20M x 2M: 204 against
// 208 us per iteration with four blocks per SM).
int vec_grid(const rbf_ctx* ctx) {
    return std::max(1, std::min(div_up(ctx->M, kVecThreads), 152 * 2));
}

// The polynomial rows of Eq. 10 in a CG solve of precision T (all null without them).
template <typename T>
struct PolyCg {
    const T* E = nullptr;   // A^T P in T
    T* pe = nullptr;        // per-block partials of E^T u
    PolyDev* pd = nullptr;
};
template <typename T>
PolyCg<T> poly_cg(rbf_ctx* ctx, bool on) {
    PolyCg<T> q;
    if (!on) return q;
    q.E = sizeof(T) == 8 ? reinterpret_cast<const T*>(ctx->pE.p) : reinterpret_cast<const T*>(ctx->pE32.p);
    q.pe = ctx->pepart.as<T>();
    q.pd = ctx->pdev.as<PolyDev>();
    return q;
}

// One CG iteration (two kernels) reading the buffers of parity P, on stream cs.
template <typename T>
void launch_iteration(rbf_ctx* ctx, const CgVec<T>& v, int P, cudaStream_t cs,
                      const PolyCg<T>& pq = PolyCg<T>()) {
    const Binned bd = view(ctx);
    CgScalars* sc = ctx->scal.as<CgScalars>();
    k_cg_spmv<T><<<spmv_grid_T<T>(ctx), kSpmvWarps * 32, 0, cs>>>(bd, bvals_dev<T>(ctx), v.u,
                                                                  v.w[P], P, sc);
    k_cg_update<T><<<vec_grid(ctx), kVecThreads, 0, cs>>>(bd, v, P, sc, ctx->partial.as<T>(),
                                                          pq.E, pq.pe, pq.pd);
}

// The solve graph of precision T: one conditional WHILE node whose body runs
// kItersPerBody CG iterations (two kernels each) and then sets the loop condition from the
// device-side state, so the whole iteration runs on the GPU without host round trips.
// Instantiated once per context, precision and workspace layout, then replayed.
template <typename T>
rbf_status cg_graph(rbf_ctx* ctx, cudaGraphExec_t* out, bool poly) {
    rbf_ctx::SolveGraph& sg = ctx->cg_graph[sizeof(T) == 8 ? 0 : 1];
    const CgVec<T> v = cg_vectors<T>(ctx);
    const PolyCg<T> pq = poly_cg<T>(ctx, poly);
    const void* key[12] = {bvals_dev<void>(ctx), v.x, v.dinv, v.bjinv, ctx->scal.p, ctx->partial.p,
                           ctx->cstart.p, ctx->rmeta.p, ctx->gdesc.p, ctx->bjoff.p, pq.E, pq.pe};
    bool hit = sg.exec && sg.ncell == ctx->g.ncell && sg.M == ctx->M && sg.gx == ctx->g.gx &&
               sg.crow == ctx->crow.p && sg.ngroup == ctx->ngroup;
    for (int k = 0; k < 12 && hit; ++k) hit = sg.key[k] == key[k];
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
        for (int k = 0; k < kItersPerBody; ++k) launch_iteration<T>(ctx, v, k & 1, cs, pq);
        k_cg_cond<<<1, 1, 0, cs>>>(ctx->scal.as<CgScalars>(), handle);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cs, &captured);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        sg.exec = nullptr;
        return cuda_fail(ctx, e, "building the CG solve graph", __FILE__, __LINE__);
    }
    sg.ncell = ctx->g.ncell;
    sg.M = ctx->M;
    sg.gx = ctx->g.gx;
    sg.crow = ctx->crow.p;
    sg.ngroup = ctx->ngroup;
    for (int k = 0; k < 12; ++k) sg.key[k] = key[k];
    *out = sg.exec;
    return RBF_OK;
}

// Start kernels of a solve of B x = bscale * b (x in the workspace holds the start vector
// when use_x0).
template <typename T, typename TB>
rbf_status cg_start(rbf_ctx* ctx, const TB* b, double bscale, bool use_x0, double tol, int maxit,
                    cudaStream_t st, bool poly = false, const double* bk = nullptr) {
    const Binned bd = view(ctx);
    const CgVec<T> v = cg_vectors<T>(ctx);
    CgScalars* sc = ctx->scal.as<CgScalars>();
    const PolyCg<T> pq = poly_cg<T>(ctx, poly);
    if (poly)
        RBF_CUDA_TRY(cudaMemcpyAsync(pq.pd->bk, bk, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CgScalars h{};
    h.tol2 = tol * tol;
    h.bscale = bscale;
    h.maxit = maxit;
    RBF_CUDA_TRY(cudaMemcpyAsync(sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, st));
    if (use_x0) {
        RBF_CUDA_TRY(cudaMemsetAsync(v.w[1], 0, sizeof(T) * ctx->M, st));
        k_spmv<T><<<spmv_grid_T<T>(ctx), kSpmvWarps * 32, 0, st>>>(bd, bvals_dev<T>(ctx), v.x, v.w[1]);
        ctx->launches += 1;
    }
    double* part = ctx->partial.as<double>();
    // per-block partials of the precision T in the first 4 vec_grid slots (both parities), the
    // start kernel's (b, b) partials after them
    k_cg_init<T, TB><<<vec_grid(ctx), kVecThreads, 0, st>>>(bd, v, b, use_x0 ? 1 : 0, sc,
                                                            reinterpret_cast<T*>(part),
                                                            part + 4 * vec_grid(ctx), pq.E, pq.pe,
                                                            pq.pd);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

// Blocks of the persistent solve kernel that fit on the device at once (0: none).
template <typename T>
int persist_grid(rbf_ctx* ctx) {
    int& per_sm = ctx->persist_blocks_per_sm[sizeof(T) == 8 ? 0 : 1];
    if (per_sm == 0) {
        int a = 0, coop = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_persist<T>, PersistCfg<T>::threads, 0) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            a = 0;
        }
        per_sm = (a > 0 && coop) ? 1 : -1;   // one block per SM
    }
    if (per_sm < 0) return 0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    return sms;
}

// Per-block partials of the persistent kernel: after the start kernel's (4 + 1) vec_grid
// slots, rounded up to an even number of doubles so that the pairs it reads as one 16-byte
// vector (double2 in FP64) stay aligned.
inline size_t persist_offset(rbf_ctx* ctx) {
    return (5 * size_t(std::max(vec_grid(ctx), 1)) + 1) & ~size_t(1);
}
template <typename T>
T* persist_partials(rbf_ctx* ctx) {
    return reinterpret_cast<T*>(ctx->partial.as<double>() + persist_offset(ctx));
}

// Preconditioned CG on the assembled B (precision T) for B x = bscale * b: start kernels on
// `st`, then the iteration loop -- one cooperative launch of the persistent kernel (single
// systems without the polynomial rows), else one launch of the solve graph.
template <typename T, typename TB>
rbf_status run_cg(rbf_ctx* ctx, const TB* b, double bscale, bool use_x0, double tol, int maxit,
                  int* iters, double* relres, int* state, cudaStream_t st, bool poly = false,
                  const double* bk = nullptr) {
    rbf_status s;
    int pgrid = (!poly && ctx->cg_persistent != 0 && ctx->T == 0) ? persist_grid<T>(ctx) : 0;
    // Automatic choice (measured on GB300): the persistent kernel wins while each block's rows
    // take at most four chunks of its update phase (FP32 terrain 1M x 100k: 14.9 against 16.2
    // us per iteration); beyond that the graph's update kernel, with more warps per SM in
    // flight, is faster in FP32 (big data 20M x 2M: 208 against 232 us), while FP64 iterations
    // are bound by the SpMV's FP64 arithmetic and keep the persistent kernel (79 against 90 us
    // at 1M x 100k, 1341 against 1382 us at 20M x 2M).
    if (pgrid > 0 && ctx->cg_persistent < 0 && sizeof(T) == 4 &&
        ctx->M > 4LL * pgrid * PersistCfg<T>::threads)
        pgrid = 0;
    bool persisted = false, started = false;
    if (pgrid > 0) {
        if ((s = ensure(ctx, ctx->partial, sizeof(double) * (persist_offset(ctx) + 5 * size_t(pgrid)),
                        st)) != RBF_OK)
            return s;
        if ((s = cg_start<T, TB>(ctx, b, bscale, use_x0, tol, maxit, st)) != RBF_OK) return s;
        started = true;
        Binned bd = view(ctx);
        CgVec<T> v = cg_vectors<T>(ctx);
        const T* B = bvals_dev<T>(ctx);
        CgScalars* sc = ctx->scal.as<CgScalars>();
        const T* pinit = reinterpret_cast<const T*>(ctx->partial.p);
        int ninit = vec_grid(ctx);
        T* pbuf = persist_partials<T>(ctx);
        int extra = ctx->cg_barrier_extra;
        void* args[] = {&bd, &v, &B, &sc, &pinit, &ninit, &pbuf, &extra};
        const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_cg_persist<T>),
                                                          dim3(pgrid), dim3(PersistCfg<T>::threads), args, 0, st);
        if (e == cudaSuccess) {
            persisted = true;
            ctx->launches += 1;
        } else {
            // not resident at once (another context holds SMs, say): the graph loop instead,
            // from the start kernel's state
            cudaGetLastError();
            ctx->persist_blocks_per_sm[sizeof(T) == 8 ? 0 : 1] = -1;
        }
    }
    if (!persisted) {
        cudaGraphExec_t ex;
        if ((s = cg_graph<T>(ctx, &ex, poly)) != RBF_OK) return s;
        if (!started)
            if ((s = cg_start<T, TB>(ctx, b, bscale, use_x0, tol, maxit, st, poly, bk)) != RBF_OK) return s;
        RBF_CUDA_TRY(cudaGraphLaunch(ex, st));
    }
    CgScalars* hs = static_cast<CgScalars*>(ctx->hpinned);
    RBF_CUDA_TRY(cudaMemcpyAsync(hs, ctx->scal.p, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    if (persisted && hs->bar_err)
        return set_err(ctx, RBF_ERR_TIMEOUT, "a grid barrier of the persistent CG solve timed out");
    if (!persisted) {
        // kernels launched by the graph: per loop pass 2 * kItersPerBody + 1; the stop is
        // detected one kernel after the last iteration, so the passes cover out_it + 1
        // iterations
        const int passes = hs->out_it / kItersPerBody + 1;
        ctx->launches += int64_t(passes) * (2 * kItersPerBody + 1);
    }
    *iters = hs->out_it;
    *relres = hs->bb > 0 ? sqrt(hs->out_rr / hs->bb) : 0.0;
    *state = hs->out_state;
    return RBF_OK;
}

// Timing hook: a solve of B x = b from x = 0 whose `reps` CG iterations are plain kernel
// launches (two per iteration) instead of the graph loop, on the solver's workspace.
template <typename T>
rbf_status bench_cg_impl(rbf_ctx* ctx, int reps, cudaStream_t st) {
    rbf_status s = cg_start<T, double>(ctx, ctx->bvec.as<double>(), 1.0, false, 0.0, 1 << 30, st);
    if (s != RBF_OK) return s;
    const CgVec<T> v = cg_vectors<T>(ctx);
    for (int k = 0; k < reps; ++k) launch_iteration<T>(ctx, v, k & 1, st);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 2 * int64_t(reps);
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

// Timing hook: `reps` CG iterations on B x = b from x = 0 (tolerance 0) in the solver's own
// loop, persistent kernel or graph as rbf_solve would choose. Synchronises `st`.
template <typename T>
rbf_status bench_cg_loop_impl(rbf_ctx* ctx, int reps, cudaStream_t st) {
    int it = 0, state = 0;
    double rel = 0.0;
    return run_cg<T, double>(ctx, ctx->bvec.as<double>(), 1.0, false, 0.0, reps, &it, &rel, &state, st);
}

rbf_status bench_cg_loop_run(rbf_ctx* ctx, int reps, cudaStream_t st) {
    return ctx->prec == RBF_FP64 ? bench_cg_loop_impl<double>(ctx, reps, st)
                                 : bench_cg_loop_impl<float>(ctx, reps, st);
}

rbf_status bench_cg_run(rbf_ctx* ctx, int reps, cudaStream_t st) {
    return ctx->prec == RBF_FP64 ? bench_cg_impl<double>(ctx, reps, st)
                                 : bench_cg_impl<float>(ctx, reps, st);
}

template <typename T>
__global__ void k_fill(T* __restrict__ v, int n, T value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = value;
}

template <typename T>
rbf_status bench_spmv_impl(rbf_ctx* ctx, int reps, cudaStream_t st) {
    rbf_status s = ensure(ctx, ctx->cgv[sizeof(T) == 8 ? 0 : 1], sizeof(T) * kCgVecs * cg_stride(ctx->M), st);
    if (s != RBF_OK) return s;
    const Binned bd = view(ctx);
    const CgVec<T> v = cg_vectors<T>(ctx);
    k_fill<T><<<div_up(ctx->M, 256), 256, 0, st>>>(v.u, ctx->M, T(1));
    RBF_CUDA_TRY(cudaMemsetAsync(v.w[0], 0, sizeof(T) * ctx->M, st));
    for (int k = 0; k < reps; ++k)
        k_spmv<T><<<spmv_grid_T<T>(ctx), kSpmvWarps * 32, 0, st>>>(bd, bvals_dev<T>(ctx), v.u, v.w[0]);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += reps + 1;
    return RBF_OK;
}

rbf_status bench_spmv_run(rbf_ctx* ctx, int reps, cudaStream_t st) {
    return ctx->prec == RBF_FP64 ? bench_spmv_impl<double>(ctx, reps, st)
                                 : bench_spmv_impl<float>(ctx, reps, st);
}

// FMA throughput probe: every thread runs kFmaChains independent FMA chains of `reps` steps
// (2 kFmaChains reps flops per thread); the result is stored only if it equals a value it
// cannot reach, which keeps the chains live.
constexpr int kFmaChains = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ sink, long long reps, T a, T b) {
    T x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (long long i = 0; i < reps; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], a, b);
    }
    T sum = T(0);
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) sum += x[k];
    if (sum == T(-12345.678)) sink[blockIdx.x] = sum;
}

rbf_status bench_fma_run(rbf_ctx* ctx, int prec, long long reps, double* flops, cudaStream_t st) {
    int sms = 0;
    RBF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = sms * 8;
    rbf_status s = ensure(ctx, ctx->scan_tmp, sizeof(double) * blocks, st);
    if (s != RBF_OK) return s;
    // a contraction toward a fixed point: the values stay finite for any reps
    if (prec == RBF_FP64)
        k_fma_peak<double><<<blocks, 256, 0, st>>>(ctx->scan_tmp.as<double>(), reps, 0.999, 1e-3);
    else
        k_fma_peak<float><<<blocks, 256, 0, st>>>(ctx->scan_tmp.as<float>(), reps, 0.999f, 1e-3f);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    *flops = 2.0 * kFmaChains * double(reps) * double(blocks) * 256.0;
    return RBF_OK;
}

// Timing hook: `reps` FP64 residual passes r = A^T (h - A x) of the refinement at the current
// FP64 iterate (stored A when the FP32 assembly kept it, else matrix-free).
rbf_status bench_residual_run(rbf_ctx* ctx, int reps, cudaStream_t st) {
    double* x64 = ctx->x.as<double>();
    double* r64 = ctx->r.as<double>();
    for (int k = 0; k < reps; ++k) {
        RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * ctx->M, st));
        rbf_status s = residual_run(ctx, x64, r64, false, st);
        if (s != RBF_OK) return s;
    }
    return RBF_OK;
}

rbf_status prec_setup_run(rbf_ctx* ctx, int prec, int min_support, int* npin_d, cudaStream_t st) {
    const Binned bd = view(ctx);
    const int nb = div_up(ctx->g.ncell, kBjWarps);
    if (prec == RBF_FP64)
        k_prec_setup<double><<<nb, kBjWarps * 32, 0, st>>>(bd, bvals_dev<double>(ctx),
                                                           ctx->support.as<int>(), min_support,
                                                           ctx->dinv.as<double>(),
                                                           ctx->bjinv.as<double>(), npin_d);
    else
        k_prec_setup<float><<<nb, kBjWarps * 32, 0, st>>>(bd, bvals_dev<float>(ctx),
                                                          ctx->support.as<int>(), min_support,
                                                          ctx->dinv32.as<float>(),
                                                          ctx->bjinv32.as<float>(), npin_d);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

void launch_resid32(rbf_ctx* ctx, const double* x64, double* r64, cudaStream_t st) {
    const int M = ctx->M;
    const CgVec<float> v = cg_vectors<float>(ctx);
    k_to_f32<<<div_up(M, 256), 256, 0, st>>>(M, x64, v.u);
    cudaMemsetAsync(v.w[0], 0, sizeof(float) * M, st);
    launch_spmv(ctx, RBF_FP32_REFINE, v.u, v.w[0], st);
    k_resid32<<<div_up(M, 256), 256, 0, st>>>(M, ctx->bvec.as<double>(), v.w[0],
                                              ctx->dinv32.as<float>(), r64);
    ctx->launches += 2;
}

void launch_spmv(rbf_ctx* ctx, int prec, const void* x, void* y, cudaStream_t st) {
    const Binned bd = view(ctx);
    if (prec == RBF_FP64)
        k_spmv<double><<<spmv_grid_T<double>(ctx), kSpmvWarps * 32, 0, st>>>(
            bd, bvals_dev<double>(ctx), static_cast<const double*>(x), static_cast<double*>(y));
    else
        k_spmv<float><<<spmv_grid_T<float>(ctx), kSpmvWarps * 32, 0, st>>>(
            bd, bvals_dev<float>(ctx), static_cast<const float*>(x), static_cast<float*>(y));
    ctx->launches += 1;
}

static rbf_status finish_status(rbf_ctx* ctx, int state) {
    if (state == kConverged) return RBF_OK;
    if (state == kBreakdown)
        return set_err(ctx, RBF_ERR_BREAKDOWN, "CG breakdown (non-positive curvature or non-finite scalar)");
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
    ENS(partial, sizeof(double) * 5 * std::max(vec_grid(ctx), 1));
    int64_t* npin_h = static_cast<int64_t*>(ctx->hpinned) + 256;
    int* npin_d = reinterpret_cast<int*>(ctx->scal.as<char>() + sizeof(CgScalars));
    RBF_CUDA_TRY(cudaMemsetAsync(npin_d, 0, sizeof(int), st));
    rbf_solve_info inf{};
    int state = kConverged;

    if (ctx->prec == RBF_FP64) {
        ENS(cgv[0], sizeof(double) * kCgVecs * cg_stride(M));
        ENS(dinv, sizeof(double) * M);
        ENS(bjinv, sizeof(double) * std::max<int64_t>(ctx->nbj, 1));
        k_prec_setup<double><<<div_up(ctx->g.ncell, kBjWarps), kBjWarps * 32, 0, st>>>(
            bd, bvals_dev<double>(ctx), ctx->support.as<int>(), min_support,
            ctx->dinv.as<double>(), ctx->bjinv.as<double>(), npin_d);
        ctx->launches += 1;
        const CgVec<double> v = cg_vectors<double>(ctx);
        if (use_c0) {
            k_to_sorted_T<double><<<div_up(M, 256), 256, 0, st>>>(c, bd.cperm, v.dinv, v.x, M);
            ctx->launches += 1;
        }
        RBF_CUDA_TRY(cudaGetLastError());
        int it = 0;
        double rel = 0.0;
        s = run_cg<double, double>(ctx, ctx->bvec.as<double>(), 1.0, use_c0 != 0, tol, maxit, &it,
                                   &rel, &state, st);
        if (s != RBF_OK) return s;
        k_from_sorted_T<double><<<div_up(M, 256), 256, 0, st>>>(v.x, bd.cperm, c, M);
        ctx->launches += 1;
        inf.iterations = it;
        inf.rel_residual = rel;
    } else {
        ENS(cgv[1], sizeof(float) * kCgVecs * cg_stride(M));
        ENS(dinv32, sizeof(float) * M);
        ENS(bjinv32, sizeof(float) * std::max<int64_t>(ctx->nbj, 1));
        k_prec_setup<float><<<div_up(ctx->g.ncell, kBjWarps), kBjWarps * 32, 0, st>>>(
            bd, bvals_dev<float>(ctx), ctx->support.as<int>(), min_support,
            ctx->dinv32.as<float>(), ctx->bjinv32.as<float>(), npin_d);
        ctx->launches += 1;
        const CgVec<float> v = cg_vectors<float>(ctx);
        double* x64 = ctx->x.as<double>();
        double* r64 = ctx->r.as<double>();
        double* nrm_d = reinterpret_cast<double*>(ctx->scal.as<char>() + sizeof(CgScalars) + 8);
        double* nrm_h = reinterpret_cast<double*>(static_cast<char*>(ctx->hpinned) + 3072);
        const float* dinv32 = ctx->dinv32.as<float>();
        // ||b|| over unpinned rows
        launch_norm2(ctx, ctx->bvec.as<double>(), dinv32, nrm_d, st);
        RBF_CUDA_TRY(cudaMemcpyAsync(nrm_h, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, st));
        // With a start vector the first residual comes from the FP32 matrix, r = b - B32 x
        // (FP32 products and sums: relative error about 1e-6 of ||b||). It only has to be far
        // more accurate than the inner tolerance, and the FP64 matrix-free residual of the
        // next refinement step replaces it; no convergence is declared on it.
        bool approx_r = false;
        if (use_c0) {
            launch_gather_sorted(c, bd.cperm, x64, M, st);
            k_mask_zero<float><<<div_up(M, 256), 256, 0, st>>>(M, x64, dinv32);
            k_to_f32<<<div_up(M, 256), 256, 0, st>>>(M, x64, v.u);
            RBF_CUDA_TRY(cudaMemsetAsync(v.w[0], 0, sizeof(float) * M, st));
            launch_spmv(ctx, RBF_FP32_REFINE, v.u, v.w[0], st);
            k_resid32<<<div_up(M, 256), 256, 0, st>>>(M, ctx->bvec.as<double>(), v.w[0], dinv32, r64);
            ctx->launches += 4;
            approx_r = true;
        } else {
            RBF_CUDA_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * M, st));
            RBF_CUDA_TRY(cudaMemcpyAsync(r64, ctx->bvec.p, sizeof(double) * M,
                                         cudaMemcpyDeviceToDevice, st));
        }
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        const double bnorm = sqrt(nrm_h[0]);
        auto norm_r64 = [&](double* out) -> rbf_status {
            launch_norm2(ctx, r64, dinv32, nrm_d, st);
            RBF_CUDA_TRY(cudaMemcpyAsync(nrm_h, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, st));
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            *out = sqrt(nrm_h[0]);
            return RBF_OK;
        };
        double rn = 0.0;
        if ((s = norm_r64(&rn)) != RBF_OK) return s;
        int total_it = 0, outer = 0, weak = 0;
        double rel = 0.0;
        state = kMaxIt;
        // Inner tolerance: each refinement step gains about -log10(inner_tol) digits; FP32
        // rounding of B limits the gain per step, not the final accuracy.
        const double inner_tol = ctx->inner_tol;
        for (outer = 0;; ++outer) {
            rel = bnorm > 0 ? rn / bnorm : 0.0;
            if ((rel <= tol && !approx_r) || rn == 0.0) {
                state = kConverged;
                break;
            }
            if (outer == ctx->max_refine) break;
            int it = 0, ist = 0;
            double irel = 0.0;
            const double itol = std::max(inner_tol, 0.5 * tol / rel);
            s = run_cg<float, double>(ctx, r64, 1.0 / rn, false, itol, maxit, &it, &irel, &ist, st);
            if (s != RBF_OK) return s;
            total_it += it;
            // An inner breakdown (FP32 rounding can make B32 indefinite when the system is
            // very ill-conditioned) ends the inner solve; its last iterate is still a usable
            // correction, and the FP64 residual below decides whether it helped.
            if (ist == kBreakdown && it == 0) {
                state = kBreakdown;
                break;
            }
            k_axpy_mixed<float><<<div_up(M, 256), 256, 0, st>>>(M, x64, v.x, rn, dinv32);
            RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
            if ((s = residual_run(ctx, x64, r64, false, st)) != RBF_OK) return s;
            k_mask_zero<float><<<div_up(M, 256), 256, 0, st>>>(M, r64, dinv32);
            ctx->launches += 2;
            approx_r = false;
            double rn_new = 0.0;
            if ((s = norm_r64(&rn_new)) != RBF_OK) return s;
            // Stalled: two steps in a row each gained less than half of what the inner solve
            // was asked for (and at most a halving), short of the tolerance -- the FP32
            // matrix cannot resolve the system. One weak step alone is retried: the FP32
            // iterates vary from run to run, and a retry is far cheaper than an FP64 finish.
            const bool done = bnorm > 0 && rn_new / bnorm <= tol;
            if (!done && !(rn_new < std::max(0.5, 2.0 * itol) * rn)) {
                if (++weak >= 2) {
                    rn = std::min(rn, rn_new);
                    ++outer;
                    state = kMaxIt;
                    break;
                }
            } else {
                weak = 0;
            }
            rn = rn_new;
        }
        inf.iterations = total_it;
        inf.refinements = outer;
        inf.rel_residual = bnorm > 0 ? rn / bnorm : 0.0;
        if (state != kConverged) {
            // Promote: assemble B in FP64 and finish with FP64 CG started from the refined
            // iterate.
            launch_scatter_orig(x64, bd.cperm, c, M, st);
            ctx->launches += 1;
            if ((s = assemble_run(ctx, ctx->kernel, RBF_FP64, st)) != RBF_OK) return s;
            ctx->prec = RBF_FP64;
            rbf_solve_info inf64{};
            s = solve_run(ctx, c, 1, tol, maxit, min_support, &inf64, st);
            inf64.iterations += total_it;
            inf64.refinements = outer;
            inf64.promoted = 1;
            if (info) *info = inf64;
            return s;
        }
        launch_scatter_orig(x64, bd.cperm, c, M, st);
        ctx->launches += 1;
    }
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->solved = true;
    RBF_CUDA_TRY(cudaMemcpyAsync(npin_h, npin_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    inf.pinned = *reinterpret_cast<int*>(npin_h);
    if (info) *info = inf;
#undef ENS
    return finish_status(ctx, state);
}

// The bordered system of Eq. 10 by iterative refinement from c = 0, k = 0: every step computes
// the FP64 residual (A^T e, P^T e) of e = h - A c - P k from the points (or the stored A),
// solves the correction with preconditioned CG on the bordered matrix in the assembly's
// precision (FP32 inner tolerance inner_tol, or FP64 to what the outer tolerance needs), and
// adds it in FP64. A stalled FP32 refinement promotes the solve to an FP64 assembly and goes on
// with FP64 inner solves from the refined iterate.
rbf_status solve_poly_run(rbf_ctx* ctx, double* c, double* kout, double tol, int maxit,
                          int min_support, rbf_solve_info* info, cudaStream_t st) {
    const int M = ctx->M;
    const Binned bd = view(ctx);
    rbf_status s;
#define ENS(buf, bytes) \
    if ((s = ensure(ctx, ctx->buf, (bytes), st)) != RBF_OK) return s;
    ENS(x, sizeof(double) * M);
    ENS(r, sizeof(double) * M);
    ENS(scal, sizeof(CgScalars) + 64);
    ENS(partial, sizeof(double) * 5 * std::max(vec_grid(ctx), 1));
    ENS(pepart, sizeof(double) * 8 * std::max(vec_grid(ctx), 1));
    int64_t* npin_h = static_cast<int64_t*>(ctx->hpinned) + 256;
    int* npin_d = reinterpret_cast<int*>(ctx->scal.as<char>() + sizeof(CgScalars));
    double* nrm_d = reinterpret_cast<double*>(ctx->scal.as<char>() + sizeof(CgScalars) + 8);
    double* nrm_h = reinterpret_cast<double*>(static_cast<char*>(ctx->hpinned) + 3072);
    PolyDev* pd = ctx->pdev.as<PolyDev>();
    double* x64 = ctx->x.as<double>();
    double* r64 = ctx->r.as<double>();
    // the row mask of the current precision (0 on pinned rows)
    auto setup = [&](int prec) -> rbf_status {
        RBF_CUDA_TRY(cudaMemsetAsync(npin_d, 0, sizeof(int), st));
        if (prec == RBF_FP64) {
            ENS(cgv[0], sizeof(double) * kCgVecs * cg_stride(M));
            ENS(dinv, sizeof(double) * M);
            ENS(bjinv, sizeof(double) * std::max<int64_t>(ctx->nbj, 1));
        } else {
            ENS(cgv[1], sizeof(float) * kCgVecs * cg_stride(M));
            ENS(dinv32, sizeof(float) * M);
            ENS(bjinv32, sizeof(float) * std::max<int64_t>(ctx->nbj, 1));
        }
        return prec_setup_run(ctx, prec, min_support, npin_d, st);
    };
    if ((s = setup(ctx->prec)) != RBF_OK) return s;
    k_poly_setup<<<1, 1, 0, st>>>(pd);
    ctx->launches += 1;
    // the mask in both precisions agrees (the support counts decide it), FP64 iterate 0
    auto mask_zero = [&](double* vv) {
        if (ctx->prec == RBF_FP64)
            k_mask_zero<double><<<div_up(M, 256), 256, 0, st>>>(M, vv, ctx->dinv.as<double>());
        else
            k_mask_zero<float><<<div_up(M, 256), 256, 0, st>>>(M, vv, ctx->dinv32.as<float>());
        ctx->launches += 1;
    };
    // ||r||^2 over unpinned rows plus the three polynomial rows
    auto norm = [&](const double* vv, const double* vk, double* out) -> rbf_status {
        // the FP32 row mask, or none: with FP64 the pinned rows are zero already
        launch_norm2(ctx, vv, ctx->prec == RBF_FP64 ? nullptr : ctx->dinv32.as<float>(), nrm_d, st);
        k_poly_norm_add<<<1, 1, 0, st>>>(vk, nrm_d);
        ctx->launches += 1;
        RBF_CUDA_TRY(cudaMemcpyAsync(nrm_h, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, st));
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        *out = sqrt(nrm_h[0]);
        return RBF_OK;
    };
    RBF_CUDA_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * M, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(r64, ctx->bvec.p, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
    RBF_CUDA_TRY(cudaMemcpyAsync(pd->rk, pd->gp + 9, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    mask_zero(r64);
    RBF_CUDA_TRY(cudaGetLastError());
    double bnorm = 0.0;
    if ((s = norm(r64, pd->rk, &bnorm)) != RBF_OK) return s;
    {
        double* flag = static_cast<double*>(ctx->hpinned) + 300;
        RBF_CUDA_TRY(cudaMemcpyAsync(flag, pd->tmp, sizeof(double), cudaMemcpyDeviceToHost, st));
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        if (*flag != 0.0)
            return set_err(ctx, RBF_ERR_ARG, "P^T P is singular: the points do not determine a linear polynomial");
    }
    double rn = bnorm;
    rbf_solve_info inf{};
    int state = kMaxIt, total_it = 0, outer = 0, weak = 0;
    const int max_outer = std::max(ctx->max_refine, 1) + 8;
    for (outer = 0;; ++outer) {
        const double rel = bnorm > 0 ? rn / bnorm : 0.0;
        if (rel <= tol || rn == 0.0) {
            state = kConverged;
            break;
        }
        if (outer >= max_outer) break;
        const bool fp64 = ctx->prec == RBF_FP64;
        const double itol = fp64 ? 0.5 * tol / rel : std::max(ctx->inner_tol, 0.5 * tol / rel);
        int it = 0, ist = 0;
        double irel = 0.0;
        if (fp64)
            s = run_cg<double, double>(ctx, r64, 1.0 / rn, false, itol, maxit, &it, &irel, &ist, st,
                                       true, pd->rk);
        else
            s = run_cg<float, double>(ctx, r64, 1.0 / rn, false, itol, maxit, &it, &irel, &ist, st,
                                      true, pd->rk);
        if (s != RBF_OK) return s;
        total_it += it;
        if (ist == kBreakdown && it == 0) {
            state = kBreakdown;
            break;
        }
        if (fp64) {
            const CgVec<double> v = cg_vectors<double>(ctx);
            k_axpy_mixed<double><<<div_up(M, 256), 256, 0, st>>>(M, x64, v.x, rn, v.dinv);
        } else {
            const CgVec<float> v = cg_vectors<float>(ctx);
            k_axpy_mixed<float><<<div_up(M, 256), 256, 0, st>>>(M, x64, v.x, rn, v.dinv);
        }
        k_poly_axpy<<<1, 1, 0, st>>>(pd, rn);
        RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
        if ((s = residual_run(ctx, x64, r64, false, st, true)) != RBF_OK) return s;
        mask_zero(r64);
        ctx->launches += 2;
        double rn_new = 0.0;
        if ((s = norm(r64, pd->rk, &rn_new)) != RBF_OK) return s;
        const bool done = bnorm > 0 && rn_new / bnorm <= tol;
        const bool weak_step = !done && !(rn_new < std::max(0.5, 2.0 * itol) * rn);
        // one weak FP32 step alone is retried (as in rbf_solve); two in a row promote
        if (weak_step && !fp64 && ++weak < 2) {
            rn = rn_new;
            continue;
        }
        if (!weak_step) weak = 0;
        if (weak_step) {
            if (fp64) {   // no progress in FP64 either
                rn = std::min(rn, rn_new);
                ++outer;
                break;
            }
            // promote: FP64 assembly (B, b, and again A^T P, P^T P, P^T h), FP64 inner solves
            // from the refined iterate (kept across the assembly, which clears PolyDev)
            double* kh = static_cast<double*>(ctx->hpinned) + 310;
            RBF_CUDA_TRY(cudaMemcpyAsync(kh, pd->k64, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            const double k0[3] = {kh[0], kh[1], kh[2]};
            if ((s = assemble_run(ctx, ctx->kernel, RBF_FP64, st, true)) != RBF_OK) return s;
            ctx->prec = RBF_FP64;
            inf.promoted = 1;
            if ((s = setup(RBF_FP64)) != RBF_OK) return s;
            k_poly_setup<<<1, 1, 0, st>>>(pd);
            ctx->launches += 1;
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            kh[0] = k0[0];
            kh[1] = k0[1];
            kh[2] = k0[2];
            RBF_CUDA_TRY(cudaMemcpyAsync(pd->k64, kh, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
            RBF_CUDA_TRY(cudaMemsetAsync(r64, 0, sizeof(double) * M, st));
            if ((s = residual_run(ctx, x64, r64, false, st, true)) != RBF_OK) return s;
            mask_zero(r64);
            if ((s = norm(r64, pd->rk, &rn_new)) != RBF_OK) return s;
        }
        rn = rn_new;
    }
    inf.iterations = total_it;
    inf.refinements = outer;
    inf.rel_residual = bnorm > 0 ? rn / bnorm : 0.0;
    launch_scatter_orig(x64, bd.cperm, c, M, st);
    k_poly_export<<<1, 1, 0, st>>>(pd, ctx->pxc, ctx->pyc, ctx->psx, ctx->psy, kout);
    ctx->launches += 2;
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->solved = true;
    RBF_CUDA_TRY(cudaMemcpyAsync(npin_h, npin_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    inf.pinned = *reinterpret_cast<int*>(npin_h);
    if (info) *info = inf;
#undef ENS
    return finish_status(ctx, state);
}

}  // namespace rbf
