// Steps (b)+(c): fused evaluation of the sparse rows of A and assembly of the
// normal equations B = A^T A, b = A^T h (Eq. 4-5, 11-12); also the matrix-free FP64
// normal residual r = A^T (h - A c) used by iterative refinement.
//
// Work decomposition: one CTA per work item = (point cell, up to kWorkPoints points of
// it). The centres that can lie within R of those points are the centres of the 3x3
// cells around the point cell -- three contiguous ranges of the sorted centre order --
// and are staged in shared memory ("candidates", n <= kMaxCand). For each sub-chunk of
// kSubChunk points the CTA fills a dense tile Phi[p][a] = phi(||x_p - xi_a|| / R)
// (zero outside the support, Eq. 18), i.e. the rows of A restricted to the candidates
// (Algorithm 1's triplets, never written to memory). The local Gram matrix
// G = Phi^T Phi (upper triangle only, Section 5) is accumulated in registers, 4x4
// entries per thread, and finally added into the stored upper triangle of B with
// atomics (entry (a, b), a <= b in the candidate order, which is the sorted order, goes to row
// s_a at the slot of column s_b; the diagonal halved, see RowMeta); b and the support counts
// are reduced per candidate.
#include <algorithm>
#include <vector>

#include "rbf_internal.h"

namespace rbf {
namespace {

constexpr int kThreads = 256;

// Adds the block-wide sums of v[0..NV-1] into out[] (one FP64 atomic per value, by thread 0).
template <int NV>
__device__ __forceinline__ void block_atomic_sum(double (&v)[NV], double* out) {
    __shared__ double red[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int j = 0; j < kThreads / 32; ++j) t += red[threadIdx.x][j];
        if (t != 0.0) atomicAdd(out + threadIdx.x, t);
    }
}

// Shared-memory layout of the candidate staging area.
template <typename CT>
struct CandSmem {
    CT* x;              // [npad] candidate coordinates (FP64 global or FP32 point-cell frame)
    CT* y;
    int* s;             // [npad] sorted centre index
    int* a9;            // [npad] local cell 0..8 (row-major in the 3x3 block)
    RowMeta* rm;        // [npad] the candidate's stored row of B (assembly only)
    double* cval;       // [npad] coefficient (residual pass only)
    float* lu;          // [npad] FP32 coordinates in the point cell's frame, units of R
    float* lv;          //        (the same arrays as x, y in the FP32 path)
};

struct LocalCells {
    int start[9], len[9], off[10], cell[9];
    int n;
};

// off[a] = cnt[0] + ... + cnt[a-1] for a < n and off[n] = the total (shared arrays), by the
// whole block; n may exceed the block size.
__device__ void block_scan_counts(const int* cnt, int n, int* off) {
    __shared__ int wtot[kThreads / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kThreads) {
        const int a = base + threadIdx.x;
        const int v = a < n ? cnt[a] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wtot[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = lane < kThreads / 32 ? wtot[lane] : 0;
#pragma unroll
            for (int o = 1; o < kThreads / 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < kThreads / 32) wtot[lane] = t;
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? wtot[w - 1] : 0) + x - v;
        if (a < n) off[a] = excl;
        __syncthreads();
        if (threadIdx.x == kThreads - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
    __syncthreads();
}

// Thread 0 describes the 3x3 block of cells around point cell `cell`.
__device__ void describe_cells(const Binned& bd, int cell, LocalCells& lc) {
    const Grid& g = bd.g;
    const int ix = cell % g.gx, iy = cell / g.gx;
    int off = 0;
    for (int k = 0; k < 9; ++k) {
        const int cx = ix - 1 + (k % 3), cy = iy - 1 + (k / 3);
        int s = 0, l = 0, cc = -1;
        if (cx >= 0 && cx < g.gx && cy >= 0 && cy < g.gy) {
            cc = cy * g.gx + cx;
            s = bd.cstart[cc];
            l = bd.cstart[cc + 1] - s;
        }
        lc.start[k] = s;
        lc.len[k] = l;
        lc.cell[k] = cc;
        lc.off[k] = off;
        off += l;
    }
    lc.off[9] = off;
    lc.n = off;
}

// Stage the candidates of the work item's 3x3 block. FP64 candidates keep global
// coordinates; FP32 candidates are moved into the point cell's local frame (units of R).
template <typename CT>
__device__ void stage_candidates(const Binned& bd, const LocalCells& lc, const CandSmem<CT>& cs,
                                 int npad, const double* c_sorted) {
    for (int a = threadIdx.x; a < npad; a += blockDim.x) {
        if (a < lc.n) {
            int k = 0;
            while (a >= lc.off[k + 1]) ++k;
            const int s = lc.start[k] + (a - lc.off[k]);
            cs.s[a] = s;
            cs.a9[a] = k;
            if (cs.rm) cs.rm[a] = bd.rmeta[s];
            cs.lu[a] = bd.cu[s] + float((k % 3) - 1);
            cs.lv[a] = bd.cv[s] + float((k / 3) - 1);
            if constexpr (sizeof(CT) == 8) {
                cs.x[a] = bd.cx[s];
                cs.y[a] = bd.cy[s];
            }
            if (cs.cval) cs.cval[a] = c_sorted ? c_sorted[s] : 0.0;
        } else {
            cs.s[a] = 0;
            cs.a9[a] = 0;
            if (cs.rm) cs.rm[a] = RowMeta{0, 0, 0, 0};
            cs.x[a] = CT(1e30);
            cs.y[a] = CT(1e30);
            cs.lu[a] = 1e30f;
            cs.lv[a] = 1e30f;
            if (cs.cval) cs.cval[a] = 0.0;
        }
    }
}

constexpr int kFillRing = 64;   // pending (point, candidate) pairs per warp: < 32 + 32

// Fill Phi[pp][a] for the points q0 .. q0+kSubChunk-1 (rows beyond p1 are zero).
// FP64: global coordinates, support decided by the exact test; counts supports if asked.
// ring: kFillRing ints per warp (FP64 only).
template <int KIND, typename T>
__device__ void fill_phi(const Binned& bd, const CandSmem<T>& cs, int n, int npad, int q0, int p1,
                         T* phi, double* hsm, int* cnt, int* ring_all) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if constexpr (sizeof(T) == 8) {
        // FP64: the warp sweeps its points' candidates with the FP32 prefilter and appends the
        // passing (point, candidate) pairs to its ring; every 32 pending pairs make one round of
        // FP64 distances, exact tests and Wendland values, one pair per lane, so the FP64 pipe
        // sees full warps of pairs that can lie inside the support, across the warp's points.
        int* ring = ring_all + warp * kFillRing;
        int head = 0, tail = 0;     // pending pairs [head, tail) (warp-uniform)
        auto round = [&](int cntp) {
            __syncwarp();
            if (lane < cntp) {
                const int e = ring[(head + lane) & (kFillRing - 1)];
                const int pp = e >> 16, a = e & 0xffff;
                const int p = q0 + pp;
                const double dx = bd.px[p] - cs.x[a], dy = bd.py[p] - cs.y[a];
                double d2;
                if (inside_exact_d2(dx, dy, bd.g.R, bd.g.R2, d2)) {
                    const double r = sqrt_fast(d2) * bd.g.invR;
                    phi[pp * npad + a] = wendland<KIND, double>(r);
                    if (cnt) atomicAdd(&cnt[a], 1);
                }
            }
            head += cntp;
            __syncwarp();
        };
        for (int pp = warp; pp < kSubChunk; pp += nw) {
            const int p = q0 + pp;
            const bool valid = p < p1;
            T* row = phi + pp * npad;
            const float up = valid ? bd.pu[p] : 1e30f;
            const float vp = valid ? bd.pv[p] : 1e30f;
            if (lane == 0 && hsm) hsm[pp] = valid ? bd.ph[p] : 0.0;
            for (int a0 = 0; a0 < npad; a0 += 32) {
                const int a = a0 + lane;
                bool pass = false;
                if (a < npad) {
                    row[a] = 0.0;
                    const float du = up - cs.lu[a], dv = vp - cs.lv[a];
                    pass = du * du + dv * dv < kPrefilterR2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (pass)
                    ring[(tail + __popc(bal & ((1u << lane) - 1u))) & (kFillRing - 1)] = (pp << 16) | a;
                tail += __popc(bal);
                if (tail - head >= 32) round(32);
            }
        }
        if (tail > head) round(tail - head);
    } else {
        for (int pp = warp; pp < kSubChunk; pp += nw) {
            const int p = q0 + pp;
            const bool valid = p < p1;
            T* row = phi + pp * npad;
            const float up = valid ? bd.pu[p] : 1e30f;
            const float vp = valid ? bd.pv[p] : 1e30f;
            for (int a = lane; a < npad; a += 32) {
                float v = 0.0f;
                const float du = up - cs.x[a], dv = vp - cs.y[a];
                const float r2 = du * du + dv * dv;
                if (r2 < 1.0f) v = wendland<KIND, float>(sqrtf(r2));
                row[a] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Assembly kernel
// ---------------------------------------------------------------------------
template <int KIND, typename T>
__global__ void __launch_bounds__(kThreads) k_assemble(Binned bd, const int4* __restrict__ work,
                                                       int npad, T* __restrict__ B,
                                                       double* __restrict__ bvec,
                                                       int* __restrict__ support,
                                                       int* __restrict__ dropped, long long boff,
                                                       int rlo, int rhi) {
    // B holds the values from offset boff on, of rows rlo .. rhi-1 only (a block of an
    // out-of-core assembly; the whole B otherwise); bvec null: no b and support counts
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LocalCells lc;
    constexpr bool kFP64 = sizeof(T) == 8;
    const int4 wi = work[blockIdx.x];
    const int cell = wi.x, p0 = wi.y, p1 = wi.z;
    if (threadIdx.x == 0) describe_cells(bd, cell, lc);
    __syncthreads();
    const int n = lc.n;

    // carve shared memory
    unsigned char* sp = smem;
    T* phi = reinterpret_cast<T*>(sp);
    sp += sizeof(T) * kSubChunk * npad;
    CandSmem<T> cs;
    cs.rm = reinterpret_cast<RowMeta*>(sp);
    sp += sizeof(RowMeta) * npad;
    cs.x = reinterpret_cast<T*>(sp);
    sp += sizeof(T) * npad;
    cs.y = reinterpret_cast<T*>(sp);
    sp += sizeof(T) * npad;
    cs.s = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    cs.a9 = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    int* cnt = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    double* hsm = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * kSubChunk;
    cs.cval = nullptr;
    int* wl = nullptr;
    if constexpr (kFP64) {
        cs.lu = reinterpret_cast<float*>(sp);
        sp += sizeof(float) * npad;
        cs.lv = reinterpret_cast<float*>(sp);
        sp += sizeof(float) * npad;
        wl = reinterpret_cast<int*>(sp);
        sp += sizeof(int) * kFillRing * (kThreads / 32);
    } else {
        cs.lu = reinterpret_cast<float*>(cs.x);
        cs.lv = reinterpret_cast<float*>(cs.y);
    }

    stage_candidates<T>(bd, lc, cs, npad, nullptr);
    for (int a = threadIdx.x; a < npad; a += blockDim.x) cnt[a] = 0;
    __syncthreads();

    const int nb = npad / 4;
    const int nblk = nb * (nb + 1) / 2;
    const int npass = (nblk + kThreads - 1) / kThreads;
    double bacc0 = 0.0, bacc1 = 0.0;   // b for candidates tid and tid + kThreads

    for (int pass = 0; pass < npass; ++pass) {
        const int blk = pass * kThreads + threadIdx.x;
        const bool active = blk < nblk;
        int bi = 0, bj = 0;
        if (active) {
            int rem = blk;
            while (rem >= nb - bi) {
                rem -= nb - bi;
                ++bi;
            }
            bj = bi + rem;
        }
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);

        for (int q0 = p0; q0 < p1; q0 += kSubChunk) {
            __syncthreads();
            fill_phi<KIND, T>(bd, cs, n, npad, q0, p1, phi, kFP64 ? hsm : nullptr,
                              (kFP64 && pass == 0 && bvec) ? cnt : nullptr, wl);
            __syncthreads();
            const int np = min(kSubChunk, p1 - q0);
            if (kFP64 && pass == 0 && bvec) {
                for (int pp = 0; pp < np; ++pp) {
                    const double hp = hsm[pp];
                    if (threadIdx.x < n) bacc0 += hp * double(phi[pp * npad + threadIdx.x]);
                    if (threadIdx.x + kThreads < n)
                        bacc1 += hp * double(phi[pp * npad + threadIdx.x + kThreads]);
                }
            }
            if (active) {
                const T* pa = phi + 4 * bi;
                const T* pb = phi + 4 * bj;
                for (int pp = 0; pp < np; ++pp) {
                    T va[4], vb[4];
                    if constexpr (kFP64) {
                        const double2 a01 = *reinterpret_cast<const double2*>(pa + pp * npad);
                        const double2 a23 = *reinterpret_cast<const double2*>(pa + pp * npad + 2);
                        const double2 b01 = *reinterpret_cast<const double2*>(pb + pp * npad);
                        const double2 b23 = *reinterpret_cast<const double2*>(pb + pp * npad + 2);
                        va[0] = a01.x; va[1] = a01.y; va[2] = a23.x; va[3] = a23.y;
                        vb[0] = b01.x; vb[1] = b01.y; vb[2] = b23.x; vb[3] = b23.y;
                    } else {
                        const float4 a4 = *reinterpret_cast<const float4*>(pa + pp * npad);
                        const float4 b4 = *reinterpret_cast<const float4*>(pb + pp * npad);
                        va[0] = a4.x; va[1] = a4.y; va[2] = a4.z; va[3] = a4.w;
                        vb[0] = b4.x; vb[1] = b4.y; vb[2] = b4.z; vb[3] = b4.w;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fma(va[u], vb[v], acc[u][v]);
                }
            }
        }
        // scatter the thread's 4x4 block of the local Gram matrix into B (upper triangle):
        // entry (a, b), a <= b, to row s_a, column s_b, whose cell row is dy above s_a's
        if (active) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = 4 * bi + u;
                if (a >= n) continue;
                const int ka = cs.a9[a];
                const RowMeta rma = cs.rm[a];
                const int sa = cs.s[a];
                if (sa < rlo || sa >= rhi) continue;   // a row of another block
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int b = 4 * bj + v;
                    if (b >= n || b < a) continue;
                    const T val = acc[u][v];
                    if (val == T(0)) continue;
                    const int dy = cs.a9[b] / 3 - ka / 3;
                    const long long slot = upper_slot(rma, sa, cs.s[b], dy);
                    if (slot >= 0)
                        atomicAdd(&B[slot - boff], b == a ? T(0.5) * val : val);
                    else
                        atomicAdd(dropped, 1);
                }
            }
        }
    }
    if (kFP64 && bvec) {
        __syncthreads();
        if (threadIdx.x < n) {
            if (bacc0 != 0.0) atomicAdd(&bvec[cs.s[threadIdx.x]], bacc0);
            if (cnt[threadIdx.x]) atomicAdd(&support[cs.s[threadIdx.x]], cnt[threadIdx.x]);
        }
        if (threadIdx.x + kThreads < n) {
            const int a = threadIdx.x + kThreads;
            if (bacc1 != 0.0) atomicAdd(&bvec[cs.s[a]], bacc1);
            if (cnt[a]) atomicAdd(&support[cs.s[a]], cnt[a]);
        }
    }
}

// ---------------------------------------------------------------------------
// Matrix-free FP64 normal residual r = A^T (h - A c), optionally with support counts.
// ---------------------------------------------------------------------------
// With the polynomial (pa): e_p also subtracts k . (u_p, v_p, 1), r_k = sum_p e_p (u_p, v_p, 1)
// is added into pa.rk, and (assembly) A^T P into pa.E, P^T P and P^T h into pa.gp. r may be
// null (only the polynomial sums of the FP64 assembly are wanted).
template <int KIND, bool POLY>
__global__ void __launch_bounds__(kThreads) k_residual(Binned bd, const int4* __restrict__ work,
                                                       int npad, const double* __restrict__ c,
                                                       double* __restrict__ r,
                                                       int* __restrict__ support,
                                                       const long long* __restrict__ woff,
                                                       double* __restrict__ astore,
                                                       const long long* __restrict__ moff,
                                                       unsigned int* __restrict__ amask,
                                                       PolyArgs pa) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LocalCells lc;
    __shared__ double esm[kSubChunk];
    __shared__ double usm[kSubChunk], vsm[kSubChunk];
    constexpr bool poly = POLY;   // the polynomial's parts are compiled only into its instance
    if constexpr (!POLY) pa = PolyArgs{};
    const double pk0 = pa.k ? pa.k[0] : 0.0, pk1 = pa.k ? pa.k[1] : 0.0, pk2 = pa.k ? pa.k[2] : 0.0;
    double eacc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // A^T P of candidates tid, tid + kThreads
    double gacc[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // P^T P (6), P^T h (3)
    double rkacc[3] = {0.0, 0.0, 0.0};
    const int4 wi = work[blockIdx.x];
    const int cell = wi.x, p0 = wi.y, p1 = wi.z;
    if (threadIdx.x == 0) describe_cells(bd, cell, lc);
    __syncthreads();
    const int n = lc.n;
    unsigned char* sp = smem;
    double* phi = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * kSubChunk * npad;
    CandSmem<double> cs;
    cs.rm = nullptr;
    cs.x = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * npad;
    cs.y = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * npad;
    cs.cval = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * npad;
    cs.s = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    cs.a9 = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    int* cnt = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    double* hsm = reinterpret_cast<double*>(sp);
    sp += sizeof(double) * kSubChunk;
    cs.lu = reinterpret_cast<float*>(sp);
    sp += sizeof(float) * npad;
    cs.lv = reinterpret_cast<float*>(sp);
    sp += sizeof(float) * npad;
    int* wl = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * kFillRing * (kThreads / 32);
    // stored A: per candidate its mask, nonzero count and offset in the sub-chunk's values
    unsigned int* amsk = reinterpret_cast<unsigned int*>(sp);
    sp += sizeof(unsigned int) * npad;
    int* acnt = reinterpret_cast<int*>(sp);
    sp += sizeof(int) * npad;
    int* aoff = reinterpret_cast<int*>(sp);

    stage_candidates<double>(bd, lc, cs, npad, c);
    for (int a = threadIdx.x; a < npad; a += blockDim.x) cnt[a] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double racc0 = 0.0, racc1 = 0.0;
    for (int q0 = p0; q0 < p1; q0 += kSubChunk) {
        __syncthreads();
        fill_phi<KIND, double>(bd, cs, n, npad, q0, p1, phi, hsm, support ? cnt : nullptr, wl);
        const int np = min(kSubChunk, p1 - q0);
        if (poly && threadIdx.x < kSubChunk) {
            const int p = q0 + threadIdx.x;
            usm[threadIdx.x] = threadIdx.x < np ? (bd.px[p] - pa.xc) * pa.sx : 0.0;
            vsm[threadIdx.x] = threadIdx.x < np ? (bd.py[p] - pa.yc) * pa.sy : 0.0;
        }
        __syncthreads();
        if (astore) {
            // Keep the nonzeros of A for later residual passes, per sub-chunk: per candidate a
            // a 32-bit mask of the sub-chunk's points in a's support, and the values packed
            // candidate after candidate (each candidate's in point order) from the start of the
            // sub-chunk's region, so a later pass reads them with coalesced loads.
            const long long q = (q0 - p0) / kSubChunk;
            double* vals = astore + woff[blockIdx.x] + q * kSubChunk * n;
            unsigned int* msk = amask + moff[blockIdx.x] + q * n;
            for (int a = threadIdx.x; a < n; a += blockDim.x) {
                // Phi is +0.0 outside the support and positive inside: an integer test of
                // its bits keeps the mask off the FP64 pipe
                unsigned int m = 0;
                for (int pp = 0; pp < np; ++pp)
                    if (__double_as_longlong(phi[pp * npad + a]) != 0) m |= 1u << pp;
                amsk[a] = m;
                acnt[a] = __popc(m);
                msk[a] = m;
            }
            __syncthreads();
            block_scan_counts(acnt, n, aoff);
            for (int a = threadIdx.x; a < n; a += blockDim.x) {
                unsigned int m = amsk[a];
                double* dst = vals + aoff[a];
                for (int j = 0; m; ++j, m &= m - 1u) dst[j] = phi[(__ffs(m) - 1) * npad + a];
            }
        }
        // e_p = h_p - sum_a Phi[p][a] c_a - k . (u_p, v_p, 1)  (one warp per point; the sum
        // is skipped for c = 0, the assembly's pass)
        for (int pp = warp; pp < np; pp += nw) {
            double s = 0.0;
            if (c) {
                for (int a = lane; a < n; a += 32) s = fma(phi[pp * npad + a], cs.cval[a], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            }
            if (lane == 0)
                esm[pp] = hsm[pp] - s - (pa.k ? fma(pk0, usm[pp], fma(pk1, vsm[pp], pk2)) : 0.0);
        }
        __syncthreads();
        if (poly && threadIdx.x < np) {
            const double u = usm[threadIdx.x], v = vsm[threadIdx.x], e = esm[threadIdx.x];
            if (pa.rk) {
                rkacc[0] = fma(e, u, rkacc[0]);
                rkacc[1] = fma(e, v, rkacc[1]);
                rkacc[2] += e;
            }
            if (pa.gp) {
                const double hp = hsm[threadIdx.x];
                gacc[0] = fma(u, u, gacc[0]);
                gacc[1] = fma(u, v, gacc[1]);
                gacc[2] += u;
                gacc[3] = fma(v, v, gacc[3]);
                gacc[4] += v;
                gacc[5] += 1.0;
                gacc[6] = fma(hp, u, gacc[6]);
                gacc[7] = fma(hp, v, gacc[7]);
                gacc[8] += hp;
            }
        }
        // r_a += sum_p Phi[p][a] e_p (and A^T P: E_a += sum_p Phi[p][a] (u_p, v_p, 1)). With
        // the masks of the stored A at hand, only the points in a's support are visited (in
        // the same order: the zero terms add nothing); the FP64 pipe bounds this pass.
        if (astore) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int a = threadIdx.x + h * kThreads;
                if (a >= n) continue;
                double acc = h ? racc1 : racc0;
                double* ea = eacc + 3 * h;
                for (unsigned int m = amsk[a]; m; m &= m - 1u) {
                    const int pp = __ffs(m) - 1;
                    const double f = phi[pp * npad + a];
                    acc = fma(f, esm[pp], acc);
                    if (pa.E) {
                        ea[0] = fma(f, usm[pp], ea[0]);
                        ea[1] = fma(f, vsm[pp], ea[1]);
                        ea[2] += f;
                    }
                }
                if (h) racc1 = acc;
                else racc0 = acc;
            }
            continue;
        }
        for (int pp = 0; pp < np; ++pp) {
            const double e = esm[pp];
            if (threadIdx.x < n) {
                const double f = phi[pp * npad + threadIdx.x];
                racc0 = fma(f, e, racc0);
                if (pa.E) {
                    eacc[0] = fma(f, usm[pp], eacc[0]);
                    eacc[1] = fma(f, vsm[pp], eacc[1]);
                    eacc[2] += f;
                }
            }
            if (threadIdx.x + kThreads < n) {
                const double f = phi[pp * npad + threadIdx.x + kThreads];
                racc1 = fma(f, e, racc1);
                if (pa.E) {
                    eacc[3] = fma(f, usm[pp], eacc[3]);
                    eacc[4] = fma(f, vsm[pp], eacc[4]);
                    eacc[5] += f;
                }
            }
        }
    }
    __syncthreads();
    const int64_t M = bd.M;
    if (threadIdx.x < n) {
        const int sa = cs.s[threadIdx.x];
        if (r && racc0 != 0.0) atomicAdd(&r[sa], racc0);
        if (support && cnt[threadIdx.x]) atomicAdd(&support[sa], cnt[threadIdx.x]);
        if (pa.E)
            for (int j = 0; j < 3; ++j)
                if (eacc[j] != 0.0) atomicAdd(&pa.E[j * M + sa], eacc[j]);
    }
    if (threadIdx.x + kThreads < n) {
        const int a = threadIdx.x + kThreads;
        const int sa = cs.s[a];
        if (r && racc1 != 0.0) atomicAdd(&r[sa], racc1);
        if (support && cnt[a]) atomicAdd(&support[sa], cnt[a]);
        if (pa.E)
            for (int j = 0; j < 3; ++j)
                if (eacc[3 + j] != 0.0) atomicAdd(&pa.E[j * M + sa], eacc[3 + j]);
    }
    if (pa.rk) block_atomic_sum<3>(rkacc, pa.rk);
    if (pa.gp) {
        __syncthreads();
        // P^T P is symmetric: the six sums fill the 3 x 3 block, then P^T h
        double full[12] = {gacc[0], gacc[1], gacc[2], gacc[1], gacc[3], gacc[4],
                           gacc[2], gacc[4], gacc[5], gacc[6], gacc[7], gacc[8]};
        block_atomic_sum<12>(full, pa.gp);
    }
}

constexpr int kPointLanes = 8;   // lanes per point in the stored residual's A c products

// The same residual from the stored nonzeros of A (written by the FP64 pass of the FP32
// assembly): no distances, square roots or Wendland evaluations, and the two FP64 products
// run over the nonzeros only. Per sub-chunk: the packed values are copied into shared memory
// with coalesced loads (their per-candidate offsets from a scan of the masks' popcounts), then
// e_p = h_p - sum_a A_pa c_a (eight lanes per point over the candidates, a value found by
// the point's rank in the candidate's mask) and r_a += sum_p A_pa e_p (one thread per candidate
// over its values).
__global__ void __launch_bounds__(kThreads) k_residual_stored(Binned bd, const int4* __restrict__ work,
                                                              int npad, const double* __restrict__ c,
                                                              double* __restrict__ r,
                                                              const long long* __restrict__ woff,
                                                              const double* __restrict__ astore,
                                                              const long long* __restrict__ moff,
                                                              const unsigned int* __restrict__ amask,
                                                              PolyArgs pa) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LocalCells lc;
    __shared__ double esm[kSubChunk];
    __shared__ double hsm[kSubChunk];
    __shared__ double usm[kSubChunk], vsm[kSubChunk];
    const double pk0 = pa.k ? pa.k[0] : 0.0, pk1 = pa.k ? pa.k[1] : 0.0, pk2 = pa.k ? pa.k[2] : 0.0;
    double rkacc[3] = {0.0, 0.0, 0.0};
    const int4 wi = work[blockIdx.x];
    const int cell = wi.x, p0 = wi.y, p1 = wi.z;
    if (threadIdx.x == 0) describe_cells(bd, cell, lc);
    __syncthreads();
    const int n = lc.n;
    double* sval = reinterpret_cast<double*>(smem);         // [kSubChunk * npad] the sub-chunk's values
    double* cval = sval + kSubChunk * npad;
    int* sidx = reinterpret_cast<int*>(cval + npad);
    unsigned int* smask = reinterpret_cast<unsigned int*>(sidx + npad);
    int* acnt = reinterpret_cast<int*>(smask + npad);
    int* aoff = acnt + npad;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        int k = 0;
        while (a >= lc.off[k + 1]) ++k;
        const int sa = lc.start[k] + (a - lc.off[k]);
        sidx[a] = sa;
        cval[a] = c ? c[sa] : 0.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double racc0 = 0.0, racc1 = 0.0;
    for (int q0 = p0; q0 < p1; q0 += kSubChunk) {
        const int np = min(kSubChunk, p1 - q0);
        const long long q = (q0 - p0) / kSubChunk;
        const double* vals = astore + woff[blockIdx.x] + q * kSubChunk * n;
        const unsigned int* msk = amask + moff[blockIdx.x] + q * n;
        __syncthreads();
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            const unsigned int m = __ldcs(msk + a);
            smask[a] = m;
            acnt[a] = __popc(m);
        }
        __syncthreads();
        block_scan_counts(acnt, n, aoff);
        // the sub-chunk's packed values, coalesced
        const int nnz = aoff[n];
        for (int i = threadIdx.x; i < nnz; i += blockDim.x) sval[i] = __ldcs(vals + i);
        if (threadIdx.x < np) {
            hsm[threadIdx.x] = bd.ph[q0 + threadIdx.x];
            if (pa.k) {
                usm[threadIdx.x] = (bd.px[q0 + threadIdx.x] - pa.xc) * pa.sx;
                vsm[threadIdx.x] = (bd.py[q0 + threadIdx.x] - pa.yc) * pa.sy;
            }
        }
        __syncthreads();
        // kPointLanes lanes per point (a warp takes 32 / kPointLanes points), so that the
        // FP64 sum over each point's lanes takes log2(kPointLanes) steps: with a whole warp per
        // point the reduction's FP64 adds, not the products, dominated the pass
        {
            const int sub = lane / kPointLanes, sl = lane % kPointLanes;
            constexpr int kPerWarp = 32 / kPointLanes;
            for (int base = warp * kPerWarp; base < np; base += nw * kPerWarp) {
                const int pp = base + sub;
                const bool ok = pp < np;
                const unsigned int below = (1u << (pp & 31)) - 1u;
                double sacc = 0.0;
                if (ok) {
                    for (int a = sl; a < n; a += kPointLanes) {
                        const unsigned int m = smask[a];
                        if ((m >> pp) & 1u) sacc = fma(sval[aoff[a] + __popc(m & below)], cval[a], sacc);
                    }
                }
#pragma unroll
                for (int o = kPointLanes / 2; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                if (ok && sl == 0)
                    esm[pp] = hsm[pp] - sacc - (pa.k ? fma(pk0, usm[pp], fma(pk1, vsm[pp], pk2)) : 0.0);
            }
        }
        __syncthreads();
        if (pa.rk && threadIdx.x < np) {
            const double e = esm[threadIdx.x];
            rkacc[0] = fma(e, usm[threadIdx.x], rkacc[0]);
            rkacc[1] = fma(e, vsm[threadIdx.x], rkacc[1]);
            rkacc[2] += e;
        }
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            unsigned int m = smask[a];
            const double* col = sval + aoff[a];
            double acc = 0.0;
            for (int j = 0; m; ++j, m &= m - 1u) acc = fma(col[j], esm[__ffs(m) - 1], acc);
            if (a == threadIdx.x) racc0 += acc;
            else racc1 += acc;
        }
    }
    __syncthreads();
    if (threadIdx.x < n && racc0 != 0.0) atomicAdd(&r[sidx[threadIdx.x]], racc0);
    if (threadIdx.x + kThreads < n && racc1 != 0.0) atomicAdd(&r[sidx[threadIdx.x + kThreads]], racc1);
    if (pa.rk) block_atomic_sum<3>(rkacc, pa.rk);
}

// Storage of A per work item: its sub-chunks x the candidates of its cell's 3x3 block, 32
// value slots (size) and one mask (msize) per sub-chunk and candidate.
__global__ void k_work_sizes(Binned bd, const int4* __restrict__ work, int nwork,
                             long long* __restrict__ size, long long* __restrict__ msize) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int4 wi = work[w];
    const Grid& g = bd.g;
    const int ix = wi.x % g.gx, iy = wi.x / g.gx;
    const int xa = max(ix - 1, 0), xb = min(ix + 1, g.gx - 1);
    long long n = 0;
    for (int r = max(iy - 1, 0); r <= min(iy + 1, g.gy - 1); ++r)
        n += bd.cstart[r * g.gx + xb + 1] - bd.cstart[r * g.gx + xa];
    const long long nsub = (wi.z - wi.y + kSubChunk - 1) / kSubChunk;
    size[w] = nsub * kSubChunk * n;
    msize[w] = nsub * n;
}

template <typename T>
size_t asm_smem(int npad, bool resid) {
    size_t b = sizeof(T) * kSubChunk * npad + 2 * sizeof(T) * npad + 3 * sizeof(int) * npad +
               sizeof(double) * kSubChunk;
    if (resid) b += sizeof(double) * npad + 3 * sizeof(int) * npad + 16;
    else b += sizeof(RowMeta) * npad;
    if (sizeof(T) == 8)   // FP32 prefilter coordinates and the per-warp pair rings
        b += 2 * sizeof(float) * npad + sizeof(int) * kFillRing * (kThreads / 32);
    return b;
}

// The Gram entries of rows [rlo, rhi) from work items [w0, w1) into B (whose first value is
// value boff of the whole B); b and the support counts too when with_b (FP64, whole B only).
template <int KIND, typename T>
rbf_status launch_assemble(rbf_ctx* ctx, cudaStream_t st, int npad, T* B, bool with_b,
                           long long boff = 0, int rlo = 0, int rhi = -1, int w0 = 0, int w1 = -1) {
    const size_t sm = asm_smem<T>(npad, false);
    auto kfn = k_assemble<KIND, T>;
    RBF_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    if (rhi < 0) rhi = ctx->M;
    if (w1 < 0) w1 = ctx->nwork;
    if (w1 <= w0) return RBF_OK;
    kfn<<<w1 - w0, kThreads, sm, st>>>(view(ctx), ctx->work.as<int4>() + w0, npad, B,
                                       with_b ? ctx->bvec.as<double>() : nullptr,
                                       ctx->support.as<int>(), ctx->stats.as<int>() + 12, boff,
                                       rlo, rhi);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    return RBF_OK;
}

template <int KIND>
rbf_status launch_residual(rbf_ctx* ctx, const double* c, double* r, bool count, cudaStream_t st,
                           int npad, const PolyArgs& pa) {
    const size_t sm = asm_smem<double>(npad, true);
    const bool poly = pa.k || pa.E || pa.gp || pa.rk;
    auto kfn = poly ? k_residual<KIND, true> : k_residual<KIND, false>;
    RBF_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    const bool store = count && ctx->astore_ok;
    kfn<<<ctx->nwork, kThreads, sm, st>>>(view(ctx), ctx->work.as<int4>(), npad, c, r,
                                          count ? ctx->support.as<int>() : nullptr,
                                          store ? ctx->woff.as<long long>() : nullptr,
                                          store ? ctx->astore.as<double>() : nullptr,
                                          store ? ctx->moff_p : nullptr,
                                          store ? ctx->amask.as<unsigned int>() : nullptr, pa);
    RBF_CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    return RBF_OK;
}

}  // namespace

PolyArgs poly_args(rbf_ctx* ctx) {
    PolyArgs pa{};
    pa.xc = ctx->pxc;
    pa.yc = ctx->pyc;
    pa.sx = ctx->psx;
    pa.sy = ctx->psy;
    return pa;
}

namespace {
// A^T P into E, P^T P and P^T h into gp (zeroed first) with the FP64 pass over the points.
rbf_status poly_sums(rbf_ctx* ctx, cudaStream_t st, bool also_b) {
    const int M = ctx->M;
    rbf_status s;
    if ((s = ensure(ctx, ctx->pE, sizeof(double) * 3 * size_t(M), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->pE32, sizeof(float) * 3 * size_t(M), st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->pdev, sizeof(PolyDev), st)) != RBF_OK) return s;
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->pE.p, 0, sizeof(double) * 3 * size_t(M), st));
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->pdev.p, 0, sizeof(PolyDev), st));
    PolyArgs pa = poly_args(ctx);
    pa.E = ctx->pE.as<double>();
    pa.gp = ctx->pdev.as<PolyDev>()->gp;
    if (ctx->nwork == 0) return RBF_OK;
    const int npad = std::max(4, (ctx->max_cand + 3) / 4 * 4);
    // with also_b the pass is the FP32 assembly's FP64 pass (b, supports, stored A); else only
    // the polynomial sums (the FP64 assembly has b and the supports already)
    double* r = also_b ? ctx->bvec.as<double>() : nullptr;
    switch (ctx->kernel) {
        case RBF_W30: return launch_residual<0>(ctx, nullptr, r, also_b, st, npad, pa);
        case RBF_W31: return launch_residual<1>(ctx, nullptr, r, also_b, st, npad, pa);
        case RBF_W32: return launch_residual<2>(ctx, nullptr, r, also_b, st, npad, pa);
        default: return launch_residual<3>(ctx, nullptr, r, also_b, st, npad, pa);
    }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        b[i] = float(a[i]);
}
}  // namespace

namespace {
// Per cell row b (and b = gy): its first sorted row, that row's value offset (quads) and the
// first assembly work item of the row's cells.
__global__ void k_band_table(Grid g, int M, int nwork, const int* __restrict__ cstart,
                             const int64_t* __restrict__ roff, const int* __restrict__ wstart,
                             long long* __restrict__ tab) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > g.gy) return;
    const int row = b < g.gy ? cstart[b * g.gx] : M;
    tab[3 * b] = row;
    tab[3 * b + 1] = roff[row];
    tab[3 * b + 2] = b < g.gy ? wstart[b * g.gx] : nwork;
}

// The pinned host copy of B, mapped into the device's address space.
rbf_status ensure_host_b(rbf_ctx* ctx, size_t bytes, cudaStream_t st) {
    bytes = std::max<size_t>(bytes, 256);
    if (ctx->bhost && ctx->bhost_bytes >= bytes) return RBF_OK;
    if (ctx->bhost) {
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFreeHost(ctx->bhost);
        ctx->bhost = ctx->bhost_dev = nullptr;
        ctx->bhost_bytes = 0;
    }
    void* p = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped) != cudaSuccess || !p) {
        cudaGetLastError();
        return set_err(ctx, RBF_ERR_ALLOC, "pinned host memory for B");
    }
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess || !d) {
        cudaGetLastError();
        cudaFreeHost(p);
        return set_err(ctx, RBF_ERR_CUDA, "device address of the host copy of B");
    }
    ctx->bhost = p;
    ctx->bhost_dev = d;
    ctx->bhost_bytes = bytes;
    return RBF_OK;
}

// Out-of-core assembly of B (Eq. 13-16: B assembled block by block within a memory bound):
// consecutive cell rows are grouped into blocks whose stored values fit b_device_mb MB; each
// block is assembled on the device from the work items of the point cells within one cell row
// of it (every point whose support touches a row of the block), keeping only the entries of
// its rows, and copied to the host copy of B, which the solver then reads through its device
// address. Blocks hold at least one cell row whatever the bound.
template <int KIND, typename T>
rbf_status assemble_blocks(rbf_ctx* ctx, cudaStream_t st, int npad) {
    const Grid& g = ctx->g;
    const int gy = g.gy;
    rbf_status s;
    if ((s = ensure(ctx, ctx->bandtab, sizeof(long long) * 3 * size_t(gy + 1), st)) != RBF_OK) return s;
    k_band_table<<<div_up(gy + 1, 256), 256, 0, st>>>(g, ctx->M, ctx->nwork, ctx->cstart.as<int>(),
                                                      ctx->roff.as<int64_t>(), ctx->wstart.as<int>(),
                                                      ctx->bandtab.as<long long>());
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    std::vector<long long> tab(3 * size_t(gy + 1));
    RBF_CUDA_TRY(cudaMemcpyAsync(tab.data(), ctx->bandtab.p, sizeof(long long) * tab.size(),
                                 cudaMemcpyDeviceToHost, st));
    RBF_CUDA_TRY(cudaStreamSynchronize(st));
    auto val = [&](int b) { return 4 * tab[3 * b + 1]; };
    const long long budget = std::max<long long>(
        4, (long long)(ctx->b_device_mb * 1048576.0 / double(sizeof(T))));
    struct Blk { int b0, b1; };
    std::vector<Blk> blocks;
    long long maxv = 0;
    for (int b = 0; b < gy;) {
        int b1 = b + 1;
        while (b1 < gy && val(b1 + 1) - val(b) <= budget) ++b1;
        blocks.push_back({b, b1});
        maxv = std::max(maxv, val(b1) - val(b));
        b = b1;
    }
    if ((s = ensure(ctx, ctx->bblock, sizeof(T) * size_t(std::max<long long>(maxv, 1)), st)) != RBF_OK)
        return s;
    T* blk = ctx->bblock.as<T>();
    char* host = static_cast<char*>(ctx->bhost);
    for (const Blk& k : blocks) {
        const long long v0 = val(k.b0), v1 = val(k.b1);
        if (v1 == v0) continue;
        const int r0 = int(tab[3 * k.b0]), r1 = int(tab[3 * k.b1]);
        const int w0 = int(tab[3 * std::max(k.b0 - 1, 0) + 2]);
        const int w1 = int(tab[3 * std::min(k.b1 + 1, gy) + 2]);
        RBF_CUDA_TRY(cudaMemsetAsync(blk, 0, sizeof(T) * size_t(v1 - v0), st));
        if ((s = launch_assemble<KIND, T>(ctx, st, npad, blk, false, v0, r0, r1, w0, w1)) != RBF_OK)
            return s;
        RBF_CUDA_TRY(cudaMemcpyAsync(host + sizeof(T) * size_t(v0), blk, sizeof(T) * size_t(v1 - v0),
                                     cudaMemcpyDeviceToHost, st));
    }
    ctx->bblocks = int64_t(blocks.size());
    return RBF_OK;
}

template <typename T>
rbf_status assemble_b(rbf_ctx* ctx, int kernel, cudaStream_t st, int npad, bool host_b, bool with_b) {
    if (host_b) {
        switch (kernel) {
            case RBF_W30: return assemble_blocks<0, T>(ctx, st, npad);
            case RBF_W31: return assemble_blocks<1, T>(ctx, st, npad);
            case RBF_W32: return assemble_blocks<2, T>(ctx, st, npad);
            default: return assemble_blocks<3, T>(ctx, st, npad);
        }
    }
    T* B = ctx->bvals.as<T>();
    switch (kernel) {
        case RBF_W30: return launch_assemble<0, T>(ctx, st, npad, B, with_b);
        case RBF_W31: return launch_assemble<1, T>(ctx, st, npad, B, with_b);
        case RBF_W32: return launch_assemble<2, T>(ctx, st, npad, B, with_b);
        default: return launch_assemble<3, T>(ctx, st, npad, B, with_b);
    }
}
}  // namespace

rbf_status assemble_run(rbf_ctx* ctx, int kernel, int prec, cudaStream_t st, bool with_poly) {
    const int M = ctx->M;
    ctx->astore_ok = false;   // rewritten below by an FP32 assembly
    ctx->poly = false;
    const size_t vb = prec == RBF_FP64 ? sizeof(double) : sizeof(float);
    rbf_status s;
    // a batch of tiles keeps B on the device (its tiles are small)
    const bool host_b = ctx->b_device_mb > 0.0 && ctx->T == 0;
    ctx->b_in_host = false;
    ctx->bblocks = 0;
    if (host_b) {
        // every value is written by the blocks' copies, which cover [0, nvals) end to end
        if (ctx->bvals.p) {
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            release(ctx, ctx->bvals);
        }
        if ((s = ensure_host_b(ctx, vb * std::max<int64_t>(ctx->nvals, 1), st)) != RBF_OK) return s;
        ctx->b_in_host = true;
    } else {
        if (ctx->bhost) {
            RBF_CUDA_TRY(cudaStreamSynchronize(st));
            cudaFreeHost(ctx->bhost);
            ctx->bhost = ctx->bhost_dev = nullptr;
            ctx->bhost_bytes = 0;
        }
        if ((s = ensure(ctx, ctx->bvals, vb * std::max<int64_t>(ctx->nvals, 1), st)) != RBF_OK) return s;
        RBF_CUDA_TRY(cudaMemsetAsync(ctx->bvals.p, 0, vb * ctx->nvals, st));
    }
    if ((s = ensure(ctx, ctx->bvec, sizeof(double) * M, st)) != RBF_OK) return s;
    if ((s = ensure(ctx, ctx->support, sizeof(int) * M, st)) != RBF_OK) return s;
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->bvec.p, 0, sizeof(double) * M, st));
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->support.p, 0, sizeof(int) * M, st));
    // stats[12]: Gram entries that found no slot in their row (none by construction)
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->stats.as<int>() + 12, 0, sizeof(int), st));
    if (with_poly) {
        // the polynomial's frame: the bounding box centred and scaled to [-1, 1]
        const Grid& g = ctx->g;
        const double w = g.gx * g.h, hh = g.gy * g.h;
        ctx->pxc = g.x0 + 0.5 * w;
        ctx->pyc = g.y0 + 0.5 * hh;
        ctx->psx = 2.0 / w;
        ctx->psy = 2.0 / hh;
    }
    auto finish_poly = [&](bool also_b) -> rbf_status {
        if (!with_poly) return RBF_OK;
        rbf_status ps = poly_sums(ctx, st, also_b);
        if (ps != RBF_OK) return ps;
        k_to_float<<<std::min(div_up(3 * int64_t(M), 256), 4096), 256, 0, st>>>(
            ctx->pE.as<double>(), ctx->pE32.as<float>(), 3 * int64_t(M));
        ctx->launches += 1;
        RBF_CUDA_TRY(cudaGetLastError());
        ctx->poly = true;
        return RBF_OK;
    };
    if (ctx->nwork == 0) return finish_poly(false);
    const int npad = std::max(4, (ctx->max_cand + 3) / 4 * 4);
    if (prec == RBF_FP64) {
        if ((s = assemble_b<double>(ctx, kernel, st, npad, host_b, true)) != RBF_OK) return s;
        if (host_b) {
            // the blocks overlap in work items: b and the support counts by the FP64 pass
            if ((s = residual_run(ctx, nullptr, ctx->bvec.as<double>(), true, st)) != RBF_OK) return s;
        }
        return finish_poly(false);
    }
    if ((s = assemble_b<float>(ctx, kernel, st, npad, host_b, false)) != RBF_OK) return s;
    // Storage for the FP64 values of A, written by the pass below and read by every later
    // residual pass (the refinement). Without room for it the residual stays matrix-free.
    ctx->astore_ok = false;
    if (ctx->store_a) {
        const int nw = ctx->nwork;
        if ((s = ensure(ctx, ctx->woff, sizeof(long long) * 2 * (nw + 1), st)) != RBF_OK) return s;
        if ((s = ensure(ctx, ctx->wsize, sizeof(long long) * 2 * nw, st)) != RBF_OK) return s;
        long long* vsize = ctx->wsize.as<long long>();
        long long* voff = ctx->woff.as<long long>();
        k_work_sizes<<<div_up(nw, 256), 256, 0, st>>>(view(ctx), ctx->work.as<int4>(), nw, vsize,
                                                      vsize + nw);
        ctx->launches += 1;
        int64_t* vs64 = reinterpret_cast<int64_t*>(vsize);
        int64_t* vo64 = reinterpret_cast<int64_t*>(voff);
        if ((s = scan_i64(ctx, vs64, vo64, nw, st)) != RBF_OK) return s;
        if ((s = scan_i64(ctx, vs64 + nw, vo64 + nw + 1, nw, st)) != RBF_OK) return s;
        long long* hp = static_cast<long long*>(ctx->hpinned) + 40;
        RBF_CUDA_TRY(cudaMemcpyAsync(hp, voff + nw, sizeof(long long), cudaMemcpyDeviceToHost, st));
        RBF_CUDA_TRY(cudaMemcpyAsync(hp + 1, voff + 2 * nw + 1, sizeof(long long),
                                     cudaMemcpyDeviceToHost, st));
        RBF_CUDA_TRY(cudaStreamSynchronize(st));
        const long long nval = hp[0], nmask = hp[1];
        if (ensure(ctx, ctx->astore, sizeof(double) * std::max<long long>(nval, 1), st) == RBF_OK &&
            ensure(ctx, ctx->amask, sizeof(unsigned int) * std::max<long long>(nmask, 1), st) == RBF_OK)
            ctx->astore_ok = true;
        else
            ctx->err.clear();   // no room: matrix-free residual
        ctx->moff_p = voff + nw + 1;
    }
    // b = A^T h and the support counts in FP64: the residual with c = 0 (with the polynomial,
    // the same pass also sums A^T P, P^T P and P^T h)
    RBF_CUDA_TRY(cudaMemsetAsync(ctx->bvec.p, 0, sizeof(double) * M, st));
    if (with_poly) return finish_poly(true);
    return residual_run(ctx, nullptr, ctx->bvec.as<double>(), true, st);
}

rbf_status residual_run(rbf_ctx* ctx, const double* c_sorted, double* r_sorted, bool count,
                        cudaStream_t st, bool poly) {
    PolyArgs pa = poly_args(ctx);
    if (poly) {
        PolyDev* pd = ctx->pdev.as<PolyDev>();
        pa.k = pd->k64;
        pa.rk = pd->rk;
        RBF_CUDA_TRY(cudaMemsetAsync(pd->rk, 0, 3 * sizeof(double), st));
    }
    if (ctx->nwork == 0) return RBF_OK;
    const double* c = c_sorted;   // nullptr stands for c = 0, i.e. r = A^T h
    const int npad = std::max(4, (ctx->max_cand + 3) / 4 * 4);
    if (!count && ctx->astore_ok) {
        const size_t sm = sizeof(double) * (kSubChunk + 1) * npad + 4 * sizeof(int) * npad + 16;
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_residual_stored, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(sm)));
        k_residual_stored<<<ctx->nwork, kThreads, sm, st>>>(view(ctx), ctx->work.as<int4>(), npad, c,
                                                            r_sorted, ctx->woff.as<long long>(),
                                                            ctx->astore.as<double>(), ctx->moff_p,
                                                            ctx->amask.as<unsigned int>(), pa);
        RBF_CUDA_TRY(cudaGetLastError());
        ctx->launches += 1;
        return RBF_OK;
    }
    switch (ctx->kernel) {
        case RBF_W30: return launch_residual<0>(ctx, c, r_sorted, count, st, npad, pa);
        case RBF_W31: return launch_residual<1>(ctx, c, r_sorted, count, st, npad, pa);
        case RBF_W32: return launch_residual<2>(ctx, c, r_sorted, count, st, npad, pa);
        default: return launch_residual<3>(ctx, c, r_sorted, count, st, npad, pa);
    }
}

}  // namespace rbf
