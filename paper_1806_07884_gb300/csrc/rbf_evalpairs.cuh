// The evaluation engine shared by the single-system and the tiled (moving-window) kernels:
// f at 32 queries by one warp as a stream of (centre, query) pairs (Eq. 3 restricted to the
// compact supports, Eq. 18).
#pragma once

#include "rbf_internal.h"

namespace rbf {

constexpr int kEvalRing = 64;        // pending pairs: < 32 before an append of <= 32

struct EvalWarpSmem {
    int s[kEvalRing];                // centre (sorted index)
    int q[kEvalRing];                // query lane
    double f[32];                    // per query: the sum so far
};

// One lane's query, located by the caller in the frame of the binned coordinates: (x, y) in
// that frame, (ix, iy) its cell of the (packed) grid, (uq, vq) its FP32 coordinates in units
// of R relative to that cell's corner.
struct EvalQuery {
    double x, y;
    int ix, iy;
    float uq, vq;
    bool valid;
};

// The frame shared by the warp's 32 queries: support radius (R, R^2, 1/R in the binned
// coordinates) and the cells a query's 3x3 neighbourhood is clamped to (a tile's band of the
// packed grid, or the whole grid).
struct EvalFrame {
    double R, R2, invR;
    int col_lo, col_hi, row_lo, row_hi;
};

// f at 32 queries by one warp, lane l owning query l: the result in the owner lane (0 for
// a lane without a query). Query after query, the lanes sweep the centres of its 3x3 cells
// (three contiguous ranges) with the FP32 prefilter and append the passing (centre, query)
// pairs to the warp's ring; whenever 32 pairs wait, the lanes take one pair each through the
// FP64 distance, exact support test and Wendland value, and a segmented shuffle reduction
// (pairs of one query are contiguous) gives each query's part of the round to one lane, which
// adds it to the query's sum in shared memory. The FP64 pipe thus sees full rounds of pairs
// inside the support, and each query's set-up runs once, in its own lane.
template <int KIND>
__device__ __forceinline__ double eval_pairs32(const Binned& bd, const double* __restrict__ c,
                                               const EvalQuery& qy, const EvalFrame& fr,
                                               int lane, EvalWarpSmem& sm) {
    const Grid& g = bd.g;
    const double x = qy.x, y = qy.y;
    const int ix = qy.ix, iy = qy.iy;
    const float uq = qy.uq, vq = qy.vq;
    sm.f[lane] = 0.0;
    __syncwarp();
    const unsigned vmask = __ballot_sync(0xffffffffu, qy.valid);
    int head = 0, tail = 0;          // pending pairs [head, tail) of the ring (warp-uniform)

    // one round: lane k takes pending pair head + k (k < cnt)
    auto round = [&](int cnt) {
        __syncwarp();
        const bool act = lane < cnt;
        const int slot = (head + lane) & (kEvalRing - 1);
        const int sidx = act ? sm.s[slot] : 0;
        const int key = act ? sm.q[slot] : -1;
        const double xq = __shfl_sync(0xffffffffu, x, key & 31);
        const double yq = __shfl_sync(0xffffffffu, y, key & 31);
        double t = 0.0;
        if (act) {
            const double dx = xq - bd.cx[sidx], dy = yq - bd.cy[sidx];
            double d2;
            if (inside_exact_d2(dx, dy, fr.R, fr.R2, d2)) {
                const double r = sqrt_fast(d2) * fr.invR;
                t = c[sidx] * wendland<KIND, double>(r);
            }
        }
        // segmented sum towards the first lane of each query's run
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double tv = __shfl_down_sync(0xffffffffu, t, o);
            const int kv = __shfl_down_sync(0xffffffffu, key, o);
            if (lane + o < 32 && kv == key) t += tv;
        }
        const int kp = __shfl_up_sync(0xffffffffu, key, 1);
        if (act && (lane == 0 || kp != key)) sm.f[key] += t;
        head += cnt;
        __syncwarp();
    };

    for (unsigned pend = vmask; pend; pend &= pend - 1) {
        const int qn = __ffs(pend) - 1;
        const int qix = __shfl_sync(0xffffffffu, ix, qn), qiy = __shfl_sync(0xffffffffu, iy, qn);
        const float quq = __shfl_sync(0xffffffffu, uq, qn), qvq = __shfl_sync(0xffffffffu, vq, qn);
        const int xa = max(qix - 1, fr.col_lo), xb = min(qix + 1, fr.col_hi);
        int rs[3], rl[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int row = qiy - 1 + d;
            if (row < fr.row_lo || row > fr.row_hi) {
                rs[d] = rl[d] = 0;
            } else {
                rs[d] = bd.cstart[row * g.gx + xa];
                rl[d] = bd.cstart[row * g.gx + xb + 1] - rs[d];
            }
        }
        const int n = rl[0] + rl[1] + rl[2];
        for (int a0 = 0; a0 < n; a0 += 32) {
            const int a = a0 + lane;
            bool pass = false;
            int s = 0;
            if (a < n) {
                const int d = a < rl[0] ? 0 : (a < rl[0] + rl[1] ? 1 : 2);
                s = rs[d] + (d == 0 ? a : (d == 1 ? a - rl[0] : a - rl[0] - rl[1]));
                // the candidate in the query cell's frame (its cell is ox, oy cells away)
                const int cc = bd.crow[s].z;
                const float ox = float(cc % g.gx - qix), oy = float(cc / g.gx - qiy);
                const float du = quq - (bd.cu[s] + ox), dv = qvq - (bd.cv[s] + oy);
                pass = du * du + dv * dv < kPrefilterR2;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const int slot = (tail + __popc(bal & ((1u << lane) - 1u))) & (kEvalRing - 1);
                sm.s[slot] = s;
                sm.q[slot] = qn;
            }
            tail += __popc(bal);
            if (tail - head >= 32) round(32);
        }
    }
    if (tail > head) round(tail - head);
    return sm.f[lane];
}

}  // namespace rbf
