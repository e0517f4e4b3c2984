// Learned warm start: radial features of each centre, a 32-64-64-1 network (BF16 weights,
// FP32 accumulation) that predicts an initial c_j, and its training (gradient by
// back-propagation, Adam). Not part of the paper, which solves from c = 0; the solver's
// answer does not depend on the start, only its iteration count does.
//
// Features of centre j: the points with r = ||x_i - xi_j|| / R < 1 fall into 16 annuli
// (bin floor(16 r)); per bin, the fraction of the support's points in it and their mean
// height over the system's height scale sigma = sqrt(mean h^2). The bin is decided from
// FP32 cell-local coordinates and, within 1e-4 of a bin edge (or of the support's edge),
// again in FP64 as sqrt(dx*dx + dy*dy) / R with every operation rounded once, so the bins
// are those of an FP64 evaluation of that expression.
//
// Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3. The FP32 master weights are rounded to
// BF16 when staged into shared memory (as FP32 values), biases and activations stay FP32,
// every product is accumulated in FP32. Prediction c0_j = sigma * y_j.
//
// Training: loss mean (y - t)^2 over a minibatch; each block back-propagates 64 samples
// (four threads per sample) and writes its partial gradient; the Adam kernel sums the
// partials in block order (deterministic) and updates the FP32 master weights.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "rbf_cg.cuh"

namespace rbf {
namespace {

constexpr int NB = 16;             // radial bins
constexpr int NF = 2 * NB;         // features
constexpr int NH = 64;             // hidden width
// offsets of the flat parameter vector
constexpr int oW1 = 0, ob1 = oW1 + NH * NF, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH,
              ob3 = oW3 + NH, kNParam = ob3 + 1;
static_assert(kNParam == RBF_MLP_NPARAM, "parameter count");

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

// Per-tile (or whole-system) sums of h^2 and point counts, one warp per cell (lanes over its
// points).
constexpr int kHWarps = 8;
__global__ void __launch_bounds__(kHWarps * 32)
    k_height_sums(Binned bd, const int* __restrict__ rowtile, double* __restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kHWarps + (threadIdx.x >> 5);
    if (c >= bd.g.ncell) return;
    const int p0 = bd.pstart[c], p1 = bd.pstart[c + 1];
    if (p1 == p0) return;
    double sum = 0.0;
    for (int p = p0 + lane; p < p1; p += 32) {
        const double h = bd.ph[p];
        sum = fma(h, h, sum);
    }
    sum = warp_sum_d(sum);
    if (lane == 0) {
        const int t = rowtile ? rowtile[c / bd.g.gx] : 0;
        atomicAdd(&acc[2 * t], sum);
        atomicAdd(&acc[2 * t + 1], double(p1 - p0));
    }
}

__global__ void k_height_scale(const double* __restrict__ acc, int T, double* __restrict__ sigma) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) sigma[t] = acc[2 * t + 1] > 0.0 ? sqrt(acc[2 * t] / acc[2 * t + 1]) : 1.0;
}

// Features, one block per cell: the threads take the candidate points of the cell's 3x3
// neighbourhood (the three rows of cells are contiguous point ranges) and test each against
// every centre of the cell (up to kFCent at a time, their cell-local coordinates staged in
// shared memory), accumulating per-centre bins with shared-memory atomics. A block per cell
// keeps dense cells (ten times the mean point count and more in clustered data) from
// serialising on one warp. The per-bin means are formed in FP32 (relative error ~1e-7).
constexpr int kFThreads = 256;
constexpr int kFCent = 64;

__global__ void __launch_bounds__(kFThreads)
    k_features_cell(Binned bd, const double* __restrict__ sigma, float* __restrict__ feat) {
    __shared__ int cnt[kFCent][NB];
    __shared__ float hs[kFCent][NB];   // FP32 height sums: native shared atomics
    __shared__ float su[kFCent], sv[kFCent];
    const Grid& g = bd.g;
    const int cell = blockIdx.x;
    const int cs = bd.cstart[cell], m = bd.cstart[cell + 1] - cs;
    if (m == 0) return;
    const int ix = cell % g.gx, iy = cell / g.gx;
    const int xa = max(ix - 1, 0), xb = min(ix + 1, g.gx - 1);
    // per row of cells: its point range and the first point of its 2nd and 3rd cell
    int r0[3], r1[3], e1[3], e2[3];
    float roy[3];
    int nrow = 0;
    for (int r = max(iy - 1, 0); r <= min(iy + 1, g.gy - 1); ++r) {
        const int* ps = bd.pstart + r * g.gx;
        r0[nrow] = ps[xa];
        e1[nrow] = xa + 1 <= xb ? ps[xa + 1] : ps[xb + 1];
        e2[nrow] = xa + 2 <= xb ? ps[xa + 2] : ps[xb + 1];
        r1[nrow] = ps[xb + 1];
        roy[nrow] = float(r - iy);
        ++nrow;
    }
    const double inv_sig = 1.0 / sigma[bd.crow[cs].w];
    for (int a0 = 0; a0 < m; a0 += kFCent) {
        const int ma = min(kFCent, m - a0);
        for (int e = threadIdx.x; e < ma * NB; e += kFThreads) {
            cnt[e / NB][e % NB] = 0;
            hs[e / NB][e % NB] = 0.0f;
        }
        for (int a = threadIdx.x; a < ma; a += kFThreads) {
            su[a] = bd.cu[cs + a0 + a];
            sv[a] = bd.cv[cs + a0 + a];
        }
        __syncthreads();
        for (int rr = 0; rr < nrow; ++rr) {
            for (int p = r0[rr] + int(threadIdx.x); p < r1[rr]; p += kFThreads) {
                // the point's cell column relative to the centre cell
                const int q = xa + (p >= e1[rr]) + (p >= e2[rr]);
                const float pux = bd.pu[p] + float(q - ix), pv = bd.pv[p] + roy[rr];
                const float ph = float(bd.ph[p]);
                for (int a = 0; a < ma; ++a) {
                    const float du = pux - su[a], dv = pv - sv[a];
                    const float r2 = du * du + dv * dv;
                    if (r2 >= kPrefilterR2) continue;
                    const float rf = sqrtf(r2) * float(NB);
                    const float fr = rf - floorf(rf);
                    int k;
                    if (fr < 1e-4f || fr > 1.0f - 1e-4f || rf > float(NB) - 1e-3f) {
                        // near a bin edge or the support's edge: decide in FP64, every
                        // operation rounded once, as sqrt(dx*dx + dy*dy) / R
                        const int s = cs + a0 + a;
                        const double dx = bd.px[p] - bd.cx[s], dy = bd.py[p] - bd.cy[s];
                        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                        const double rr2 = __ddiv_rn(__dsqrt_rn(d2), g.R);
                        if (!(rr2 < 1.0)) continue;
                        k = int(floor(double(NB) * rr2));
                    } else {
                        if (rf >= float(NB)) continue;
                        k = int(rf);
                    }
                    atomicAdd(&cnt[a][k], 1);
                    atomicAdd(&hs[a][k], ph);
                }
            }
        }
        __syncthreads();
        // 16 threads per centre, one per bin; every thread takes every pass (the shuffles
        // below involve the whole warp)
        for (int a1 = 0; a1 < ma; a1 += kFThreads / NB) {
            const int a = a1 + (threadIdx.x >> 4);
            const int k = threadIdx.x & (NB - 1);
            const bool ok = a < ma;
            const int ck = ok ? cnt[a][k] : 0;
            // support count: the 16 bins of this centre (the other half-warp holds another)
            int n = ck;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o, NB);
            if (ok) {
                const int s = cs + a0 + a;
                float* out = feat + (long long)bd.cperm[s] * NF;
                out[k] = float(ck) / float(max(n, 1));
                out[NB + k] = ck > 0 ? hs[a][k] / float(ck) * float(inv_sig) : 0.0f;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------

struct __align__(16) SmemW {
    float W1[NH * NF], b1[NH], W2[NH * NH], b2[NH], W3[NH], b3;
};

__device__ __forceinline__ float bf16r(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

__device__ void stage_weights(const float* __restrict__ p, SmemW& w) {
    for (int i = threadIdx.x; i < NH * NF; i += blockDim.x) w.W1[i] = bf16r(p[oW1 + i]);
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) w.W2[i] = bf16r(p[oW2 + i]);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        w.b1[i] = p[ob1 + i];
        w.b2[i] = p[ob2 + i];
        w.W3[i] = bf16r(p[oW3 + i]);
    }
    if (threadIdx.x == 0) w.b3 = p[ob3];
}

constexpr int kFwdThreads = 128;

// y_i for feature rows i < n (one thread per row).
__global__ void __launch_bounds__(kFwdThreads)
    k_mlp_forward(const float* __restrict__ params, const float* __restrict__ feat, long long n,
                  float* __restrict__ y) {
    __shared__ SmemW w;
    stage_weights(params, w);
    __syncthreads();
    const long long i = blockIdx.x * (long long)kFwdThreads + threadIdx.x;
    if (i >= n) return;
    float x[NF];
    const float4* xr = reinterpret_cast<const float4*>(feat + i * NF);
#pragma unroll
    for (int k = 0; k < NF / 4; ++k) {
        const float4 q = xr[k];
        x[4 * k] = q.x;
        x[4 * k + 1] = q.y;
        x[4 * k + 2] = q.z;
        x[4 * k + 3] = q.w;
    }
    float a1[NH];
#pragma unroll
    for (int o = 0; o < NH; ++o) {
        float z = w.b1[o];
        const float4* wr = reinterpret_cast<const float4*>(w.W1 + o * NF);
#pragma unroll
        for (int k = 0; k < NF / 4; ++k) {
            const float4 q = wr[k];
            z = fmaf(q.x, x[4 * k], z);
            z = fmaf(q.y, x[4 * k + 1], z);
            z = fmaf(q.z, x[4 * k + 2], z);
            z = fmaf(q.w, x[4 * k + 3], z);
        }
        a1[o] = fmaxf(z, 0.0f);
    }
    float out = w.b3;
    for (int o = 0; o < NH; ++o) {
        float z = w.b2[o];
        const float4* wr = reinterpret_cast<const float4*>(w.W2 + o * NH);
#pragma unroll
        for (int k = 0; k < NH / 4; ++k) {
            const float4 q = wr[k];
            z = fmaf(q.x, a1[4 * k], z);
            z = fmaf(q.y, a1[4 * k + 1], z);
            z = fmaf(q.z, a1[4 * k + 2], z);
            z = fmaf(q.w, a1[4 * k + 3], z);
        }
        out = fmaf(w.W3[o], fmaxf(z, 0.0f), out);
    }
    y[i] = out;
}

// c0[cperm[s]] = sigma_tile * y[cperm[s]] for every sorted centre s.
__global__ void k_warm_scale(Binned bd, const double* __restrict__ sigma, const float* __restrict__ y,
                             double* __restrict__ c0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bd.M) return;
    const int j = bd.cperm[s];
    c0[j] = sigma[bd.crow[s].w] * double(y[j]);
}

// The network's training target of every centre: t[cperm[s]] = c[cperm[s]] / sigma_tile
// (c in the caller's order), the inverse of k_warm_scale.
__global__ void k_mlp_targets(Binned bd, const double* __restrict__ sigma,
                              const double* __restrict__ c, float* __restrict__ t) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bd.M) return;
    const int j = bd.cperm[s];
    t[j] = float(c[j] / sigma[bd.crow[s].w]);
}

constexpr int kGS = 64;           // samples per gradient block
constexpr int kGT = 4 * kGS;      // threads: four per sample
constexpr int kPad = NH + 1;      // padded activation rows

struct SmemG {
    SmemW w;
    float X[kGS][NF + 1];
    float A1[kGS][kPad];          // relu(z1)
    float A2[kGS][kPad];          // relu(z2)
    float D2[kGS][kPad];          // dL/dz2
    float D1[kGS][kPad];          // dL/dz1
    float dy[kGS];
    float y[kGS];
};

// Partial gradient (and loss) of the minibatch's samples b*64 .. b*64+63 (sample i is
// idx[i] when idx is given), scaled by 1/n_total, written to part[b][0 .. kNParam] (the
// loss share at index kNParam).
__global__ void __launch_bounds__(kGT)
    k_mlp_grad(const float* __restrict__ params, const float* __restrict__ feat,
               const float* __restrict__ target, const int* __restrict__ idx, long long n,
               float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char gsm[];
    SmemG& S = *reinterpret_cast<SmemG*>(gsm);
    stage_weights(params, S.w);
    const int tid = threadIdx.x;
    const int sl = tid >> 2, q = tid & 3;          // sample slot, quarter of the hidden units
    const long long i = blockIdx.x * (long long)kGS + sl;
    const bool valid = i < n;
    const long long row = valid ? (idx ? (long long)idx[i] : i) : 0;
    for (int k = q; k < NF; k += 4) S.X[sl][k] = valid ? feat[row * NF + k] : 0.0f;
    __syncthreads();
    // forward, layer 1: this thread's 16 hidden units
    for (int o = q * 16; o < q * 16 + 16; ++o) {
        float z = S.w.b1[o];
        for (int k = 0; k < NF; ++k) z = fmaf(S.w.W1[o * NF + k], S.X[sl][k], z);
        S.A1[sl][o] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    float yp = 0.0f;
    for (int o = q * 16; o < q * 16 + 16; ++o) {
        float z = S.w.b2[o];
        for (int k = 0; k < NH; ++k) z = fmaf(S.w.W2[o * NH + k], S.A1[sl][k], z);
        const float a = fmaxf(z, 0.0f);
        S.A2[sl][o] = a;
        yp = fmaf(S.w.W3[o], a, yp);
    }
    // the four quarters of a sample are consecutive lanes
    yp += __shfl_xor_sync(0xffffffffu, yp, 1);
    yp += __shfl_xor_sync(0xffffffffu, yp, 2);
    const float inv_n = 1.0f / float(n);
    if (q == 0) {
        const float yy = yp + S.w.b3;
        const float e = valid ? yy - target[row] : 0.0f;
        S.y[sl] = e;
        S.dy[sl] = 2.0f * e * inv_n;
    }
    __syncthreads();
    // backward: dz2 = dy W3 [z2 > 0] (a2 > 0 iff z2 > 0), then dz1 = (W2^T dz2) [z1 > 0]
    const float dys = S.dy[sl];
    for (int o = q * 16; o < q * 16 + 16; ++o) S.D2[sl][o] = S.A2[sl][o] > 0.0f ? dys * S.w.W3[o] : 0.0f;
    __syncthreads();
    for (int k = q * 16; k < q * 16 + 16; ++k) {
        float d = 0.0f;
        for (int o = 0; o < NH; ++o) d = fmaf(S.w.W2[o * NH + k], S.D2[sl][o], d);
        S.D1[sl][k] = S.A1[sl][k] > 0.0f ? d : 0.0f;
    }
    __syncthreads();
    // weight gradients over the block's samples
    float* out = part + (long long)blockIdx.x * (kNParam + 1);
    for (int e = tid; e < NH * NF; e += kGT) {
        const int o = e / NF, k = e % NF;
        float g = 0.0f;
        for (int s = 0; s < kGS; ++s) g = fmaf(S.D1[s][o], S.X[s][k], g);
        out[oW1 + e] = g;
    }
    for (int e = tid; e < NH * NH; e += kGT) {
        const int o = e / NH, k = e % NH;
        float g = 0.0f;
        for (int s = 0; s < kGS; ++s) g = fmaf(S.D2[s][o], S.A1[s][k], g);
        out[oW2 + e] = g;
    }
    for (int o = tid; o < NH; o += kGT) {
        float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
        for (int s = 0; s < kGS; ++s) {
            g1 += S.D1[s][o];
            g2 += S.D2[s][o];
            g3 = fmaf(S.dy[s], S.A2[s][o], g3);
        }
        out[ob1 + o] = g1;
        out[ob2 + o] = g2;
        out[oW3 + o] = g3;
    }
    if (tid == 0) {
        float g = 0.0f, L = 0.0f;
        for (int s = 0; s < kGS; ++s) {
            g += S.dy[s];
            L = fmaf(S.y[s], S.y[s], L);
        }
        out[ob3] = g;
        out[kNParam] = L * inv_n;
    }
}

// Sum of the partials in block order (FP64); optionally an Adam step on the FP32 master
// weights (step t >= 1) or just the gradient into grad.
__global__ void k_mlp_reduce_adam(const float* __restrict__ part, int nblk, float* __restrict__ params,
                                  float* __restrict__ m, float* __restrict__ v, int step, double lr,
                                  float* __restrict__ grad, double* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNParam) return;
    double g = 0.0;
    for (int b = 0; b < nblk; ++b) g += double(part[(long long)b * (kNParam + 1) + p]);
    if (p == kNParam) {
        if (loss) *loss = g;
        return;
    }
    if (grad) grad[p] = float(g);
    if (step > 0) {
        const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
        const double mm = b1 * double(m[p]) + (1.0 - b1) * g;
        const double vv = b2 * double(v[p]) + (1.0 - b2) * g * g;
        m[p] = float(mm);
        v[p] = float(vv);
        const double mh = mm / (1.0 - pow(b1, double(step)));
        const double vh = vv / (1.0 - pow(b2, double(step)));
        params[p] = float(double(params[p]) - lr * mh / (sqrt(vh) + eps));
    }
}

}  // namespace

// ---- host side ----

// sigma per tile (T) or for the whole system (1) into ctx->sigma.
static rbf_status height_scales(rbf_ctx* ctx, cudaStream_t st) {
    const int T = std::max(ctx->T, 1);
    rbf_status s;
    if ((s = ensure(ctx, ctx->sigma, sizeof(double) * 3 * T, st)) != RBF_OK) return s;
    double* acc = ctx->sigma.as<double>() + T;
    RBF_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 2 * T, st));
    k_height_sums<<<div_up(ctx->g.ncell, kHWarps), kHWarps * 32, 0, st>>>(
        view(ctx), ctx->T > 0 ? ctx->rowtile.as<int>() : nullptr, acc);
    k_height_scale<<<div_up(T, 256), 256, 0, st>>>(acc, T, ctx->sigma.as<double>());
    ctx->launches += 2;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status features_run(rbf_ctx* ctx, float* feat, double* sigma_out, cudaStream_t st) {
    rbf_status s = height_scales(ctx, st);
    if (s != RBF_OK) return s;
    // one block per cell (cells without centres return at once)
    k_features_cell<<<ctx->g.ncell, kFThreads, 0, st>>>(
        view(ctx), ctx->sigma.as<double>(), feat);
    ctx->launches += 1;
    if (sigma_out)
        RBF_CUDA_TRY(cudaMemcpyAsync(sigma_out, ctx->sigma.p, sizeof(double) * std::max(ctx->T, 1),
                                     cudaMemcpyDeviceToDevice, st));
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status mlp_forward_run(rbf_ctx* ctx, const float* params, const float* feat, int64_t n, float* y,
                           cudaStream_t st) {
    if (n <= 0) return RBF_OK;
    k_mlp_forward<<<div_up(n, kFwdThreads), kFwdThreads, 0, st>>>(params, feat, n, y);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status mlp_targets_run(rbf_ctx* ctx, const double* c, float* target, cudaStream_t st) {
    // the height scales of the binned system (tiles)
    rbf_status s = height_scales(ctx, st);
    if (s != RBF_OK) return s;
    k_mlp_targets<<<div_up(ctx->M, 256), 256, 0, st>>>(view(ctx), ctx->sigma.as<double>(), c, target);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status warm_start_run(rbf_ctx* ctx, const float* params, double* c0, cudaStream_t st) {
    const int M = ctx->M;
    rbf_status s;
    if ((s = ensure(ctx, ctx->feat, sizeof(float) * (size_t(M) * NF + M), st)) != RBF_OK) return s;
    float* feat = ctx->feat.as<float>();
    float* y = feat + size_t(M) * NF;
    if ((s = features_run(ctx, feat, nullptr, st)) != RBF_OK) return s;
    if ((s = mlp_forward_run(ctx, params, feat, M, y, st)) != RBF_OK) return s;
    k_warm_scale<<<div_up(M, 256), 256, 0, st>>>(view(ctx), ctx->sigma.as<double>(), y, c0);
    ctx->launches += 1;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

rbf_status mlp_step_run(rbf_ctx* ctx, float* params, float* m, float* v, int step, double lr,
                        const float* feat, const float* target, const int* idx, int64_t n,
                        float* grad, double* loss, cudaStream_t st) {
    const int nblk = div_up(n, kGS);
    rbf_status s = ensure(ctx, ctx->mlp_part, sizeof(float) * size_t(nblk) * (kNParam + 1), st);
    if (s != RBF_OK) return s;
    RBF_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(sizeof(SmemG))));
    k_mlp_grad<<<nblk, kGT, sizeof(SmemG), st>>>(params, feat, target, idx, n, ctx->mlp_part.as<float>());
    k_mlp_reduce_adam<<<div_up(kNParam + 1, 256), 256, 0, st>>>(ctx->mlp_part.as<float>(), nblk, params,
                                                                m, v, step, lr, grad, loss);
    ctx->launches += 2;
    RBF_CUDA_TRY(cudaGetLastError());
    return RBF_OK;
}

}  // namespace rbf
