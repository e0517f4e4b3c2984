// Device-side definitions shared by the librbf kernels: the Wendland basis
// functions, the uniform cell grid, the context layout and CUDA error helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rbf.h"

namespace rbf {

// Largest number of centres in a 3x3 cell neighbourhood that the assembly and
// residual kernels stage in shared memory (a point's candidate list).
constexpr int kMaxCand = 384;
// Points per staged sub-chunk of the fused assembly / residual passes.
constexpr int kSubChunk = 32;
// Largest cell (centres per cell) whose diagonal block is inverted for the block-Jacobi
// preconditioner; larger cells fall back to the scalar diagonal.
constexpr int kMaxBlock = 32;
// Points per assembly work item (one CTA); larger cells are split.
constexpr int kWorkPoints = 256;
// Relative enlargement of the cell side over R, so that a pair closer than R is never
// more than one computed cell apart whatever the rounding of the cell index.
constexpr double kCellMargin = 1.0 + 1.0 / 1073741824.0;

// ---------------------------------------------------------------------------
// Wendland functions phi_{3,s}(r), r = ||x - xi|| / R in [0, 1) (Table 2, Eq. 18).
// Callers apply the cut-off (r >= 1 -> 0) themselves. KIND 2 is phi_{3,2} / 3.
// ---------------------------------------------------------------------------
template <int KIND, typename T>
__device__ __forceinline__ T wendland(T r) {
    const T t = T(1) - r;
    const T t2 = t * t;
    if constexpr (KIND == 0) {
        return t2;
    } else if constexpr (KIND == 1) {
        const T t4 = t2 * t2;
        return t4 * (T(4) * r + T(1));
    } else if constexpr (KIND == 2) {
        const T t6 = t2 * t2 * t2;
        return t6 * ((T(35) * r + T(18)) * r + T(3)) * T(1.0 / 3.0);
    } else {
        const T t4 = t2 * t2;
        const T t8 = t4 * t4;
        return t8 * (((T(32) * r + T(25)) * r + T(8)) * r + T(1));
    }
}

// Exact form of the support test ||x - xi|| / R < 1 in FP64 with the operation order
// sqrt(dx*dx + dy*dy) / R (separately rounded products and sum, IEEE sqrt and division),
// so that integer support counts agree bit for bit with a CPU evaluation of the same
// expression. The division is only evaluated for pairs within 1e-9 of the boundary.
__device__ __forceinline__ bool inside_exact(double dx, double dy, double R, double R2) {
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (d2 < R2 * (1.0 - 1e-9)) return true;
    if (d2 > R2 * (1.0 + 1e-9)) return false;
    return __ddiv_rn(__dsqrt_rn(d2), R) < 1.0;
}

// The same test, also handing out the separately rounded squared distance it computed.
__device__ __forceinline__ bool inside_exact_d2(double dx, double dy, double R, double R2, double& d2) {
    d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (d2 < R2 * (1.0 - 1e-9)) return true;
    if (d2 > R2 * (1.0 + 1e-9)) return false;
    return __ddiv_rn(__dsqrt_rn(d2), R) < 1.0;
}

// Square root of a >= 0 for distances whose Wendland values feed sums checked to far above
// FP64 rounding (surfaces, B, b): the FP32 hardware estimate y of 1/sqrt(a) (relative error e,
// about 2^-22) and one Newton step on the square root itself, s <- s + y (a - s^2) / 2 from
// s = a y, which leaves a relative error of about e^2 (~3e-14). Four FP64 operations besides
// the two conversions -- this GPU's FP64 pipe is what the evaluation and the assembly's FP64
// pass are bound by -- against eight for sqrt_nr. The range test runs in FP32; outside FP32's
// normal range (and at 0) it falls back to sqrt.
__device__ __forceinline__ double sqrt_fast(double a) {
    const float af = float(a);
    if (!(af > 1e-30f && af < 1e30f)) return sqrt(a);
    const double y = double(rsqrtf(af));
    const double s = a * y;
    return fma(0.5 * y, fma(-s, s, a), s);
}

// Square root of a >= 0 in FP64 by Newton-Raphson iteration for the reciprocal square root,
// y <- y (3 - a y^2) / 2, seeded with the FP32 hardware estimate rsqrtf (about 23 correct
// bits; the step doubles them to about 46), followed by one Newton step on sqrt itself,
// s <- s + y (a - s^2) / 2, which squares the remaining relative error (below FP64 rounding).
// About seven FP64 operations instead of a full IEEE square root; the result is within a few
// units in the last place of sqrt(a) (checked against sqrt by the library's self-test entry
// point).
__device__ __forceinline__ double sqrt_nr(double a) {
    if (!(a > 0.0)) return 0.0;
    if (a < 1e-30 || a > 1e30) return sqrt(a);   // outside the FP32 seed's normal range
    double y = double(rsqrtf(float(a)));
    y = y * fma(-0.5 * a, y * y, 1.5);
    const double s = a * y;
    return fma(0.5 * y, fma(-s, s, a), s);
}

// Lower bound on the squared distance, in units of R^2, above which an FP32 test from
// cell-local coordinates (absolute error about 1e-7 R per coordinate) certainly means
// outside the support; pairs below it get the exact FP64 test.
constexpr float kPrefilterR2 = 1.00002f;

// ---------------------------------------------------------------------------
// Uniform grid of square cells of side h = R * kCellMargin over a bounding box.
// Cell key = iy * gx + ix (row-major, x fastest); items outside are clamped.
// ---------------------------------------------------------------------------
struct Grid {
    double x0, y0;     // lower-left corner
    double h, invh;    // cell side and its inverse
    double R, invR, R2;
    int gx, gy;        // cells per axis
    int ncell;         // gx * gy
};

__device__ __forceinline__ int cell_ix(const Grid& g, double x) {
    double f = floor((x - g.x0) * g.invh);
    f = fmin(fmax(f, 0.0), double(g.gx - 1));
    return int(f);
}
__device__ __forceinline__ int cell_iy(const Grid& g, double y) {
    double f = floor((y - g.y0) * g.invh);
    f = fmin(fmax(f, 0.0), double(g.gy - 1));
    return int(f);
}

// Stored upper triangle of B (Section 5 keeps only the upper triangle), row by row in the
// cell-sorted centre order, where a cell's centres are ordered by x (then by input index), so
// that the centres of one cell row ("band") are ordered by x. Row s keeps B[s][t] for the
// t >= s that can be nonzero -- centres closer than 2R, i.e. inside the 2R disc around xi_s --
// as three contiguous column ranges of the sorted order:
//   seg 0: its own band, t in [s, e0): x_t < x_s + 2R
//   seg 1: the band above, the centres whose x lies within the half-chord of the 2R disc at
//          that band's lower edge
//   seg 2: two bands above, likewise (empty when that edge is 2R or more above xi_s)
// (a small relative margin widens each range, so FP32 rounding of the assembly's support
// test can never place an entry outside it). Each range is widened to column bounds that are
// multiples of 4 (lo rounded down, hi rounded up) and the three are stored back to back from
// an offset that is a multiple of 4, so the value of column t always sits at an offset equal
// to t modulo 4: a lane reads the values of a column quad (t..t+3, t a multiple of 4) with one
// aligned 4-vector load. Slots whose column is outside the row's own range (t < s in seg 0,
// the widening) hold exact zeros.
// The diagonal value is stored halved: the SpMV adds every stored value once to the row sum
// and once to the column sum, so a halved diagonal counts once in y = B x with no special
// case. Readers of B itself (preconditioner set-up, export) double it.
struct __align__(16) RowMeta {
    unsigned int off;   // offset of the row's first stored value (column s & ~3), in quads
    int lo1, lo2;       // first column (a multiple of 4) of seg 1 and seg 2
    unsigned int len;   // stored quads of seg 0 | seg 1 << 10 | seg 2 << 20 (10 bits each)
};
constexpr int kLenBits = 10;
constexpr int kMaxSegQuads = (1 << kLenBits) - 1;
__host__ __device__ __forceinline__ int seg_quads(unsigned int len, int k) {
    return int((len >> (kLenBits * k)) & unsigned(kMaxSegQuads));
}

// Relative widening of the 2R disc that bounds each row's column ranges.
constexpr double kDiscMargin = 1.0 + 1e-5;

// Rows of one row group: consecutive rows of one band whose column ranges one warp sweeps
// together (lanes over the union of the rows' ranges, column sums kept in registers across
// the rows).
constexpr int kGroupRows = 8;

// A row group and the union of its rows' column ranges per segment (bounds multiples of 4,
// in column quads), which is what the SpMV's lanes sweep.
struct __align__(16) GroupDesc {
    int r0, n;          // first row and number of rows (1 .. kGroupRows)
    int lo0, q0;        // seg 0 union: columns [lo0, lo0 + 4 q0)
    int lo1, q1;        // seg 1 union
    int lo2, q2;        // seg 2 union
};

// What the SpMV reads of a row group before its values: the GroupDesc and the RowMeta of its
// rows (zeros past n) in one 160-byte record, fetched by ten lanes in one round trip.
constexpr int kGroupRecInt4 = 2 + kGroupRows;
struct __align__(16) GroupRec {
    GroupDesc d;
    RowMeta rows[kGroupRows];
};

// Offset of B[s][t] (s <= t, t in band(s) + k) in the value array, or -1 if the row keeps no
// slot for t.
__host__ __device__ __forceinline__ long long upper_slot(const RowMeta& rm, int s, int t, int k) {
    const int lo = k == 0 ? (s & ~3) : (k == 1 ? rm.lo1 : rm.lo2);
    const int n0 = 4 * seg_quads(rm.len, 0), n1 = 4 * seg_quads(rm.len, 1);
    const int len = 4 * seg_quads(rm.len, k);
    const int base = k == 0 ? 0 : (k == 1 ? n0 : n0 + n1);
    const int d = t - lo;
    if (d < 0 || d >= len) return -1;
    return 4LL * rm.off + base + d;
}

// Linear polynomial of Section 3 (Eq. 6-10), P_i = (x_i, y_i, 1), handled in a centred and
// scaled frame u = (x - xc) sx, v = (y - yc) sy (|u|, |v| <= 1 over the bounding box), which
// spans the same functions and keeps the polynomial block of Eq. 10 well scaled. Arguments of
// the FP64 passes over the points; null pointers switch the parts off.
struct PolyArgs {
    double xc, yc, sx, sy;   // the frame
    const double* k;         // [3] coefficients (of u, v, 1) of the current iterate (residual)
    double* E;               // [3 * M] A^T P, column-major (u, v, 1), sorted order (assembly)
    double* gp;              // [12] P^T P (row-major 3 x 3) then P^T h (assembly)
    double* rk;              // [3] P^T (h - A c - P k) (residual)
};

// Views of the context's device buffers passed by value to kernels.
struct Binned {
    Grid g;
    int M, N;
    const int* cstart;      // [ncell+1] first sorted centre of each cell
    const int* pstart;      // [ncell+1] first sorted point of each cell
    const double* cx;       // [M] sorted centre coordinates (FP64, global frame)
    const double* cy;
    const float* cu;        // [M] centre coordinates local to its cell, units of R (FP32)
    const float* cv;
    const double* px;       // [N] sorted point coordinates and heights (FP64)
    const double* py;
    const double* ph;
    const float* pu;        // [N] point coordinates local to its cell, units of R (FP32)
    const float* pv;
    const int* cperm;       // [M] sorted -> caller centre index
    const RowMeta* rmeta;   // [M] stored row of B of each sorted centre
    const GroupRec* gdesc;  // [ngroup] row groups (description and rows' RowMeta), row order
    int ngroup;
    const int64_t* bjoff;   // [ncell+1] offset of each cell's inverse diagonal block
    const int4* crow;       // [M] {first sorted centre, centre count, cell, tile} of each centre's cell
};

// ---------------------------------------------------------------------------
// Host-side error helpers
// ---------------------------------------------------------------------------
#define RBF_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::rbf::cuda_fail(ctx, _e, #expr, __FILE__, __LINE__); \
    } while (0)

rbf_status cuda_fail(rbf_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

}  // namespace rbf
