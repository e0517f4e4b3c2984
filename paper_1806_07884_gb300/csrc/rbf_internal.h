// Host-side context of librbf and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rbf_common.cuh"

// Device state of the linear polynomial of Section 3 (Eq. 10): the assembly's P^T P and P^T h,
// the inverse of P^T P (the preconditioner's block of the three polynomial rows), the FP64
// iterate and residual of the polynomial unknowns, and the CG recurrences of the three rows
// (kept in FP64 whatever the solver's precision: one thread updates them per iteration).
struct PolyDev {
    double gp[12];       // P^T P (row-major 3 x 3), then P^T h
    double ginv[9];      // (P^T P)^-1
    double k64[3];       // FP64 iterate (coefficients of u, v, 1)
    double rk[3];        // FP64 residual P^T (h - A c - P k)
    double uk[2][3];     // CG: preconditioned residual u of the three rows, by iteration parity
    double xk[3], pk[3], sk[3], rkc[3];   // CG: solution, direction, s = K p, residual
    double bk[3];        // right-hand side of the three rows in the current CG solve
    double tmp[4];
};

// A device buffer obtained from the context's allocator.
struct rbf_buf {
    void* p = nullptr;
    size_t bytes = 0;
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct rbf_ctx {
    int device = 0;
    rbf_alloc_fn alloc = nullptr;
    rbf_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;

    // ---- binning (rbf_bin) ----
    rbf::Grid g{};
    int M = 0, N = 0;
    int max_cand = 0;          // largest 3x3 neighbourhood centre count
    int max_cell_pts = 0;      // largest points-per-cell count
    int nwork = 0;             // assembly work items
    int64_t nvals = 0;         // stored B values (rows of the upper triangle, see RowMeta)
    bool binned = false;

    rbf_buf ccount, pcount;    // [ncell] counts, reused as scratch
    rbf_buf cstart, pstart;    // [ncell+1]
    rbf_buf ckey, crank;       // [M]
    rbf_buf pkey, prank;       // [N]
    rbf_buf cx, cy, cu, cv, cperm;      // [M]
    rbf_buf px, py, ph, pu, pv;         // [N]
    rbf_buf rmeta;             // [M] RowMeta: the stored row of B of each sorted centre
    rbf_buf rsize, roff;       // [M], [M+1] int64: row lengths and offsets (pairs of values)
    rbf_buf gcount, gstart;    // [gy], [gy+1]: row groups per cell row and their first index
    rbf_buf gdesc;             // [ngroup] GroupDesc
    int ngroup = 0;            // row groups of the stored B
    rbf_buf wcount, wstart;    // [ncell], [ncell+1]
    rbf_buf bjsize, bjoff;     // [ncell], [ncell+1] int64: inverse diagonal blocks (m <= 32)
    rbf_buf crow;              // [M] int4 {cell start, cell count, cell, tile} per sorted centre
    int64_t nbj = 0;           // values of all inverse diagonal blocks
    rbf_buf work;              // [nwork] int4 {cell, p0, p1, 0}
    rbf_buf scan_tmp;          // block sums of the device scans
    rbf_buf stats;             // small int counters read back by rbf_bin

    // ---- assembly (rbf_assemble) ----
    int kernel = -1;
    int prec = -1;
    bool assembled = false;
    rbf_buf bvals;             // B values (double or float)
    // B beyond device memory (rbf_set_param "b_device_mb" > 0): the values live in pinned host
    // memory mapped into the device's address space (over NVLink-C2C on GB300), assembled in
    // blocks of cell rows through the device buffer bblock of at most b_device_mb MB
    double b_device_mb = 0.0;
    bool b_in_host = false;    // the last assembly's B lives in host memory
    void* bhost = nullptr;     // pinned host copy of B
    size_t bhost_bytes = 0;
    void* bhost_dev = nullptr; // its device address
    rbf_buf bblock;            // device block of B under assembly
    rbf_buf bandtab;           // [3 (gy + 1)] per cell row: first row, its value offset, first work item
    int64_t bblocks = 0;       // blocks of the last out-of-core assembly
    rbf_buf bvec;              // [M] b = A^T h, sorted order (FP64)
    rbf_buf support;           // [M] points inside each support, sorted order
    // FP64 values of A per work item (points x candidates of the cell's 3x3 block), kept by
    // the FP32 assembly for the refinement's residual passes
    rbf_buf astore, amask, woff, wsize;   // values, masks, their offsets per work item
    const long long* moff_p = nullptr;    // mask offsets (second half of woff)
    bool astore_ok = false;
    int store_a = 1;           // rbf_set_param("store_a")

    // ---- linear polynomial (Section 3, Eq. 6-10): rbf_assemble_poly / rbf_solve_poly ----
    bool poly = false;         // the last assembly added the polynomial blocks of Eq. 10
    double pxc = 0.0, pyc = 0.0, psx = 1.0, psy = 1.0;   // frame u = (x - xc) sx, v = (y - yc) sy
    rbf_buf pE, pE32;          // [3 M] A^T P (FP64), and its FP32 copy for the FP32 solver
    rbf_buf pdev;              // PolyDev
    rbf_buf pepart;            // per-block partial sums of E^T u (both parities)

    // ---- solver workspace ----
    // FP64 refinement vectors (sorted order): the solution and the matrix-free residual
    rbf_buf x, r;
    // CG workspace per precision ([0] FP64, [1] FP32): kCgVecs vectors of length M (x, u, p,
    // r[2], s[2], w[2] -- r, s, w double-buffered by iteration parity) and dinv
    rbf_buf cgv[2], dinv, dinv32;
    rbf_buf bjinv, bjinv32;    // inverse diagonal cell blocks (block-Jacobi preconditioner)
    rbf_buf partial;           // per-block partial sums
    rbf_buf scal;              // device scalars (struct CgScalars)
    rbf_buf csort;             // [M] FP64 coefficients in sorted order (evaluation)
    void* hpinned = nullptr;   // pinned host scratch for scalar read-back (4 KiB)
    int64_t launches = 0;      // kernels launched by this context (graph nodes included)
    int spmv_blocks_per_sm[2] = {0, 0};   // occupancy of the SpMV kernels, [0] FP64, [1] FP32
    int persist_blocks_per_sm[2] = {0, 0};  // of the persistent solve kernel (-1: not resident)
    int cg_persistent = -1;          // single systems' CG loop: 1 persistent kernel, 0 graph,
                                     // -1 chosen by size and precision
    int cg_barrier_extra = 0;        // test hook: the persistent solve's barriers never complete
    // solver parameters (rbf_set_param)
    double inner_tol = 1e-3;   // relative tolerance of each FP32 inner solve
    int max_refine = 30;       // FP64 refinement steps of RBF_FP32_REFINE
    cudaStream_t capture_stream = nullptr;   // private stream used only to capture graphs
    // CG solve graphs (conditional WHILE loop), [0] FP64, [1] FP32, and what they were built for
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        int ncell = 0, M = 0, gx = 0, ngroup = 0;
        const void* crow = nullptr;
        const void* key[12] = {};
    };
    SolveGraph cg_graph[2];
    bool solved = false;       // solver workspace exists

    // ---- batched tiles (rbf_bin_tiles / rbf_solve_tiles) ----
    int T = 0;                       // tiles packed into this system (0: one plain system)
    std::vector<rbf_tile> tiles;     // the caller's tile descriptors
    rbf_buf tdesc;                   // [T] per-tile placement (device)
    rbf_buf rowtile;                 // [gy] tile owning each cell row, -1 between bands
    rbf_buf tcg;                     // per-tile CG scalars and results
    rbf_buf twork;                   // per-tile cell and row ranges, CG work lists
    rbf_buf tred;                    // per-tile reductions (norms, pinned counts, scales)
    rbf_buf qoff;                    // [T+1] query offsets of rbf_eval_tiles
    void* hbt = nullptr;             // pinned host mirror of tcg / tred
    size_t hbt_bytes = 0;
    // launch configuration of the batched CG loop, [0] FP64, [1] FP32
    struct TileTuning {
        int spmv_bps = 0, chunk = 0, nt = 0;   // SpMV blocks per SM, cells per SpMV item,
                                               // update block size (0: not chosen yet)
        double us_per_iter = 0.0;              // measured by the autotuner (0: not tuned)
        int ngroup = 0, M = 0;                 // shape it was chosen for
        int64_t nvals = 0;
    };
    TileTuning tune[2];
    int autotune = 1;                // tune on the first batched solve of a new shape
    bool no_tune_now = false;        // a promotion's FP64 finish: keep the default
    int force_bps = 0, force_chunk = 0, force_nt = 0;   // fixed configuration (0: automatic)
    struct TileGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key[13] = {};
        int T = 0, M = 0, ngroup = 0, bps = 0, chunk = 0, nt = 0;
    };
    TileGraph bt_graph[2];

    // ---- moving window (rbf_bin_windows): the windows are the tiles of a batch ----
    bool win_on = false;             // the batch was laid out by rbf_bin_windows
    int win_wx = 0, win_wy = 0;
    double win_overlap = 0.0, win_margin = 0.0, win_bbox[4] = {0.0, 0.0, 1.0, 1.0};
    int64_t win_M = 0, win_N = 0;    // centres and points summed over the windows
    rbf_buf win_eval;                // grid evaluation: per window its node ranges, item offsets
    rbf_buf win_edges;               // window bounds: per axis data lo / hi, extended lo / hi
    rbf_buf win_count;               // per window: centre and point counts, scatter cursors
    rbf_buf win_off;                 // per window: first centre, first point (and the totals)
    rbf_buf win_c;                   // the windows' centres (x then y), window after window
    rbf_buf win_cidx;                // input index of each of them
    rbf_buf win_p;                   // the windows' points (x, y, h), window after window

    // ---- learned warm start (rbf_features / rbf_warm_start / rbf_mlp_*) ----
    rbf_buf sigma;                   // [T or 1] height scales, then 2 T sums
    rbf_buf feat;                    // [M x 32] features and [M] network outputs
    rbf_buf mlp_part;                // per-block partial gradients
};

namespace rbf {

// The stored B values as the kernels address them: the device buffer, or the mapped host copy
// when the last assembly kept B in host memory.
template <typename T>
inline T* bvals_dev(const rbf_ctx* ctx) {
    return static_cast<T*>(ctx->b_in_host ? ctx->bhost_dev : ctx->bvals.p);
}

rbf_status set_err(rbf_ctx* ctx, rbf_status s, const char* msg);
rbf_status ensure(rbf_ctx* ctx, rbf_buf& b, size_t bytes, cudaStream_t st);
void release(rbf_ctx* ctx, rbf_buf& b);
Binned view(const rbf_ctx* ctx);

// rbf_bin.cu
rbf_status bin_run(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                   const double* py, const double* h, cudaStream_t st);
// exclusive scan of n int32 counts into n+1 outputs (int32 or int64), device-wide
rbf_status scan_i32(rbf_ctx* ctx, const int* in, int* out, int n, cudaStream_t st);
rbf_status scan_i64(rbf_ctx* ctx, const int64_t* in, int64_t* out, int n, cudaStream_t st);

// rbf_batch.cu: the tile-aware parts of the binning of a batched system
rbf_status tiles_count(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                       const double* py, const double* h, cudaStream_t st);
rbf_status tiles_scatter(rbf_ctx* ctx, const double* cx, const double* cy, const double* px,
                         const double* py, const double* h, cudaStream_t st);
rbf_status tiles_scatter_centres(rbf_ctx* ctx, const double* cx, const double* cy, cudaStream_t st);
rbf_status tiles_group_ranges(rbf_ctx* ctx, cudaStream_t st);
void tiles_release(rbf_ctx* ctx);
rbf_status bin_tiles_run(rbf_ctx* ctx, const rbf_tile* tiles, int T, const double* cx,
                         const double* cy, int64_t Mtot, const double* px, const double* py,
                         const double* h, int64_t Ntot, cudaStream_t st);
rbf_status solve_tiles_run(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                           int min_support, rbf_tile_info* tinfo, rbf_solve_info* info,
                           cudaStream_t st);
rbf_status autotune_run(rbf_ctx* ctx, cudaStream_t st);
// timing hooks of a batched system: the batched SpMV alone, or whole batched CG iterations
rbf_status bench_tiles_run(rbf_ctx* ctx, int reps, bool spmv_only, cudaStream_t st);
rbf_status window_bin_run(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M,
                          const double* px, const double* py, const double* h, int64_t N,
                          double R, const double* bbox, int wx, int wy, double overlap,
                          double margin, cudaStream_t st);
rbf_status window_eval_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                           int64_t Q, int nx, int ny, const double* box, double* f, cudaStream_t st);
rbf_status eval_tiles_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                          const int64_t* qoff, int nx, int ny, double* f, cudaStream_t st);

// rbf_mlp.cu
rbf_status features_run(rbf_ctx* ctx, float* feat, double* sigma_out, cudaStream_t st);
rbf_status mlp_forward_run(rbf_ctx* ctx, const float* params, const float* feat, int64_t n, float* y,
                           cudaStream_t st);
rbf_status warm_start_run(rbf_ctx* ctx, const float* params, double* c0, cudaStream_t st);
rbf_status mlp_targets_run(rbf_ctx* ctx, const double* c, float* target, cudaStream_t st);
rbf_status mlp_step_run(rbf_ctx* ctx, float* params, float* m, float* v, int step, double lr,
                        const float* feat, const float* target, const int* idx, int64_t n,
                        float* grad, double* loss, cudaStream_t st);

// rbf_assemble.cu (with_poly: also A^T P, P^T P and P^T h of Eq. 10)
rbf_status assemble_run(rbf_ctx* ctx, int kernel, int prec, cudaStream_t st, bool with_poly = false);

// r = A^T (h - A c) in FP64 (c in sorted order), from the stored A or matrix-free. With
// count_support the support counts are recomputed. With the polynomial of the last assembly,
// poly = true also subtracts P k (k = PolyDev::k64) and writes P^T (h - A c - P k) to
// PolyDev::rk.
rbf_status residual_run(rbf_ctx* ctx, const double* c_sorted, double* r_sorted,
                        bool count_support, cudaStream_t st, bool poly = false);
// the frame of the polynomial and the device pointers of PolyDev for the FP64 passes
PolyArgs poly_args(rbf_ctx* ctx);

// rbf_solve.cu
rbf_status solve_run(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                     int min_support, rbf_solve_info* info, cudaStream_t st);
// the bordered system of Eq. 10 (after an assembly with the polynomial); k: DEVICE, 3 doubles
// (a_x, a_y, a_0) in the caller's coordinates
rbf_status solve_poly_run(rbf_ctx* ctx, double* c, double* k, double tol, int maxit,
                          int min_support, rbf_solve_info* info, cudaStream_t st);

// rbf_eval.cu
rbf_status eval_points_run(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                           int64_t Q, double* f, cudaStream_t st);
rbf_status eval_grid_run(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                         double* f, cudaStream_t st, const double* k = nullptr);
rbf_status eval_points_poly_run(rbf_ctx* ctx, const double* c, const double* k, const double* qx,
                                const double* qy, int64_t Q, double* f, cudaStream_t st);
rbf_status diag_sqrt_run(const double* a, double* out, int64_t n, cudaStream_t st);
rbf_status layout_stats_run(rbf_ctx* ctx, rbf_layout_stats* out, cudaStream_t st);
rbf_status export_upper_run(rbf_ctx* ctx, int64_t cap, int32_t* row, int32_t* col, double* val,
                            double* bvec, int32_t* support, int64_t* nnz, cudaStream_t st);

// preconditioner set-up of the assembled B (precision prec): dinv / dinv32 and the inverse
// diagonal cell blocks; pinned centres counted into *npin_d
rbf_status prec_setup_run(rbf_ctx* ctx, int prec, int min_support, int* npin_d, cudaStream_t st);
// y += B x over all cells (precision prec; x, y sorted order)
void launch_spmv(rbf_ctx* ctx, int prec, const void* x, void* y, cudaStream_t st);
// r64 = b - B32 x64 on unpinned rows (FP32 assembly; uses the FP32 CG workspace's u and w[0])
void launch_resid32(rbf_ctx* ctx, const double* x64, double* r64, cudaStream_t st);

rbf_status bench_spmv_run(rbf_ctx* ctx, int reps, cudaStream_t st);
rbf_status bench_cg_run(rbf_ctx* ctx, int reps, cudaStream_t st);
rbf_status bench_cg_loop_run(rbf_ctx* ctx, int reps, cudaStream_t st);
rbf_status bench_fma_run(rbf_ctx* ctx, int prec, long long reps, double* flops, cudaStream_t st);
rbf_status bench_residual_run(rbf_ctx* ctx, int reps, cudaStream_t st);

// permutation helpers (rbf_solve.cu)
void launch_gather_sorted(const double* c_orig, const int* cperm, double* c_sorted, int M,
                          cudaStream_t st);
void launch_scatter_orig(const double* c_sorted, const int* cperm, double* c_orig, int M,
                         cudaStream_t st);

inline int div_up(int64_t a, int64_t b) { return int((a + b - 1) / b); }

}  // namespace rbf
