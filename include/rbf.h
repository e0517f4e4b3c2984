/*
 * librbf -- compactly supported RBF least-squares surface approximation of
 * scattered 2.5-D data on one GB300 (sm_103a).
 *
 * Method (Majdisova & Skala, "Big Geo Data Surface Approximation using Radial
 * Basis Functions: A Comparative Study"):
 *   f(x) = sum_{j=1..M} c_j phi(||x - xi_j|| / R)                    (Eq. 3)
 *   A_ij = phi(||x_i - xi_j|| / R),  N x M, N >> M,  A c ~= h       (Eq. 4-5)
 *   c solves the normal equations  B c = b,  B = A^T A,  b = A^T h   (Section 2, Eq. 11-12)
 *   phi is a Wendland function of Table 2 (cut-off of Eq. 18), R = 1/alpha.
 *
 * Pipeline and entry points:
 *   rbf_bin        bin centres and points into a uniform grid of cell size R
 *                  (replaces the kd-tree range query of Algorithm 1)
 *   rbf_assemble   evaluate each point's sparse row of A and accumulate the
 *                  upper triangle of B and b in one fused pass (Eq. 11-13);
 *                  A is never stored
 *   rbf_solve      Jacobi-preconditioned CG on B c = b (FP64), or FP32 CG inside
 *                  FP64 iterative refinement with a matrix-free FP64 residual
 *   rbf_eval       f at arbitrary query points (Eq. 3); rbf_eval_grid on a grid
 *   rbf_bin_tiles, rbf_solve_tiles
 *                  many independent tiles of uneven size binned, assembled (rbf_assemble)
 *                  and solved together, each kernel launched once for the whole batch
 *   rbf_bin_windows, rbf_eval_windows
 *                  the moving window (Section 7): overlapping windows of one domain fitted
 *                  as a batch of tiles and blended by a partition of unity
 *
 * Conventions (all entry points):
 *   - Array arguments are DEVICE pointers owned by the caller unless stated
 *     otherwise; they must stay valid until the work on `stream` completes.
 *     `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Calls are asynchronous on `stream` except where a result must come back
 *     to the host (rbf_bin, rbf_solve): those synchronise `stream` before return.
 *   - Errors are returned as rbf_status; no exception crosses this boundary.
 *     rbf_last_error(ctx) gives a message for the last failure on that context.
 *   - Device-side failures (CG breakdown, non-convergence) are reported through the status
 *     of rbf_solve / rbf_solve_tiles; no kernel traps, and no kernel spins on a flag set by
 *     another block, so none can hang.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef RBF_H_
#define RBF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBF_OK = 0,
    RBF_ERR_ARG = 1,            /* invalid argument (size, pointer, NaN, order of calls) */
    RBF_ERR_ALLOC = 2,          /* workspace allocation failed */
    RBF_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    RBF_ERR_NOT_CONVERGED = 4,  /* solver hit maxit before reaching tol */
    RBF_ERR_BREAKDOWN = 5,      /* CG breakdown: p^T B p <= 0 or a non-finite scalar */
    RBF_ERR_LIMIT = 6,          /* input exceeds a documented kernel limit */
    RBF_ERR_TIMEOUT = 7         /* a grid barrier of the persistent CG solve (rbf_solve)
                                   waited longer than 2 s; the context stays usable */
} rbf_status;

/* Wendland functions phi_{3,s}(r), r = ||x - xi|| / R, zero for r >= 1 (Table 2, Eq. 18).
 * RBF_W32 is not in Table 2: it is (1-r)^6 (35 r^2 + 18 r + 3) / 3, scaled so phi(0) = 1. */
typedef enum { RBF_W30 = 0, RBF_W31 = 1, RBF_W32 = 2, RBF_W33 = 3 } rbf_kernel;

/* Arithmetic of the assembled matrix and of the CG iterations. */
typedef enum {
    RBF_FP64 = 0,          /* B, b and CG in FP64 */
    RBF_FP32_REFINE = 1    /* B and inner CG in FP32 (FP32 accumulation); FP64 matrix-free
                              residual A^T (h - A c) and FP64 correction updates of c */
} rbf_prec;

typedef struct rbf_ctx rbf_ctx;

/* Workspace allocator. alloc returns a device pointer of at least `bytes` bytes usable on
 * `stream` (NULL on failure); free releases it. user is passed through. When both are NULL
 * the library uses cudaMalloc / cudaFree. */
typedef void* (*rbf_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*rbf_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Result of rbf_solve. */
typedef struct {
    int iterations;          /* total CG iterations (inner iterations for RBF_FP32_REFINE) */
    int refinements;         /* outer FP64 refinement steps (0 for RBF_FP64) */
    double rel_residual;     /* ||b - B c||_2 / ||b||_2 at exit, over unpinned centres.
                                For RBF_FP32_REFINE this is the FP64 matrix-free
                                ||A^T(h - A c)||_2 / ||A^T h||_2 */
    int64_t pinned;          /* centres with fewer than min_support points in support */
    int promoted;            /* 1 if RBF_FP32_REFINE stopped making progress (the FP32 matrix
                                cannot resolve a system this ill-conditioned) and the solve was
                                finished by an FP64 assembly and FP64 CG started from the
                                refined iterate; the context's assembly is FP64 afterwards */
} rbf_solve_info;

/* One tile of a batch (rbf_bin_tiles): an independent fitting problem of the same kind as
 * rbf_bin's, whose centres and points are ranges of concatenated arrays. */
typedef struct {
    int64_t c0, M;           /* centres c0 .. c0+M-1 of the concatenated centre arrays, M >= 1 */
    int64_t p0, N;           /* points p0 .. p0+N-1 of the concatenated point arrays, N >= 0 */
    double R;                /* support radius of this tile, > 0 */
    double bbox[4];          /* {x0, y0, x1, y1} of this tile (items outside are clamped) */
} rbf_tile;

/* Per-tile result of rbf_solve_tiles. */
typedef struct {
    int iterations;          /* CG iterations of this tile (summed over refinement steps) */
    int refinements;         /* FP64 refinement steps this tile took part in */
    double rel_residual;     /* as rbf_solve_info.rel_residual, over this tile's centres */
    int64_t pinned;          /* centres of this tile with fewer than min_support points */
    int status;              /* rbf_status of this tile: RBF_OK, RBF_ERR_NOT_CONVERGED or
                                RBF_ERR_BREAKDOWN */
    int promoted;            /* 1 if this tile was finished by FP64 CG after its FP32
                                refinement stalled or ran out of steps; tiles that converged
                                in FP32 keep their refined iterate */
} rbf_tile_info;

/* Create / destroy a context bound to CUDA device `device`. alloc / free_fn (both or
 * neither; NULL: cudaMalloc / cudaFree) supply the workspace: device memory of at least
 * `bytes`, aligned to 256 bytes (as cudaMalloc's), usable on `stream`; a NULL or misaligned
 * result makes the call that needed it return RBF_ERR_ALLOC. */
rbf_status rbf_create(rbf_ctx** out, int device, rbf_alloc_fn alloc, rbf_free_fn free_fn,
                      void* user);
rbf_status rbf_destroy(rbf_ctx* ctx);
const char* rbf_last_error(const rbf_ctx* ctx);

/* Step (a): bin M centres (cx, cy) and N points (px, py) with heights h into a uniform
 * grid of cell side R (plus a 2^-30 relative margin) over bbox = {x0, y0, x1, y1}
 * (HOST array of 4 doubles). Items outside bbox are clamped to the edge cells, which
 * stays correct. The context keeps cell-sorted copies of the inputs (within a cell, centres
 * ordered by x) and the permutation back to the caller's centre order, and lays out the
 * sparse B (Section 5: symmetric, only the upper triangle stored): row s keeps the columns
 * t >= s of the centres within 2R of xi_s (a slightly wider superset), as three contiguous
 * ranges of the sorted order, one per cell row. Requires M >= 1, N >= 1, R > 0, finite
 * coordinates and heights. Synchronises `stream`.
 * Returns RBF_ERR_LIMIT if some 3x3 cell neighbourhood holds more than
 * rbf_max_candidates() centres, a cell more than 16384 centres, one cell row more than 4092
 * centres within 2R of a centre, or the stored B more than 2^34 values. */
rbf_status rbf_bin(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M,
                   const double* px, const double* py, const double* h, int64_t N,
                   double R, const double* bbox, void* stream);

/* Largest number of centres in one 3x3 cell neighbourhood that rbf_bin accepts. */
int rbf_max_candidates(void);

/* Steps (b)+(c): one fused pass over the binned points computes every nonzero
 * A_ij = phi(||x_i - xi_j|| / R) (Algorithm 1 semantics: a pair counts iff
 * ||x_i - xi_j|| < R) and accumulates B = A^T A (upper triangle, Eq. 11-13) and b = A^T h
 * (Section 2) in the precision `prec`; also counts the data points inside each support.
 * Asynchronous. Requires a preceding rbf_bin. */
rbf_status rbf_assemble(rbf_ctx* ctx, rbf_kernel kernel, rbf_prec prec, void* stream);

/* Step (d): solve B c = b (Section 2) by Jacobi-preconditioned CG.
 * c       : device array of M doubles in the caller's centre order; on entry the
 *           starting guess if use_c0 != 0 (else ignored), on exit the weights.
 * tol     : stop when the relative residual (see rbf_solve_info) <= tol.
 * maxit   : iteration limit (for RBF_FP32_REFINE: per inner solve; at most 30 outer steps).
 * min_support: centres whose support disc holds fewer data points are removed from
 *           the system and get c_j = 0 (the paper leaves empty supports undefined).
 * info    : HOST pointer, may be NULL.
 * Each CG solve runs as one cooperative launch of a persistent kernel (SpMV and vector update
 * of every iteration separated by grid barriers) or as one launch of a CUDA graph looping over
 * the two kernels of an iteration ("cg_persistent"; the graph also where the device cannot
 * hold the persistent grid at once). Both give the same iterates up to the order of FP
 * additions.
 * Synchronises `stream`. Returns RBF_ERR_NOT_CONVERGED / RBF_ERR_BREAKDOWN with c
 * holding the last iterate, RBF_ERR_TIMEOUT if a barrier wait of the persistent kernel ran
 * out. With RBF_FP32_REFINE, a refinement step that no longer reduces
 * the FP64 residual promotes the solve to FP64 (see rbf_solve_info.promoted). */
rbf_status rbf_solve(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                     int min_support, rbf_solve_info* info, void* stream);

/* Step (e): f(q) = sum_j c_j phi(||q - xi_j|| / R) (Eq. 3) at Q query points.
 * c: device, M doubles in the caller's centre order; qx, qy: device, Q doubles;
 * f: device, Q doubles (output). Uses the centres binned by the last rbf_bin and
 * the kernel of the last rbf_assemble. Asynchronous. */
rbf_status rbf_eval(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                    int64_t Q, double* f, void* stream);

/* Step (e) on the node-centred nx x ny grid over box = {x0, y0, x1, y1} (HOST array):
 * node (i, j) = (x0 + j (x1-x0)/(nx-1), y0 + i (y1-y0)/(ny-1)); f is a device array of
 * nx*ny doubles, row-major f[i*nx + j]. Asynchronous. */
rbf_status rbf_eval_grid(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                         double* f, void* stream);

/* ---- linear polynomial reproduction (Section 3, Eq. 6-10) ----
 * The approximant gains a linear polynomial, f(x) = sum_j c_j phi(||x - xi_j|| / R)
 * + a_x x + a_y y + a_0 (Eq. 6-7), and (c, a_x, a_y, a_0) minimise ||A c + P k - h||_2, row i
 * of P being (x_i, y_i, 1) (Eq. 8-9): the bordered normal system of Eq. 10,
 *     [A^T A  A^T P] [c]   [A^T h]
 *     [P^T A  P^T P] [k] = [P^T h],
 * solved as one SPD system (least squares: no orthogonality constraint rows). Centres with
 * fewer than min_support points in their support leave the system (c_j = 0) as in rbf_solve;
 * the three polynomial unknowns always stay. Single systems only (a batched context returns
 * RBF_ERR_ARG). */

/* As rbf_assemble, and also A^T P (M x 3), P^T P and P^T h in FP64 (the polynomial handled in
 * the bounding box's centred, scaled frame, which spans the same functions). Asynchronous. */
rbf_status rbf_assemble_poly(rbf_ctx* ctx, rbf_kernel kernel, rbf_prec prec, void* stream);

/* Solve Eq. 10 after rbf_assemble_poly: iterative refinement from c = 0, k = 0 whose every
 * step takes the FP64 residual (A^T e, P^T e), e = h - A c - P k, from the points, and solves
 * the correction by CG on the bordered matrix in the assembly's precision (FP32 B and
 * A^T P with FP32 inner tolerance "inner_tol", or FP64), preconditioned by the cells' inverse
 * diagonal blocks and (P^T P)^-1. A stalled FP32 refinement is finished with an FP64 assembly
 * (info->promoted). c: DEVICE, M doubles in the caller's centre order (output); k: DEVICE, 3
 * doubles (a_x, a_y, a_0) in the caller's coordinates (output). tol: on
 * ||(A^T e, P^T e)||_2 / ||(A^T h, P^T h)||_2 (info->rel_residual). maxit: per inner solve.
 * Synchronises `stream`. Returns RBF_ERR_ARG if P^T P is singular (collinear points),
 * RBF_ERR_NOT_CONVERGED / RBF_ERR_BREAKDOWN with c, k holding the last iterate. */
rbf_status rbf_solve_poly(rbf_ctx* ctx, double* c, double* k, double tol, int maxit,
                          int min_support, rbf_solve_info* info, void* stream);

/* f(q) = sum_j c_j phi(||q - xi_j|| / R) + a_x q_x + a_y q_y + a_0 (Eq. 6-7) at Q query
 * points (as rbf_eval); k: DEVICE, 3 doubles. Asynchronous. */
rbf_status rbf_eval_poly(rbf_ctx* ctx, const double* c, const double* k, const double* qx,
                         const double* qy, int64_t Q, double* f, void* stream);

/* The same on the node-centred nx x ny grid over box (as rbf_eval_grid). Asynchronous. */
rbf_status rbf_eval_grid_poly(rbf_ctx* ctx, const double* c, const double* k, int nx, int ny,
                              const double* box, double* f, void* stream);

/* Solver parameters (HOST call, takes effect at the next rbf_solve):
 *   "inner_tol"        relative tolerance of each FP32 inner solve of RBF_FP32_REFINE, in
 *                      (0, 1); default 1e-3
 *   "max_refinements"  FP64 refinement steps of RBF_FP32_REFINE, in [0, 1000]; default 30
 *   "store_a"          1 (default): the FP32 assembly keeps the FP64 values of A (points x
 *                      candidate centres of each cell's 3x3 block, ~8 x N x 9 x centres per cell
 *                      bytes) so that the refinement's residual passes read them instead of
 *                      recomputing them; 0 (or no room for them): matrix-free residual
 *   "autotune"         1 (default): rbf_solve_tiles times the candidate launch
 *                      configurations of its CG loop on the first solve of a system of a
 *                      new shape and keeps the fastest (see rbf_autotune); 0: it uses the
 *                      forced values below, else a fixed default
 *   "spmv_blocks_per_sm", "spmv_chunk", "update_threads"
 *                      force the batched CG's SpMV blocks per SM (1..8), row groups per
 *                      SpMV work item (1..64) and update block size (128, 256 or 512); 0 =
 *                      automatic
 *   "cg_persistent"    how rbf_solve runs its CG loop: 1 as one cooperative launch of the
 *                      persistent kernel, 0 as the CUDA graph of two kernels per iteration,
 *                      -1 (default) the persistent kernel for FP64 and for FP32 systems of at
 *                      most 4 x (SMs) x 768 centres, else the graph (the faster of the two on
 *                      GB300 at each size)
 *   "cg_barrier_test"  test hook, 0 (default) or 1: the persistent kernel's barriers wait for
 *                      one block more than its grid has, so the first wait runs out (2 s) and
 *                      rbf_solve returns RBF_ERR_TIMEOUT
 *   "b_device_mb"      0 (default): B lives in device memory. > 0 (single systems; takes effect
 *                      at the next rbf_assemble / rbf_assemble_poly): B too large for the
 *                      device -- the block-wise assembly of Section 5 (Eq. 13-16). The stored
 *                      values of B live in pinned, device-mapped host memory (read by the
 *                      solver over the host link) and are assembled on the device in blocks of
 *                      consecutive cell rows whose values fit this many MB (at least one cell
 *                      row per block), each block copied out when done. The values are those
 *                      of the in-device assembly up to the order of the FP additions. The
 *                      host buffer is freed by rbf_destroy or the next in-device assembly.
 *                      Pinned host memory that cannot be had returns RBF_ERR_ALLOC.
 * Returns RBF_ERR_ARG for an unknown name or a value out of range. */
rbf_status rbf_set_param(rbf_ctx* ctx, const char* name, double value);

/* Diagnostics: number of stored B values (the upper rows the SpMV streams) and bytes per
 * value of the last assembly; sizes of the cell grid. HOST outputs, any may be NULL. */
rbf_status rbf_get_layout(const rbf_ctx* ctx, int64_t* nvals, int* value_bytes, int* gx,
                          int* gy);

/* Diagnostics of the stored B after an assembly. */
typedef struct {
    int64_t stored_values;   /* values the SpMV streams (as rbf_get_layout's nvals) */
    int64_t nonzeros;        /* stored values that are not exactly zero: the nonzeros of the
                                upper triangle of B, diagonal included (Eq. 11-12) */
    int64_t row_groups;      /* row groups (up to 8 consecutive rows) the SpMV sweeps */
    int64_t dropped;         /* Gram entries of the last assembly that found no slot in their
                                row: 0 by construction (any other value is a library defect) */
    int64_t host_blocks;     /* 0: B in device memory; else the blocks of cell rows of the
                                last out-of-core assembly (B in host memory, "b_device_mb") */
} rbf_layout_stats;

/* Fill *out (HOST) for the last assembly; counts the nonzeros on the GPU. Requires a
 * preceding rbf_assemble. Synchronises `stream`. */
rbf_status rbf_get_layout_stats(rbf_ctx* ctx, rbf_layout_stats* out, void* stream);

/* Diagnostics: copy the assembled B as COO triplets (upper triangle incl. diagonal,
 * caller's centre indices) into DEVICE arrays of capacity cap; *nnz gets the count.
 * Entries that are exactly zero are skipped. Synchronises `stream`. */
rbf_status rbf_export_upper(rbf_ctx* ctx, int64_t cap, int32_t* row, int32_t* col,
                            double* val, double* bvec, int32_t* support, int64_t* nnz,
                            void* stream);

/* Diagnostics: number of kernels this context has launched since rbf_create (kernels
 * inside replayed CUDA graphs included). HOST output. */
rbf_status rbf_get_launch_count(const rbf_ctx* ctx, int64_t* launches);

/* Diagnostics / timing: launch the solver's SpMV kernel y += B x (Section 4's y = Q x on
 * this library's cell-blocked symmetric storage) `reps` times on `stream` with x = 1, in the
 * launch configuration a CG iteration uses, on the solver's workspace (which it allocates if
 * needed and overwrites). Requires a preceding rbf_assemble. On a batched context (after
 * rbf_solve_tiles) it launches the batched SpMV with every tile running. Asynchronous. */
rbf_status rbf_bench_spmv(rbf_ctx* ctx, int reps, void* stream);

/* Diagnostics / timing: run `reps` preconditioned CG iterations on B c = b from c = 0 with
 * every iteration's two kernels launched individually on `stream` (the solver normally loops
 * inside one CUDA graph), so that the kernels can be timed or profiled one by one. Uses and
 * overwrites the solver's workspace; requires a preceding rbf_solve (rbf_solve_tiles on a
 * batched context, where the iterations are batched ones with every tile running).
 * Asynchronous. */
rbf_status rbf_bench_cg(rbf_ctx* ctx, int reps, void* stream);

/* Diagnostics / timing: run `reps` (>= 1) preconditioned CG iterations on B c = b from c = 0
 * (tolerance 0) in the solver's own loop -- the persistent kernel or the graph, as rbf_solve
 * chooses ("cg_persistent") -- so that time / reps is the loop's cost per iteration. Uses and
 * overwrites the solver's workspace; requires a preceding rbf_solve on a single system.
 * Synchronises `stream`. */
rbf_status rbf_bench_cg_loop(rbf_ctx* ctx, int reps, void* stream);

/* Diagnostics / timing: the device's FMA throughput in precision `prec` (RBF_FP64: FP64;
 * RBF_FP32_REFINE: FP32): one kernel in which every thread of 8 blocks per SM runs 8
 * independent FMA chains of `reps` (1 .. 2^32) steps; *flops (HOST) gets the floating-point
 * operations it performs (2 per FMA). Time it with events on `stream`. Asynchronous. */
rbf_status rbf_bench_fma(rbf_ctx* ctx, int prec, int64_t reps, double* flops, void* stream);

/* Diagnostics / timing: `reps` FP64 residual passes r = A^T (h - A x) of the FP32 refinement
 * at the current iterate (reading the stored A when the FP32 assembly kept it), as every
 * refinement step runs them. Requires a preceding rbf_solve on a single system without the
 * polynomial. Asynchronous. */
rbf_status rbf_bench_residual(rbf_ctx* ctx, int reps, void* stream);

/* Batched step (a): bin T independent tiles (HOST array `tiles`) into one packed system.
 * cx, cy: DEVICE arrays of Mtot centre coordinates; px, py, h: DEVICE arrays of Ntot point
 * coordinates and heights; tile t owns centres [c0, c0+M) and points [p0, p0+N). The centre
 * ranges of all tiles must partition [0, Mtot) and the point ranges of the tiles with N > 0
 * must partition [0, Ntot) (any order of tiles). Each tile is fitted exactly as rbf_bin +
 * rbf_assemble + rbf_solve would fit it alone: A_ij = phi(||x_i - xi_j|| / R_t) over the
 * tile's own points and centres only. Internally each tile is moved to its own frame
 * (x - x0_t) / R_t, where its support radius is 1, and gets its own band of cell rows of one
 * shared grid, two empty rows apart, so the packed B is block diagonal by tile.
 * Follow with rbf_assemble (one launch for all tiles) and rbf_solve_tiles; rbf_solve,
 * rbf_eval and rbf_eval_grid reject a batched context. Synchronises `stream`.
 * Returns RBF_ERR_ARG for overlapping or non-covering ranges, RBF_ERR_LIMIT if the packed
 * grid exceeds 2^24 cells or a 3x3 neighbourhood more than rbf_max_candidates() centres. */
rbf_status rbf_bin_tiles(rbf_ctx* ctx, const rbf_tile* tiles, int T, const double* cx,
                         const double* cy, int64_t Mtot, const double* px, const double* py,
                         const double* h, int64_t Ntot, void* stream);

/* Batched step (d): solve every tile's normal equations B_t c_t = b_t with its own CG
 * (own step lengths, own stopping test, own iteration count), all tiles advancing together
 * in one CUDA graph whose kernels each cover every tile still running. c: DEVICE array of
 * Mtot doubles in the caller's concatenated centre order (start guess if use_c0). tol,
 * maxit, min_support as for rbf_solve, applied per tile. tile_info: HOST array of T entries
 * (may be NULL); info: HOST totals (may be NULL): iterations = largest per-tile count,
 * refinements = most refinement steps, rel_residual = largest per-tile value, pinned = sum,
 * promoted = 1 if any tile was finished in FP64 (later solves on this context then run in
 * FP64, as for rbf_solve). Synchronises `stream`. Returns
 * RBF_OK when every tile converged, else RBF_ERR_BREAKDOWN if some tile broke down, else
 * RBF_ERR_NOT_CONVERGED; c holds every tile's last iterate in all cases. */
rbf_status rbf_solve_tiles(rbf_ctx* ctx, double* c, int use_c0, double tol, int maxit,
                           int min_support, rbf_tile_info* tile_info, rbf_solve_info* info,
                           void* stream);

/* Batched step (e): f(q) = sum_j c_j phi(||q - xi_j|| / R_t) over the centres of tile t for
 * queries grouped by tile: tile t's queries are qx, qy [qoff[t], qoff[t+1]) (DEVICE arrays;
 * qoff a HOST array of T+1 non-decreasing offsets with qoff[0] = 0), values into f at the
 * same positions (DEVICE). c: DEVICE, Mtot doubles in the caller's concatenated order.
 * Requires rbf_bin_tiles + rbf_assemble. Synchronises `stream`. */
rbf_status rbf_eval_tiles(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                          const int64_t* qoff, double* f, void* stream);

/* Batched step (e) on each tile's own node-centred nx x ny grid over the tile's bbox (as
 * rbf_eval_grid): tile t's node (i, j) at f[t*nx*ny + i*nx + j] (DEVICE, T*nx*ny doubles).
 * Asynchronous. */
rbf_status rbf_eval_tiles_grid(rbf_ctx* ctx, const double* c, int nx, int ny, double* f,
                               void* stream);

/* ---- Moving window (the "moving window" the paper names as future work, Section 7) ----
 * A large domain is cut into wx x wy overlapping windows fitted independently -- each window
 * is one tile of the batched fit -- and the surface blends the windows' local surfaces with a
 * partition of unity. Window (i, j) (row-major, j slow; tile j wx + i):
 *   core box        [a_i, a_{i+1}] x [b_j, b_{j+1}], a_i = x0 + (x1 - x0) i / wx, likewise b_j
 *   extended box    the core box grown by `overlap` on its inner sides, closed; a side on the
 *                   domain's boundary is open to infinity (items outside bbox belong to the
 *                   edge windows)
 *   data box        the extended box grown by `margin` on its inner sides
 *   points, centres those in the data box (an item can belong to several windows); a centre
 *                   at the data box's edge keeps about half of its support's points, so with
 *                   margin >= R a window's system is about as well conditioned as the whole
 *                   domain's, and the window's surface inside its extended box has every
 *                   centre within R
 *   weight          the product over the inner sides of s((q - (a_i - overlap)) / (2 overlap))
 *                   and s(((a_{i+1} + overlap) - q) / (2 overlap)), s(t) = t^2 (3 - 2t) on
 *                   [0, 1] (0 below, 1 above): neighbours' weights sum to one across their
 *                   common band; with overlap 0, steps (q >= a_i, q < a_{i+1})
 *   surface         f(q) = sum_w weight_w(q) f_w(q) / sum_w weight_w(q) over the windows whose
 *                   extended box holds q, f_w the window's own fit (Eq. 3 on its centres)
 * Use: rbf_bin_windows, then rbf_assemble and rbf_solve_tiles (c: DEVICE, the Mtot weights of
 * rbf_window_sizes, window after window; rbf_window_centres maps them to input centres), then
 * rbf_eval_windows / rbf_eval_windows_grid. The windows' centre and point order within a window
 * comes from atomics: results agree from run to run up to the order of FP additions. */

/* Lay the windows out over bbox = {x0, y0, x1, y1} (HOST; x1 > x0, y1 > y0) and bin them as
 * a batch: cx, cy (M centres), px, py, h (N points) DEVICE arrays in the caller's order; R > 0
 * the support radius of every window; 1 <= wx, wy, wx wy <= 65536; overlap >= 0; margin >= 0
 * (R is the usual choice). Synchronises `stream`. Returns RBF_ERR_ARG for a window without centres (fewer windows or a
 * larger overlap), RBF_ERR_LIMIT as rbf_bin_tiles. */
rbf_status rbf_bin_windows(rbf_ctx* ctx, const double* cx, const double* cy, int64_t M,
                           const double* px, const double* py, const double* h, int64_t N,
                           double R, const double* bbox, int wx, int wy, double overlap,
                           double margin, void* stream);

/* Centres (Mtot) and points (Ntot) summed over the windows of the last rbf_bin_windows (HOST
 * outputs): the length of rbf_solve_tiles' c. */
rbf_status rbf_window_sizes(const rbf_ctx* ctx, int64_t* Mtot, int64_t* Ntot);

/* idx[k] (DEVICE, capacity cap >= Mtot) = the input index of the centre behind weight k.
 * Asynchronous. */
rbf_status rbf_window_centres(rbf_ctx* ctx, int64_t* idx, int64_t cap, void* stream);

/* The blended surface at Q query points (qx, qy, f DEVICE) from the windows' weights c (DEVICE,
 * Mtot values as rbf_solve_tiles returns them). Asynchronous. */
rbf_status rbf_eval_windows(rbf_ctx* ctx, const double* c, const double* qx, const double* qy,
                            int64_t Q, double* f, void* stream);

/* The same on the node-centred nx x ny grid over box (HOST {x0, y0, x1, y1}); f[i nx + j]
 * (DEVICE, nx ny values). Each window's node range is computed on the host and copied from
 * pageable memory, which waits for the work already queued on `stream`; the evaluation itself
 * is queued asynchronously. The windows' values are summed into f with atomics, so repeated
 * calls agree up to the order of FP additions. */
rbf_status rbf_eval_windows_grid(rbf_ctx* ctx, const double* c, int nx, int ny, const double* box,
                                 double* f, void* stream);

/* Autotuner of the batched CG loop: on the assembled batched system, times CG iterations in
 * each candidate launch configuration (SpMV blocks per SM x row groups per work item, then the
 * update block size) with CUDA events on `stream` and keeps the fastest for systems of this
 * shape. Overwrites the solver workspace. Synchronises `stream`. */
rbf_status rbf_autotune(rbf_ctx* ctx, void* stream);

/* The launch configuration of the batched CG loop for the precision of the last assembly
 * (HOST outputs, any may be NULL): SpMV blocks per SM, row groups per SpMV work item, update block
 * size, and the measured time of one iteration in microseconds (0 if not tuned). */
rbf_status rbf_get_tuning(const rbf_ctx* ctx, int* spmv_blocks_per_sm, int* spmv_chunk,
                          int* update_threads, double* us_per_iteration);

/* ---- learned warm start (not in the paper: a start vector for the solver) ----
 * A 32-64-64-1 network predicts c_j from 32 radial features of the data around centre j;
 * rbf_solve / rbf_solve_tiles started from that guess (use_c0 = 1) reach the same solution,
 * in fewer iterations when the guess is good. Parameters: a flat FP32 DEVICE vector of
 * RBF_MLP_NPARAM values: W1 (row-major 64 x 32), b1 (64), W2 (row-major 64 x 64), b2 (64),
 * W3 (64), b3 (1); the weights (not the biases) are rounded to BF16 where they enter a
 * product, every product is accumulated in FP32. */
#define RBF_MLP_NFEAT 32
#define RBF_MLP_NPARAM 6337

/* Features of every binned centre (after rbf_bin or rbf_bin_tiles): row j of feat (DEVICE,
 * M x 32 floats, caller's centre order, 16-byte aligned) holds, for the 16 annuli
 * k/16 <= ||x_i - xi_j|| / R < (k+1)/16 of the support, the fraction of the support's
 * points in annulus k (0..15) and their mean height divided by sigma (16..31; 0 when
 * empty), sigma = sqrt(mean h^2) over the system's (the tile's) points. The annulus of a
 * point is that of an FP64 evaluation of sqrt(dx*dx + dy*dy) / R. sigma: DEVICE array of T
 * (batched) or 1 doubles, may be NULL. Asynchronous. */
rbf_status rbf_features(rbf_ctx* ctx, float* feat, double* sigma, void* stream);

/* y[i] = network(feat row i) for i < n (DEVICE arrays; feat 16-byte aligned). The context
 * supplies the device and the launch accounting only. Asynchronous. */
rbf_status rbf_mlp_forward(rbf_ctx* ctx, const float* params, const float* feat, int64_t n,
                           float* y, void* stream);

/* One training step on the minibatch of n samples: sample i is feature row idx[i] (or i when
 * idx is NULL) of feat with target target[idx[i]] (DEVICE arrays). Computes the loss
 * mean (y - t)^2 and its gradient by back-propagation (with respect to the BF16-rounded
 * weights as they enter the products, and the biases); with step >= 1 also applies Adam
 * step number `step` (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) to params, m and v
 * (DEVICE, RBF_MLP_NPARAM floats each; m = v = 0 before step 1); with step = 0 nothing is
 * updated. grad (DEVICE, RBF_MLP_NPARAM floats) and loss (DEVICE, 1 double) receive the
 * gradient and the loss when not NULL. The gradient is summed in a fixed order
 * (deterministic). Asynchronous. */
rbf_status rbf_mlp_train_step(rbf_ctx* ctx, float* params, float* m, float* v, int step,
                              double lr, const float* feat, const float* target,
                              const int32_t* idx, int64_t n, float* grad, double* loss,
                              void* stream);

/* The warm start c0 (DEVICE, M doubles, caller's order) of the binned system:
 * c0_j = sigma * network(features of centre j), sigma per tile for a batch. Asynchronous. */
rbf_status rbf_warm_start(rbf_ctx* ctx, const float* params, double* c0, void* stream);

/* Training targets of the network for the binned system and weights c (DEVICE, M doubles,
 * caller's order): target[j] = c_j / sigma, sigma as for rbf_features (per tile for a batch);
 * target: DEVICE, M floats, caller's order. The inverse of rbf_warm_start's scaling.
 * Asynchronous. */
rbf_status rbf_mlp_targets(rbf_ctx* ctx, const double* c, float* target, void* stream);

/* Evaluation with no allocation at all (the paper has no counterpart; this is a service to
 * callers that cannot allocate device memory where they need the surface -- e.g. code that
 * runs while its own memory pool is locked or inside a fixed device-memory budget, or a
 * C/Fortran host that owns every device buffer and keeps no library context). Computes
 * f[q] = sum_j c[j] phi(||(qx[q], qy[q]) - (cx[j], cy[j])|| / R) for q < Q, the same value
 * as rbf_eval, from caller-owned DEVICE arrays cx, cy, c (M values each), qx, qy (Q values)
 * into the caller-owned DEVICE array f (Q values); bbox is a HOST array {x0, y0, x1, y1}.
 * The centres are binned into a scratch area that is a static device array of 2.6 MB
 * reserved when the library is loaded (each GPU that loads the library keeps it until the
 * process exits); nothing is allocated and no context is used.
 * Limits: M <= 65536 and at most 65536 cells of side R over bbox, else RBF_ERR_LIMIT (no
 * work queued). The scratch address belongs to the CUDA context current on the calling
 * thread: the first call in each context (the device's primary context unless the caller made
 * another one current; a context created after a device reset counts as new) looks it up, so
 * make that first call before any stream capture. Every call on a device shares the scratch:
 * calls whose GPU work overlaps (other streams or threads) race; calls ordered on one stream
 * are safe. The order in which a cell's centres are summed comes from atomic counters, so two
 * identical calls can differ in the last bits; the value agrees with rbf_eval to rounding.
 * Asynchronous on `stream`. */
rbf_status rbf_eval_noalloc(const double* cx, const double* cy, const double* c, int64_t M,
                            double R, const double* bbox, rbf_kernel kernel, const double* qx,
                            const double* qy, int64_t Q, double* f, void* stream);

/* Self-test of the device square roots used for distances, both seeded by the FP32 hardware
 * estimate of 1/sqrt: for each a[i] >= 0 (DEVICE, n values) writes out[3i] = the two-step
 * Newton-Raphson root (within a few units in the last place), out[3i+1] = the one-step root of
 * the evaluation and the FP64 assembly pass (relative error ~3e-14) and out[3i+2] = CUDA's
 * sqrt(a[i]) (DEVICE, 3n values). Asynchronous. */
rbf_status rbf_selftest_sqrt(const double* a, double* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RBF_H_ */
