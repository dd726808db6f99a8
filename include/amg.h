/*
 * amg.h - C ABI of libamg, the GPU (sm_103a) solve phase of the edge-matrix
 * ("auxiliary topology") algebraic multigrid method of Kogler & Schoeberl,
 * "An algebraic multigrid method based on an auxiliary topology with edge
 * matrices".
 *
 * The library solves A u = f (Sec. 2, eq. (auf)) by the conjugate gradient
 * method preconditioned with one V-cycle (Sec. 7): on every level a
 * block-l1 Jacobi smoother (Sec. 7, blocks = the dofs of one vertex), the
 * restriction P^T r and the prolongation P e (Sec. 3, Algorithm tg) with the
 * auxiliary smoothed prolongation of Sec. 6 (Def. aux_sp), Galerkin coarse
 * matrices A_{l+1} = P_l^T A_l P_l (Sec. 6), and the regularised coarsest
 * solve of Sec. 3 after Lemma eet_is_diag.
 *
 * Conventions that hold for every entry point:
 *  - Every call returns an int status (AMG_OK or a negative AMG_ERR_*); the
 *    message of the last failure is returned by amg_last_error(ctx).  No
 *    call aborts the process or throws across the ABI.
 *  - BSR matrices: n_rows x n_cols blocks of br x bc doubles, int32 rowptr
 *    (n_rows+1, rowptr[0] = 0, non-decreasing) and colidx (nnzb, strictly
 *    increasing within a row, 0 <= colidx < n_cols), values row-major per
 *    block.  Host arrays passed in are owned by the caller and copied.
 *  - Vectors are interleaved per vertex ("AoS": dof r of vertex i at
 *    i*k + r).  Pointers named *_dev are device pointers owned by the
 *    caller, on the device the context was created for; the library uses
 *    them on the context's stream and returns only after that stream is
 *    synchronised, unless stated otherwise.
 *  - All internal device buffers, CUDA graphs and streams belong to the
 *    context until amg_destroy.
 */
#ifndef AMG_H
#define AMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_ctx amg_ctx;

/* Block-sparse-row matrix (host arrays, caller-owned, copied on upload). */
typedef struct {
  int32_t n_rows, n_cols; /* block rows / block columns                     */
  int32_t br, bc;         /* block dimensions                               */
  int64_t nnzb;           /* number of stored blocks                        */
  const int32_t *rowptr;  /* n_rows + 1                                     */
  const int32_t *colidx;  /* nnzb, sorted ascending within each row         */
  const double *vals;     /* nnzb * br * bc, row-major blocks               */
} amg_bsr;

/* Same layout, filled by the library (caller allocates the arrays). */
typedef struct {
  int32_t n_rows, n_cols, br, bc;
  int64_t nnzb;
  int32_t *rowptr;
  int32_t *colidx;
  double *vals;
} amg_bsr_out;

/* A hierarchy given by the finest matrix and the prolongations.
 * P[l] maps level l+1 to level l (n_rows = rows of A_l, n_cols = rows of
 * A_{l+1}); A0.bc == P[0].br and P[l].bc == P[l+1].br.  The coarse matrices
 * are built on the device by the Galerkin product (Sec. 6). */
typedef struct {
  amg_bsr A0;
  int32_t n_levels;       /* number of levels, >= 1; P has n_levels-1 items */
  const amg_bsr *P;
} amg_hierarchy;

enum {
  AMG_OK = 0,
  AMG_ERR_ARG = -1,            /* invalid argument / malformed matrix        */
  AMG_ERR_CUDA = -2,           /* a CUDA runtime call failed                 */
  AMG_ERR_NOT_SPD = -3,        /* CG breakdown (p^T A p <= 0 or NaN)         */
  AMG_ERR_NO_CONVERGENCE = -4, /* maxit reached before rtol                  */
  AMG_ERR_TIMEOUT = -5,        /* reserved for a bounded device wait that
                                  ran out; no entry point has such a wait,
                                  so none returns it today                  */
  AMG_ERR_STATE = -6           /* call out of order (e.g. no hierarchy yet)  */
};

/* Precision of the V-cycle (the outer CG is always FP64). */
enum {
  AMG_PREC_FP64 = 0,          /* FP64 values, vectors and accumulation        */
  AMG_PREC_FP32_VCYCLE = 1,   /* V-cycle matrices, smoother blocks, vectors
                                 and accumulation in FP32; coarsest solve FP64 */
  AMG_PREC_BF16_STORAGE = 2,  /* as FP32 but A_l, P_l, R_l stored in BF16     */
  AMG_PREC_BF16_COARSE = 3    /* as FP32, with A_l, P_l, R_l of the levels
                                 l >= 1 stored in BF16 (level 0 in FP32): the
                                 coarse operators move half the bytes, while
                                 A_0, whose rounding to BF16 spoils the
                                 smoother on coefficient jumps, stays FP32.
                                 Not accepted by amg_batch_create.            */
};

/* Smoother of the V-cycle.
 *  AMG_SMOOTHER_L1_JACOBI  block-l1 Jacobi (Sec. 7) on every level.
 *  AMG_SMOOTHER_LEARNED    level 0 uses the blocks of amg_set_learned_smoother
 *                          (set by that call, not accepted by the uploads).
 *  AMG_SMOOTHER_HYBRID_GS  block-l1 hybrid Gauss-Seidel, the other form of the
 *                          l1 smoothers Sec. 7 cites, read for one device:
 *                          the block rows of every level are coloured at
 *                          upload (greedy in smallest-last order: rows
 *                          removed by least remaining degree, ties by the
 *                          smallest index, coloured in reverse, each the
 *                          smallest colour no already coloured neighbour
 *                          holds: a distance-1 colouring) and a sweep visits
 *                          the colour classes in order, every row of a class
 *                          x_v <- x_v + M_v^+ (b - A x)_v with the values of
 *                          the classes before (one launch per class; a level
 *                          0 with a SELL-32 copy also keeps one in colour
 *                          order and sweeps its large classes from it, one
 *                          thread per row); M_v = A_vv + diag of the
 *                          |entries| coupling v to rows of its own class
 *                          (none for a distance-1 colouring).
 *                          Forward sweep before the coarse correction,
 *                          backward sweep after it (the V-cycle stays
 *                          symmetric).  Not available to amg_batch_create,
 *                          amg_vcycle_static or amg_set_learned_smoother. */
enum {
  AMG_SMOOTHER_L1_JACOBI = 0,
  AMG_SMOOTHER_LEARNED = 1,
  AMG_SMOOTHER_HYBRID_GS = 2
};

/* Create a context (library plumbing, no counterpart in the paper) on CUDA
 * device `device`.  `cuda_stream` is a
 * cudaStream_t owned by the caller (not the legacy default stream: the CG is
 * captured into a CUDA graph), or NULL to let the library create a blocking
 * stream, ordered with the legacy default stream.
 * On success *ctx receives the context.  Errors: AMG_ERR_ARG (ctx NULL),
 * AMG_ERR_CUDA. */
int amg_create(amg_ctx **ctx, int device, void *cuda_stream);

/* Release every device buffer, graph and owned stream (plumbing).  NULL is
 * a no-op. */
void amg_destroy(amg_ctx *ctx);

/* Message of the last failed call on ctx ("" if none; plumbing). Valid until the next
 * call on ctx. */
const char *amg_last_error(const amg_ctx *ctx);

/* Upload a hierarchy and prepare the solve phase on the device:
 *   - validates every matrix (sizes, rowptr monotone, colidx sorted and in
 *     range, matching block dims between levels) -> AMG_ERR_ARG,
 *   - builds R_l = P_l^T explicitly (Sec. 3, restriction),
 *   - computes A_{l+1} = P_l^T A_l P_l on the device (Sec. 6, amg_galerkin),
 *   - computes the block-l1 smoother blocks M_v^+ (Sec. 7 and the pseudo
 *     smoother of Sec. 3 after Lemma eet_is_diag) in FP64 on the device,
 *   - factorises the regularised coarsest matrix A_L + (I - E_L E_L^T)
 *     (Sec. 3 after Lemma eet_is_diag) in FP64 on the device and stores
 *     its inverse,
 *   - for AMG_PREC_FP32_VCYCLE / AMG_PREC_BF16_STORAGE, keeps FP32 / BF16
 *     copies of the level operators (AMG_PREC_BF16_COARSE: FP32 copies of
 *     level 0's, BF16 copies of the coarser levels').
 * Replaces any previous hierarchy of ctx. */
int amg_upload_hierarchy(amg_ctx *ctx, const amg_hierarchy *h, int precision, int smoother);

/* Recompute A_{level+1} = P_level^T A_level P_level on the device (the
 * Galerkin triple product of Sec. 6, Sec. 3 eq. for the coarse system) as a
 * segmented SpGEMM: symbolic (sorted unique block columns per coarse row,
 * every structurally reached block kept) then numeric.  If out is not NULL
 * the result is copied to the caller's host arrays: out->rowptr must hold
 * n_rows+1 entries and colidx / vals at least nnzb / nnzb*k*k entries as
 * reported by amg_level_info(level+1).  0 <= level < n_levels-1. */
int amg_galerkin(amg_ctx *ctx, int level, amg_bsr_out *out);

/* Sizes of level `level` of the hierarchy (Sec. 3: A_l, P_l): block rows,
 * block size and stored blocks of A_l, and of P_l (0 on the coarsest level).
 * Any output pointer may be NULL. */
int amg_level_info(const amg_ctx *ctx, int level, int32_t *n_rows, int32_t *block,
                   int64_t *nnzb_A, int64_t *nnzb_P, int32_t *n_levels);

/* Copy A_level (the Galerkin operator of Sec. 3, as held on the device,
 * FP64) to caller host arrays sized as reported by amg_level_info. */
int amg_download_matrix(amg_ctx *ctx, int level, int32_t *rowptr, int32_t *colidx, double *vals);

/* Copy the smoother blocks M_v^+ of `level` (block-l1 Jacobi, Sec. 7;
 * n_rows * k * k doubles, row-major per block) to host memory `minv`. */
int amg_download_smoother(amg_ctx *ctx, int level, double *minv);

/* Copy the coarsest-level inverse (A_L + I - E_L E_L^T)^{-1} (Sec. 3 after
 * Lemma eet_is_diag; n x n doubles, n = n_rows * k of the coarsest level)
 * to host memory. */
int amg_download_coarse_inverse(amg_ctx *ctx, double *cinv);

/* --- single steps of the V-cycle, FP64, device vectors of level `level` ---
 * Errors of every single step: AMG_ERR_STATE without a hierarchy,
 * AMG_ERR_ARG for a level out of range (restriction / prolongation: the
 * coarsest level too) or a NULL required vector, AMG_ERR_CUDA. */

/* y = A_l x (BSR SpMV with the level operator of Algorithm tg). */
int amg_spmv(amg_ctx *ctx, int level, const double *x_dev, double *y_dev);
/* r = b - A_l x (the residual of Algorithm tg). */
int amg_residual(amg_ctx *ctx, int level, const double *b_dev, const double *x_dev, double *r_dev);
/* One block-l1 Jacobi sweep x_out = x_in + M^+ (b - A_l x_in) (Algorithm tg,
 * pre- and post-smoothing; M symmetric so M^{-T} = M^{-1}).  x_in == NULL
 * means x_in = 0, i.e. x_out = M^+ b.  x_out must not alias x_in. */
int amg_smooth(amg_ctx *ctx, int level, const double *b_dev, const double *x_in_dev, double *x_out_dev);
/* b_{l+1} = R_l r_l = P_l^T r_l (restriction, Algorithm tg). */
int amg_restrict(amg_ctx *ctx, int level, const double *r_dev, double *bc_dev);
/* x_l += P_l e_{l+1} (prolongation and correction, Algorithm tg). */
int amg_prolong_add(amg_ctx *ctx, int level, const double *ec_dev, double *x_dev);
/* x = (A_L + I - E_L E_L^T)^{-1} b on the coarsest level (Sec. 3 after Lemma eet_is_diag). */
int amg_coarse_solve(amg_ctx *ctx, const double *b_dev, double *x_dev);

/* z = B^{-1} r: one V-cycle (Algorithm tg applied recursively, one pre- and
 * one post-smoothing sweep, zero initial guess) on the finest level, in the
 * context's precision.  nrhs vectors stored one after another. */
int amg_vcycle(amg_ctx *ctx, const double *r_dev, double *z_dev, int nrhs);

/* Colour of every block row of level `level` under AMG_SMOOTHER_HYBRID_GS
 * (colour_out: n_rows int32, host; may be NULL) and the number of colours.
 * 0 <= level < n_levels - 1.  Errors: AMG_ERR_STATE (no hierarchy or another
 * smoother), AMG_ERR_ARG. */
int amg_smoother_colouring(amg_ctx *ctx, int level, int32_t *colour_out, int32_t *n_colours);

/* Solve A_0 u = f by FP64 PCG with one V-cycle as preconditioner (Sec. 7).
 * u_dev holds the initial guess on entry and the solution on return.  Stops
 * when the recurrence residual satisfies ||r||_2 <= rtol ||f||_2 or after
 * maxit iterations (AMG_ERR_NO_CONVERGENCE).  The whole iteration runs on
 * the device as one CUDA graph with a device-side while loop.  iters_out /
 * relres_out receive the iteration count and the final recurrence relative
 * residual per right-hand side (may be NULL).  For the mixed precisions the
 * CG uses the flexible (Polak-Ribiere) beta.  With the double-float CG
 * operator (amg_set_cg_operator) the residual is replaced by the true one
 * f - A_0 u (FP64 operator) at every 10^3 drop of its norm and when it meets
 * the tolerance, and the iteration stops only when the true residual meets
 * it; relres_out then reports the true residual.  f = 0 with u = 0 returns at
 * once (0 iterations, relres 0).  Errors: AMG_ERR_STATE (no hierarchy),
 * AMG_ERR_ARG (NULL vector, nrhs < 1, rtol < 0, maxit < 0),
 * AMG_ERR_NOT_SPD (CG breakdown), AMG_ERR_NO_CONVERGENCE (u holds the last
 * iterate), AMG_ERR_CUDA; with several right-hand sides the first failure
 * is returned after all of them ran. */
int amg_pcg_solve(amg_ctx *ctx, const double *f_dev, double *u_dev, int nrhs, double rtol,
                  int maxit, int *iters_out, double *relres_out);

/* As amg_pcg_solve (PCG of Sec. 7) but f_host / u_host are host arrays
 * (pinned or pageable);
 * the host->device copy of f and u and the device->host copy of u happen
 * inside the call on the context's stream (end-to-end use). */
int amg_pcg_solve_host(amg_ctx *ctx, const double *f_host, double *u_host, int nrhs,
                       double rtol, int maxit, int *iters_out, double *relres_out);

/* z = B^{-1} r for one right-hand side, exactly as amg_vcycle, but with the
 * V-cycle's work vectors in a fixed 16 MiB device array of the library
 * instead of buffers of the context, and without allocating anything.  It
 * serves callers that cannot allocate device memory while it runs: code
 * running where a framework's caching allocator already holds the free
 * device memory (a cudaMalloc there fails or forces the framework to give
 * back its cache), and code with a memory budget fixed in advance.  (The
 * paper has no counterpart: it is an execution variant of the V-cycle.)
 *  - The hierarchy must be uploaded before (amg_upload_hierarchy /
 *    amg_setup allocate; this call does not).
 *  - The array holds 4 vectors per level (256-byte aligned) of the
 *    V-cycle precision; a hierarchy that needs more than 16 MiB is
 *    rejected with AMG_ERR_ARG and a message giving the size.
 *  - The first call on a device is its set-up: it looks up the array's
 *    device address with that device current.  Under lazy module loading
 *    (the CUDA default) this also loads the array's module, and the driver
 *    reserves its 16 MiB at that moment.  Make that first call while
 *    16 MiB are free; later calls allocate nothing.
 *  - The call returns after synchronising the context's stream.
 *  - Every GPU that loads the library holds the array until the process
 *    exits.  All calls on a device share it and it keeps the last call's
 *    contents (nothing in it needs to start at zero); calls that overlap on
 *    the GPU (two contexts, two streams) race on it and must be serialised. */
int amg_vcycle_static(amg_ctx *ctx, const double *r_dev, double *z_dev);

/* Execution mode of amg_pcg_solve* (the PCG of Sec. 7; no counterpart in
 * the paper: a GPU scheduling choice): enable != 0 (default) runs the whole
 * iteration as one CUDA graph with a device-side while loop; enable == 0
 * launches the same kernels one by one and reads the loop condition back
 * after every iteration (a kernel-by-kernel view for profilers, which do not
 * see inside graphs with conditional nodes).  Results are identical. */
int amg_set_pcg_graph(amg_ctx *ctx, int enable);

/* Programmatic dependent launch of the solve-phase kernels (no counterpart
 * in the paper; default on): every V-cycle and CG kernel is launched with
 * programmatic stream serialization and waits at its start for the previous
 * kernel of the stream to complete (griddepcontrol.wait), so that its launch
 * overlaps the predecessor's drain.  enable = 0 launches them plainly.
 * Results are identical.  If a graph build refuses the programmatic
 * launches, the library turns them off. */
int amg_set_launch_overlap(amg_ctx *ctx, int enable);

/* Kernel launches of one amg_pcg_solve (one right-hand side; the V-cycle of
 * Algorithm tg and the CG steps of Sec. 7): *fixed + iterations *
 * *per_iteration. */
int amg_pcg_launches(const amg_ctx *ctx, int32_t *per_iteration, int32_t *fixed);

/* Storage layout of the level operators, applied by the next
 * amg_upload_hierarchy / amg_setup:
 *   AMG_LAYOUT_AUTO             SELL-32 copy (one thread per block row) for
 *                               operators with >= 16 * 32 rows per SM and at
 *                               most 32 blocks per row (A_0), 64
 *                               (rectangular P_l, R_l) or 96 (A_l, l >= 1);
 *                               warp-per-row BSR kernels (one warp streams a
 *                               block row, shuffle reduction) for the rest
 *                               (default)
 *   AMG_LAYOUT_SELL_SHORT_ROWS  SELL-32 for every operator with at most 32
 *                               blocks per row, warp-per-row kernels for the
 *                               rest
 *   AMG_LAYOUT_WARP_ROWS        warp-per-row BSR kernels only
 *   AMG_LAYOUT_ROW_LANES        row-lane BSR kernels only (one lane per
 *                               scalar row of a block row, no reduction)
 *   AMG_LAYOUT_BLOCK_LANES      block-lane BSR kernels only (one warp per
 *                               block row, one whole block per lane)
 *   AMG_LAYOUT_SELL_SPLIT       as AMG_LAYOUT_SELL_SHORT_ROWS, with the
 *                               sorted copies of P_l and R_l run by one warp
 *                               per output row of a slice (the block rows'
 *                               br output rows on br warps)
 * Under AMG_LAYOUT_AUTO the upload also times, for every V-cycle operator
 * but A_0 (whose SELL-32 copy the CG kernels read), the warp-row, row-lane
 * and block-lane kernels and the SELL-32 copy where there is one (for P_l
 * and R_l in both the thread-per-row and the split form) on the operator
 * itself and keeps the fastest.  With the environment variable
 * AMG_TUNE_CACHE naming a file, choices recorded there are reused without
 * timing and new ones appended (a profiled process then applies the kernels
 * an earlier plain process chose).
 * The SELL-32 copies of the transfer operators P_l, R_l and of the coarse
 * A_l (rows of varying length) hold, inside each window of 256 rows, the
 * rows sorted by length, so that each slice of 32 rows carries little
 * padding; A_0 keeps its rows in order.
 * The result of every operator is the same up to the order of the sums. */
enum {
  AMG_LAYOUT_AUTO = 0,
  AMG_LAYOUT_SELL_SHORT_ROWS = 1,
  AMG_LAYOUT_WARP_ROWS = 2,
  AMG_LAYOUT_ROW_LANES = 3,
  AMG_LAYOUT_BLOCK_LANES = 4,
  AMG_LAYOUT_SELL_SPLIT = 5
};
int amg_set_layout_policy(amg_ctx *ctx, int policy);

/* Arithmetic of the CG operator q = A_0 p of the PCG (Sec. 7; no counterpart
 * in the paper: an execution choice of GB300, whose FP64 pipe (about 2 FMA
 * per clock per SM) is slower than its memory for 2x2 / 3x3 FP64 blocks):
 *   AMG_CG_FP64          FP64 fused multiply-adds.
 *   AMG_CG_DOUBLE_FLOAT  every FP64 value of A_0 (scaled by a power
 *                        of two so that max |a| < 1) and of p is held as a pair
 *                        of FP32 numbers hi + lo (48 significant bits, same 8
 *                        bytes), products are formed exactly with FP32 fused
 *                        multiply-adds (Dekker's two-product) and summed with
 *                        Knuth's two-sum (the double-float arithmetic of
 *                        Dekker 1971 / Bailey's double-float method), the
 *                        low parts of each block summed on their own and
 *                        two-summed into the row's low word; q is returned
 *                        in FP64.  Each term carries a relative error
 *                        of about 2^-47 (FP64: 2^-53); p.q, the CG scalars and
 *                        all vector updates stay FP64.  Entries of p below
 *                        about 2^-102 in magnitude lose low-word bits (FP32
 *                        gradual underflow); below 2^-126 they count as zero
 *                        in the product.
 *   AMG_CG_AUTO          (default) double-float with the FP32 / BF16-storage
 *                        V-cycles, FP64 with the FP64 V-cycle.
 * It applies to A_0 with 2x2 or 3x3 blocks and a SELL-32 copy (see
 * amg_set_layout_policy); elsewhere the FP64 kernel runs.  With the
 * double-float operator the PCG replaces the recurrence residual by the true
 * one, f - A_0 u with the FP64 operator, whenever r.r has dropped by 10^6
 * since the start or the last replacement and when it meets the tolerance
 * (residual replacement, van der Vorst and Ye); the stop is decided on the
 * true residual.  The setting takes effect at the next amg_pcg_solve*.
 * Errors: AMG_ERR_ARG (unknown mode). */
enum { AMG_CG_FP64 = 0, AMG_CG_DOUBLE_FLOAT = 1, AMG_CG_AUTO = 2 };
int amg_set_cg_operator(amg_ctx *ctx, int mode);

/* q = A_0 p with the CG operator of the PCG (Sec. 7) in the arithmetic
 * amg_set_cg_operator selects (device vectors of level 0; a single step for
 * parity checks).  Errors: AMG_ERR_STATE (no hierarchy), AMG_ERR_ARG (NULL
 * vector, A_0 block size other than 2 or 3), AMG_ERR_CUDA. */
int amg_cg_operator(amg_ctx *ctx, const double *p_dev, double *q_dev);

/* Per-kernel timing of the CG steps of one PCG iteration (Sec. 7; a
 * measurement aid, no counterpart in the paper), the V-cycle excluded: kind
 * 0 rho = r.z (and beta), 1 p = z + beta p, 2 q = A_0 p with the per-block
 * partials of p.q (the CG operator, in the arithmetic amg_set_cg_operator
 * selects), 3 alpha = rho / p.q, 4 x += alpha p, r -= alpha q with the
 * partials of r.r, 5 the loop decision.  Each kernel is launched reps times
 * on the context's stream after one warm launch and timed with CUDA events;
 * us receives microseconds per launch and bytes its algorithmic bytes
 * (operator values, indices and slice pointers once, every vector it reads
 * or writes once).  The CG vectors of the context are overwritten (the next
 * solve starts afresh).  Up to max_entries entries are written; *n_entries
 * receives the total (6).  Errors: AMG_ERR_STATE (no hierarchy),
 * AMG_ERR_ARG, AMG_ERR_CUDA. */
int amg_profile_pcg(amg_ctx *ctx, int reps, int32_t *kind, double *us, double *bytes,
                    int max_entries, int32_t *n_entries);

/* Per-kernel timing of one V-cycle (Algorithm tg) in the context's
 * precision (a measurement aid, no counterpart in the paper): every step
 * (kind 0 pre-smoothing x = M^+ b, 1 residual t = b - A x, 2 restriction,
 * 3 prolongation x += P y, 4 post-smoothing, 5 coarsest solve) of every
 * level is launched reps times on the context's stream (after one warm
 * launch) and timed with CUDA events; us receives microseconds per launch
 * and bytes its algorithmic bytes (values, indices, row pointers, each
 * input and output vector once).  The work vectors of the context are
 * overwritten.  Up to max_entries entries are written; *n_entries receives
 * the total. */
int amg_profile_vcycle(amg_ctx *ctx, int reps, int32_t *level, int32_t *kind, double *us, double *bytes,
                       int max_entries, int32_t *n_entries);

/* Text listing every level operator (A_l, P_l, R_l of Sec. 3) with its
 * size and the kernel that applies it (after the tuner); owned by ctx,
 * valid until the next call. */
const char *amg_describe(amg_ctx *ctx);

/* Wall-clock seconds of the last amg_setup: [0] host setup (edge matrices,
 * Algorithm 1, prolongations), [1] device Galerkin products and transfers,
 * [2] smoothers / coarsest inverse / layouts, [3] total. */
int amg_setup_times(const amg_ctx *ctx, double *times4);

/* Measure the device's FP64 and FP32 fused-multiply-add throughput (GFLOP/s)
 * with a short synthetic kernel (no counterpart in the paper: it provides the
 * arithmetic peak against which the FP64 sparse kernels, bound by the FP64
 * pipe on sm_103a, are reported).  Takes a few tens of milliseconds. */
int amg_probe_fma_rate(amg_ctx *ctx, double *fp64_gflops, double *fp32_gflops);

/* Cumulative device time (ms, CUDA events) of the last amg_pcg_solve* call
 * (the PCG of Sec. 7). */
int amg_last_solve_ms(const amg_ctx *ctx, float *ms);


/* ------------------------------------------------------------------------
 * Setup: build the hierarchy from the finite element problem (host setup of
 * the paper's method + device Galerkin products), then prepare the solve
 * phase exactly as amg_upload_hierarchy does.
 * ---------------------------------------------------------------------- */

/* The problem of Sec. 2 before the Dirichlet elimination: elasticity
 * (Problem epseps, block = dim or 0) or the scalar problem (Problem gg,
 * block = 1, 1 x 1 blocks; its kernel transfers are the identity and its
 * finest edge / vertex weights E^{ij} = |A_ij|, M^i = max{0, A_ii -
 * sum_{j != i} |A_ij|}, Sec. 4). */
typedef struct {
  int32_t dim;              /* spatial dimension, 2 or 3                          */
  int32_t n_vertices;       /* all mesh vertices, Dirichlet ones included         */
  const double *coords;     /* n_vertices * dim vertex positions (host)           */
  const uint8_t *dirichlet; /* n_vertices flags, 1 = clamped vertex (may be NULL) */
  amg_bsr A_full;           /* stiffness matrix over all vertices (Neumann)       */
  int32_t block;            /* dofs per vertex: 0 or dim (elasticity), 1 (scalar) */
} amg_problem;

/* Parameters of the setup and the readings taken where the paper is silent:
 *  sigma        threshold of Algorithm 1 for mu_s, mu_p, mu_g and mu_D
 *               (not given; 30: the least work to 1e-8 on 3D elasticity
 *               with coefficient jumps; larger values lower the operator
 *               complexity but merge across the jumps)
 *  delta        stabilisation of mu_p / mu_g (Sec. 5, delta = 1)
 *  passes_*     matching passes on the first / later levels (Sec. 7: 5 / 4)
 *  omega        damping of Def. aux_sp (not given; 2/3)
 *  cap_*        row caps of the smoothed prolongation (Sec. 7: 8 first
 *               level / 6 later for real-matrix rows, 4 for auxiliary rows)
 *  coarse_max   stop when a level has at most this many vertices
 *               (0: min(1000, max(64, ceil(n_0 / 10^4))))
 *  min_ratio    stop when a level shrinks by less than this factor
 *  max_levels   upper bound on the number of levels
 *  host_threads OpenMP threads of this call's host setup (0: the process
 *               default); lets independent setups run side by side
 *  device_setup 1 (default): the coarse edge / vertex matrices (Thm.
 *               cemats) and the auxiliary smoothed prolongation (Def.
 *               aux_sp) are built on the device for the agglomerates that
 *               Algorithm 1 finds on the host, and (with
 *               device_pair_measure) Algorithm 1's pair measure mu_p (Lemma
 *               mu2) is evaluated on the device for its batches of candidate
 *               pairs (>= 512 pairs; the greedy loop and the mu_g tests stay
 *               on the host); 0: all on the host
 *  device_pair_measure 1: with device_setup, mu_p as above on the device;
 *               0 (default): mu_p on the host, in the same parallel pass as
 *               the mu_g tests, which a 16-core host finishes sooner than
 *               the device path (same hierarchy: a matter of speed only)
 *  keep_topology 1: keep the coarse topologies the device stages build, for
 *               amg_download_topology (host memory: a level's edge and
 *               vertex matrices); 0 (default): drop them
 *  scalar_only  1: Algorithm 1 with the scalar measure mu_s alone (the
 *               candidate of minimal mu_s is taken; the paper's choice for
 *               the scalar problem and the comparison of Sec. 5); 0 (default)
 * The device stages run for elasticity (2D / 3D); the scalar problem builds
 * its coarse topology and prolongation on the host.
 * A vertex is "standard" (real matrix row in P_s) when its row touches at
 * most cap agglomerates, does not couple to D and is kernel-exact; the
 * auxiliary rows use the own agglomerate and the 3 others with the largest
 * sum of tr E^{il}. */
typedef struct {
  double sigma;
  int32_t delta;
  int32_t passes_first, passes_later;
  double omega;
  int32_t cap_S_first, cap_S_later, cap_A;
  int32_t coarse_max;
  double min_ratio;
  int32_t max_levels;
  int32_t host_threads;
  int32_t device_setup;
  int32_t keep_topology;
  int32_t scalar_only;
  int32_t device_pair_measure;
} amg_setup_params;

/* Fill *p with the defaults listed above (the readings of Sec. 5, 6, 7). */
void amg_default_setup_params(amg_setup_params *p);

/* Build the hierarchy of `prob` on ctx: A_0 = A_full restricted to the free
 * vertices (Sec. 2, eq. (auf)); per level: edge/vertex matrices (Thm.
 * deng_elast, Thm. cemats), Algorithm 1, tentative P (Def. pwp / pwp_el),
 * auxiliary smoothed P_s (Def. aux_sp) on the host, A_{l+1} = P_s^T A_l P_s
 * on the device; then smoothers and the coarsest inverse as in
 * amg_upload_hierarchy.  params may be NULL (defaults).  Replaces any
 * previous hierarchy.  Errors: AMG_ERR_ARG (malformed problem),
 * AMG_ERR_CUDA. */
int amg_setup(amg_ctx *ctx, const amg_problem *prob, const amg_setup_params *params, int precision,
              int smoother);

/* Wall-clock seconds of the last amg_setup's device stages: the Galerkin
 * products with their transfers, the coarse edge / vertex matrices with the
 * smoothed prolongation, and the device evaluation of Algorithm 1's pair
 * measure mu_p (the upload of each matching pass's topology and the batches
 * of candidate pairs it takes; counted inside the host part of
 * amg_setup_times, whose greedy loop waits on it).  Any pointer may be
 * NULL. */
int amg_setup_device_split(const amg_ctx *ctx, double *galerkin_s, double *topology_prolongation_s,
                           double *pair_measure_s);

/* The coarse topology of level `level` (>= 1) built by amg_setup's device
 * stages (Thm. cemats: edge matrices E^{IJ} of the coarse edges (ei < ej),
 * vertex matrices M^I, vertex positions = agglomerate centroids), kept when
 * amg_setup_params.keep_topology was set.  Sizes first (NULL arrays): n
 * vertices, m edges, k x k blocks; then ei / ej (m), E (m k k), M (n k k),
 * pos (n d) into caller host arrays (any may be NULL).  Errors:
 * AMG_ERR_STATE (nothing kept for that level), AMG_ERR_ARG. */
int amg_download_topology(amg_ctx *ctx, int level, int32_t *n_vertices, int64_t *n_edges, int32_t *k,
                          int32_t *ei, int32_t *ej, double *E, double *M, double *pos);

/* Size of P_level, the auxiliary smoothed prolongation (Def. aux_sp) built
 * by amg_setup (0 <= level < n_levels-1): rows, columns, block dims and
 * stored blocks.  Any pointer may be NULL. */
int amg_prolongation_info(const amg_ctx *ctx, int level, int32_t *n_rows, int32_t *n_cols,
                          int32_t *br, int32_t *bc, int64_t *nnzb);

/* Copy P_level (Def. aux_sp, FP64) to caller host arrays sized by
 * amg_prolongation_info. */
int amg_download_prolongation(amg_ctx *ctx, int level, int32_t *rowptr, int32_t *colidx,
                              double *vals);

/* ------------------------------------------------------------------------
 * Batched solve: many independent systems, several load cases each
 * ---------------------------------------------------------------------- */

typedef struct amg_batch amg_batch;

/* Group n_systems contexts (each with an uploaded hierarchy, all on one
 * device and with one V-cycle precision) for batched solves with nrhs load
 * cases per system (nrhs = 1 or 6).  The contexts must outlive the batch and
 * must not be re-uploaded while it exists.  The batch allocates its own
 * multi-load-case work vectors and builds ONE CUDA graph: a device-side
 * while loop of FP64 PCG (Sec. 7) over all systems in lockstep, where every
 * step (each V-cycle step of each level, each CG step) is one grouped launch
 * covering every system, and every matrix block read serves all load cases.
 * Creation also runs the autotuner: each grouped block-sparse product is
 * timed with every tile (lanes per block row 32/16/8 x warps per block 8/4;
 * the SELL-32 copy with 4 or 2 slices per block for 2x2, 3x3, 2x3 and 3x6
 * blocks, which every system's A_0 and P_0 receive, P_0's with
 * length-sorted slices as in the single-system layout; block lanes, 8 or 16
 * lanes per block row with one whole block per lane, for 6x6 and 6x3
 * blocks) and the fastest is kept (amg_batch_describe lists the choices).
 * The CG product q = A_0 p runs in double-float arithmetic (as described
 * at amg_set_cg_operator) when the contexts' CG operator setting, read at
 * creation, asks for it (AMG_CG_DOUBLE_FLOAT, or AMG_CG_AUTO with the FP32
 * or BF16-storage V-cycle; the same setting on every context) and every A_0
 * has 2x2 or 3x3 blocks; otherwise in FP64.  The batched loop stops on every
 * load case's recurrence residual in either arithmetic.
 * Errors: AMG_ERR_ARG (also: a context with AMG_SMOOTHER_HYBRID_GS or
 * AMG_PREC_BF16_COARSE), AMG_ERR_STATE (a context without hierarchy),
 * AMG_ERR_CUDA. */
int amg_batch_create(amg_batch **batch, amg_ctx *const *systems, int n_systems, int nrhs);
void amg_batch_destroy(amg_batch *batch);
const char *amg_batch_last_error(const amg_batch *batch);

/* Text listing the grouped launches of the batch (init, one iteration of
 * the PCG of Sec. 7 with its V-cycle, tail) with the tile the autotuner
 * chose and its time; owned by the batch. */
const char *amg_batch_describe(const amg_batch *batch);

/* Kernel launches of one batched PCG solve (Sec. 7): *fixed + iterations *
 * *per_iteration, where iterations is the largest iteration count over all
 * load cases. */
int amg_batch_launches(const amg_batch *batch, int32_t *per_iteration, int32_t *fixed);

/* Layout of the stacked vectors (right-hand sides f and solutions u of
 * A_0 u = f, Sec. 2, per system and load case): system s occupies [offset, offset +
 * nrhs * n_dofs) with its nrhs load cases one after another (each n_dofs
 * long); *total is the full length.  Any pointer may be NULL. */
int amg_batch_layout(const amg_batch *batch, int s, int64_t *offset, int64_t *n_dofs,
                     int64_t *total);

/* Solve all systems and load cases by FP64 PCG with one V-cycle as
 * preconditioner (Sec. 7) with one graph launch.  f_dev / u_dev
 * are stacked device vectors (amg_batch_layout); u_dev holds the initial
 * guesses and receives the solutions.  Every load case stops when its
 * recurrence residual reaches rtol * ||f|| (it is then frozen) or after
 * maxit iterations.  iters_out / relres_out (n_systems * nrhs, may be NULL)
 * receive per load case the iterations and final relative residual, ms_out
 * the device time of the graph.  AMG_ERR_NO_CONVERGENCE / AMG_ERR_NOT_SPD
 * if some load case failed. */
int amg_batch_pcg_solve(amg_batch *batch, const double *f_dev, double *u_dev, double rtol,
                        int maxit, int *iters_out, double *relres_out, float *ms_out);

/* amg_batch_pcg_solve (Sec. 7) with the stacked f / u in HOST memory (pinned for
 * full copy speed): the copies to and from the device are part of the call
 * and of *ms_out (end-to-end device time). */
int amg_batch_pcg_solve_host(amg_batch *batch, const double *f_host, double *u_host, double rtol,
                             int maxit, int *iters_out, double *relres_out, float *ms_out);

/* ------------------------------------------------------------------------
 * Learned smoother of the finest level (an extension: the paper has no
 * learned component; 3D elasticity, 3x3 blocks)
 *
 * A per-vertex MLP 13 -> 64 -> 64 -> 6 (ReLU) maps the features of vertex v
 * to a lower-triangular factor L; the smoother block is
 * B_v = (L L^T + 1e-6 I) / tr A_vv (SPD by construction) and replaces the
 * block-l1 Jacobi block of level 0, damped by omega = 4 / (3 * 1.05 * lambda)
 * with lambda the largest Ritz value of 30 Lanczos steps on B A (the
 * smoother x += omega B r converges iff omega lambda_max(BA) < 2, which
 * keeps the V-cycle an SPD preconditioner).
 * Features (13, FP32): A_vv's 6 unique entries (00, 11, 22, 01, 02, 12) /
 * tr A_vv; the same entries of sum_j c^{vj} t t^T over v's off-diagonal
 * blocks (t = x_j - x_v, c^{vj} = mean |entry| of A_vj: the displacement
 * part of the finest edge matrices of Thm. deng_elast and its Remark)
 * / (tr A_vv * mean |t|^2); degree / 14.
 * Training target (row-major 3x3): [(A_{N(v),N(v)})^{-1}]_{vv} * tr A_vv,
 * N(v) = v and its neighbours (at most 15).
 * Parameters (AMG_MLP_PARAMS floats): W1 (64 x 13, row-major), b1 (64),
 * W2 (64 x 64), b2 (64), W3 (6 x 64), b3 (6); outputs L00, L10, L11, L20,
 * L21, L22.  The network keeps FP32 master weights for Adam and computes
 * with their BF16 copy, FP32 activations and FP32 accumulation.
 * ---------------------------------------------------------------------- */

#define AMG_MLP_PARAMS 5446

typedef struct amg_mlp amg_mlp;

/* (Learned-smoother extension, no counterpart in the paper.)  Network on
 * `device` with He-normal weights (splitmix64 stream from
 * `seed`, Box-Muller) and zero biases.  Errors: AMG_ERR_ARG, AMG_ERR_CUDA. */
int amg_mlp_create(amg_mlp **mlp, int device, uint64_t seed);
void amg_mlp_destroy(amg_mlp *mlp);
const char *amg_mlp_last_error(const amg_mlp *mlp);
int amg_mlp_n_params(void);

/* (Extension.)  Copy the parameters to host `params` (AMG_MLP_PARAMS floats): the FP32
 * master weights (working = 0) or the BF16 weights the kernels compute with,
 * widened to FP32 (working = 1). */
int amg_mlp_get_params(amg_mlp *mlp, float *params, int working);

/* (Extension.)  Set the master weights (host FP32), refresh the BF16 copy, clear Adam. */
int amg_mlp_set_params(amg_mlp *mlp, const float *params);

/* (Extension; features from the finest edge matrices of Thm. deng_elast.)
 * Features of the level-0 vertices of ctx: coords_host (n_0 x 3 FP64,
 * host) are the vertex positions; X_dev receives n_0 x 13 FP32 (device),
 * tr_dev (device, may be NULL) n_0 traces.  Errors: AMG_ERR_STATE (no
 * hierarchy), AMG_ERR_ARG (not 3x3 blocks, a vertex without positive
 * diagonal block), AMG_ERR_CUDA. */
int amg_learned_features(amg_ctx *ctx, const double *coords_host, float *X_dev, double *tr_dev);

/* (Extension.)  Patch-inverse targets of the level-0 vertices (n_0 x 9, device; either
 * pointer may be NULL), computed in FP64 (dense Cholesky per patch).
 * AMG_ERR_ARG if a vertex has more than 15 neighbours or a singular patch. */
int amg_learned_targets(amg_ctx *ctx, float *T32_dev, double *T64_dev);

/* (Extension.)  Mean loss (1/n) sum_v ||L L^T + 1e-6 I - T_v||_F^2 over n samples
 * (X_dev n x 13, T_dev n x 9, device) and its gradient (host, may be NULL),
 * with the BF16 weights. */
int amg_mlp_loss_grad(amg_mlp *mlp, const float *X_dev, const float *T_dev, int64_t n, double *loss,
                      float *grad_host);

/* (Extension.)  Adam (beta 0.9 / 0.999, eps 1e-8, step lr) over `epochs` passes of n
 * samples in minibatches of `batch` (>= 32), the order of each pass a
 * splitmix64 Fisher-Yates shuffle from `seed`; epoch_loss (host, may be
 * NULL) receives the mean minibatch loss of every pass.  All on the device. */
int amg_mlp_train(amg_mlp *mlp, const float *X_dev, const float *T_dev, int64_t n, int epochs, int batch,
                  float lr, uint64_t seed, double *epoch_loss);

/* (Extension.)  Outputs (n x 6 FP32, device) of the network for n feature rows. */
int amg_mlp_infer(amg_mlp *mlp, const float *X_dev, int64_t n, float *out_dev);

/* (Extension; replaces the block-l1 Jacobi smoother of Sec. 7 on level 0.)
 * Replace the level-0 smoother blocks of ctx by the damped learned blocks
 * omega * B_v (features from coords_host as in amg_learned_features);
 * lambda_out / omega_out (may be NULL) receive the Lanczos estimate and the
 * damping.  The PCG graph stays valid (same buffers).  Errors: AMG_ERR_STATE
 * (no hierarchy or one level), AMG_ERR_ARG, AMG_ERR_NOT_SPD, AMG_ERR_CUDA. */
int amg_set_learned_smoother(amg_ctx *ctx, amg_mlp *mlp, const double *coords_host, double *lambda_out,
                             double *omega_out);

/* Restore the block-l1 Jacobi smoother (Sec. 7) of level 0. */
int amg_reset_smoother(amg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* AMG_H */
