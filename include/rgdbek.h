/*
 * rgdbek.h — C ABI of the GB300 (sm_103a) RGDBEK solver library.
 *
 * RGDBEK (Randomized Greedy Double Block Extended Kaczmarz, arXiv 2509.19267)
 * solves A x = b for A in R^{m x n}, consistent or not (Eq. 1), and converges
 * to the minimum-norm least-squares solution x* = A^+ b (Theorem 2.3).  One
 * outer iteration (Algorithm 1) is:
 *   1. column weights eps^z_j = (A_j^T z_k)^2 / ||A_j||^2            (Section 2)
 *   2. draw ceil(eta_col * n) columns with probability proportional to eps^z;
 *      the column block U_k is the set of distinct drawn indices
 *   3. z_{k+1} = z_k - A_U A_U^+ z_k                                  (Eq. 4)
 *   4. row weights eps^x_i = (b_i - z_{k+1,i} - A^(i) x_k)^2 / ||A^(i)||^2
 *   5. draw ceil(eta_row * m) rows the same way -> row block J_k
 *   6. x_{k+1} = x_k + (A^J)^+ (b^J - z_{k+1}^J - A^J x_k)           (Eq. 4)
 * with x_0 = 0 (or a given x_0, option warm_start) and z_0 = b.  The block
 * pseudo-inverse products are computed by LSQR started from zero (Remark
 * 3.1), which gives minimum-norm solutions: in the column step on A_U with
 * unit columns (the projection A_U A_U^+ z does not depend on the
 * least-squares solution taken), in the row step first on A^J with unit rows
 * (the same minimum-norm solution whenever the block system is consistent,
 * which it is in exact arithmetic since the row residual lies in range(A);
 * solved again unscaled when LSQR finds it inconsistent at rounding level).
 *
 * Every pointer argument marked "device" is CUDA device memory of the
 * current device; "host" pointers are ordinary CPU memory.  All device work
 * of a handle runs on the handle's stream (rgdbek_set_stream).  Handles are
 * not thread-safe: use one handle per stream.  No function throws; every
 * int-returning function returns a status code below.
 */
#ifndef RGDBEK_H
#define RGDBEK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define RGDBEK_OK 0                 /* converged / done                          */
#define RGDBEK_NOT_CONVERGED 1      /* iteration cap reached; x holds x_k        */
#define RGDBEK_ERR_INVALID_ARG (-1) /* bad size, option or null pointer          */
#define RGDBEK_ERR_NONFINITE (-2)   /* NaN or Inf met in b, A or a weight        */
#define RGDBEK_ERR_CUDA (-3)        /* a CUDA runtime call failed                */
#define RGDBEK_ERR_OOM (-4)         /* device allocation failed                  */
#define RGDBEK_ERR_TIMEOUT (-5)     /* time budget or a device wait limit hit    */
#define RGDBEK_ERR_BAD_CSR (-6)     /* row pointers, column order or range wrong */

/* ---- selection rules ----------------------------------------------------- */
#define RGDBEK_SELECT_RANDOM 0 /* Algorithm 1: draws proportional to the weights */
#define RGDBEK_SELECT_GREEDY 1 /* GDBEK threshold sets {j: eps_j >= eta max eps} */

/* ---- stopping rules (tested on x_k before each iteration) ---------------- */
#define RGDBEK_STOP_AUTO 0     /* same as RGDBEK_STOP_NORMAL                      */
#define RGDBEK_STOP_REL_RES 1  /* ||b - A x|| / ||b|| <= tol (consistent systems) */
#define RGDBEK_STOP_NORMAL 2   /* ||A^T (b - A x)|| / ||A^T b|| <= tol            */
#define RGDBEK_STOP_RSE 3      /* ||A x - b||^2 / ||b||^2 <= tol (Section 3.1)    */

/* ---- arithmetic of the solve ------------------------------------------------ */
#define RGDBEK_PRECISION_FP64 0  /* everything in FP64                          */
/* FP32 inner iterations wrapped in FP64 iterative refinement.  Every update
 * of x lies in range(A^T), so A^+ (b - A x) = x* - x for the limit x* = A^+ b
 * (Theorem 2.3): the solve repeats, in FP64,
 *   t = b - A x, ||A^T t||, the stopping test on x
 * and then runs Algorithm 1 entirely in FP32 (A's values rounded to float,
 * float vectors, weights, sampling, LSQR with Kahan-compensated dot
 * products) on A d = t / ||t|| from d = 0, to the stopping rule's relative
 * measure tau = min(0.5, max(RGDBEK_FP32_REFINE_TOL_MIN, 0.5 tol / measure))
 * or until that inner solve stops making progress, and adds ||t|| d to x in
 * FP64.  Rounding t / ||t|| to float bounds what an FP32 step resolves (for
 * least squares, near kappa(A) u_32 ||b - A x*|| / ||b|| in the
 * normal-equation measure), so once an FP32 step fails to halve the FP64
 * measure the remaining steps solve the same refinement system with the FP64
 * iteration (short solves: their z starts near the final residual).  The
 * returned x, the stopping rule and its tolerance are FP64; the limit is
 * A^+ b up to FP64 rounding when A has full column rank.  With a nontrivial
 * null space, FP32 rounding leaves components in it that no refinement
 * removes (relative size about 1e-7).  The inner LSQR tolerance of FP32
 * steps is raised to at least RGDBEK_FP32_INNER_TOL.  stats.iters counts the
 * outer iterations of all inner solves, stats.refinements the FP64 steps. */
#define RGDBEK_PRECISION_FP32_INNER 1
#define RGDBEK_FP32_INNER_TOL 1e-6
#define RGDBEK_FP32_REFINE_TOL_MIN 1e-5

typedef struct rgdbek_s *rgdbek_t;

typedef struct {
    double eta_col;        /* column block fraction eta of Algorithm 1, in (0, 1]  */
    double eta_row;        /* row block fraction, in (0, 1]                         */
    int selection;         /* RGDBEK_SELECT_*                                       */
    double inner_tol;      /* LSQR: stop when ||B^T r|| <= tol ||B||_F ||r|| or
                              ||r|| <= tol ||c||                                    */
    int inner_max;         /* LSQR step cap per block (>= 1)                        */
    int stop_rule;         /* RGDBEK_STOP_*                                         */
    double time_budget_s;  /* wall-clock cap of one solve on the device, 0 = none   */
    uint64_t system_id;    /* second word of the Philox key                         */
    int blocks_per_sm;     /* persistent grid: CTAs per SM, 0 = largest that fits   */
    int threads_per_block; /* solve kernels: 0 = automatic (512, or 1024 when
                              max(m, n) exceeds 2048 per CTA); else a multiple
                              of 32 in [64, 1024]                                   */
    int precision;         /* RGDBEK_PRECISION_*                                    */
    int batch_team;        /* CTAs per system in rgdbek_solve_batched (read from the
                              first handle): 0 = the size rgdbek_tune_batched found,
                              else about one system per team                        */
    int warm_start;        /* 1: x holds x_0 on entry to rgdbek_solve (z_0 = b still);
                              the limit is then A^+ b + (I - A^+ A) x_0, since the
                              method never changes x_0's null-space part.  0: x_0 = 0 */
    double inner_adapt;    /* > 0: the inner tolerance of outer iteration k is
                              max(inner_tol, min(0.1, inner_adapt * r_k)), r_k the
                              stopping rule's measure of x_k (looser block solves
                              while x_k is far from the target; the outer test and
                              its tolerance are unchanged).  0 (default): inner_tol */
    int col_team;          /* two-team schedule of rgdbek_solve (and of the solves of
                              rgdbek_backward and the FP32 form): the column steps of
                              Algorithm 1 (the z recurrence, which does not depend on
                              x) run one outer iteration ahead of the row steps, on
                              col_team CTAs of the grid with barriers of their own,
                              while the other CTAs run the row steps.  0 = automatic
                              (a quarter of the grid when the solved system has at
                              least four times as many rows as columns, where the row
                              step dominates; otherwise one team, as also when
                              inner_adapt > 0, whose inner tolerance ties the column
                              step to x, or when the grid is below 8 CTAs), -1 = one
                              team runs every phase
                              in turn, k > 0 = k CTAs (at most half the grid).  The
                              iterates are the same either way up to the rounding of
                              the reductions; rgdbek_solve_batched always runs one
                              team per system */
    int smem_per_cta;      /* dynamic shared memory (bytes) of each CTA of rgdbek_solve's
                              kernel, where the inner solves keep their chunk of the
                              block and of its vectors: 0 = 96 KB (more shrinks the
                              L1 cache that the full-matrix passes gather through),
                              else a multiple of 1024, at least 32768, capped at what
                              the GPU allows beside the kernel's static shared
                              memory.  Batched solves use 96 KB */
} rgdbek_options;

typedef struct {
    int64_t iters;      /* outer iterations run                                  */
    int64_t inner_u;    /* LSQR steps summed over the column steps               */
    int64_t inner_j;    /* LSQR steps summed over the row steps                  */
    int64_t sum_nu;     /* sum over iterations of |U_k|                          */
    int64_t sum_nj;     /* sum over iterations of |J_k|                          */
    int64_t sum_nnz_u;  /* sum of nnz(A_U) over iterations                       */
    int64_t sum_nnz_j;  /* sum of nnz(A^J) over iterations                       */
    int64_t lsqr_nnz_u; /* sum over iterations of (LSQR steps) x nnz(A_U)        */
    int64_t lsqr_nnz_j; /* sum over iterations of (LSQR steps) x nnz(A^J)        */
    int64_t lsqr_n_u;   /* sum over iterations of (LSQR steps) x |U_k|           */
    int64_t lsqr_n_j;   /* sum over iterations of (LSQR steps) x |J_k|           */
    double rel_res;     /* ||b - A x|| / ||b|| of the returned x                 */
    double normal_res;  /* ||A^T (b - A x)|| / ||A^T b|| of the returned x       */
    double rse;         /* rel_res^2, the paper's RSE                            */
    int status;         /* same as the return code of the solve                  */
    /* device time (ms, globaltimer of CTA 0) spent per phase kind, in the order
     * of RGDBEK_PHASE_NAMES: set-up, column pass, column selection, A_U
     * extraction, LSQR on A_U, z update, row selection, A^J extraction, LSQR on
     * A^J, residual pass, and the FP64 refinement steps of the FP32 form.  With
     * two teams (option col_team) each team's rank 0 times its own phases and
     * the two are added: the column team's run beside the row team's, so the
     * sum exceeds the solve's time; the row team's waits for the column team
     * count as column pass */
    double phase_ms[11];
    int64_t refinements; /* FP64 refinement steps (RGDBEK_PRECISION_FP32_INNER)   */
} rgdbek_stats;

#define RGDBEK_NUM_PHASES 11
#define RGDBEK_PHASE_NAMES                                                            \
    "setup", "col_pass", "col_select", "col_extract", "col_lsqr", "z_update", "row_select", \
        "row_extract", "row_lsqr", "residual_pass", "refine"

typedef struct {
    int64_t m, n, nnz;
    int grid;              /* CTAs of the persistent solve kernel                */
    int threads_per_block;
    int lanes_per_row;     /* lanes that share one CSR row in the A x passes     */
    int lanes_per_col;     /* lanes that share one CSC column in the A^T z passes */
    int num_sms;
    int64_t device_bytes;  /* device memory the handle uses (with its matrix)    */
    int col_team;          /* CTAs of the column team of the next rgdbek_solve
                              (option col_team resolved; 0 = one team)          */
    int smem_per_cta;      /* dynamic shared memory per CTA of rgdbek_solve      */
} rgdbek_info_t;

/* Fills *opt with the defaults: eta_col = eta_row = 0.5 (the paper's
 * sequential experiments, Section 3.1), random selection, inner_tol = 1e-10,
 * inner_max = 200, stop_rule = AUTO, no time budget, system_id = 0,
 * automatic launch shape, precision = FP64. */
void rgdbek_default_options(rgdbek_options *opt);

/* Creates a solver for the m x n matrix A given in CSR form (Eq. 1).
 *   row_ptr  int64[m + 1], row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz
 *   col_idx  int32[nnz], strictly increasing within each row, in [0, n)
 *   vals     double[nnz], finite
 * ptr_is_device: 0 = the three arrays are host memory, 1 = device memory.
 * The arrays are copied; the caller keeps ownership.  The handle builds and
 * owns a CSC copy of A (so A^T products need no atomics), the squared row
 * and column norms, and all workspace.  opt may be NULL (defaults).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Requires m >= 1, n >= 1, nnz >= 0, m and n below 2^31.
 * Errors: INVALID_ARG, BAD_CSR (the CSR checks above), NONFINITE, OOM, CUDA.
 * On error *h is set to NULL and nothing is leaked. */
int rgdbek_create(rgdbek_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, int ptr_is_device,
                  const rgdbek_options *opt, void *stream);

/* Releases everything the handle owns (after synchronising its stream). */
void rgdbek_destroy(rgdbek_t h);

/* A new handle for the same matrix as `base`: it shares base's read-only
 * device arrays (CSR, CSC, squared norms; nothing is copied or rebuilt) and
 * owns its own workspace and control block, so that several right-hand
 * sides of one matrix can be solved at once (rgdbek_solve_batched over the
 * derived handles) with one copy of A in memory.  opt may be NULL (base's
 * options); stream as in rgdbek_create.  The shared arrays live until the
 * last handle using them is destroyed, in any order.  The current device
 * must be base's.  Errors: INVALID_ARG, OOM, CUDA. */
int rgdbek_create_like(rgdbek_t base, const rgdbek_options *opt, void *stream, rgdbek_t *out);

/* Replaces the options (validated as in rgdbek_create). */
int rgdbek_set_options(rgdbek_t h, const rgdbek_options *opt);

/* Sets the stream used by every later call on the handle. */
int rgdbek_set_stream(rgdbek_t h, void *stream);

/* Launch shape and sizes of the handle. */
int rgdbek_get_info(rgdbek_t h, rgdbek_info_t *info);

/* Algorithm 1 on the device: x_0 = 0, z_0 = b, iterate until the stopping
 * rule holds for x_k (tested before each iteration, so b = 0 returns at once),
 * or max_iter iterations ran, or both blocks of an iteration are empty (x can
 * no longer change; reported as converged).
 *   b  device double[m]  (read only)
 *   x  device double[n]  (output; x_k of the last test)
 *   seed  first word of the Philox key; (seed, system_id, k) fixes every draw
 *   st  host, may be NULL
 * The whole solve is one persistent cooperative kernel: no host round trip
 * per iteration.  The call returns after the kernel has finished (it
 * synchronises the handle's stream to read the status).
 * Returns OK, NOT_CONVERGED, NONFINITE (b or a weight not finite), TIMEOUT,
 * INVALID_ARG, CUDA. */
int rgdbek_solve(rgdbek_t h, const double *b, double *x, double tol, int64_t max_iter,
                 uint64_t seed, rgdbek_stats *st);

/* rgdbek_solve with host buffers: copies b (host double[m]) to the device,
 * solves, and copies x back into host double[n].  Page-locked host memory
 * gives the fastest copies. */
int rgdbek_solve_host(rgdbek_t h, const double *b_host, double *x_host, double tol,
                      int64_t max_iter, uint64_t seed, rgdbek_stats *st);

/* Solves nsys independent systems in ONE persistent cooperative launch:
 * system i on handle hs[i] (its matrix, options and workspace; the handles
 * must be distinct, on one device, with the same block size and precision)
 * with device buffers b[i], x[i], tolerance tol[i] and system_id i (seed
 * shared).  The grid is cut into teams of `team` CTAs (options.batch_team of
 * hs[0], or the tuned size, see rgdbek_tune_batched); each team solves its
 * share of the systems one after another with barriers among its own CTAs,
 * each system to its own stopping rule or cap (a per-system convergence
 * mask: a finished system frees its team for the next one).  Systems are
 * assigned largest first to the least loaded team (work ~ nnz + m + n).
 * The launch runs on hs[0]'s stream after the other handles' streams are
 * synchronised.  st: host array of nsys records, may be NULL.  Returns the
 * worst status (the most negative error, else NOT_CONVERGED if any system
 * hit the cap).  Device scratch of about 600 B per system is allocated and
 * freed inside the call. */
int rgdbek_solve_batched(int nsys, rgdbek_t *hs, const double *const *b, double *const *x,
                         const double *tol, int64_t max_iter, uint64_t seed,
                         rgdbek_stats *st);

/* Autotuner of the batched solve: runs the batch for probe_iters outer
 * iterations with each candidate team size (1, 2, 4, 8, 19, 38, 76, 152 CTAs
 * per system, those not above the grid) and the automatic block, then, at
 * the fastest team size and unless hs[0] fixes threads_per_block, with each
 * shape of the solve kernel (512 and 1024 threads).  Each launch is timed
 * with CUDA events; the fastest team size and block are kept in hs[0] for
 * later rgdbek_solve_batched calls with batch_team = 0 (and
 * threads_per_block = 0).  *team_out and *block_out (0 = automatic; may be
 * NULL) receive them; ms_out (host double[RGDBEK_BATCH_TEAM_CANDIDATES + 2],
 * may be NULL) the time of each team size and then of the 512- and
 * 1024-thread shapes (-1 where skipped).  The x buffers are overwritten by
 * the probe solves, which run their full length whatever the handles'
 * time_budget_s.  Returns OK or the first error. */
#define RGDBEK_BATCH_TEAM_CANDIDATES 8
int rgdbek_tune_batched(int nsys, rgdbek_t *hs, const double *const *b, double *const *x,
                        const double *tol, int64_t probe_iters, uint64_t seed, int *team_out,
                        int *block_out, double *ms_out);

/* Autotuner of the block fraction eta (Section 2: a larger eta gives larger
 * blocks, so costlier iterations but fewer of them; which wins depends on the
 * matrix and on the GPU).  For each candidate c (host array of ncand values in
 * (0, 1]; candidates NULL with ncand 0 takes the RGDBEK_ETA_CANDIDATES values
 * 0.05, 0.1, 0.2, 0.3, 0.5) it runs probe_iters outer iterations with
 * eta_col = eta_row = c from x0 = 0 on b (device, m) into x (device, n,
 * overwritten), times them with CUDA events, and scores the decrease of the
 * stopping rule's measure (1 at x0 = 0) as -ln(measure) per second.  The
 * handle keeps the best candidate as eta_col and eta_row; *eta_out receives
 * it and rate_out (host double[ncand], may be NULL) every score.  The probe
 * is short, so the score favours the early rate of decrease; the probes run
 * their full length whatever the handle's time_budget_s.  Returns OK or the
 * first error (the options are then left as they were). */
#define RGDBEK_ETA_CANDIDATES 5
int rgdbek_tune_eta(rgdbek_t h, const double *b, double *x, const double *candidates,
                    int ncand, int64_t probe_iters, uint64_t seed, double *eta_out,
                    double *rate_out);

/* Autotuner of the single solve's kernel shape: runs probe_iters outer
 * iterations from x0 = 0 on b (device, m) into x (device, n, overwritten)
 * with 512 and with 1024 threads per CTA, times each with CUDA events, and
 * sets the handle's threads_per_block to the faster.  *block_out receives it
 * and ms_out (host double[2], may be NULL) the two times; the probes run
 * their full length whatever the handle's time_budget_s.  Returns OK or the
 * first error (the options are then left as they were). */
int rgdbek_tune(rgdbek_t h, const double *b, double *x, int64_t probe_iters, uint64_t seed,
                int *block_out, double *ms_out);

/* Autotuner of the two-team schedule (option col_team): runs probe_iters
 * outer iterations from x0 = 0 on b (device, m) into x (device, n,
 * overwritten) with one team and with column teams of 2/16, 3/16, 4/16 and
 * 5/16 of the grid (RGDBEK_COL_TEAM_CANDIDATES runs, in that order), times
 * each with CUDA events on the handle's stream and keeps the fastest as the
 * handle's col_team.  The right split depends on how the column step's work
 * (the z recurrence) compares with the row step's on the matrix.  *col_team_out
 * (may be NULL) receives it (-1 = one team); ms_out (host
 * double[RGDBEK_COL_TEAM_CANDIDATES], may be NULL) each time, -1 where skipped
 * (grids below 8 CTAs run one team).  The probes run their full length
 * whatever the handle's time_budget_s.  Returns OK or the first error (the
 * options are then left as they were). */
#define RGDBEK_COL_TEAM_CANDIDATES 5
int rgdbek_tune_teams(rgdbek_t h, const double *b, double *x, int64_t probe_iters,
                      uint64_t seed, int *col_team_out, double *ms_out);

/* Autotuner of the work split of the full-matrix passes (A^T z and b - A x
 * of every outer iteration, the FP64 passes of the refinement loop and the
 * component SpMVs): for each candidate of RGDBEK_SPMV_LANE_CANDIDATES lanes
 * per CSR row (1, 2, 4, 8, 16, 32) it times reps launches of the CSR product
 * (after one warm-up launch), and likewise per CSC column for the CSC
 * product, with CUDA events on the handle's stream, and keeps the fastest of
 * each for the handle (rgdbek_get_info reports them as lanes_per_row /
 * lanes_per_col).  The sums of each pass are taken in a different order per
 * lane count, so a solve's rounding (not its limit) depends on the choice.
 * us_out: host double[2 * RGDBEK_SPMV_LANE_CANDIDATES] (may be NULL), the
 * median time in microseconds of each candidate, CSR first.  The handle's
 * workspace serves as input and output vectors (zeros).  Returns OK,
 * INVALID_ARG (reps < 1), CUDA. */
#define RGDBEK_SPMV_LANE_CANDIDATES 6
int rgdbek_tune_spmv(rgdbek_t h, int reps, int *lanes_row, int *lanes_col, double *us_out);

/* Sets the lanes per row / column of the full-matrix passes by hand (powers
 * of two in [1, 32]; the default is about sixteen entries per lane). */
int rgdbek_set_pass_lanes(rgdbek_t h, int lanes_row, int lanes_col);

/* Implicit adjoint of the solve (reverse-mode gradient).  The method
 * converges to x = A^+ b, the minimum-norm least-squares solution (the
 * convergence theorem of Section 2).  Given the gradient g = dL/dx of a loss
 * at that x, the derivative of the pseudo-inverse (Golub and Pereyra 1973,
 * along perturbations that keep rank(A)) gives
 *   dL/db    = w                         with w = A^+T g
 *   dL/dA_ij = r_i v_j - w_i x_j         with r = b - A x, v = A^+ w
 *              [+ u_i p_j]               with u = A^+T x, p = (I - A^+ A) g
 * The bracketed term is zero when A has full column rank; it is added only
 * with flags = RGDBEK_ADJ_RANK_TERM.  Each of w, v, u and A^+(A g) is an
 * Algorithm 1 solve on the device from a zero start (w and u on A^T, using
 * the handle's CSC arrays as the CSR form of A^T), with the handle's options,
 * tolerance tol and cap max_iter; solve i (w, v, u, q in that order) uses
 * seed + i.  The paper itself has no adjoint; this call builds on its solver.
 *   b          device double[m]   right-hand side of the forward solve
 *   x          device double[n]   the forward solution
 *   grad_x     device double[n]   g
 *   grad_b     device double[m]   output dL/db, or NULL
 *   grad_vals  device double[nnz] output dL/dA at the stored entries, in the
 *                                 CSR order given to rgdbek_create; or NULL
 *                                 (then only w is solved for)
 *   st         host rgdbek_stats[4] (w, v, u, q solves; unused ones zeroed),
 *              or NULL
 * The handle owns a scratch area of 4m + 2n doubles, allocated on the first
 * call and freed by rgdbek_destroy.  Returns OK, NOT_CONVERGED (some solve hit
 * max_iter; the gradients are still written), or the first error of a solve
 * (its outputs are then not written), INVALID_ARG (a NULL input, tol < 0,
 * max_iter < 0, unknown flag bits), OOM, CUDA. */
#define RGDBEK_ADJ_RANK_TERM 1
int rgdbek_backward(rgdbek_t h, const double *b, const double *x, const double *grad_x,
                    double *grad_b, double *grad_vals, double tol, int64_t max_iter,
                    uint64_t seed, int flags, rgdbek_stats *st);

/* Records the blocks of each iteration of the next solves into device
 * buffers: counts int64[count_cap][4] = (|U_k|, |J_k|, LSQR steps of the
 * column step, of the row step); lists int32[list_cap] = U_0, J_0, U_1, J_1,
 * ... concatenated.  Recording stops silently when either buffer is full.
 * Pass NULLs to turn recording off. */
int rgdbek_set_trace(rgdbek_t h, int64_t *counts, int64_t count_cap, int32_t *lists,
                     int64_t list_cap);

/* Records, for each of the first iters_cap outer iterations k of the next
 * solves, the two vectors the blocks of iteration k are drawn from (Section 2,
 * Algorithm 1), so that a caller can replay the selections on the host:
 *   g  device double[iters_cap][n]: row k = A^T z_k, whose squares over the
 *      squared column norms are the column weights eps^z
 *   r  device double[iters_cap][m]: row k = b - z_{k+1} - A x_k, whose squares
 *      over the squared row norms are the row weights eps^x
 * Either may be NULL; both NULL turns recording off (iters_cap is then
 * ignored).  With either given, iters_cap >= 1 (else INVALID_ARG).  The caller
 * owns the buffers and keeps them alive while recording is on; rgdbek_solve
 * (not the transposed or batched solves) writes them. */
int rgdbek_set_trace_vectors(rgdbek_t h, double *g, double *r, int64_t iters_cap);

/* ---- component entry points (each runs the same device code the solve
 *      kernel uses; for tests and measurement) ------------------------------ */

/* y = A x: x device double[n], y device double[m]  (CSR product). */
int rgdbek_spmv(rgdbek_t h, const double *x, double *y);

/* The FP32 form's products with the float copy of A (values rounded to float,
 * made on first use and kept with the matrix): transposed = 0 gives y = A x
 * (x device float[n], y device float[m], CSR), transposed = 1 gives
 * y = A^T x (x device float[m], y device float[n], CSC); each lane's share of a
 * line is summed with Kahan compensation, the lanes then in float.  Errors:
 * INVALID_ARG, OOM (the float copy), CUDA. */
int rgdbek_spmv_f32(rgdbek_t h, int transposed, const float *x, float *y);

/* g = A^T z: z device double[m], g device double[n]  (CSC product). */
int rgdbek_spmv_t(rgdbek_t h, const double *z, double *g);

/* Residual weights of Section 2: which = 0 gives eps_j = v_j^2/||A_j||^2
 * (v device double[n]), which = 1 gives eps_i = v_i^2/||A^(i)||^2 (v device
 * double[m]); eps is 0 where the norm is 0.  eps: device output of the same
 * length; eps_max: host, receives the maximum.  NONFINITE if a weight is NaN
 * or Inf. */
int rgdbek_weights(rgdbek_t h, int which, const double *v, double *eps, double *eps_max);

/* Largest number of draws per weight that the samplers accept: s must not
 * exceed RGDBEK_MAX_DRAWS_PER_ENTRY * len (Algorithm 1 itself draws at most
 * len, since eta <= 1).  Each draw costs a search over the prefix sums, so a
 * bound on s is a bound on the time one sampling kernel can run. */
#define RGDBEK_MAX_DRAWS_PER_ENTRY 16

/* Block selection of Algorithm 1 on given weights eps (device double[len],
 * nonnegative, finite; len <= max(m, n)): s draws (0 <= s <=
 * RGDBEK_MAX_DRAWS_PER_ENTRY * len, else INVALID_ARG) with probability
 * eps_j / sum eps, Philox key (seed, sysid), counter (k, phase, t/4, 0);
 * the sorted distinct drawn indices go to idx (device int32[len]) and their
 * number to *count (host).  All-zero weights give an empty block.  With
 * selection = GREEDY in the handle's options the block is instead
 * {j : eps_j >= eta eps_max} with eta = eta_col (phase 0) or eta_row
 * (phase 1), and s, seed, sysid, k are ignored. */
int rgdbek_sample(rgdbek_t h, const double *eps, int64_t len, int64_t s, uint64_t seed,
                  uint64_t sysid, int64_t k, int phase, int32_t *idx, int64_t *count);

/* Largest len accepted by rgdbek_sample_noalloc. */
#define RGDBEK_NOALLOC_MAX_LEN 262144

/* The block selection of rgdbek_sample (random rule only) for callers that
 * cannot allocate device memory when they draw a block: an application whose
 * memory pool already holds the GPU's memory, a latency-critical loop that
 * cannot accept the device synchronisation cudaMalloc / cudaFree may cause,
 * or a plugin whose host forbids allocation after start-up.  The paper has no
 * counterpart; this is an entry point for deploying the sampler.
 *   eps    device double[len], nonnegative and finite, 1 <= len <=
 *          RGDBEK_NOALLOC_MAX_LEN (larger len: INVALID_ARG, nothing launched)
 *   s      number of draws, 0 <= s <= RGDBEK_MAX_DRAWS_PER_ENTRY * len (else
 *          INVALID_ARG, nothing launched)
 *   idx    device int32[len] output: the sorted distinct drawn indices
 *   count  device int64 output: their number, -1 if a weight is negative or
 *          not finite, -2 if the kernel gave up a device wait
 *   stream cudaStream_t the work is queued on (NULL = legacy default stream)
 * The draws are those of rgdbek_sample with the same (s, seed, sysid, k,
 * phase).  The call only queues work and returns (no host synchronisation);
 * results are valid once the stream has reached them.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch memory (about 3.4 MB) is
 * one static device array that every GPU loading the library holds until the
 * process exits.  All calls on a device share that array, which keeps the
 * last call's contents; each call resets what must start from zero.  Calls
 * whose work overlaps on the GPU (e.g. on two streams) race on the array and
 * must be ordered by the caller.  The first call on a device, with that
 * device current, looks up the array's device address and the launch shape
 * (cudaGetSymbolAddress, occupancy queries); make that first call before any
 * stream capture.  If that look-up fails the call returns CUDA and the next
 * call on the device tries it again.  Returns OK, INVALID_ARG or CUDA. */
int rgdbek_sample_noalloc(const double *eps, int64_t len, int64_t s, uint64_t seed,
                          uint64_t sysid, int64_t k, int phase, int32_t *idx, int64_t *count,
                          void *stream);

/* Copies the squared row norms (device double[m]) and squared column norms
 * (device double[n]) computed at creation; either may be NULL. */
int rgdbek_get_norms(rgdbek_t h, double *row_norms2, double *col_norms2);

/* Copies the handle's CSC form of A: col_ptr device int64[n + 1], row_idx
 * device int32[nnz] (increasing within each column), vals device double[nnz]. */
int rgdbek_get_csc(rgdbek_t h, int64_t *col_ptr, int32_t *row_idx, double *vals);

/* Human-readable name of a status code (static storage). */
const char *rgdbek_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RGDBEK_H */
