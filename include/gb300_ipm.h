/*
 * gb300_ipm.h -- C ABI of the GB300-native pivoting-free interior-point solver.
 *
 * The method (arXiv 2508.16094): problem (1)  min f(x) s.t. g(x) >= 0  is solved
 * by a primal-dual interior-point method. Every iteration linearises the KKT
 * conditions (2) into the regularised Newton system (3) and condenses it into
 * the primal condensed system (5)
 *
 *     K d_x = -r_p,   K = W + delta_p I + J^T D J,   D = (delta_d I + Lambda^{-1} S)^{-1},
 *
 * which is symmetric positive definite (Sec. 3, "Pivoting-Free IPM"), so it is
 * factored by a supernodal Cholesky that never pivots after a fill-reducing
 * ordering computed once on the host and reused (Sec. 2, "GPU Direct Solvers
 * for Optimization"), followed by triangular solves and iterative refinement
 * (Sec. 2, "Numerical Pivoting": perturbation error corrected by refinement).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an ipm_status and never aborts the process; on error
 *    ipm_last_error(ctx) returns a message owned by the context.
 *  - Pointers named h_* are host memory, d_* are device memory of the GPU the
 *    context was created on. Device buffers are owned by the caller; they are
 *    read or written only during the call, on the context's stream.
 *  - Index arrays are int32 (int64 for CSR/CSC offsets), values float64.
 *  - J is the m x n constraint Jacobian pattern in CSR (rows sorted ascending,
 *    no duplicates). W (optional) is the pattern of the Hessian of the
 *    Lagrangian, lower triangle, CSC. Value arrays follow these patterns' nnz
 *    order.
 *  - Bounds l <= x <= u (+-INFINITY for none) are rows of g with Jacobian rows
 *    +-e_i. Their D entries act on the diagonal of K only. The constraint
 *    vector has m_tot = m + (#finite l) + (#finite u) rows, ordered: the m rows
 *    of J, then the finite lower bounds by ascending variable, then the finite
 *    upper bounds by ascending variable. s, lambda and D have length m_tot.
 *  - Orderings are new->old: perm[k] is the original index of the k-th
 *    eliminated variable.
 *  - Call order: ipm_create -> kkt_analyze -> ipm_set_workspace -> kkt_assemble
 *    -> kkt_factor -> kkt_solve (any number of times). ipm_solve runs the whole
 *    method after ipm_set_workspace. A call out of order returns IPM_ERR_STATE.
 */
#ifndef GB300_IPM_H
#define GB300_IPM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IPM_API __attribute__((visibility("default")))
#else
#define IPM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipm_ctx ipm_ctx;

typedef enum {
  IPM_OK = 0,
  IPM_ERR_ARG = 1,         /* invalid argument (null pointer, size, pattern) */
  IPM_ERR_STATE = 2,       /* call out of order */
  IPM_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  IPM_ERR_NOMEM = 4,       /* workspace too small, or the factor does not fit the device */
  IPM_ERR_NOT_SPD = 5,     /* a pivot of the Cholesky factorisation was not positive */
  IPM_ERR_NUMERIC = 6,     /* NaN/Inf met, or refinement could not reach its tolerance */
  IPM_ERR_MAXITER = 7,     /* interior-point iteration limit reached */
  IPM_ERR_TIMEOUT = 8,     /* a bounded device-side wait ran out */
  IPM_ERR_STALL = 9,       /* the interior-point method stopped making progress */
  IPM_ERR_UNSUPPORTED = 10 /* feature not available for this configuration */
} ipm_status;

/* Arithmetic of the numeric factorisation (storage type in brackets). */
typedef enum {
  IPM_FP64 = 0, /* FP64 FMA                                             [FP64] */
  IPM_FP32 = 1, /* FP32 FMA                                             [FP32] */
  IPM_TF32 = 2, /* TF32 tensor cores (tcgen05), FP32 accumulate (TMEM)  [FP32] */
  IPM_BF16 = 3, /* BF16 tensor cores (tcgen05), FP32 accumulate (TMEM)  [FP32] */
  IPM_TF32X3 = 4 /* TF32 tensor cores, 3-term split A_lo B + A B_lo + A B: about
                    FP32-accurate products; FP32 accumulate (TMEM)      [FP32] */
} ipm_precision;

typedef enum {
  IPM_REFINE_NONE = 0, /* one solve with the factor */
  IPM_REFINE_IR = 1,   /* FP64 iterative refinement, then PCG if it stalls */
  IPM_REFINE_PCG = 2   /* FP64 conjugate gradients preconditioned by the factor */
} ipm_refine;

typedef struct {
  int32_t max_iter;      /* interior-point iteration limit (500) */
  double tol;            /* scaled KKT residual tolerance (1e-8) */
  double delta_p;        /* primal regularisation of (3) (1e-8) */
  double delta_d;        /* dual regularisation of (3) (1e-8) */
  int32_t precision;     /* ipm_precision of kkt_factor inside ipm_solve (IPM_FP64) */
  int32_t storage_fp64;  /* 1: size the factor storage for FP64 values (needed by IPM_FP64
                            and by fallback_fp64); 0: FP32 storage only. -1: automatic */
  int32_t refine;        /* ipm_refine used inside ipm_solve (IPM_REFINE_PCG: the condensed
                            matrix of an LP/QP is SPD, and CG preconditioned by the factor
                            needs fewer solves than refinement; the grid NLP, whose matrix
                            may be indefinite, refines with IPM_REFINE_IR instead) */
  int32_t ir_max;        /* refinement steps per solve (10) */
  double ir_tol;         /* stop once ||b - K x||_inf <= ir_tol ||b||_inf (1e-10) */
  int32_t pcg_max;       /* PCG iterations per solve (100) */
  int32_t fallback_fp64; /* after a linear solve that misses accept_tol with a TF32/BF16/FP32
                            factor, or a low-precision factor that had to perturb pivots or
                            met a pivot of the wrong sign, refactor in the most accurate
                            arithmetic the storage allows (FP64 with FP64 storage, else the
                            split TF32), solve again and keep that arithmetic for the rest of
                            ipm_solve; a step taken with a low-precision factor after which the
                            KKT residual exceeds 10x the previous one is taken back (the
                            iterate before it is restored) and redone in that arithmetic.
                            Counted in ipm_result.fp64_fallbacks (0). When precision is below
                            that arithmetic, ipm_solve allocates n + 2 m_tot doubles on the
                            context's stream for the kept iterate */
  double accept_tol;     /* a solve that misses ir_tol but reaches accept_tol is used (1e-6) */
  int32_t verbose;       /* print one line per interior-point iteration to stderr */
  int32_t warm_start;    /* 1: ipm_solve starts from the x, s, lambda it is given (0) */
  int32_t learned;       /* stale-factor reuse inside ipm_solve (needs an FP32-storage factor):
                            0 off; 1 PCG with the learned correction; 2 PCG with the stale
                            factor alone (E = 0 ablation) (0) */
  int32_t learned_probes;/* probes per training sample (1..8); > 0 also reserves the learned
                            buffers when learned = 0 (0) */
  int32_t learned_pcg_max; /* PCG iterations allowed before falling back to refactoring (30) */
  int32_t formulation;   /* linear system solved for each Newton direction of (3), read by
                            kkt_analyze (Sec. 3, "Condensed KKT Systems"); the bound rows are
                            folded into H = W + delta_p I + D_l + D_u in the last two:
                            IPM_FORM_PRIMAL (5)  K = W + delta_p I + J^T D J (order n, SPD);
                            IPM_FORM_DUAL (6)    D_G^{-1} + A H^{-1} A^T (order m, SPD; W
                                                 diagonal or absent);
                            IPM_FORM_AUGMENTED (4)  [H, A^T; A, -D_G^{-1}] (order n + m,
                                                 quasi-definite, signed LDL^T in FP64/FP32)
                            (IPM_FORM_PRIMAL) */
  int32_t cg_escalate;   /* with fallback_fp64: an interior-point iteration whose two solves
                            took more than this many CG steps with a factor below the
                            fallback arithmetic moves ipm_solve to that arithmetic from the
                            next iteration on (a cheaper factor no longer pays for its extra
                            CG steps); counted in ipm_result.fp64_fallbacks. 0: off (0) */
  int32_t fp64_tc;       /* read by kkt_analyze: 1 runs every FP64 Cholesky factorisation (IPM_FP64,
                            and the FP64 fallback) with its dense updates on the tensor cores:
                            each FP64 operand split into 7 BF16 slices, the slice products summed
                            exactly in FP32 and combined in FP64 (Ozaki scheme; about FP64-
                            accurate, Sec. 6 on the precision of condensed KKT systems); the
                            diagonal blocks stay on the FP64 pipe. Sizes FP64 storage plus 14
                            bytes per factor entry of slices. The signed LDL^T of (4) keeps the
                            FMA path. Long updates are split over CTAs and summed with FP64
                            atomics, so results may differ between runs in the last bits. The
                            slices keep each 128-column row window to 56 bits of its largest
                            entry, so a factorisation that meets a non-positive pivot is redone
                            on the FMA pipe before the status is returned (counted in
                            ipm_result.fp64_tc_rechecks) (0) */
} ipm_options;

typedef enum {
  IPM_FORM_PRIMAL = 0,
  IPM_FORM_DUAL = 1,
  IPM_FORM_AUGMENTED = 2
} ipm_formulation;

/* Default options (values in brackets above). */
IPM_API void ipm_default_options(ipm_options *opts);

typedef struct {
  int64_t n;               /* variables */
  int64_t m_tot;           /* rows of g including finite bounds */
  int64_t nnz_k;           /* entries of the lower triangle of K (diagonal included) */
  int64_t nnz_l;           /* entries of L (sum of column counts) */
  int32_t nsuper;          /* supernodes after relaxed amalgamation */
  int32_t nlevels;         /* levels of the supernodal elimination tree */
  int32_t max_front;       /* largest frontal matrix order */
  int32_t max_ncol;        /* widest supernode */
  double flops;            /* algorithmic factor flops: sum over columns of colcount^2 */
  int64_t factor_entries;  /* stored entries of the supernodal panels (with padding) */
  int64_t update_entries;  /* stored entries of all update matrices */
  int64_t workspace_bytes; /* bytes ipm_set_workspace needs (from the storage option) */
} ipm_symbolic_info;

typedef struct {
  int32_t iterations;   /* refinement or PCG iterations */
  int32_t used_pcg;     /* 1 if PCG ran */
  double rel_residual;  /* final ||b - K x||_inf / ||b||_inf in FP64 */
} ipm_solve_info;

typedef struct {
  int32_t status;           /* ipm_status of the solve */
  int32_t iterations;       /* interior-point iterations */
  int32_t factorizations;   /* numeric factorisations (including retries) */
  int32_t regularizations;  /* delta_p increases after a non-positive pivot */
  int32_t refine_steps;     /* total refinement steps */
  int32_t pcg_steps;        /* total PCG iterations */
  int32_t fp64_fallbacks;   /* refactorisations in the fallback arithmetic after a missed
                               tolerance (see ipm_options.fallback_fp64) */
  int32_t perturbed_pivots; /* low-precision pivots replaced (static pivoting) */
  double objective;         /* f(x) at the returned point */
  double kkt;               /* scaled KKT residual (see ipm_solve) */
  double primal_res, dual_res, compl_res, mu;
  double worst_rel_residual;/* largest linear-solve residual accepted */
  double time_total_ms, time_assemble_ms, time_factor_ms, time_solve_ms, time_other_ms;
  int32_t learned_skips;     /* iterations that reused the held factor (no factorisation) */
  int32_t learned_pcg_steps; /* PCG iterations spent with the held factor */
  int32_t fp64_tc_rechecks;  /* FP64 tensor-core factorisations (options.fp64_tc) whose failed
                                pivot was redone by the FMA-pipe FP64 factor of the same matrix */
} ipm_result;

/* Create a solver context for a problem with n variables and m general
 * constraint rows (Sec. 1, problem (1); Sec. 3, KKT conditions (2)).
 * j_rowptr/j_col: host CSR pattern of J (m x n). w_colptr/w_row: host lower
 * CSC pattern of W (NULL for an LP). l/u: host bounds, length n (NULL = none).
 * stream: a cudaStream_t (NULL = default stream) on the current device.
 * Copies everything it needs; keeps no caller pointer. Touches no GPU memory.
 * Errors: IPM_ERR_ARG for a malformed pattern (unsorted or out-of-range). */
IPM_API ipm_status ipm_create(int32_t n, int32_t m, const int64_t *h_j_rowptr, const int32_t *h_j_col,
                      const int64_t *h_w_colptr, const int32_t *h_w_row, const double *h_l,
                      const double *h_u, const ipm_options *opts, void *stream, ipm_ctx **out);

/* The pattern of a problem as one argument: J (m x n, CSR), W (lower CSC, both
 * pointers NULL for an LP) and the bounds (length n, NULL = none, +-INFINITY
 * allowed), all host memory. */
typedef struct {
  const int64_t *j_rowptr;
  const int32_t *j_col;
  const int64_t *w_colptr;
  const int32_t *w_row;
  const double *l, *u;
} ipm_pattern;

/* ipm_create with the pattern given as one struct (copied; no pointer kept).
 * Errors: IPM_ERR_ARG for p == NULL; otherwise as ipm_create. */
IPM_API ipm_status ipm_create_pattern(int32_t n, int32_t m, const ipm_pattern *p,
                                      const ipm_options *opts, void *stream, ipm_ctx **out);

/* Replace the options of a context (copied). Takes effect at the next call;
 * storage_fp64 is read by kkt_analyze only. Errors: IPM_ERR_ARG for NULL. */
IPM_API ipm_status ipm_set_options(ipm_ctx *ctx, const ipm_options *opts);

/* Symbolic analysis with the ordering given (Sec. 2: the fill-reducing
 * reordering is computed once on the host and reused): pattern of
 * K = W + J^T J + I, elimination tree, postorder, column counts, supernodes
 * with relaxed amalgamation, supernode row structures, level sets and every
 * index map the numeric phase uses. Host only; no GPU work.
 * h_perm: length n, new->old, or NULL for the identity.
 * info (may be NULL) receives sizes and the workspace the numeric phase needs.
 * Errors: IPM_ERR_ARG if h_perm is not a permutation. */
IPM_API ipm_status kkt_analyze(ipm_ctx *ctx, const int32_t *h_perm, ipm_symbolic_info *info);

/* Hand the context a caller-owned device buffer of at least
 * info.workspace_bytes bytes (256-byte aligned). Uploads the symbolic data.
 * The buffer must stay valid until ipm_destroy or the next call of this
 * function. Errors: IPM_ERR_NOMEM if too small, IPM_ERR_CUDA on upload failure. */
IPM_API ipm_status ipm_set_workspace(ipm_ctx *ctx, void *d_buf, size_t bytes);

/* Assembly of the primal condensed matrix, Eq. (5):
 *   K = W + J^T diag(D_J) J + diag(D_bounds) + delta_p I
 * on the fixed pattern, in FP64 (products summed in ascending J row).
 * d_wvals: W values (NULL if no W). d_jvals: J values. d_D: length m_tot.
 * The values are copied into the workspace (kkt_solve's refinement evaluates
 * K x from them), so the caller's buffers may be released after the call.
 * Errors: IPM_ERR_STATE before ipm_set_workspace. */
IPM_API ipm_status kkt_assemble(ipm_ctx *ctx, const double *d_wvals, const double *d_jvals,
                        const double *d_D, double delta_p);

/* Supernodal multifrontal Cholesky P K P^T = L L^T without pivoting (Sec. 2,
 * "LDL^T Factorization"; Sec. 3, SPD condensed system), level by level over
 * the elimination tree (Sec. 2: tree-level parallelism), in the given
 * ipm_precision. FP64 reports the first non-positive pivot: returns
 * IPM_ERR_NOT_SPD with *bad_col = that column in the final ordering (the
 * smallest such column). Lower precisions replace a non-positive pivot by a
 * large value (static pivoting; counted in ipm_last_perturbed) and return
 * IPM_OK; refinement in kkt_solve corrects the perturbation. With
 * options.fp64_tc (set before kkt_analyze), FP64 runs the dense updates on the
 * tensor cores (BF16 slices, Sec. 6 on the precision of condensed systems);
 * a factorisation that meets a non-positive pivot there is redone on the FMA
 * pipe, whose first failing column is the one reported.
 * Errors: IPM_ERR_STATE before kkt_assemble; IPM_ERR_NOMEM if the storage was
 * sized for FP32 and FP64 is requested; IPM_ERR_UNSUPPORTED if fp64_tc is set
 * but was not at kkt_analyze (no slice storage). */
IPM_API ipm_status kkt_factor(ipm_ctx *ctx, int32_t precision, int32_t *bad_col);

/* Solve K x = b with the current factor: x = P^T L^{-T} L^{-1} P b, then FP64
 * refinement on the residual b - K x computed matrix-free from W, J, D
 * (Sec. 2, refinement; ipm_refine). d_b, d_x: nrhs right-hand sides and
 * solutions of length n each, stored one after the other (column k at offset
 * k n), original numbering (may alias). Each right-hand side is solved and
 * refined on its own; info (may be NULL) receives the summed iterations and
 * the largest final relative residual.
 * Errors: IPM_ERR_ARG for nrhs < 1; IPM_ERR_STATE before kkt_factor;
 * IPM_ERR_NUMERIC if a residual misses accept_tol (the other right-hand sides
 * are still solved). */
IPM_API ipm_status kkt_solve(ipm_ctx *ctx, const double *d_b, double *d_x, int32_t nrhs,
                     int32_t refine, ipm_solve_info *info);

/* The whole method on the LP/QP  min c^T x + 1/2 x^T W x  s.t.  J x >= b,
 * l <= x <= u  (Sec. 3): Mehrotra predictor-corrector on the primal condensed
 * system (5), fraction-to-the-boundary step lengths and the barrier update as
 * device map/reduce kernels (Sec. 1: "map or reduce operations").
 * d_jvals, d_b (length m), d_c (length n), d_wvals (NULL for an LP): problem
 * data. d_x (n), d_s and d_lambda (m_tot): outputs. res may be NULL.
 * Scaled KKT residual: max(||g - s||_inf / max(1, ||bfull||_inf),
 * ||grad f - J^T lambda||_inf / max(1, ||c||_inf), ||s .* lambda||_inf /
 * max(1, |f(x)|)), bfull = [b; l_finite; -u_finite].
 * Returns IPM_OK when it reaches opts.tol, else IPM_ERR_MAXITER/NUMERIC/... */
IPM_API ipm_status ipm_solve(ipm_ctx *ctx, const double *d_jvals, const double *d_b, const double *d_c,
                     const double *d_wvals, double *d_x, double *d_s, double *d_lambda,
                     ipm_result *res);

/* One Newton direction of (3) at (x, s, lambda) with complementarity target w
 * (length m_tot; w = mu e for the barrier step), through D, assembly, factor,
 * solve with refinement and the recovery d_lambda = D (w/lambda - g - J d_x),
 * d_s = -s + w/lambda - (s/lambda) d_lambda. All arrays are device memory.
 * Used to check one step of the method in isolation. */
IPM_API ipm_status ipm_newton_direction(ipm_ctx *ctx, const double *d_jvals, const double *d_b,
                                const double *d_c, const double *d_wvals, const double *d_x,
                                const double *d_s, const double *d_lambda, const double *d_w,
                                double *d_dx, double *d_ds, double *d_dlambda);

/* --- batched MPC QPs (Sec. 6: batch solvers) ------------------------------
 * Many small QPs of one family solved by one persistent launch: instance i is
 *   min 1/2 sum_k (x_{k+1}^T Q_i x_{k+1} + u_k^T R_i u_k)
 *   s.t. x_{k+1} = A_k x_k + B_k u_k (k = 0..T_i-1, x_0 given), |u| <= u_max, |x| <= x_max,
 * with 12 states and 4 inputs, the dynamics written as pairs of inequalities
 * (Sec. 1: equalities as pairs of inequalities). Each instance runs the same
 * Mehrotra method on the condensed system (5), which is block tridiagonal
 * with 16 x 16 blocks (stage variables (u_k, x_{k+1})) and factored by a
 * sequential block Cholesky without pivoting. */
typedef struct {
  int32_t count;          /* instances */
  const int32_t *h_T;     /* host, horizons T_i >= 1 */
  const double *d_A;      /* device, (sum T) x 12 x 12, stages of instance 0 first */
  const double *d_B;      /* device, (sum T) x 12 x 4 */
  const double *d_Q;      /* device, count x 12 (diagonal of Q_i) */
  const double *d_R;      /* device, count x 4 (diagonal of R_i) */
  const double *d_x0;     /* device, count x 12 */
  double u_max, x_max;    /* box bounds */
} ipm_mpc_batch;

typedef struct {
  int32_t precision;          /* IPM_FP64, or IPM_FP32: FP32 block factor and solves with
                                 two FP64 refinement steps per solve */
  int32_t instances_per_cta;  /* 2, 4, 8 or 16 (16 lanes per instance) */
  int32_t ctas;               /* persistent grid size, 0 = automatic */
} ipm_mpc_config;

/* Workspace bytes for a batch (host only). */
IPM_API ipm_status ipm_mpc_workspace_bytes(const ipm_mpc_batch *b, size_t *bytes);
/* Upload the horizons, stage offsets and the longest-first instance queue into
 * the workspace (256-byte aligned device buffer). Call once per batch shape. */
IPM_API ipm_status ipm_mpc_prepare(const ipm_mpc_batch *b, void *d_work, size_t bytes, void *stream);
/* Solve every instance to the scaled KKT residual tol (same definition as
 * ipm_solve, with c = 0). Launches only kernels (a queue reset and the
 * persistent solver) on stream, so the call can be captured in a CUDA graph.
 * Outputs (device): d_z ((sum T) x 16, may be NULL), d_obj, d_kkt, d_iters,
 * d_status (ipm_status per instance). */
IPM_API ipm_status ipm_solve_batched(const ipm_mpc_batch *b, const ipm_mpc_config *cfg,
                                     void *d_work, size_t bytes, double tol, int32_t max_iter,
                                     void *stream, double *d_z, double *d_obj, double *d_kkt,
                                     int32_t *d_iters, int32_t *d_status);
/* Autotuner: times instances_per_cta in {2, 4, 8, 16} x four grid sizes (a
 * quarter, half, one and two times the CTAs that fill the SMs' lanes; the
 * smaller grids leave fewer slots than instances, so the work queue balances
 * uneven horizons) for the precision in best->precision on this batch (one
 * warm-up solve, then the mean of two timed solves per shape) and writes the
 * fastest shape to best; h_ms (may be NULL) receives the 16 timings in that
 * order (float[16]). */
IPM_API ipm_status ipm_mpc_autotune(const ipm_mpc_batch *b, void *d_work, size_t bytes, double tol,
                                    int32_t max_iter, void *stream, double *d_z, double *d_obj,
                                    double *d_kkt, int32_t *d_iters, int32_t *d_status,
                                    ipm_mpc_config *best, float *h_ms);

/* --- symbolic analysis of batched patterns on the GPU ----------------------
 * Sec. 2 computes the fill-reducing ordering and the analysis once, serially,
 * and reuses them; Sec. 6 names batch solvers for many problems of one family
 * as the open direction. For a batch of constraint-Jacobian patterns J_b
 * (m_b x n_b, CSR; the problems' K_b = J_b^T J_b + I, a W that is diagonal
 * adds nothing) with orderings P_b, one launch computes per pattern, in the
 * final numbering (P_b followed by the postorder, children and roots visited
 * in ascending order, as kkt_analyze numbers columns): the elimination tree,
 * the column counts of L (diagonal included) and the starts of the
 * fundamental supernodes. The results are exactly those of kkt_analyze on the
 * same pattern (the tree, postorder and counts are unique). */
typedef struct {
  int32_t count;            /* patterns */
  const int32_t *h_n;       /* host: variables of each pattern */
  const int32_t *h_m;       /* host: rows of J of each pattern */
  const int64_t *h_nnz;     /* host: entries of J of each pattern */
  const int64_t *d_rowptr;  /* device: m_b + 1 offsets into d_col per pattern (absolute
                               offsets), patterns one after the other */
  const int32_t *d_col;     /* device: column indices in [0, n_b) (any order within a row) */
  const int32_t *d_perm;    /* device: orderings new -> old, n_b each, one after the other;
                               NULL for the identity */
} ipm_pattern_batch;

/* Workspace bytes of ipm_symbolic_batched (host only). Errors: IPM_ERR_ARG. */
IPM_API ipm_status ipm_symbolic_batched_workspace(const ipm_pattern_batch *b, size_t *bytes);
/* One launch on `stream` over every pattern (one CTA per pattern); returns
 * after the stream has finished it. Outputs (device, n_b entries per pattern,
 * one after the other): d_post (final numbering new -> original index),
 * d_parent (elimination tree in the final numbering, -1 at roots), d_colcount,
 * d_sstart (1 where a fundamental supernode starts). d_work: at least the
 * workspace bytes, 256-byte aligned, owned by the caller.
 * Errors: IPM_ERR_NOMEM for a small or misaligned workspace; IPM_ERR_ARG if a
 * pattern has a column index or an ordering entry out of range (or a repeated
 * ordering entry): *h_bad (may be NULL) receives the first such pattern, -1
 * if none; IPM_ERR_CUDA if a CUDA call fails. */
IPM_API ipm_status ipm_symbolic_batched(const ipm_pattern_batch *b, void *d_work, size_t bytes,
                                        void *stream, int32_t *d_post, int32_t *d_parent,
                                        int32_t *d_colcount, int32_t *d_sstart, int32_t *h_bad);

/* --- grid NLP (the nonlinear problem class of Sec. 2, equalities as pairs) ---
 * min 1/2 ||u - u_t||^2 + alpha/2 ||v||^2 over u, v on an nx x nx grid of
 * interior points (spacing h = 1/(nx+1), u = 0 on the boundary) subject to
 * h(x) = -Lap_h u + c3 u^3 - v = 0, written as the rows h >= 0 and -h >= 0, and
 * v_lo <= v <= v_hi when v_bounded. Variables x = [u; v] (index ix + nx iy),
 * n = m = 2 nx^2. The library evaluates f, h, J (6 entries per row: u at the
 * five-point stencil in ascending column order, then v) and the diagonal
 * Hessian of the Lagrangian W = diag(1 - 6 c3 u (lambda^+ - lambda^-), alpha)
 * in its own kernels. */
typedef struct {
  int32_t nx;          /* grid points per side */
  double alpha;        /* weight of ||v||^2 */
  double v_lo, v_hi;   /* bounds of v (used when v_bounded) */
  int32_t cubic;       /* 1: the u^3 term is present */
  int32_t v_bounded;   /* 1: v_lo <= v <= v_hi */
} ipm_grid_nlp;

/* n, m and nnz(J) of the problem. */
IPM_API ipm_status ipm_grid_nlp_sizes(const ipm_grid_nlp *p, int32_t *n, int32_t *m,
                                      int64_t *nnz_j);
/* Host arrays of the patterns the context must be created with: J (CSR,
 * m + 1 and nnz_j entries), W (lower CSC, diagonal: n + 1 and n entries) and
 * the bounds l, u (n each, +-INFINITY where absent). Any may be NULL. */
IPM_API ipm_status ipm_grid_nlp_pattern(const ipm_grid_nlp *p, int64_t *h_jrowptr,
                                        int32_t *h_jcol, int64_t *h_wcolptr, int32_t *h_wrow,
                                        double *h_l, double *h_u);
/* Interior-point method on the grid NLP (Sec. 2: Newton system (3) condensed
 * to Eq. (5) at every iterate, W the Hessian of L = f - lambda^T (g - s)).
 * The context must have been created with the patterns above. Rules: start
 * x = 0, s = max(g, 1), lambda = 1, mu = 0.1; monotone barrier update
 * mu <- max(tol/10, min(0.2 mu, mu^1.5)) once the scaled barrier error is at
 * most 10 mu; complementarity target mu (no corrector); one common step from
 * the fraction to the boundary (tau = max(0.99, 1 - mu)) shortened by halving
 * (at most 10 times) until the merit f - mu sum ln s + nu ||g - s||_1 decreases
 * by 1e-4 alpha times its directional derivative (up to 10 eps |merit|). A
 * non-positive pivot raises delta_p 100-fold and refactors; an FP32 factor
 * that had to perturb a pivot (or whose solve misses its tolerance) is redone
 * in FP64 when fallback_fp64 is set and the storage holds FP64 (else delta_p
 * is raised), and the remaining iterations factor in FP64; with the same
 * setting, a low-precision step after which the KKT residual exceeds 10x the
 * previous one is taken back (x, s, lambda, mu and the merit penalty
 * restored) and redone in FP64. The pair formulation makes
 * the interior degenerate (both slacks of a pair vanish): on fine grids the
 * dual residual can stall above tol while the objective has converged.
 * d_ut: target (nx^2, device); d_x (n), d_s, d_lambda (m_tot): outputs (device).
 * Allocates 4 n + 6 m_tot + nnz(J) doubles of scratch on the context's stream
 * for the call. res: as for ipm_solve. Errors: IPM_ERR_ARG if the context's
 * pattern is not the grid NLP's; otherwise as ipm_solve. */
IPM_API ipm_status ipm_solve_grid_nlp(ipm_ctx *ctx, const ipm_grid_nlp *p, const double *d_ut,
                                      double *d_x, double *d_s, double *d_lambda,
                                      ipm_result *res);

/* A nonlinear problem min f(x) s.t. g_G(x) >= 0 (m general rows), l <= x <= u
 * (Sec. 1, problem (1)) given by evaluation callbacks on the context's
 * patterns (J: m x n from ipm_create; W: its lower CSC pattern of the Hessian
 * of the Lagrangian). The callbacks run the caller's device code on `stream`
 * (the context's stream) and return 0 on success; any other value ends the
 * solve with IPM_ERR_NUMERIC.
 *   eval(user, d_x, d_f, d_grad, d_g, d_jvals): at x (n), f (one device
 *     double), grad f (n), g_G(x) (m) and the values of J = dg_G/dx in the
 *     pattern's CSR order;
 *   hess(user, d_x, d_lambda, d_wvals): the values, in W's pattern order, of
 *     the Hessian of f - lambda_G^T g_G at x, lambda_G = the first m entries of
 *     d_lambda. */
typedef struct {
  void *user;
  int32_t (*eval)(void *user, const double *d_x, double *d_f, double *d_grad, double *d_g,
                  double *d_jvals, void *stream);
  int32_t (*hess)(void *user, const double *d_x, const double *d_lambda, double *d_wvals,
                  void *stream);
} ipm_nlp;

/* The interior-point method for a nonlinear problem through its callbacks,
 * with the rules of ipm_solve_grid_nlp (monotone barrier, common step with
 * the l1-merit backtracking, inertia by regularisation, the low-precision
 * ladder with the take-back of a step that made the KKT residual grow
 * tenfold, acceptance on the normwise backward error). The starting point is
 * the box midpoint (1 inside a one-sided bound, 0 without bounds); the KKT
 * residual scales the primal part by the largest finite bound (at least 1).
 * Outputs and errors as ipm_solve; allocates 3 n + 6 m_tot + nnz(J) + nnz(W)
 * doubles on the context's stream for the call. Grid NLP: ipm_solve_grid_nlp
 * is this solver with the library's own evaluation kernels. */
IPM_API ipm_status ipm_solve_nlp(ipm_ctx *ctx, const ipm_nlp *p, double *d_x, double *d_s,
                                 double *d_lambda, ipm_result *res);

/* One problem for ipm_solve_problem: an LP or QP (the values of J, b, c and
 * W on the context's pattern, device memory, d_wvals NULL for an LP), the
 * grid NLP (its parameters, host, and the target d_ut, device) or a
 * nonlinear problem given by callbacks (fns). */
typedef enum { IPM_PROBLEM_LPQP = 0, IPM_PROBLEM_GRID_NLP = 1, IPM_PROBLEM_NLP = 2 } ipm_problem_kind;
typedef struct {
  int32_t kind; /* ipm_problem_kind */
  const double *d_jvals, *d_b, *d_c, *d_wvals;
  const ipm_grid_nlp *nlp;
  const double *d_ut;
  const ipm_nlp *fns;
} ipm_problem;

/* Solve one problem: ipm_solve for IPM_PROBLEM_LPQP, ipm_solve_grid_nlp for
 * IPM_PROBLEM_GRID_NLP, ipm_solve_nlp for IPM_PROBLEM_NLP, with the same
 * outputs. Errors: IPM_ERR_ARG for NULL or an unknown kind; otherwise those of
 * the call it makes. */
IPM_API ipm_status ipm_solve_problem(ipm_ctx *ctx, const ipm_problem *p, double *d_x, double *d_s,
                                     double *d_lambda, ipm_result *res);

/* --- learned correction of a stale factor --------------------------------
 * Not in the paper (its iterative-solver discussion in Sec. 1 is the nearest
 * passage). A per-variable network (8 features -> 32 -> 32 -> 17, tanh; 1905
 * FP32 weights W1[32x8], b1, W2[32x32], b2, W3[17x32], b3, row-major) maps the
 * change between the matrix a held factor L_s was computed from and the current
 * K of Eq. (5) to Delta = diag(exp(o_0)) and U = 0.1 o_{1..16} (n x 16) so that
 *   M^{-1} = P^T L_s^{-T} (Delta + U U^T)^{-1} L_s^{-1} P
 * preconditions PCG on K (Woodbury identity, 16 x 16 capacitance in FP64).
 * ipm_solve with options.learned = 1 then skips the refactorisation of an
 * iteration whenever both PCG solves reach ir_tol within learned_pcg_max
 * iterations, and refactors otherwise; learned = 2 is the ablation Delta = 1,
 * U = 0 (plain stale factor). Training minimises the relative probe loss
 *   sum_z ||Delta^{-1} (w_z - Delta z - U (U^T z))||^2 / (probes n),
 *   w_z = L_s^{-1} P K P^T L_s^{-T} z,
 * on iterates of the method itself; features, targets, loss, gradients and
 * Adam run in this library's kernels, with fixed-order reductions (the same
 * call gives the same bits). The learned buffers are sized at kkt_analyze:
 * options.learned != 0 or learned_probes > 0 must be set before it (else
 * ipm_set_options returns IPM_ERR_STATE), and the factor must be stored in
 * FP32 (precision TF32, TF32X3 or FP32). Features of variable i (stored at its
 * permuted index): log(K_ii / K_s,ii); log of the ratio of its bound-row
 * weights / 10; asinh of the signed and absolute change of sum_r J_ri^2 D_r,
 * relative to K_s,ii; log10(mu) / 10; log(mu / mu_s) / 10; log(bound weight /
 * K_ii) / 10; x_i / 10 (clamped as documented in the kernels). */
IPM_API int32_t ipm_learned_param_count(void);
/* Copy the weights out (h_get, may be NULL) and/or in (h_set, may be NULL;
 * setting resets the Adam moments). Host arrays of ipm_learned_param_count()
 * floats. IPM_ERR_STATE before ipm_set_workspace or without learned buffers. */
IPM_API ipm_status ipm_learned_weights(ipm_ctx *ctx, float *h_get, const float *h_set);
/* One training sample against the factor the last ipm_solve iteration left
 * held (its iterate recorded by ipm_solve) at the iterate (d_x, d_s,
 * d_lambda): features d_feat (n x 8, permuted index) and targets d_w
 * (probes x n) for the probes d_z (probes x n, permuted index), probes =
 * min(8, max(1, learned_probes)). All device memory owned by the caller.
 * IPM_ERR_STATE without a held FP32 factor recorded by ipm_solve (a direct
 * kkt_factor call, or a cold-started ipm_solve, drops it). */
IPM_API ipm_status ipm_learned_sample(ipm_ctx *ctx, const double *d_jvals, const double *d_x,
                                      const double *d_s, const double *d_lambda,
                                      const float *d_z, float *d_feat, float *d_w);
/* Loss and its gradient w.r.t. the weights for one sample (no update); h_loss,
 * h_grad (param_count floats) are host pointers and may be NULL. */
IPM_API ipm_status ipm_learned_loss_grad(ipm_ctx *ctx, const float *d_feat, const float *d_z,
                                         const float *d_w, double *h_loss, float *h_grad);
/* steps Adam updates (learning rate lr, beta 0.9 / 0.999) on one sample;
 * h_loss (host, may be NULL): loss before the last update. */
IPM_API ipm_status ipm_learned_train(ipm_ctx *ctx, const float *d_feat, const float *d_z,
                                     const float *d_w, float lr, int32_t steps, double *h_loss);

/* --- inspection (host copies; for tests and tools) --------------------- */

/* Copy the symbolic analysis to host arrays (each may be NULL). Sizes: perm,
 * parent, colcount: n; super: nsuper+1; sparent, slevel: nsuper; srp: nsuper+1;
 * sri: srp[nsuper]. Numbering is the final one (given ordering + postorder). */
IPM_API ipm_status kkt_symbolic_export(const ipm_ctx *ctx, int32_t *h_perm, int32_t *h_parent,
                               int32_t *h_colcount, int32_t *h_super, int32_t *h_sparent,
                               int32_t *h_slevel, int64_t *h_srp, int32_t *h_sri);

/* Assembled K values in the order of the lower CSC pattern of K in the
 * ORIGINAL numbering (columns ascending, rows ascending): h_out has nnz_k. */
IPM_API ipm_status kkt_export_assembled(ipm_ctx *ctx, double *h_out);

/* Entries L(i, j) of the current factor for count (i, j) pairs in the final
 * numbering (h_rows, h_cols; 0 for entries outside the structure), as FP64. */
IPM_API ipm_status kkt_factor_entries(ipm_ctx *ctx, int64_t count, const int32_t *h_rows,
                              const int32_t *h_cols, double *h_out);

/* Test of the bounded device-side waits: in the next launch of the persistent
 * FP32 triangular solve (kkt_solve with an FP32-storage factor) every wait
 * polls its flag at most `spins` times, and the task at position
 * `withheld_task` of the solve's task order (0 = the first block of the first
 * front's forward sweep) is abandoned by the CTA that takes it, so the tasks
 * that need its result wait until their limit runs out. That kkt_solve then
 * returns IPM_ERR_TIMEOUT; the context stays usable. Applies to one launch
 * only; a position past the launch's tasks withholds nothing.
 * Errors: IPM_ERR_ARG for spins == 0 or a negative position. */
IPM_API ipm_status kkt_test_solve_timeout(ipm_ctx *ctx, uint32_t spins, int32_t withheld_task);

/* Low-precision pivots replaced by the last kkt_factor. */
IPM_API int32_t ipm_last_perturbed(const ipm_ctx *ctx);

/* Measurement: average duration in milliseconds (CUDA events on the
 * context's stream) of reps back-to-back launches of one of this library's
 * kernels on the context's current data. kernel 0: the assembly kernel of
 * Eq. (5) on the inputs of the last kkt_assemble (rewrites the same K);
 * 1: the persistent FP32 triangular solve (both sweeps) with the current
 * FP32-storage factor; 2: the FP64 level-scheduled triangular solve with the
 * current FP64 factor; 3 and 4: the persistent FP32 solve's forward sweep
 * alone and its backward sweep alone. The solves overwrite the context's
 * solve scratch only.
 * Errors: IPM_ERR_STATE if the data the kernel needs is missing. */
IPM_API ipm_status kkt_time_kernel(ipm_ctx *ctx, int32_t kernel, int32_t reps, double *ms);

/* --- allocation-free solve -------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they need a solve (code running while a
 * memory pool is locked or exhausted, allocation-free callbacks of another
 * library, or a framework whose allocator must not be re-entered).
 *
 * kkt_solve_noalloc: x = P^T L^{-T} L^{-1} P b with the current factor, like
 * kkt_solve(..., IPM_REFINE_NONE, ...), but its working vectors live in a
 * static device array of kkt_solve_noalloc_capacity() doubles (8 MiB) that
 * every GPU loading this library holds until the process exits. It calls no
 * cudaMalloc/cudaFree and no allocating library routine.
 *  - d_b, d_x: device, length n, original numbering (may not alias).
 *  - Size limit: n + (update-vector entries of the plan) + 2464 doubles must fit
 *    the array, else IPM_ERR_NOMEM with the sizes in ipm_last_error (checked
 *    right after kkt_analyze, before any GPU work).
 *  - When the array is committed: ipm_set_workspace looks up its device
 *    address for the current device (once per device), which loads the part of
 *    this library that holds it and so commits the 8 MiB on that device while
 *    the caller is handing over memory anyway. kkt_solve_noalloc itself then
 *    only reads the cached address: it loads no module and commits nothing.
 *  - The device current at the call must be the one that was current at
 *    ipm_set_workspace (the workspace's device); otherwise IPM_ERR_ARG and no
 *    launch.
 *  - Every call on a device shares the one array, which keeps the last call's
 *    contents; calls that overlap on the GPU (other streams, other contexts,
 *    other threads) race on it and must be serialised by the caller.
 * Errors: IPM_ERR_STATE before kkt_factor, IPM_ERR_ARG on a device mismatch,
 * IPM_ERR_CUDA if a launch fails. */
IPM_API ipm_status kkt_solve_noalloc(ipm_ctx *ctx, const double *d_b, double *d_x);
IPM_API int64_t kkt_solve_noalloc_capacity(void);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts). Read it before and after a call to count that call's launches. */
IPM_API int64_t ipm_kernel_launches(void);

IPM_API const char *ipm_last_error(const ipm_ctx *ctx);
IPM_API void ipm_destroy(ipm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GB300_IPM_H */
