/*
 * libmlmc -- the data-parallel hot path of mixed-precision multilevel Monte
 * Carlo (MPML) for -div(a grad u) = f on the unit square with a lognormal
 * random coefficient, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Martinek, Carson, Scheichl, "Exploiting Inexact Computations in
 * Multilevel Monte Carlo and Other Sampling Methods", arXiv 2503.05533.
 * Passages are cited as Sec./Eq./Alg. of that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids.  A grid with n cells per side has (n+1)^2 nodes (x_i, y_j) =
 *    (i/n, j/n); a nodal array stores node (i, j) at index j*(n+1) + i
 *    ("dense nodal layout").  Batches of S grids are contiguous:
 *    sample s starts at s*(n+1)^2.  Level l uses n_l = n0 * m^l.
 *  - Memory.  Every array argument documented "device" is a device pointer
 *    owned by the caller (e.g. allocated by PyTorch); the library never frees
 *    it.  "host" arrays are ordinary host memory.  The context owns its own
 *    workspaces (basis tables, solver scratch) and frees them in mlmc_destroy.
 *  - Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls enqueue work on it and return without
 *    synchronising, except where a call says it synchronises.
 *  - Errors.  Every call returns an mlmc_status and never aborts, traps or
 *    exits.  On failure the context records a message, mlmc_last_error(ctx).
 *    Device-side waits are bounded: a wait that runs out makes the call return
 *    MLMC_E_TIMEOUT with the GPU still usable.
 */
#ifndef LIBMLMC_H
#define LIBMLMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLMC_MAX_LEVELS 16

typedef enum {
    MLMC_OK = 0,
    MLMC_E_ARG = 1,          /* invalid argument: null pointer, size out of range, bad enum */
    MLMC_E_NOMEM = 2,        /* a device or host allocation failed */
    MLMC_E_CUDA = 3,         /* a CUDA runtime call failed; text in mlmc_last_error */
    MLMC_E_NOCONV = 4,       /* some solve stopped before its tolerance (see per-solve flags) */
    MLMC_E_NONFINITE = 5,    /* a non-finite value appeared (coefficient overflow, NaN input) */
    MLMC_E_TIMEOUT = 6,      /* a bounded device-side wait ran out; the kernel returned early */
    MLMC_E_UNSUPPORTED = 7   /* a valid request this build does not implement */
} mlmc_status;

/* Arithmetic of a solve's inner (correction) solver and storage of its
 * coefficient, Alg. 2.1 precisions (u_f, u_s) in Sec. 2.3.  The outer
 * residual r = b - A x and the update x += d are always FP64 (u = u_r =
 * double).  S = storage only: the coefficient is stored in 16 bits and
 * widened to FP32 inside the stencil, all Krylov arithmetic being FP32. */
typedef enum {
    MLMC_FP64 = 0,    /* inner FP64, coefficient FP64 (plain double solve)       */
    MLMC_FP32 = 1,    /* inner FP32, coefficient stored FP32                     */
    MLMC_BF16S = 2,   /* inner FP32, coefficient stored bfloat16                 */
    MLMC_FP16S = 3,   /* inner FP32, coefficient stored IEEE half                */
    MLMC_FP64TC = 4,  /* fields only: FP64 field from the tensor-core contraction
                         (see mlmc_sample_fields); not an inner precision        */
    MLMC_FP8S = 5     /* Cholesky factor only: stored FP8 E4M3 (4 exponent and 3
                         mantissa bits, the quarter precision q43 of Sec. 5.2)   */
} mlmc_prec;

/* Solvers of the correction equation in the refinement (Alg. 2.1): the Krylov
 * methods of Sec. 2.2, and the banded Cholesky factorisation of Sec. 5.2,
 * computed once per system in the precision `prec` (IEEE half, bfloat16,
 * single or double storage; FP32 arithmetic below double) and reused by every
 * correction solve.  The Cholesky solver takes grids of 2 to 128 cells. */
typedef enum { MLMC_CG = 0, MLMC_MINRES = 1, MLMC_CHOLESKY = 2 } mlmc_solver;
/* Preconditioner of the inner solves (CG and MINRES). */
typedef enum { MLMC_PC_JACOBI = 0, MLMC_PC_MG = 1 } mlmc_precond;   /* Sec. 2.2 */

/* per-solve flag bits (int32 arrays returned by the solves) */
#define MLMC_F_CONVERGED 1   /* ||b - A x||_2 / ||b||_2 < delta reached (Eq. (2.1), C = 1) */
#define MLMC_F_MAXIT     2   /* iteration budget exhausted before delta */
#define MLMC_F_STAGNATED 4   /* an outer refinement step reduced the residual by less than 2x */
#define MLMC_F_NONFINITE 8   /* NaN / Inf in the residual (e.g. coefficient overflow, Sec. 5.2) */
#define MLMC_F_TIMEOUT   16  /* a bounded wait of the solve's row pipeline ran out; the solve stopped early */

/* Random log-coefficient, log a(x) = sum_{k<K} xi_k Phi_k(x), xi_k ~ N(0,1). */
typedef struct {
    int kind;          /* 0: separable exponential covariance sigma2 exp(-|dx1|/corr_len - |dx2|/corr_len)
                          1: the paper's field, Sec. 5.1 Eq. (5.2): Phi_j = sigma j^-q sin(2 pi j x1) cos(2 pi j x2)
                          2: one spatially constant mode, Phi_0 = sigma                                    */
    int K;             /* number of terms, 1 <= K <= 256 (kind 2: K = 1)                                  */
    double sigma2;     /* variance sigma^2 > 0                                                             */
    double corr_len;   /* correlation length (kind 0), > 0                                                 */
    double q;          /* decay exponent (kind 1)                                                          */
} mlmc_field;

/* The level hierarchy and QoI of Problem 4.5 (Sec. 4.3) and Sec. 5.1. */
typedef struct {
    int n0;            /* cells per side on level 0 (h_0 = 1/n0), 2 <= n0                                 */
    int m;             /* refinement factor between levels, m >= 2 (h_l = h_0 m^-l)                        */
    int L_max;         /* finest level that may be used, 0 <= L_max < MLMC_MAX_LEVELS, n0 m^L_max <= 2048  */
    mlmc_field field;
    int qoi;           /* 0: Q = int_D u_h ; 1: Q = int_B u_h over the box B below                         */
    double box[4];     /* x0, x1, y0, y1 of B (sides on grid lines of level 0)                              */
    double f;          /* constant right-hand side f (Sec. 5.1 uses f = 1)                                 */
    uint64_t seed;     /* Philox key                                                                       */
} mlmc_problem;

typedef struct mlmc_ctx mlmc_ctx;

/* Level accumulator for Y_l = Q_l - Q_{l-1} (Eq. (4.1)): count, Welford mean
 * and sum of squared deviations (s_l^2 = m2 / n, Eq. (4.2)), and
 * Kahan-compensated sums of Y and Y^2. */
typedef struct {
    int64_t n;
    double mean, m2;
    double sum, sum_c, sumsq, sumsq_c;
} mlmc_acc;

/* ------------------------------------------------------------------------- */
/* Context                                                                    */

/* Create a context on CUDA device `device`: validates `prob`, builds the KL
 * basis tables for every level grid 0..L_max on the host and uploads them.
 * *out is set to NULL on failure; the message is then in mlmc_last_error(NULL). */
mlmc_status mlmc_create(const mlmc_problem* prob, int device, mlmc_ctx** out);
void mlmc_destroy(mlmc_ctx* ctx);                 /* NULL is ignored */
/* The Philox key of this context's samples (mlmc_problem.seed).  Nothing the
 * context built depends on it (the KL basis, the workspaces), so estimates with
 * new seeds reuse the context. */
mlmc_status mlmc_set_seed(mlmc_ctx* ctx, uint64_t seed);
const char* mlmc_last_error(const mlmc_ctx* ctx); /* never NULL; "" when no error */
const char* mlmc_version(void);
int64_t mlmc_launch_count(void);                  /* kernels launched by this library so far (process) */

/* ------------------------------------------------------------------------- */
/* A1 + A2: random inputs and the coefficient field (Sec. 5.1, Eq. (5.2);
 * independence of levels, Sec. 4.1).
 *
 * xi[s][k] = Phi^-1(u) with u from Philox4x32-10 (key = seed, counter =
 * (sample lo, sample hi, level, k >> 1), words (0,1) for even k and (2,3) for
 * odd k, u = (M + 1/2) 2^-52 for the 52-bit M = (w_a << 20) | (w_b >> 12)) and
 * Wichura's AS241 inverse normal; sample indices are first .. first+S-1.
 * a[s][v] = exp(sum_k xi[s][k] Phi_k(x_v)) on the (n_l+1)^2 nodes of level l.
 *   xi    device FP64 [S][K], out (may be NULL when not wanted)
 *   a     device, out: S rows of the (n_l+1)^2 nodal values, row s at a + s a_ld
 *         elements, by field_prec:
 *         MLMC_FP64   FP64; contraction and exp on the FP64 pipe (plain FP64 form);
 *         MLMC_FP32   FP32; tensor-core contraction with split FP16 operands
 *                     (hi + 2^-11 lo) and FP32 accumulation, then expf: about
 *                     1e-6 relative error;
 *         MLMC_FP64TC FP64; tensor-core contraction with an exactly accumulated
 *                     integer lead slice and two FP16 correction slices per
 *                     operand, log a as a float-float pair, exp in float-float
 *                     (Tang's table-driven method): log a within about 1e-9
 *                     (a bound in terms of sum |xi_k| and sum |Phi_k| is given
 *                     in kl_tc.cu), the master coefficient of the mixed form.
 *   a_ld  elements from one row of `a` to the next: 0 (dense, (n_l+1)^2) or at
 *         least (n_l+1)^2; the gap is not written.  Rows of whole 128-byte lines
 *         (a_ld a multiple of 32, `a` 128-byte aligned) let the tensor-core FP32
 *         synthesis store full lines straight from its accumulators; other
 *         pitches go through a shared-memory staging step (the estimate pads
 *         its fields this way).
 * S = 0 is a no-op.  Errors: MLMC_E_ARG for level outside [0, L_max], S < 0,
 * null a with S > 0, a_ld nonzero and below (n_l+1)^2, field_prec not
 * FP64/FP32/FP64TC. */
mlmc_status mlmc_sample_fields(mlmc_ctx* ctx, int level, uint64_t first, int S,
                               double* xi, void* a, int64_t a_ld, mlmc_prec field_prec, void* stream);

/* A2 alone: the same field from caller-given coefficients xi (device FP64
 * [S][K]) on the grid of level `level`, rows a_ld apart as above.  Used by the
 * gradient path. */
mlmc_status mlmc_synthesize_fields(mlmc_ctx* ctx, int level, int S, const double* xi,
                                   void* a, int64_t a_ld, mlmc_prec field_prec, void* stream);

/* ------------------------------------------------------------------------- */
/* A3 + A4: the P1 stiffness operator applied matrix-free (Sec. 3.1; uniform
 * grid, cells split along the SW-NE diagonal, a_T = mean of its vertex values,
 * which makes A a 5-point operator).  y = A x on the (n-1)^2 interior nodes,
 * y = 0 on boundary nodes; x's boundary values are ignored (Dirichlet u = 0).
 *   a  device [S][(a_n+1)^2] nodal coefficient, FP64 (a_prec = MLMC_FP64) or
 *      FP32 (MLMC_FP32); a_n = n or a multiple of n (the grid-n operator then
 *      uses every (a_n/n)-th node: a coarse view of a fine field)
 *   x, y  device [S][(n+1)^2], FP64 if vec_prec == MLMC_FP64 else FP32
 *   op_prec  storage of the coefficient inside the operator (MLMC_FP64 needs
 *      vec_prec FP64; FP32/BF16S/FP16S need vec_prec FP32)
 * Errors: MLMC_E_ARG for n < 2, S < 0, a_n % n != 0, inconsistent precisions. */
mlmc_status mlmc_apply_operator(int n, int S, const void* a, mlmc_prec a_prec, int a_n,
                                mlmc_prec op_prec, const void* x, void* y, mlmc_prec vec_prec,
                                void* stream);

/* ------------------------------------------------------------------------- */
/* A5 + A6 + A7: solve S independent systems A(a_s) x_s = b (b_i = f h^2) to
 * relative residual delta (Eq. (2.1) with C = 1; accuracy choice Eq. (4.12))
 * by iterative refinement (Alg. 2.1): r = b - A x in FP64 with the FP64
 * operator of the master coefficient; stop when ||r|| / ||b|| < delta; else
 * solve A d = r approximately with the inner Krylov method (CG or MINRES,
 * Sec. 2.2, preconditioned by the context's choice: a geometric multigrid
 * V-cycle by default, or Jacobi; mlmc_set_precond) in precision `prec`, and
 * x += d in FP64.  All S solves run in one kernel launch.  Then Q_s = G(u_s) (Problem 4.5; the QoI of
 * the context's problem).
 *   n      cells per side of the solve grid, 2 <= n <= 2048
 *   a      device master coefficient, S rows of (a_n+1)^2 nodes, FP64 or FP32 (a_prec)
 *   a_n    grid of `a`: n, or a multiple of n (coarse member of a level pair)
 *   a_ld   elements from one row of `a` to the next: 0 (dense, (a_n+1)^2) or at
 *          least (a_n+1)^2 (e.g. rows padded by mlmc_sample_fields)
 *   delta  target relative residual, > 0
 *   max_iters  inner-iteration budget per solve (summed over refinement steps)
 *   u      device FP64 [S][(n+1)^2] solution (dense nodal, zero boundary) or NULL
 *   Q      device FP64 [S] out
 *   iters  device int32 [S] inner iterations, or NULL
 *   relres device FP64 [S] final ||b - A x|| / ||b|| (FP64), or NULL
 *   flags  device int32 [S] MLMC_F_* bits, or NULL
 * Every system is solved start to finish by one group of threads (a CTA, a
 * quarter CTA or a warp, by grid size), all systems of the call in one launch.
 * Asynchronous: the call enqueues the solve on `stream` and returns; Q, u,
 * iters, relres and flags are valid once `stream` has been synchronised.
 * Per-solve failures are in `flags`; a bounded wait that ran out is reported
 * by the context's next synchronising call (mlmc_sync, mlmc_level_stats,
 * mlmc_estimate, mlmc_profile_get) as MLMC_E_TIMEOUT.  With profiling on
 * (mlmc_profile_enable) the call synchronises to read the launch's counters. */
mlmc_status mlmc_level_solve(mlmc_ctx* ctx, int n, int S, const void* a, mlmc_prec a_prec, int a_n,
                             int64_t a_ld, mlmc_prec prec, mlmc_solver solver, double delta, int max_iters,
                             double* u, double* Q, int32_t* iters, double* relres, int32_t* flags,
                             void* stream);

/* Wait for the work this context enqueued on `stream` and report what the
 * asynchronous calls could not: MLMC_E_TIMEOUT when a bounded device-side wait
 * of a synthesis or a solve ran out since the last synchronising call.
 * The calls of one context share its workspaces, so the work each call
 * enqueues starts on the device after the work of the context's previous call,
 * whatever stream either used. */
mlmc_status mlmc_sync(mlmc_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------- */
/* Allocation-free variant of mlmc_level_solve.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * a host application or plug-in framework that owns all device memory and
 * hands the library only its own buffers, or a serving loop that forbids
 * allocation after start-up (cudaMalloc can synchronise the device, and it
 * fails once a memory pool has reserved the device).  It solves like
 * mlmc_level_solve with the Jacobi preconditioner (same kernel and outputs)
 * but takes no context and calls no cudaMalloc, cudaFree or allocating library
 * routine, on the device or the host: the solver's scratch (vectors,
 * descriptors, error word) lives in one file-scope __device__ array of
 * MLMC_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits, and the descriptors are written there by a kernel.
 *   device  CUDA device to run on (made current for the call, then restored)
 *   n, S, a, a_prec, a_n, prec, delta, max_iters: as mlmc_level_solve (CG only)
 *   qoi, box, f: the QoI and right-hand side of mlmc_problem (box host [4], read
 *           only when qoi == 1)
 *   Q, iters, relres, flags: device outputs as in mlmc_level_solve (iters,
 *           relres, flags may be NULL)
 * Capacity: a batch needs about (24 + 4 p_v + 2 p_s) (n+1)(n+8) bytes per system
 * (p_v, p_s: vector and coefficient storage bytes) plus a few words;
 * a batch beyond MLMC_NOALLOC_SCRATCH_BYTES is rejected with MLMC_E_ARG and a
 * message in mlmc_last_error(NULL), as are the argument errors of
 * mlmc_level_solve and a QoI box that is not finite, ordered, inside the unit
 * square and on grid lines of the n-cell grid.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call uses the same
 * array and leaves its contents behind; the call clears what must start at
 * zero.  Calls whose work overlaps on the GPU (other threads or streams) race
 * on the array: issue them one after another.  Every call synchronises
 * `stream` and copies the kernel's error word to the host, so it cannot be
 * called while a stream is being captured. */
#define MLMC_NOALLOC_SCRATCH_BYTES (64ull << 20)
mlmc_status mlmc_level_solve_noalloc(int device, int n, int S, const void* a, mlmc_prec a_prec, int a_n,
                                     mlmc_prec prec, double delta, int max_iters, int qoi, const double* box,
                                     double f, double* Q, int32_t* iters, double* relres, int32_t* flags,
                                     void* stream);

/* ------------------------------------------------------------------------- */
/* A8: level statistics.  Y_s = Qf[s] - Qc[s] (Qc NULL at level 0), Eq. (4.1);
 * the batch's (n, mean, m2, Kahan sums) is computed on the device in a fixed
 * order and merged into *acc (host) with Chan's pairwise update.
 * Synchronises `stream`.  S = 0 leaves *acc unchanged. */
mlmc_status mlmc_level_stats(mlmc_ctx* ctx, int S, const double* Qf, const double* Qc,
                             mlmc_acc* acc, void* stream);

/* Host-side Chan merge of two accumulators: *into <- *into (+) *other. */
void mlmc_acc_merge(mlmc_acc* into, const mlmc_acc* other);

/* ------------------------------------------------------------------------- */
/* A9: the accuracy rule, Eq. (4.7): delta_l = (kp h_l^beta1)^(1/beta2) for
 * l < L and delta_L = min((kp h_L^beta1)^(1/beta2), (kp h_L^alpha1)^(1/alpha2));
 * for the P1 problem (alpha1, alpha2, beta1, beta2) = (2, 1, 4, 2), Eq. (4.12).
 * prec[l] is this library's choice of inner precision for accuracy delta_l on
 * grid h_l, from the conditions of Cor. 3.4 with kappa(A) ~ contrast h^-2
 * (Lemma 3.3): FP64 when contrast h^-2 u_single > 0.5 (condition 1 fails
 * for single); else FP16-stored coefficient (MLMC_FP16S) when delta_l >= 1e-4
 * (a refinement step then contracts the residual by ~u_half, so at most two
 * steps are needed); else FP32.  `contrast` <= 0 means 1.
 *   h      host [L+1] mesh sizes, decreasing, > 0
 *   delta  host [L+1] out;  prec host [L+1] out (may be NULL)
 * Pure host code (no GPU). */
mlmc_status mlmc_adapt_precision(int L, const double* h, double kp, double alpha1, double alpha2,
                                 double beta1, double beta2, double contrast,
                                 double* delta, mlmc_prec* prec);

/* ------------------------------------------------------------------------- */
/* A10 + A11: the estimate loop, Alg. 4.1, with every round's samples of all
 * levels solved in one resident-solve launch. */
typedef enum {
    MLMC_FORM_MIXED = 0,          /* per-level accuracy delta_l (Eq. (4.12)), per-level inner precision  */
    MLMC_FORM_FP64_ADAPTIVE = 1,  /* per-level delta_l, FP64 inner                                        */
    MLMC_FORM_FP64_FIXED = 2      /* standard MLMC: fixed accuracy fixed_delta on all levels, FP64         */
} mlmc_form;

typedef struct {
    double tol;            /* target RMSE TOL (variance budget TOL^2/2, bias test below)            */
    int L_start;           /* finest level of the first round: 1 = Alg. 4.1; L_max = fixed hierarchy */
    int N_init;            /* samples on a newly started level (Alg. 4.1, N_init), >= 2             */
    double kp;             /* k_p of Eq. (4.7), in (0, 1); the paper uses 0.05                       */
    double alpha1, alpha2, beta1, beta2;   /* rates of Lemma 4.6 (2, 1, 4, 2)                      */
    double alpha;          /* bias rate in the bias test (2)                                         */
    double gamma;          /* cost model C_l = m^(gamma l) (Alg. 4.1 "estimate C_l"), e.g. 2         */
    double r;              /* bias-test constant: |Y_hat_L| <= (r m^alpha - 1) TOL / sqrt(2), r = 1    */
    int form;              /* mlmc_form                                                              */
    double fixed_delta;    /* accuracy of MLMC_FORM_FP64_FIXED (e.g. 1e-10)                          */
    int force_prec;        /* -1: per-level rule of mlmc_adapt_precision; else an mlmc_prec for all  */
    int solver;            /* mlmc_solver                                                            */
    int max_iters;         /* inner-iteration budget per solve                                       */
    int max_rounds;        /* safety cap on Alg. 4.1 rounds                                          */
    const int64_t* fixed_N;/* non-NULL: no adaptivity, exactly fixed_N[l] samples on levels 0..L_start */
    double contrast;       /* contrast estimate for the precision rule (<= 0: 1)                     */
    int mixed_field;       /* master coefficient of the mixed form: MLMC_FP64TC (default; FP64 from
                              the tensor cores, as the FP64 refinement residual of Alg. 2.1 needs) or
                              MLMC_FP32 (the FP32 tensor-core field, about 1e-6 relative)            */
    int prec_rule;         /* inner precision of the mixed form's Krylov solves: 0 (default) the rule of
                              mlmc_adapt_precision with `contrast`; 1 calibrated: each level's contrast
                              is measured on its own fields (max over samples of max(a) / min(a),
                              which bounds kappa(A) / kappa(Laplacian), Lemma 3.3), FP64 where Cor. 3.4's
                              condition contrast h^-2 u_single <= 0.5 fails, and a 16-bit stored
                              coefficient IEEE half where a and D^-1 fit its normal range
                              (min a >= 6.2e-5, max a <= 4e3), else bfloat16                        */
    int chol_table;        /* Cholesky solver, mixed form: the per-level precisions (u_f u_s u u_r) of
                              Sec. 5.2.  0 (default): Table 1 (right), hhss on level 0, ssss on level 1,
                              ssdd above; 1: the quarter-precision setting, qhhh on level 0 and hhss
                              above.  The FP64 forms use dddd.                                        */
    const struct mlmc_result_s* resume;   /* checkpoint: NULL (fresh start) or the result of an
                              earlier adaptive estimate of the same problem and form (e.g. one stopped
                              by max_rounds, or saved to disk and read back).  The estimate continues
                              Alg. 4.1 from that state: its level accumulators, finest level and sample
                              counts (new samples take the next indices, so an interrupted and resumed
                              run draws exactly the samples of an uninterrupted one), its calibrated-
                              rule state and its counters.  tol, max_rounds and the budgets may differ.
                              Not with fixed_N.                                                       */
    const char* log_path;  /* NULL, or a file to which the estimate appends one JSON object per Alg. 4.1
                              round (one line each): round, L, samples and next targets per level,
                              level means and variances, delta_l, the current RMSE estimate, the bias
                              and sample-count tests, elapsed seconds                                   */
} mlmc_options;

typedef struct mlmc_result_s {
    double estimate;                 /* Q_hat = sum_l Y_hat_l (Eq. (4.1))                        */
    double rmse;                     /* sqrt(bias^2 + sum_l s_l^2 / N_l), bias = |Y_hat_L|/(m^alpha-1) */
    double var_est;                  /* sum_l s_l^2 / N_l                                          */
    int L;                           /* finest level used                                         */
    int rounds;                      /* Alg. 4.1 rounds                                           */
    int bias_failed;                 /* bias test still failing at L_max                          */
    int32_t flags_or;                /* OR of all per-solve flags                                 */
    int64_t N[MLMC_MAX_LEVELS];      /* samples per level                                         */
    double Yhat[MLMC_MAX_LEVELS];    /* level means                                               */
    double s2[MLMC_MAX_LEVELS];      /* level variances (1/N normalisation, Eq. (4.2))            */
    double delta[MLMC_MAX_LEVELS];   /* accuracy used per level (fine member)                     */
    int32_t prec[MLMC_MAX_LEVELS];   /* inner precision used per level                            */
    int64_t inner_iters[MLMC_MAX_LEVELS];   /* inner iterations summed over the level's solves    */
    int64_t dofs[MLMC_MAX_LEVELS];   /* unknowns solved per level (fine + coarse members)         */
    mlmc_acc acc[MLMC_MAX_LEVELS];   /* final level accumulators                                  */
    double seconds;                  /* wall time of the call                                     */
    int64_t fp64_retries[MLMC_MAX_LEVELS];  /* mixed form: solves re-run with FP64 inner arithmetic
                                               after their low-precision refinement stagnated or ran
                                               out of iterations (Cor. 3.4 conditions failed)     */
    double contrast[MLMC_MAX_LEVELS];       /* calibrated rule: measured contrast per level (else 0) */
    double a_min[MLMC_MAX_LEVELS];          /* calibrated rule: smallest and largest nodal coefficient */
    double a_max[MLMC_MAX_LEVELS];          /* seen per level (else 0); kept for a resumed estimate   */
} mlmc_result;

/* Fill *opts with the paper's defaults: kp 0.05, (2,1,4,2), alpha 2, gamma 2,
 * r 1, N_init 100, L_start 1, mixed form with an MLMC_FP64TC master field, CG,
 * fixed_delta 1e-10. */
void mlmc_default_options(mlmc_options* opts);

/* Run Alg. 4.1 on the GPU; synchronises; results in *res (host). */
mlmc_status mlmc_estimate(mlmc_ctx* ctx, const mlmc_options* opts, mlmc_result* res);

/* The same host loop with a caller-supplied level sampler instead of the GPU
 * (for testing the loop without a GPU).  sampler(user, level, first, count,
 * delta[L+1], Y[count]) fills Y with count samples of Y_level and returns 0
 * (non-zero aborts with MLMC_E_ARG).  The cost model is m^(gamma l). */
typedef int (*mlmc_sampler_fn)(void* user, int level, int64_t first, int count,
                               const double* delta, double* Y);
mlmc_status mlmc_estimate_host(int m, int L_max, int n0, const mlmc_options* opts,
                               mlmc_sampler_fn sampler, void* user, mlmc_result* res);

/* ------------------------------------------------------------------------- */
/* A12: dQ/dxi for S samples on level grid `level` (QoI of the context).
 * Field from xi (device FP64 [S][K]); the forward solve A x = b and the
 * adjoint solve A lambda = g (g_i = G(phi_i)) run together in one resident-solve
 * launch, to accuracy delta in precision prec; then
 * G_v = -(1/3) sum_{T contains v} |T| grad(lambda_h).grad(u_h)|_T and
 * dQ/dxi[s][k] = sum_v Phi_k(x_v) a_v G_v (the transposed KL contraction).
 * u is recomputed here rather than kept from an earlier forward pass (the
 * autograd wrapper's forward stores only Q).  The field is FP64: from the FP64
 * contraction when prec == MLMC_FP64, else from the tensor-core contraction
 * (MLMC_FP64TC of mlmc_sample_fields).
 *   Q      device FP64 [S] out;  dQdxi  device FP64 [S][K] out
 * Asynchronous like mlmc_level_solve: results are valid once `stream` has been
 * synchronised. */
mlmc_status mlmc_adjoint_grad(mlmc_ctx* ctx, int level, int S, const double* xi, mlmc_prec prec,
                              double delta, int max_iters, double* Q, double* dQdxi, void* stream);

/* ------------------------------------------------------------------------- */
/* Preconditioner of this context's inner solves, CG and MINRES (mlmc_level_solve,
 * mlmc_estimate, mlmc_adjoint_grad).
 *  - MLMC_PC_JACOBI: z = D^-1 r.
 *  - MLMC_PC_MG (default): one geometric multigrid V-cycle, the optimal solver
 *    that the cost model of Sec. 4 assumes (cost per sample proportional to the
 *    unknowns).  Coarse grids n/2, n/4, ... while even and at least 4 cells, the
 *    nodal coefficient injected at the coarse nodes and the P1 operator
 *    re-discretised on it; P1 interpolation on the SW-NE triangulation and its
 *    transpose; nu damped-Jacobi sweeps (damping omega) before and after the
 *    coarse correction; coarse_sweeps Jacobi sweeps on the coarsest grid.  The
 *    V-cycle is a fixed symmetric positive definite linear map, so CG stays
 *    CG and MINRES stays preconditioned MINRES.
 * nu in {1, 2}, coarse_sweeps even and >= 2, 0 < omega < 1; 0 keeps the current
 * value (defaults nu = 1, coarse_sweeps = 8, omega = 0.8).  Stopping is still
 * on the FP64 residual of the refinement (Alg. 2.1). */
mlmc_status mlmc_set_precond(mlmc_ctx* ctx, mlmc_precond pc, int nu, int coarse_sweeps, double omega);

/* Multigrid hierarchy depth: grids are halved while even and the half keeps at
 * least min_cells cells (2..64; default 4), so the coarsest grid has between
 * min_cells and 2 min_cells - 1 cells (or is the solve grid itself). */
mlmc_status mlmc_set_mg_coarsest(mlmc_ctx* ctx, int min_cells);

/* Full-multigrid start of multigrid-preconditioned CG (on = 1, the default; 0
 * off).  The first inner solve of a refinement (Alg. 2.1: x = 0, r = b) starts
 * from the nested-iteration guess instead of zero: r restricted down the
 * V-cycle's hierarchy, the coarsest grid smoothed, and on each finer grid the
 * prolonged coarser solution improved by one V-cycle.  The inner tolerance and
 * the FP64 stopping test are unchanged; MINRES and Jacobi-CG start from zero. */
mlmc_status mlmc_set_full_multigrid(mlmc_ctx* ctx, int on);

/* Working precision u (of the iterate x) and residual precision u_r of the
 * refinement of this context's Cholesky solves (MLMC_CHOLESKY): (u, u_r) one of
 * (MLMC_FP64, MLMC_FP64) (default), (MLMC_FP32, MLMC_FP64), (MLMC_FP32,
 * MLMC_FP32) or (MLMC_FP16S, MLMC_FP16S) (x and the residual stored in IEEE
 * half, formed in FP32).  With the factor precision `prec` of mlmc_level_solve
 * (MLMC_FP8S, MLMC_FP16S, MLMC_BF16S, MLMC_FP32 or MLMC_FP64) they form the
 * quadruple (u_f, u_s = u_f, u, u_r) of Sec. 5.2, e.g. (half, half, single,
 * single) for `hhss`.  mlmc_estimate with the Cholesky solver sets these per
 * level itself (mlmc_options.chol_table). */
mlmc_status mlmc_set_cholesky_precision(mlmc_ctx* ctx, mlmc_prec u, mlmc_prec u_r);

/* Inner tolerance of the refinement (Alg. 2.1) for this context's solves: each
 * inner solve stops at ||r_k|| <= tau ||r_0|| with tau = clamp(theta delta /
 * rho, tau_min, 0.5), rho the current relative residual.  theta = 0 keeps the
 * current value (default 0.3); tau_min <= 0 restores the per-precision floor
 * (1e-14 FP64, 1e-6 FP32, 1e-3 BF16 storage, 1e-4 FP16 storage), the accuracy
 * an inner solve in that precision can be relied on to reach.  Stopping and
 * the result are always judged on the FP64 residual. */
mlmc_status mlmc_set_inner_tolerance(mlmc_ctx* ctx, double theta, double tau_min);

/* A11: launch-setting autotuner of this context's resident solves (off by
 * default).  When on, the first launch of each new launch shape -- inner
 * precision, solver, preconditioner, and the batch's grid sizes with their
 * system counts rounded down to powers of two -- is solved once per candidate
 * setting, changing one setting at a time from the library's own rules:
 *   - the group size of n = 91..128 systems (mlmc_debug_set_medium_items);
 *   - the row-pipeline depth of Jacobi-preconditioned CG (0, 2, 4 slots);
 *   - the V-cycle's coarsest grid (4 or 16 sweeps on it, or one halving less
 *     with 16; mlmc_set_mg_coarsest), its smoother damping (0.7, 0.9), the
 *     deepest coarse grid kept in shared memory (32 cells) and its smoothing
 *     sweeps (1, 2);
 *   - the inner tolerance factor theta (0.1, 0.3, 0.6) and its floor tau_min
 *     (0.3, 1 or 3 times the precision's default, unless the context sets one;
 *     mlmc_set_inner_tolerance).
 * Each candidate is timed twice with CUDA events; a change is kept when at
 * least 1% faster, and the fastest setting is cached in the context for the
 * shape.  Every candidate solves the same systems to the same delta, so
 * results agree to the solve tolerance whatever is chosen.  A launch that
 * tunes synchronises its stream (mlmc_level_solve included). */
mlmc_status mlmc_set_autotune(mlmc_ctx* ctx, int on);

/* Samples solved ahead in mlmc_estimate (on = 1, the default; 0 off).  A round
 * of Alg. 4.1 also solves, on each of its levels that the last estimate on
 * this context took further, the next samples up to 1.25 times the count that
 * level ended with there, as long as they add at most a tenth of the round's
 * unknowns; they run beside the round's
 * own solves, on SMs the finest level's few large systems leave idle.  If the
 * next round asks for them (same delta and precision class), it takes their
 * QoIs, iteration counts and flags instead of solving again.  The result does
 * not depend on it: a sample's field and solve do not depend on the batch it is
 * solved in (with the autotuner off; with it on, each launch shape's chosen
 * settings apply, as for any batch), the level statistics are taken over
 * exactly the samples each round asks for, and every counter of a sample counts
 * in the round that asks for it.  Levels with a member whose thread-group size
 * follows the rest of its launch (91 <= n <= 128) are not solved ahead,
 * nor is anything with fixed_N or under the calibrated precision rule. */
mlmc_status mlmc_set_sample_ahead(mlmc_ctx* ctx, int on);
typedef struct {
    char shape[192];       /* the launch shape, as text                                        */
    int prec, solver, precond;
    int med_items, ring, nu;   /* chosen settings; -3 (and nu 0) means the context's own rule    */
    int mg_min, mg_coarse; /* chosen coarsening bound and coarsest-grid sweeps; 0: the context's  */
    double mg_omega;       /* chosen smoother damping; 0: the context's                           */
    int mg_smem;           /* largest coarse grid kept in shared memory; 0: the library's rule (64) */
    double theta;          /* chosen inner tolerance factor; 0 means the context's (0.3)       */
    double tau_min;        /* chosen floor of the inner tolerance; < 0 means the precision's    */
    double best_ms, default_ms;   /* launch time with the chosen and with the default settings */
    int trials;            /* timed trial launches                                              */
} mlmc_tune_entry;
int mlmc_autotune_count(const mlmc_ctx* ctx);                  /* shapes tuned so far */
mlmc_status mlmc_autotune_entry(const mlmc_ctx* ctx, int i, mlmc_tune_entry* out);   /* in tuning order */

/* Diagnostics.  Timeout of every bounded device-side wait of this context, in
 * seconds (default 10): the tensor-core synthesis waits on its TMA copies and
 * MMAs, and the large CG solves wait on the bulk row copies of their pipeline.
 * Used to test the MLMC_E_TIMEOUT path. */
mlmc_status mlmc_set_wait_timeout(mlmc_ctx* ctx, double seconds);

/* Measurement.  With profiling on, the context records CUDA events on the
 * launching stream around every resident solve and tensor-core synthesis
 * launch and, after each solve, derives the launch's algorithmic bytes from
 * the per-system inner-iteration and refinement counts:
 *   per unknown and inner iteration 8 p_v + 2 p_s bytes with Jacobi (plus p_s
 *   for its inverse diagonal; p_v vector bytes, p_s coefficient storage bytes),
 *   or that plus the V-cycle's bytes with multigrid; per unknown and
 *   refinement step (residual from x and the FP64 edge weights, update)
 *   40 + 3 p_v bytes; plus 24 + p_m + p_s bytes per unknown for set-up and
 *   the QoI (p_m master coefficient bytes).
 * The synthesis counts its FP32 output (4 bytes per node and sample) plus one
 * read of both split operands, and 3 x 2 S_pad K_pad N_pad executed tensor
 * FLOPs (three MMAs per split product).  Event times are resolved lazily. */
typedef struct {
    int64_t solve_launches;
    double solve_ms;           /* summed event time of the resident-solve launches */
    double solve_bytes;        /* their algorithmic bytes */
    int64_t inner_iters;       /* inner iterations summed over systems */
    int64_t unknown_iters;     /* sum over systems of interior unknowns x inner iterations */
    int64_t kl_launches;
    double kl_ms, kl_bytes, kl_flops;
    int64_t h2d_bytes, d2h_bytes;  /* host<->device bytes moved by this context's calls */
    double solve_busy_ms;      /* union of the resident-solve launches' intervals on the device timeline
                                  (launches on concurrent streams counted once), since profiling was
                                  switched on or reset */
    double solve_flops;        /* arithmetic operations of the resident solves, counted per unknown as
                                  the kernels execute them: a stencil point 28 (nodal coefficient) or 12
                                  (stored FP64 edge weights); per inner iteration two stencil sweeps with
                                  their recurrences and dots, plus the V-cycle with multigrid; per
                                  refinement step the FP64 residual and its dots (20) and the update;
                                  set-up (edge weights, inverse diagonal) and the QoI */
    double chol_bits;          /* Cholesky solves: the memory cost model of Sec. 5.2 -- bits of every
                                  entry computed and stored while solving: the factor's nonzeros
                                  (N (bw+1) - bw (bw+1)/2, bw = n - 1) in u_f, x_0 in u, each residual in
                                  u_r, each correction and update in u */
} mlmc_profile;
mlmc_status mlmc_profile_enable(mlmc_ctx* ctx, int on);
mlmc_status mlmc_profile_get(mlmc_ctx* ctx, mlmc_profile* out);   /* synchronises the device */
mlmc_status mlmc_profile_reset(mlmc_ctx* ctx);

/* Diagnostics.  Make every bounded wait of this context's tensor-core KL
 * synthesis, and the first row-copy wait of each team of a large CG solve,
 * expect 16 * extra bytes that never arrive (extra = 0 restores normal
 * operation), so that the wait runs out after the timeout.  The synthesis then
 * records MLMC_E_TIMEOUT in its error word, waits (bounded) for its own copies,
 * frees its tensor memory and returns; the next synchronising call of the
 * context (mlmc_level_solve, mlmc_level_stats, mlmc_estimate,
 * mlmc_adjoint_grad, mlmc_profile_get) returns MLMC_E_TIMEOUT.  The solve stops
 * at its next reduction, flags the system MLMC_F_TIMEOUT, waits (bounded) for
 * its copies in flight, and mlmc_level_solve returns MLMC_E_TIMEOUT.  Exists
 * only to test those paths; the GPU stays usable. */
mlmc_status mlmc_debug_set_wait_extra(mlmc_ctx* ctx, int extra);

/* Diagnostics.  Slots per team of the row pipeline of this context's large CG
 * solves (n >= 91, one 512-thread CTA per system; used for grids whose rows
 * are a multiple of 128 cells wide).  -1 chooses automatically (default): the
 * deepest of 4..2 that fits shared memory when the launch has at least one
 * system of its largest size per SM and the solve is Jacobi-preconditioned,
 * else none (the multigrid V-cycle uses that shared memory for its coarse
 * levels).  0 turns the pipeline off (rows are read with
 * plain cached loads); 2..4 cap the depth.  The arithmetic is the same either
 * way, so results are bit-identical; exists to measure the pipeline and to test
 * that identity. */
mlmc_status mlmc_debug_set_solve_ring(mlmc_ctx* ctx, int ring);

/* Diagnostics: forced allocation failure (process-wide).  With after >= 0 the
 * library's (after+1)-th next device allocation fails as if the device were out
 * of memory, once; after = -1 disarms.  The failing call returns MLMC_E_NOMEM
 * with the allocation named in mlmc_last_error, the context stays usable, and
 * the next call allocates afresh.  The allocation-free entry point never
 * allocates and is unaffected. */
mlmc_status mlmc_debug_fail_allocation(int64_t after);

/* Diagnostics.  Group size of this context's solves: a system of n cells has
 * (n - 1) ((n - 1)/4 + 1) four-node chunks; up to 512 chunks it is solved by
 * one warp, up to `items` chunks by a 128-thread quarter of a CTA (four
 * systems per CTA), above that by a whole 512-thread CTA.  -1 (default)
 * chooses per launch: 4096 (n = 91..128 in quarters) when the launch also
 * holds systems at least twice their size and those systems plus the
 * mid-size quarters need no more CTAs than the GPU has SMs, else 2048
 * (n <= 90 in quarters).  Reduction orders follow the group size, so results
 * agree to the solve tolerance, not bit for bit.
 * Errors: MLMC_E_ARG unless items is -1 or 512 <= items <= 16384 (n <= 256). */
mlmc_status mlmc_debug_set_medium_items(mlmc_ctx* ctx, int items);

#ifdef __cplusplus
}
#endif
#endif /* LIBMLMC_H */
