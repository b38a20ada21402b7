/*
 * glm_sur.h -- C ABI of the GB300 (sm_103a) library for GLS estimation of
 * Seemingly Unrelated Regressions (SUR) models by PCG-Aug.
 *
 * The method (Foschi, "Preconditioned Conjugate Gradient methods for the
 * estimation of General Linear Models"):
 *   SUR model (Sec. 1, eq. SURdefs):  y = vec(Y),  X = (+)_i X_i (M x n_i blocks),
 *                                      Sigma = Omega (x) I_M,  Omega G x G, PSD.
 *   GLS as the augmented system eq. (aug1):  [Sigma X; X^T 0][w; b] = [y; 0].
 *   Solved by Algorithm glmpcg2 (PCG-Aug) with the indefinite preconditioner
 *   eq. (invprec) and D = I (Sec. 4.3): every step applies Sigma as U * Omega
 *   and the per-block OLS projection Pi_i = I - Q_i Q_i^T from a Householder
 *   QR X_i = Q_i R_i computed once; the estimate is z = X*^T (y - Sigma w)
 *   with X*^T xi = vec(R_i^-1 Q_i^T xi_i).
 *
 * Conventions common to every entry point
 *   - All matrix arguments are DEVICE pointers to float64 data in column-major
 *     order unless stated otherwise; the caller owns them and they need only be
 *     valid for the duration of the call (work is stream-ordered: "the call"
 *     ends when the stream reaches it).  Outputs are written into caller
 *     buffers.  The handle owns every other allocation.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is asynchronous with respect to the host except where noted.
 *   - The return value reports host-side validation, allocation and launch
 *     errors.  Conditions found on the device (rank deficiency, breakdown,
 *     stagnation, non-convergence, non-finite data) are written to the
 *     per-right-hand-side status array and read with glm_sur_get_status.
 *   - No exception crosses the ABI.  A handle must not be used from two host
 *     threads at once; different handles are independent.
 */
#ifndef GLM_SUR_H
#define GLM_SUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* glm_sur_stream_t;   /* == cudaStream_t */

typedef struct glm_sur_ctx* glm_sur_t;          /* opaque handle */

typedef enum {
  GLM_SUR_OK = 0,
  GLM_SUR_INVALID_ARG = 1,     /* bad size, null pointer, unsupported option      */
  GLM_SUR_RANK_DEFICIENT = 2,  /* some X_i not of full column rank (|R_jj| tiny)   */
  GLM_SUR_BREAKDOWN = 3,       /* d_i = u^T Sigma u <= 0 or not finite (Sec. 2)    */
  GLM_SUR_STAGNATED = 4,       /* c_i = r^T Pi r stopped decreasing (Sec. 3.2)     */
  GLM_SUR_NOT_CONVERGED = 5,   /* maxit reached                                    */
  GLM_SUR_TIMEOUT = 6,         /* a bounded device wait gave up                    */
  GLM_SUR_NONFINITE = 7,       /* NaN/Inf in inputs                                */
  GLM_SUR_OOM = 8,             /* device allocation failed                         */
  GLM_SUR_CUDA_ERROR = 9       /* a CUDA runtime call failed                       */
} glm_sur_status;

enum {
  GLM_SUR_PREC_FP64 = 0,          /* every step in float64                          */
  GLM_SUR_PREC_FP32_REFINE = 1    /* float32 bulk iterations inside a float64
                                     iterative-refinement loop                     */
};

typedef struct {
  int precision;          /* GLM_SUR_PREC_*                                         */
  double tol;             /* stop a column when sqrt(c_i / c_1) <= tol              */
  int maxit;              /* iteration cap of one PCG run (<= 0: m - n + 1)         */
  int stagnation_window;  /* W: stagnated if c has no new minimum for W steps (0: off) */
  double inner_tol;       /* FP32_REFINE: relative reduction per inner solve        */
  int max_refine;         /* FP32_REFINE: cap on outer (refinement) steps           */
  int chunk;              /* iterations per captured CUDA graph launch (even, >= 2) */
  double inner_shift;     /* FP32_REFINE: the inner solves use Omega + s I with
                             s = inner_shift * max_i omega_ii (0 disables); the
                             float64 residual always uses Omega itself        */
  int reduce_rows;        /* setup only: 1 = solve the row-reduced model of Remark
                             rem:reduction (M' = n rows), when M >= 2 n,
                             n <= 2048 and W = [X_1 ... X_G] has full column
                             rank (otherwise the model is kept whole).  On a
                             reduced handle the residual is the reduced
                             system's (responses Q^T y_i), and tol and relres
                             are relative to the M-row model's ||P y||, whose
                             square is the reduced ||P' y'||^2 plus the
                             energy of y outside range(W) (taken as it is
                             scaled by a preconditioner block).  The
                             adjoint solve and PCG-NE need no such term    */
  int step_kernels;       /* GLM_SUR_STEP_*: kernels of the float32 bulk steps   */
  int precond;            /* GLM_SUR_PRECOND_*: the block D of the preconditioner
                             of eq. (invprec), D = D0 (x) I_M               */
  int algorithm;          /* GLM_SUR_ALG_*: Algorithm glmpcg2 or glmpcg3      */
} glm_sur_opts;

enum {
  GLM_SUR_ALG_GLMPCG2 = 0,  /* Algorithm glmpcg2 (default): u_{i+1} = Pi r_{i+1}
                               + mu_i u_i, run in the reduced form of eq. (urwProj) */
  GLM_SUR_ALG_GLMPCG3 = 1   /* Algorithm glmpcg3: the direction s_{i+1} = r_{i+1}
                               + mu_i s_i is carried unprojected and u_i = Pi s_i
                               is recomputed every step (two more passes over Q
                               per step); w_{i+1} = w_i - lambda_i u_i, r_{i+1} =
                               r_i - lambda_i (Sigma u_i + X X*^T s_i) with
                               X X*^T s = s - Pi s.  Float64 only, no
                               restrictions (GLM_SUR_INVALID_ARG otherwise); a
                               column stops at tol, on breakdown or at maxit
                               (no stagnation window).                     */
};

enum {
  GLM_SUR_PRECOND_IDENTITY = 0,  /* D = I (Sec. 4.3)                             */
  GLM_SUR_PRECOND_SCALED = 1,    /* D = alpha I, alpha = max_i omega_ii          */
  GLM_SUR_PRECOND_DIAG = 2       /* D = diag(Sigma) = diag(Omega) (x) I_M (the two
                                    choices of the VAR experiments).  With D0 =
                                    diag(delta), PCG-Aug with D runs the iterates
                                    of PCG-Aug with D = I on the row-scaled model
                                    (y_i, X_i divided by sqrt(delta_i), Omega by
                                    sqrt(delta_a delta_b)); solves run that model
                                    and return the same b.  relres refers to it;
                                    a delta_i <= 0 is taken as 1.  Not with
                                    restrictions (GLM_SUR_INVALID_ARG).
                                    glm_sur_get_w and glm_sur_backward map back
                                    to the given model: w = S w~, dL/dy = S
                                    dL/dy~, dL/dOmega = D0^-1/2 dL/dOmega~
                                    D0^-1/2 (S = D0^-1/2 (x) I_M; b does not
                                    depend on D0).                              */
};

enum {
  GLM_SUR_STEP_AUTO = 0,  /* fused two-pass step with the Sigma-apply on the
                             tensor cores (tcgen05, three tf32 products) when
                             k is 8 or 16, G <= 64, n_i <= 32 and
                             sum_i 4 ceil(n_i / 4) <= 2048; otherwise SIMT */
  GLM_SUR_STEP_SIMT = 1   /* four launches per step, Sigma-apply on the FP32
                             FMA pipe                                        */
};

/* Default options: FP64, tol 1e-13, maxit m-n+1, W = 25, inner_tol 1e-5,
 * max_refine 8, chunk 16, inner_shift 0, reduce_rows 0, step_kernels AUTO,
 * algorithm GLMPCG2,
 * precond IDENTITY.  A column that stops without
 * converging (stagnation, breakdown, maxit) returns its best saved iterate:
 * w is saved whenever c falls below a quarter of the c of the previous save. */
void glm_sur_default_opts(glm_sur_opts* opts);

/*
 * glm_sur_setup -- factor the regressors once (Sec. 3.2: the factorisations
 * the preconditioner needs do not change between steps; Sec. 4.3: X_i = Q_i R_i).
 *
 *   out    : receives the new handle (host pointer).
 *   G      : number of equations, 1 <= G <= 1024.  Solves need G <= 156:
 *            they stage Omega (G x ceil4(G) float64) in shared memory, and
 *            glm_sur_solve returns GLM_SUR_INVALID_ARG for a larger G.
 *   M      : observations per equation (>= max n_i).
 *   n_i    : HOST array of G block widths, 1 <= n_i <= 64.
 *   X      : DEVICE, M x n column-major with leading dimension ldx >= M,
 *            n = sum n_i; columns offs_i .. offs_i + n_i - 1 hold X_i
 *            (i.e. X = [X_1 ... X_G] = W of Remark rem:reduction).
 *   Omega  : DEVICE, G x G symmetric positive semi-definite (Sec. 1).
 *   opts   : HOST, may be NULL for defaults.
 * The handle keeps Q_i (explicit thin factor, M x n_i), R_i and Omega.
 * Errors: INVALID_ARG on bad sizes; OOM; CUDA_ERROR.  Rank deficiency of an
 * X_i is detected on the device and reported by glm_sur_get_setup_status.
 */
glm_sur_status glm_sur_setup(glm_sur_t* out, int G, int64_t M, const int* n_i,
                             const double* X, int64_t ldx, const double* Omega,
                             const glm_sur_opts* opts, glm_sur_stream_t stream);

/* Synchronises the handle's last setup and returns GLM_SUR_OK or
 * GLM_SUR_RANK_DEFICIENT (a block with |R_jj| <= n_i * eps * max|R|). */
glm_sur_status glm_sur_get_setup_status(glm_sur_t h);

/* Replace Omega (DEVICE, G x G) without refactoring X (Sec. 4.3: the QRs
 * depend on X only). */
glm_sur_status glm_sur_set_omega(glm_sur_t h, const double* Omega, glm_sur_stream_t stream);

/* Replace the options used by later solves. */
glm_sur_status glm_sur_set_opts(glm_sur_t h, const glm_sur_opts* opts);

/*
 * glm_sur_solve -- Algorithm glmpcg2 (PCG-Aug) with D = I, one independent PCG
 * per right-hand side, started at w_1 = 0, z_1 = 0; returns
 * b = z_hat = X*^T (y - Sigma w) (step 10 of the algorithm).
 *
 *   Y      : DEVICE, m x k column-major (m = G*M), column j = vec(Y_j),
 *            leading dimension ldy >= m.
 *   k      : number of right-hand sides, 1 <= k <= 64.
 *   b      : DEVICE output, n x k column-major, leading dimension ldb >= n.
 *   iters  : DEVICE output (nullable), k ints: PCG steps taken per column
 *            (summed over inner solves for FP32_REFINE).
 *   relres : DEVICE output (nullable), k doubles: final sqrt(c/c_1) per column
 *            (FP32_REFINE: the float64 true residual ||P(y - Sigma w)|| / ||P y||).
 * The final w (float64, m x k) stays in the handle for glm_sur_backward.
 * FP32_REFINE synchronises the stream once per refinement step.
 */
glm_sur_status glm_sur_solve(glm_sur_t h, const double* Y, int64_t ldy, int k,
                             double* b, int64_t ldb, int* iters, double* relres,
                             glm_sur_stream_t stream);

/*
 * glm_sur_set_restrictions -- linear restrictions C b = d on the parameters
 * (Sec. 4.1): the model becomes the GLM of eq. (RGLM1setup) with
 * Sigma_aug = diag(Omega (x) I_M, 0), X_aug = [(+)X_i; C], y_aug = [y; d],
 * and the preconditioner of eq. (invprec) with D = I, whose X* and Pi are
 * those of eq. (rglm1m): N = X_aug^T X_aug = (+)R_i^T R_i + C^T C is formed
 * and inverted once here (float64 Cholesky).
 *   C  : DEVICE, kc x n column-major, ldc >= kc (copied).  kc = 0 removes
 *        the restrictions.  n <= 25600.
 * A singular N (the restrictions and the X_i do not determine b) is reported
 * by glm_sur_get_setup_status as GLM_SUR_RANK_DEFICIENT.  Restricted solves
 * run in float64 (FP32_REFINE returns GLM_SUR_INVALID_ARG).
 */
glm_sur_status glm_sur_set_restrictions(glm_sur_t h, const double* C, int64_t ldc, int kc,
                                        glm_sur_stream_t stream);

/*
 * glm_sur_solve_restricted -- glm_sur_solve for a handle with restrictions:
 * Algorithm glmpcg2 on the restricted GLM (at most m + kc - n + 1 steps in
 * exact arithmetic, Sec. 4.1), b = X*^T (y_aug - Sigma_aug w).
 *   d  : DEVICE, kc x k column-major, ldd >= kc; NULL means d = 0.
 * Other arguments as glm_sur_solve.  (glm_sur_solve on a restricted handle
 * solves with d = 0.)
 */
glm_sur_status glm_sur_solve_restricted(glm_sur_t h, const double* Y, int64_t ldy, const double* d,
                                        int64_t ldd, int k, double* b, int64_t ldb, int* iters,
                                        double* relres, glm_sur_stream_t stream);

/*
 * glm_sur_mvrglm_setup -- the restricted multivariate GLM of Sec.
 * "Multivariate linear models with parameters restrictions" (MVRGLM):
 * Y = Z0 B + U (Y, U: M x G; B: N x G), vec(U) ~ (0, Omega0 (x) I_M), with
 * k_i linear restrictions C_i b_i = gamma_i on column i of B (no
 * cross-equation restrictions).  Setup factors Z0 = Q0 R0 (model reduction,
 * M rows -> N) and, for every equation, the updating QRD [R0; C_i] =
 * Qt_i R_i (eq. MvRGLMQRi); each step of Algorithm glmpcg2 then applies
 * Qt_i, Qt_i^T and R_i^-T with Sigma = Omega0 (x) I_N on the reduced rows and
 * 0 on the restriction rows (eq. RGLM1setup).  At most sum_i k_i + 1 steps in
 * exact arithmetic (m + k - n + 1 with m = n = G N).
 *   Z0     : DEVICE, M x N column-major, ldz >= M; full column rank
 *            (GLM_SUR_RANK_DEFICIENT otherwise, GLM_SUR_NONFINITE for a
 *            NaN / Inf entry).  1 <= N <= 64, M >= N.
 *   Omega0 : DEVICE, G x G (symmetric; positive definite on the null space
 *            of the restricted regressors).
 *   k_i    : HOST, G counts, 0 <= k_i <= N.
 *   C      : DEVICE, (sum k_i) x N column-major, ldc >= sum k_i: rows
 *            k_1 + ... + k_{i-1} .. + k_i - 1 hold C_i (full row rank each);
 *            NULL when every k_i is 0.
 *   opts   : as glm_sur_setup (reduce_rows is ignored: the model reduction
 *            is always applied); precond D0 = alpha I or diag(Omega0) scales
 *            every row of equation i, the restriction rows included (D_C of
 *            eq. (3) = delta_i I).
 * Solves: glm_sur_solve (gamma = 0, e.g. exclusion restrictions) and
 * glm_sur_solve_restricted with d = gamma ((sum k_i) x k column-major, ldd >=
 * sum k_i), Y in the layout of glm_sur_solve (column j = vec(Y_j), ldy >=
 * G M), b = vec(B) (G N x k, ldb >= G N).  glm_sur_set_omega,
 * glm_sur_set_opts and glm_sur_get_status apply; glm_sur_backward,
 * glm_sur_solve_ne, glm_sur_set_restrictions, glm_sur_get_w and
 * glm_sur_get_factors return GLM_SUR_INVALID_ARG.  Release with
 * glm_sur_destroy.
 */
glm_sur_status glm_sur_mvrglm_setup(glm_sur_t* out, int G, int64_t M, int N, const double* Z0, int64_t ldz,
                                    const double* Omega0, const int* k_i, const double* C, int64_t ldc,
                                    const glm_sur_opts* opts, glm_sur_stream_t stream);

/*
 * glm_sur_solve_ne -- PCG-NE, the comparator of the paper's Monte-Carlo study
 * (Sec. "Statistical properties of the PCG-Aug estimator") and experiments
 * (Sec. "Experimental Tests"): the conjugate gradient method of Algorithm pcg
 * with K = I on the normal equations (X^T Sigma^-1 X) beta = X^T Sigma^-1 y,
 * beta_1 = 0, in float64 whatever opts.precision says.  X = (+) Q_i R_i is
 * applied through the setup factors and Sigma^-1 = Omega^-1 (x) I_M, with
 * Omega^-1 from a Cholesky factorisation of the handle's Omega (the
 * preconditioner block opts.precond does not apply: PCG-NE has none).  A
 * column stops when ||f_i|| <= opts.tol ||f_1|| (f = A beta - h, the
 * gradient of Algorithm pcg) with status GLM_SUR_OK, or after opts.maxit
 * steps (0: 4 n) with GLM_SUR_NOT_CONVERGED; a non-positive p^T A p gives
 * GLM_SUR_BREAKDOWN.  In exact arithmetic it ends within n steps; on an
 * ill-conditioned X^T Sigma^-1 X it needs many more (the paper's point).
 * Arguments as glm_sur_solve; iters and relres (= ||f|| / ||f_1||) per
 * column; glm_sur_get_status reports the columns.  Row-reduced handles
 * (opts.reduce_rows) run it on the reduced model.
 * GLM_SUR_INVALID_ARG: Omega not numerically positive definite (a pivot of
 * its Cholesky factorisation below 1e-13 of its largest diagonal entry; the
 * normal equations need Sigma^-1), a handle with restrictions, or bad sizes.
 * glm_sur_get_w and glm_sur_backward are refused until the next glm_sur_solve.
 */
glm_sur_status glm_sur_solve_ne(glm_sur_t h, const double* Y, int64_t ldy, int k, double* b, int64_t ldb,
                                int* iters, double* relres, glm_sur_stream_t stream);

/*
 * glm_sur_backward -- adjoint of the last glm_sur_solve for a loss L(b).
 * K = [[Sigma, X], [X^T, 0]] of eq. (aug1) is symmetric, so with
 * (lam; mu) = K^-1 (0; dL/db):  dL/dy = lam  and  dL/dK = -(lam; mu)(w; b)^T,
 * whose Sigma part gives dL/domega_ab = -sum_t Lam[t, a] W[t, b] (M x G
 * matrices of lam and of the forward w, summed over the k right-hand sides).
 * lam = lam_1 + lam_2: lam_1 = Q_i R_i^-T (dL/db)_i meets X^T lam_1 = dL/db,
 * and lam_2 is the w of eq. (aug1) for y' = -Sigma lam_1, found by the same
 * PCG-Aug iteration (Algorithm glmpcg2) and precision as the forward solve.
 * Only the forward's converged w is needed: no iterate is stored.
 *   dL_db     : DEVICE, n x k column-major, ldg >= n.
 *   dL_dY     : DEVICE output (nullable), m x k column-major, ldy >= m:
 *               dL/dy per right-hand side, same layout as Y of glm_sur_solve.
 *   dL_dOmega : DEVICE output (nullable), G x G column-major, ldo >= G:
 *               (G_Omega + G_Omega^T) / 2, the gradient with respect to a
 *               symmetric Omega, summed over the right-hand sides.
 *   iters, relres : DEVICE outputs (nullable, k): of the adjoint solve.
 * k must equal the k of the last solve; the handle must have no
 * restrictions, and neither Omega nor the precision or stagnation window
 * may have changed since that solve (GLM_SUR_INVALID_ARG otherwise).  Afterwards glm_sur_get_status reports the
 * adjoint solve, and glm_sur_get_w still returns the forward w, so the call
 * may be repeated with another dL/db.
 */
glm_sur_status glm_sur_backward(glm_sur_t h, const double* dL_db, int64_t ldg, int k, double* dL_dY,
                                int64_t ldy, double* dL_dOmega, int64_t ldo, int* iters, double* relres,
                                glm_sur_stream_t stream);

/* Synchronises and copies the per-column status of the last solve (k values,
 * glm_sur_status codes) into the HOST array `status`. */
glm_sur_status glm_sur_get_status(glm_sur_t h, int* status, int k);

/* Copies the float64 w of the last solve (m x k column-major, DEVICE, ldw >= m)
 * into a caller buffer; Sigma w is the GLM residual of eq. (aug1).
 * GLM_SUR_INVALID_ARG on a handle set up with reduce_rows (w of the rows
 * outside range(W) is not formed). */
glm_sur_status glm_sur_get_w(glm_sur_t h, double* w, int64_t ldw, glm_sur_stream_t stream);

/* Copies the factors of glm_sur_setup into caller buffers (both DEVICE):
 * Q (M x n column-major, ldq >= M): the thin Q_i side by side, [Q_1 ... Q_G];
 * R (sum_i n_i^2 doubles): R_i row-major n_i x n_i, blocks in order.
 * Either pointer may be NULL.  GLM_SUR_INVALID_ARG on a handle set up with
 * reduce_rows (its factors are those of the reduced model). */
glm_sur_status glm_sur_get_factors(glm_sur_t h, double* Q, int64_t ldq, double* R, glm_sur_stream_t stream);

/* Kernels of the PCG steps of the last solve: 1 = fused two-pass float32
 * step with the Sigma-apply on the tensor cores, 0 = four launches per step
 * on the SIMT pipes, -1 = no solve yet.  Host-side query. */
int glm_sur_step_path(glm_sur_t h);

/* Number of kernel launches (including the nodes of replayed CUDA graphs)
 * this handle has issued since glm_sur_setup.  Host-side counter. */
int64_t glm_sur_launch_count(glm_sur_t h);

/* Measurement helper.  Runs `reps` PCG steps of the configuration of the last
 * solve (same k and precision; float32 bulk steps for FP32_REFINE) on the
 * handle's buffers, with the stop tests disabled, and writes the mean device
 * time in milliseconds of each launch of one step into the HOST array ms[5]:
 * ms[0] Sigma-apply step, ms[1] projection partials, ms[2] reduction and
 * scalar step, ms[3] projection update, ms[4] the whole step.  Events are
 * recorded on `stream`.  Synchronous.  Destroys the stored w (glm_sur_get_w
 * fails until the next solve). */
glm_sur_status glm_sur_profile_steps(glm_sur_t h, int reps, double* ms, glm_sur_stream_t stream);

/*
 * glm_sur_ols_static -- per-block least squares b_i = R_i^-1 Q_i^T y_i
 * (the ordinary least-squares estimate of every equation, from the factors
 * the handle already holds), for callers that must not allocate device
 * memory: code whose device memory is owned by another allocator or fully
 * reserved up front, or that must not trigger the implicit synchronisation
 * a cudaMalloc/cudaFree can cause.  It allocates nothing: its intermediate
 * sums live in one fixed 4 MiB device array inside the library (every GPU
 * that loads the library keeps it until the process exits).  There is no
 * counterpart in the paper; it is a service of this library.
 *
 *   Y  : DEVICE, m x k column-major (m = G*M, column j = vec(Y_j)), ldy >= m.
 *   b  : DEVICE output, n x k column-major, ldb >= n.
 * Limit: (n' * k) * 2 <= 524288 doubles, n' = sum_i 4*ceil(n_i/4); larger
 * requests return GLM_SUR_INVALID_ARG before any device work.
 * Call it with the handle's device current (GLM_SUR_INVALID_ARG otherwise).
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current; under CUDA's lazy module
 * loading that first call also loads the library's module that holds the
 * array (which reserves the 4 MiB on the device and may synchronise), so
 * make that first call outside any latency-critical region and before any
 * stream capture.  All calls share the array: calls that may
 * run at the same time on the GPU (different streams without ordering)
 * race and must be serialised by the caller.  Nothing in the array needs
 * clearing between calls: each call writes every entry it reads.
 * GLM_SUR_INVALID_ARG on a handle set up with reduce_rows.
 */
glm_sur_status glm_sur_ols_static(glm_sur_t h, const double* Y, int64_t ldy, int k,
                                  double* b, int64_t ldb, glm_sur_stream_t stream);

void glm_sur_destroy(glm_sur_t h);
const char* glm_sur_status_string(glm_sur_status s);

/* ------------------------------------------------------------------------
 * Batches of independent SUR instances (uneven G, M, n_i), each solved with
 * the same method: float32 PCG-Aug steps (Algorithm glmpcg2, D = I) inside
 * a float64 iterative-refinement loop, b = X*^T (y - Sigma w); one
 * persistent launch for the whole batch, one CTA per instance at a time.
 * ------------------------------------------------------------------------ */
typedef struct glm_sur_batch_ctx* glm_sur_batch_t;

/*
 * glm_sur_batch_setup -- factor every block of every instance (TSQR).
 *   count : number of instances.
 *   G, M  : HOST arrays (count): equations (1..32) and observations of each.
 *   n_i   : HOST array of sum_j G[j] block widths (1..32, <= M of the
 *           instance), instance by instance.  Padded width per instance
 *           n' = sum_i 4 ceil(n_i / 4) <= 512.
 *   X     : DEVICE, the instances' [X_1 ... X_G] (M_j x n_j column-major,
 *           ld = M_j) one after another.
 *   Omega : DEVICE, the instances' Omega_j (G_j x G_j column-major) one after
 *           another.
 *   opts  : tol (float64 residual ||P(y - Sigma w)|| / ||P y||), inner_tol,
 *           max_refine and reduce_rows are used; may be NULL.  reduce_rows = 1
 *           solves every instance with M_j >= 2 n_j on the n_j rows of its
 *           projection onto range([X_1 ... X_G]) (Remark rem:reduction: Q_W
 *           by Cholesky QR twice at setup, one float64 product Q_W^T Y_j per
 *           instance and solve; tol and relres then refer to the reduced
 *           system); when some W_j has no full column rank the whole batch
 *           is kept unreduced.  The float64 residual of a
 *           refined solve settles at a few 1e-13 on instances of this size,
 *           so a tol below that ends in GLM_SUR_NOT_CONVERGED after
 *           max_refine refinement steps with b still at full accuracy.
 */
glm_sur_status glm_sur_batch_setup(glm_sur_batch_t* out, int count, const int* G, const int* M,
                                   const int* n_i, const double* X, const double* Omega,
                                   const glm_sur_opts* opts, glm_sur_stream_t stream);
glm_sur_status glm_sur_batch_get_setup_status(glm_sur_batch_t h);

/*
 * glm_sur_batch_solve -- k in {1, 2, 4, 8} right-hand sides per instance.
 *   Y      : DEVICE, the instances' m_j x k column-major blocks (m_j = G_j M_j,
 *            ld = m_j, column c = vec(Y_c)) one after another.
 *   b      : DEVICE output, the instances' n_j x k column-major blocks.
 *   iters, relres : DEVICE outputs (nullable), count x k (instance-major):
 *            float32 steps summed over refinement steps; final float64
 *            relative residual.
 * The first solve with a given k tunes the tile height (three timed
 * launches, glm_sur_batch_tile reports them); later solves replay one
 * captured launch while Y, b, iters and relres stay the same.
 */
glm_sur_status glm_sur_batch_solve(glm_sur_batch_t h, const double* Y, int k, double* b, int* iters,
                                   double* relres, glm_sur_stream_t stream);
/* Synchronises; HOST status (count x k); returns the first status other than
 * GLM_SUR_OK / GLM_SUR_STAGNATED. */
glm_sur_status glm_sur_batch_get_status(glm_sur_batch_t h, int* status);
/* Work of the last batch solve, per instance (HOST arrays of count, either
 * nullable): float32 PCG steps its CTA ran over all refinement rounds (the
 * unit of the per-step traffic), and SM clock cycles from its start to its
 * end.  Synchronises. */
glm_sur_status glm_sur_batch_get_work(glm_sur_batch_t h, int* steps, long long* cycles);
/* Tile height chosen by the autotuner (0 before the first solve); tune_ms
 * (HOST, 3, nullable) receives the timed candidates (8, 16, 32 rows; 0 = not
 * timed: tuning stops once a candidate is 10% slower than the best). */
int glm_sur_batch_tile(glm_sur_batch_t h, float* tune_ms);
/* CTAs of the persistent batch launch (SMs x CTAs resident per SM at the
 * chosen tile height; 0 before the first solve, -1 for a NULL handle).
 * Host-side query. */
int glm_sur_batch_grid(glm_sur_batch_t h);
int64_t glm_sur_batch_launch_count(glm_sur_batch_t h);
void glm_sur_batch_destroy(glm_sur_batch_t h);

/* Library build information (static string). */
const char* glm_sur_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GLM_SUR_H */
