/*
 * nys.h -- C ABI of the GB300 (sm_103a) Nys-IP-PMM normal-equations solver.
 *
 * The library solves separable convex QPs (Section 1, problems (P)/(D)):
 *     min 1/2 x^T Q x + c^T x   s.t.  A x = b,  x >= 0,     Q = diag(q), q >= 0,
 * and their generalisation (P~)/(D~) with free variables (x_F free) and
 * box-constrained variables (0 <= x_J <= u_J) of the section on free and
 * box-constrained variables (nys_problem.var_kind),
 * by the randomized-Nystrom-preconditioned IP-PMM of arxiv 2404.14524
 * (Algorithm 6 with the predictor-corrector of Algorithm 5 and the Newton
 * solve of Algorithm 4).  Every step of the solve runs in this library's CUDA
 * kernels; the caller only provides memory and a CUDA stream.
 *
 * Conventions for every entry point below:
 *  - A is dense and row-major, m x n, leading dimension lda >= n (elements).
 *  - Tall m x ell panels (Omega, Y, U) are column-major with leading
 *    dimension ld >= m (elements).
 *  - "device" pointers are CUDA device (or managed) memory on the handle's
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    pointer it passes; the handle owns only its internal workspace.
 *  - All work is issued on the handle's stream.  Entry points that return a
 *    scalar through a host pointer synchronise that stream before returning.
 *  - Return value: NYS_OK (0), a negative error, or a positive warning.  No
 *    entry point aborts, traps or throws; after an error the message is
 *    available from nys_last_error(h).  Invalid sizes or NULL pointers give
 *    NYS_ERR_ARG before any device work is issued.
 */
#ifndef NYS_H
#define NYS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nys_solver* nys_handle;

typedef enum {
    NYS_OK = 0,
    NYS_ERR_ARG = -1,             /* invalid argument (size, pointer, dtype, ell)     */
    NYS_ERR_CUDA = -2,            /* a CUDA runtime call failed                       */
    NYS_ERR_NUMERIC = -3,         /* NaN/Inf met in an iterate or a reduction         */
    NYS_ERR_CORE_BREAKDOWN = -4,  /* chol(Omega^T Y_nu) hit a non-positive pivot      */
    NYS_ERR_TIMEOUT = -5,         /* a bounded device-side wait expired               */
    NYS_ERR_NOMEM = -6,           /* workspace allocation failed / problem too large  */
    NYS_WARN_MAXITER = 1,         /* IPM reached max_ipm_iter before the tolerance    */
    NYS_WARN_PCG_MAXITER = 2      /* some PCG solve stopped at max_pcg_iter           */
} nys_status;

typedef enum { NYS_F64 = 0, NYS_F32 = 1, NYS_BF16 = 2, NYS_FP8E4M3 = 3 } nys_dtype;

/* Solver options.  Defaults (nys_default_options): tol 1e-6, ell 20,
 * max_ipm_iter 200, max_pcg_iter 1000, seed 0, rho0 = delta0 = 8 (Algorithm 6,
 * second step), reg_floor 5e-10 (the floor seen in Tables 7-8), no forced
 * counts, start_mode 0, reuse_pcg 0, adapt_cost 0, ell_min 0. */
typedef struct {
    double tol;                   /* relative KKT tolerance of the termination test  */
    int ell;                      /* Nystrom sketch size (clamped to m)               */
    int max_ipm_iter;
    int max_pcg_iter;
    unsigned long long seed;      /* key of the counter-based Gaussian stream         */
    int precision_mode;           /* 0 = FP64 form (A must be NYS_F64); 1 = precision */
                                  /*   form, BF16 inner operator; 2 = precision form, */
                                  /*   FP8 E4M3 inner operator with per-row scales    */
                                  /*   (1 and 2: A must be NYS_F32)                   */
    double rho0, delta0, reg_floor;
    /* Parity mode (optional, host arrays): run exactly forced_pcg_iters[s] PCG
     * iterations in Newton solve s (predictor, corrector, predictor, ...), and
     * exactly forced_ipm_iters IPM iterations when >= 0. */
    const int* forced_pcg_iters;
    int n_forced_pcg;
    int forced_ipm_iters;
    /* Start point: 0 = the problem's x0, y0, z0 (and w0, s0); 1 = the
     * practical initial point of the supplement's construction: candidate
     * x~ = u/2 + A^T (A A^T + 10 I)^{-1} (b - A u/2) and
     * y~ = (A A^T + 10 I)^{-1} A (c + Q x~), both by Nystrom PCG on A A^T
     * (Omega of the first IPM iteration, relative residual 1e-10; not counted
     * in pcg_iters_total / pcg_log), z~ = c - A^T y~ + Q x~ (halved on J),
     * s~_J = -z~_J, w~_J = u_J - x~_J, then the shifts that make x, w, z, s
     * strictly positive (the denominator of the dual shift sums x~ + delta_p:
     * the printed x~ + delta_d is read as the primal shift).  With 1 the
     * problem's x0, y0, z0, w0, s0 are ignored and may be NULL. */
    int start_mode;
    /* Preconditioner reuse (the paper suggests reusing the preconditioner
     * between IPM iterations without giving a rule): 0 = a fresh sketch and
     * Nystrom factor in every IPM iteration (Algorithm 6 as written); R > 0 =
     * keep the previous iteration's factor (U, Lambda; P^{-1} is rebuilt with
     * the current delta) while both PCG solves of the previous iteration took
     * at most R iterations. */
    int reuse_pcg;
    /* Sketch size per IPM iteration (Algorithm 6, "choose sketch size l_k"):
     * 0 = every factor has the problem's ell (l_max).  C > 0 = adaptive: with
     * a factor taken to cost about C * l / l_max PCG iterations, iteration k
     * is followed by a doubled sketch when its two PCG solves took more than
     * 2 C l_k / l_max iterations and by a halved one when they took fewer than
     * C l_k / (2 l_max), within [ell_min, l_max]; the first factor uses
     * ell_min (0 = max(1, l_max / 8)).  Omega_k of size l_k is the first l_k
     * columns of the l_max-wide Omega_k.  Not combined with reuse_pcg or with
     * nys_solve_batched (NYS_ERR_ARG); a resumed solve starts again at
     * ell_min. */
    int adapt_cost;
    int ell_min;
} nys_options;

/* One QP.  With host == 0 all pointers are device pointers; with host == 1
 * they are host pointers and nys_solve stages them to the device itself
 * (copies included in nys_result.seconds).  x0, y0, z0 is the strictly
 * interior start point (x0 > 0, z0 > 0; unused with options.start_mode 1).
 * Warm start (resume from a saved state): lam0 and zeta0 are the PMM
 * estimates lambda, zeta (NULL = y0, x0 as in Algorithm 6), the options'
 * rho0/delta0 carry rho and delta, k0 is the index of the first IPM
 * iteration (it selects the Gaussian test matrix Omega_k), and with
 * has_peu_ref = 1 peu_ref_p / peu_ref_d are the relative primal / dual
 * infeasibilities recorded at the last re-centring of lambda / zeta
 * (has_peu_ref = 0: those of the start point, as in a fresh solve).
 *
 * PMM parameter update (Algorithm 6, last step; the paper fixes its outcome
 * in Tables 7-8: rho_0 = delta_0 = 8, independent decrease, floor 5e-10):
 * after each iteration r = |mu_new - mu_old| / max(mu_new, mu_old); lambda is
 * re-centred on y and delta shrinks by 1 - r when the relative primal
 * infeasibility fell to 95% of its value at lambda's last re-centring (or
 * meets tol, or that value already met tol), else delta shrinks by
 * 1 - (2/3) r and lambda stays; zeta, rho likewise with the dual
 * infeasibility and x.  Both parameters are floored at reg_floor. */
typedef struct {
    int m, n;
    int a_dtype;                  /* nys_dtype of A                                   */
    const void* A;                /* m x n row-major                                  */
    long long lda;
    const double *b, *c, *q;      /* m, n, n                                          */
    const double *x0, *y0, *z0;   /* n, m, n                                          */
    int host;
    const double *lam0, *zeta0;   /* m, n, or NULL                                    */
    int k0;
    int ell;                      /* sketch size for this problem (0 = the handle's), */
                                  /* clamped to the handle's ell and to m             */
    /* Free and box-constrained variables, problems (P~)/(D~).  var_kind NULL:
     * every x_j >= 0 (problem (P)); u, w0, s0 are then ignored.  Otherwise n
     * kinds: 0 = x_j >= 0 (set I), 1 = free (F), 2 = 0 <= x_j <= u_j (J).
     * The iteration is Algorithm 5 with Algorithm 4 in its general form: the
     * slack w = u - x and the multiplier s of x_J <= u_J move with the primal
     * and the dual step; z0 is ignored on F (z_F = 0).  On J, u must be
     * finite and s0, w0 positive (u and s0 are required when some kind is 2;
     * entries outside J are ignored).  An invalid kind or J entry gives
     * NYS_ERR_ARG (checked on the device before the first iteration).
     * Termination: ||(Ax - b, x_J + w_J - u_J)|| / (1 + ||(b, u_J)||),
     * ||c + Qx - A^T y - z + s|| / (1 + ||c||) and
     * mu = (x_IJ^T z_IJ + w_J^T s_J) / (|I u J| + |J|) all <= tol. */
    const signed char* var_kind;  /* n, or NULL                                       */
    const double* u;              /* n: upper bounds (read on J)                      */
    const double* w0;             /* n: start of w on J (NULL = u - x0)               */
    const double* s0;             /* n: start of s on J                               */
    int has_peu_ref;              /* 1: peu_ref_p, peu_ref_d below are used (resume)  */
    double peu_ref_p, peu_ref_d;
    /* Parity mode for this problem alone (optional): with forced_override = 1
     * these replace the options' forced_pcg_iters / n_forced_pcg /
     * forced_ipm_iters (same meaning; host array), so that each problem of a
     * batch can follow its own recorded counts. */
    int forced_override;
    const int* forced_pcg_iters;
    int n_forced_pcg;
    int forced_ipm_iters;
} nys_problem;

/* Result.  x, y, z are caller-allocated outputs (n, m, n) in the same memory
 * space as the problem (device, or host when problem.host == 1).  On an error
 * they hold the last complete iterate.  lam, zeta (m, n; NULL = not wanted)
 * receive the final PMM estimates, which with rho/delta and ipm_iters make a
 * resumable state. */
typedef struct {
    double *x, *y, *z;
    double *lam, *zeta;
    int status;                   /* nys_status of the solve                          */
    int ipm_iters;
    int pcg_iters_total;
    int refine_steps;
    double rel_primal;            /* ||Ax - b|| / (1 + ||b||)  ((P~): see var_kind)    */
    double rel_dual;              /* ||c + Qx - A^T y - z (+ s)|| / (1 + ||c||)        */
    double mu;                    /* x^T z / n  ((P~): see var_kind)                   */
    double rel_gap;               /* |pobj - dobj| / (1 + |pobj|)                      */
    double rho, delta;            /* final PMM regularisation                          */
    double seconds;               /* wall time inside nys_solve                        */
    double pcg_seconds;           /* device time of the PCG solves (CUDA events on the */
                                  /*   handle's stream around each solve; in a batch,  */
                                  /*   each problem's share of the launches it shared, */
                                  /*   in proportion to its PCG iterations)            */
    int* pcg_log;                 /* optional host array: PCG iterations per Newton   */
    int pcg_log_cap;              /*   solve, in order (capacity in entries)           */
    int pcg_log_len;              /* entries written                                   */
    double *w, *s;                /* n each, NULL = not wanted: final slack and bound */
                                  /*   multiplier of a (P~) problem (0 outside J)     */
    int sketches;                 /* Nystrom factors built (= ipm_iters unless reused) */
    double peu_ref_p, peu_ref_d;  /* final references of the PMM update (resumable    */
                                  /*   state together with lam, zeta, rho, delta)      */
    int* ell_log;                 /* optional host array: sketch size of each factor  */
    int ell_log_cap;              /*   built, in order (capacity in entries)           */
    int ell_log_len;              /* entries written                                   */
    int device_iteration;         /* 1: the device-resident iteration ran (one graph  */
                                  /*   launch per IPM iteration), 0: host phases       */
} nys_result;

/* Fill *opt with the defaults listed above. */
void nys_default_options(nys_options* opt);

/* Create a solver handle for problems up to max_m x max_n.  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream).  Allocates the workspace
 * (O(max_m*ell + max_n*ell + ell^2) doubles plus split-reduction buffers) on
 * the current device.  Errors: NYS_ERR_ARG, NYS_ERR_NOMEM, NYS_ERR_CUDA. */
int nys_create(nys_handle* h, const nys_options* opt, int max_m, int max_n, int max_batch,
               void* cuda_stream);

/* Solve one QP with Algorithm 6 (IP-PMM, Nystrom PCG for every Newton system).
 * Termination: rel_primal, rel_dual and mu all <= tol.  Returns the status
 * also stored in r->status. */
int nys_solve(nys_handle h, const nys_problem* p, nys_result* r);

/* Solve `count` independent QPs (the batching form), each exactly as
 * nys_solve would, with up to max_batch of them in flight at once; each
 * in-flight problem owns a private worker solver (workspace, CUDA stream,
 * cached graphs) sized for the handle's max_m x max_n.  When every problem is
 * of kind (P) and the form is FP64, each worker advances its problem with the
 * device-resident iteration (one graph launch per IPM iteration) at its own
 * pace, one host thread keeping the workers fed, and the number in flight is
 * autotuned on the first call (see nys_batch_inflight); otherwise the
 * problems run in lock-step groups whose PCG solves share thread-block
 * cluster launches.  p[i] and r[i] follow nys_solve's conventions (device or
 * host memory per problem).  The handle must have been created with
 * max_batch >= 1.  Returns the worst status (negative errors first); each
 * r[i].status holds its own.  All work is complete on return.  A problem's
 * results do not depend on the batch it is in or on the number in flight;
 * they depend on its PCG cluster plan, which is the fixed rule's unless the
 * plan autotuner (nys_batch_plan) has chosen one for its shape bucket. */
int nys_solve_batched(nys_handle h, int count, const nys_problem* p, nys_result* r);

/* Problems in flight chosen for this handle's batches by timed trials (0
 * until a batch of at least 128 problems with max_batch >= 16 has run on the
 * device-resident path): in-flight counts of 8, 16, 24, 32, 48, 64, ..., up
 * to the number of hardware queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless
 * set) and max_batch, are scored by the PCG work completed per second over
 * 0.8 s each, a larger count kept only when it beats the best by 3 %.  Untuned batches run
 * max_batch at once; NYS_BATCH_TUNE=0 keeps max_batch. */
int nys_batch_inflight(nys_handle h);

/* The PCG cluster plan the batching form's autotuner chose for problems of
 * this shape (the bucket of m rounded up to 64, n rounded up to 512, the same
 * ell = min(ell option, m, the problem's ell)).  Before a batch of at least
 * 128 problems with max_batch >= 16 on the device-resident path starts
 * (NYS_BATCH_TUNE and NYS_BATCH_PLAN_TUNE not 0), every bucket this handle
 * has not seen is tuned:
 * each cluster plan with A in shared memory that fits (16, 8 or 4 CTAs) runs
 * 16 forced PCG iterations of a synthetic system of the bucket's first
 * shape, and the plan with the least time x max(CTAs, SMs / hardware queues)
 * is kept (no more problems run at once than CUDA_DEVICE_MAX_CONNECTIONS
 * queues, 8 unless set, so a narrower plan is charged that share of the
 * SMs).  Buckets whose A fits no cluster's shared memory keep the fixed
 * rule's plan reading A from L2 (*ctas = 0): alone on the GPU a trial finds
 * A in L2, which a full batch does not.
 * Later problems of the bucket, in this and later calls, run it when it fits
 * their exact shape.  Writes *ctas (4, 8, 16; 0 when the bucket keeps the
 * fixed rule's plan) and *a_smem (1: A in shared memory); returns 1 when the
 * bucket has been tuned, 0 when not, NYS_ERR_ARG on bad arguments. */
int nys_batch_plan(nys_handle h, int m, int n, int ell, int* ctas, int* a_smem);

int nys_destroy(nys_handle h);

/* Gradients of a loss L(x*) through the solutions of `count` solved QPs (the
 * differentiation form).  At each final iterate the transposed regularised
 * KKT system J^T lam = (dL/dx, 0, 0), J the Newton matrix of Eq. Newton at
 * the final (x, z, rho, delta), is reduced exactly like Eq. normal-eq:
 *   (A D A^T + delta I) lam2 = A D g,   lam1 = D (g - A^T lam2),
 * solved by Nystrom PCG (a fresh sketch at the final D, relative tolerance
 * eta), and
 *   dL/dc = -lam1, dL/db = lam2, dL/dq = -lam1 .* x, dL/dA = y lam1^T - lam2 x^T.
 * p[i], r[i]: the problems and results of the forward solves (device
 * problems, FP64 A; x, y, z, rho, delta are read from r[i]).  Device arrays,
 * QPs concatenated in order: dL_dx, dL_dc, dL_dq (sum n_i), dL_db (sum m_i),
 * dL_dA (sum m_i n_i, each QP row-major m_i x n_i; FP64).  Any output may be
 * NULL.  Problems (P) only: a problem with var_kind set gives NYS_ERR_ARG.
 * Returns the worst status over the QPs. */
int nys_adjoint(nys_handle h, int count, const nys_problem* p, const nys_result* r, const double* dL_dx,
                double eta, double* dL_dc, double* dL_db, double* dL_dq, double* dL_dA);

/* Message of the last error recorded on h (static storage owned by h). */
const char* nys_last_error(nys_handle h);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all handles; a counter for instrumentation, not a synchronisation). */
unsigned long long nys_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Step-level entry points (device pointers).  Each is one step of the solve,
 * exposed so that it can be called and checked on its own.
 * ------------------------------------------------------------------------- */

/* D = (Q + Theta^{-1} + rho I)^{-1} with Theta = X Z^{-1}, i.e.
 * D_j = 1 / (q_j + z_j / x_j + rho)  (Section 2.1.2, below Eq. delta_z).
 * x, z, q, D: device, length n.  x > 0 is required (not checked). */
int nys_scaling(nys_handle h, int n, const double* x, const double* z, const double* q,
                double rho, double* D);

/* out = (N + delta I) v with N = A diag(D) A^T (Eq. normal-eq): one streaming
 * pass of A for t = D .* (A^T v) and one for A t.  A: device, a_dtype must be
 * NYS_F64.  D: device n; v, out: device m (out must not alias v). */
int nys_normal_matvec(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
                      const double* D, double delta, const double* v, double* out);

/* The precision form's operator: out = A_r (D .* (A_r^T v)) + delta v with A_r
 * stored in reduced precision (a_dtype NYS_BF16, or NYS_FP32) and given as two
 * row-major copies, A (m x n, lda) and AT = A^T (n x m, ldat); products and
 * sums in FP32 (Eq. normal-eq in the precision of the inner PCG solves).
 * D, v, out: FP64 device.  The handle must be a precision-form handle
 * (precision_mode 1); A and AT 16-byte aligned. */
int nys_normal_matvec_lp(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
                         const void* AT, long long ldat, const double* D, double delta, const double* v,
                         double* out);

/* FP8 storage of the precision form's matrix (the per-row-scaled FP8
 * variant of Eq. normal-eq's operator): s_r = max_c |A[r, c]| / 448
 * (448 = the largest finite E4M3 value; s_r = 1 for an all-zero row) and
 * Q[r, c] = E4M3(A[r, c] / s_r), round to nearest, saturating, so that
 * A ~ diag(s) Q.  A: FP32 device m x n (lda >= n).  Outputs (device,
 * caller-allocated): Q, m x ldq bytes (ldq >= n); QT = Q^T, n x ldqt bytes
 * (ldqt >= m); padding columns are zeroed; row_scale: FP32, m. */
int nys_quantize_fp8(nys_handle h, int m, int n, const float* A, long long lda, void* Q, long long ldq,
                     void* QT, long long ldqt, float* row_scale);

/* out = diag(s) Q (D .* (Q^T (s .* v))) + delta v with (Q, QT, s) from
 * nys_quantize_fp8: the FP8 operator of the inner PCG solves of
 * precision_mode 2, FP32 products and sums.  Q, QT: device bytes, rows 16-byte
 * aligned for the vectorised path (ldq, ldqt multiples of 16); D, v, out: FP64
 * device.  The handle must have precision_mode 2. */
int nys_normal_matvec_fp8(nys_handle h, int m, int n, const void* Q, long long ldq, const void* QT,
                          long long ldqt, const float* row_scale, const double* D, double delta, const double* v,
                          double* out);

/* (N + delta I) v = A (D .* (A^T v)) + delta v, as nys_normal_matvec, for
 * callers that cannot allocate device memory (code running inside a stream
 * capture or under a memory pool that a cudaMalloc would disturb, hosts that
 * forbid allocation after start-up, plugins that only receive pointers): it
 * takes no handle and allocates nothing.  The paper has no counterpart; this
 * is an interface of this library.
 * Scratch: one fixed 8 MiB device array inside the library, held by every
 * GPU that loads it until exit; n <= 1,048,576 (larger n returns
 * NYS_ERR_NOMEM).  The first call on a device, with that device current,
 * looks up the array's device address (make it before any stream capture).
 * The address is cached per device for the life of the process: after a
 * cudaDeviceReset of that device no further call may be made.
 * All calls share the array: calls that may overlap on the GPU race and must
 * be serialised by the caller.  A: FP64 row-major m x n (lda >= n); D: n;
 * v, out: m (out must not alias v); all device pointers; work is issued on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream) and not waited
 * for.  Errors: NYS_ERR_ARG, NYS_ERR_NOMEM, NYS_ERR_CUDA. */
int nys_normal_matvec_noalloc(int m, int n, const double* A, long long lda, const double* D, double delta,
                              const double* v, double* out, void* cuda_stream);

/* Omega_k (m x ell, leading dimension ld): entry (i, j) is the standard normal
 * deviate of Algorithm 1's first step drawn from the SplitMix64 stream of
 * Steele, Lea and Flood (2014) keyed by `seed`, at stream positions 2c and
 * 2c + 1 with c = (k*ell + j)*m + i, via u = ((bits >> 11) + 1/2) 2^-53 and
 * Box-Muller sqrt(-2 ln u1) cos(2 pi u2).  Omega: device. */
int nys_gaussian(nys_handle h, unsigned long long seed, int k, int m, int ell, double* Omega,
                 int ld);

/* Sketch Y = N Omega = A (D .* (A^T Omega)) (Algorithm 1, second step).
 * Omega, Y: device m x ell (column-major, leading dimension ld); D: device n.
 * a_dtype NYS_F64: FP64 arithmetic.  a_dtype NYS_F32 (precision-form handle
 * only, else NYS_ERR_ARG): the precision form's sketch on the tensor cores --
 * A (FP32) and Omega rounded to BF16 (Omega via FP32), T = A^T Omega with FP32
 * accumulation, T' = BF16(D .* T), Y = A T' with FP32 accumulation, widened
 * to FP64; Omega is not modified. */
int nys_sketch(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
               const double* D, int ell, const double* Omega, double* Y, int ld);

/* Nystrom factor from a sketch (Algorithm 1, steps 3-8): nu = eps(||Y||_F),
 * Y_nu = Y + nu Omega, C = chol(Omega^T Y_nu) (upper, after symmetrising),
 * B = Y_nu C^{-1}, thin SVD B = U Sigma V^T, lam = max(0, Sigma^2 - nu),
 * sorted descending.  Y, Omega: device m x ell inputs (not modified);
 * U: device m x ell output (same ld); lam: device ell output; *nu: host.
 * Errors: NYS_ERR_CORE_BREAKDOWN if the Cholesky meets a pivot <= 0. */
int nys_nystrom(nys_handle h, int m, int ell, const double* Y, const double* Omega, int ld,
                double* U, double* lam, double* nu);

/* out = P_Nys^{-1} r (Eq. Nys_precond_inv):
 * (lam_ell + delta) U (Lam + delta I)^{-1} U^T r + (I - U U^T) r, with
 * lam_ell the last (smallest) entry of lam.  U: device m x ell (ld);
 * lam: device ell; r, out: device m (out must not alias r). */
int nys_precond_apply(nys_handle h, int m, int ell, const double* U, int ld, const double* lam,
                      double delta, const double* r, double* out);

/* Preconditioned CG for (N + delta I) dy = xi from dy = 0 (Section 2.2 with
 * P_Nys), N = A diag(D) A^T.  Stops at the top of an iteration once the
 * recursive residual satisfies ||r|| <= eta ||xi||, or after max_iter
 * iterations; forced_iters >= 0 runs exactly that many.  *iters and
 * *res_norm (host) receive the iteration count and final ||r||.
 * Returns NYS_WARN_PCG_MAXITER if the tolerance was not met. */
int nys_pcg(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
            const double* D, double delta, int ell, const double* U, int ld, const double* lam,
            const double* xi, double* dy, double eta, int max_iter, int forced_iters,
            int* iters, double* res_norm);

/* The same PCG on the precision form's operators (the inner solves of
 * precision_mode 1 and 2 and their final stage): the FP32 matrix A (device,
 * m x n, lda) is first copied into the handle's operator storage, then
 * (N_r + delta I) dy = xi is solved with N_r = A_r diag(D) A_r^T for
 * op_dtype NYS_BF16 (BF16 copies, FP32 sums), NYS_FP8E4M3 (E4M3 copies with
 * per-row scales, FP32 sums; precision_mode 2 handles only) or NYS_F32 (the
 * FP32 matrix with float-float sums, the problem's own operator).  Vectors
 * FP64; other arguments and results as nys_pcg.  The handle must be a
 * precision-form handle. */
int nys_pcg_lp(nys_handle h, int m, int n, const float* A, long long lda, int op_dtype, const double* D,
               double delta, int ell, const double* U, int ld, const double* lam, const double* xi, double* dy,
               double eta, int max_iter, int forced_iters, int* iters, double* res_norm);

/* Which implementation nys_pcg / nys_solve use for an FP64 system of this
 * size (the same arithmetic in each; they differ only in summation order):
 *   NYS_ROUTE_CLUSTER_SMEM  one thread-block cluster, A's column bands in
 *                           shared memory (small A);
 *   NYS_ROUTE_CLUSTER_L2    one thread-block cluster, A read from L2;
 *   NYS_ROUTE_COOPERATIVE   one cooperative grid-wide launch;
 *   NYS_ROUTE_GRAPH         one CUDA-graph launch of per-step kernels.
 * The choice depends only on (m, n, ell), the device and the environment
 * variable NYS_PCG_PATH (cluster | cooperative | graph) read at nys_create
 * (with "cluster", systems whose A does not fit on chip use a cluster that
 * reads A from L2).
 * Returns the route, or NYS_ERR_ARG for a null handle or sizes <= 0.
 * The paper has no counterpart: its PCG runs on a CPU. */
enum { NYS_ROUTE_CLUSTER_SMEM = 0, NYS_ROUTE_CLUSTER_L2 = 1, NYS_ROUTE_COOPERATIVE = 2, NYS_ROUTE_GRAPH = 3 };
int nys_pcg_route(nys_handle h, int m, int n, int ell);

/* Newton direction through the normal equations (Algorithm 4 with I = all):
 * xi_au = -X^{-1} r_xz; xi = r_p + A D (r_d + xi_au); (N + delta I) dy = xi by
 * the PCG above; dx = D (A^T dy - r_d - xi_au); dz = X^{-1} (r_xz - Z dx).
 * Vectors: device; r_d, r_xz, x, z, D, dx, dz length n; r_p, dy length m. */
int nys_newton(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
               const double* x, const double* z, const double* D, double delta,
               const double* r_d, const double* r_p, const double* r_xz,
               int ell, const double* U, int ld, const double* lam,
               double eta, int max_iter, int forced_iters,
               double* dx, double* dy, double* dz, int* iters);

/* C = A B^T on the tcgen05 tensor cores, BF16 inputs, FP32 accumulation: the
 * two products of the sketch (Algorithm 1, second step) in the precision form
 * are of this shape (A^T Omega with A^T stored row-major, and A T').
 * A: M x K, B: N x K, both BF16 row-major with K contiguous, leading
 * dimensions multiples of 8 elements, 16-byte aligned; C: FP32 column-major
 * M x N, ldc >= M.  N <= 512.  Device pointers.  Kernel: a CTA pair per
 * 256-row stripe (tcgen05.mma.cta_group::2) with the k-blocks split evenly
 * over the resident pairs, partial tiles summed in a fixed order; or, where
 * clusters of two cannot run or the partial tiles do not fit the handle's
 * workspace, one CTA per 128-row stripe with split-K.  The environment
 * variable NYS_UMMA_PAIR=0 / 1 forces the one-CTA / the pair kernel (1: a
 * CUDA error when the pair kernel cannot run).  NYS_ERR_ARG if M x N (padded)
 * exceeds the handle's workspace. */
int nys_gemm_bf16(nys_handle h, int M, int N, int K, const void* A, long long lda, const void* B,
                  long long ldb, float* C, long long ldc);

/* Fraction-to-boundary step (Eq. stepsize-p / stepsize-d):
 * *alpha = 0.995 min{1, min over dv_i < 0 of -v_i / dv_i}.
 * v, dv: device length n; *alpha: host. */
int nys_step_length(nys_handle h, int n, const double* v, const double* dv, double* alpha);

#ifdef __cplusplus
}
#endif
#endif /* NYS_H */
