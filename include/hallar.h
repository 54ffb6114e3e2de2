/*
 * hallar.h -- C ABI of the B300 (sm_103a) HALLaR hot-path library.
 *
 * HALLaR (the hybrid low-rank augmented Lagrangian method) solves
 *
 *   (P)  min C.X  s.t.  A(X) = b,  X psd,  tr X <= tau^2          (Section 1, eq. P)
 *
 * through the factorisation X = UU^T, U in R^{n x r}.  Its data-parallel hot
 * path is a handful of operator evaluations on U (Section 4):
 *
 *   T  = A~(UU^T) = [C.UU^T ; A_1.UU^T ; ... ; A_m.UU^T]   (eq. A tilde operator)
 *   p' = p + beta (A(UU^T) - b)                            (eq. Grad U Space)
 *   W  = (C + A*(p')) U,   grad_U L_beta(UU^T; p) = 2W      (eqs. Grad U Space,
 *                                                            Adjoint calculation)
 *   lambda_min, v_min of G = C + A*(p')                     (Alg. 1 step 7)
 *
 * and the HALLaR loop (Alg. 1, ADAP-AIPP / ADAP-FISTA of Appendix A) that
 * drives them to a relative KKT tolerance (eq. termination2).
 *
 * Problem data.  C = C_sparse + C_J * 11^T + C_I * I, with C_sparse a
 * symmetric matrix in full CSR (both triangles; the diagonal may be stored).
 * The constraint family fixes the A_l:
 *   HALLAR_DIAG      A_i = e_i e_i^T, i = 0..n-1 (m = n).  Max-Cut SDP.
 *   HALLAR_EDGE      A_l = (e_i e_j^T + e_j e_i^T)/2 for pair l = (i, j), i != j,
 *                    so A_l.X = X_ij; optionally followed by a trace row A = I.
 *                    Lovasz theta SDP (eq. lovasz).
 *   HALLAR_OBSERVED  the EDGE family on pairs (i, n1 + j), i < n1, j < n - n1.
 *                    Matrix completion SDP (eq. matcomp-sdp).
 * Constraint l of the pair list is row l of b / p / residuals; the trace row,
 * when present, is the last one.  T has m + 1 entries, T[0] = C.UU^T.
 *
 * Memory and pointers.  A handle owns every device buffer it allocates and
 * frees them in hallar_destroy.  Arguments of hallar_create are HOST arrays,
 * copied to the device once (Section 3.1: data resident on the GPU).  Every
 * array argument of the other calls may be a host or a device pointer: the
 * library asks the CUDA runtime which it is and stages host arrays through
 * its own device buffers.  Factor arrays (U, W) are row-major n x r with
 * leading dimension r and hold double for HALLAR_FP64 handles and float for
 * HALLAR_MIXED handles; every other floating array is double.  Work is
 * issued on the handle's stream (hallar_options.stream, NULL = a stream the
 * handle creates); calls return after their results are complete.
 *
 * Errors.  Every call returns a hallar_status and never aborts, traps or
 * exits; hallar_last_error(h) describes the last failure on h.  Input
 * validation (indices in range, C symmetric, finite values, sizes) happens
 * on the host before any kernel runs.  Kernels never spin on a flag.
 *
 * Precision.  HALLAR_FP64 keeps every quantity in double.  HALLAR_MIXED keeps
 * U, the row dot products and the SpMM in float with float accumulation; the
 * multipliers p, the residuals r, p', the reductions (C.UU^T, p^T r,
 * ||r||^2), Lanczos (basis, orthogonalisation, Ritz values), the dual update,
 * the KKT norms and the Frank-Wolfe and line-search scalars stay in double.
 *
 * Limits.  n < 2^31, stored nonzeros < 2^31, r <= 256; hallar_solve takes
 * r_cap <= 89 (its rank trim diagonalises an (r_cap+1)^2 Gram matrix).
 *
 * Beyond the single problem (none of these has a counterpart in the paper):
 * hallar_server_* runs whole solves concurrently under an HBM budget
 * (continuous batching), hallar_batch_* evaluates the fused operator of many
 * stacked instances in one launch, hallar_check_problem validates a problem
 * on the host alone, and hallar_grad_diag_noalloc is a handle-free gradient
 * that allocates nothing.
 */
#ifndef HALLAR_H
#define HALLAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hallar_ctx* hallar_t;

typedef enum {
  HALLAR_OK = 0,
  HALLAR_EINVAL = 1,    /* bad argument: null pointer, size or index out of
                           range, non-finite value, asymmetric C            */
  HALLAR_ENOMEM = 2,    /* device allocation failed                        */
  HALLAR_ECUDA = 3,     /* CUDA runtime error (message in last_error)      */
  HALLAR_ENOTCONV = 4,  /* iteration limit reached before the tolerance    */
  HALLAR_ETIMEOUT = 5,  /* wall-clock limit reached before the tolerance   */
  HALLAR_ERANK = 6,     /* rank would exceed the cap and trimming failed   */
  HALLAR_ENUMERIC = 7   /* a NaN or Inf appeared in a reduction            */
} hallar_status;

typedef enum { HALLAR_DIAG = 0, HALLAR_EDGE = 1, HALLAR_OBSERVED = 2 } hallar_family;
typedef enum { HALLAR_FP64 = 0, HALLAR_MIXED = 1 } hallar_precision;

/* Parameters of the method.  The paper fixes none of sigma, chi, lambda_0,
 * beta_0 or the epsilon_t / beta_t schedules (Alg. 1 remarks, Appendix A);
 * hallar_default_options fills this library's choices. */
typedef struct {
  double tol;             /* relative KKT tolerance of eq. termination2 (1e-5)    */
  double sigma;           /* ADAP-FISTA success parameter sigma (0.3)             */
  double chi;             /* ADAP-FISTA parameter chi in (0,1) (0.5)              */
  double lambda0;         /* initial ADAP-AIPP prox stepsize (1)                  */
  double beta0;           /* initial penalty beta_1 (1)                           */
  double beta_max;        /* cap of the penalty schedule, in units of
                           * 1 + ||C||_1 (1e8)                                    */
  double eps_decay;       /* epsilon_{t+1} = eps_decay * epsilon_t (0.5)          */
  double eps1_rel;        /* epsilon_1 = eps1_rel (1 + tau^2 ||C||_1) (1e-2)      */
  double lanczos_tol_rel; /* Ritz residual tol = this * epsilon_t / tau^2 (0.5)   */
  double time_limit_s;    /* wall-clock limit of hallar_solve (3600)              */
  double lambda_kappa;    /* > 0: every ADAP-AIPP call starts at the prox stepsize
                           * lambda_kappa / beta_t (the subproblem's curvature grows
                           * with the penalty); 0: lambda starts at lambda0 and is
                           * carried over between calls (0)                       */
  int32_t r_cap;          /* maximum factor rank; the Gram trim keeps r_cap (32)  */
  int32_t max_outer;      /* AL iterations (300)                                  */
  int32_t max_hlr;        /* HLR iterations per AL iteration (100)                */
  int32_t max_aipp;       /* ADAP-AIPP iterations per call (20000)                */
  int32_t max_fista;      /* ADAP-FISTA iterations per call (400)                 */
  int32_t lanczos_kmax;   /* Lanczos basis size before a restart (300)            */
  int32_t precision;      /* hallar_precision                                     */
  int32_t verbose;        /* 1: one line per AL iteration on stderr; 2: also one
                           * per ADAP-AIPP call; 3: also ADAP-AIPP's step-2 test
                           * (device printf, stdout)                            */
  int32_t promote;        /* HALLAR_MIXED only (1): when ADAP-AIPP's prox steps no
                           * longer move the float factor (four ADAP-AIPP calls of
                           * one AL iteration end on a step that left W
                           * unchanged), the solve continues in FP64 from its own
                           * iterate (factor widened exactly; p, beta, lambda
                           * carried over) and returns the solution as float.
                           * 0: never                                           */
  uint64_t seed;          /* seed of the Lanczos start vectors (SplitMix64)       */
  void* stream;           /* cudaStream_t to issue on; NULL: the handle's own     */
} hallar_options;

/* Counters and results of hallar_solve.  pval = C.UU^T, dval = -b^T p -
 * tau^2 theta, and the three relative residuals of eq. termination2. */
typedef struct {
  double pval, dval, theta, lam_min_S;
  double rel_primal, rel_gap, rel_dual, kkt;
  double beta, seconds;
  int32_t rank, converged;
  int32_t outer_iters, hlr_iters, aipp_iters, fista_iters, fista_failures;
  int32_t lanczos_iters, fw_steps, trims;
  int32_t promoted_at;    /* AL iteration after which a mixed solve went on in
                           * FP64 (options.promote), 0 if it did not */
  int64_t grad_evals, value_evals, kernel_launches;
} hallar_result;

/* Fill *opt with the defaults listed above.  HALLAR_EINVAL for opt == NULL. */
hallar_status hallar_default_options(hallar_options* opt);

/* Build a problem on the current CUDA device (Section 3.1: C, A and b are
 * copied to the GPU once and stay resident).
 *   n              order of X (> 0).
 *   n1             HALLAR_OBSERVED only: rows of the observed block; else 0.
 *   C_rowptr[n+1], C_col[nnz], C_val[nnz]: symmetric sparse part of C in
 *                  full CSR (host); C_rowptr NULL means an empty sparse part.
 *   C_J, C_I       implicit C_J 11^T + C_I I added to C.
 *   family         hallar_family.
 *   m_pairs        EDGE / OBSERVED: number of pairs; DIAG: must be 0.
 *   cons_i, cons_j [m_pairs] pair indices (host).
 *   has_trace_row  EDGE / OBSERVED: 1 adds the constraint tr X = b[m-1].
 *   b              [m] right-hand side (host), m = n (DIAG) or
 *                  m_pairs + has_trace_row.
 *   tau2           tau^2 > 0, the trace bound of the spectraplex.
 *   opt            NULL for defaults; copied.
 *   out            receives the handle (NULL on failure).
 * Errors: HALLAR_EINVAL (validation), HALLAR_ENOMEM, HALLAR_ECUDA. */
hallar_status hallar_create(int64_t n, int64_t n1,
                            const int64_t* C_rowptr, const int32_t* C_col,
                            const double* C_val, double C_J, double C_I,
                            int32_t family, int64_t m_pairs,
                            const int32_t* cons_i, const int32_t* cons_j,
                            int32_t has_trace_row, const double* b, double tau2,
                            const hallar_options* opt, hallar_t* out);

/* T = A~(UU^T) (eq. A tilde operator; the sum of Alg. 2 / Alg. 3).
 *   U  [n x r] factor (host or device), r in [1, 256].
 *   T  [m + 1] doubles (host or device): T[0] = C.UU^T, T[1+l] = A_l.UU^T. */
hallar_status hallar_eval_A(hallar_t h, const void* U, int32_t r, double* T);

/* One fused gradient evaluation (eqs. AL function, Grad U Space, Adjoint
 * calculation): with r_l = A_l.UU^T - b_l and p' = p + beta r,
 *   W     [n x r] = (C + A*(p')) U   (the U-gradient of L_beta is 2W),
 *   g_val [1]     = C.UU^T + p^T r + beta/2 ||r||^2   (host; may be NULL),
 *   resid [m]     = r                                  (may be NULL).
 * p is [m] doubles.  U and W must not overlap. */
hallar_status hallar_grad(hallar_t h, const void* U, int32_t r, const double* p,
                          double beta, void* W, double* g_val, double* resid);

/* Change of the AL value g(U) = L_beta(UU^T; p) between two factors,
 * g(Y) - g(X) (eq. AL function): the quantity the step-2 tests of ADAP-FISTA
 * (Appendix A.1) and ADAP-AIPP (Appendix A) compare.  It is formed without
 * cancellation from the differences of the pair products,
 * <Y_a,Y_b> - <X_a,X_b> = <D_a,Y_b> + <X_a,D_b> with D = Y - X, by the same
 * kernel hallar_solve runs.
 *   X, Y  [n x r] factors (host or device, the handle's precision), r in [1, 256].
 *   p     [m] multipliers (doubles), beta the penalty.
 *   rX    [m] r_X = A(XX^T) - b (doubles, host or device), or NULL: then the
 *         library evaluates it with one pass of the fused operator.
 *   dg    (host) receives g(Y) - g(X).
 *   rY    [m] out (doubles, host or device) or NULL: r_Y = r_X + A(YY^T) - A(XX^T).
 * In the mixed form p and r_X are read as float copies and r_Y is formed in
 * float (the solver keeps its residuals in the factor type). */
hallar_status hallar_value_change(hallar_t h, const void* X, const void* Y, int32_t r,
                                  const double* p, double beta, const double* rX, double* dg,
                                  double* rY);

/* Rank trim (not in the paper; the solver applies it when a Frank-Wolfe step
 * (eq. tilde Y) would take the factor above hallar_options.r_cap):
 * Yout = Y Q_k, where Q_k holds the k leading eigenvectors of the Gram Y^T Y,
 * so Yout Yout^T is the best rank-k approximation of YY^T (Eckart-Young).
 *   Y     [n x r] (host or device, the handle's precision), 1 <= k <= r <= 90.
 *   Yout  [n x k] out (host or device), leading dimension k.
 *   eigs  [r] out (host, may be NULL): the Gram eigenvalues, descending.
 * The Gram is accumulated in FP64; its eigenvectors come from cyclic Jacobi
 * rotations on the host. */
hallar_status hallar_trim_rank(hallar_t h, const void* Y, int32_t r, int32_t k, void* Yout,
                               double* eigs);

/* Goemans-Williamson hyperplane rounding of a Max-Cut factor (not in the
 * paper, which stops at the SDP solution; the standard way to turn the
 * Max-Cut SDP's X = UU^T into a cut).  For each trial t the caller's normal
 * g_t gives x_i = sign(<U_i, g_t>) (+1 at zero, in double), and the trial's
 * cut value is -x^T C x (= (1/4) x^T L x, the weight of the cut edges, for
 * C = -L/4).
 *   U      [n x r] factor (host or device, the handle's precision), 1 <= r <= 256.
 *   G      [trials x r] doubles, row t the normal of trial t (host or device).
 *   x_best [n] int8 out (host or device, may be NULL): the best trial's signs.
 *   cuts   [trials] doubles out (host): each trial's cut value.
 * HALLAR_EINVAL for a handle that is not HALLAR_DIAG. */
hallar_status hallar_maxcut_round(hallar_t h, const void* U, int32_t r, const double* G,
                                  int32_t trials, int8_t* x_best, double* cuts);

/* Entries of X = UU^T at index pairs, X_ab = <U_a, U_b> (double).  For a
 * matrix-completion problem (HALLAR_OBSERVED, eq. matcomp-sdp) the
 * recovered matrix is X's off-diagonal block: M^_ij = X_{i, n1 + j}.
 *   U       [n x r] factor (host or device), 1 <= r <= 256.
 *   a, b    [count] int32 row indices in [0, n) (host or device; host pairs
 *           are range-checked, device pairs are the caller's to keep in range).
 *   out     [count] doubles (host or device). */
hallar_status hallar_factor_entries(hallar_t h, const void* U, int32_t r, const int32_t* a,
                                    const int32_t* b, int64_t count, double* out);

/* Minimum eigenpair of G = C + A*(p') (Alg. 1 step 7, eq. Grad X Space) by
 * Lanczos in FP64 with partial reorthogonalisation (the basis is swept
 * against when Simon's estimate of the loss of orthogonality passes
 * sqrt(eps)), restarted from the Ritz vector every kmax steps, until
 * ||G v - lambda v|| <= tol or 50 restarts.
 *   pshift [m]  p' (doubles).
 *   v0     [n]  start vector, or NULL for the SplitMix64 vector of opt.seed.
 *   lambda_min (host), v [n] (unit), iters (host), resid (host): outputs;
 *   v, iters, resid may be NULL.
 * Returns HALLAR_ENOTCONV (with the best Ritz pair written) when the
 * tolerance was not met. */
hallar_status hallar_min_eig(hallar_t h, const double* pshift, double tol,
                             int32_t kmax, const double* v0, double* lambda_min,
                             double* v, int32_t* iters, double* resid);

/* Run HALLaR (Alg. 1) from U0 [n x r0] (projected onto the ball ||U||_F <= tau
 * when outside it) and p0 [m] (NULL = 0) to the relative KKT tolerance of
 * eq. termination2.  The final factor and multipliers stay on the device;
 * read them with hallar_get_solution.  res (host) may be NULL.
 * Returns HALLAR_OK on convergence, HALLAR_ENOTCONV / HALLAR_ETIMEOUT when a
 * limit was hit first (res still filled). */
hallar_status hallar_solve(hallar_t h, const void* U0, int32_t r0, const double* p0,
                           hallar_result* res);

/* Copy the last solve's factor U [n x rank] (leading dimension rank; needs
 * r_capacity >= rank) and multipliers p [m] out (host or device).  U and p
 * may be NULL; rank (host) receives the rank when non-NULL. */
hallar_status hallar_get_solution(hallar_t h, void* U, int32_t r_capacity, double* p,
                                  int32_t* rank);

/* Kernel timing.  Kernel classes: 0 = the fused constraint map + shift +
 * SpMM (hallar_grad, and every gradient of hallar_solve), 1 = the
 * value-change kernel of the ADAP-FISTA / ADAP-AIPP tests, 2 = the Lanczos
 * basis passes.  op = 1 clears the counters and starts timing (a CUDA event
 * pair on the handle's stream around every launch of those kernels), op = 2
 * stops timing, op = 0 only reads.  ms[3], launches[3], bytes[3] and
 * bytes_padded[3] (host, may be NULL) receive, per class since the last
 * clear, the summed kernel milliseconds, the launch counts and the summed
 * bytes: every input array read once and every output written once,
 * gathered neighbour rows not counted; `bytes` counts the r columns of each
 * factor row and per-row / per-constraint vectors at the element size the
 * kernel reads (4 bytes in the mixed form), `bytes_padded` the stored
 * leading dimension (r rounded up to 16 bytes) instead of r.  Timing adds
 * two event records per timed launch (see hallar_profile_sampling). */
hallar_status hallar_profile(hallar_t h, int32_t op, double* ms, int64_t* launches,
                             double* bytes, double* bytes_padded);

/* Sampled kernel timing: with every = k > 1, hallar_profile times only every
 * k-th launch of each kernel class (the 1st, (k+1)-th, ...) and counts the
 * bytes and launches of the timed ones, so the average launch duration is
 * measured at 1/k of the event overhead.  every = 1 (the default) times
 * every launch.  HALLAR_EINVAL for every < 1. */
hallar_status hallar_profile_sampling(hallar_t h, int32_t every);

/* Allocation-free fused gradient for the diagonal (Max-Cut) family.  The
 * paper has no counterpart: it exists for callers that cannot let a library
 * call cudaMalloc -- applications that hand out device memory only from their
 * own pool or arena and account for every byte, and hot paths where an
 * allocation (or the device-wide synchronisation of a later cudaFree) would
 * stall work queued on other streams.  It computes what hallar_grad
 * computes for a HALLAR_DIAG problem (A_i = e_i e_i^T, b, C), from arrays
 * the caller owns, with no handle:
 *   rowptr[n+1], col[nnz], cval[nnz]  off-diagonal entries of C (device,
 *                                     full symmetric CSR, int32 indices),
 *   cdiag[n]   diagonal of C (plus any C_I),  b[n], p[n]   (device),
 *   U[n x r]   factor, W[n x r] = (C + Diag(p + beta r)) U   (device, double,
 *              row-major with leading dimension r, 16-byte aligned),
 *   resid[n]   r = diag(UU^T) - b (device; may be NULL),
 *   g_out[1]   C.UU^T + p^T r + beta/2 |r|^2 (device),
 *   stream     cudaStream_t to issue on (NULL: the legacy default stream),
 *   errbuf     optional host buffer for a message on failure.
 * Limits: 2 <= r <= 64 with r even, n < 2^31; anything else returns
 * HALLAR_EINVAL with a message.  The call only enqueues work on `stream`
 * and returns; it allocates nothing.  Its scratch (per-block partial sums
 * and an arrival counter) is one static device array of about 29 KB that
 * every GPU loading this library holds until exit; all calls share it and
 * it keeps the last call's contents, the counter is cleared at the start of
 * each call, and calls whose kernels overlap on the GPU race on it.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again
 * when the device's context was re-created (after cudaDeviceReset); make
 * that first call before any stream capture. */
hallar_status hallar_grad_diag_noalloc(int64_t n, int32_t r, const int32_t* rowptr,
                                       const int32_t* col, const double* cval,
                                       const double* cdiag, const double* b, const double* p,
                                       double beta, const double* U, double* W, double* resid,
                                       double* g_out, void* stream, char* errbuf,
                                       int32_t errbuf_len);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of whole solves.  The paper solves one problem
 * at a time (Section 5); this engine, which has no counterpart there, keeps a
 * FIFO of solve requests and runs up to max_inflight of them at once, each in
 * its own handle on its own CUDA stream driven by a worker thread, so their
 * kernels overlap on the device.  A request is admitted when a worker is free
 * and its estimated device footprint (hallar_solve_footprint) fits in what the
 * HBM budget has left; requests that arrive while others run wait in the
 * queue and are admitted as workers and memory free up.  Problem data, the
 * factor and the multipliers stay on the device from admission to the end
 * of the solve.  Every kernel is deterministic and handles share no device
 * state, so a request's result does not depend on what else is in flight.
 * ------------------------------------------------------------------------- */
typedef struct hallar_server* hallar_server_t;

typedef struct {
  double hbm_budget_bytes;  /* summed footprint of the solves admitted at once (> 0) */
  int32_t max_inflight;     /* solves on the device at once, 1..256                  */
  int32_t device;           /* CUDA device of every solve                            */
} hallar_server_options;

/* One solve request: the arguments of hallar_create, the start factor and the
 * options.  Every array is a HOST array; hallar_server_submit copies them, so
 * the caller may release them when it returns.  U0 is n x r0, row-major,
 * double for HALLAR_FP64 and float for HALLAR_MIXED (opt.precision); C_nnz is
 * the length of C_col / C_val (C_rowptr[n]).  opt.stream is ignored. */
typedef struct {
  int64_t n, n1;
  const int64_t* C_rowptr;
  const int32_t* C_col;
  const double* C_val;
  int64_t C_nnz;
  double C_J, C_I;
  int32_t family;
  int64_t m_pairs;
  const int32_t* cons_i;
  const int32_t* cons_j;
  int32_t has_trace_row;
  const double* b;
  double tau2;
  const void* U0;
  int32_t r0;
  hallar_options opt;
} hallar_request;

/* Aggregate counters of a server; latencies are from submit to completion. */
typedef struct {
  int64_t submitted, admitted, completed, failed, queued, inflight, max_inflight_seen;
  double bytes_inflight, peak_bytes_inflight;
  double p50_latency_s, p99_latency_s, mean_latency_s, max_latency_s;
  double first_submit_to_last_done_s;
} hallar_server_stats;

/* Estimated device bytes of one solve of req (problem data, the solver's
 * factors and vectors, the Lanczos basis, staging and reduction buffers, plus
 * 5 % and 64 MB of allocator slack; a mixed request with opt.promote counts
 * its factor buffers at 8 bytes an entry, what they hold after a promotion);
 * host arithmetic only.  -1 if req is NULL. */
int64_t hallar_solve_footprint(const hallar_request* req);

/* Start a server (worker threads; no device memory until requests run).
 * HALLAR_EINVAL for bad options, HALLAR_ECUDA if the device is unusable. */
hallar_status hallar_server_create(const hallar_server_options* opt, hallar_server_t* out);

/* Queue a solve.  *ticket (host) identifies it for hallar_server_wait.
 * HALLAR_EINVAL for a NULL or malformed request (sizes, null arrays),
 * HALLAR_ENOMEM when its footprint exceeds the whole budget.  Problems that
 * only hallar_create detects (asymmetric C, bad indices) complete with that
 * status. */
hallar_status hallar_server_submit(hallar_server_t s, const hallar_request* req,
                                   int64_t* ticket);

/* Wait for a ticket.  timeout_s < 0 waits without limit.  When the call
 * itself does not complete the ticket, *rank and *latency_s are set to -1:
 * HALLAR_ETIMEOUT when the request is still queued or running at the
 * timeout (the ticket stays valid), HALLAR_EINVAL for an unknown ticket or
 * U_capacity below the rank.  A completed solve that hit its own time limit
 * also returns HALLAR_ETIMEOUT, with its rank and latency (>= 0).  On
 * completion the ticket is released and the call returns the solve's status:
 *   res        (host, may be NULL) the hallar_result of the solve,
 *   U          (host, may be NULL) n x *rank factor, leading dimension
 *              U_capacity >= rank, in the request's precision,
 *   p          (host, may be NULL) the m multipliers,
 *   rank       (host, may be NULL) rank of U,
 *   latency_s  (host, may be NULL) seconds from submit to completion. */
hallar_status hallar_server_wait(hallar_server_t s, int64_t ticket, double timeout_s,
                                 hallar_result* res, void* U, int32_t U_capacity, double* p,
                                 int32_t* rank, double* latency_s);

/* Counters (host).  Latency percentiles over every completed request. */
hallar_status hallar_server_get_stats(hallar_server_t s, hallar_server_stats* st);

/* Stop the server: queued requests are dropped, running solves finish, the
 * workers exit and every result not yet waited for is released.  No other
 * call on s may run concurrently with this one or follow it. */
void hallar_server_destroy(hallar_server_t s);

/* Message of the last failure of a server call ("" if none), copied for the
 * calling thread: valid until that thread's next call of this function. */
const char* hallar_server_last_error(hallar_server_t s);

/* ---------------------------------------------------------------------------
 * Batching: many uneven instances in one launch.  The paper evaluates one
 * problem's operators at a time (Section 4); this layer, which has no
 * counterpart there, stacks `count` instances into one segmented problem --
 * instance k owns rows [row_off[k], row_off[k+1]) of a stacked factor and
 * constraints [cons_off[k], cons_off[k+1]) -- and evaluates the fused
 * constraint map + shift + SpMM of every instance in one launch of a
 * grid-stride kernel sized to one wave of resident blocks, with per-instance
 * penalties and per-instance reductions (summed per instance in a fixed
 * order, so results are deterministic for a given kernel shape).  Supported
 * instances: HALLAR_DIAG, HALLAR_EDGE and HALLAR_OBSERVED without the trace
 * row and with C_J = 0 (Max-Cut and matrix completion); others return
 * HALLAR_EINVAL.  The kernel shape (lanes per row, chunks per lane) for a
 * factor width is chosen on the first call with that width: by timing the
 * candidate shapes on the call's own data (autotune = 1; the choice is then
 * fixed for the batch) or by the built-in rule (autotune = 0).
 * ------------------------------------------------------------------------- */
typedef struct hallar_batch* hallar_batch_t;

/* Stack count >= 1 problems given as hallar_request (their U0, r0 and opt
 * are ignored) in the precision `precision` on `stream` (NULL: a stream the
 * batch creates).  Problem arrays are host arrays, copied.  HALLAR_EINVAL for
 * an unsupported or invalid instance (hallar_batch_last_error(NULL) names
 * it), HALLAR_ENOMEM, HALLAR_ECUDA. */
hallar_status hallar_batch_create(int32_t count, const hallar_request* problems,
                                  int32_t precision, int32_t autotune, void* stream,
                                  hallar_batch_t* out);

/* Layout (host pointers, any may be NULL): row_off[count+1], cons_off[count+1],
 * the stacked order n_total and constraint count m_total. */
hallar_status hallar_batch_layout(hallar_batch_t b, int64_t* row_off, int64_t* cons_off,
                                  int64_t* n_total, int64_t* m_total);

/* The fused operator of every instance in one launch (plus one per-instance
 * reduction launch):
 *   U     [n_total x r] stacked factors, row-major, leading dimension r, in
 *         the batch precision (host or device),
 *   p     [m_total] multipliers, beta [count] penalties (host or device),
 *   W     [n_total x r] out: W_k = (C_k + A_k*(p'_k)) U_k (host or device),
 *   g     [count] out: g_k = C_k.U_kU_k^T + p_k^T r_k + beta_k/2 |r_k|^2,
 *   resid [m_total] out or NULL: r = A(UU^T) - b per constraint.
 * 1 <= r <= 256.  Returns when the results are complete. */
hallar_status hallar_batch_grad(hallar_batch_t b, const void* U, int32_t r, const double* p,
                                const double* beta, void* W, double* g, double* resid);

/* Kernel shape used for factor width r (host pointers): lanes per row G,
 * 16-byte chunks per lane K, tuned = 1 when the autotuner timed it.
 * HALLAR_EINVAL before the first hallar_batch_grad with that width. */
hallar_status hallar_batch_shape(hallar_batch_t b, int32_t r, int32_t* G, int32_t* K,
                                 int32_t* tuned);

/* Free every resource of b (NULL is a no-op). */
void hallar_batch_destroy(hallar_batch_t b);

/* Message of the last failure on b; for b == NULL the last failure of
 * hallar_batch_create on this thread. */
const char* hallar_batch_last_error(hallar_batch_t b);

/* Validate a problem exactly as hallar_create does and build its merged CSR
 * on the host, without touching a device (arguments as for hallar_create;
 * no options).  On success m (constraints), nnz_merged (stored entries of
 * the merged CSR: off-diagonal C entries plus both orientations of every
 * pair) and c_norm1 (induced 1-norm of C, the scale of eq. termination2)
 * are written to the non-NULL host pointers.  Errors: HALLAR_EINVAL with
 * the reason in hallar_last_error(NULL), HALLAR_ENOMEM. */
hallar_status hallar_check_problem(int64_t n, int64_t n1, const int64_t* C_rowptr,
                                   const int32_t* C_col, const double* C_val, double C_J,
                                   double C_I, int32_t family, int64_t m_pairs,
                                   const int32_t* cons_i, const int32_t* cons_j,
                                   int32_t has_trace_row, const double* b, double tau2,
                                   int64_t* m, int64_t* nnz_merged, double* c_norm1);

/* Merged support of general sparse data matrices (Section 4.1, eqs.
 * support S ell and index list; the pattern S and lists L_ij that Alg. 4
 * forms M from): the host half of general HSLR/SDPA input (Section 3.2).
 *   n          order of the matrices (> 0); m: constraints (>= 0).
 *   count      listed entries; ell[k] in 0..m (0 = C), 0 <= ii[k] <= jj[k] < n
 *              (each symmetric matrix by its upper triangle), val[k] finite.
 *              Entries repeated for one (l, i, j) are summed; entries that are
 *              or sum to exactly 0 are dropped.
 * Outputs (host, written when non-NULL; call once with NULL arrays for the
 * sizes): *nnz_S stored pattern entries (both triangles: the diagonal once,
 * every off-diagonal pair twice), *nnz_L list entries; rowptr[n+1] and
 * col[nnz_S] the CSR of the pattern (columns ascending); for stored entry e,
 * its list L_ij is lidx/lval[lptr[e] .. lptr[e+1]) (lptr[nnz_S+1]), matrices
 * ascending, so M_ij = sum over the list of p~[lidx] * lval.
 * Host arithmetic only.  Errors: HALLAR_EINVAL (reason in
 * hallar_last_error(NULL)), HALLAR_ENOMEM. */
hallar_status hallar_merge_general(int64_t n, int64_t m, int64_t count, const int32_t* ell,
                                   const int32_t* ii, const int32_t* jj, const double* val,
                                   int64_t* nnz_S, int64_t* nnz_L, int64_t* rowptr,
                                   int32_t* col, int64_t* lptr, int32_t* lidx, double* lval);

/* Problem sizes of a handle (host pointers; any may be NULL). */
hallar_status hallar_get_sizes(hallar_t h, int64_t* n, int64_t* m, int64_t* nnz_merged,
                               int32_t* precision);

/* Free every resource of h (NULL is a no-op). */
void hallar_destroy(hallar_t h);

/* Message of the last failure on h ("" if none); for h == NULL, the last
 * failure of hallar_create on this thread.  Valid until the next call on h. */
const char* hallar_last_error(hallar_t h);

/* Name of a status code. */
const char* hallar_status_string(hallar_status s);

#ifdef __cplusplus
}
#endif

#endif /* HALLAR_H */
