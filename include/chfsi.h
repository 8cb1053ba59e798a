/*
 * chfsi.h -- C ABI of the GB300 ChFSI library (libchfsi.so).
 *
 * Chebyshev Filtered Subspace Iteration for sequences of correlated dense
 * Hermitian eigenproblems, after Berljafa, Wortmann and Di Napoli, "An
 * Optimized and Scalable Eigensolver for Sequences of Eigenvalue Problems"
 * (arXiv 1404.4161): Algorithm 1 (ChFSI), Algorithm 2 (the Chebyshev filter
 * with per-vector degrees), Sec. 3.2 (degree optimisation).
 *
 * Conventions for every entry point:
 *  - Complex numbers are complex128 stored as interleaved (re, im) doubles.
 *    A "complex n x k matrix" is n*k such pairs, column-major, leading
 *    dimension n (column j starts at element j*n).
 *  - Pointers are DEVICE pointers unless the parameter name ends in _host.
 *    The caller owns every buffer it passes; the library never frees or
 *    keeps a caller pointer beyond the call.
 *  - Work is issued on the stream given to chfsi_init (a cudaStream_t passed
 *    as void*; NULL = the legacy default stream).  Entry points that return
 *    host-visible results (stats, *_host outputs) synchronise that stream
 *    before returning; the others are stream-ordered.
 *  - Return value: CHFSI_OK or one of the error codes below.  No entry point
 *    exits the process or traps on the device.  chfsi_strerror() names a
 *    code; chfsi_last_error() gives a message for the last failure on ctx.
 *  - Not thread-safe per context: one host thread per chfsi_ctx at a time.
 *  - Diagnostics: with the environment variable CHFSI_VERBOSE=1 the solvers
 *    print one line per outer loop on stderr (loop, active and locked
 *    columns, residual range of the wanted pairs, filter interval, summed
 *    degrees).  This adds a device-to-host copy per loop.
 */
#ifndef CHFSI_H
#define CHFSI_H

#ifdef __cplusplus
extern "C" {
#endif

#define CHFSI_OK 0
#define CHFSI_EINVAL 1      /* bad argument: sizes, NULL pointer, options  */
#define CHFSI_ENOMEM 2      /* device allocation failed                     */
#define CHFSI_ENOCONV 3     /* max_loops reached before nev pairs converged */
#define CHFSI_EBREAKDOWN 4  /* QR breakdown: filtered block rank-deficient  */
#define CHFSI_ENAN 5        /* NaN or Inf met in a reduction                */
#define CHFSI_ETIMEOUT 6    /* a bounded device wait gave up                */
#define CHFSI_ECUDA 7       /* CUDA runtime error                           */
#define CHFSI_ENOTSUP 8     /* configuration not supported on this device   */
#define CHFSI_ETOOBIG 9     /* n*k above the static scratch of               */
                            /* chfsi_filter_static (CHFSI_FILTER_STATIC_MAX_NK) */

/* Arithmetic of the filter (the other steps always run in FP64). */
#define CHFSI_PREC_FP64 0   /* complex FP64 filter on the FP64 pipe          */
#define CHFSI_PREC_MIXED 1  /* split-precision tensor-core filter while the  */
                            /* largest wanted residual > switch_tol, then    */
                            /* FP64 filter sweeps to tol                     */
#define CHFSI_PREC_TC 2     /* split-precision tensor-core filter in every   */
                            /* loop; from the second loop on it filters the  */
                            /* residual block (chfsi_filter_refine), so its  */
                            /* error scales with the residual: no FP64 sweep */

/* Split format of the tensor-core filter (CHFSI_PREC_MIXED / _TC): each
 * operand x = x0 + x1 + x2 in bf16 pieces (x0 = bf16(x), x1 = bf16(x - x0),
 * x2 = bf16(x - x0 - x1)), FP32 accumulation in TMEM. */
#define CHFSI_SPLIT_BF16X3 0 /* x0 y0 + x0 y1 + x1 y0: 3 products, ~2^-16     */
#define CHFSI_SPLIT_BF16X6 1 /* adds x0 y2 + x1 y1 + x2 y0: 6 products,       */
                             /* ~2^-20 (the FP32 accumulation dominates)    */
#define CHFSI_SPLIT_ADAPTIVE 2 /* the solver uses BF16X6 for the refinement  */
                             /* form while 2^-16 x 1.7 x the largest wanted */
                             /* residual exceeds tol/3, else BF16X3; the     */
                             /* single-step entry points use BF16X3         */

/* Engine of the FP64 products (H Q, Gram matrices, block products). */
#define CHFSI_GEMM_FP64 0   /* DFMA kernels on the FP64 pipe                 */
#define CHFSI_GEMM_OZAKI 1  /* FP64-accurate emulation on the BF16 tensor    */
                            /* cores: 7 x 7-bit error-free slices, 28 slice  */
                            /* products, exact FP32 chunk sums (~2^-48 of    */
                            /* row scale x column scale per product)         */

/* Degree model (degree optimisation of Alg. 1). */
#define CHFSI_DEG_ANALYTIC 0 /* Single Optimization rule of Sec. 3.2         */
#define CHFSI_DEG_MLP 1      /* learned predictor; analytic rule as fallback */

typedef struct chfsi_ctx chfsi_ctx;

typedef struct chfsi_opts {
  int precision;       /* CHFSI_PREC_FP64 / _MIXED / _TC      (FP64)       */
  int split;           /* CHFSI_SPLIT_*                       (ADAPTIVE)   */
  int degree_model;    /* CHFSI_DEG_*                         (ANALYTIC)   */
  int deg_cold;        /* first-loop degree, random start     (20)         */
  int deg_warm;        /* first-loop degree, warm start       (8)          */
  int deg_min;         /* lower clamp of the degree rule      (1)          */
  int deg_max;         /* upper clamp of the degree rule      (36)         */
  int deg_extra;       /* margin added to the rule's ceiling  (1)          */
  int lanczos_steps;   /* Lanczos steps for the bounds        (20)         */
  int max_loops;       /* outer-loop limit                    (50)         */
  double switch_tol;   /* MIXED: residual below which FP64 takes over (1e-4) */
  unsigned long long seed; /* SplitMix64 seed of the Lanczos start (1)     */
  int profile;         /* 1: time every FP64 GEMM and tensor-core filter */
                       /* launch with CUDA events into chfsi_stats (0)    */
  int mlp_extra;       /* DEG_MLP: margin added to the learned degree (2) */
  int step0;           /* sequence index of the next problem solved (0):  */
                       /* the step feature of the degree MLP and traces   */
  int f64_gemm;        /* CHFSI_GEMM_FP64 / CHFSI_GEMM_OZAKI        (FP64) */
  int warm_rr;         /* 1: on a warm start, Rayleigh-Ritz the starting  */
                       /* block before the first filter, so the first loop */
                       /* gets per-vector degrees and (CHFSI_PREC_TC) the  */
                       /* refinement form (0: the paper's uniform deg)     */
  int warm_resid;      /* 1: on a warm start, the Rayleigh quotients and  */
                       /* residuals of the starting block on the new H    */
                       /* (one product H X, no reduced eigensolve): pairs */
                       /* already converged lock, the first loop gets     */
                       /* per-vector degrees and (CHFSI_PREC_TC) the      */
                       /* refinement form; 0: the uniform deg_warm (0)    */
  int autotune;        /* 1: the tensor-core filter times its candidate   */
                       /* tilings (column block width x tile grouping)    */
                       /* on the first launch of each (n, k/32, split)    */
                       /* shape and keeps the fastest for the context;    */
                       /* results do not depend on the tiling (1)         */
} chfsi_opts;

/* Per-problem statistics (host struct, filled when non-NULL). */
typedef struct chfsi_stats {
  int status;               /* return code of this problem               */
  int loops;                /* outer loops (filter + QR + RR)            */
  int loops_lowp;           /* loops whose filter ran split-precision    */
  int n_locked;             /* converged pairs at exit                   */
  long long col_degrees;    /* sum over loops of sum_j m_j               */
  long long col_degrees_lowp; /* the part done by the tensor-core filter */
  double beta;              /* Lanczos upper bound of the spectrum       */
  double norm_h;            /* ||H||_est used to normalise residuals     */
  double max_resid;         /* largest residual of the nev wanted pairs  */
  double ms_total;          /* wall time of the solve on the stream      */
  double ms_lanczos, ms_filter, ms_qr, ms_rr, ms_resid, ms_lock;
  double filter_flops;      /* useful filter flops, 8 n^2 sum m_j        */
  long long filter_launches; /* filter-step kernel launches              */
  long long launches;       /* all kernel launches of this solve         */
  /* per-kernel device time (opts.profile = 1; zero otherwise): */
  double k_f64_ms;          /* FP64 complex GEMM kernels (H Q, Gram, ...) */
  double k_f64_flops;       /* their flops, 8 per complex multiply-add   */
  long long k_f64_launches;
  double k_tc_ms;           /* tcgen05 filter-step kernel                */
  double k_tc_flops;        /* its useful complex flops, 8 n^2 k_active  */
  long long k_tc_launches;
  double k_solver_ms;       /* FP32 start of the reduced eigensolve on    */
                            /* dense quotients (tridiagonal reduction and */
                            /* the tridiagonal eigenpairs)                */
  long long k_solver_calls;
  int loops_mlp;            /* loops whose degrees came from the MLP     */
  int mlp_fallback;         /* 1 if the MLP stalled and the analytic rule */
                            /* took over for the rest of this problem     */
  double k_f64_exec_flops;  /* flops the FP64 GEMM kernels executed: with */
                            /* the tensor-core engine S(S+1)/2 BF16 slice */
                            /* products per product (S slices), else     */
                            /* k_f64_flops                                */
  /* more per-kernel device times (opts.profile = 1): */
  double k_cholinv_ms;      /* inverse-Cholesky kernel of the QR step    */
  double k_lanczos_ms;      /* Lanczos kernels of the spectral bounds    */
  double k_slice_ms;        /* operand slicers of the tensor-core engine */
  double k_eigctl_ms;       /* control kernels of the reduced eigensolve */
                            /* (analysis, cluster rotations)             */
  double k_tc_exec_flops;   /* flops the tensor-core filter executed: 3 or */
                            /* 6 BF16 products per complex product         */
} chfsi_stats;

/* ---- context ---------------------------------------------------------- */

/* Fill *opts with the defaults shown above. */
void chfsi_default_opts(chfsi_opts* opts);

/* Create a context bound to the current CUDA device and `stream`.
 * opts may be NULL (defaults).  Workspaces are allocated lazily and grown
 * on demand; they belong to the context.  Returns EINVAL, ENOMEM, ECUDA or
 * ENOTSUP (device is not sm_103 when the MIXED path is asked for). */
int chfsi_init(chfsi_ctx** ctx, const chfsi_opts* opts, void* stream);

/* Replace the options of an existing context (same validation as init). */
int chfsi_set_opts(chfsi_ctx* ctx, const chfsi_opts* opts);

/* Release the context and all its device memory.  NULL is ignored. */
void chfsi_free(chfsi_ctx* ctx);

const char* chfsi_strerror(int code);
const char* chfsi_last_error(const chfsi_ctx* ctx);

/* ---- the solver (Alg. 1) ---------------------------------------------- */

/* Solve one problem: the nev lowest eigenpairs of the Hermitian H
 * (Alg. 1; Alg. 2 for the filter).
 *  H      complex n x n, Hermitian, read only (shift and scale of Alg. 2
 *         are folded into the filter; H is never written).
 *  X      complex n x (nev+nex); in: starting block X0, out: the block of
 *         Ritz vectors, the locked (converged) pairs first, ascending.
 *  evals  n_ev = nev+nex doubles (device), ascending within the locked part
 *         and within the rest, matching X's columns.
 *  warm_host  NULL for a random start, else two doubles {lam_1, lam_k} of
 *         the previous problem (Alg. 1 Require line): gamma and alpha.
 *  Requires 1 <= nev, 1 <= nex, nev + nex <= n.  On ENOCONV X holds the
 *  last block of Ritz vectors; on any other error X is left unchanged. */
int chfsi_solve(chfsi_ctx* ctx, const double* H, int n, int nev, int nex,
                double* X, double tol, double* evals,
                const double* warm_host, chfsi_stats* stats_host);

/* Solve a correlated sequence (Definitions 1-2, Sec. 2.2): problem l+1
 * starts from problem l's Ritz vectors and its lam_1, lam_k.
 *  H      array of N device pointers to complex n x n Hermitian matrices
 *         (the array itself is in host memory).
 *  X      in: X0 for the first problem; out: the Ritz vectors of the last.
 *  evals  N x (nev+nex) doubles (device), row l = problem l.
 *  stats_host  NULL or N structs. */
int chfsi_solve_sequence(chfsi_ctx* ctx, const double* const* H_host, int N,
                         int n, int nev, int nex, double* X, double tol,
                         double* evals, chfsi_stats* stats_host);

/* Same as chfsi_solve_sequence with every buffer in HOST memory: the call
 * copies each H to the device (double-buffered against the solve of the
 * previous problem), X in and out, and evals out. */
int chfsi_solve_sequence_host(chfsi_ctx* ctx, const double* const* H_host, int N,
                              int n, int nev, int nex, double* X_host, double tol,
                              double* evals_host, chfsi_stats* stats_host);

/* One independent sequence of chfsi_solve_batched. */
typedef struct chfsi_problem {
  const double* const* H_host; /* host array of `steps` device pointers to */
                               /* complex n x n Hermitian matrices          */
  int n, nev, nex;
  double* X;                   /* device, complex n x (nev+nex): in X0,     */
                               /* out the Ritz block of the last step        */
  double* evals;               /* device, steps x (nev+nex) doubles          */
  int warm;                    /* in: 1 = X holds the Ritz vectors of an     */
                               /* earlier step of this sequence and          */
                               /* lam_lo, lam_hi its lambda_1, lambda_k (the */
                               /* first step starts warm); 0 = random X0     */
  double lam_lo, lam_hi;       /* in (warm = 1) / out: lambda_1, lambda_k of */
                               /* the last step solved                       */
} chfsi_problem;

/* Many independent sequences (k-point style) solved in lockstep: at each
 * step l, problem p starts from its step l-1 Ritz block (at l = 0 from X
 * as the problem's warm field says), and every outer loop filters all
 * unconverged problems in ONE
 * batched persistent tensor-core launch (opts.precision CHFSI_PREC_TC or
 * CHFSI_PREC_MIXED; FP64 filters run per problem), followed by each
 * problem's QR, Rayleigh-Ritz, residuals, locking and degrees.
 *  stats_host  NULL or steps * P structs, entry l * P + p; with
 *  opts.profile the batch's kernel times are reported in entry l * P. */
int chfsi_solve_batched(chfsi_ctx* ctx, int P, chfsi_problem* probs, int steps,
                        double tol, chfsi_stats* stats_host);

/* Generalized problem A c = lambda B c (A Hermitian, B Hermitian positive
 * definite; the form the paper's FLAPW sequences come in, Sec. 3): the
 * input of Alg. 1 is the reduction to standard form H = L^-1 A L^-H with
 * B = L L^H (Cholesky), and c = L^-H y.  Here B = R^H R with R = L^H; the
 * inverse factor W = R^-1 = L^-H comes from the library's inverse-Cholesky
 * kernel (FP64), H = W^H A W and C = W Y from the context's FP64 product
 * engine.
 *  A, B   complex n x n (device), read only.
 *  X      in: starting block of H (a random block, or in a sequence the
 *         previous problem's Y, as in the paper); out: Y, the Ritz vectors
 *         of H (as chfsi_solve).
 *  C      complex n x (nev+nex) (device) out: W Y, the generalized
 *         eigenvectors (C^H B C = I).
 *  evals, warm_host, stats_host as chfsi_solve.
 *  EBREAKDOWN when B is not numerically positive definite.  The context
 *  keeps three n x n workspaces for the reduction. */
int chfsi_solve_generalized(chfsi_ctx* ctx, const double* A, const double* B, int n, int nev,
                            int nex, double* X, double* C, double tol, double* evals,
                            const double* warm_host, chfsi_stats* stats_host);

/* ---- the steps of the hot path, one entry point each ------------------ */

/* Alg. 1 (spectral bounds): s-step Lanczos with full reorthogonalisation from the
 * SplitMix64 start vector of `seed` (entry j = u(2j) + i u(2j+1), u(t) =
 * 2 (splitmix64_t >> 11) 2^-53 - 1).  out_host[0..3] = {beta = theta_max +
 * ||f||, theta_min, theta_max, ||H||_est = max(|theta_min|, |theta_max|)}. */
int chfsi_lanczos(chfsi_ctx* ctx, const double* H, int n, int steps,
                  unsigned long long seed, double* out_host);

/* Alg. 2: filter the k columns of Y0 (complex n x k) with degrees
 * degrees_host[0..k-1] (>= 1, ascending), Y_m,j = C_{m_j}(Hs) Y0_j /
 * C_{m_j}(gamma_hat), Hs = (H - cI)/e, gamma_hat = (lam1 - c)/e.  Result in
 * Y (complex n x k; may not alias Y0).  precision = CHFSI_PREC_FP64 or
 * CHFSI_PREC_MIXED (tensor-core split product with the context's split
 * format). */
int chfsi_filter(chfsi_ctx* ctx, const double* H, int n, int k, const double* Y0,
                 const int* degrees_host, double lam1, double c, double e,
                 double* Y, int precision);

/* One problem of chfsi_filter_batched (same meaning as chfsi_filter's
 * arguments; every pointer is a device pointer except degrees_host). */
typedef struct chfsi_filter_item {
  const double* H;          /* complex n x n Hermitian                     */
  int n, k;
  const double* Y0;         /* complex n x k, ascending-degree columns      */
  const int* degrees_host;  /* k ints >= 1, ascending                       */
  double lam1, c, e;
  double* Y;                /* complex n x k output (not aliasing Y0)       */
} chfsi_filter_item;

/* Alg. 2 for P independent problems of any sizes in one persistent,
 * cooperative tensor-core launch (split precision as CHFSI_PREC_MIXED):
 * one CTA per SM walks a list of (step, problem, tile) work items; a step
 * of a problem starts when that problem's previous step is complete
 * (bounded device waits; CHFSI_ETIMEOUT if one gives up).  Results equal
 * chfsi_filter(..., CHFSI_PREC_MIXED) problem by problem. */
int chfsi_filter_batched(chfsi_ctx* ctx, int P, const chfsi_filter_item* items);

/* Alg. 2 in refinement form (not in the paper): for Ritz pairs (Y, ritz)
 * of H and R = H Y - Y diag(ritz), returns Y_m = p_m(H) Y exactly as
 * chfsi_filter would, computed as Y psi_m(ritz) + D_m: psi_m is the
 * filter's scalar recurrence on each Ritz value (FP64) and D_m the same
 * three-term recurrence driven by R (D_0 = 0, D_1 = a_0 R, D_{i+1} =
 * a_i (H D_i - c D_i) + b_i D_{i-1} + a_i psi_i(ritz) R), computed with
 * the split-precision tensor-core product.  Its error is the split
 * precision times ||R|| rather than times ||Y||.
 *  Y, R   complex n x k (device), columns in ascending-degree order.
 *  ritz   k doubles (device); degrees_host as for chfsi_filter.
 *  Yout   complex n x k (device), may not alias Y or R. */
int chfsi_filter_refine(chfsi_ctx* ctx, const double* H, int n, int k, const double* Y,
                        const double* R, const double* ritz, const int* degrees_host,
                        double lam1, double c, double e, double* Yout);

/* Complex GEMM with either engine: C = alpha op(A) B + beta C, op(A) = A
 * (op_a = 0) or A^H (op_a = 1); op(A) is m x k, B k x n, C m x n, all
 * column-major complex with leading dimensions lda, ldb, ldc (device).
 * engine = CHFSI_GEMM_FP64 or CHFSI_GEMM_OZAKI.  The building block of
 * Rayleigh-Ritz (H Q, Q^H Z, Q W) and CholQR (Y^H Y, Y R^-1). */
int chfsi_zgemm(chfsi_ctx* ctx, int op_a, int m, int n, int k, double alpha, const double* A,
                int lda, const double* B, int ldb, double beta, double* C, int ldc, int engine);

/* Alg. 1 (QR step): orthonormalise the k columns of Y (complex n x k, in
 * place) against the nl orthonormal columns of L (complex n x nl; may be
 * NULL when nl = 0) by two block Gram-Schmidt passes and CholQR2 (shifted
 * CholQR3 when the Gram matrix is not numerically positive definite).
 * With the FP64 engine (opts.f64_gemm = CHFSI_GEMM_FP64) the result is the
 * unique Q with R's diagonal real positive.  With CHFSI_GEMM_OZAKI the first
 * Cholesky pass runs in FP32 arithmetic and, when it leaves
 * ||I - Y^H Y||_F <= 0.1, the second is the polar correction
 * Y (I - F)^{-1/2}, F = I - Y^H Y (binomial series): the result is then an
 * orthonormal basis of the same span, not the Cholesky one (FP64 CholQR2
 * otherwise).  EBREAKDOWN if the block is rank-deficient. */
int chfsi_orthonormalize(chfsi_ctx* ctx, int n, int nl, const double* L, int k,
                         double* Y);

/* Alg. 1: Rayleigh-Ritz on orthonormal Q (complex n x k):
 * Z = HQ, G = Q^H Z (Hermitianised), G W = W Lambda, Y = QW, HY = ZW.
 * Y and HY: complex n x k outputs; evals: k doubles, ascending.  The k x k
 * eigensolve is this library's: FP32 eigenvectors (Householder
 * tridiagonalisation, Sturm multisection, inverse iteration) or W = I when
 * G is nearly diagonal, refined to FP64 accuracy (first-order updates,
 * exact rotations on clusters of close eigenvalues, Newton-Schulz) with the
 * products of opts.f64_gemm.  The FP32 start needs k <= about 5600
 * (EINVAL above). */
int chfsi_rayleigh_ritz(chfsi_ctx* ctx, const double* H, int n, int k,
                        const double* Q, double* Y, double* HY, double* evals);

/* Residuals r_j = ||HY_j - evals_j Y_j||_2 / norm_h (k doubles out). */
int chfsi_residuals(chfsi_ctx* ctx, int n, int k, const double* HY,
                    const double* Y, const double* evals, double norm_h,
                    double* resid);

/* Sec. 3.2 Single Optimization: m_j = ceil(ln(r_j/tol)/acosh|t_j|) +
 * deg_extra, t_j = (ritz_j - c)/e, clamped to [deg_min, deg_max], deg_max
 * when |t_j| <= 1; columns j >= n_wanted are capped at the largest wanted
 * degree.  ritz, resid: k doubles; degrees: k ints (all device). */
int chfsi_degrees(chfsi_ctx* ctx, int k, const double* ritz, const double* resid,
                  double c, double e, double tol, int n_wanted, int* degrees);

/* Tilings the autotuner chose in this context (opts.autotune): 6 ints per
 * entry in entries_host {n, k rounded up to 32, bf16 pieces (2 or 3),
 * column block width, blocks per tile group, time of the winning trial in
 * microseconds}; at most max_entries are written, *n_entries_host gets the
 * total.  The paper has no counterpart: its Sec. 4 tunes the algorithmic
 * block size and the process grid of the distributed GEMMs by hand. */
int chfsi_autotune_table(chfsi_ctx* ctx, int max_entries, int* entries_host,
                         int* n_entries_host);

/* Alg. 1 / Sec. 4 (columns sorted by degree so that the filter runs on a
 * shrinking suffix): stable ascending sort of k columns by degree.
 *  deg         k ints (device), each >= 1.
 *  perm        k ints (device): perm[r] = the column of rank r; equal
 *              degrees keep their column order.
 *  deg_sorted  k ints (device): deg[perm[r]]. */
int chfsi_sort_degrees(chfsi_ctx* ctx, int k, const int* deg, int* perm, int* deg_sorted);

/* Alg. 1 locking, out of order (Sec. 4): among ka active Ritz pairs in
 * ascending order, lock every pair whose residual is <= tol and whose
 * position is below n_wanted_left (= nev - pairs already locked).
 *  ritz, resid  ka doubles each (device).
 *  lock_idx     ka ints (device): positions of the locked pairs, ascending.
 *  act_idx      ka ints (device): positions of the others, ascending.
 *  counts_host  2 ints: {locked, still active}. */
int chfsi_lock(chfsi_ctx* ctx, int ka, const double* ritz, const double* resid,
               int n_wanted_left, double tol, int* lock_idx, int* act_idx, int* counts_host);

/* ---- filter without device allocation ---------------------------------- */

/* Largest n*k accepted by chfsi_filter_static. */
#define CHFSI_FILTER_STATIC_MAX_NK 262144

/* The FP64 Chebyshev filter of chfsi_filter (same arguments and result as
 * precision CHFSI_PREC_FP64), for callers that cannot allocate device
 * memory on the call path: applications that reserve the whole device for
 * their own memory pool at start-up, so a further cudaMalloc fails or
 * fragments that pool, and latency-bound code that cannot accept the
 * implicit device synchronisation of cudaMalloc / cudaFree.  The paper has
 * no counterpart; this is a deployment variant of the filter step.
 *
 * It needs no context and allocates nothing: its three recurrence buffers
 * are one static device array of 3 * CHFSI_FILTER_STATIC_MAX_NK complex128
 * elements (12 MiB) that every GPU which loads this library keeps until the
 * process exits.  Work is issued on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and is stream-ordered; the call returns without
 * synchronising.
 *
 * The first call in each CUDA context of a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and keeps
 * it for that context; after a device reset, or a released and re-created
 * primary context, the next call looks it up again.  Make the first call on
 * a device (and the first after a reset) before any stream capture.  All
 * calls share the one array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race and give wrong
 * results; serialise them.  The buffers are fully written before they are
 * read, so no earlier contents leak into a result.
 *
 * Returns CHFSI_ETOOBIG when n * k > CHFSI_FILTER_STATIC_MAX_NK (no work is
 * issued), CHFSI_EINVAL for the argument errors of chfsi_filter and when Y
 * overlaps Y0 or H in memory, CHFSI_ECUDA when the address lookup or a
 * launch fails. */
int chfsi_filter_static(const double* H, int n, int k, const double* Y0,
                        const int* degrees_host, double lam1, double c, double e,
                        double* Y, void* stream);

/* ---- learned degree predictor (not in the paper) ---------------------- */

/* Traces for training (Alg. 1 degree decisions and their outcome).
 * chfsi_trace_enable(ctx, cap) starts recording, into a device buffer of
 * cap rows owned by the context (cap = 0 stops and frees it): for every
 * active column of every loop after the first, its features (see the MLP
 * below), the degree it was given, its residual before and after that
 * filter.  chfsi_trace_dataset writes the complete rows of wanted columns
 * as training pairs: x (rows x 5 floats, row-major) and y = realised decay
 * per degree / acosh|t| clipped to [0.02, 1.5] (rows floats), both device
 * buffers of max_rows; *n_rows_host gets the number written. */
int chfsi_trace_enable(chfsi_ctx* ctx, int capacity_rows);
int chfsi_trace_dataset(chfsi_ctx* ctx, float* x, float* y, int max_rows, int* n_rows_host);

/* The network: 5 features -> 64 tanh -> 64 tanh -> 1 linear, weights
 * kept in the context as FP32 masters with FP16 copies for the products
 * (FP32 accumulation).  Parameter vector layout (CHFSI_MLP_NPARAM floats):
 * W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3[1]. */
#define CHFSI_MLP_NPARAM (64 * 5 + 64 + 64 * 64 + 64 + 64 + 1)

/* Copy parameters host -> context (resets the optimiser state) / out. */
int chfsi_mlp_set_params(chfsi_ctx* ctx, const float* params_host);
int chfsi_mlp_get_params(chfsi_ctx* ctx, float* params_host);

/* Features of column j: t = (ritz - c)/e; x = {clip(t, -8, 8), log10(r)/10,
 * acosh(max|t|, 1), clip((gamma - c)/e, -8, 8), min(step, 9)/10} (the
 * sequence index saturates at the tenth problem).  The output y is
 * the predicted ratio of the realised decay per degree to acosh|t|; with
 * opts.degree_model = CHFSI_DEG_MLP the solver turns it into
 * m = ceil(ln(max(r, tol)/tol) / (acosh|t| clip(y, 0.02, 1.5))) + mlp_extra,
 * clamped to [4, 60] (60 when |t| <= 1), and uses the analytic rule for a
 * non-finite prediction and for the rest of a problem whose loop did not
 * make progress (nothing locked and the residual fell by less than 10x). */

/* Forward pass: x (B x 5 floats, row-major, device) -> y (B floats). */
int chfsi_mlp_forward(chfsi_ctx* ctx, int B, const float* x, float* y);

/* One training step on a batch: loss = 0.5 mean((y - target)^2), gradients
 * by the backward kernels, then Adam (lr, beta1 0.9, beta2 0.999, eps
 * 1e-8).  grads (CHFSI_MLP_NPARAM floats, device) may be NULL; loss_host
 * may be NULL. */
int chfsi_mlp_train_step(chfsi_ctx* ctx, int B, const float* x, const float* target,
                         float lr, float* grads, float* loss_host);

#ifdef __cplusplus
}
#endif
#endif /* CHFSI_H */
