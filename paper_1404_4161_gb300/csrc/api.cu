// C ABI and solver core of the ChFSI library.
//
// Host-side orchestration of Algorithm 1 (ChFSI) of arXiv 1404.4161 over
// device kernels: Lanczos bounds of the spectrum, the Chebyshev filter of
// Algorithm 2, orthonormalisation against the locked block, Rayleigh-Ritz,
// residuals, locking and degree optimisation.  Every arithmetic step runs in
// this library's kernels, the k x k Cholesky inverse and the Hermitian
// eigensolve of the reduced problems included.  The host only reads a small
// control block per loop (converged count, interval, sorted degrees) to size
// the next launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <vector>

#include "common.cuh"

#include <atomic>

static std::atomic<long long> g_launches{0};
long long chfsi_launch_counter() { return g_launches.load(std::memory_order_relaxed); }
void chfsi_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local KernelTimer* g_kt = nullptr;
KernelTimer* kt_current() { return g_kt; }
void kt_install(KernelTimer* t) { g_kt = t; }

int kt_begin(cudaStream_t st) {
  KernelTimer* t = g_kt;
  if (!t) return -1;
  if ((int)t->ev.size() < 2 * (t->used + 1)) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      CHFSI_CUDA_TRY(cudaEventCreate(&e));
      t->ev.push_back(e);
    }
    t->cat.resize(t->ev.size() / 2);
    t->flops.resize(t->ev.size() / 2);
    t->flops_exec.resize(t->ev.size() / 2);
  }
  const int slot = t->used++;
  CHFSI_CUDA_TRY(cudaEventRecord(t->ev[2 * slot], st));
  return slot;
}

void kt_end(cudaStream_t st, int slot, int cat, double flops, double flops_exec) {
  KernelTimer* t = g_kt;
  if (!t || slot < 0) return;
  CHFSI_CUDA_TRY(cudaEventRecord(t->ev[2 * slot + 1], st));
  t->cat[slot] = cat;
  t->flops[slot] = flops;
  t->flops_exec[slot] = flops_exec < 0.0 ? flops : flops_exec;
}

void kt_resolve(KernelTimer* t) {
  if (!t) return;
  for (int i = 0; i < t->used; ++i) {
    float ms = 0.f;
    CHFSI_CUDA_TRY(cudaEventElapsedTime(&ms, t->ev[2 * i], t->ev[2 * i + 1]));
    t->ms[t->cat[i]] += ms;
    t->fl[t->cat[i]] += t->flops[i];
    t->fx[t->cat[i]] += t->flops_exec[i];
    t->n[t->cat[i]] += 1;
  }
  t->used = 0;
}

// ===================================================== workspace & ctx ====
void* ws_get(chfsi_ctx* ctx, const char* name, size_t bytes) {
  DevBuf& b = ctx->ws[name];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) CHFSI_CUDA_TRY(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    const size_t want = (bytes + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      b.p = nullptr;
      throw ChfsiError{CHFSI_ENOMEM, std::string("cudaMalloc(") + name + ", " +
                                         std::to_string(want) + " B) failed"};
    }
    b.bytes = want;
  }
  return b.p;
}

void ws_free_all(chfsi_ctx* ctx) {
  for (auto& kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  ctx->ws.clear();
}

void* pinned_get(chfsi_ctx* ctx, size_t bytes) {
  if (ctx->pinned_bytes < bytes) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    const size_t want = std::max<size_t>(bytes, 1 << 16);
    CHFSI_CUDA_TRY(cudaHostAlloc(&ctx->pinned, want, cudaHostAllocDefault));
    ctx->pinned_bytes = want;
  }
  return ctx->pinned;
}

namespace {

int run_guarded(chfsi_ctx* ctx, const std::function<void()>& body);

void validate_opts(const chfsi_opts& o) {
  CHFSI_REQUIRE(o.precision == CHFSI_PREC_FP64 || o.precision == CHFSI_PREC_MIXED ||
                    o.precision == CHFSI_PREC_TC,
                "opts.precision");
  CHFSI_REQUIRE(o.split == CHFSI_SPLIT_BF16X3 || o.split == CHFSI_SPLIT_BF16X6 ||
                    o.split == CHFSI_SPLIT_ADAPTIVE,
                "opts.split");
  CHFSI_REQUIRE(o.degree_model == CHFSI_DEG_ANALYTIC || o.degree_model == CHFSI_DEG_MLP,
                "opts.degree_model");
  CHFSI_REQUIRE(o.deg_min >= 1 && o.deg_max >= o.deg_min && o.deg_max <= 512,
                "opts.deg_min/deg_max");
  CHFSI_REQUIRE(o.deg_cold >= 1 && o.deg_warm >= 1, "opts.deg_cold/deg_warm");
  CHFSI_REQUIRE(o.deg_extra >= 0, "opts.deg_extra");
  CHFSI_REQUIRE(o.lanczos_steps >= 2 && o.lanczos_steps <= 200, "opts.lanczos_steps");
  CHFSI_REQUIRE(o.max_loops >= 1, "opts.max_loops");
  CHFSI_REQUIRE(o.switch_tol > 0.0, "opts.switch_tol");
  CHFSI_REQUIRE(o.mlp_extra >= 0 && o.step0 >= 0, "opts.mlp_extra/step0");
  CHFSI_REQUIRE((o.warm_rr == 0 || o.warm_rr == 1) && (o.warm_resid == 0 || o.warm_resid == 1),
                "opts.warm_rr/warm_resid");
  CHFSI_REQUIRE(o.autotune == 0 || o.autotune == 1, "opts.autotune");
  CHFSI_REQUIRE(o.f64_gemm == CHFSI_GEMM_FP64 || o.f64_gemm == CHFSI_GEMM_OZAKI,
                "opts.f64_gemm");
}

inline double2* C2(double* p) { return reinterpret_cast<double2*>(p); }
inline const double2* C2(const double* p) { return reinterpret_cast<const double2*>(p); }

// ------------------------------------------------------------ Lanczos ----
// out4_dev = {beta, theta_min, theta_max, norm_h} (device).
// ------------------------------------------------------- FP64 filter ----
void filter_f64(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y0,
                const int* deg, double lam1, double c, double e, double2* Yout) {
  const size_t blk = sizeof(double2) * (size_t)n * k;
  double2* F[3] = {(double2*)ws_get(ctx, "flt0", blk), (double2*)ws_get(ctx, "flt1", blk),
                   (double2*)ws_get(ctx, "flt2", blk)};
  filter_f64_recurrence(ctx->stream, H, n, k, Y0, deg, lam1, c, e, Yout, F);
}

// ------------------------------------------------ FP64 product engines ----
bool use_oz(chfsi_ctx* ctx) { return ctx->opts.f64_gemm == CHFSI_GEMM_OZAKI; }

// C = alpha A^H B + beta C
void gemm_cn(chfsi_ctx* ctx, int K1, int K2, int Nr, const double2* A, int lda,
             const double2* B, int ldb, double2* C, int ldc, double alpha = 1.0,
             double beta = 0.0) {
  if (use_oz(ctx))
    oz_gemm_cn(ctx, K1, K2, Nr, A, lda, B, ldb, C, ldc, alpha, beta);
  else
    zgemm_cn(ctx, K1, K2, Nr, A, lda, B, ldb, C, ldc, alpha, beta);
}

// C = alpha A B + beta C (C may be the same buffer as the beta term only)
// (oz_ns: slices of the tensor-core engine, 0 = by the product's size)
void gemm_nn(chfsi_ctx* ctx, int M, int N, int K, const double2* A, int lda, const double2* B,
             int ldb, double2* C, int ldc, double alpha = 1.0, double beta = 0.0,
             int oz_ns = 0) {
  if (use_oz(ctx)) {
    oz_gemm_nn(ctx, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, oz_ns);
    return;
  }
  EpiNN ep;
  ep.alpha = alpha;
  ep.beta = beta;
  ep.P = beta != 0.0 ? C : nullptr;
  ep.ldp = ldc;
  ep.D = C;
  ep.ldd = ldc;
  zgemm_nn(ctx->stream, M, N, K, A, lda, B, ldb, ep);
}

// ------------------------------------------------- orthonormalisation ----
// Y <- Y (I - F)^{-1/2} for the Hermitian F = I - Y^H Y with ||F||_F = f <
// 1: the binomial series sum_m c_m F^m, c_0 = 1, c_m = c_{m-1} (2m-1)/(2m),
// summed by Horner's rule to the first M with f^{M+1} / (1 - f) <= 2^-53,
// so Y^H Y = I to rounding.  This is the symmetric (polar) orthonormal
// basis of span(Y); its first-order term is the Newton-Schulz step
// (3I - Y^H Y)/2.
void polar_orthonormalize(chfsi_ctx* ctx, int n, int k, double2* Y, const double2* F, double f) {
  cudaStream_t st = ctx->stream;
  int M = 0;
  while (M < 60 && std::pow(f, M + 1) / (1.0 - f) > 0x1p-53) ++M;
  if (M == 0) return;
  std::vector<double> c(M + 1);
  c[0] = 1.0;
  for (int m = 1; m <= M; ++m) c[m] = c[m - 1] * (2.0 * m - 1.0) / (2.0 * m);
  double2* W = (double2*)ws_get(ctx, "pol_W", sizeof(double2) * (size_t)k * k);
  double2* Tk = (double2*)ws_get(ctx, "pol_T", sizeof(double2) * (size_t)k * k);
  shift_identity(st, k, nullptr, c[M], W);
  // the k x k products take the slice count of the problem's n-sized ones
  const int ns = oz_slices_for(n);
  for (int m = M - 1; m >= 0; --m) {
    gemm_nn(ctx, k, k, k, F, k, W, k, Tk, k, 1.0, 0.0, ns);  // F W
    shift_identity(st, k, Tk, c[m], W);                      // c_m I + F W
  }
  double2* T = (double2*)ws_get(ctx, "qr_T", sizeof(double2) * (size_t)n * k);
  gemm_nn(ctx, n, k, k, Y, n, W, k, T, n);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(Y, T, sizeof(double2) * (size_t)n * k, cudaMemcpyDeviceToDevice,
                                 st));
}

// The QR step of Alg. 1 on the device: two block Gram-Schmidt passes against the
// locked block, column normalisation, then CholQR2 (a shifted Cholesky QR
// pass first when the Gram matrix is not numerically positive definite).
//
// adaptive (the solver with the tensor-core FP64 products): the first
// Cholesky pass runs in FP32 arithmetic -- it only has to precondition the
// block -- and the second is replaced by the polar correction above when
// ||I - Y^H Y||_F <= 0.1 after it.  The result is then an orthonormal
// basis of the same span (not the Cholesky one), which is all that
// Rayleigh-Ritz needs.  When the FP32 factorisation breaks down or leaves
// the block further from orthonormal, the FP64 CholQR2 below takes over.
void orthonormalize_dev(chfsi_ctx* ctx, int n, int nl, const double2* L, int k, double2* Y,
                        bool adaptive = false) {
  cudaStream_t st = ctx->stream;
  if (k <= 0) return;
  // Y -= L (L^H Y).  Whatever is left along L (rounding, ~u ||Y||) is
  // multiplied by ||R^-1|| ~ 1/sigma_min(Y) in the first Cholesky pass, so
  // one more projection follows that pass (the block is well conditioned
  // by then and the second pass keeps what it leaves).
  auto project = [&](int passes) {
    if (nl <= 0) return;
    double2* P = (double2*)ws_get(ctx, "qr_P", sizeof(double2) * (size_t)nl * k);
    for (int pass = 0; pass < passes; ++pass) {
      gemm_cn(ctx, nl, k, n, L, n, Y, n, P, nl);
      gemm_nn(ctx, n, k, nl, L, n, P, nl, Y, n, -1.0, 1.0);
    }
  };
  project(2);
  double* cn = (double*)ws_get(ctx, "qr_cn", sizeof(double) * k);
  column_norms(st, n, k, Y, n, cn);
  scale_columns_inv(st, n, k, Y, n, cn);
  double2* G = (double2*)ws_get(ctx, "qr_G", sizeof(double2) * (size_t)k * k);
  double2* T = (double2*)ws_get(ctx, "qr_T", sizeof(double2) * (size_t)n * k);
  if (adaptive) {
    gemm_cn(ctx, k, k, n, Y, n, Y, n, G, k);
    hermitianize(st, k, G, k);
    if (cholinv_upper_f32(ctx, k, G) == 0) {
      gemm_nn(ctx, n, k, k, Y, n, G, k, T, n);
      CHFSI_CUDA_TRY(cudaMemcpyAsync(Y, T, sizeof(double2) * (size_t)n * k,
                                     cudaMemcpyDeviceToDevice, st));
      project(1);
      gemm_cn(ctx, k, k, n, Y, n, Y, n, G, k);
      hermitianize(st, k, G, k);
      double2* F = (double2*)ws_get(ctx, "qr_F", sizeof(double2) * (size_t)k * k);
      const double f = identity_defect(ctx, k, G, F);
      if (f <= 0.1) {
        polar_orthonormalize(ctx, n, k, Y, F, f);
        return;
      }
    }
  }
  double* shift = (double*)ws_get(ctx, "qr_shift", sizeof(double));
  int passes = 2;
  bool shifted = false;
  for (int pass = 0; pass < passes; ++pass) {
    gemm_cn(ctx, k, k, n, Y, n, Y, n, G, k);
    hermitianize(st, k, G, k);
    if (shifted && pass == 0) {
      cholqr_shift(st, n, k, G, k, shift);
      add_diag(st, k, G, k, shift);
    }
    int info = cholinv_upper(ctx, k, G);  // G <- R^{-1}, R^H R = G
    if (info != 0) {
      if (pass == 0 && !shifted) {
        shifted = true;
        passes = 3;
        pass = -1;  // restart with the shifted first pass
        continue;
      }
      throw ChfsiError{CHFSI_EBREAKDOWN, "CholQR: Gram matrix not positive definite (info " +
                                             std::to_string(info) + ")"};
    }
    gemm_nn(ctx, n, k, k, Y, n, G, k, T, n);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(Y, T, sizeof(double2) * (size_t)n * k,
                                   cudaMemcpyDeviceToDevice, st));
    if (pass < passes - 1) project(1);
    if (adaptive && pass == passes - 2) {
      // Before the last pass: when the block is already orthonormal to
      // 1e-8, one Newton-Schulz step Y (3I - Y^H Y)/2 leaves it orthonormal
      // to the Gram's accuracy (error ~ the square of 1e-8) and replaces the
      // last Cholesky pass.
      gemm_cn(ctx, k, k, n, Y, n, Y, n, G, k);
      if (deviation_from_identity(ctx, k, G) <= 1e-8) {
        ns_matrix(st, k, G, G);
        gemm_nn(ctx, n, k, k, Y, n, G, k, T, n);
        CHFSI_CUDA_TRY(cudaMemcpyAsync(Y, T, sizeof(double2) * (size_t)n * k,
                                       cudaMemcpyDeviceToDevice, st));
        break;
      }
    }
  }
}

// ----------------------------------------------------- Rayleigh-Ritz ----
void rayleigh_ritz_dev(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Q,
                       double2* Y, double2* HY, double* evals, const std::string& hprefix = "",
                       bool* h_sliced = nullptr) {
  cudaStream_t st = ctx->stream;
  double2* Z = (double2*)ws_get(ctx, "rr_Z", sizeof(double2) * (size_t)n * k);
  double2* G = (double2*)ws_get(ctx, "rr_G", sizeof(double2) * (size_t)k * k);
  if (use_oz(ctx)) {
    const bool fresh = !(h_sliced && *h_sliced);
    oz_hemm(ctx, hprefix, H, n, Q, k, Z, fresh);
    if (h_sliced) *h_sliced = true;
  } else {
    EpiNN ep;
    ep.D = Z;
    ep.ldd = n;
    zgemm_nn(st, n, k, n, H, n, Q, n, ep);
  }
  gemm_cn(ctx, k, k, n, Q, n, Z, n, G, k);
  hermitianize(st, k, G, k);
  // The reduced eigensolver is iterative: never hand it NaN or Inf.
  if (any_nonfinite(ctx, (size_t)2 * k * k, (const double*)G))
    throw ChfsiError{CHFSI_ENAN, "NaN/Inf in the Rayleigh quotient"};
  reduced_eigh_mixed(ctx, k, G, evals, !use_oz(ctx));
  gemm_nn(ctx, n, k, k, Q, n, G, k, Y, n);
  gemm_nn(ctx, n, k, k, Z, n, G, k, HY, n);
}

// ------------------------------------------------- one problem's state --
// Alg. 1 for one problem, split into phases so that several problems can
// share a batched filter launch: init (checks, Lanczos, interval), filter,
// post (QR, Rayleigh-Ritz, residuals, locking, degrees), finish (output).
struct Problem {
  chfsi_ctx* ctx = nullptr;
  const chfsi_opts* o = nullptr;
  cudaStream_t st = nullptr;
  std::string pre;  // workspace-name prefix (one per concurrent problem)
  const double2* H = nullptr;
  int n = 0, nev = 0, nex = 0, k = 0, step = 0;
  double2* X = nullptr;
  double* evals_out = nullptr;
  double tol = 0.0;
  chfsi_stats* stats_out = nullptr;
  bool mixed = false, tc_all = false;
  double2 *Xact = nullptr, *Yf = nullptr, *Yrr = nullptr, *HY = nullptr, *Lk = nullptr,
          *Rblk = nullptr;
  double *lam = nullptr, *res = nullptr, *lamL = nullptr, *resL = nullptr, *lam_act = nullptr,
         *bnd = nullptr;
  int *lock_idx = nullptr, *act_idx = nullptr, *deg = nullptr, *perm = nullptr,
      *deg_sorted = nullptr;
  LoopCtl* ctl = nullptr;
  double beta = 0, norm_h = 0, alpha = 0, gamma = 0, max_resid_wanted = INFINITY;
  int ka = 0, nl = 0, loops = 0, status = CHFSI_ENOCONV;
  bool use_mlp = false, lowp_on = false, done = false, warm_start = false;
  std::vector<int> degs;
  chfsi_stats S;
  long long launches0 = 0, fl0 = 0;
  long long sdeg = 0;
  cudaEvent_t ev[9] = {};
  double* psi = nullptr;  // refinement tables of the current loop
  double* fR = nullptr;
  bool h_sliced = false;  // tensor-core slices of H built for this problem
  int slot = 0;           // operand slot of the tensor-core filter
  bool have_R = false;    // residual block of the current Ritz pairs built

  void* ws(const char* name, size_t bytes) { return ws_get(ctx, (pre + name).c_str(), bytes); }
  void mark(int i) { CHFSI_CUDA_TRY(cudaEventRecord(ev[i], st)); }
  double ms(int a, int b) {
    float t = 0.f;
    CHFSI_CUDA_TRY(cudaEventElapsedTime(&t, ev[a], ev[b]));
    return (double)t;
  }
  ~Problem() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }

  void init(chfsi_ctx* c, const std::string& prefix, const double2* H_, int n_, int nev_,
            int nex_, double2* X_, double tol_, double* evals_, const double* warm,
            chfsi_stats* stats_, int step_) {
    ctx = c;
    o = &ctx->opts;
    st = ctx->stream;
    pre = prefix;
    H = H_;
    n = n_;
    nev = nev_;
    nex = nex_;
    k = nev + nex;
    X = X_;
    tol = tol_;
    evals_out = evals_;
    stats_out = stats_;
    step = step_;
    CHFSI_REQUIRE(H && X && evals_out, "NULL buffer");
    CHFSI_REQUIRE(nev >= 1 && nex >= 1 && k <= n, "need 1 <= nev, 1 <= nex, nev + nex <= n");
    CHFSI_REQUIRE(tol > 0.0, "tol must be > 0");
    mixed = o->precision == CHFSI_PREC_MIXED;
    tc_all = o->precision == CHFSI_PREC_TC;
    if ((mixed || tc_all) && !tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
    std::memset(&S, 0, sizeof(S));
    launches0 = chfsi_launch_counter();
    for (auto& e : ev) CHFSI_CUDA_TRY(cudaEventCreate(&e));
    mark(0);
    const size_t blk = sizeof(double2) * (size_t)n * k;
    Xact = (double2*)ws("s_Xact", blk);
    Yf = (double2*)ws("s_Yf", blk);
    Yrr = (double2*)ws("s_Yrr", blk);
    HY = (double2*)ws("s_HY", blk);
    Lk = (double2*)ws("s_Lk", sizeof(double2) * (size_t)n * nev);
    lam = (double*)ws("s_lam", sizeof(double) * k);
    res = (double*)ws("s_res", sizeof(double) * k);
    lamL = (double*)ws("s_lamL", sizeof(double) * nev);
    resL = (double*)ws("s_resL", sizeof(double) * nev);
    Rblk = tc_all ? (double2*)ws("s_Rblk", blk) : nullptr;
    lam_act = (double*)ws("s_lamact", sizeof(double) * k);
    int* iws = (int*)ws("s_int", sizeof(int) * 5 * (size_t)k);
    lock_idx = iws;
    act_idx = iws + k;
    deg = iws + 2 * k;
    perm = iws + 3 * k;
    deg_sorted = iws + 4 * k;
    bnd = (double*)ws("s_bnd", sizeof(double) * 4);
    ctl = (LoopCtl*)ws("s_ctl", sizeof(LoopCtl));
    char* hp = (char*)pinned_get(ctx, 1024 + sizeof(int) * (size_t)k + sizeof(double) * k);
    double* bnd_h = (double*)(hp + 512);

    if (any_nonfinite(ctx, (size_t)2 * n * k, (const double*)X))
      throw ChfsiError{CHFSI_ENAN, "NaN/Inf in the starting block"};
    if (any_nonfinite(ctx, (size_t)2 * n * n, (const double*)H))
      throw ChfsiError{CHFSI_ENAN, "NaN/Inf in H"};
    // Alg. 1: bounds of the spectrum (Lanczos, Sec. 3.1).
    lanczos_dev(ctx, H, n, o->lanczos_steps, o->seed, bnd);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(bnd_h, bnd, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    int* lz_err_h = (int*)(hp + 640);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(lz_err_h, lanczos_error_word(ctx), sizeof(int),
                                   cudaMemcpyDeviceToHost, st));
    mark(1);
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    if (*lz_err_h)
      throw ChfsiError{CHFSI_ETIMEOUT, "Lanczos: a bounded grid barrier gave up (code " +
                                           std::to_string(*lz_err_h) + ")"};
    S.ms_lanczos = ms(0, 1);
    beta = bnd_h[0];
    norm_h = bnd_h[3];
    if (!std::isfinite(beta) || !std::isfinite(norm_h) || norm_h <= 0.0)
      throw ChfsiError{CHFSI_ENAN, "Lanczos bounds are not finite"};
    S.beta = beta;
    S.norm_h = norm_h;
    // split pieces of H for the tensor-core filter, once per problem
    if (mixed || tc_all)
      tc_filter_prepare(ctx, slot, H, n, o->split == CHFSI_SPLIT_BF16X3 ? 2 : 3);
    int deg0;
    if (warm) {
      warm_start = true;
      gamma = warm[0];
      alpha = warm[1];
      deg0 = o->deg_warm;
    } else {
      gamma = bnd_h[1];
      alpha = gamma + (beta - gamma) * (double)k / (double)n;
      deg0 = o->deg_cold;
    }
    CHFSI_REQUIRE(alpha < beta, "filter interval is empty (alpha >= beta)");
    copy_columns(st, n, k, X, n, Xact, n);
    degs.assign(k, deg0);
    ka = k;
    nl = 0;
    use_mlp = o->degree_model == CHFSI_DEG_MLP;
    trace_abandon(ctx);
    lowp_on = mixed;
    if (warm && o->warm_rr) {
      // Rayleigh-Ritz on the (orthonormal) warm block: residuals, locking
      // and degrees are known before the first filter.
      mark(3);
      mark(4);
      rayleigh_ritz_dev(ctx, H, n, ka, Xact, Yrr, HY, lam, pre, &h_sliced);
      mark(5);
      residual_norms(st, n, ka, HY, Yrr, lam, norm_h, res);
      mark(6);
      after_rr();
      S.ms_rr += ms(4, 5);
    } else if (warm && o->warm_resid) {
      // The warm block (the previous problem's Ritz vectors, orthonormal)
      // on the new H: its Rayleigh quotients and residuals from one product
      // H X, without a reduced eigensolve.  Converged pairs lock at once,
      // the first loop gets per-vector degrees from the rule of Sec. 3.2,
      // and with CHFSI_PREC_TC the refinement form of the filter, which
      // holds for any diagonal of shifts.
      mark(3);
      mark(4);
      hx_product(Xact, Yf);  // Yf <- H Xact (scratch)
      rayleigh_quotients(st, n, ka, Yf, Xact, res);
      sort_by_value(st, ka, res, perm);
      gather_values(st, ka, res, perm, lam);
      gather_columns(st, n, ka, Xact, n, perm, Yrr, n);
      gather_columns(st, n, ka, Yf, n, perm, HY, n);
      mark(5);
      residual_norms(st, n, ka, HY, Yrr, lam, norm_h, res);
      mark(6);
      after_rr();
      S.ms_rr += ms(4, 5);
    }
  }

  // Z = H Y (n x ka) with the engine of the FP64 products; the tensor-core
  // slices of H are made once per problem and shared with Rayleigh-Ritz.
  void hx_product(const double2* Y, double2* Z) {
    if (use_oz(ctx)) {
      oz_hemm(ctx, pre, H, n, Y, ka, Z, !h_sliced);
      h_sliced = true;
    } else {
      EpiNN ep;
      ep.D = Z;
      ep.ldd = n;
      zgemm_nn(st, n, ka, n, H, n, Y, n, ep);
    }
  }

  double c_() const { return 0.5 * (alpha + beta); }
  double e_() const { return 0.5 * (beta - alpha); }

  // Start of a loop: which filter this problem's loop uses.
  enum FilterKind { F64 = 0, TC_PLAIN = 1, TC_DEFECT = 2 };
  FilterKind begin_loop() {
    ++loops;
    if (lowp_on && !(max_resid_wanted > o->switch_tol)) lowp_on = false;
    sdeg = 0;
    for (int j = 0; j < ka; ++j) sdeg += degs[j];
    mark(2);
    fl0 = chfsi_launch_counter();
    if (tc_all) return have_R ? TC_DEFECT : TC_PLAIN;
    if (lowp_on) return TC_PLAIN;
    return F64;
  }

  // bf16 pieces of the tensor-core filter in this loop.  Adaptive: the
  // refinement form's error is about 2^-16 x 1.7 times the residual with two
  // pieces (3 products); three pieces (6 products) while that would not
  // stay below a third of tol.
  int split_pieces(FilterKind kind) const {
    if (o->split == CHFSI_SPLIT_BF16X3) return 2;
    if (o->split == CHFSI_SPLIT_BF16X6) return 3;
    return (kind == TC_DEFECT && max_resid_wanted * 1.7 * 0x1p-16 > tol / 3.0) ? 3 : 2;
  }

  // The filter of this loop run by this problem alone.
  void filter_single(FilterKind kind) {
    if (kind == F64) {
      filter_f64(ctx, H, n, ka, Xact, degs.data(), gamma, c_(), e_(), Yf);
      return;
    }
    TcBatchItem it = batch_item(kind);
    tc_filter_launch(ctx, 1, &it, split_pieces(kind));
    after_batch(kind);
  }

  // Work item of this loop's filter for a batched launch.
  TcBatchItem batch_item(FilterKind kind) {
    TcBatchItem it;
    it.H = H;
    it.n = n;
    it.k = ka;
    it.src = Xact;
    it.R = nullptr;
    it.fR = nullptr;
    it.deg = degs.data();
    it.lam1 = gamma;
    it.c = c_();
    it.e = e_();
    it.out = Yf;
    it.slot = slot;
    it.h_ready = true;
    if (kind == TC_DEFECT) {
      tc_defect_tables(ctx, pre, ka, lam_act, degs.data(), gamma, c_(), e_(), &psi, &fR);
      it.R = Rblk;
      it.fR = fR;
    }
    return it;
  }
  void after_batch(FilterKind kind) {
    if (kind == TC_DEFECT) tc_defect_combine(st, n, ka, Xact, deg_sorted, psi, Yf);
  }

  // Rest of the loop; sets done when nev pairs are locked.
  void post(FilterKind kind) {
    if (kind != F64) {
      S.loops_lowp++;
      S.col_degrees_lowp += sdeg;
    }
    S.col_degrees += sdeg;
    S.filter_launches += chfsi_launch_counter() - fl0;
    mark(3);
    orthonormalize_dev(ctx, n, nl, Lk, ka, Yf, use_oz(ctx));
    mark(4);
    rayleigh_ritz_dev(ctx, H, n, ka, Yf, Yrr, HY, lam, pre, &h_sliced);
    mark(5);
    residual_norms(st, n, ka, HY, Yrr, lam, norm_h, res);
    trace_finish(ctx, ka, res);
    mark(6);
    after_rr();
    S.ms_filter += ms(2, 3);
    S.ms_qr += ms(3, 4);
    S.ms_rr += ms(4, 5);
    S.ms_resid += ms(5, 6);
    S.ms_lock += ms(6, 7);
  }

  // Locking, interval update, degrees and sort after a Rayleigh-Ritz step.
  void after_rr() {
    lock_select(st, ka, lam, res, nev - nl, tol, gamma, ctl, lock_idx, act_idx);
    char* hp = (char*)pinned_get(ctx, 1024 + sizeof(int) * (size_t)k + sizeof(double) * k);
    LoopCtl* ctl_h = (LoopCtl*)(hp + 256);
    int* deg_h = (int*)(hp + 1024);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(ctl_h, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, st));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    if (use_oz(ctx)) {
      const int e = oz_check_error(ctx);
      if (e)
        throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up (code " +
                                             std::to_string(e) + ")"};
    }
    if (ctl_h->nonfinite) throw ChfsiError{CHFSI_ENAN, "NaN/Inf in Ritz values or residuals"};
    const int n_new = ctl_h->n_new_locked;
    gather_columns(st, n, n_new, Yrr, n, lock_idx, Lk + (size_t)nl * n, n);
    gather_values(st, n_new, lam, lock_idx, lamL + nl);
    gather_values(st, n_new, res, lock_idx, resL + nl);
    nl += n_new;
    ka = ctl_h->k_active;
    gamma = ctl_h->gamma;
    // The learned degrees stall: nothing locked and the residual fell by
    // less than 10x -> the analytic rule for the rest of this problem.
    if (use_mlp && S.loops_mlp > 0 && n_new == 0 &&
        ctl_h->max_resid_wanted > 0.1 * max_resid_wanted) {
      use_mlp = false;
      S.mlp_fallback = 1;
    }
    max_resid_wanted = ctl_h->max_resid_wanted;
    if (verbose()) log_loop(n_new, ctl_h);
    if (nl >= nev) {
      status = CHFSI_OK;
      done = true;
      mark(7);
      CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      // Courant-Fischer makes the largest Ritz value of the block an upper
      // bound of lambda_k; on a warm start the interval keeps the tightest
      // bound seen (the previous problem's lambda_k first), so that a buffer
      // column the low-precision filter spoiled cannot push alpha up.
      alpha = warm_start ? std::min(alpha, ctl_h->alpha) : ctl_h->alpha;
      const double c2 = c_(), e2 = e_();
      // First loop of a warm start from the residuals of the starting block
      // (opts.warm_resid): the buffer columns keep the uniform deg_warm (a
      // higher degree makes them near combinations of the amplified wanted
      // directions, an ill-conditioned block).
      const bool warm_first = warm_start && loops == 0;
      const int bcap = warm_first ? o->deg_warm : (1 << 30);
      const int extra = o->deg_extra;
      if (use_mlp) {
        mlp_degrees(ctx, ka, lam, res, act_idx, c2, e2, gamma, step, tol, deg);
        degree_cap_buffer(st, ka, nev - nl, deg, bcap);
        S.loops_mlp++;
      } else {
        degrees_analytic(st, ka, lam, res, act_idx, c2, e2, tol, nev - nl, o->deg_min,
                         o->deg_max, extra, deg, bcap);
      }
      trace_record(ctx, ka, lam, res, act_idx, deg, c2, e2, gamma, step, nev - nl);
      sort_by_degree(st, ka, deg, act_idx, perm, deg_sorted);
      gather_columns(st, n, ka, Yrr, n, perm, Xact, n);
      if (tc_all) {
        residual_block(st, n, ka, HY, Yrr, lam, perm, Rblk, lam_act);
        have_R = true;
      }
      CHFSI_CUDA_TRY(cudaMemcpyAsync(deg_h, deg_sorted, sizeof(int) * ka,
                                     cudaMemcpyDeviceToHost, st));
      mark(7);
      CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
      degs.assign(deg_h, deg_h + ka);
      if (loops >= o->max_loops) done = true;
    }
  }

  // CHFSI_VERBOSE=1: one line per loop on stderr (diagnostics only).
  static bool verbose() {
    static const bool v = [] {
      const char* e = std::getenv("CHFSI_VERBOSE");
      return e && e[0] == '1';
    }();
    return v;
  }
  void log_loop(int n_new, const LoopCtl* c) {
    std::vector<double> r(ka + n_new);
    CHFSI_CUDA_TRY(cudaMemcpy(r.data(), res, sizeof(double) * r.size(), cudaMemcpyDeviceToHost));
    std::vector<double> l(ka + n_new);
    CHFSI_CUDA_TRY(cudaMemcpy(l.data(), lam, sizeof(double) * l.size(), cudaMemcpyDeviceToHost));
    const int nw = std::min((int)r.size(), nev - (nl - n_new));
    std::vector<double> w(r.begin(), r.begin() + std::max(nw, 0));
    std::sort(w.begin(), w.end());
    int worst = 0;
    for (int j = 1; j < nw; ++j)
      if (r[j] > r[worst]) worst = j;
    std::fprintf(stderr,
                 "[chfsi] step %d loop %d n %d k_act %d locked %d (+%d) wanted resid: min %.2e "
                 "med %.2e max %.2e (col %d, ritz %.6f) alpha %.4f gamma %.4f sum_deg %lld\n",
                 step, loops, n, (int)r.size(), nl, n_new, w.empty() ? 0.0 : w.front(),
                 w.empty() ? 0.0 : w[w.size() / 2], w.empty() ? 0.0 : w.back(), worst,
                 nw > 0 ? l[worst] : 0.0, c->alpha, c->gamma, sdeg);
  }

  // Output: locked pairs ascending, then the remaining active block.
  int finish() {
    int* permL = perm;
    sort_by_value(st, nl, lamL, permL);
    gather_columns(st, n, nl, Lk, n, permL, X, n);
    gather_values(st, nl, lamL, permL, evals_out);
    gather_columns(st, n, ka, Yrr, n, act_idx, X + (size_t)nl * n, n);
    gather_values(st, ka, lam, act_idx, evals_out + nl);
    char* hp = (char*)pinned_get(ctx, 1024 + sizeof(int) * (size_t)k + sizeof(double) * k);
    double* rl_h = (double*)(hp + 1024);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(rl_h, resL, sizeof(double) * std::max(nl, 1),
                                   cudaMemcpyDeviceToHost, st));
    mark(8);
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    double mr = 0.0;
    for (int j = 0; j < std::min(nl, nev); ++j) mr = std::max(mr, rl_h[j]);
    S.max_resid = (nl >= nev) ? mr : INFINITY;
    S.loops = loops;
    S.n_locked = nl;
    S.status = status;
    S.ms_total = ms(0, 8);
    S.filter_flops = 8.0 * (double)n * (double)n * (double)S.col_degrees;
    S.launches = chfsi_launch_counter() - launches0;
    return status;
  }
};

void copy_kernel_times(chfsi_stats& S, const KernelTimer& t) {
  S.k_f64_ms = t.ms[KT_F64];
  S.k_f64_flops = t.fl[KT_F64];
  S.k_f64_launches = t.n[KT_F64];
  S.k_tc_ms = t.ms[KT_TC];
  S.k_tc_flops = t.fl[KT_TC];
  S.k_tc_launches = t.n[KT_TC];
  S.k_solver_ms = t.ms[KT_SOLVER];
  S.k_solver_calls = t.n[KT_SOLVER];
  S.k_f64_exec_flops = t.fx[KT_F64];
  S.k_cholinv_ms = t.ms[KT_CHOLINV];
  S.k_lanczos_ms = t.ms[KT_LANCZOS];
  S.k_slice_ms = t.ms[KT_SLICE];
  S.k_eigctl_ms = t.ms[KT_EIGCTL];
  S.k_tc_exec_flops = t.fx[KT_TC];
}

struct TimerScope {
  KernelTimer* t;
  explicit TimerScope(KernelTimer* x) : t(x) { kt_install(x); }
  ~TimerScope() {
    kt_install(nullptr);
    if (t)
      for (auto e : t->ev) cudaEventDestroy(e);
  }
};

int solve_one(chfsi_ctx* ctx, const double2* H, int n, int nev, int nex, double2* X,
              double tol, double* evals_out, const double* warm, chfsi_stats* stats,
              int step) {
  KernelTimer timer;
  TimerScope scope(ctx->opts.profile ? &timer : nullptr);
  Problem pb;
  pb.init(ctx, "", H, n, nev, nex, X, tol, evals_out, warm, stats, step);
  while (!pb.done && pb.loops < ctx->opts.max_loops) {
    const Problem::FilterKind kind = pb.begin_loop();
    pb.filter_single(kind);
    pb.post(kind);
    if (ctx->opts.profile) kt_resolve(&timer);
  }
  const int status = pb.finish();
  if (ctx->opts.profile) {
    kt_resolve(&timer);
    copy_kernel_times(pb.S, timer);
  }
  if (stats) *stats = pb.S;
  return status;
}

// P independent problems in lockstep: one batched tensor-core filter launch
// per loop for every problem whose loop uses the split-precision filter,
// then each problem's QR, Rayleigh-Ritz and locking.
int solve_batch(chfsi_ctx* ctx, int P, const double2* const* H, const int* n, const int* nev,
                const int* nex, double2* const* X, double tol, double* const* evals,
                const double* warm /* 2P or null */, chfsi_stats* stats, int step,
                double* ms_filter_total) {
  KernelTimer timer;
  TimerScope scope(ctx->opts.profile ? &timer : nullptr);
  std::vector<Problem> pbs(P);
  for (int p = 0; p < P; ++p) {
    pbs[p].slot = p;
    pbs[p].init(ctx, "b" + std::to_string(p) + ".", H[p], n[p], nev[p], nex[p], X[p], tol,
                evals[p], warm ? warm + 2 * p : nullptr, stats ? stats + p : nullptr, step);
  }
  cudaEvent_t e0, e1;
  CHFSI_CUDA_TRY(cudaEventCreate(&e0));
  CHFSI_CUDA_TRY(cudaEventCreate(&e1));
  double filt_ms = 0.0;
  for (;;) {
    std::vector<int> act;
    for (int p = 0; p < P; ++p)
      if (!pbs[p].done && pbs[p].loops < ctx->opts.max_loops) act.push_back(p);
    if (act.empty()) break;
    std::vector<Problem::FilterKind> kind(P, Problem::F64);
    std::vector<TcBatchItem> items;
    std::vector<int> in_batch;
    int ns = 2;
    for (int p : act) {
      kind[p] = pbs[p].begin_loop();
      if (kind[p] != Problem::F64) {
        items.push_back(pbs[p].batch_item(kind[p]));
        in_batch.push_back(p);
        ns = std::max(ns, pbs[p].split_pieces(kind[p]));
      }
    }
    CHFSI_CUDA_TRY(cudaEventRecord(e0, ctx->stream));
    if (!items.empty()) tc_filter_launch(ctx, (int)items.size(), items.data(), ns);
    for (int p : in_batch) pbs[p].after_batch(kind[p]);
    for (int p : act)
      if (kind[p] == Problem::F64) pbs[p].filter_single(kind[p]);
    CHFSI_CUDA_TRY(cudaEventRecord(e1, ctx->stream));
    CHFSI_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    CHFSI_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    filt_ms += t;
    for (int p : act) pbs[p].post(kind[p]);
    if (ctx->opts.profile) kt_resolve(&timer);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int status = CHFSI_OK;
  for (int p = 0; p < P; ++p) {
    const int s = pbs[p].finish();
    if (s != CHFSI_OK && status == CHFSI_OK) status = s;
    if (stats) stats[p] = pbs[p].S;
  }
  if (ctx->opts.profile && stats && P > 0) {
    kt_resolve(&timer);
    copy_kernel_times(stats[0], timer);  // batch totals reported on problem 0
  }
  if (ms_filter_total) *ms_filter_total = filt_ms;
  return status;
}

int run_guarded(chfsi_ctx* ctx, const std::function<void()>& body) {
  try {
    body();
    ctx->last_error.clear();
    return CHFSI_OK;
  } catch (const ChfsiError& e) {
    ctx->last_error = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    ctx->last_error = e.what();
    return CHFSI_ECUDA;
  }
}

}  // namespace

// ============================================================ C ABI =====
extern "C" {

void chfsi_default_opts(chfsi_opts* o) {
  if (!o) return;
  o->precision = CHFSI_PREC_FP64;
  o->split = CHFSI_SPLIT_ADAPTIVE;
  o->degree_model = CHFSI_DEG_ANALYTIC;
  o->deg_cold = 20;
  o->deg_warm = 8;
  o->deg_min = 1;
  o->deg_max = 36;
  o->deg_extra = 1;
  o->lanczos_steps = 20;
  o->max_loops = 50;
  o->switch_tol = 1e-4;
  o->seed = 1ull;
  o->profile = 0;
  o->mlp_extra = 2;
  o->step0 = 0;
  o->f64_gemm = CHFSI_GEMM_FP64;
  o->warm_rr = 0;
  o->warm_resid = 0;
  o->autotune = 1;
}

const char* chfsi_strerror(int code) {
  switch (code) {
    case CHFSI_OK: return "ok";
    case CHFSI_EINVAL: return "invalid argument";
    case CHFSI_ENOMEM: return "out of device memory";
    case CHFSI_ENOCONV: return "not converged within max_loops";
    case CHFSI_EBREAKDOWN: return "orthonormalisation breakdown (rank-deficient block)";
    case CHFSI_ENAN: return "NaN or Inf encountered";
    case CHFSI_ETIMEOUT: return "device wait timed out";
    case CHFSI_ECUDA: return "CUDA runtime error";
    case CHFSI_ENOTSUP: return "not supported on this device";
    case CHFSI_ETOOBIG: return "n*k exceeds the static scratch of chfsi_filter_static";
    default: return "unknown error";
  }
}

const char* chfsi_last_error(const chfsi_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "no context";
}

int chfsi_init(chfsi_ctx** out, const chfsi_opts* opts, void* stream) {
  if (!out) return CHFSI_EINVAL;
  *out = nullptr;
  chfsi_ctx* ctx = new chfsi_ctx();
  if (opts) ctx->opts = *opts; else chfsi_default_opts(&ctx->opts);
  ctx->stream = (cudaStream_t)stream;
  int rc = run_guarded(ctx, [&] {
    validate_opts(ctx->opts);
    CHFSI_CUDA_TRY(cudaGetDevice(&ctx->device));
    cudaDeviceProp p;
    CHFSI_CUDA_TRY(cudaGetDeviceProperties(&p, ctx->device));
    ctx->sm_count = p.multiProcessorCount;
    ctx->cc_major = p.major;
    ctx->cc_minor = p.minor;
    for (auto& e : ctx->ev) CHFSI_CUDA_TRY(cudaEventCreate(&e));
    if (ctx->opts.precision != CHFSI_PREC_FP64 && !tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
    mlp_create(ctx);
  });
  if (rc != CHFSI_OK) {
    chfsi_free(ctx);
    return rc;
  }
  *out = ctx;
  return CHFSI_OK;
}

int chfsi_set_opts(chfsi_ctx* ctx, const chfsi_opts* opts) {
  if (!ctx || !opts) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    validate_opts(*opts);
    if (opts->precision != CHFSI_PREC_FP64 && !tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
    ctx->opts = *opts;
  });
}

void chfsi_free(chfsi_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  tc_filter_release(ctx);
  mlp_destroy(ctx);
  ws_free_all(ctx);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

int chfsi_solve(chfsi_ctx* ctx, const double* H, int n, int nev, int nex, double* X,
                double tol, double* evals, const double* warm_host, chfsi_stats* stats) {
  if (!ctx) return CHFSI_EINVAL;
  int status = CHFSI_OK;
  int rc = run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1, "n must be >= 1");
    status = solve_one(ctx, C2(H), n, nev, nex, C2(X), tol, evals, warm_host, stats,
                       ctx->opts.step0);
  });
  if (rc != CHFSI_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  if (status == CHFSI_ENOCONV) ctx->last_error = "max_loops reached";
  return status;
}

int chfsi_solve_generalized(chfsi_ctx* ctx, const double* A, const double* B, int n, int nev,
                            int nex, double* X, double* C, double tol, double* evals,
                            const double* warm_host, chfsi_stats* stats) {
  if (!ctx) return CHFSI_EINVAL;
  int status = CHFSI_OK;
  int rc = run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && nev >= 1 && nex >= 1 && nev + nex <= n, "bad generalized sizes");
    CHFSI_REQUIRE(A && B && X && C && evals && C != X, "bad generalized buffers");
    cudaStream_t st = ctx->stream;
    const size_t nn = sizeof(double2) * (size_t)n * n;
    double2* W = (double2*)ws_get(ctx, "gen_W", nn);
    double2* T = (double2*)ws_get(ctx, "gen_T", nn);
    double2* Hs = (double2*)ws_get(ctx, "gen_H", nn);
    if (any_nonfinite(ctx, (size_t)2 * n * n, B))
      throw ChfsiError{CHFSI_ENAN, "NaN/Inf in B"};
    // B = R^H R, W = R^-1 = L^-H
    CHFSI_CUDA_TRY(cudaMemcpyAsync(W, B, nn, cudaMemcpyDeviceToDevice, st));
    const int info = cholinv_upper(ctx, n, W);
    if (info != 0)
      throw ChfsiError{CHFSI_EBREAKDOWN, "B is not numerically positive definite (minor " +
                                             std::to_string(info) + ")"};
    // H = W^H A W (= L^-1 A L^-H), Hermitianised
    gemm_nn(ctx, n, n, n, C2(A), n, W, n, T, n);
    gemm_cn(ctx, n, n, n, W, n, T, n, Hs, n);
    hermitianize(st, n, Hs, n);
    status = solve_one(ctx, Hs, n, nev, nex, C2(X), tol, evals, warm_host, stats,
                       ctx->opts.step0);
    // C = W Y (= L^-H Y)
    gemm_nn(ctx, n, nev + nex, n, W, n, C2(X), n, C2(C), n);
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  });
  if (rc != CHFSI_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  if (status == CHFSI_ENOCONV) ctx->last_error = "max_loops reached";
  return status;
}

int chfsi_solve_sequence(chfsi_ctx* ctx, const double* const* H, int N, int n, int nev,
                         int nex, double* X, double tol, double* evals, chfsi_stats* stats) {
  if (!ctx) return CHFSI_EINVAL;
  int status = CHFSI_OK;
  int rc = run_guarded(ctx, [&] {
    CHFSI_REQUIRE(H && N >= 1 && n >= 1, "bad sequence arguments");
    const int k = nev + nex;
    double warm[2];
    double* wh = (double*)pinned_get(ctx, 1024 + sizeof(int) * (size_t)(k + 8) +
                                              sizeof(double) * (size_t)(k + 8));
    for (int l = 0; l < N; ++l) {
      CHFSI_REQUIRE(H[l] != nullptr, "NULL H in sequence");
      double* ev = evals + (size_t)l * k;
      const int s = solve_one(ctx, C2(H[l]), n, nev, nex, C2(X), tol, ev, l ? warm : nullptr,
                              stats ? stats + l : nullptr, ctx->opts.step0 + l);
      if (s != CHFSI_OK && status == CHFSI_OK) status = s;
      CHFSI_CUDA_TRY(cudaMemcpyAsync(wh, ev, sizeof(double), cudaMemcpyDeviceToHost,
                                     ctx->stream));
      CHFSI_CUDA_TRY(cudaMemcpyAsync(wh + 1, ev + k - 1, sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
      CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      warm[0] = wh[0];
      warm[1] = wh[1];
    }
  });
  return rc != CHFSI_OK ? rc : status;
}

int chfsi_solve_sequence_host(chfsi_ctx* ctx, const double* const* H, int N, int n, int nev,
                              int nex, double* X_host, double tol, double* evals_host,
                              chfsi_stats* stats) {
  if (!ctx) return CHFSI_EINVAL;
  int status = CHFSI_OK;
  int rc = run_guarded(ctx, [&] {
    CHFSI_REQUIRE(H && N >= 1 && n >= 1 && X_host && evals_host, "bad sequence arguments");
    const int k = nev + nex;
    const size_t hb = sizeof(double2) * (size_t)n * n;
    double* Hd[2] = {(double*)ws_get(ctx, "hs_H0", hb), (double*)ws_get(ctx, "hs_H1", hb)};
    double* Xd = (double*)ws_get(ctx, "hs_X", sizeof(double2) * (size_t)n * k);
    double* Ed = (double*)ws_get(ctx, "hs_E", sizeof(double) * (size_t)N * k);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(Xd, X_host, sizeof(double2) * (size_t)n * k,
                                   cudaMemcpyHostToDevice, ctx->stream));
    double warm[2];
    double* wh = (double*)pinned_get(ctx, 1024 + sizeof(int) * (size_t)(k + 8) +
                                              sizeof(double) * (size_t)(k + 8));
    for (int l = 0; l < N; ++l) {
      CHFSI_REQUIRE(H[l] != nullptr, "NULL H in sequence");
      double* hd = Hd[l & 1];
      CHFSI_CUDA_TRY(cudaMemcpyAsync(hd, H[l], hb, cudaMemcpyHostToDevice, ctx->stream));
      double* ev = Ed + (size_t)l * k;
      const int s = solve_one(ctx, C2((const double*)hd), n, nev, nex, C2(Xd), tol, ev,
                              l ? warm : nullptr, stats ? stats + l : nullptr,
                              ctx->opts.step0 + l);
      if (s != CHFSI_OK && status == CHFSI_OK) status = s;
      CHFSI_CUDA_TRY(cudaMemcpyAsync(wh, ev, sizeof(double), cudaMemcpyDeviceToHost,
                                     ctx->stream));
      CHFSI_CUDA_TRY(cudaMemcpyAsync(wh + 1, ev + k - 1, sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
      CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      warm[0] = wh[0];
      warm[1] = wh[1];
    }
    CHFSI_CUDA_TRY(cudaMemcpyAsync(X_host, Xd, sizeof(double2) * (size_t)n * k,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    CHFSI_CUDA_TRY(cudaMemcpyAsync(evals_host, Ed, sizeof(double) * (size_t)N * k,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  });
  return rc != CHFSI_OK ? rc : status;
}

int chfsi_solve_batched(chfsi_ctx* ctx, int P, chfsi_problem* probs, int steps,
                        double tol, chfsi_stats* stats) {
  if (!ctx) return CHFSI_EINVAL;
  int status = CHFSI_OK;
  int rc = run_guarded(ctx, [&] {
    CHFSI_REQUIRE(P >= 1 && probs && steps >= 1, "bad batched arguments");
    std::vector<const double2*> H(P);
    std::vector<int> n(P), nev(P), nex(P);
    std::vector<double2*> X(P);
    std::vector<double*> ev(P);
    std::vector<double> warm(2 * (size_t)P);
    bool any_warm = false, all_warm = true;
    for (int p = 0; p < P; ++p) {
      CHFSI_REQUIRE(probs[p].H_host && probs[p].X && probs[p].evals, "NULL in a problem");
      CHFSI_REQUIRE(probs[p].warm == 0 || probs[p].warm == 1, "bad warm flag");
      n[p] = probs[p].n;
      nev[p] = probs[p].nev;
      nex[p] = probs[p].nex;
      X[p] = C2(probs[p].X);
      warm[2 * p] = probs[p].lam_lo;
      warm[2 * p + 1] = probs[p].lam_hi;
      any_warm = any_warm || probs[p].warm;
      all_warm = all_warm && probs[p].warm;
    }
    CHFSI_REQUIRE(any_warm == all_warm, "the problems of a batch start all warm or all cold");
    for (int l = 0; l < steps; ++l) {
      for (int p = 0; p < P; ++p) {
        H[p] = C2(probs[p].H_host[l]);
        CHFSI_REQUIRE(H[p] != nullptr, "NULL H in a batched sequence");
        ev[p] = probs[p].evals + (size_t)l * (nev[p] + nex[p]);
      }
      const int s = solve_batch(ctx, P, H.data(), n.data(), nev.data(), nex.data(), X.data(),
                                tol, ev.data(), (l || all_warm) ? warm.data() : nullptr,
                                stats ? stats + (size_t)l * P : nullptr, ctx->opts.step0 + l,
                                nullptr);
      if (s != CHFSI_OK && status == CHFSI_OK) status = s;
      double* wh = (double*)pinned_get(ctx, sizeof(double) * 2 * (size_t)P + 64);
      for (int p = 0; p < P; ++p) {
        const int k = nev[p] + nex[p];
        CHFSI_CUDA_TRY(cudaMemcpyAsync(wh + 2 * p, ev[p], sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream));
        CHFSI_CUDA_TRY(cudaMemcpyAsync(wh + 2 * p + 1, ev[p] + k - 1, sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream));
      }
      CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      std::copy(wh, wh + 2 * P, warm.begin());
    }
    for (int p = 0; p < P; ++p) {
      probs[p].lam_lo = warm[2 * p];
      probs[p].lam_hi = warm[2 * p + 1];
    }
  });
  return rc != CHFSI_OK ? rc : status;
}

int chfsi_sort_degrees(chfsi_ctx* ctx, int k, const int* deg, int* perm, int* deg_sorted) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(k >= 0, "bad k");
    if (k == 0) return;
    CHFSI_REQUIRE(deg && perm && deg_sorted, "bad sort buffers");
    sort_by_degree(ctx->stream, k, deg, nullptr, perm, deg_sorted);
  });
}

int chfsi_lock(chfsi_ctx* ctx, int ka, const double* ritz, const double* resid,
               int n_wanted_left, double tol, int* lock_idx, int* act_idx, int* counts_host) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(ka >= 1 && n_wanted_left >= 0 && tol > 0.0, "bad locking arguments");
    CHFSI_REQUIRE(ritz && resid && lock_idx && act_idx && counts_host, "bad locking buffers");
    LoopCtl* ctl = (LoopCtl*)ws_get(ctx, "api_ctl", sizeof(LoopCtl));
    lock_select(ctx->stream, ka, ritz, resid, n_wanted_left, tol, 0.0, ctl, lock_idx, act_idx);
    LoopCtl* h = (LoopCtl*)pinned_get(ctx, 256);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(h, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, ctx->stream));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    counts_host[0] = h->n_new_locked;
    counts_host[1] = h->k_active;
  });
}

int chfsi_autotune_table(chfsi_ctx* ctx, int max_entries, int* entries_host,
                         int* n_entries_host) {
  if (!ctx || !n_entries_host || max_entries < 0) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(max_entries == 0 || entries_host, "bad table buffer");
    *n_entries_host = tc_tuning_table(ctx, max_entries, entries_host);
  });
}

int chfsi_lanczos(chfsi_ctx* ctx, const double* H, int n, int steps, unsigned long long seed,
                  double* out_host) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(H && out_host && n >= 1 && steps >= 2, "bad Lanczos arguments");
    double* d = (double*)ws_get(ctx, "api_bnd", sizeof(double) * 4);
    lanczos_dev(ctx, C2(H), n, steps, seed, d);
    int* err_h = (int*)pinned_get(ctx, 64);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(out_host, d, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                                   ctx->stream));
    CHFSI_CUDA_TRY(cudaMemcpyAsync(err_h, lanczos_error_word(ctx), sizeof(int),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (*err_h)
      throw ChfsiError{CHFSI_ETIMEOUT, "Lanczos: a bounded grid barrier gave up (code " +
                                           std::to_string(*err_h) + ")"};
  });
}

int chfsi_filter(chfsi_ctx* ctx, const double* H, int n, int k, const double* Y0,
                 const int* degrees_host, double lam1, double c, double e, double* Y,
                 int precision) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && k >= 0 && k <= n, "bad filter sizes");
    if (k == 0) return;
    CHFSI_REQUIRE(H && Y0 && Y && degrees_host && Y0 != Y, "bad filter buffers");
    CHFSI_REQUIRE(e > 0.0 && lam1 != c, "bad filter interval");
    for (int j = 0; j < k; ++j) {
      CHFSI_REQUIRE(degrees_host[j] >= 1, "degrees must be >= 1");
      CHFSI_REQUIRE(j == 0 || degrees_host[j] >= degrees_host[j - 1],
                    "degrees must be ascending");
    }
    if (precision == CHFSI_PREC_MIXED || precision == CHFSI_PREC_TC) {
      if (!tc_filter_supported(ctx))
        throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
      tc_filter_run(ctx, C2(H), n, k, C2(Y0), degrees_host, lam1, c, e, C2(Y),
                    ctx->opts.split == CHFSI_SPLIT_BF16X6 ? 3 : 2);
    } else {
      CHFSI_REQUIRE(precision == CHFSI_PREC_FP64, "bad precision");
      filter_f64(ctx, C2(H), n, k, C2(Y0), degrees_host, lam1, c, e, C2(Y));
    }
  });
}

int chfsi_filter_batched(chfsi_ctx* ctx, int P, const chfsi_filter_item* items) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(P >= 0 && (P == 0 || items), "bad batch");
    if (!tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
    std::vector<TcBatchItem> v;
    for (int p = 0; p < P; ++p) {
      const chfsi_filter_item& it = items[p];
      CHFSI_REQUIRE(it.n >= 1 && it.k >= 0 && it.k <= it.n, "bad batched filter sizes");
      if (it.k == 0) continue;
      CHFSI_REQUIRE(it.H && it.Y0 && it.Y && it.degrees_host && it.Y0 != it.Y,
                    "bad batched filter buffers");
      CHFSI_REQUIRE(it.e > 0.0 && it.lam1 != it.c, "bad filter interval");
      for (int j = 0; j < it.k; ++j) {
        CHFSI_REQUIRE(it.degrees_host[j] >= 1, "degrees must be >= 1");
        CHFSI_REQUIRE(j == 0 || it.degrees_host[j] >= it.degrees_host[j - 1],
                      "degrees must be ascending");
      }
      TcBatchItem b;
      b.H = C2(it.H);
      b.n = it.n;
      b.k = it.k;
      b.src = C2(it.Y0);
      b.R = nullptr;
      b.fR = nullptr;
      b.deg = it.degrees_host;
      b.lam1 = it.lam1;
      b.c = it.c;
      b.e = it.e;
      b.out = C2(it.Y);
      b.slot = (int)v.size();
      b.h_ready = false;
      v.push_back(b);
    }
    tc_filter_launch(ctx, (int)v.size(), v.data(), ctx->opts.split == CHFSI_SPLIT_BF16X6 ? 3 : 2);
  });
}

int chfsi_filter_refine(chfsi_ctx* ctx, const double* H, int n, int k, const double* Y,
                        const double* R, const double* ritz, const int* degrees_host,
                        double lam1, double c, double e, double* Yout) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && k >= 0 && k <= n, "bad filter sizes");
    if (k == 0) return;
    CHFSI_REQUIRE(H && Y && R && ritz && Yout && degrees_host && Yout != Y && Yout != R,
                  "bad filter buffers");
    CHFSI_REQUIRE(e > 0.0 && lam1 != c, "bad filter interval");
    for (int j = 0; j < k; ++j) {
      CHFSI_REQUIRE(degrees_host[j] >= 1, "degrees must be >= 1");
      CHFSI_REQUIRE(j == 0 || degrees_host[j] >= degrees_host[j - 1],
                    "degrees must be ascending");
    }
    if (!tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "split-precision filter needs an sm_103 device"};
    int* dd = (int*)ws_get(ctx, "api_deg", sizeof(int) * k);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(dd, degrees_host, sizeof(int) * k, cudaMemcpyHostToDevice,
                                   ctx->stream));
    tc_filter_run_defect(ctx, C2(H), n, k, C2(Y), C2(R), ritz, degrees_host, dd, lam1, c, e,
                         C2(Yout), ctx->opts.split == CHFSI_SPLIT_BF16X6 ? 3 : 2);
  });
}

int chfsi_zgemm(chfsi_ctx* ctx, int op_a, int m, int n, int k, double alpha, const double* A,
                int lda, const double* B, int ldb, double beta, double* C, int ldc, int engine) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(m >= 0 && n >= 0 && k >= 0 && (op_a == 0 || op_a == 1), "bad zgemm shape");
    if (m == 0 || n == 0) return;
    CHFSI_REQUIRE(A && B && C, "bad zgemm buffers");
    CHFSI_REQUIRE(engine == CHFSI_GEMM_FP64 || engine == CHFSI_GEMM_OZAKI, "bad engine");
    if (engine == CHFSI_GEMM_OZAKI && !tc_filter_supported(ctx))
      throw ChfsiError{CHFSI_ENOTSUP, "tensor-core GEMM needs an sm_103 device"};
    const int saved = ctx->opts.f64_gemm;
    ctx->opts.f64_gemm = engine;
    try {
      if (op_a == 1) {
        CHFSI_REQUIRE(lda >= k && ldb >= k && ldc >= m, "bad leading dimensions");
        gemm_cn(ctx, m, n, k, C2(A), lda, C2(B), ldb, C2(C), ldc, alpha, beta);
      } else {
        CHFSI_REQUIRE(lda >= m && ldb >= k && ldc >= m, "bad leading dimensions");
        gemm_nn(ctx, m, n, k, C2(A), lda, C2(B), ldb, C2(C), ldc, alpha, beta);
      }
    } catch (...) {
      ctx->opts.f64_gemm = saved;
      throw;
    }
    ctx->opts.f64_gemm = saved;
    if (engine == CHFSI_GEMM_OZAKI) {
      const int e = oz_check_error(ctx);
      if (e)
        throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up (code " +
                                             std::to_string(e) + ")"};
    }
  });
}

int chfsi_orthonormalize(chfsi_ctx* ctx, int n, int nl, const double* L, int k, double* Y) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && nl >= 0 && k >= 0 && nl + k <= n, "bad QR sizes");
    CHFSI_REQUIRE(Y && (nl == 0 || L), "bad QR buffers");
    orthonormalize_dev(ctx, n, nl, C2(L), k, C2(Y), use_oz(ctx));
  });
}

int chfsi_rayleigh_ritz(chfsi_ctx* ctx, const double* H, int n, int k, const double* Q,
                        double* Y, double* HY, double* evals) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && k >= 1 && k <= n, "bad RR sizes");
    CHFSI_REQUIRE(H && Q && Y && HY && evals, "bad RR buffers");
    rayleigh_ritz_dev(ctx, C2(H), n, k, C2(Q), C2(Y), C2(HY), evals);
  });
}

int chfsi_residuals(chfsi_ctx* ctx, int n, int k, const double* HY, const double* Y,
                    const double* evals, double norm_h, double* resid) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(n >= 1 && k >= 0 && norm_h > 0.0, "bad residual arguments");
    if (k == 0) return;
    CHFSI_REQUIRE(HY && Y && evals && resid, "bad residual buffers");
    residual_norms(ctx->stream, n, k, C2(HY), C2(Y), evals, norm_h, resid);
  });
}

int chfsi_degrees(chfsi_ctx* ctx, int k, const double* ritz, const double* resid, double c,
                  double e, double tol, int n_wanted, int* degrees) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(k >= 0 && e > 0.0 && tol > 0.0, "bad degree arguments");
    if (k == 0) return;
    CHFSI_REQUIRE(ritz && resid && degrees, "bad degree buffers");
    const chfsi_opts& o = ctx->opts;
    degrees_analytic(ctx->stream, k, ritz, resid, nullptr, c, e, tol, n_wanted, o.deg_min,
                     o.deg_max, o.deg_extra, degrees);
  });
}

int chfsi_trace_enable(chfsi_ctx* ctx, int capacity_rows) {
  if (!ctx || capacity_rows < 0) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] { trace_enable(ctx, capacity_rows); });
}

int chfsi_trace_dataset(chfsi_ctx* ctx, float* x, float* y, int max_rows, int* n_rows_host) {
  if (!ctx || !n_rows_host || max_rows < 0) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(max_rows == 0 || (x && y), "bad dataset buffers");
    *n_rows_host = max_rows ? trace_dataset(ctx, x, y, max_rows) : 0;
  });
}

int chfsi_mlp_set_params(chfsi_ctx* ctx, const float* params_host) {
  if (!ctx || !params_host) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] { mlp_set_params(ctx, params_host); });
}

int chfsi_mlp_get_params(chfsi_ctx* ctx, float* params_host) {
  if (!ctx || !params_host) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] { mlp_get_params(ctx, params_host); });
}

int chfsi_mlp_forward(chfsi_ctx* ctx, int B, const float* x, float* y) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(B >= 0, "bad batch");
    if (B == 0) return;
    CHFSI_REQUIRE(x && y, "bad MLP buffers");
    mlp_forward(ctx, B, x, y);
  });
}

int chfsi_mlp_train_step(chfsi_ctx* ctx, int B, const float* x, const float* target, float lr,
                         float* grads, float* loss_host) {
  if (!ctx) return CHFSI_EINVAL;
  return run_guarded(ctx, [&] {
    CHFSI_REQUIRE(B >= 1 && x && target && lr > 0.f, "bad MLP training arguments");
    float* loss_dev = (float*)ws_get(ctx, "mlp_loss", sizeof(float));
    mlp_train_step(ctx, B, x, target, lr, grads, loss_dev);
    if (loss_host) {
      CHFSI_CUDA_TRY(cudaMemcpyAsync(loss_host, loss_dev, sizeof(float), cudaMemcpyDeviceToHost,
                                     ctx->stream));
      CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
  });
}

}  // extern "C"
