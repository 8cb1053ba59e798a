// Shared definitions of the ChFSI CUDA library: the context, workspace
// management, error plumbing and the launch wrappers each .cu file exports
// to the solver core (api.cu).  Device code is sm_103a only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/chfsi.h"

// ---------------------------------------------------------------- errors --
struct ChfsiError {
  int code;
  std::string msg;
};

#define CHFSI_CUDA_TRY(call)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      throw ChfsiError{CHFSI_ECUDA, std::string(#call) + ": " +                \
                                        cudaGetErrorString(e_)};               \
  } while (0)

#define CHFSI_REQUIRE(cond, text)                                              \
  do {                                                                         \
    if (!(cond)) throw ChfsiError{CHFSI_EINVAL, text};                         \
  } while (0)

// Optional per-launch timing of the kernel families.  When a
// timer is installed for the calling thread (solver with opts.profile),
// kt_begin / kt_end bracket a launch with CUDA events on its stream and
// kt_resolve adds the elapsed times after the stream has been synchronised.
// Categories: FP64 products (Ozaki or DFMA GEMMs), the tensor-core filter,
// the FP32 start of the reduced eigensolve (tridiagonal reduction and
// eigenpairs), the inverse-Cholesky kernel, the Lanczos kernels, the Ozaki
// operand slicers, and the control kernels of the reduced eigensolve.
enum KtCat {
  KT_F64 = 0, KT_TC = 1, KT_SOLVER = 2, KT_CHOLINV = 3, KT_LANCZOS = 4, KT_SLICE = 5,
  KT_EIGCTL = 6, KT_NCAT = 7
};
struct KernelTimer {
  std::vector<cudaEvent_t> ev;
  std::vector<int> cat;
  std::vector<double> flops;
  std::vector<double> flops_exec;
  int used = 0;
  double ms[KT_NCAT] = {};
  double fl[KT_NCAT] = {};
  double fx[KT_NCAT] = {};  // executed flops (tensor-core slice products)
  long long n[KT_NCAT] = {};
};
KernelTimer* kt_current();
void kt_install(KernelTimer* t);
int kt_begin(cudaStream_t st);                       // -1 when no timer
// flops: the operation's own count (FP64-equivalent for the Ozaki GEMM);
// flops_exec: what the hardware executed (default: flops).
void kt_end(cudaStream_t st, int slot, int cat, double flops, double flops_exec = -1.0);
void kt_resolve(KernelTimer* t);

// Kernel launches issued by this library (all contexts, all threads).
long long chfsi_launch_counter();
void chfsi_count_launch();

// Check the launch just issued (configuration errors only; asynchronous
// faults surface at the next synchronising call) and count it.
inline void chfsi_check_launch(const char* what) {
  chfsi_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw ChfsiError{CHFSI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ------------------------------------------------------------- context ----
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Tensor-core filter state kept per context (split copies of H and the
// Y operand buffers); defined in filter_tc.cu.
struct TcFilterState;

struct MlpState;

struct chfsi_ctx {
  chfsi_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  std::string last_error;
  std::unordered_map<std::string, DevBuf> ws;
  void* pinned = nullptr;  // small page-locked control buffer
  size_t pinned_bytes = 0;
  TcFilterState* tc = nullptr;
  MlpState* mlp = nullptr;
  cudaEvent_t ev[16] = {};
};

// Device buffer named `name` with at least `bytes` bytes (grown on demand;
// contents are not preserved when it grows).
void* ws_get(chfsi_ctx* ctx, const char* name, size_t bytes);
void ws_free_all(chfsi_ctx* ctx);
void* pinned_get(chfsi_ctx* ctx, size_t bytes);

// ------------------------------------------------- FP64 dense kernels ------
// All complex matrices are double2 (re, im), column-major.

// Epilogue of the NN product acc = A(M x K) B(K x N):
//   v = alpha * (acc - shift * S) + beta * P;  D = v;  F = v for columns
//   c < fin_end (F may be null).  S, P may be null when shift, beta are 0.
// D may alias P (each element is read then written by one thread).
struct EpiNN {
  double alpha = 1.0, shift = 0.0, beta = 0.0;
  const double2* S = nullptr;
  int lds = 0;
  const double2* P = nullptr;
  int ldp = 0;
  double2* D = nullptr;
  int ldd = 0;
  double2* F = nullptr;
  int ldf = 0;
  int fin_end = 0;
};

void zgemm_nn(cudaStream_t st, int M, int N, int K, const double2* A, int lda,
              const double2* B, int ldb, const EpiNN& ep);

// Alg. 2 in FP64 on the k degree-sorted columns of Y0 (deg ascending, host)
// into Yout; F: three caller-owned n x k work buffers.
void filter_f64_recurrence(cudaStream_t st, const double2* H, int n, int k, const double2* Y0,
                           const int* deg, double lam1, double c, double e, double2* Yout,
                           double2* const F[3]);

// C (K1 x K2, ldc) = alpha * A^H B + beta * C, A: Nr x K1, B: Nr x K2 (split
// over the long dimension Nr, partial sums reduced in a fixed order).
void zgemm_cn(chfsi_ctx* ctx, int K1, int K2, int Nr, const double2* A, int lda,
              const double2* B, int ldb, double2* C, int ldc, double alpha = 1.0,
              double beta = 0.0);


void hermitianize(cudaStream_t st, int k, double2* G, int ldg);
void add_diag(cudaStream_t st, int k, double2* G, int ldg, const double* shift_dev);
void column_norms(cudaStream_t st, int n, int k, const double2* Y, int ldy, double* out);
void scale_columns_inv(cudaStream_t st, int n, int k, double2* Y, int ldy, const double* norms);
void residual_norms(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                    const double* lam, double norm_h, double* out);
// lam_j = Re(y_j^H hy_j) / (y_j^H y_j) for the k columns (ld n).
void rayleigh_quotients(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                        double* lam);
void gather_columns(cudaStream_t st, int n, int k, const double2* src, int lds,
                    const int* idx, double2* dst, int ldd);
void gather_values(cudaStream_t st, int k, const double* src, const int* idx, double* dst);
void copy_columns(cudaStream_t st, int n, int k, const double2* src, int lds, double2* dst,
                  int ldd);
// Shift for shifted CholQR from trace(G) (Fukaya et al., SISC 2020).
void cholqr_shift(cudaStream_t st, int n, int k, const double2* G, int ldg, double* shift);
int any_nonfinite(chfsi_ctx* ctx, size_t count, const double* v);
// max |G - I| (synchronises) and T = (3I - G)/2 for a Newton-Schulz step.
double deviation_from_identity(chfsi_ctx* ctx, int k, const double2* G);
void ns_matrix(cudaStream_t st, int k, const double2* G, double2* T);
// F = I - G (k x k) and ||F||_F (synchronises).
double identity_defect(chfsi_ctx* ctx, int k, const double2* G, double2* F);
// W = c I + T (T may be null: W = c I); W may alias T.
void shift_identity(cudaStream_t st, int k, const double2* T, double c, double2* W);

// Lanczos bounds of the spectrum (lanczos.cu): out4_dev = {theta_max +
// beta_m, theta_min, theta_max, max|theta|}; NaN when a bounded wait of the
// persistent kernel gave up, with the code in *lanczos_error_word(ctx).
void lanczos_dev(chfsi_ctx* ctx, const double2* H, int n, int steps, unsigned long long seed,
                 double* out4_dev);
const int* lanczos_error_word(chfsi_ctx* ctx);

// W = R^{-1} in place for the Hermitian positive definite G = R^H R (k x k,
// ld k; cholinv.cu).  Returns 0 or the order of the first leading minor
// that is not positive definite (W then incomplete); synchronises.
int cholinv_upper(chfsi_ctx* ctx, int k, double2* G);
// The same with FP32 arithmetic (FP64 storage): a preconditioning pass.
int cholinv_upper_f32(chfsi_ctx* ctx, int k, double2* G);

// Loop control: locking, interval update, degrees, sorting (small_ops.cu).
struct LoopCtl {
  int n_new_locked;
  int k_active;
  int deg_max;
  int nonfinite;
  double alpha;
  double gamma;
  double max_resid_wanted;
  double pad;
};

void lock_select(cudaStream_t st, int ka, const double* lam, const double* resid,
                 int n_wanted_left, double tol, double gamma_in, LoopCtl* ctl,
                 int* lock_idx, int* act_idx);
// buffer_cap: upper clamp of the buffer columns' degrees (besides the
// largest wanted degree).
void degrees_analytic(cudaStream_t st, int k, const double* ritz, const double* resid,
                      const int* idx, double c, double e, double tol, int n_wanted,
                      int deg_min, int deg_max, int deg_extra, int* deg_out,
                      int buffer_cap = 1 << 30);
void sort_by_degree(cudaStream_t st, int k, const int* deg, const int* idx_or_null,
                    int* perm, int* deg_sorted);
void sort_by_value(cudaStream_t st, int k, const double* val, int* perm);
void degree_cap_buffer(cudaStream_t st, int k, int n_wanted, int* deg, int buffer_cap = 1 << 30);

// Tensor-core split-precision filter (filter_tc.cu): one persistent launch
// runs every step of Alg. 2 for one or many problems.  ns = bf16 pieces per
// operand: 2 (3 products, ~2^-16) or 3 (6 products, ~2^-20 with the FP32
// accumulation).
int tc_filter_supported(chfsi_ctx* ctx);
// A pieces of H (n x n) in operand slot `slot` (kept until the slot is
// prepared again): a solver prepares each problem's H once.
void tc_filter_prepare(chfsi_ctx* ctx, int slot, const double2* H, int n, int pieces);
// One problem of a filter launch.  Plain form: src = Y0, R = fR = null.
// Refinement form: R = residual block, fR = forcing table ((m_k + 1) x k,
// row i for step i); out receives D.  slot: operand slot of the problem;
// h_ready: its A pieces are already those of H (tc_filter_prepare).
struct TcBatchItem {
  const double2* H;
  int n, k;
  const double2* src;
  const double2* R;
  const double* fR;
  const int* deg;  // host, ascending
  double lam1, c, e;
  double2* out;
  int slot;
  bool h_ready;
};
void tc_filter_launch(chfsi_ctx* ctx, int P, const TcBatchItem* items, int ns);
// Autotuned tilings of this context: 6 ints per entry {n, k bucket (k rounded
// up to 32), pieces, block width, group, microseconds}; returns the count.
int tc_tuning_table(chfsi_ctx* ctx, int max_entries, int* out);
void tc_filter_run(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y0,
                   const int* deg_host, double lam1, double c, double e, double2* Yout, int ns);
void tc_filter_run_defect(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y,
                          const double2* Rres, const double* lam, const int* deg_host,
                          const int* deg_dev, double lam1, double c, double e, double2* Yout,
                          int ns);
void tc_filter_release(chfsi_ctx* ctx);
void tc_defect_tables(chfsi_ctx* ctx, const std::string& prefix, int k, const double* lam,
                      const int* deg_host, double lam1, double c, double e, double** psi,
                      double** fR);
void tc_defect_combine(cudaStream_t st, int n, int k, const double2* Y, const int* deg_dev,
                       const double* psi, double2* out);
// R[:, j] = HY[:, perm[j]] - lam[perm[j]] Y[:, perm[j]], lam_out[j] = lam[perm[j]].
void residual_block(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                    const double* lam, const int* perm, double2* R, double* lam_out);

// FP64-accurate GEMMs on the tensor cores (gemm_ozaki.cu).
void oz_hemm(chfsi_ctx* ctx, const std::string& prefix, const double2* H, int n,
             const double2* Q, int k, double2* Z, bool reslice_h);
// ns = slices per operand: 6 (~2^-41 of the row x column scales), 7
// (~2^-48) or 8 (~2^-55); 0 = by size (oz_slices_for).
void oz_gemm_cn(chfsi_ctx* ctx, int k1, int k2, int n, const double2* L, int ldl,
                const double2* R, int ldr, double2* C, int ldc, double alpha, double beta,
                int ns = 0);
void oz_gemm_nn(chfsi_ctx* ctx, int m, int k2, int k1, const double2* S, int lds,
                const double2* W, int ldw, double2* C, int ldc, double alpha, double beta,
                int ns = 0);
// Slices for a product whose largest dimension is `dim`: 7 up to 6144, 8
// above.  The products' error grows with the reduction length (the
// n-sized Gram and H Q products): with 7 slices the residuals of an
// n = 8192 warm solve stall near 1e-10 (12 loops instead of 4) and an
// n = 13000 solve does not reach it; 8 slices cost ~30% more tensor work.
int oz_slices_for(int dim);
int oz_check_error(chfsi_ctx* ctx);
// Reduced Hermitian eigensolve: FP32 eigenpairs refined to FP64 accuracy
// (eig_mixed.cu); eigenvectors overwrite G, eigenvalues ascending in w.
// Products FP64-accurate on the tensor cores, or FP64 on the CUDA cores
// when f64_products is set.
void reduced_eigh_mixed(chfsi_ctx* ctx, int k, double2* G, double* w, bool f64_products);
// FP32-accurate eigenvectors of the Hermitian G (k x k, ld k) into W (k x k,
// ld k), columns in ascending eigenvalue order (eig_trd.cu).
// W = Q Z runs on the engine that f64_products selects.
void trd_eigvecs_f32(chfsi_ctx* ctx, int k, const double2* G, double2* W, bool f64_products);

// Degree MLP (mlp.cu).
void mlp_create(chfsi_ctx* ctx);
void mlp_destroy(chfsi_ctx* ctx);
void mlp_set_params(chfsi_ctx* ctx, const float* host);
void mlp_get_params(chfsi_ctx* ctx, float* host);
void mlp_forward(chfsi_ctx* ctx, int B, const float* x, float* y);
void mlp_train_step(chfsi_ctx* ctx, int B, const float* x, const float* target, float lr,
                    float* grads, float* loss_dev);
void mlp_degrees(chfsi_ctx* ctx, int k, const double* ritz, const double* resid,
                 const int* idx, double c, double e, double gamma, int step, double tol,
                 int* deg_out);
void trace_enable(chfsi_ctx* ctx, int cap);
bool trace_on(chfsi_ctx* ctx);
void trace_record(chfsi_ctx* ctx, int k, const double* ritz, const double* resid,
                  const int* idx, const int* deg, double c, double e, double gamma, int step,
                  int n_wanted);
void trace_finish(chfsi_ctx* ctx, int k, const double* resid);
void trace_abandon(chfsi_ctx* ctx);
int trace_dataset(chfsi_ctx* ctx, float* x, float* y, int max_rows);
