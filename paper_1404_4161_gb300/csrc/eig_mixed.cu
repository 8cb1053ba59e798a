// Reduced Hermitian eigensolve of the Rayleigh-Ritz step (Alg. 1,
// G W = W Lambda for the k x k Rayleigh quotient) in mixed precision.
//
// GB300's FP64 pipe makes LAPACK-style k x k eigensolvers slow (about
// 14 ms at k = 320 in FP64).  Here the eigenpairs are first computed in
// FP32 (cuSOLVER, the FP32 pipe is ~64x wider), then refined to FP64
// accuracy by the iterative refinement of Ogita and Aishima ("Iterative
// refinement for symmetric eigenvalue decomposition", Japan J. Indust.
// Appl. Math. 35, 2018), written here for complex Hermitian matrices:
//     R = I - W^H W,  S = W^H G W,  lam_i = Re s_ii / (1 - r_ii),
//     delta = 2 (||S - diag(lam)||_F + ||G||_2 ||R||_F),
//     E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)   if |lam_i - lam_j| > delta,
//            r_ij / 2                                 otherwise,
//     W <- W + W E.
// Each step roughly squares the error; its k x k x k products run on the
// FP64-accurate tensor-core GEMM with 8 slices per operand (~2^-56 of the
// row and column scales: the refinement needs the diagonal of W^H G W to
// FP64 accuracy).  After each step one Newton-Schulz step
// W <- W (3I - W^H W)/2 restores orthonormality (the update loses it at
// second order, which would widen the next step's cluster threshold).
#include <cuComplex.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

__global__ void to_c64_kernel(size_t n, const double2* __restrict__ a, cuComplex* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_cuComplex((float)a[i].x, (float)a[i].y);
}

__global__ void to_c128_kernel(size_t n, const cuComplex* __restrict__ a, double2* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

// lam_i = Re S_ii / Re M_ii (M = W^H W, so 1 - r_ii = m_ii); partial
// Frobenius sums of S - diag(lam) and R = I - M per block -> part[2 b],
// part[2 b + 1].
__global__ void __launch_bounds__(256)
oa_stats_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
                double* __restrict__ lam, double* __restrict__ part) {
  __shared__ double sh[2][8];
  double s1 = 0.0, s2 = 0.0;
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 s = S[t], m = M[t];
    if (i == j) {
      const double l = s.x / m.x;
      lam[i] = l;
      const double ds = s.x - l;
      s1 += ds * ds + s.y * s.y;
      const double r = 1.0 - m.x;
      s2 += r * r + m.y * m.y;
    } else {
      s1 += s.x * s.x + s.y * s.y;
      s2 += m.x * m.x + m.y * m.y;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s1;
    sh[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// delta = 2 (||S - D||_F + normG ||R||_F) from the partial sums.
__global__ void oa_delta_kernel(int nparts, const double* part, const double* normG,
                                double* delta) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int p = 0; p < nparts; ++p) {
    a += part[2 * p];
    b += part[2 * p + 1];
  }
  *delta = 2.0 * (sqrt(a) + *normG * sqrt(b));
}

// E_ij of the refinement step (R = I - M).
__global__ void oa_e_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
                            const double* __restrict__ lam, const double* __restrict__ delta,
                            double2* __restrict__ E) {
  const size_t total = (size_t)k * k;
  const double dl = *delta;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 m = M[t];
    const double2 r = make_double2((i == j ? 1.0 : 0.0) - m.x, -m.y);
    const double d = lam[j] - lam[i];
    double2 e;
    if (fabs(d) > dl) {
      const double2 s = S[t];
      e = make_double2((s.x + lam[j] * r.x) / d, (s.y + lam[j] * r.y) / d);
    } else {
      e = make_double2(0.5 * r.x, 0.5 * r.y);
    }
    E[t] = e;
  }
}

// T = (3 I - M) / 2
__global__ void ns_kernel(int k, const double2* __restrict__ M, double2* __restrict__ T) {
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 m = M[t];
    T[t] = make_double2(0.5 * ((i == j ? 3.0 : 0.0) - m.x), -0.5 * m.y);
  }
}

__global__ void norm_from_w32_kernel(int k, const float* w, double* out) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int i = 0; i < k; ++i) m = fmax(m, fabs((double)w[i]));
  *out = m;
}

unsigned grid_k2(int k) {
  const size_t t = (size_t)k * k;
  return (unsigned)std::min<size_t>((t + 255) / 256, 1024);
}

}  // namespace

// Eigenvalues (ascending) into w, eigenvectors into G (k x k, ld k).
void reduced_eigh_mixed(chfsi_ctx* ctx, int k, double2* G, double* w) {
  cudaStream_t st = ctx->stream;
  const size_t kk = (size_t)k * k;
  cuComplex* G32 = (cuComplex*)ws_get(ctx, "eig_g32", sizeof(cuComplex) * kk);
  float* w32 = (float*)ws_get(ctx, "eig_w32", sizeof(float) * k);
  double2* W = (double2*)ws_get(ctx, "eig_W", sizeof(double2) * kk);
  double2* W2 = (double2*)ws_get(ctx, "eig_W2", sizeof(double2) * kk);
  double2* GW = (double2*)ws_get(ctx, "eig_GW", sizeof(double2) * kk);
  double2* S = (double2*)ws_get(ctx, "eig_S", sizeof(double2) * kk);
  double2* M = (double2*)ws_get(ctx, "eig_M", sizeof(double2) * kk);
  double2* E = (double2*)ws_get(ctx, "eig_E", sizeof(double2) * kk);
  double* lam = (double*)ws_get(ctx, "eig_lam", sizeof(double) * k);
  double* scal = (double*)ws_get(ctx, "eig_scal", sizeof(double) * (2 * 1024 + 8));
  double* normG = scal;
  double* delta = scal + 1;
  double* part = scal + 8;
  int* perm = (int*)ws_get(ctx, "eig_perm", sizeof(int) * k);

  to_c64_kernel<<<grid_k2(k), 256, 0, st>>>(kk, G, G32);
  chfsi_check_launch("to_c64");
  int lwork = 0;
  CHFSI_SOLVER_TRY(cusolverDnCheevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                               CUBLAS_FILL_MODE_LOWER, k, G32, k, w32, &lwork));
  cuComplex* work = (cuComplex*)ws_get(ctx, "eig_work32", sizeof(cuComplex) * (size_t)std::max(lwork, 1));
  int* info = (int*)ws_get(ctx, "eig_info", sizeof(int));
  const int slot = kt_begin(st);
  CHFSI_SOLVER_TRY(cusolverDnCheevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                    k, G32, k, w32, work, lwork, info));
  kt_end(st, slot, KT_SOLVER, 0.0);
  to_c128_kernel<<<grid_k2(k), 256, 0, st>>>(kk, G32, W);
  chfsi_check_launch("to_c128");
  norm_from_w32_kernel<<<1, 32, 0, st>>>(k, w32, normG);
  chfsi_check_launch("norm_w32");
  const unsigned nparts = grid_k2(k);
  for (int it = 0; it < 2; ++it) {
    oz_gemm_nn(ctx, k, k, k, G, k, W, k, GW, k, 1.0, 0.0, 8);     // G W
    oz_gemm_cn(ctx, k, k, k, W, k, GW, k, S, k, 1.0, 0.0, 8);     // S = W^H G W
    oz_gemm_cn(ctx, k, k, k, W, k, W, k, M, k, 1.0, 0.0, 8);      // M = W^H W
    oa_stats_kernel<<<nparts, 256, 0, st>>>(k, S, M, lam, part);
    chfsi_check_launch("oa_stats");
    oa_delta_kernel<<<1, 32, 0, st>>>((int)nparts, part, normG, delta);
    chfsi_check_launch("oa_delta");
    oa_e_kernel<<<grid_k2(k), 256, 0, st>>>(k, S, M, lam, delta, E);
    chfsi_check_launch("oa_e");
    CHFSI_CUDA_TRY(cudaMemcpyAsync(W2, W, sizeof(double2) * kk, cudaMemcpyDeviceToDevice, st));
    oz_gemm_nn(ctx, k, k, k, W, k, E, k, W2, k, 1.0, 1.0, 8);     // W + W E
    // Newton-Schulz: the update above loses orthogonality at second order,
    // which would otherwise widen the next step's cluster threshold delta
    oz_gemm_cn(ctx, k, k, k, W2, k, W2, k, M, k, 1.0, 0.0, 8);
    ns_kernel<<<grid_k2(k), 256, 0, st>>>(k, M, E);
    chfsi_check_launch("ns");
    oz_gemm_nn(ctx, k, k, k, W2, k, E, k, W, k, 1.0, 0.0, 8);
  }
  // The refinement update can lose orthogonality at first order for pairs
  // just outside the cluster threshold (E_ij ~ s_ij / gap), more than one
  // Newton-Schulz step repairs; the Ritz vectors Q W must be orthonormal to
  // rounding, or the locked block stops being one.  Newton-Schulz until
  // max |W^H W - I| <= 1e-13 (quadratic: a few steps at most).
  for (int extra = 0; extra < 6; ++extra) {
    oz_gemm_cn(ctx, k, k, k, W, k, W, k, M, k, 1.0, 0.0, 8);
    if (deviation_from_identity(ctx, k, M) <= 1e-13) break;  // synchronises
    ns_kernel<<<grid_k2(k), 256, 0, st>>>(k, M, E);
    chfsi_check_launch("ns");
    CHFSI_CUDA_TRY(cudaMemcpyAsync(W2, W, sizeof(double2) * kk, cudaMemcpyDeviceToDevice, st));
    oz_gemm_nn(ctx, k, k, k, W2, k, E, k, W, k, 1.0, 0.0, 8);
  }
  double2* Wf = W;
  // Eigenvalues as the Rayleigh quotients of the final vectors: the lam of
  // a refinement step are quotients of that step's input and lag a step
  // behind for pairs the FP32 start mixes (gap near u_32 ||G||).
  oz_gemm_nn(ctx, k, k, k, G, k, Wf, k, GW, k, 1.0, 0.0, 8);
  oz_gemm_cn(ctx, k, k, k, Wf, k, GW, k, S, k, 1.0, 0.0, 8);
  oz_gemm_cn(ctx, k, k, k, Wf, k, Wf, k, M, k, 1.0, 0.0, 8);
  oa_stats_kernel<<<nparts, 256, 0, st>>>(k, S, M, lam, part);
  chfsi_check_launch("oa_stats");
  // ascending order (refinement keeps the FP32 order except inside ties)
  sort_by_value(st, k, lam, perm);
  gather_values(st, k, lam, perm, w);
  gather_columns(st, k, k, Wf, k, perm, G, k);
  const int e = oz_check_error(ctx);  // also synchronises
  if (e)
    throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up (code " +
                                         std::to_string(e) + ")"};
  int* hinfo = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  if (*hinfo != 0)
    throw ChfsiError{CHFSI_ECUDA, "FP32 reduced eigensolve failed (info " + std::to_string(*hinfo) + ")"};
}
