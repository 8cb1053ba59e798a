// FP64 complex dense kernels of the ChFSI path: the NN product with the
// fused three-term-recurrence epilogue (the FP64 Chebyshev filter step of
// Alg. 2, and H*Q of the Rayleigh-Ritz step of Alg. 1), the
// split-K conjugate-transpose product for the tall-skinny Gram and
// projection matrices (QR and Rayleigh-Ritz of Alg. 1), the Hermitian mat-vec of the
// Lanczos bounds (Alg. 1, Sec. 3.1), and the column reductions for residuals.
//
// GB300 runs FP64 on a narrow pipe (about 1.1 TFLOP/s for the whole GPU),
// so these kernels are bound by DFMA issue at any practical size: a 32 x 32
// complex output tile per 256-thread CTA with a 2 x 2 register tile keeps
// the pipe fed, and grids are sized to cover all 152 SMs several times.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int TB = 32;   // output tile edge (complex elements)
constexpr int TK = 16;   // K chunk staged in shared memory

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// conj(a) * b accumulated.
__device__ __forceinline__ void cmac_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__global__ void __launch_bounds__(256)
zgemm_nn_kernel(int M, int N, int K, const double2* __restrict__ A, int lda,
                const double2* __restrict__ B, int ldb, EpiNN ep) {
  __shared__ double2 As[TK][TB + 1];
  __shared__ double2 Bs[TK][TB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.x * TB, col0 = blockIdx.y * TB;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int e = threadIdx.x; e < TB * TK; e += 256) {
      const int r = e & (TB - 1), kk = e >> 5;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[gr + (size_t)gk * lda] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int e = threadIdx.x; e < TB * TK; e += 256) {
      const int kk = e & (TK - 1), c = e >> 4;
      const int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (gk < K && gc < N) ? B[gk + (size_t)gc * ldb] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const double2 a0 = As[kk][tx], a1 = As[kk][tx + 16];
      const double2 b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
      cmac(acc[0][0], a0, b0);
      cmac(acc[0][1], a0, b1);
      cmac(acc[1][0], a1, b0);
      cmac(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = col0 + ty + 16 * j;
    if (c >= N) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = row0 + tx + 16 * i;
      if (r >= M) continue;
      double2 v = acc[i][j];
      if (ep.shift != 0.0) {
        const double2 s = ep.S[r + (size_t)c * ep.lds];
        v.x = fma(-ep.shift, s.x, v.x);
        v.y = fma(-ep.shift, s.y, v.y);
      }
      v.x *= ep.alpha;
      v.y *= ep.alpha;
      if (ep.beta != 0.0) {
        const double2 p = ep.P[r + (size_t)c * ep.ldp];
        v.x = fma(ep.beta, p.x, v.x);
        v.y = fma(ep.beta, p.y, v.y);
      }
      ep.D[r + (size_t)c * ep.ldd] = v;
      if (ep.F != nullptr && c < ep.fin_end) ep.F[r + (size_t)c * ep.ldf] = v;
    }
  }
}

// Partial[z] (K1 x K2) = A[rows of chunk z]^H B[rows of chunk z].
__global__ void __launch_bounds__(256)
zgemm_cn_part_kernel(int K1, int K2, int Nr, int chunk, const double2* __restrict__ A,
                     int lda, const double2* __restrict__ B, int ldb,
                     double2* __restrict__ part) {
  __shared__ double2 As[TK][TB + 1];
  __shared__ double2 Bs[TK][TB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * TB, j0 = blockIdx.y * TB;
  const int rbeg = blockIdx.z * chunk;
  const int rend = min(Nr, rbeg + chunk);
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int r0 = rbeg; r0 < rend; r0 += TK) {
#pragma unroll
    for (int e = threadIdx.x; e < TB * TK; e += 256) {
      const int rr = e & (TK - 1), c = e >> 4;
      const int gr = r0 + rr;
      As[rr][c] = (gr < rend && i0 + c < K1) ? A[gr + (size_t)(i0 + c) * lda]
                                             : make_double2(0.0, 0.0);
      Bs[rr][c] = (gr < rend && j0 + c < K2) ? B[gr + (size_t)(j0 + c) * ldb]
                                             : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < TK; ++rr) {
      const double2 a0 = As[rr][tx], a1 = As[rr][tx + 16];
      const double2 b0 = Bs[rr][ty], b1 = Bs[rr][ty + 16];
      cmac_conj(acc[0][0], a0, b0);
      cmac_conj(acc[0][1], a0, b1);
      cmac_conj(acc[1][0], a1, b0);
      cmac_conj(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  double2* out = part + (size_t)blockIdx.z * K1 * K2;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = j0 + ty + 16 * j;
    if (c >= K2) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = i0 + tx + 16 * i;
      if (r < K1) out[r + (size_t)c * K1] = acc[i][j];
    }
  }
}

__global__ void zgemm_cn_reduce_kernel(int K1, int K2, int splits, const double2* part,
                                       double2* C, int ldc, double alpha, double beta) {
  const size_t total = (size_t)K1 * K2;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < splits; ++z) {
      const double2 p = part[(size_t)z * total + t];
      s.x += p.x;
      s.y += p.y;
    }
    const int i = (int)(t % K1), j = (int)(t / K1);
    double2* c = C + i + (size_t)j * ldc;
    double2 v = make_double2(alpha * s.x, alpha * s.y);
    if (beta != 0.0) {
      v.x = fma(beta, c->x, v.x);
      v.y = fma(beta, c->y, v.y);
    }
    *c = v;
  }
}

// y[r] = sum_j conj(H[j, r]) x[j]  (= (H x)[r] for Hermitian H).
template <int NT>
__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < NT / 32) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;  // valid in thread 0
}

__global__ void __launch_bounds__(256)
column_norms_kernel(int n, const double2* __restrict__ Y, int ldy, double* out) {
  __shared__ double sh[8];
  const double2* y = Y + (size_t)blockIdx.x * ldy;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) s += y[r].x * y[r].x + y[r].y * y[r].y;
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

__global__ void scale_columns_inv_kernel(int n, int k, double2* Y, int ldy,
                                         const double* norms) {
  const int c = blockIdx.y;
  const double inv = 1.0 / norms[c];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double2 v = Y[r + (size_t)c * ldy];
    v.x *= inv;
    v.y *= inv;
    Y[r + (size_t)c * ldy] = v;
  }
}

__global__ void __launch_bounds__(256)
residual_norms_kernel(int n, const double2* __restrict__ HY, const double2* __restrict__ Y,
                      const double* lam, double inv_norm, double* out) {
  __shared__ double sh[8];
  const size_t off = (size_t)blockIdx.x * n;
  const double l = lam[blockIdx.x];
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) {
    const double2 h = HY[off + r], y = Y[off + r];
    const double dx = h.x - l * y.x, dy = h.y - l * y.y;
    s += dx * dx + dy * dy;
  }
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s) * inv_norm;
}

// lam_j = Re(y_j^H hy_j) / (y_j^H y_j): the Rayleigh quotient of column j.
__global__ void __launch_bounds__(256)
rayleigh_quotients_kernel(int n, const double2* __restrict__ HY, const double2* __restrict__ Y,
                          double* lam) {
  __shared__ double sh[8];
  const size_t off = (size_t)blockIdx.x * n;
  double num = 0.0, den = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) {
    const double2 h = HY[off + r], y = Y[off + r];
    num += y.x * h.x + y.y * h.y;
    den += y.x * y.x + y.y * y.y;
  }
  num = block_sum<256>(num, sh);
  den = block_sum<256>(den, sh);
  if (threadIdx.x == 0) lam[blockIdx.x] = num / den;
}

__global__ void hermitianize_kernel(int k, double2* G, int ldg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i > j || j >= k) return;
  double2 a = G[i + (size_t)j * ldg], b = G[j + (size_t)i * ldg];
  if (i == j) {
    G[i + (size_t)j * ldg] = make_double2(a.x, 0.0);
    return;
  }
  const double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  G[i + (size_t)j * ldg] = v;
  G[j + (size_t)i * ldg] = make_double2(v.x, -v.y);
}


__global__ void add_diag_kernel(int k, double2* G, int ldg, const double* shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) G[i + (size_t)i * ldg].x += *shift;
}

__global__ void gather_columns_kernel(int n, const double2* __restrict__ src, int lds,
                                      const int* __restrict__ idx, double2* __restrict__ dst,
                                      int ldd) {
  const int c = blockIdx.y;
  const int sc = idx ? idx[c] : c;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    dst[r + (size_t)c * ldd] = src[r + (size_t)sc * lds];
}

__global__ void gather_values_kernel(int k, const double* src, const int* idx, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) dst[i] = src[idx[i]];
}

// Shifted CholQR shift s = 11 (n k + k (k + 1)) u ||Y||_2^2 with the
// bound ||Y||_2^2 <= trace(G) (Fukaya, Kannan, Nakatsukasa, Yamamoto,
// Yanagisawa, SIAM J. Sci. Comput. 42 (2020), Sec. 3).
__global__ void cholqr_shift_kernel(int n, int k, const double2* G, int ldg, double* shift) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += 256) s += G[i + (size_t)i * ldg].x;
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) {
    const double u = 1.1102230246251565e-16;
    *shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * u * s;
  }
}

__global__ void nonfinite_kernel(size_t count, const double* v, int* flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) *flag = 1;
}

__global__ void residual_block_kernel(int n, const double2* __restrict__ HY,
                                      const double2* __restrict__ Y, const double* lam,
                                      const int* __restrict__ perm, double2* __restrict__ R,
                                      double* lam_out) {
  const int j = blockIdx.y;
  const int sj = perm[j];
  const double l = lam[sj];
  if (blockIdx.x == 0 && threadIdx.x == 0) lam_out[j] = l;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const size_t es = (size_t)r + (size_t)sj * n;
    const double2 h = HY[es], y = Y[es];
    R[(size_t)r + (size_t)j * n] = make_double2(h.x - l * y.x, h.y - l * y.y);
  }
}

int grid_for(size_t work, int per_block, int cap = 4096) {
  size_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

}  // namespace

// ======================================================== host wrappers ===
void zgemm_nn(cudaStream_t st, int M, int N, int K, const double2* A, int lda,
              const double2* B, int ldb, const EpiNN& ep) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((M + TB - 1) / TB, (N + TB - 1) / TB);
  const int slot = kt_begin(st);
  zgemm_nn_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
  chfsi_check_launch("zgemm_nn");
  kt_end(st, slot, KT_F64, 8.0 * M * (double)N * K);
}

void zgemm_cn(chfsi_ctx* ctx, int K1, int K2, int Nr, const double2* A, int lda,
              const double2* B, int ldb, double2* C, int ldc, double alpha, double beta) {
  if (K1 <= 0 || K2 <= 0) return;
  const int tiles = ((K1 + TB - 1) / TB) * ((K2 + TB - 1) / TB);
  int splits = (4 * ctx->sm_count + tiles - 1) / tiles;
  const int max_splits = (Nr + 63) / 64;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  int chunk = (Nr + splits - 1) / splits;
  chunk = (chunk + TK - 1) / TK * TK;
  splits = (Nr + chunk - 1) / chunk;
  if (splits < 1) splits = 1;
  double2* part = (double2*)ws_get(ctx, "cn_part", sizeof(double2) * (size_t)splits * K1 * K2);
  dim3 grid((K1 + TB - 1) / TB, (K2 + TB - 1) / TB, splits);
  const int slot = kt_begin(ctx->stream);
  zgemm_cn_part_kernel<<<grid, 256, 0, ctx->stream>>>(K1, K2, Nr, chunk, A, lda, B, ldb, part);
  chfsi_check_launch("zgemm_cn_part");
  kt_end(ctx->stream, slot, KT_F64, 8.0 * K1 * (double)K2 * Nr);
  zgemm_cn_reduce_kernel<<<grid_for((size_t)K1 * K2, 256, 2048), 256, 0, ctx->stream>>>(
      K1, K2, splits, part, C, ldc, alpha, beta);
  chfsi_check_launch("zgemm_cn_reduce");
}


void hermitianize(cudaStream_t st, int k, double2* G, int ldg) {
  if (k <= 0) return;
  hermitianize_kernel<<<dim3((k + 127) / 128, k), 128, 0, st>>>(k, G, ldg);
  chfsi_check_launch("hermitianize");
}


void add_diag(cudaStream_t st, int k, double2* G, int ldg, const double* shift_dev) {
  add_diag_kernel<<<(k + 255) / 256, 256, 0, st>>>(k, G, ldg, shift_dev);
  chfsi_check_launch("add_diag");
}

void column_norms(cudaStream_t st, int n, int k, const double2* Y, int ldy, double* out) {
  if (k <= 0) return;
  column_norms_kernel<<<k, 256, 0, st>>>(n, Y, ldy, out);
  chfsi_check_launch("column_norms");
}

void scale_columns_inv(cudaStream_t st, int n, int k, double2* Y, int ldy,
                       const double* norms) {
  if (k <= 0) return;
  scale_columns_inv_kernel<<<dim3(grid_for(n, 256, 64), k), 256, 0, st>>>(n, k, Y, ldy, norms);
  chfsi_check_launch("scale_columns_inv");
}

void residual_norms(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                    const double* lam, double norm_h, double* out) {
  if (k <= 0) return;
  residual_norms_kernel<<<k, 256, 0, st>>>(n, HY, Y, lam, 1.0 / norm_h, out);
  chfsi_check_launch("residual_norms");
}

void rayleigh_quotients(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                        double* lam) {
  if (k <= 0) return;
  rayleigh_quotients_kernel<<<k, 256, 0, st>>>(n, HY, Y, lam);
  chfsi_check_launch("rayleigh_quotients");
}

void gather_columns(cudaStream_t st, int n, int k, const double2* src, int lds, const int* idx,
                    double2* dst, int ldd) {
  if (k <= 0) return;
  gather_columns_kernel<<<dim3(grid_for(n, 256, 64), k), 256, 0, st>>>(n, src, lds, idx, dst,
                                                                        ldd);
  chfsi_check_launch("gather_columns");
}

void copy_columns(cudaStream_t st, int n, int k, const double2* src, int lds, double2* dst,
                  int ldd) {
  gather_columns(st, n, k, src, lds, nullptr, dst, ldd);
}

void gather_values(cudaStream_t st, int k, const double* src, const int* idx, double* dst) {
  if (k <= 0) return;
  gather_values_kernel<<<(k + 255) / 256, 256, 0, st>>>(k, src, idx, dst);
  chfsi_check_launch("gather_values");
}

void cholqr_shift(cudaStream_t st, int n, int k, const double2* G, int ldg, double* shift) {
  cholqr_shift_kernel<<<1, 256, 0, st>>>(n, k, G, ldg, shift);
  chfsi_check_launch("cholqr_shift");
}

int any_nonfinite(chfsi_ctx* ctx, size_t count, const double* v) {
  int* flag = (int*)ws_get(ctx, "nf_flag", sizeof(int));
  CHFSI_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  nonfinite_kernel<<<grid_for(count, 256, 1024), 256, 0, ctx->stream>>>(count, v, flag);
  chfsi_check_launch("nonfinite");
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return *h;
}






void residual_block(cudaStream_t st, int n, int k, const double2* HY, const double2* Y,
                    const double* lam, const int* perm, double2* R, double* lam_out) {
  if (k <= 0) return;
  residual_block_kernel<<<dim3(grid_for(n, 256, 64), k), 256, 0, st>>>(n, HY, Y, lam, perm, R,
                                                                        lam_out);
  chfsi_check_launch("residual_block");
}

namespace {
// max |G - I| over a k x k matrix: per-block maxima then one block.
__global__ void __launch_bounds__(256) dev_from_identity_kernel(int k, const double2* G,
                                                                double* part) {
  __shared__ double sh[8];
  double m = 0.0;
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 g = G[t];
    m = fmax(m, fmax(fabs(g.x - (i == j ? 1.0 : 0.0)), fabs(g.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < 8; ++w) r = fmax(r, sh[w]);
    part[blockIdx.x] = r;
  }
}
__global__ void max_reduce_kernel(int n, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double r = 0.0;
  for (int i = 0; i < n; ++i) r = fmax(r, part[i]);
  *out = r;
}
// T = (3 I - G) / 2
__global__ void ns_matrix_kernel(int k, const double2* __restrict__ G, double2* __restrict__ T) {
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 g = G[t];
    T[t] = make_double2(0.5 * ((i == j ? 3.0 : 0.0) - g.x), -0.5 * g.y);
  }
}
// F = I - G and per-block partial sums of |F_ij|^2
__global__ void __launch_bounds__(256) identity_defect_kernel(int k, const double2* __restrict__ G,
                                                              double2* __restrict__ F,
                                                              double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 g = G[t];
    const double2 f = make_double2((i == j ? 1.0 : 0.0) - g.x, -g.y);
    F[t] = f;
    s += f.x * f.x + f.y * f.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < 8; ++w) r += sh[w];
    part[blockIdx.x] = r;
  }
}
__global__ void sum_sqrt_kernel(int n, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double r = 0.0;
  for (int i = 0; i < n; ++i) r += part[i];
  *out = sqrt(r);
}
// W = c I + (T or 0)
__global__ void shift_identity_kernel(int k, const double2* __restrict__ T, double c,
                                      double2* __restrict__ W) {
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    double2 v = T ? T[t] : make_double2(0.0, 0.0);
    if (i == j) v.x += c;
    W[t] = v;
  }
}
}  // namespace

double identity_defect(chfsi_ctx* ctx, int k, const double2* G, double2* F) {
  const unsigned nb = (unsigned)std::min<size_t>(((size_t)k * k + 255) / 256, 512);
  double* part = (double*)ws_get(ctx, "idf_part", sizeof(double) * (nb + 2));
  identity_defect_kernel<<<nb, 256, 0, ctx->stream>>>(k, G, F, part);
  chfsi_check_launch("identity_defect");
  sum_sqrt_kernel<<<1, 32, 0, ctx->stream>>>((int)nb, part, part + nb);
  chfsi_check_launch("sum_sqrt");
  double* h = (double*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, part + nb, sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return *h;
}

void shift_identity(cudaStream_t st, int k, const double2* T, double c, double2* W) {
  shift_identity_kernel<<<(unsigned)std::min<size_t>(((size_t)k * k + 255) / 256, 1024), 256, 0,
                          st>>>(k, T, c, W);
  chfsi_check_launch("shift_identity");
}

double deviation_from_identity(chfsi_ctx* ctx, int k, const double2* G) {
  const unsigned nb = (unsigned)std::min<size_t>(((size_t)k * k + 255) / 256, 512);
  double* part = (double*)ws_get(ctx, "dfi_part", sizeof(double) * (nb + 2));
  dev_from_identity_kernel<<<nb, 256, 0, ctx->stream>>>(k, G, part);
  chfsi_check_launch("dev_from_identity");
  max_reduce_kernel<<<1, 32, 0, ctx->stream>>>((int)nb, part, part + nb);
  chfsi_check_launch("max_reduce");
  double* h = (double*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, part + nb, sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return *h;
}

void ns_matrix(cudaStream_t st, int k, const double2* G, double2* T) {
  ns_matrix_kernel<<<(unsigned)std::min<size_t>(((size_t)k * k + 255) / 256, 1024), 256, 0, st>>>(
      k, G, T);
  chfsi_check_launch("ns_matrix");
}

// Alg. 2 in FP64 (readings R1, R2 of the column ranges): Y_1 = sigma_1/e
// (H - cI) Y_0 on all k columns, then for i = 1 .. m_k - 1 the step
// Y_{i+1} = 2 sigma_{i+1}/e (H - cI) Y_i - sigma_{i+1} sigma_i Y_{i-1} on the
// columns whose degree exceeds i; a column's result goes to Yout at the step
// that reaches its degree.  deg (host) ascending; F: three n x k work
// buffers (caller-owned, fully written before they are read).
void filter_f64_recurrence(cudaStream_t st, const double2* H, int n, int k, const double2* Y0,
                           const int* deg, double lam1, double c, double e, double2* Yout,
                           double2* const F[3]) {
  auto buf = [&](int i) -> const double2* { return i == 0 ? Y0 : F[i % 3]; };
  const int mk = deg[k - 1];
  const double sigma1 = e / (lam1 - c);
  int s = (int)(std::upper_bound(deg, deg + k, 1) - deg);
  {
    EpiNN ep;
    ep.alpha = sigma1 / e;
    ep.shift = c;
    ep.S = Y0;
    ep.lds = n;
    ep.D = F[1];
    ep.ldd = n;
    ep.F = Yout;
    ep.ldf = n;
    ep.fin_end = s;
    zgemm_nn(st, n, k, n, H, n, Y0, n, ep);
  }
  double sigma = sigma1;
  for (int i = 1; i < mk; ++i) {
    const double sn = 1.0 / (2.0 / sigma1 - sigma);
    const int s_new = (int)(std::upper_bound(deg, deg + k, i + 1) - deg);
    const double2* cur = buf(i);
    const double2* prev = buf(i - 1);
    double2* nxt = F[(i + 1) % 3];
    const size_t off = (size_t)s * n;
    EpiNN ep;
    ep.alpha = 2.0 * sn / e;
    ep.shift = c;
    ep.S = cur + off;
    ep.lds = n;
    ep.beta = -sn * sigma;
    ep.P = prev + off;
    ep.ldp = n;
    ep.D = nxt + off;
    ep.ldd = n;
    ep.F = Yout + off;
    ep.ldf = n;
    ep.fin_end = s_new - s;
    zgemm_nn(st, n, k - s, n, H, n, cur + off, n, ep);
    sigma = sn;
    s = s_new;
  }
}
