// Inverse Cholesky factor of the CholQR step (QR step of Alg. 1): for the
// Hermitian positive definite Gram matrix G = R^H R (k x k) compute
// W = R^{-1} (upper triangular) in place, in FP64, in ONE persistent
// cooperative kernel.
//
// Left-looking by block columns of width 32: with W known for the leading
// J = 32 j columns,
//   X   = W_{0:J,0:J}^H A_{0:J,j}       (= R_{0:J,j}, the panel of R)
//   S   = A_jj - X^H X                  (Schur complement, 32 x 32)
//   R_jj = chol(S),  W_jj = R_jj^{-1}   (one CTA, in shared memory)
//   W_{0:J,j} = -(W_{0:J,0:J} X) W_jj
// so the factor and its inverse come out together and no triangular solve
// is needed.  GB300's FP64 pipe is narrow (about 2 DFMA per clock per SM),
// so every product is spread over all SMs: one warp per output entry (or
// per row and 8 columns) with the lanes along the reduction.  Four bounded
// grid barriers per block column (grid_sync.cuh).  The strict lower
// triangle of A is never read and is zeroed at the start.
//
// info: 0, or i (1-based) when the leading minor of order i is not
// (numerically) positive definite -- the pivot is <= 0 or not finite; W is
// then incomplete.
#include "common.cuh"
#include "grid_sync.cuh"

namespace {

constexpr int CI_THREADS = 512;
constexpr int CI_WARPS = CI_THREADS / 32;
constexpr int CI_B = 32;     // block column width
constexpr int CI_YG = 8;     // columns per warp task in the panel products
constexpr int CI_ROWS = 4;   // rows per CTA batch in the W update

struct CiArgs {
  int k, ld;
  double2* G;     // in: A (upper part), out: W = R^{-1}, strict lower zero
  double2* X;     // scratch, k x 32 column-major (ld k)
  double2* S;     // scratch, 32 x 32 column-major
  int* info;      // 0 or the failing pivot (1-based)
  unsigned* bar;  // barrier counter (zero at launch)
  int* flags;     // [0] abort, [1] error code
};

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
// acc += conj(a) * b
__device__ __forceinline__ void cmac_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * b
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__global__ void __launch_bounds__(CI_THREADS, 1) cholinv_kernel(CiArgs a) {
  __shared__ double2 Rs[CI_B][CI_B + 1];   // diagonal block: S, then R_jj
  __shared__ double2 Ws[CI_B][CI_B + 1];   // W_jj
  __shared__ double2 Zs[CI_ROWS][CI_B];    // rows of W_{0:J,0:J} X
  __shared__ int ok_sh, fail_sh;
  const int k = a.k, ld = a.ld;
  double2* G = a.G;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * CI_WARPS + warp, nwarps = gridDim.x * CI_WARPS;
  unsigned nbar = 0;

  // strict lower triangle of the output is zero (never read as input)
  for (size_t e = (size_t)blockIdx.x * CI_THREADS + threadIdx.x; e < (size_t)k * k;
       e += (size_t)gridDim.x * CI_THREADS) {
    const int r = (int)(e % k), c = (int)(e / k);
    if (r > c) G[(size_t)r + (size_t)c * ld] = make_double2(0.0, 0.0);
  }

  const int nb = (k + CI_B - 1) / CI_B;
  for (int j = 0; j < nb; ++j) {
    const int c0 = j * CI_B, bw = min(CI_B, k - c0), J = c0;
    const int ngy = (bw + CI_YG - 1) / CI_YG;

    // ---- (a) X = W_{0:J,0:J}^H A_{0:J,j}: X[x][y] = sum_{l<=x} conj(W[l][x]) A[l][c0+y]
    if (J > 0) {
      for (int t = gwarp; t < J * ngy; t += nwarps) {
        const int x = t / ngy, y0 = (t - x * ngy) * CI_YG;
        double2 acc[CI_YG];
#pragma unroll
        for (int u = 0; u < CI_YG; ++u) acc[u] = make_double2(0.0, 0.0);
        const double2* wcol = G + (size_t)x * ld;
        for (int l = lane; l <= x; l += 32) {
          const double2 w = __ldcg(wcol + l);
#pragma unroll
          for (int u = 0; u < CI_YG; ++u)
            if (y0 + u < bw) cmac_conj(acc[u], w, __ldcg(G + (size_t)l + (size_t)(c0 + y0 + u) * ld));
        }
#pragma unroll
        for (int u = 0; u < CI_YG; ++u) {
          const double2 s = warp_sum2(acc[u]);
          if (lane == 0 && y0 + u < bw) a.X[(size_t)x + (size_t)(y0 + u) * k] = s;
        }
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 11, &ok_sh)) return;
    }

    // ---- (b) S = A_jj - X^H X (upper part), one warp per entry ----------
    for (int t = gwarp; t < bw * bw; t += nwarps) {
      const int x = t % bw, y = t / bw;
      if (x > y) continue;
      double2 acc = make_double2(0.0, 0.0);
      for (int l = lane; l < J; l += 32)
        cmac_conj(acc, __ldcg(a.X + (size_t)l + (size_t)x * k), __ldcg(a.X + (size_t)l + (size_t)y * k));
      acc = warp_sum2(acc);
      if (lane == 0) {
        const double2 g = __ldcg(G + (size_t)(c0 + x) + (size_t)(c0 + y) * ld);
        a.S[x + CI_B * y] = make_double2(g.x - acc.x, g.y - acc.y);
      }
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 12, &ok_sh)) return;

    // ---- (c) R_jj = chol(S), W_jj = R_jj^{-1} on CTA 0 -----------------
    if (blockIdx.x == 0) {
      for (int e = threadIdx.x; e < CI_B * CI_B; e += CI_THREADS) {
        const int x = e % CI_B, y = e / CI_B;
        double2 v = make_double2(x == y ? 1.0 : 0.0, 0.0);
        if (x < bw && y < bw && x <= y) v = __ldcg(a.S + x + CI_B * y);
        Rs[x][y] = v;
        Ws[x][y] = make_double2(0.0, 0.0);
      }
      if (threadIdx.x == 0) fail_sh = 0;
      __syncthreads();
      for (int c = 0; c < bw; ++c) {
        const double piv = Rs[c][c].x;
        if (!(piv > 0.0) || !isfinite(piv)) {  // uniform across the CTA
          if (threadIdx.x == 0) {
            fail_sh = 1;
            *a.info = c0 + c + 1;
          }
          break;
        }
        const double r = sqrt(piv), ir = 1.0 / r;
        __syncthreads();  // everyone has read the pivot
        if (threadIdx.x > c && threadIdx.x < bw) {
          Rs[c][threadIdx.x].x *= ir;
          Rs[c][threadIdx.x].y *= ir;
        }
        if (threadIdx.x == 0) Rs[c][c] = make_double2(r, 0.0);
        __syncthreads();
        for (int e = threadIdx.x; e < CI_B * CI_B; e += CI_THREADS) {
          const int x = e % CI_B, y = e / CI_B;
          if (x > c && x <= y && y < bw) {
            const double2 u = Rs[c][x], v = Rs[c][y];
            // Rs[x][y] -= conj(u) * v
            Rs[x][y].x -= u.x * v.x + u.y * v.y;
            Rs[x][y].y -= u.x * v.y - u.y * v.x;
          }
        }
        __syncthreads();
      }
      __syncthreads();
      if (!fail_sh) {
        // back substitution, bottom row first: W[x][y] = -(sum_{x<l<=y} R[x][l] W[l][y]) / R[x][x]
        for (int x = bw - 1; x >= 0; --x) {
          const int y = threadIdx.x;
          if (y >= x && y < bw) {
            const double id = 1.0 / Rs[x][x].x;
            if (y == x) {
              Ws[x][x] = make_double2(id, 0.0);
            } else {
              double2 s = make_double2(0.0, 0.0);
              for (int l = x + 1; l <= y; ++l) cmac(s, Rs[x][l], Ws[l][y]);
              Ws[x][y] = make_double2(-s.x * id, -s.y * id);
            }
          }
          __syncthreads();
        }
        for (int e = threadIdx.x; e < bw * bw; e += CI_THREADS) {
          const int x = e % bw, y = e / bw;
          G[(size_t)(c0 + x) + (size_t)(c0 + y) * ld] = x <= y ? Ws[x][y] : make_double2(0.0, 0.0);
        }
      }
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 13, &ok_sh)) return;
    if (__ldcg(a.info) != 0) return;

    // ---- (d) W_{0:J,j} = -(W_{0:J,0:J} X) W_jj, rows by CTA ------------
    if (J > 0) {
      for (int base = blockIdx.x; base < J; base += CI_ROWS * gridDim.x) {
        // Z rows x = base + q * gridDim.x, q < CI_ROWS
        for (int t = warp; t < CI_ROWS * ngy; t += CI_WARPS) {
          const int q = t / ngy, y0 = (t - q * ngy) * CI_YG;
          const int x = base + q * gridDim.x;
          if (x >= J) continue;
          double2 acc[CI_YG];
#pragma unroll
          for (int u = 0; u < CI_YG; ++u) acc[u] = make_double2(0.0, 0.0);
          for (int l = x + lane; l < J; l += 32) {
            const double2 w = __ldcg(G + (size_t)x + (size_t)l * ld);
#pragma unroll
            for (int u = 0; u < CI_YG; ++u)
              if (y0 + u < bw) cmac(acc[u], w, __ldcg(a.X + (size_t)l + (size_t)(y0 + u) * k));
          }
#pragma unroll
          for (int u = 0; u < CI_YG; ++u) {
            const double2 s = warp_sum2(acc[u]);
            if (lane == 0 && y0 + u < bw) Zs[q][y0 + u] = s;
          }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < CI_ROWS * bw; e += CI_THREADS) {
          const int q = e / bw, y = e - q * bw;
          const int x = base + q * gridDim.x;
          if (x >= J) continue;
          double2 s = make_double2(0.0, 0.0);
          for (int mm = 0; mm <= y; ++mm)
            cmac(s, Zs[q][mm], __ldcg(G + (size_t)(c0 + mm) + (size_t)(c0 + y) * ld));
          G[(size_t)x + (size_t)(c0 + y) * ld] = make_double2(-s.x, -s.y);
        }
        __syncthreads();
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 14, &ok_sh)) return;
    }
  }
}

}  // namespace

int cholinv_upper(chfsi_ctx* ctx, int k, double2* G) {
  cudaStream_t st = ctx->stream;
  if (k <= 0) return 0;
  static int per_sm = -1;
  if (per_sm < 0)
    CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholinv_kernel,
                                                                 CI_THREADS, 0));
  CHFSI_REQUIRE(per_sm >= 1, "cholinv: kernel does not fit on an SM");
  const int grid = std::max(1, std::min(ctx->sm_count, (k + 1) / 2));
  CiArgs a;
  a.k = k;
  a.ld = k;
  a.G = G;
  a.X = (double2*)ws_get(ctx, "ci_X", sizeof(double2) * (size_t)k * CI_B);
  a.S = (double2*)ws_get(ctx, "ci_S", sizeof(double2) * CI_B * CI_B);
  char* sync = (char*)ws_get(ctx, "ci_sync", 64);
  a.bar = (unsigned*)sync;
  a.flags = (int*)(sync + 16);
  a.info = (int*)(sync + 32);
  CHFSI_CUDA_TRY(cudaMemsetAsync(sync, 0, 64, st));
  void* args[] = {&a};
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)cholinv_kernel, dim3(grid), dim3(CI_THREADS),
                                             args, 0, st));
  chfsi_check_launch("cholinv");
  kt_end(st, slot, KT_SOLVER, 0.0);
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, a.flags, 3 * sizeof(int) + 8, cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  // h[0] abort, h[1] error code, h[2..3] padding, h[4] info
  if (h[1] != 0)
    throw ChfsiError{CHFSI_ETIMEOUT, "cholinv: a bounded grid barrier gave up (code " +
                                         std::to_string(h[1]) + ")"};
  return h[4];
}
