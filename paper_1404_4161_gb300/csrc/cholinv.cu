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
// is needed.  GB300's FP64 pipe is narrow (about 2 DFMA per clock per SM,
// and a warp-wide FP64 instruction costs its full width even with idle
// lanes), so the products are laid out with the 32 columns of the block on
// the lanes -- no FP64 shuffle reductions -- and spread over all SMs: a
// warp per row of X and of W_{0:J,0:J} X, a warp per (row, 64-row chunk)
// of the Schur sums.  The rows of W_{0:J,0:J} X are formed next to those
// sums, before the diagonal block is factored, so only the small product
// with W_jj follows it.  The diagonal block (CTA 0) forms each pivot's
// square root and reciprocal once; its inverse is a column-oriented
// substitution with the columns over the warps.  Up to four bounded grid
// barriers per block column (grid_sync.cuh).  The strict lower triangle of
// A is never read and is zeroed at the start.
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
constexpr int CI_CH = 64;    // rows per partial sum of the Schur complement

struct CiArgs {
  int k, ld;
  double2* G;     // in: A (upper part), out: W = R^{-1}, strict lower zero
  double2* X;     // scratch, k x 32 row-major (X[l * 32 + y])
  double2* S;     // scratch, ceil(k / 64) partial 32 x 32 Schur sums
  int* info;      // 0 or the failing pivot (1-based)
  unsigned* bar;  // barrier counter (zero at launch)
  int* flags;     // [0] abort, [1] error code
};

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
  __shared__ double2 Rs[CI_B][CI_B + 1];   // CTA 0: working Schur complement
  __shared__ double2 Ws[CI_B][CI_B + 1];   // W_jj (CTA 0 computes, all CTAs copy)
  __shared__ double2 Bs[CI_B][CI_B + 1];   // CTA 0: right-hand sides of the inverse
  __shared__ double invd[CI_B];            // 1 / R_jj[x][x]
  __shared__ double pv[2];                 // current pivot: 1/r, 1/piv
  __shared__ int ok_sh, fail_sh;
  extern __shared__ double2 Zs[];          // rpc x 32: rows of W_{0:J,0:J} X owned here
  const int k = a.k, ld = a.ld;
  double2* G = a.G;
  double2* X = a.X;                        // row-major: X[l * 32 + y]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * CI_WARPS + warp, nwarps = gridDim.x * CI_WARPS;
  const int P = gridDim.x;
  unsigned nbar = 0;

  // strict lower triangle of the output is zero (never read as input)
  for (size_t e = (size_t)blockIdx.x * CI_THREADS + threadIdx.x; e < (size_t)k * k;
       e += (size_t)P * CI_THREADS) {
    const int r = (int)(e % k), c = (int)(e / k);
    if (r > c) G[(size_t)r + (size_t)c * ld] = make_double2(0.0, 0.0);
  }

  const int nb = (k + CI_B - 1) / CI_B;
  for (int j = 0; j < nb; ++j) {
    const int c0 = j * CI_B, bw = min(CI_B, k - c0), J = c0;
    const int nch = (J + CI_CH - 1) / CI_CH;  // row chunks of the Schur sums
    const bool ylane = lane < bw;
    const double2* acol = G + (size_t)(c0 + lane) * ld;  // column c0 + lane of A

    // ---- (a) X[x][y] = sum_{l<=x} conj(W[l][x]) A[l][c0+y]; warp per row, lane = y
    if (J > 0) {
      for (int x = gwarp; x < J; x += nwarps) {
        const double2* wcol = G + (size_t)x * ld;
        double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
        int l = 0;
        for (; l + 1 <= x; l += 2) {
          const double2 w0 = __ldcg(wcol + l), w1 = __ldcg(wcol + l + 1);
          if (ylane) {
            cmac_conj(acc0, w0, __ldcg(acol + l));
            cmac_conj(acc1, w1, __ldcg(acol + l + 1));
          }
        }
        if (l <= x && ylane) cmac_conj(acc0, __ldcg(wcol + l), __ldcg(acol + l));
        if (ylane) X[(size_t)x * CI_B + lane] = make_double2(acc0.x + acc1.x, acc0.y + acc1.y);
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 11, &ok_sh)) return;
    }

    // ---- (b) partial Schur sums Sp[ch][x][y] = sum_{l in chunk} conj(X[l][x]) X[l][y]
    //      (warp per (x, chunk), lane = y), and the rows of Z = W_{0:J,0:J} X
    //      owned by this CTA (warp per row, lane = y; kept in shared memory)
    if (J > 0) {
      for (int t = gwarp; t < bw * nch; t += nwarps) {
        const int x = t % bw, ch = t / bw;
        const int l0 = ch * CI_CH, l1 = min(J, l0 + CI_CH);
        double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
        int l = l0;
        for (; l + 1 < l1; l += 2) {
          const double2 p0 = __ldcg(X + (size_t)l * CI_B + x), p1 = __ldcg(X + (size_t)(l + 1) * CI_B + x);
          if (ylane && lane >= x) {
            cmac_conj(acc0, p0, __ldcg(X + (size_t)l * CI_B + lane));
            cmac_conj(acc1, p1, __ldcg(X + (size_t)(l + 1) * CI_B + lane));
          }
        }
        if (l < l1 && ylane && lane >= x)
          cmac_conj(acc0, __ldcg(X + (size_t)l * CI_B + x), __ldcg(X + (size_t)l * CI_B + lane));
        if (ylane && lane >= x)
          a.S[(size_t)ch * CI_B * CI_B + x + CI_B * lane] = make_double2(acc0.x + acc1.x, acc0.y + acc1.y);
      }
      const int rows = (J - (int)blockIdx.x + P - 1) / P;  // rows x = blockIdx.x + q P < J
      for (int q = warp; q < rows; q += CI_WARPS) {
        const int x = blockIdx.x + q * P;
        double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
        int l = x;
        for (; l + 1 < J; l += 2) {
          const double2 w0 = __ldcg(G + (size_t)x + (size_t)l * ld);
          const double2 w1 = __ldcg(G + (size_t)x + (size_t)(l + 1) * ld);
          if (ylane) {
            cmac(acc0, w0, __ldcg(X + (size_t)l * CI_B + lane));
            cmac(acc1, w1, __ldcg(X + (size_t)(l + 1) * CI_B + lane));
          }
        }
        if (l < J && ylane) cmac(acc0, __ldcg(G + (size_t)x + (size_t)l * ld), __ldcg(X + (size_t)l * CI_B + lane));
        if (ylane) Zs[q * CI_B + lane] = make_double2(acc0.x + acc1.x, acc0.y + acc1.y);
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 12, &ok_sh)) return;
    }

    // ---- (c) R_jj = chol(A_jj - X^H X), W_jj = R_jj^{-1} on CTA 0 -------
    if (blockIdx.x == 0) {
      for (int e = threadIdx.x; e < CI_B * CI_B; e += CI_THREADS) {
        const int x = e % CI_B, y = e / CI_B;
        double2 v = make_double2(x == y ? 1.0 : 0.0, 0.0);
        if (x < bw && y < bw && x <= y) {
          v = __ldcg(G + (size_t)(c0 + x) + (size_t)(c0 + y) * ld);
          for (int ch = 0; ch < nch; ++ch) {  // fixed order
            const double2 sp = __ldcg(a.S + (size_t)ch * CI_B * CI_B + x + CI_B * y);
            v.x -= sp.x;
            v.y -= sp.y;
          }
        }
        Rs[x][y] = v;
        Bs[x][y] = make_double2(x == y ? 1.0 : 0.0, 0.0);
      }
      if (threadIdx.x == 0) fail_sh = 0;
      __syncthreads();
      // right-looking; the pivot's square root and reciprocal are formed
      // once (thread 0) and shared: FP64 sqrt and division are long
      // sequences on the narrow FP64 pipe
      for (int c = 0; c < bw; ++c) {
        if (threadIdx.x == 0) {
          const double piv = Rs[c][c].x;
          if (!(piv > 0.0) || !isfinite(piv)) {
            fail_sh = 1;
            *a.info = c0 + c + 1;
          } else {
            const double r = sqrt(piv), ir = 1.0 / r;
            pv[0] = ir;
            pv[1] = ir * ir;
            invd[c] = ir;
            Rs[c][c] = make_double2(r, 0.0);
          }
        }
        __syncthreads();
        if (fail_sh) break;
        const double ip = pv[1];
        // Rs[x][y] -= conj(Rs[c][x]) Rs[c][y] / piv for c < x <= y (warp ~ y, lane = x)
        for (int y = c + 1 + warp; y < bw; y += CI_WARPS) {
          const int x = lane;
          if (x > c && x <= y) {
            const double2 u = Rs[c][x], v = Rs[c][y];
            const double vr = v.x * ip, vi = v.y * ip;
            Rs[x][y].x -= u.x * vr + u.y * vi;
            Rs[x][y].y -= u.x * vi - u.y * vr;
          }
        }
        __syncthreads();
        // row c of R: Rs[c][y] * (1/r), y > c (read above, written now)
        if (threadIdx.x > c && threadIdx.x < bw) {
          Rs[c][threadIdx.x].x *= pv[0];
          Rs[c][threadIdx.x].y *= pv[0];
        }
      }
      __syncthreads();
      if (!fail_sh) {
        // W = R^{-1} by column-oriented back substitution, columns over the
        // warps and the update of the remaining right-hand side over the
        // lanes (no reductions): for l = y..0: w_l = b_l / R_ll,
        // b_x -= R_xl w_l (x < l)
        for (int y = warp; y < bw; y += CI_WARPS) {
          for (int l = y; l >= 0; --l) {
            const double2 b = Bs[l][y];
            const double2 w = make_double2(b.x * invd[l], b.y * invd[l]);
            if (lane < l) {
              const double2 r = Rs[lane][l];
              Bs[lane][y].x -= r.x * w.x - r.y * w.y;
              Bs[lane][y].y -= r.x * w.y + r.y * w.x;
            }
            if (lane == 0) Ws[l][y] = w;
            __syncwarp();
          }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < bw * bw; e += CI_THREADS) {
          const int x = e % bw, y = e / bw;
          G[(size_t)(c0 + x) + (size_t)(c0 + y) * ld] = x <= y ? Ws[x][y] : make_double2(0.0, 0.0);
        }
      }
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 13, &ok_sh)) return;
    if (__ldcg(a.info) != 0) return;

    // ---- (d) W_{0:J,j} = -Z W_jj for the rows owned by this CTA ---------
    if (J > 0 && (int)blockIdx.x < J) {
      for (int e = threadIdx.x; e < bw * bw; e += CI_THREADS) {
        const int x = e % bw, y = e / bw;
        Ws[x][y] = __ldcg(G + (size_t)(c0 + x) + (size_t)(c0 + y) * ld);
      }
      __syncthreads();
      const int rows = (J - (int)blockIdx.x + P - 1) / P;
      for (int e = threadIdx.x; e < rows * CI_B; e += CI_THREADS) {
        const int q = e / CI_B, y = e - q * CI_B;
        if (y >= bw) continue;
        const int x = blockIdx.x + q * P;
        double2 s = make_double2(0.0, 0.0);
        for (int mm = 0; mm <= y; ++mm) cmac(s, Zs[q * CI_B + mm], Ws[mm][y]);
        G[(size_t)x + (size_t)(c0 + y) * ld] = make_double2(-s.x, -s.y);
      }
    }
    if (J > 0 && !gsync::grid_sync(a.bar, a.flags, nbar++, 14, &ok_sh)) return;
  }
}

}  // namespace

int cholinv_upper(chfsi_ctx* ctx, int k, double2* G) {
  cudaStream_t st = ctx->stream;
  if (k <= 0) return 0;
  const int grid = std::max(1, std::min(ctx->sm_count, (k + 1) / 2));
  const int rpc = (k + grid - 1) / grid;  // rows of each block column per CTA
  const size_t smem = sizeof(double2) * (size_t)rpc * CI_B;
  CHFSI_REQUIRE(smem <= 160 * 1024, "cholinv: k too large");
  static size_t smem_set = 0;
  if (smem > smem_set) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(cholinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)std::max<size_t>(smem, 48 * 1024)));
    smem_set = std::max<size_t>(smem, 48 * 1024);
  }
  int per_sm = 0;
  CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholinv_kernel,
                                                               CI_THREADS, smem));
  CHFSI_REQUIRE(per_sm >= 1, "cholinv: kernel does not fit on an SM");
  CiArgs a;
  a.k = k;
  a.ld = k;
  a.G = G;
  a.X = (double2*)ws_get(ctx, "ci_X", sizeof(double2) * (size_t)k * CI_B);
  a.S = (double2*)ws_get(ctx, "ci_S", sizeof(double2) * CI_B * CI_B * (size_t)((k + CI_CH - 1) / CI_CH + 1));
  char* sync = (char*)ws_get(ctx, "ci_sync", 64);
  a.bar = (unsigned*)sync;
  a.flags = (int*)(sync + 16);
  a.info = (int*)(sync + 32);
  CHFSI_CUDA_TRY(cudaMemsetAsync(sync, 0, 64, st));
  void* args[] = {&a};
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)cholinv_kernel, dim3(grid), dim3(CI_THREADS),
                                             args, smem, st));
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
