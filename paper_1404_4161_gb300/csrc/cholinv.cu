// Inverse Cholesky factor of the CholQR step (QR step of Alg. 1): for the
// Hermitian positive definite Gram matrix G = R^H R (k x k) compute
// W = R^{-1} (upper triangular) in place, in ONE persistent cooperative
// kernel, with FP64 or FP32 arithmetic (storage is FP64 either way).
//
// Left-looking by block columns of width 32: with W known for the leading
// J = 32 j columns,
//   X   = W_{0:J,0:J}^H A_{0:J,j}       (= R_{0:J,j}, the panel of R)
//   S   = A_jj - X^H X                  (Schur complement, 32 x 32)
//   R_jj = chol(S),  W_jj = R_jj^{-1}   (one CTA, in shared memory)
//   W_{0:J,j} = -(W_{0:J,0:J} X) W_jj
// so the factor and its inverse come out together and no triangular solve
// is needed.  The three products are "one CTA per output row": the 32
// columns of the block sit on the lanes, the 16 warps of the CTA split the
// reduction index and their partial sums are added in shared memory in a
// fixed order -- short latency chains, no FP64 shuffle reductions (GB300's
// FP64 pipe is about 2 DFMA per clock per SM, and a warp-wide FP64
// instruction costs its full width).  The rows of W_{0:J,0:J} X are formed
// next to S, before the diagonal block is factored, so only the small
// product with W_jj follows it.  The diagonal block (CTA 0) forms each
// pivot's square root and reciprocal once; its inverse is a
// column-oriented substitution with the columns over the warps.  Up to four
// bounded grid barriers per block column (grid_sync.cuh).  The strict
// lower triangle of A is never read and is zeroed at the start.
//
// info: 0, or i (1-based) when the leading minor of order i is not
// (numerically, in the arithmetic used) positive definite -- the pivot is
// <= 0 or not finite; W is then incomplete.
#include "common.cuh"
#include "grid_sync.cuh"

namespace {

constexpr int CI_THREADS = 512;
constexpr int CI_WARPS = CI_THREADS / 32;
constexpr int CI_B = 32;    // block column width
constexpr int CI_RB = 4;    // output rows per CTA batch in the panel products

template <typename R>
struct Cx;
template <>
struct Cx<double> {
  using T = double2;
};
template <>
struct Cx<float> {
  using T = float2;
};

__device__ __forceinline__ double2 to_c(double2 v, double2) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float2) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }

template <typename C>
__device__ __forceinline__ C ldg_c(const double2* p) {
  return to_c(__ldcg(p), C{});
}
// acc += conj(a) * b
template <typename C>
__device__ __forceinline__ void cmac_conj(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * b
template <typename C>
__device__ __forceinline__ void cmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

struct CiArgs {
  int k, ld;
  double2* G;     // in: A (upper part), out: W = R^{-1}, strict lower zero
  void* X;        // scratch, k x 32 row-major (X[l * 32 + y]), arithmetic type
  void* S;        // scratch, 32 x 32 column-major Schur complement
  int* info;      // 0 or the failing pivot (1-based)
  unsigned* bar;  // barrier counter (zero at launch)
  int* flags;     // [0] abort, [1] error code
};

// Sum of red[q][0..15][lane] in a fixed order.
template <typename C>
__device__ __forceinline__ C sum_warps(const C (*red)[CI_WARPS][CI_B], int q, int lane) {
  C s = red[q][0][lane];
#pragma unroll
  for (int w = 1; w < CI_WARPS; ++w) {
    s.x += red[q][w][lane].x;
    s.y += red[q][w][lane].y;
  }
  return s;
}

template <typename R>
__global__ void __launch_bounds__(CI_THREADS, 1) cholinv_kernel(CiArgs a) {
  using C = typename Cx<R>::T;
  __shared__ R invd[CI_B];               // 1 / R_jj[x][x]
  __shared__ R pv[2];                    // current pivot: 1/r, 1/piv
  __shared__ int ok_sh, fail_sh;
  // dynamic shared memory: Rs, Ws, Bs (32 x 33 each), red, then Zs
  extern __shared__ __align__(16) unsigned char ci_dyn[];
  C(*Rs)[CI_B + 1] = reinterpret_cast<C(*)[CI_B + 1]>(ci_dyn);  // CTA 0: Schur complement, then R_jj
  C(*Ws)[CI_B + 1] = Rs + CI_B;          // W_jj (CTA 0 computes, all CTAs copy)
  C(*Bs)[CI_B + 1] = Ws + CI_B;          // CTA 0: right-hand sides of the inverse
  C(*red)[CI_WARPS][CI_B] = reinterpret_cast<C(*)[CI_WARPS][CI_B]>(Bs + CI_B);
  C* Zs = reinterpret_cast<C*>(red + CI_RB);  // rpc x 32: rows of W_{0:J,0:J} X owned here
  const int k = a.k, ld = a.ld;
  double2* G = a.G;
  C* X = reinterpret_cast<C*>(a.X);
  C* S = reinterpret_cast<C*>(a.S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = gridDim.x, bid = blockIdx.x;
  const C zero = {R(0), R(0)};
  unsigned nbar = 0;

  // strict lower triangle of the output is zero (never read as input)
  for (size_t e = (size_t)bid * CI_THREADS + threadIdx.x; e < (size_t)k * k;
       e += (size_t)P * CI_THREADS) {
    const int r = (int)(e % k), c = (int)(e / k);
    if (r > c) G[(size_t)r + (size_t)c * ld] = make_double2(0.0, 0.0);
  }

  const int nb = (k + CI_B - 1) / CI_B;
  for (int j = 0; j < nb; ++j) {
    const int c0 = j * CI_B, bw = min(CI_B, k - c0), J = c0;
    const bool ylane = lane < bw;
    const double2* acol = G + (size_t)(c0 + (ylane ? lane : 0)) * ld;  // column c0 + lane of A
    const int rows = J > bid ? (J - bid + P - 1) / P : 0;  // rows x = bid + q P < J

    // ---- (a) X[x][y] = sum_{l<=x} conj(W[l][x]) A[l][c0+y] -------------
    if (J > 0) {
      for (int q0 = 0; q0 < rows; q0 += CI_RB) {
        const int nq = min(CI_RB, rows - q0);
        for (int qq = 0; qq < nq; ++qq) {
          const int x = bid + (q0 + qq) * P;
          const double2* wcol = G + (size_t)x * ld;
          C acc0 = zero, acc1 = zero;
          int l = warp;
          for (; l + CI_WARPS <= x; l += 2 * CI_WARPS) {
            const C w0 = ldg_c<C>(wcol + l), w1 = ldg_c<C>(wcol + l + CI_WARPS);
            if (ylane) {
              cmac_conj(acc0, w0, ldg_c<C>(acol + l));
              cmac_conj(acc1, w1, ldg_c<C>(acol + l + CI_WARPS));
            }
          }
          if (l <= x && ylane) cmac_conj(acc0, ldg_c<C>(wcol + l), ldg_c<C>(acol + l));
          red[qq][warp][lane] = C{acc0.x + acc1.x, acc0.y + acc1.y};
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nq * CI_B; t += CI_THREADS) {
          const int qq = t / CI_B, y = t % CI_B;
          if (y < bw) X[(size_t)(bid + (q0 + qq) * P) * CI_B + y] = sum_warps(red, qq, y);
        }
        __syncthreads();
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 11, &ok_sh)) return;
    }

    // ---- (b) S = A_jj - X^H X (CTA x mod P owns row x) and the rows of
    //      Z = W_{0:J,0:J} X owned by this CTA (kept in shared memory) ----
    for (int x = bid; x < bw; x += P) {
      C acc0 = zero, acc1 = zero;
      int l = warp;
      for (; l + CI_WARPS < J; l += 2 * CI_WARPS) {
        const C p0 = __ldcg(X + (size_t)l * CI_B + x);
        const C p1 = __ldcg(X + (size_t)(l + CI_WARPS) * CI_B + x);
        if (ylane) {
          cmac_conj(acc0, p0, __ldcg(X + (size_t)l * CI_B + lane));
          cmac_conj(acc1, p1, __ldcg(X + (size_t)(l + CI_WARPS) * CI_B + lane));
        }
      }
      if (l < J && ylane)
        cmac_conj(acc0, __ldcg(X + (size_t)l * CI_B + x), __ldcg(X + (size_t)l * CI_B + lane));
      red[0][warp][lane] = C{acc0.x + acc1.x, acc0.y + acc1.y};
      __syncthreads();
      if (threadIdx.x < bw && threadIdx.x >= x) {
        const int y = threadIdx.x;
        const C s = sum_warps(red, 0, y);
        const C g = ldg_c<C>(G + (size_t)(c0 + x) + (size_t)(c0 + y) * ld);
        S[x + CI_B * y] = C{g.x - s.x, g.y - s.y};
      }
      __syncthreads();
    }
    if (J > 0) {
      for (int q0 = 0; q0 < rows; q0 += CI_RB) {
        const int nq = min(CI_RB, rows - q0);
        for (int qq = 0; qq < nq; ++qq) {
          const int x = bid + (q0 + qq) * P;
          C acc0 = zero, acc1 = zero;
          int l = x + warp;
          for (; l + CI_WARPS < J; l += 2 * CI_WARPS) {
            const C w0 = ldg_c<C>(G + (size_t)x + (size_t)l * ld);
            const C w1 = ldg_c<C>(G + (size_t)x + (size_t)(l + CI_WARPS) * ld);
            if (ylane) {
              cmac(acc0, w0, __ldcg(X + (size_t)l * CI_B + lane));
              cmac(acc1, w1, __ldcg(X + (size_t)(l + CI_WARPS) * CI_B + lane));
            }
          }
          if (l < J && ylane)
            cmac(acc0, ldg_c<C>(G + (size_t)x + (size_t)l * ld), __ldcg(X + (size_t)l * CI_B + lane));
          red[qq][warp][lane] = C{acc0.x + acc1.x, acc0.y + acc1.y};
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nq * CI_B; t += CI_THREADS) {
          const int qq = t / CI_B, y = t % CI_B;
          Zs[(q0 + qq) * CI_B + y] = sum_warps(red, qq, y);
        }
        __syncthreads();
      }
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 12, &ok_sh)) return;

    // ---- (c) R_jj = chol(S), W_jj = R_jj^{-1} on CTA 0 -----------------
    if (bid == 0) {
      for (int e = threadIdx.x; e < CI_B * CI_B; e += CI_THREADS) {
        const int x = e % CI_B, y = e / CI_B;
        C v = C{x == y ? R(1) : R(0), R(0)};
        if (x < bw && y < bw && x <= y) v = __ldcg(S + x + CI_B * y);
        Rs[x][y] = v;
        Bs[x][y] = C{x == y ? R(1) : R(0), R(0)};
      }
      if (threadIdx.x == 0) fail_sh = 0;
      __syncthreads();
      // right-looking; the pivot's square root and reciprocal are formed
      // once (thread 0) and shared
      for (int c = 0; c < bw; ++c) {
        if (threadIdx.x == 0) {
          const R piv = Rs[c][c].x;
          if (!(piv > R(0)) || !isfinite(piv)) {
            fail_sh = 1;
            *a.info = c0 + c + 1;
          } else {
            const R r = sqrt(piv), ir = R(1) / r;
            pv[0] = ir;
            pv[1] = ir * ir;
            invd[c] = ir;
            Rs[c][c] = C{r, R(0)};
          }
        }
        __syncthreads();
        if (fail_sh) break;
        const R ip = pv[1];
        // Rs[x][y] -= conj(Rs[c][x]) Rs[c][y] / piv for c < x <= y (warp ~ y, lane = x)
        for (int y = c + 1 + warp; y < bw; y += CI_WARPS) {
          const int x = lane;
          if (x > c && x <= y) {
            const C u = Rs[c][x], v = Rs[c][y];
            const R vr = v.x * ip, vi = v.y * ip;
            Rs[x][y].x -= u.x * vr + u.y * vi;
            Rs[x][y].y -= u.x * vi - u.y * vr;
          }
        }
        __syncthreads();
        // row c of R: Rs[c][y] / r, y > c (read above, written now)
        if (threadIdx.x > c && threadIdx.x < bw) {
          Rs[c][threadIdx.x].x *= pv[0];
          Rs[c][threadIdx.x].y *= pv[0];
        }
      }
      __syncthreads();
      if (!fail_sh) {
        // W = R^{-1} by column-oriented back substitution, columns over the
        // warps and the update of the remaining right-hand side over the
        // lanes: for l = y..0: w_l = b_l / R_ll, b_x -= R_xl w_l (x < l)
        for (int y = warp; y < bw; y += CI_WARPS) {
          for (int l = y; l >= 0; --l) {
            const C b = Bs[l][y];
            const C w = C{b.x * invd[l], b.y * invd[l]};
            if (lane < l) {
              const C r = Rs[lane][l];
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
          G[(size_t)(c0 + x) + (size_t)(c0 + y) * ld] =
              x <= y ? to_d(Ws[x][y]) : make_double2(0.0, 0.0);
        }
      }
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 13, &ok_sh)) return;
    if (__ldcg(a.info) != 0) return;

    // ---- (d) W_{0:J,j} = -Z W_jj for the rows owned by this CTA ---------
    if (rows > 0) {
      for (int e = threadIdx.x; e < bw * bw; e += CI_THREADS) {
        const int x = e % bw, y = e / bw;
        Ws[x][y] = ldg_c<C>(G + (size_t)(c0 + x) + (size_t)(c0 + y) * ld);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < rows * CI_B; e += CI_THREADS) {
        const int q = e / CI_B, y = e - q * CI_B;
        if (y >= bw) continue;
        C s = zero;
        for (int mm = 0; mm <= y; ++mm) cmac(s, Zs[q * CI_B + mm], Ws[mm][y]);
        G[(size_t)(bid + q * P) + (size_t)(c0 + y) * ld] = to_d(C{-s.x, -s.y});
      }
    }
    if (J > 0 && !gsync::grid_sync(a.bar, a.flags, nbar++, 14, &ok_sh)) return;
  }
}

template <typename R>
int cholinv_run(chfsi_ctx* ctx, int k, double2* G) {
  using C = typename Cx<R>::T;
  cudaStream_t st = ctx->stream;
  if (k <= 0) return 0;
  const int grid = std::max(1, std::min(ctx->sm_count, (k + 1) / 2));
  const int rpc = (k + grid - 1) / grid;  // rows of each block column per CTA
  const size_t smem =
      sizeof(C) * (3 * (size_t)CI_B * (CI_B + 1) + (size_t)CI_RB * CI_WARPS * CI_B + (size_t)rpc * CI_B);
  CHFSI_REQUIRE(smem <= 200 * 1024, "cholinv: k too large");
  static bool attr = false;
  if (!attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(cholinv_kernel<R>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  int per_sm = 0;
  CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholinv_kernel<R>,
                                                               CI_THREADS, smem));
  CHFSI_REQUIRE(per_sm >= 1, "cholinv: kernel does not fit on an SM");
  CiArgs a;
  a.k = k;
  a.ld = k;
  a.G = G;
  a.X = ws_get(ctx, "ci_X", sizeof(double2) * (size_t)k * CI_B);
  a.S = ws_get(ctx, "ci_S", sizeof(double2) * CI_B * CI_B);
  char* sync = (char*)ws_get(ctx, "ci_sync", 64);
  a.bar = (unsigned*)sync;
  a.flags = (int*)(sync + 16);
  a.info = (int*)(sync + 32);
  CHFSI_CUDA_TRY(cudaMemsetAsync(sync, 0, 64, st));
  void* args[] = {&a};
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)cholinv_kernel<R>, dim3(grid),
                                             dim3(CI_THREADS), args, smem, st));
  chfsi_check_launch("cholinv");
  kt_end(st, slot, KT_CHOLINV, 0.0);
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, a.flags, 3 * sizeof(int) + 8, cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  // h[0] abort, h[1] error code, h[2..3] padding, h[4] info
  if (h[1] != 0)
    throw ChfsiError{CHFSI_ETIMEOUT, "cholinv: a bounded grid barrier gave up (code " +
                                         std::to_string(h[1]) + ")"};
  return h[4];
}

}  // namespace

int cholinv_upper(chfsi_ctx* ctx, int k, double2* G) { return cholinv_run<double>(ctx, k, G); }
int cholinv_upper_f32(chfsi_ctx* ctx, int k, double2* G) { return cholinv_run<float>(ctx, k, G); }
