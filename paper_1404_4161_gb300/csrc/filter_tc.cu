// Split-precision Chebyshev filter on the GB300 tensor cores (tcgen05 +
// TMEM + TMA), sm_103a.
//
// Each step of the Alg. 2 recurrence computes Y_{i+1} = a_i (H Y_i - c Y_i) +
// b_i Y_{i-1} on the active (still unfinished) suffix of the degree-sorted
// block.  The complex product is one real GEMM
//
//     [Hr | Hi] (n x 2n)  *  B (2n x 2k)  ->  [.. Zr_j, Zi_j ..] (n x 2k)
//
// with B's columns interleaved per complex column j: column 2j holds
// (Yr_j ; -Yi_j) and column 2j+1 holds (Yi_j ; Yr_j), so the real and
// imaginary parts of each output element sit in adjacent accumulator
// columns.  A = [Hr | Hi] is built once per problem (row r of A is the
// conjugate of column r of the Hermitian H, read contiguously).
//
// Split format BF16x3: x = hi + lo with hi = bf16(x), lo = bf16(x - hi);
// the product uses hi*hi + hi*lo + lo*hi, all accumulated in one FP32 TMEM
// accumulator (the lo*lo term is below the kept precision).
//
// Kernel layout (one 128 x N output tile per CTA, 256 threads):
//   warp 0 lane 0: TMA producer (A_hi, A_lo, B_hi, B_lo tiles per K block)
//   warp 1 lane 0: tcgen05.mma issuer (3 products x 4 K-steps per block)
//   warp 2:        TMEM allocation / release
//   warps 4-7:     epilogue: tcgen05.ld -> recurrence -> FP32 master of
//                  Y_{i+1}, bf16 hi/lo B operand of the next step, FP64
//                  output for columns that finish at this step.
// Every mbarrier wait is bounded (globaltimer); on timeout the CTA sets an
// error word, lets the other roles drain and releases its TMEM.
//
// "Defect" form (iterative refinement of the filter, not in the paper):
// for Ritz vectors Y with values Lambda and residual block R = HY - Y
// Lambda, the filtered block is p(H) Y = Y psi(Lambda) + D, where psi is
// the scalar recurrence applied to each Ritz value and D follows the same
// three-term recurrence driven by R:
//     D_0 = 0,  D_1 = a_0 R,
//     D_{i+1} = a_i (H D_i - c D_i) + b_i D_{i-1} + a_i psi_i(lambda_j) R_j.
// D is of the size of the residual, so computing it in split precision
// leaves an error of (split precision) x (residual) instead of the split
// precision itself; Y psi(Lambda) is formed in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_ptx.cuh"

namespace {

using namespace tcx;

// ------------------------------------------------------------ kernel ----
struct StepParams {
  int n;          // rows of H
  int ka;         // active complex columns in this launch
  int P;          // row pitch (elements) of the A and B operand arrays
  int ntile;      // N of a tile (real columns, multiple of 16)
  int stages;
  int kblocks;    // ceil(2n / 64)
  uint32_t tmem_cols;
  float a, c, b;  // recurrence scalars of this step
  const float2* cur;    // FP32 master of Y_i (n x ka, ld n), active columns
  const float2* prev;   // FP32 master of Y_{i-1} (null when b == 0)
  const double2* R;     // defect forcing block (null in plain form)
  const double* fR;     // per-column forcing coefficient a_i psi_i(lambda_j)
  float2* next;         // FP32 master of Y_{i+1}
  __nv_bfloat16* bh;    // next B operand, hi (row 2j = column 2j of B), offset
  __nv_bfloat16* bl;    //   to the active start
  double2* out;         // finished columns (c < fin_end) in FP64
  int fin_end;
  int* err;
};

__global__ void __launch_bounds__(NTHREADS, 1)
tc_filter_step_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                      const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                      int b_row0, StepParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int N = p.ntile;
  const uint32_t a_bytes = BM * BK * 2;        // 16 KB per A split
  const uint32_t b_bytes = (uint32_t)N * BK * 2;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  uint64_t* bars = (uint64_t*)(smem + (size_t)p.stages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + p.stages;
  uint64_t* accf = bars + 2 * p.stages;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* abort_sh = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * N;  // first real column of this tile (active-relative)

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(tmem_slot, p.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int kb = 0; kb < p.kblocks; ++kb) {
      const int s = kb % p.stages;
      const uint32_t ph = (uint32_t)(kb / p.stages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, abort_sh, p.err, 1)) break;
      unsigned char* st = smem + (size_t)s * stage_bytes;
      mbar_arrive_expect_tx(&full[s], stage_bytes);
      tma_load_2d(st, &mAh, &full[s], kb * BK, m0);
      tma_load_2d(st + a_bytes, &mAl, &full[s], kb * BK, m0);
      tma_load_2d(st + 2 * a_bytes, &mBh, &full[s], kb * BK, b_row0 + n0);
      tma_load_2d(st + 2 * a_bytes + b_bytes, &mBl, &full[s], kb * BK, b_row0 + n0);
      issued = kb + 1;
    }
    if (*abort_sh) {
      // Let the copies still in flight land before the CTA releases its
      // shared memory (bounded wait on each stage's last armed phase).
      for (int kb = (issued > p.stages ? issued - p.stages : 0); kb < issued; ++kb) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[kb % p.stages], (uint32_t)(kb / p.stages) & 1u) &&
               globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = idesc_bf16(BM, N);
    bool ok = true;
    for (int kb = 0; kb < p.kblocks && ok; ++kb) {
      const int s = kb % p.stages;
      const uint32_t ph = (uint32_t)(kb / p.stages) & 1u;
      if (!mbar_wait(&full[s], ph, abort_sh, p.err, 2)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
      const uint64_t dAh = desc_sw128(sa), dAl = desc_sw128(sa + a_bytes);
      const uint64_t dBh = desc_sw128(sa + 2 * a_bytes), dBl = desc_sw128(sa + 2 * a_bytes + b_bytes);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 B along K
        const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
        umma_bf16(tmem, dAh + adv, dBh + adv, idesc, acc0);
        umma_bf16(tmem, dAh + adv, dBl + adv, idesc, 1u);
        umma_bf16(tmem, dAl + adv, dBh + adv, idesc, 1u);
      }
      umma_commit(&empty[s]);
    }
    if (ok) umma_commit(accf);
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    const bool ok = mbar_wait(accf, 0u, abort_sh, p.err, 3);
    tc_fence_after();
    if (ok) {
      const int n = p.n;
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        __syncwarp();
        tmem_ld16(tq + (uint32_t)c0, v);  // warp-collective: all lanes take part
        if (row >= n) continue;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = (n0 + c0) / 2 + t;  // active-relative complex column
          if (j >= p.ka) break;
          const size_t e = (size_t)row + (size_t)j * n;
          const float2 cu = p.cur[e];
          float re = p.a * (v[2 * t] - p.c * cu.x);
          float im = p.a * (v[2 * t + 1] - p.c * cu.y);
          if (p.prev) {
            const float2 pv = p.prev[e];
            re = fmaf(p.b, pv.x, re);
            im = fmaf(p.b, pv.y, im);
          }
          if (p.R) {
            const double f = p.fR[j];
            const double2 rr = p.R[e];
            re += (float)(f * rr.x);
            im += (float)(f * rr.y);
          }
          p.next[e] = make_float2(re, im);
          __nv_bfloat16 h, l;
          const size_t r0 = (size_t)(2 * j) * p.P, r1 = r0 + p.P;
          split_bf16(re, h, l);
          p.bh[r0 + row] = h;  p.bl[r0 + row] = l;          // column 2j, top:   Yr
          p.bh[r1 + n + row] = h;  p.bl[r1 + n + row] = l;  // column 2j+1, bottom: Yr
          split_bf16(im, h, l);
          p.bh[r1 + row] = h;  p.bl[r1 + row] = l;          // column 2j+1, top: Yi
          split_bf16(-im, h, l);
          p.bh[r0 + n + row] = h;  p.bl[r0 + n + row] = l;  // column 2j, bottom: -Yi
          if (j < p.fin_end) p.out[e] = make_double2((double)re, (double)im);
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, p.tmem_cols);
  }
}

// ------------------------------------------------- operand preparation --
// Row r of A = [Re H[r, :] | Im H[r, :]]; for Hermitian H, H[r, x] =
// conj(H[x, r]), so row r is read from column r (contiguous).
__global__ void repack_h_kernel(int n, int P, const double2* __restrict__ H,
                                __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al) {
  const int r = blockIdx.y;
  const double2* col = H + (size_t)r * n;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < 2 * n; x += gridDim.x * blockDim.x) {
    const double v = (x < n) ? col[x].x : -col[x - n].y;
    const __nv_bfloat16 h = __double2bfloat16(v);
    const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
    Ah[(size_t)r * P + x] = h;
    Al[(size_t)r * P + x] = l;
  }
}

// B operand + FP32 master of an n x k block.  Plain form: src = Y0 (scale
// 1).  Defect form: src = R, scale = a_0 (D_1 = a_0 R).  Columns below
// fin_end are also written to out (FP64) when out is not null.
__global__ void split_block_kernel(int n, int k, int P, const double2* __restrict__ src,
                                   double scale, float2* __restrict__ master,
                                   __nv_bfloat16* __restrict__ bh, __nv_bfloat16* __restrict__ bl,
                                   double2* __restrict__ out, int fin_end) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const size_t e = (size_t)r + (size_t)j * n;
    const double2 s = src[e];
    const float re = (float)(scale * s.x), im = (float)(scale * s.y);
    master[e] = make_float2(re, im);
    if (out && j < fin_end) out[e] = make_double2(scale * s.x, scale * s.y);
    __nv_bfloat16 h, l;
    const size_t r0 = (size_t)(2 * j) * P, r1 = r0 + P;
    split_bf16(re, h, l);
    bh[r0 + r] = h;  bl[r0 + r] = l;
    bh[r1 + n + r] = h;  bl[r1 + n + r] = l;
    split_bf16(im, h, l);
    bh[r1 + r] = h;  bl[r1 + r] = l;
    split_bf16(-im, h, l);
    bh[r0 + n + r] = h;  bl[r0 + n + r] = l;
  }
}

// psi[i * k + j] = psi_i(lambda_j): the filter's scalar recurrence on each
// Ritz value (psi_0 = 1, psi_1 = a_0 (lambda - c), psi_{i+1} = a_i (lambda -
// c) psi_i + b_i psi_{i-1}).  coef = {a_0, (a_i, b_i) for i >= 1}.
__global__ void psi_table_kernel(int k, int m, const double* __restrict__ lam, double c,
                                 const double* __restrict__ coef, double* __restrict__ psi) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const double t = lam[j] - c;
  double p0 = 1.0, p1 = coef[0] * t;
  psi[j] = p0;
  if (m >= 1) psi[(size_t)k + j] = p1;
  for (int i = 1; i < m; ++i) {
    const double p2 = coef[2 * i - 1] * t * p1 + coef[2 * i] * p0;
    psi[(size_t)(i + 1) * k + j] = p2;
    p0 = p1;
    p1 = p2;
  }
}

// Y'_j = Y_j psi_{m_j}(lambda_j) + D_j (FP64), in place on D.
__global__ void defect_combine_kernel(int n, int k, const double2* __restrict__ Y,
                                      const int* __restrict__ deg, const double* __restrict__ psi,
                                      double2* __restrict__ D) {
  const int j = blockIdx.y;
  const double f = psi[(size_t)deg[j] * k + j];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const size_t e = (size_t)r + (size_t)j * n;
    const double2 y = Y[e];
    double2 d = D[e];
    d.x = fma(f, y.x, d.x);
    d.y = fma(f, y.y, d.y);
    D[e] = d;
  }
}

// out[i * k + j] = psi[i * k + j] * a[i]
__global__ void scale_rows_kernel(int rows, int k, const double* __restrict__ psi,
                                  const double* __restrict__ a, double* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * k) return;
  out[t] = psi[t] * a[t / k];
}

// ------------------------------------------------------------ host ------
// Tile N (real columns, multiple of 16, <= 256) for `cols` active real
// columns and `mtiles` row tiles: fewest waves over the SMs, then the
// smallest per-CTA width (a fixed per-tile cost of 32 columns is added).
int pick_ntile(int cols, int mtiles, int sms) {
  int best = 256;
  double best_cost = 1e300;
  for (int N = 32; N <= 256; N += 16) {
    const int tiles = mtiles * ((cols + N - 1) / N);
    const int waves = (tiles + sms - 1) / sms;
    const double cost = (double)waves * (N + 32);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = N;
    }
  }
  return best;
}

}  // namespace

struct TcFilterState {
  int n = 0, P = 0, kcap = 0;
  __nv_bfloat16* A = nullptr;  // A_hi then A_lo, n x P each
  __nv_bfloat16* B = nullptr;  // 2 buffers x (hi, lo) x (2 kcap) x P
  float2* M = nullptr;         // 3 FP32 masters, n x kcap each
  int* err = nullptr;
  size_t a_elems = 0, b_elems = 0;
  bool attr_set = false;
};

int tc_filter_supported(chfsi_ctx* ctx) { return ctx->cc_major == 10 && ctx->cc_minor == 3; }

void tc_filter_release(chfsi_ctx* ctx) {
  TcFilterState* s = ctx->tc;
  if (!s) return;
  cudaFree(s->A);
  cudaFree(s->B);
  cudaFree(s->M);
  cudaFree(s->err);
  delete s;
  ctx->tc = nullptr;
}

static void tc_reserve(chfsi_ctx* ctx, int n, int k) {
  if (!ctx->tc) ctx->tc = new TcFilterState();
  TcFilterState* s = ctx->tc;
  const int P = (2 * n + 7) / 8 * 8;  // 16-byte row pitch for TMA
  if (s->n != n || s->P != P || !s->A) {
    cudaFree(s->A);
    s->A = nullptr;
    s->a_elems = (size_t)n * P;
    CHFSI_CUDA_TRY(cudaMalloc(&s->A, sizeof(__nv_bfloat16) * 2 * s->a_elems));
    s->n = n;
    s->P = P;
    s->kcap = 0;
  }
  if (k > s->kcap) {
    cudaFree(s->B);
    cudaFree(s->M);
    s->B = nullptr;
    s->M = nullptr;
    s->b_elems = (size_t)2 * k * P;
    CHFSI_CUDA_TRY(cudaMalloc(&s->B, sizeof(__nv_bfloat16) * 4 * s->b_elems));
    CHFSI_CUDA_TRY(cudaMalloc(&s->M, sizeof(float2) * 3 * (size_t)n * k));
    s->kcap = k;
  }
  if (!s->err) {
    CHFSI_CUDA_TRY(cudaMalloc(&s->err, sizeof(int)));
    CHFSI_CUDA_TRY(cudaMemsetAsync(s->err, 0, sizeof(int), ctx->stream));
  }
  if (!s->attr_set) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(tc_filter_step_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    s->attr_set = true;
  }
}

void tc_repack_h(cudaStream_t st, int n, int P, const double2* H, void* Ah, void* Al) {
  dim3 grid((2 * n + 255) / 256, n);
  repack_h_kernel<<<grid, 256, 0, st>>>(n, P, H, (__nv_bfloat16*)Ah, (__nv_bfloat16*)Al);
  chfsi_check_launch("repack_h");
}

void tc_split_block(cudaStream_t st, int n, int k, int P, const double2* src, double scale,
                    float2* master, void* bh, void* bl, double2* out, int fin_end) {
  split_block_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(
      n, k, P, src, scale, master, (__nv_bfloat16*)bh, (__nv_bfloat16*)bl, out, fin_end);
  chfsi_check_launch("split_block");
}

void tc_filter_prepare(chfsi_ctx* ctx, const double2* H, int n) {
  tc_reserve(ctx, n, 1);
  TcFilterState* s = ctx->tc;
  dim3 grid((2 * n + 255) / 256, n);
  repack_h_kernel<<<grid, 256, 0, ctx->stream>>>(n, s->P, H, s->A, s->A + s->a_elems);
  chfsi_check_launch("repack_h");
}

namespace {

struct TcRun {
  chfsi_ctx* ctx;
  TcFilterState* s;
  int n, k;
  CUtensorMap mAh, mAl;
  __nv_bfloat16* bh(int buf) { return s->B + (size_t)buf * 2 * s->b_elems; }
  __nv_bfloat16* bl(int buf) { return bh(buf) + s->b_elems; }
  float2* master(int i) { return s->M + (size_t)(i % 3) * n * k; }
};

void launch_step(TcRun& R, int bufB_in, int bufB_out, int s_col, int ka, float a, float c,
                 float b, const float2* cur, const float2* prev, const double2* Rsrc,
                 const double* fR, float2* next, double2* out, int fin_end) {
  TcFilterState* s = R.s;
  const int n = R.n, P = s->P;
  const int cols = 2 * ka;
  const int mtiles = (n + BM - 1) / BM;
  const int N = pick_ntile(cols, mtiles, R.ctx->sm_count);
  const uint32_t stage_bytes = 2u * BM * BK * 2 + 2u * N * BK * 2;
  int stages = (int)((220u * 1024u) / stage_bytes);
  stages = std::max(2, std::min(stages, 6));
  const size_t smem = 1024 + (size_t)stages * stage_bytes + 8 * (2 * stages + 1) + 16;
  uint32_t tcols = 32;
  while ((int)tcols < N) tcols <<= 1;
  CUtensorMap mBh = make_map(R.bh(bufB_in), 2 * n, 2 * R.k, P, N);
  CUtensorMap mBl = make_map(R.bl(bufB_in), 2 * n, 2 * R.k, P, N);
  StepParams p;
  p.n = n;
  p.ka = ka;
  p.P = P;
  p.ntile = N;
  p.stages = stages;
  p.kblocks = (2 * n + BK - 1) / BK;
  p.tmem_cols = tcols;
  p.a = a;
  p.c = c;
  p.b = b;
  p.cur = cur + (size_t)s_col * n;
  p.prev = prev ? prev + (size_t)s_col * n : nullptr;
  p.R = Rsrc ? Rsrc + (size_t)s_col * n : nullptr;
  p.fR = fR ? fR + s_col : nullptr;
  p.next = next + (size_t)s_col * n;
  p.bh = R.bh(bufB_out) + (size_t)(2 * s_col) * P;
  p.bl = R.bl(bufB_out) + (size_t)(2 * s_col) * P;
  p.out = out + (size_t)s_col * n;
  p.fin_end = fin_end;
  p.err = s->err;
  dim3 grid((cols + N - 1) / N, mtiles);
  const int slot = kt_begin(R.ctx->stream);
  tc_filter_step_kernel<<<grid, NTHREADS, smem, R.ctx->stream>>>(R.mAh, R.mAl, mBh, mBl,
                                                                 2 * s_col, p);
  chfsi_check_launch("tc_filter_step");
  kt_end(R.ctx->stream, slot, KT_TC, 8.0 * (double)n * n * ka);
}

void check_err(chfsi_ctx* ctx) {
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, ctx->tc->err, sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (*h) {
    CHFSI_CUDA_TRY(cudaMemsetAsync(ctx->tc->err, 0, sizeof(int), ctx->stream));
    throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core filter: pipeline wait timed out (code " +
                                         std::to_string(*h) + ")"};
  }
}

// Shared driver of both forms.  Plain: Y_0 = Y0, recurrence of Alg. 2.
// Defect: D_0 = 0, D_1 = a_0 R, forcing a_i psi_i R; output D (combined
// with Y psi by the caller).
void run_filter(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* src,
                const double2* Rdef, const double* psi_dev, const int* deg, double lam1,
                double c, double e, double2* out) {
  tc_reserve(ctx, n, k);
  TcFilterState* s = ctx->tc;
  // Rebuilt on every call: the same device buffer may hold a new H.
  tc_filter_prepare(ctx, H, n);
  TcRun R{ctx, s, n, k, {}, {}};
  R.mAh = make_map(s->A, 2 * n, n, s->P, BM);
  R.mAl = make_map(s->A + s->a_elems, 2 * n, n, s->P, BM);
  cudaStream_t st = ctx->stream;
  const bool defect = Rdef != nullptr;
  const int mk = deg[k - 1];
  const double sigma1 = e / (lam1 - c);
  int sidx = (int)(std::upper_bound(deg, deg + k, 1) - deg);
  // Y_1 (plain) or D_1 (defect).
  if (!defect) {
    split_block_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(n, k, s->P, src, 1.0,
                                                                 R.master(0), R.bh(0), R.bl(0),
                                                                 nullptr, 0);
    chfsi_check_launch("split_block");
    launch_step(R, 0, 1, 0, k, (float)(sigma1 / e), (float)c, 0.f, R.master(0), nullptr,
                nullptr, nullptr, R.master(1), out, sidx);
  } else {
    split_block_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(n, k, s->P, Rdef, sigma1 / e,
                                                                 R.master(1), R.bh(1), R.bl(1),
                                                                 out, sidx);
    chfsi_check_launch("split_block");
  }
  double sigma = sigma1;
  for (int i = 1; i < mk; ++i) {
    const double sn = 1.0 / (2.0 / sigma1 - sigma);
    const int s_new = (int)(std::upper_bound(deg, deg + k, i + 1) - deg);
    const float2* prev = (i == 1 && defect) ? nullptr : R.master(i - 1);
    launch_step(R, i & 1, (i + 1) & 1, sidx, k - sidx, (float)(2.0 * sn / e), (float)c,
                (float)(-sn * sigma), R.master(i), prev, defect ? Rdef : nullptr,
                defect ? psi_dev + (size_t)i * k : nullptr, R.master(i + 1), out, s_new - sidx);
    sigma = sn;
    sidx = s_new;
  }
  check_err(ctx);
}

}  // namespace

void tc_filter_run(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y0,
                   const int* deg_host, double lam1, double c, double e, double2* Yout) {
  run_filter(ctx, H, n, k, Y0, nullptr, nullptr, deg_host, lam1, c, e, Yout);
}

// Refinement-form tables for one problem: psi[i][j] = psi_i(lambda_j) and
// the forcing coefficients fR[i][j] = a_i psi_i(lambda_j), (m_k + 1) x k each,
// in context workspaces named after `prefix`.
void tc_defect_tables(chfsi_ctx* ctx, const std::string& prefix, int k, const double* lam,
                      const int* deg_host, double lam1, double c, double e, double** psi_out,
                      double** fR_out) {
  const int mk = deg_host[k - 1];
  std::vector<double> coef(2 * mk + 1, 0.0);
  const double sigma1 = e / (lam1 - c);
  coef[0] = sigma1 / e;
  double sigma = sigma1;
  for (int i = 1; i < mk; ++i) {
    const double sn = 1.0 / (2.0 / sigma1 - sigma);
    coef[2 * i - 1] = 2.0 * sn / e;
    coef[2 * i] = -sn * sigma;
    sigma = sn;
  }
  std::vector<double> ai(mk + 1, 0.0);
  for (int i = 1; i < mk; ++i) ai[i] = coef[2 * i - 1];
  double* dcoef = (double*)ws_get(ctx, (prefix + "tc_coef").c_str(), sizeof(double) * coef.size());
  double* dai = (double*)ws_get(ctx, (prefix + "tc_ai").c_str(), sizeof(double) * (mk + 1));
  double* psi = (double*)ws_get(ctx, (prefix + "tc_psi").c_str(), sizeof(double) * (size_t)(mk + 1) * k);
  double* fR = (double*)ws_get(ctx, (prefix + "tc_fR").c_str(), sizeof(double) * (size_t)(mk + 1) * k);
  double* hbuf = (double*)pinned_get(ctx, sizeof(double) * (coef.size() + ai.size()) + 64);
  std::copy(coef.begin(), coef.end(), hbuf);
  std::copy(ai.begin(), ai.end(), hbuf + coef.size());
  CHFSI_CUDA_TRY(cudaMemcpyAsync(dcoef, hbuf, sizeof(double) * coef.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(dai, hbuf + coef.size(), sizeof(double) * ai.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
  psi_table_kernel<<<(k + 127) / 128, 128, 0, ctx->stream>>>(k, mk, lam, c, dcoef, psi);
  chfsi_check_launch("psi_table");
  scale_rows_kernel<<<(unsigned)(((size_t)(mk + 1) * k + 255) / 256), 256, 0, ctx->stream>>>(
      mk + 1, k, psi, dai, fR);
  chfsi_check_launch("scale_rows");
  // the host staging buffer is reused by the next call: finish the copies
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *psi_out = psi;
  *fR_out = fR;
}

void tc_defect_combine(cudaStream_t st, int n, int k, const double2* Y, const int* deg_dev,
                       const double* psi, double2* out) {
  defect_combine_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(n, k, Y, deg_dev, psi, out);
  chfsi_check_launch("defect_combine");
}

// Defect form: Y (Ritz vectors, degree-sorted), R = HY - Y Lambda (same
// order), lam (Ritz values, device, same order), deg_dev (device copy of
// the degrees).  Yout = p(H) Y per column.
void tc_filter_run_defect(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y,
                          const double2* Rres, const double* lam, const int* deg_host,
                          const int* deg_dev, double lam1, double c, double e, double2* Yout) {
  double *psi, *fR;
  tc_defect_tables(ctx, "", k, lam, deg_host, lam1, c, e, &psi, &fR);
  run_filter(ctx, H, n, k, Y, Rres, fR, deg_host, lam1, c, e, Yout);
  tc_defect_combine(ctx->stream, n, k, Y, deg_dev, psi, Yout);
}
