// FP64-accurate complex GEMM on the BF16 tensor cores (Ozaki scheme).
//
// GB300 issues FP64 on a narrow pipe (~1.1 TFLOP/s), while its BF16 tensor
// cores run ~1.9 PFLOP/s.  This kernel computes the FP64 products of the
// Rayleigh-Ritz step (Z = H Q, Alg. 1) to ~2^-43 accuracy with
// error-free splitting (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59,
// 2012): every operand row (A) and column (B) is scaled by a power of two
// to [-1, 1] and cut into S slices of 7-bit signed digits (S = 7 for the
// n-sized products up to n = 6144 and 8 above, 8 for the k x k ones of the
// reduced eigensolve)
//     x / scale = sum_{p=1..S} d_p 2^{-7p},  |d_1| <= 128, |d_p| <= 64,
// which BF16 represents exactly.  Digit products are exact (<= 2^14).  The
// sum of the pairs with p + q = t over a K chunk of 512 is at most
// 512 * 2^14 = 2^23 for t = 2 and 512 (2 * 2^13 + (t - 3) 2^12) =
// 2^21 (t + 1) for t >= 3, within 2^24 for t <= 7: the FP32 tensor-core
// accumulation of those groups (one TMEM accumulator each) is exact, and
// the groups t = 8, 9 carry weights 2^-7t <= 2^-56 of the leading one, so
// their FP32 rounding stays below 2^-78 of it.  Pairs with p + q > S + 1 are dropped: with
// the slicing remainder (< 2^-7S) they bound the error by ~2^-(7S-1)
// |scale_row| |scale_col| per product.  S(S+1)/2 slice products (28 for
// S = 7, 36 for S = 8) per output tile and K step.
//
// The complex product is the real GEMM of the filter kernels:
// C (M x 2N) = A (M x 2K) * B (2K x 2N), A rows [Re S | Im S] of the left
// factor, B columns interleaved (Re T_j ; -Im T_j), (Im T_j ; Re T_j).
//
// Kernel layout (one 128 x 64 output tile per CTA, 384 threads):
//   warp 0 lane 0: TMA producer (S A slices + S B slices per 32-wide K block)
//   warp 1 lane 0: tcgen05.mma issuer (S(S+1)/2 slice pairs per 16-wide K step)
//   warp 2:        TMEM allocation (S groups x 64 columns)
//   warps 4-11:    epilogue: after every 512-wide K chunk, drain the S
//                  group accumulators into double-float running sums (two
//                  warps per TMEM lane quarter, one per half of the
//                  columns); at the end scale back and store FP64.
// Waits are bounded as in the filter kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int OZ_SIZE_SWITCH = 6144;  // above: 8 slices for the n-sized products
constexpr int OZ_BETA = 7;     // bits per slice
constexpr int OZ_BK = 32;      // K block (64-byte swizzle rows)
constexpr int OZ_N = 64;       // tile columns (real)
constexpr int OZ_KC = 512;     // exact-accumulation K chunk
constexpr int OZ_THREADS = 384;

// Shared-memory descriptor, K-major, 64-byte swizzle: SBO = 8 rows x 64 B.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Error-free sum of two floats (Knuth): s + err = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bp = s - a;
  err = (a - (s - bp)) + (b - bp);
}

struct OzParams {
  int M, N2, K2;       // rows, real columns (2 x complex), real K (2 x complex)
  int kblocks;         // ceil(K2 / 32)
  int kb_per_split;    // K blocks per split
  int stages;
  const double* sA;    // row scales (powers of two), M
  const double* sB;    // column scales, N2
  double2* C;          // output (complex, column-major, ldc) or partial buffer
  int ldc;
  size_t split_stride; // elements between split partials (0: no split)
  int* err;
};

// OZ_S slices per operand; pairs with p + q <= OZ_S + 1; one TMEM group
// (64 columns) per t = p + q, so OZ_S <= 8.
template <int OZ_S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
               OzParams p) {
  constexpr int OZ_GROUPS = OZ_S;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_slice = BM * OZ_BK * 2;     // 8 KB
  const uint32_t b_slice = OZ_N * OZ_BK * 2;   // 4 KB
  const uint32_t stage_bytes = OZ_S * (a_slice + b_slice);
  uint64_t* bars = (uint64_t*)(smem + (size_t)p.stages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + p.stages;
  uint64_t* accf = bars + 2 * p.stages;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = (uint32_t*)(acce + 1);
  volatile int* abort_sh = (volatile int*)(tmem_slot + 1);
  int* ep_count = (int*)(tmem_slot + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * OZ_N;
  const int kb0 = blockIdx.z * p.kb_per_split;
  const int kb1 = min(p.kblocks, kb0 + p.kb_per_split);
  const int nchunks = (kb1 - kb0 + OZ_KC / OZ_BK - 1) / (OZ_KC / OZ_BK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 1);
    *abort_sh = 0;
    *ep_count = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = kb0, i = 0; kb < kb1; ++kb, ++i) {
      const int s = i % p.stages;
      const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, abort_sh, p.err, 11)) break;
      unsigned char* st = smem + (size_t)s * stage_bytes;
      mbar_arrive_expect_tx(&full[s], stage_bytes);
      for (int sl = 0; sl < OZ_S; ++sl)
        tma_load_3d(st + sl * a_slice, &mA, &full[s], kb * OZ_BK, m0, sl);
      for (int sl = 0; sl < OZ_S; ++sl)
        tma_load_3d(st + OZ_S * a_slice + sl * b_slice, &mB, &full[s], kb * OZ_BK, n0, sl);
      issued = i + 1;
    }
    if (*abort_sh) {
      for (int i = (issued > p.stages ? issued - p.stages : 0); i < issued; ++i) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[i % p.stages], (uint32_t)(i / p.stages) & 1u) &&
               globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(BM, OZ_N);
    bool ok = true;
    int i = 0;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      if (!mbar_wait(acce, ((uint32_t)ch & 1u) ^ 1u, abort_sh, p.err, 12)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int kbc0 = kb0 + ch * (OZ_KC / OZ_BK);
      const int kbc1 = min(kb1, kbc0 + OZ_KC / OZ_BK);
      for (int kb = kbc0; kb < kbc1; ++kb, ++i) {
        const int s = i % p.stages;
        const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
        if (!mbar_wait(&full[s], ph, abort_sh, p.err, 13)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
        const uint32_t sb = sa + OZ_S * a_slice;
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)((kk * 32) >> 4);
          const bool first_k = (kb == kbc0) && (kk == 0);
          uint32_t seen = 0;  // groups written in this K step
#pragma unroll
          for (int pa = 0; pa < OZ_S; ++pa) {
#pragma unroll
            for (int qb = 0; qb < OZ_S; ++qb) {
              const int t = pa + qb;  // 0-based: p + q - 2
              if (t > OZ_S - 1) continue;
              const int g = t;
              const uint32_t acc = (first_k && !(seen & (1u << g))) ? 0u : 1u;
              seen |= 1u << g;
              umma_bf16(tmem + (uint32_t)(g * OZ_N), desc_sw64(sa + pa * a_slice) + adv,
                        desc_sw64(sb + qb * b_slice) + adv, idesc, acc);
            }
          }
        }
        umma_commit(&empty[s]);
      }
      if (!ok) break;
      umma_commit(accf);
    }
  } else if (warp >= 4) {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns of half
    // h = (w - 4) / 4; running sums in double-float (hi, lo).
    const int q = warp & 3;
    const int h = (warp - 4) >> 2;
    const int row = m0 + q * 32 + lane;
    const int c_begin = h * (OZ_N / 2);
    float shi[OZ_N / 2], slo[OZ_N / 2];
#pragma unroll
    for (int c = 0; c < OZ_N / 2; ++c) {
      shi[c] = 0.f;
      slo[c] = 0.f;
    }
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    bool ok = true;
    for (int ch = 0; ch < nchunks; ++ch) {
      if (!mbar_wait(accf, (uint32_t)ch & 1u, abort_sh, p.err, 14)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // chunk value in units of 2^-14: sum_{g} 2^{-7 g} S_{g+2}, added into
      // the (hi, lo) running sums group by group with error-free sums
#pragma unroll
      for (int g = 0; g < OZ_GROUPS; ++g) {
        const float sc = ldexpf(1.f, -OZ_BETA * g);
#pragma unroll
        for (int cc = 0; cc < OZ_N / 2; cc += 16) {
          float v[16];
          __syncwarp();
          tmem_ld16(tq + (uint32_t)(g * OZ_N + c_begin + cc), v);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            float s2, e2;
            two_sum(shi[cc + c], v[c] * sc, s2, e2);
            shi[cc + c] = s2;
            slo[cc + c] += e2;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < OZ_N / 2; ++c) {  // renormalise
        const float t2 = shi[c] + slo[c];
        slo[c] = slo[c] - (t2 - shi[c]);
        shi[c] = t2;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        const int arrived = atomicAdd(ep_count, 1);
        if (arrived == 8 * ch + 7) mbar_arrive(acce);
      }
    }
    if (ok && row < p.M) {
      const double rs = p.sA[row] * 6.103515625e-05;  // 2^-14
#pragma unroll
      for (int c = 0; c < OZ_N / 2; c += 2) {
        const int gc = n0 + c_begin + c;  // even real column = real part
        if (gc >= p.N2) break;
        const int j = gc >> 1;
        const double re = ((double)shi[c] + (double)slo[c]) * rs * p.sB[gc];
        const double im = ((double)shi[c + 1] + (double)slo[c + 1]) * rs * p.sB[gc + 1];
        double2* out = p.C + blockIdx.z * p.split_stride + (size_t)row + (size_t)j * p.ldc;
        *out = make_double2(re, im);
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- operand slicing ------------------------------------------------------
// Integer-only slicing (the FP64 pipe is too narrow for per-digit FP64 math):
// |x| and the row/column maximum come from the IEEE bit patterns, the scaled
// value N = round(x 2^(7 NS) / 2^s) is formed by shifting the 53-bit
// significand, and the digits are balanced base-128 digits of N (least
// significant first, d in [-64, 63], the leading digit takes the rest and
// stays within +-128).  sum_p d_p 2^{-7p} = N 2^{-7 NS} exactly, and
// |x / 2^s - N 2^{-7 NS}| <= 2^{-7 NS - 1}.

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// s with 2^s > |x| for the largest |x| whose bit pattern is `mb` (0 -> 0).
__device__ __forceinline__ int pow2_exponent(unsigned long long mb) {
  if (mb == 0) return 0;
  const int e = (int)(mb >> 52);                // biased exponent
  if (e == 0) return -1022;                     // subnormal: 2^-1022 > |x|
  return e - 1023 + 1;                          // |x| < 2^(e - 1022)
}

template <int NS>
__device__ __forceinline__ void slice_value(double x, int s, __nv_bfloat16* out, size_t stride) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const bool neg = (bits >> 63) != 0;
  const int e = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (e != 0) m |= 1ull << 52;
  // x = m 2^(max(e,1) - 1075); N = round(m 2^sh), sh = max(e,1) - 1075 + 7 NS - s
  const int sh = (e ? e : 1) - 1075 + 7 * NS - s;
  long long N = 0;
  if (m != 0) {
    if (sh >= 0) {
      N = (long long)(m << sh);  // |x| < 2^s keeps N below 2^(7 NS) <= 2^56
    } else if (sh > -64) {
      const int r = -sh;
      N = (long long)((m + (1ull << (r - 1))) >> r);
    }
  }
  if (neg) N = -N;
#pragma unroll
  for (int p = NS - 1; p > 0; --p) {
    int d = (int)(N & 127);
    if (d >= 64) d -= 128;
    N = (N - d) >> 7;
    out[(size_t)p * stride] = __int2bfloat16_rn(d);
  }
  out[0] = __int2bfloat16_rn((int)N);
}

__device__ unsigned long long block_max_bits(unsigned long long v, unsigned long long* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u > v ? u : v;
    }
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  const unsigned long long r = sh[0];
  __syncthreads();
  return r;
}

// A rows from conjugated columns of S (rows x cols, column-major, lds):
// row i = [Re S[:, i] | -Im S[:, i]]  (for Hermitian H this is row i of H;
// for S = Q it is row i of Q^H).  With mu (device scalar) the diagonal
// entry S[i, i] is taken as S[i, i] - mu.  Slices: [sl][i][x], pitch P.
template <int NS>
__global__ void __launch_bounds__(256)
oz_slice_a_conjcols_kernel(int rows, int lds, const double2* __restrict__ S, int P,
                           __nv_bfloat16* __restrict__ out, size_t slice_stride,
                           double* __restrict__ scale, const double* __restrict__ mu) {
  __shared__ unsigned long long sh[8];
  const int i = blockIdx.x;
  const double2* col = S + (size_t)i * lds;
  const double shift = mu ? *mu : 0.0;
  unsigned long long m = 0;
  for (int x = threadIdx.x; x < rows; x += 256) {
    const double re = (x == i) ? col[x].x - shift : col[x].x;
    const unsigned long long a = abs_bits(re), b = abs_bits(col[x].y);
    m = a > m ? a : m;
    m = b > m ? b : m;
  }
  const int se = pow2_exponent(block_max_bits(m, sh));
  if (threadIdx.x == 0) scale[i] = ldexp(1.0, se);
  __nv_bfloat16* o = out + (size_t)i * P;
  for (int x = threadIdx.x; x < rows; x += 256) {
    const double re = (x == i) ? col[x].x - shift : col[x].x;
    slice_value<NS>(re, se, o + x, slice_stride);
    slice_value<NS>(-col[x].y, se, o + rows + x, slice_stride);
  }
}

// mu = mean of Re diag(H) (one block).
__global__ void __launch_bounds__(256) oz_diag_mean_kernel(int n, const double2* H, double* mu) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += H[(size_t)i * n + i].x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    *mu = t / n;
  }
}

// C += mu Q (n x k, both column-major)
__global__ void oz_add_shift_kernel(int n, int k, const double* mu, const double2* Q,
                                    double2* C) {
  const size_t total = (size_t)n * k;
  const double m = *mu;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const double2 q = Q[t];
    double2 c = C[t];
    c.x = fma(m, q.x, c.x);
    c.y = fma(m, q.y, c.y);
    C[t] = c;
  }
}

// A rows from rows of S (rows x cols, column-major, lds): row r =
// [Re S[r, :] | Im S[r, :]].  A block takes 32 rows; the maximum pass reads
// 32 consecutive rows per column (coalesced) and combines the row maxima in
// shared memory.
template <int NS>
__global__ void __launch_bounds__(256)
oz_slice_a_rows_kernel(int nrows, int cols, int lds, const double2* __restrict__ S, int P,
                       __nv_bfloat16* __restrict__ out, size_t slice_stride,
                       double* __restrict__ scale) {
  __shared__ unsigned long long shm[8][32];
  __shared__ int sexp[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + tx;
  unsigned long long m = 0;
  if (r < nrows)
    for (int x = ty; x < cols; x += 8) {
      const double2 v = S[(size_t)r + (size_t)x * lds];
      const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
  shm[ty][tx] = m;
  __syncthreads();
  if (ty == 0) {
    unsigned long long mm = 0;
    for (int t = 0; t < 8; ++t) mm = shm[t][tx] > mm ? shm[t][tx] : mm;
    const int se = pow2_exponent(mm);
    sexp[tx] = se;
    if (r < nrows) scale[r] = ldexp(1.0, se);
  }
  __syncthreads();
  // 32 x 32 tiles through shared memory so that the slice stores run along
  // the row (coalesced) while the loads run down the column.
  __shared__ double2 tile[32][33];
  const int r0 = blockIdx.x * 32;
  for (int x0 = 0; x0 < cols; x0 += 32) {
#pragma unroll
    for (int c = ty; c < 32; c += 8) {
      const int x = x0 + c;
      tile[c][tx] = (r < nrows && x < cols) ? S[(size_t)r + (size_t)x * lds] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int x = x0 + tx;
#pragma unroll
    for (int rr = ty; rr < 32; rr += 8) {
      if (r0 + rr < nrows && x < cols) {
        const double2 v = tile[tx][rr];
        __nv_bfloat16* o = out + (size_t)(r0 + rr) * P;
        slice_value<NS>(v.x, sexp[rr], o + x, slice_stride);
        slice_value<NS>(v.y, sexp[rr], o + cols + x, slice_stride);
      }
    }
    __syncthreads();
  }
}

// B from T (rows x cols complex, column-major, ldt): real column 2j =
// (Re T_j ; -Im T_j), 2j + 1 = (Im T_j ; Re T_j); stored K-major (row 2j of
// B^T), slices [sl][2j][x], pitch P; scale per real column (same for the
// pair).
template <int NS>
__global__ void __launch_bounds__(256)
oz_slice_b_kernel(int rows, int ldt, const double2* __restrict__ T, int P,
                  __nv_bfloat16* __restrict__ out, size_t slice_stride,
                  double* __restrict__ scale) {
  __shared__ unsigned long long sh[8];
  const int j = blockIdx.x;
  const double2* col = T + (size_t)j * ldt;
  unsigned long long m = 0;
  for (int x = threadIdx.x; x < rows; x += 256) {
    const unsigned long long a = abs_bits(col[x].x), b = abs_bits(col[x].y);
    m = a > m ? a : m;
    m = b > m ? b : m;
  }
  const int se = pow2_exponent(block_max_bits(m, sh));
  if (threadIdx.x == 0) {
    scale[2 * j] = ldexp(1.0, se);
    scale[2 * j + 1] = ldexp(1.0, se);
  }
  __nv_bfloat16* o0 = out + (size_t)(2 * j) * P;
  __nv_bfloat16* o1 = o0 + P;
  for (int x = threadIdx.x; x < rows; x += 256) {
    const double re = col[x].x, im = col[x].y;
    slice_value<NS>(re, se, o0 + x, slice_stride);
    slice_value<NS>(-im, se, o0 + rows + x, slice_stride);
    slice_value<NS>(im, se, o1 + x, slice_stride);
    slice_value<NS>(re, se, o1 + rows + x, slice_stride);
  }
}

__global__ void oz_reduce_kernel(int M, int Nc, int splits, const double2* part,
                                 size_t split_stride, int ldp, double2* C, int ldc,
                                 double alpha, double beta) {
  const size_t total = (size_t)M * Nc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), j = (int)(t / M);
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < splits; ++z) {
      const double2 v = part[z * split_stride + i + (size_t)j * ldp];
      s.x += v.x;
      s.y += v.y;
    }
    double2* c = C + i + (size_t)j * ldc;
    double2 o = make_double2(alpha * s.x, alpha * s.y);
    if (beta != 0.0) {
      o.x = fma(beta, c->x, o.x);
      o.y = fma(beta, c->y, o.y);
    }
    *c = o;
  }
}

CUtensorMap make_map3(const void* base, int inner, int rows, int P, int slices, int box_inner,
                      int box_rows, size_t slice_stride_elems) {
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)slices};
  const cuuint64_t strides[2] = {(cuuint64_t)P * 2, (cuuint64_t)slice_stride_elems * 2};
  const cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base),
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw ChfsiError{CHFSI_ECUDA, "cuTensorMapEncodeTiled (3d) failed (" + std::to_string((int)r) + ")"};
  return m;
}

}  // namespace

// Sliced operand storage and the launch.
struct OzOperand {
  __nv_bfloat16* data = nullptr;  // ns slices
  int ns = 6;
  double* scale = nullptr;
  int rows = 0;      // M (A) or 2N (B)
  int K2 = 0;        // real K
  int P = 0;         // pitch (elements)
  size_t stride = 0; // elements per slice
};

static void oz_alloc(chfsi_ctx* ctx, const std::string& name, OzOperand& o, int rows, int K2,
                     int ns) {
  o.ns = ns;
  o.rows = rows;
  o.K2 = K2;
  o.P = (K2 + 7) / 8 * 8;
  o.stride = (size_t)rows * o.P;
  o.data = (__nv_bfloat16*)ws_get(ctx, (name + ".sl").c_str(),
                                  sizeof(__nv_bfloat16) * ns * o.stride + 256);
  o.scale = (double*)ws_get(ctx, (name + ".sc").c_str(), sizeof(double) * (rows + 8));
}

// C (M x Nc complex) = alpha * left * right + beta * C, where the left factor
// is given as A rows (already sliced) and the right factor as B (sliced).
template <int OZ_S>
static void oz_run_t(chfsi_ctx* ctx, const OzOperand& A, const OzOperand& B, double2* C,
                     int ldc, double alpha, double beta) {
  cudaStream_t st = ctx->stream;
  const int M = A.rows, N2 = B.rows, K2 = A.K2;
  const int kblocks = (K2 + OZ_BK - 1) / OZ_BK;
  const int mt = (M + BM - 1) / BM, nt = (N2 + OZ_N - 1) / OZ_N;
  const int tiles = mt * nt;
  // Split K.  One CTA fits per SM, so the time is about (number of waves)
  // x (K blocks per unit + a fixed set-up and drain): pick the split that
  // minimises that -- e.g. 320 tiles on 152 SMs take 3 waves unsplit (the
  // last one 16 CTAs), 13 waves of 1/6 of K split 6 ways; the 30 tiles of
  // a k x k product fill the GPU split 5 ways -- plus a small charge per
  // split for the FP64 partials that oz_reduce adds up.  The exact-sum
  // chunks (512 of K) are counted from each split's start, so any split
  // stays exact.
  int kb_per = kblocks, splits = 1;
  double best = 1e30;
  for (int s = 1; s <= std::min(kblocks, 64); ++s) {
    const int kp = (kblocks + s - 1) / s;
    const int se = (kblocks + kp - 1) / kp;
    if (se != s) continue;
    const double waves = std::ceil((double)tiles * se / ctx->sm_count);
    // a unit also pays a fixed set-up and drain of about 8 K blocks
    const double cost = waves * (kp + 8.0) / (kblocks + 8.0) + (se > 1 ? 0.03 * se : 0.0);
    if (cost < best - 1e-9) {
      best = cost;
      kb_per = kp;
      splits = se;
    }
  }
  const uint32_t stage_bytes = OZ_S * (BM * OZ_BK * 2 + OZ_N * OZ_BK * 2);
  int stages = (int)((220u * 1024u) / stage_bytes);
  stages = std::max(2, std::min(stages, 4));
  const size_t smem = 1024 + (size_t)stages * stage_bytes + 8 * (2 * stages + 2) + 32;
  static bool attr = false;
  if (!attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<OZ_S>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  CUtensorMap mA = make_map3(A.data, K2, M, A.P, OZ_S, OZ_BK, BM, A.stride);
  CUtensorMap mB = make_map3(B.data, K2, N2, B.P, OZ_S, OZ_BK, OZ_N, B.stride);
  int* err = (int*)ws_get(ctx, "oz_err", sizeof(int));
  CHFSI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int Nc = N2 / 2;
  OzParams p;
  p.M = M;
  p.N2 = N2;
  p.K2 = K2;
  p.kblocks = kblocks;
  p.kb_per_split = kb_per;
  p.stages = stages;
  p.sA = A.scale;
  p.sB = B.scale;
  p.err = err;
  const bool direct = splits == 1 && alpha == 1.0 && beta == 0.0;
  double2* part = nullptr;
  if (direct) {
    p.C = C;
    p.ldc = ldc;
    p.split_stride = 0;
  } else {
    part = (double2*)ws_get(ctx, "oz_part", sizeof(double2) * (size_t)splits * M * Nc);
    p.C = part;
    p.ldc = M;
    p.split_stride = (size_t)M * Nc;
  }
  dim3 grid(nt, mt, splits);
  const int slot = kt_begin(st);
  oz_gemm_kernel<OZ_S><<<grid, OZ_THREADS, smem, st>>>(mA, mB, p);
  chfsi_check_launch("oz_gemm");
  kt_end(st, slot, KT_F64, 8.0 * (double)M * Nc * (K2 / 2),
         (double)(OZ_S * (OZ_S + 1) / 2) * 2.0 * (double)M * N2 * K2);
  if (!direct) {
    const size_t total = (size_t)M * Nc;
    oz_reduce_kernel<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0, st>>>(
        M, Nc, splits, part, (size_t)M * Nc, M, C, ldc, alpha, beta);
    chfsi_check_launch("oz_reduce");
  }
}

static void oz_run(chfsi_ctx* ctx, const OzOperand& A, const OzOperand& B, double2* C, int ldc,
                   double alpha, double beta) {
  if (A.ns == 8)
    oz_run_t<8>(ctx, A, B, C, ldc, alpha, beta);
  else if (A.ns == 7)
    oz_run_t<7>(ctx, A, B, C, ldc, alpha, beta);
  else
    oz_run_t<6>(ctx, A, B, C, ldc, alpha, beta);
}

int oz_check_error(chfsi_ctx* ctx) {
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, ws_get(ctx, "oz_err", sizeof(int)), sizeof(int),
                                 cudaMemcpyDeviceToHost, ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return *h;
}

template <int NS>
static void oz_slice_a_conj(cudaStream_t st, int nrows_S, int lds, const double2* S, int count,
                            const OzOperand& A, const double* mu) {
  const int slot = kt_begin(st);
  oz_slice_a_conjcols_kernel<NS><<<count, 256, 0, st>>>(nrows_S, lds, S, A.P, A.data, A.stride,
                                                        A.scale, mu);
  chfsi_check_launch("oz_slice_a_conj");
  kt_end(st, slot, KT_SLICE, 0.0);
}
template <int NS>
static void oz_slice_a_row(cudaStream_t st, int cols, int lds, const double2* S, int count,
                           const OzOperand& A) {
  const int slot = kt_begin(st);
  oz_slice_a_rows_kernel<NS><<<(count + 31) / 32, 256, 0, st>>>(count, cols, lds, S, A.P, A.data,
                                                                A.stride, A.scale);
  chfsi_check_launch("oz_slice_a_rows");
  kt_end(st, slot, KT_SLICE, 0.0);
}
template <int NS>
static void oz_slice_bb(cudaStream_t st, int rows, int ldt, const double2* T, int count,
                        const OzOperand& B) {
  const int slot = kt_begin(st);
  oz_slice_b_kernel<NS><<<count, 256, 0, st>>>(rows, ldt, T, B.P, B.data, B.stride, B.scale);
  chfsi_check_launch("oz_slice_b");
  kt_end(st, slot, KT_SLICE, 0.0);
}
#define OZ_DISPATCH(ns, fn, ...)          \
  do {                                    \
    if ((ns) == 8) fn<8>(__VA_ARGS__);    \
    else if ((ns) == 7) fn<7>(__VA_ARGS__); \
    else fn<6>(__VA_ARGS__);              \
  } while (0)

// Z (n x k) = H Q with H Hermitian n x n, both complex column-major,
// computed as (H - mu I) Q + mu Q with mu = mean(Re diag H): the diagonal of
// a dense Hermitian matrix is often far larger than its other entries and
// would otherwise set each row's scale.  The sliced H - mu I is kept in the
// workspace named after `prefix` and rebuilt when reslice_h is set.
int oz_slices_for(int dim) { return dim > OZ_SIZE_SWITCH ? 8 : 7; }

void oz_hemm(chfsi_ctx* ctx, const std::string& prefix, const double2* H, int n,
             const double2* Q, int k, double2* Z, bool reslice_h) {
  OzOperand A, B;
  const int ns = oz_slices_for(n);
  oz_alloc(ctx, prefix + "ozH", A, n, 2 * n, ns);
  double* mu = (double*)ws_get(ctx, (prefix + "ozH.mu").c_str(), sizeof(double));
  if (reslice_h) {
    oz_diag_mean_kernel<<<1, 256, 0, ctx->stream>>>(n, H, mu);
    chfsi_check_launch("oz_diag_mean");
    OZ_DISPATCH(ns, oz_slice_a_conj, ctx->stream, n, n, H, n, A, mu);
  }
  oz_alloc(ctx, "ozQ", B, 2 * k, 2 * n, ns);
  OZ_DISPATCH(ns, oz_slice_bb, ctx->stream, n, n, Q, k, B);
  oz_run(ctx, A, B, Z, n, 1.0, 0.0);
  const size_t total = (size_t)n * k;
  oz_add_shift_kernel<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0,
                        ctx->stream>>>(n, k, mu, Q, Z);
  chfsi_check_launch("oz_add_shift");
}

// C (k1 x k2) = alpha * L^H R + beta * C with L n x k1, R n x k2.
void oz_gemm_cn(chfsi_ctx* ctx, int k1, int k2, int n, const double2* L, int ldl,
                const double2* R, int ldr, double2* C, int ldc, double alpha, double beta,
                int ns) {
  if (ns <= 0) ns = oz_slices_for(std::max(n, std::max(k1, k2)));
  OzOperand A, B;
  oz_alloc(ctx, "ozL", A, k1, 2 * n, ns);
  OZ_DISPATCH(ns, oz_slice_a_conj, ctx->stream, n, ldl, L, k1, A, nullptr);
  oz_alloc(ctx, "ozR", B, 2 * k2, 2 * n, ns);
  OZ_DISPATCH(ns, oz_slice_bb, ctx->stream, n, ldr, R, k2, B);
  oz_run(ctx, A, B, C, ldc, alpha, beta);
}

// C (m x k2) = alpha * S W + beta * C with S m x k1 (lds), W k1 x k2 (ldw).
void oz_gemm_nn(chfsi_ctx* ctx, int m, int k2, int k1, const double2* S, int lds,
                const double2* W, int ldw, double2* C, int ldc, double alpha, double beta,
                int ns) {
  if (ns <= 0) ns = oz_slices_for(std::max(m, std::max(k1, k2)));
  OzOperand A, B;
  oz_alloc(ctx, "ozS", A, m, 2 * k1, ns);
  OZ_DISPATCH(ns, oz_slice_a_row, ctx->stream, k1, lds, S, m, A);
  oz_alloc(ctx, "ozW", B, 2 * k2, 2 * k1, ns);
  OZ_DISPATCH(ns, oz_slice_bb, ctx->stream, k1, ldw, W, k2, B);
  oz_run(ctx, A, B, C, ldc, alpha, beta);
}
