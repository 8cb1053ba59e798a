// Spectral bounds of Alg. 1 (Sec. 3.1): m steps of Lanczos with full
// reorthogonalisation from a SplitMix64 start vector, then the extreme
// eigenvalues of the tridiagonal by Sturm-count multisection.
//
// The m steps run in ONE persistent cooperative kernel.  CTA g owns the
// index range [g*chunk, (g+1)*chunk) twice over: as columns of H for the
// mat-vec (w = H x = H^H x, so column c gives entry c; coalesced reads of
// H, streamed past L1/L2) and as rows for every vector operation.
//
// The mat-vec does 4 real FMAs per 16 bytes of H: on GB300's narrow FP64
// pipe that is ALU-bound at about a third of HBM speed.  It therefore reads
// H as FP32 hi/lo pairs (split once per call, same 16 bytes per entry) and
// runs on the FP32 pipe: exact hi*hi products (TwoProd), double-float sums,
// hi*lo cross terms by FMA (about 2^-44 relative per partial sum); the
// partial sums and everything after them are FP64.  The
// mat-vec therefore hands each CTA exactly the rows it owns and needs no
// grid barrier; a step has three: after the partial dots of each of the
// two Gram-Schmidt passes and after the partial norms.  Partial sums are
// written per CTA and every CTA reduces them in the same fixed order, so
// all CTAs hold bitwise identical coefficients and the result does not
// depend on timing.  Every wait is bounded (grid_sync.cuh).
#include "common.cuh"
#include "grid_sync.cuh"

namespace {

constexpr int LZ_THREADS = 512;
constexpr int LZ_WARPS = LZ_THREADS / 32;

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long t) {
  unsigned long long z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry j of the start vector: real and imaginary parts uniform in [-1, 1)
// from draws 2j and 2j+1 of SplitMix64 (53-bit fractions).
__device__ __forceinline__ double2 start_entry(unsigned long long seed, int j) {
  const double sc = 1.1102230246251565e-16;  // 2^-53
  const unsigned long long a = splitmix64_at(seed, 2ull * j) >> 11;
  const unsigned long long b = splitmix64_at(seed, 2ull * j + 1ull) >> 11;
  return make_double2((double)a * sc * 2.0 - 1.0, (double)b * sc * 2.0 - 1.0);
}

struct LzArgs {
  int n, m;
  int chunk;     // indices owned per CTA
  int seg, nseg; // mat-vec column segments (rows per segment, count)
  const float4* Hs;  // H split into FP32 pairs: (re_hi, re_lo, im_hi, im_lo)
  double2* V;     // n x (m + 1), column-major
  double2* xbuf;  // 2 x n: the finished w of the previous step (ping-pong)
  float4* xs;     // 2 x n: the same vectors split into FP32 pairs
  double2* p1;    // gridDim.x x (m + 1) partial dots, first pass
  double2* p2;    // same, second pass
  double* pn;     // gridDim.x partial squared norms
  double* ab;     // alpha[0..m-1], beta[0..m] (beta[m] = start norm)
  unsigned* bar;  // barrier arrival counter (zero at launch)
  int* flags;     // [0] abort, [1] error code
  unsigned long long seed;
};

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc += conj(a) * b
__device__ __forceinline__ void cmac_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ float4 split_c(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih,
                     __double2float_rn(v.y - (double)ih));
}

// Double-float accumulator (hi, lo) for one real sum.
struct DF {
  float hi, lo;
};
// hi + p exactly as (hi', err) (Knuth's TwoSum); err goes to lo.
// (Explicitly rounded intrinsics: no FMA contraction may touch these.)
__device__ __forceinline__ void df_add(DF& s, float p) {
  const float t = __fadd_rn(s.hi, p);
  const float bp = __fsub_rn(t, s.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
  s.hi = t;
}
// s += a * b with the product exact (TwoProd by FMA)
__device__ __forceinline__ void df_mac(DF& s, float a, float b) {
  const float p = __fmul_rn(a, b);
  s.lo = __fadd_rn(s.lo, fmaf(a, b, -p));
  df_add(s, p);
}

// acc += conj(h) x for h, x given as FP32 pairs.  The hi*hi products are
// exact (TwoProd) and summed as double-float; the hi*lo cross terms are
// below 2^-24 of them and go into the low word by plain FMAs; lo*lo
// (2^-48) is dropped.  Relative accuracy about 2^-44 per partial sum.
__device__ __forceinline__ void cmac_conj_split(DF& re, DF& im, float4 h, float4 x) {
  // Re: hr xr + hi xi      Im: hr xi - hi xr
  df_mac(re, h.x, x.x);
  df_mac(re, h.z, x.z);
  re.lo = fmaf(h.x, x.y, re.lo);
  re.lo = fmaf(h.y, x.x, re.lo);
  re.lo = fmaf(h.z, x.w, re.lo);
  re.lo = fmaf(h.w, x.z, re.lo);
  df_mac(im, h.x, x.z);
  df_mac(im, -h.z, x.x);
  im.lo = fmaf(h.x, x.w, im.lo);
  im.lo = fmaf(h.y, x.z, im.lo);
  im.lo = fmaf(-h.z, x.y, im.lo);
  im.lo = fmaf(-h.w, x.x, im.lo);
}

__global__ void split_h_kernel(size_t count, const double2* __restrict__ H, float4* __restrict__ Hs) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    Hs[i] = split_c(__ldcs(H + i));
}

// Sum of the per-CTA partials P[g * ld + i], g = 0..G-1, by one warp in a
// fixed order (lane-strided, then a butterfly): identical in every CTA.
__device__ __forceinline__ double2 reduce_partials(const double2* P, int ld, int i, int G,
                                                   int lane) {
  double2 s = make_double2(0.0, 0.0);
  for (int g = lane; g < G; g += 32) {
    const double2 v = __ldcg(P + (size_t)g * ld + i);
    s.x += v.x;
    s.y += v.y;
  }
  return warp_sum2(s);
}

__global__ void __launch_bounds__(LZ_THREADS, 1)
lanczos_persistent_kernel(LzArgs a) {
  extern __shared__ double2 lz_sm[];
  const int n = a.n, m = a.m, G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * a.chunk;
  const int nown = max(0, min(n, r0 + a.chunk) - r0);
  double2* segp = lz_sm;                                // chunk * nseg mat-vec partials
  double2* wl = segp + (size_t)a.chunk * a.nseg;        // chunk: own rows of w
  double2* h = wl + a.chunk;                            // m + 1 coefficients
  double* red = reinterpret_cast<double*>(h + m + 1);   // LZ_WARPS scratch
  __shared__ int ok_sh;
  __shared__ double bscal[2];  // [0] current beta, [1] alpha accumulator
  unsigned nbar = 0;
  const int ldp = m + 1;

  // Start vector: own rows into xbuf[0], partial norm, barrier, beta[m].
  double sq = 0.0;
  for (int t = threadIdx.x; t < nown; t += LZ_THREADS) {
    const double2 s = start_entry(a.seed, r0 + t);
    a.xbuf[r0 + t] = s;
    a.xs[r0 + t] = split_c(s);
    wl[t] = s;
    sq += s.x * s.x + s.y * s.y;
  }
  sq = warp_sum(sq);
  if (lane == 0) red[warp] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < LZ_WARPS; ++w) s += red[w];
    a.pn[blockIdx.x] = s;
  }
  if (!gsync::grid_sync(a.bar, a.flags, nbar++, 1, &ok_sh)) return;
  if (warp == 0) {
    double s = 0.0;
    for (int g = lane; g < G; g += 32) s += __ldcg(a.pn + g);
    s = warp_sum(s);
    if (lane == 0) {
      bscal[0] = sqrt(s);
      if (blockIdx.x == 0) a.ab[m + m] = sqrt(s);  // beta[m]
    }
  }
  __syncthreads();
  {
    const double inv = 1.0 / bscal[0];
    for (int t = threadIdx.x; t < nown; t += LZ_THREADS)
      a.V[r0 + t] = make_double2(wl[t].x * inv, wl[t].y * inv);
  }

  for (int j = 0; j < m; ++j) {
    // ---- w = H x / beta_prev on the owned columns (x = finished w) ------
    const float4* x = a.xs + (size_t)(j & 1) * n;
    const double inv_b = 1.0 / bscal[0];
    const int ntask = nown * a.nseg;
    for (int t = warp; t < ntask; t += LZ_WARPS) {
      const int cl = t / a.nseg, s = t - cl * a.nseg;
      const float4* col = a.Hs + (size_t)(r0 + cl) * n;
      const int rs = s * a.seg, re = min(n, rs + a.seg);
      // eight 16-byte loads of H in flight per lane, two accumulator pairs
      DF ar[2] = {{0.f, 0.f}, {0.f, 0.f}}, ai[2] = {{0.f, 0.f}, {0.f, 0.f}};
      int r = rs + lane;
      for (; r + 224 < re; r += 256) {
        float4 hv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) hv[u] = __ldcs(col + r + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) cmac_conj_split(ar[u & 1], ai[u & 1], hv[u], __ldcg(x + r + 32 * u));
      }
      for (; r < re; r += 32) cmac_conj_split(ar[0], ai[0], __ldcs(col + r), __ldcg(x + r));
      double2 acc0 = make_double2(((double)ar[0].hi + (double)ar[0].lo) + ((double)ar[1].hi + (double)ar[1].lo),
                                  ((double)ai[0].hi + (double)ai[0].lo) + ((double)ai[1].hi + (double)ai[1].lo));
      acc0 = warp_sum2(acc0);
      if (lane == 0) segp[t] = acc0;
    }
    if (threadIdx.x == 0) bscal[1] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < nown; t += LZ_THREADS) {
      double2 s = make_double2(0.0, 0.0);
      for (int q = 0; q < a.nseg; ++q) {
        s.x += segp[t * a.nseg + q].x;
        s.y += segp[t * a.nseg + q].y;
      }
      wl[t] = make_double2(s.x * inv_b, s.y * inv_b);
    }
    __syncthreads();

    // ---- two classical Gram-Schmidt passes against V[:, 0..j] ----------
    const int J = j + 1;
    for (int pass = 0; pass < 2; ++pass) {
      double2* P = pass == 0 ? a.p1 : a.p2;
      for (int i = warp; i < J; i += LZ_WARPS) {
        const double2* v = a.V + (size_t)i * n + r0;
        double2 d = make_double2(0.0, 0.0);
        for (int t = lane; t < nown; t += 32) cmac_conj(d, v[t], wl[t]);
        d = warp_sum2(d);
        if (lane == 0) P[(size_t)blockIdx.x * ldp + i] = d;
      }
      if (!gsync::grid_sync(a.bar, a.flags, nbar++, 2 + pass, &ok_sh)) return;
      for (int i = warp; i < J; i += LZ_WARPS) {
        const double2 s = reduce_partials(P, ldp, i, G, lane);
        if (lane == 0) h[i] = s;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nown; t += LZ_THREADS) {
        double2 w = wl[t];
        for (int i = 0; i < J; ++i) {
          const double2 v = a.V[(size_t)i * n + r0 + t], c = h[i];
          w.x -= v.x * c.x - v.y * c.y;
          w.y -= v.x * c.y + v.y * c.x;
        }
        wl[t] = w;
      }
      if (threadIdx.x == 0) bscal[1] += h[j].x;
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ab[j] = bscal[1];  // alpha_j

    // ---- beta_j = ||w||, x for the next step, v_{j+1} = w / beta_j -------
    double2* xn = a.xbuf + (size_t)((j + 1) & 1) * n;
    sq = 0.0;
    for (int t = threadIdx.x; t < nown; t += LZ_THREADS) {
      const double2 w = wl[t];
      xn[r0 + t] = w;
      a.xs[(size_t)((j + 1) & 1) * n + r0 + t] = split_c(w);
      sq += w.x * w.x + w.y * w.y;
    }
    sq = warp_sum(sq);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < LZ_WARPS; ++w) s += red[w];
      a.pn[blockIdx.x] = s;
    }
    if (!gsync::grid_sync(a.bar, a.flags, nbar++, 4, &ok_sh)) return;
    if (warp == 0) {
      double s = 0.0;
      for (int g = lane; g < G; g += 32) s += __ldcg(a.pn + g);
      s = warp_sum(s);
      if (lane == 0) {
        bscal[0] = sqrt(s);
        if (blockIdx.x == 0) a.ab[m + j] = sqrt(s);  // beta_j
      }
    }
    __syncthreads();
    const double inv = 1.0 / bscal[0];
    for (int t = threadIdx.x; t < nown; t += LZ_THREADS)
      a.V[(size_t)(j + 1) * n + r0 + t] = make_double2(wl[t].x * inv, wl[t].y * inv);
  }
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x
// (Sturm sequence count with the LDL^T pivots).
__device__ int sturm_count(int m, const double* a, const double* b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    const double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - ((i > 0) ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Extreme eigenvalues of the Lanczos tridiagonal by multisection on Sturm
// counts: one warp, each round splits the bracket into 33 parts and keeps
// the part holding the wanted eigenvalue (5 bits per round instead of 1).
// out4 = {theta_max + beta_m, theta_min, theta_max, max|theta|}, beta_m the
// norm of the last residual vector.  Nothing is written after a timeout of
// the Lanczos kernel (flags[1] != 0): out4 is then NaN.
__global__ void tridiag_bounds_kernel(int m_in, const double* a, const double* b, double* out,
                                      const int* flags) {
  const int lane = threadIdx.x & 31;
  if (flags[1] != 0) {
    if (lane < 4) out[lane] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  // Steps after an (almost) invariant Krylov space are not used: the
  // recurrence stops at the first beta_j <= 1e-14 max(|alpha_j|, 1).
  int m = m_in;
  for (int j = 0; j < m_in; ++j)
    if (!(b[j] > 1e-14 * fmax(fabs(a[j]), 1.0))) {
      m = j + 1;
      break;
    }
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = ((i > 0) ? fabs(b[i - 1]) : 0.0) + ((i < m - 1) ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  double th[2];
  for (int which = 0; which < 2; ++which) {
    const int target = which == 0 ? 1 : m;  // smallest x with count(x) >= target
    double l = lo - 1e-12 * fabs(lo) - 1e-300, h = hi + 1e-12 * fabs(hi) + 1e-300;
    for (int it = 0; it < 40; ++it) {
      const double step = (h - l) / 33.0;
      const double x = l + step * (lane + 1);
      const bool ge = sturm_count(m, a, b, x) >= target;
      const unsigned mask = __ballot_sync(0xffffffffu, ge);
      // first lane whose point has count >= target: new bracket (x_{f-1}, x_f]
      const int f = mask ? __ffs(mask) - 1 : 32;
      const double nl = l + step * f;
      const double nh = (f < 32) ? l + step * (f + 1) : h;
      if (!(nl < nh) || (nl == l && nh == h)) break;
      l = nl;
      h = nh;
      if (h - l <= 4e-16 * fmax(fabs(l), fabs(h))) break;
    }
    th[which] = 0.5 * (l + h);
  }
  if (lane == 0) {
    out[1] = th[0];
    out[2] = th[1];
    out[0] = th[1] + b[m - 1];
    out[3] = fmax(fabs(th[0]), fabs(th[1]));
  }
}

}  // namespace

void lanczos_dev(chfsi_ctx* ctx, const double2* H, int n, int steps, unsigned long long seed,
                 double* out4_dev) {
  cudaStream_t st = ctx->stream;
  const int m = std::min(steps, n);
  const int seg = std::max(1024, ((n + 7) / 8 + 31) / 32 * 32);
  const int nseg = (n + seg - 1) / seg;
  static int per_sm = -1;
  static size_t per_sm_smem = 0;
  // grid: one CTA per SM (or as many as fit), at least 8 indices per CTA
  int G = std::max(1, std::min(ctx->sm_count, (n + 7) / 8));
  int chunk = (n + G - 1) / G;
  size_t smem = sizeof(double2) * ((size_t)chunk * nseg + chunk + m + 1) + sizeof(double) * 32;
  CHFSI_REQUIRE(smem <= 200 * 1024, "Lanczos: n too large for the persistent kernel");
  if (per_sm < 0 || per_sm_smem != smem) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(lanczos_persistent_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)std::max<size_t>(smem, 48 * 1024)));
    CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, lanczos_persistent_kernel, LZ_THREADS, smem));
    per_sm_smem = smem;
  }
  CHFSI_REQUIRE(per_sm >= 1, "Lanczos: persistent kernel does not fit on an SM");

  LzArgs a;
  a.n = n;
  a.m = m;
  a.chunk = chunk;
  a.seg = seg;
  a.nseg = nseg;
  float4* Hs = (float4*)ws_get(ctx, "lz_Hs", sizeof(float4) * (size_t)n * n);
  split_h_kernel<<<ctx->sm_count * 8, 256, 0, st>>>((size_t)n * n, H, Hs);
  chfsi_check_launch("split_h");
  a.Hs = Hs;
  a.V = (double2*)ws_get(ctx, "lz_V", sizeof(double2) * (size_t)n * (m + 1));
  a.xbuf = (double2*)ws_get(ctx, "lz_x", sizeof(double2) * 2 * (size_t)n);
  a.xs = (float4*)ws_get(ctx, "lz_xs", sizeof(float4) * 2 * (size_t)n);
  a.p1 = (double2*)ws_get(ctx, "lz_p1", sizeof(double2) * (size_t)G * (m + 1));
  a.p2 = (double2*)ws_get(ctx, "lz_p2", sizeof(double2) * (size_t)G * (m + 1));
  a.pn = (double*)ws_get(ctx, "lz_pn", sizeof(double) * (size_t)G);
  a.ab = (double*)ws_get(ctx, "lz_ab", sizeof(double) * (2 * (size_t)m + 2));
  a.bar = (unsigned*)ws_get(ctx, "lz_sync", 64);
  a.flags = (int*)((char*)a.bar + 16);
  a.seed = seed;
  CHFSI_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, st));
  void* args[] = {&a};
  const int lz_slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)lanczos_persistent_kernel, dim3(G),
                                             dim3(LZ_THREADS), args, smem, st));
  chfsi_check_launch("lanczos_persistent");
  tridiag_bounds_kernel<<<1, 32, 0, st>>>(m, a.ab, a.ab + m, out4_dev, a.flags);
  chfsi_check_launch("tridiag_bounds");
  kt_end(st, lz_slot, KT_LANCZOS, 0.0);
}

const int* lanczos_error_word(chfsi_ctx* ctx) {
  return (const int*)((char*)ws_get(ctx, "lz_sync", 64) + 20);
}
