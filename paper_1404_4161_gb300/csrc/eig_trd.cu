// Starting eigenvectors of the reduced Hermitian eigensolve (Rayleigh-Ritz
// step of Alg. 1, G W = W Lambda for the k x k Rayleigh quotient G), to
// FP32 accuracy, without a library eigensolver.  The refinement in
// eig_mixed.cu takes them to FP64 accuracy.
//
//  1. Householder reduction G = Q T Q^H to real symmetric tridiagonal T in
//     FP32 arithmetic (one persistent cooperative launch).  Step j
//     annihilates column j below the subdiagonal with H_j = I - tau v v^H,
//     v = (1, x_2 / (x_1 - beta), ...), beta = -sign(Re x_1) ||x||, so that
//     H_j^H x = beta e_1 with beta real; the trailing block becomes
//     A - v w^H - w v^H with p = tau A v, w = p - (tau/2)(p^H v) v.  Row i
//     of the working matrix lives in the shared memory of CTA i mod G (in
//     global memory when it does not fit), next to row i of Q = H_0 H_1 ...,
//     which is updated in the same pass (q_i <- q_i - tau (q_i . v) v^H).
//     Every CTA recomputes the reflector from the published column (the
//     same data in the same order, so the same bits everywhere); a step
//     needs one grid barrier, after p.
//  2. Eigenvalues of T by multisection of Sturm counts in FP32: one warp
//     per eigenvalue, its 32 lanes count the eigenvalues below 32 points of
//     the current interval (counts of a backward stable recurrence, so the
//     result is within a few FP32 ulps of ||T||).
//  3. Eigenvectors of T by inverse iteration in FP64 (tridiagonal LU with
//     partial pivoting, three solves from a pseudo-random start), all in
//     parallel; the vectors of each run of eigenvalues closer than
//     1e-5 ||T|| are then orthonormalised together (modified Gram-Schmidt),
//     an orthonormal basis of the run's invariant subspace.
//  4. W = Q Z, Z the real eigenvectors of T: on the tensor cores (the
//     FP64-accurate complex GEMM with 6 slices) or, for the FP64 engine, as
//     an FP64 GEMM.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "grid_sync.cuh"

namespace {

constexpr int TRD_THREADS = 256;
constexpr int TRD_WARPS = TRD_THREADS / 32;
constexpr double CLUSTER_REL = 1e-5;  // runs of eigenvalues closer than this x ||T||
constexpr int INV_ITERS = 3;
constexpr int IB = 8;  // rows per batch of the inverse iteration's loads

struct TrdArgs {
  int k, rows;        // order; rows per CTA
  const double2* G;   // k x k, column-major, Hermitian
  float2* gA;         // rows in global memory (gridDim.x * rows * k each for A and Q), or null
  double2* Qh;        // out: Q^H, column-major (conj(Q) row-major)
  double* d;          // out: diagonal of T (k)
  double* e;          // out: off-diagonal of T (k - 1)
  float2* colpub;     // [2][k]: column j + 1 of the rows below it, before step j's update
  float2* pbuf;       // [2][k]: p = tau A v
  double2* part;      // [2][gridDim.x]: per-CTA partial sums of p^H v
  unsigned* bar;
  int* flags;         // [0] abort word, [1] error code
};

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // red may still be read from an earlier use
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < TRD_WARPS; ++w) s += red[w];
  return s;
}

// One grid barrier per step: every CTA holds the column to annihilate (xs)
// in shared memory.  At step j the owners publish column j + 1 of their
// rows as it stands before step j's update; after the barrier every CTA
// knows v and w and forms the next column itself, x' = c - v conj(w_1) -
// w conj(v_1) (c the published column), so no second barrier is needed.
// The published buffers alternate between two halves by step parity: a CTA
// can be at most one step ahead of the slowest one.
__global__ void __launch_bounds__(TRD_THREADS, 1) trd_kernel(TrdArgs a) {
  extern __shared__ __align__(16) unsigned char trd_sm[];
  __shared__ int ok_sh;
  __shared__ double sc[8];
  const int k = a.k, R = a.rows, G = gridDim.x, c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* vs = (float2*)trd_sm;  // v (k)
  float2* wv = vs + k;           // w (k)
  float2* xs = wv + k;           // column to annihilate (k)
  float2* ps = xs + k;           // p, all rows (k)
  float2* cps = ps + k;          // published column (k)
  double* red = (double*)(cps + k);
  float2* A = a.gA ? a.gA + (size_t)c * R * k : (float2*)(red + 2 * TRD_WARPS + 2);
  float2* Q = a.gA ? a.gA + ((size_t)G + c) * R * k : A + (size_t)R * k;

  // rows i = c + r G: A[i][l] = conj(G(l, i)) = G(i, l); Q = I
  for (int r = 0; r < R; ++r) {
    const int i = c + r * G;
    for (int l = tid; l < k; l += TRD_THREADS) {
      float2 v = make_float2(0.f, 0.f), q = make_float2(0.f, 0.f);
      if (i < k) {
        const double2 g = a.G[(size_t)i * k + l];
        v = make_float2((float)g.x, -(float)g.y);
        q = make_float2(i == l ? 1.f : 0.f, 0.f);
      }
      A[(size_t)r * k + l] = v;
      Q[(size_t)r * k + l] = q;
    }
  }
  for (int t = tid; t + 1 < k; t += TRD_THREADS) {  // x of step 0: G(1 + t, 0)
    const double2 g = a.G[1 + t];
    xs[t] = make_float2((float)g.x, (float)g.y);
  }
  __syncthreads();

  unsigned nb = 0;
  for (int j = 0; j + 1 < k; ++j) {
    const int m = k - j - 1, par = j & 1;
    float2* cp = a.colpub + (size_t)par * k;
    float2* pb = a.pbuf + (size_t)par * k;
    double2* pt = a.part + (size_t)par * G;
    double s2 = 0.0;
    for (int t = 1 + tid; t < m; t += TRD_THREADS)
      s2 += (double)xs[t].x * xs[t].x + (double)xs[t].y * xs[t].y;
    s2 = block_sum(s2, red);
    if (tid == 0) {
      const float ar = xs[0].x, ai = xs[0].y;
      float tr = 0.f, ti = 0.f, beta = ar, scr = 0.f, sci = 0.f;
      if (s2 > 0.0 || ai != 0.f) {
        beta = -copysignf(sqrtf((float)((double)ar * ar + (double)ai * ai + s2)), ar);
        const float rb = 1.f / beta;
        tr = (beta - ar) * rb;
        ti = -ai * rb;
        const float dr = ar - beta, rden = 1.f / (dr * dr + ai * ai);  // 1 / (x_1 - beta)
        scr = dr * rden;
        sci = -ai * rden;
      }
      sc[0] = tr;
      sc[1] = ti;
      sc[2] = scr;
      sc[3] = sci;
      if (c == 0) a.e[j] = beta;
      if (c == j % G) a.d[j] = (double)A[(size_t)(j / G) * k + j].x;
    }
    __syncthreads();
    {
      const float scr = (float)sc[2], sci = (float)sc[3];
      for (int t = tid; t < m; t += TRD_THREADS) {
        const float2 xt = xs[t];
        vs[t] = t == 0 ? make_float2(1.f, 0.f)
                       : make_float2(xt.x * scr - xt.y * sci, xt.x * sci + xt.y * scr);
      }
    }
    __syncthreads();
    const float tr = (float)sc[0], ti = (float)sc[1];

    // own rows: Q row update (all rows), p_i = tau (A v)_i (rows i > j),
    // and column j + 1 published for rows i >= j + 2
    double pvr = 0.0, pvi = 0.0;
    for (int r = warp; r < R; r += TRD_WARPS) {
      const int i = c + r * G;
      if (i >= k) break;
      float2* Qr = Q + (size_t)r * k + (j + 1);
      float qr = 0.f, qi = 0.f;
      for (int t = lane; t < m; t += 32) {
        const float2 q = Qr[t], v = vs[t];
        qr += q.x * v.x - q.y * v.y;
        qi += q.x * v.y + q.y * v.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        qr += __shfl_xor_sync(0xffffffffu, qr, o);
        qi += __shfl_xor_sync(0xffffffffu, qi, o);
      }
      // f = tau (q_i . v); q_i[l] -= f conj(v_l)
      const float fr = tr * qr - ti * qi, fi = tr * qi + ti * qr;
      for (int t = lane; t < m; t += 32) {
        const float2 v = vs[t];
        float2 q = Qr[t];
        q.x -= fr * v.x + fi * v.y;
        q.y -= fi * v.x - fr * v.y;
        Qr[t] = q;
      }
      if (i <= j) continue;
      const float2* Ar = A + (size_t)r * k + (j + 1);
      if (lane == 0 && i >= j + 2) __stcg(cp + (i - j - 2), Ar[0]);
      float sr = 0.f, si = 0.f;
      for (int t = lane; t < m; t += 32) {
        const float2 av = Ar[t], v = vs[t];
        sr += av.x * v.x - av.y * v.y;
        si += av.x * v.y + av.y * v.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      const float pr = tr * sr - ti * si, pi = tr * si + ti * sr;
      if (lane == 0) {
        __stcg(pb + (i - j - 1), make_float2(pr, pi));
        const float2 vi = vs[i - j - 1];  // conj(p_i) v_i
        pvr += (double)pr * vi.x + (double)pi * vi.y;
        pvi += (double)pr * vi.y - (double)pi * vi.x;
      }
    }
    __syncthreads();
    if (lane == 0) {
      red[2 * warp] = pvr;
      red[2 * warp + 1] = pvi;
    }
    __syncthreads();
    if (tid == 0) {
      double2 s = make_double2(0.0, 0.0);
      for (int w = 0; w < TRD_WARPS; ++w) {
        s.x += red[2 * w];
        s.y += red[2 * w + 1];
      }
      __stcg(pt + c, s);
    }
    if (!gsync::grid_sync(a.bar, a.flags, nb++, 31, &ok_sh)) return;

    // every load of the other CTAs' results at once: p, the published
    // column and the partial sums of p^H v (fixed order)
    for (int t = tid; t < m; t += TRD_THREADS) {
      ps[t] = __ldcg(pb + t);
      if (t + 1 < m) cps[t] = __ldcg(cp + t);
    }
    if (warp == 0) {
      double sr = 0.0, si = 0.0;
      for (int q = lane; q < G; q += 32) {
        const double2 pp = __ldcg(pt + q);
        sr += pp.x;
        si += pp.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) {  // alpha = -tau (p^H v) / 2
        sc[4] = -0.5 * (sc[0] * sr - sc[1] * si);
        sc[5] = -0.5 * (sc[0] * si + sc[1] * sr);
      }
    }
    __syncthreads();
    const float alr = (float)sc[4], ali = (float)sc[5];
    for (int t = tid; t < m; t += TRD_THREADS) {  // w = p + alpha v
      const float2 p = ps[t], v = vs[t];
      wv[t] = make_float2(p.x + alr * v.x - ali * v.y, p.y + alr * v.y + ali * v.x);
    }
    __syncthreads();
    // A[i][l] -= v_i conj(w_l) + w_i conj(v_l) on own rows i > j
    for (int r = 0; r < R; ++r) {
      const int i = c + r * G;
      if (i >= k) break;
      if (i <= j) continue;
      const float2 vi = vs[i - j - 1], wi = wv[i - j - 1];
      float2* Ar = A + (size_t)r * k + (j + 1);
      for (int t = tid; t < m; t += TRD_THREADS) {
        const float2 vl = vs[t], wl = wv[t];
        float2 av = Ar[t];
        av.x -= vi.x * wl.x + vi.y * wl.y + wi.x * vl.x + wi.y * vl.y;
        av.y -= vi.y * wl.x - vi.x * wl.y + wi.y * vl.x - wi.x * vl.y;
        Ar[t] = av;
      }
    }
    // next column: x'_t = c_t - v_{t+1} conj(w_0) - w_{t+1} conj(v_0), v_0 = 1
    {
      const float2 w0 = wv[0];
      for (int t = tid; t + 1 < m; t += TRD_THREADS) {
        const float2 cv = cps[t], v = vs[t + 1], w = wv[t + 1];
        xs[t] = make_float2(cv.x - (v.x * w0.x + v.y * w0.y) - w.x,
                            cv.y - (v.y * w0.x - v.x * w0.y) - w.y);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && c == (k - 1) % G) a.d[k - 1] = (double)A[(size_t)((k - 1) / G) * k + (k - 1)].x;
  // Q^H column-major = conj(Q) row-major
  for (int r = 0; r < R; ++r) {
    const int i = c + r * G;
    if (i >= k) break;
    for (int l = tid; l < k; l += TRD_THREADS) {
      const float2 q = Q[(size_t)r * k + l];
      a.Qh[(size_t)i * k + l] = make_double2((double)q.x, -(double)q.y);
    }
  }
}

// Eigenvalue j (ascending) of the symmetric tridiagonal T by multisection:
// one warp per eigenvalue; count(x) = number of eigenvalues below x from
// the signs of the LDL^T pivots of T - xI in FP32.
__global__ void __launch_bounds__(256)
tri_bisect_kernel(int k, const double* __restrict__ d, const double* __restrict__ e,
                  double* __restrict__ lam, double* __restrict__ tnorm_out) {
  extern __shared__ float tri_sm[];
  float* sd = tri_sm;
  float* se2 = tri_sm + k;
  __shared__ float rlo[8], rhi[8], rem[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float lo = FLT_MAX, hi = -FLT_MAX, em = 0.f;
  for (int i = tid; i < k; i += blockDim.x) {
    const float di = (float)d[i];
    const float el = i > 0 ? (float)fabs(e[i - 1]) : 0.f;
    const float er = i + 1 < k ? (float)fabs(e[i]) : 0.f;
    sd[i] = di;
    se2[i] = er * er;
    lo = fminf(lo, di - el - er);
    hi = fmaxf(hi, di + el + er);
    em = fmaxf(em, er * er);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    em = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, o));
  }
  if (lane == 0) {
    rlo[warp] = lo;
    rhi[warp] = hi;
    rem[warp] = em;
  }
  __syncthreads();
  lo = rlo[0];
  hi = rhi[0];
  em = rem[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    lo = fminf(lo, rlo[w]);
    hi = fmaxf(hi, rhi[w]);
    em = fmaxf(em, rem[w]);
  }
  const float tn = fmaxf(fabsf(lo), fabsf(hi));
  const float pivmin = FLT_MIN * fmaxf(1.f, em);
  lo -= 4.f * FLT_EPSILON * tn + pivmin;
  hi += 4.f * FLT_EPSILON * tn + pivmin;
  if (blockIdx.x == 0 && tid == 0) *tnorm_out = (double)tn;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= k) return;
  float a = lo, b = hi;
  for (int it = 0; it < 8; ++it) {
    if (b - a <= 2.f * FLT_EPSILON * fmaxf(fabsf(a), fabsf(b)) + pivmin) break;
    const float x = a + (b - a) * (float)(lane + 1) * (1.f / 33.f);
    int cnt = 0;
    float q = 1.f;
    for (int i = 0; i < k; ++i) {
      q = (sd[i] - x) - (i > 0 ? __fdividef(se2[i - 1], q) : 0.f);
      if (fabsf(q) < pivmin) q = -pivmin;
      cnt += q < 0.f;
    }
    const unsigned above = __ballot_sync(0xffffffffu, cnt > j);
    const int f = above ? __ffs(above) - 1 : 32;
    const float xa = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
    const float xb = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
    if (f > 0) a = xa;
    if (f < 32) b = xb;
  }
  if (lane == 0) lam[j] = 0.5 * ((double)a + (double)b);
}

__device__ __forceinline__ double start_value(int i, int j) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1) +
                         0xD1B54A32D192ED03ull * (unsigned long long)(j + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0);  // in [0.5, 1.5)
}

// Inverse iteration for the eigenvectors of T (FP64), one thread per
// eigenvector, 8 threads per CTA (the FP64 pipe is the limit: spread the
// threads over the SMs; measured 14% faster than 32 per CTA at k = 320).  Work arrays are k x k, interleaved by slot
// (element i of the thread's vector at [i * k + slot]) so that a warp's
// accesses coalesce; every recurrence carries its value in registers.
// zt: element i of eigenvector j at zt[i * k + j].  For a run of close
// eigenvalues (FP32 shifts cannot tell them apart) the run's vectors come
// from distinct pseudo-random starts, so they span the run's invariant
// subspace; tri_runs_mgs_kernel orthonormalises them afterwards.
__global__ void __launch_bounds__(32)
tri_invit_kernel(int k, const double* __restrict__ d, const double* __restrict__ e,
                 const double* __restrict__ lam, const double* __restrict__ tnorm_p,
                 double* __restrict__ zt, double* __restrict__ R0, double* __restrict__ U1,
                 double* __restrict__ U2, double* __restrict__ Lm, double* __restrict__ ya,
                 double* __restrict__ yb, unsigned char* __restrict__ piv) {
  const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (j0 >= k) return;
  const double tn = fmax(*tnorm_p, DBL_MIN);
  const int j1 = j0 + 1;
  const size_t K = (size_t)k;
  const double tiny = DBL_EPSILON * tn;
  auto rec = [&](double u) { return 1.0 / (fabs(u) < tiny ? (u < 0.0 ? -tiny : tiny) : u); };
  for (int j = j0; j < j1; ++j) {
    const double sigma = lam[j];
    // LU with partial pivoting of T - sigma I: row i of U is (1/R0, U1, U2).
    // Loops run in batches of IB rows: a batch's loads are issued together,
    // then its part of the recurrence runs on registers.
    double al = d[0] - sigma;
    double cu = k > 1 ? e[0] : 0.0;
    for (int i0 = 0; i0 + 1 < k; i0 += IB) {
      double bb[IB], dd[IB], ee[IB];
#pragma unroll
      for (int u = 0; u < IB; ++u) {
        const int i = i0 + u;
        bb[u] = i + 1 < k ? e[i] : 0.0;
        dd[u] = i + 1 < k ? d[i + 1] : 0.0;
        ee[u] = i + 2 < k ? e[i + 1] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < IB; ++u) {
        const int i = i0 + u;
        if (i + 1 >= k) break;
        const size_t o = (size_t)i * K + j0;
        const double b = bb[u], an = dd[u] - sigma, cn = ee[u];
        if (fabs(b) <= fabs(al)) {
          const double l = al != 0.0 ? b / al : 0.0;
          R0[o] = rec(al);
          U1[o] = cu;
          U2[o] = 0.0;
          Lm[o] = l;
          piv[o] = 0;
          al = an - l * cu;
          cu = cn;
        } else {
          const double l = al / b;
          R0[o] = rec(b);
          U1[o] = an;
          U2[o] = cn;
          Lm[o] = l;
          piv[o] = 1;
          al = cu - l * an;
          cu = -l * cn;
        }
      }
    }
    {
      const size_t o = (size_t)(k - 1) * K + j0;
      R0[o] = rec(al);
      U1[o] = 0.0;
      U2[o] = 0.0;
      Lm[o] = 0.0;
      piv[o] = 0;
    }
    for (int i = 0; i < k; ++i) ya[(size_t)i * K + j0] = start_value(i, j);
    double scale = 1.0;  // applied to ya when it is read
    for (int it = 0; it < INV_ITERS; ++it) {
      // forward: yb = (row operations of the LU) (scale ya)
      double carry = scale * ya[j0];
      for (int i0 = 0; i0 + 1 < k; i0 += IB) {
        double yn[IB], lm[IB];
        unsigned char pv[IB];
#pragma unroll
        for (int u = 0; u < IB; ++u) {
          const int i = i0 + u;
          const size_t o = (size_t)i * K + j0;
          yn[u] = i + 1 < k ? ya[o + K] : 0.0;
          lm[u] = i + 1 < k ? Lm[o] : 0.0;
          pv[u] = i + 1 < k ? piv[o] : 0;
        }
#pragma unroll
        for (int u = 0; u < IB; ++u) {
          const int i = i0 + u;
          if (i + 1 >= k) break;
          const size_t o = (size_t)i * K + j0;
          const double y = scale * yn[u];
          if (pv[u]) {
            yb[o] = y;
            carry = carry - lm[u] * y;
          } else {
            yb[o] = carry;
            carry = y - lm[u] * carry;
          }
        }
      }
      yb[(size_t)(k - 1) * K + j0] = carry;
      // back substitution: ya = U^-1 yb
      double z1 = 0.0, z2 = 0.0, ss = 0.0;
      for (int i1 = k - 1; i1 >= 0; i1 -= IB) {
        double yv[IB], r0[IB], u1[IB], u2[IB];
#pragma unroll
        for (int u = 0; u < IB; ++u) {
          const int i = i1 - u;
          const size_t o = (size_t)(i >= 0 ? i : 0) * K + j0;
          yv[u] = i >= 0 ? yb[o] : 0.0;
          r0[u] = i >= 0 ? R0[o] : 0.0;
          u1[u] = i >= 0 ? U1[o] : 0.0;
          u2[u] = i >= 0 ? U2[o] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < IB; ++u) {
          const int i = i1 - u;
          if (i < 0) break;
          const double z = (yv[u] - u1[u] * z1 - u2[u] * z2) * r0[u];
          ya[(size_t)i * K + j0] = z;
          z2 = z1;
          z1 = z;
          ss += z * z;
        }
      }
      scale = ss > 0.0 ? 1.0 / sqrt(ss) : 1.0;
    }
    for (int i = 0; i < k; ++i) zt[(size_t)i * K + j] = scale * ya[(size_t)i * K + j0];
  }
}

// Runs of eigenvalues closer than CLUSTER_REL ||T||: modified Gram-Schmidt,
// twice, over the run's vectors in index order (one warp per run, its lanes
// over the rows), so the run yields an orthonormal basis of its invariant
// subspace.
__global__ void __launch_bounds__(256)
tri_runs_mgs_kernel(int k, const double* __restrict__ lam, const double* __restrict__ tnorm_p,
                    double* __restrict__ zt) {
  const int lane = threadIdx.x & 31;
  const int j0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (j0 >= k) return;  // uniform across the warp
  const double ctol = CLUSTER_REL * fmax(*tnorm_p, DBL_MIN);
  if (j0 > 0 && lam[j0] - lam[j0 - 1] < ctol) return;  // not the first of its run
  int j1 = j0 + 1;
  while (j1 < k && lam[j1] - lam[j1 - 1] < ctol) ++j1;
  if (j1 - j0 < 2) return;
  const size_t K = (size_t)k;
  for (int j = j0 + 1; j < j1; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int p = j0; p < j; ++p) {
        double dot = 0.0;
        for (int i = lane; i < k; i += 32) dot += zt[(size_t)i * K + p] * zt[(size_t)i * K + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        for (int i = lane; i < k; i += 32) zt[(size_t)i * K + j] -= dot * zt[(size_t)i * K + p];
      }
    double ss = 0.0;
    for (int i = lane; i < k; i += 32) ss += zt[(size_t)i * K + j] * zt[(size_t)i * K + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double r = ss > 0.0 ? 1.0 / sqrt(ss) : 1.0;
    for (int i = lane; i < k; i += 32) zt[(size_t)i * K + j] *= r;
  }
}

// Z (k x k complex, column-major) from the interleaved real eigenvectors.
__global__ void z_complex_kernel(int k, const double* __restrict__ zt, double2* __restrict__ Z) {
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t % k, j = t / k;  // Z(i, j)
    Z[t] = make_double2(zt[i * k + j], 0.0);
  }
}

bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char* s = std::getenv("CHFSI_VERBOSE");
    v = (s && *s && *s != '0') ? 1 : 0;
  }
  return v == 1;
}

}  // namespace

void trd_eigvecs_f32(chfsi_ctx* ctx, int k, const double2* G, double2* W, bool f64_products) {
  cudaStream_t st = ctx->stream;
  const size_t kk = (size_t)k * k;
  // grid: about four rows per CTA, at most one CTA per SM (measured at k = 320
  // to 1000: 4 rows per CTA beat 8, whose cheaper grid barrier does not make
  // up for the longer per-step products)
  const int Gc = std::max(1, std::min(ctx->sm_count, (k + 3) / 4));
  const int R = (k + Gc - 1) / Gc;
  const size_t base = sizeof(float2) * 5 * (size_t)k + sizeof(double) * (2 * TRD_WARPS + 2);
  const size_t rows_bytes = sizeof(float2) * 2 * (size_t)R * k;
  // the five k-vectors of a step stay in shared memory: k <= about 5600
  CHFSI_REQUIRE(base <= 220 * 1024, "reduced eigensolve: k too large for the FP32 start");
  const bool in_smem = base + rows_bytes <= 200 * 1024;
  const size_t smem = in_smem ? base + rows_bytes : base;
  static size_t attr_smem = 0;
  if (smem > 48 * 1024 && smem > attr_smem) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(trd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr_smem = smem;
  }
  int per_sm = 0;
  CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trd_kernel, TRD_THREADS,
                                                               smem));
  CHFSI_REQUIRE(per_sm >= 1, "tridiagonal reduction does not fit on an SM");

  TrdArgs a;
  a.k = k;
  a.rows = R;
  a.G = G;
  a.gA = in_smem ? nullptr
                 : (float2*)ws_get(ctx, "trd_rows", sizeof(float2) * 2 * (size_t)Gc * R * k);
  a.Qh = (double2*)ws_get(ctx, "trd_Qh", sizeof(double2) * kk);
  a.d = (double*)ws_get(ctx, "trd_d", sizeof(double) * (k + 1));
  a.e = (double*)ws_get(ctx, "trd_e", sizeof(double) * (k + 1));
  a.colpub = (float2*)ws_get(ctx, "trd_c", sizeof(float2) * 2 * (size_t)k);
  a.pbuf = (float2*)ws_get(ctx, "trd_p", sizeof(float2) * 2 * (size_t)k);
  a.part = (double2*)ws_get(ctx, "trd_part", sizeof(double2) * 2 * (size_t)Gc);
  a.bar = (unsigned*)ws_get(ctx, "trd_sync", 64);
  a.flags = (int*)((char*)a.bar + 16);
  double* lam = (double*)ws_get(ctx, "trd_lam", sizeof(double) * (k + 1));
  double* tnorm = lam + k;
  double* zt = (double*)ws_get(ctx, "trd_zt", sizeof(double) * kk);
  double* lu = (double*)ws_get(ctx, "trd_lu", sizeof(double) * 6 * kk);
  unsigned char* piv = (unsigned char*)ws_get(ctx, "trd_piv", kk);
  double2* Z = (double2*)ws_get(ctx, "trd_Z", sizeof(double2) * kk);

  const bool v = verbose();
  cudaEvent_t t[4] = {};
  if (v)
    for (auto& x : t) CHFSI_CUDA_TRY(cudaEventCreate(&x));
  if (v) CHFSI_CUDA_TRY(cudaEventRecord(t[0], st));
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, st));
  void* args[] = {&a};
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)trd_kernel, dim3(Gc), dim3(TRD_THREADS), args,
                                             smem, st));
  chfsi_check_launch("trd");
  if (v) CHFSI_CUDA_TRY(cudaEventRecord(t[1], st));
  const size_t bis_smem = sizeof(float) * 2 * (size_t)k;  // d and e^2 of T
  static size_t bis_attr = 0;
  if (bis_smem > 48 * 1024 && bis_smem > bis_attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(tri_bisect_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bis_smem));
    bis_attr = bis_smem;
  }
  tri_bisect_kernel<<<(k + 7) / 8, 256, bis_smem, st>>>(k, a.d, a.e, lam, tnorm);
  chfsi_check_launch("tri_bisect");
  tri_invit_kernel<<<(k + 7) / 8, 8, 0, st>>>(k, a.d, a.e, lam, tnorm, zt, lu, lu + kk,
                                                   lu + 2 * kk, lu + 3 * kk, lu + 4 * kk,
                                                   lu + 5 * kk, piv);
  chfsi_check_launch("tri_invit");
  tri_runs_mgs_kernel<<<(unsigned)(((size_t)k * 32 + 255) / 256), 256, 0, st>>>(k, lam, tnorm, zt);
  chfsi_check_launch("tri_runs_mgs");
  z_complex_kernel<<<(unsigned)std::min<size_t>((kk + 255) / 256, 4096), 256, 0, st>>>(k, zt, Z);
  chfsi_check_launch("z_complex");
  kt_end(st, slot, KT_SOLVER, 0.0);
  if (v) CHFSI_CUDA_TRY(cudaEventRecord(t[2], st));
  if (f64_products)  // W = Q Z
    zgemm_cn(ctx, k, k, k, a.Qh, k, Z, k, W, k, 1.0, 0.0);
  else
    oz_gemm_cn(ctx, k, k, k, a.Qh, k, Z, k, W, k, 1.0, 0.0, 6);
  if (v) CHFSI_CUDA_TRY(cudaEventRecord(t[3], st));
  int* h = (int*)pinned_get(ctx, 256) + 40;
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, a.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  if (*h)
    throw ChfsiError{CHFSI_ETIMEOUT,
                     "tridiagonal reduction: a bounded wait gave up (code " + std::to_string(*h) +
                         ")"};
  if (v) {
    float ms[3];
    for (int i = 0; i < 3; ++i) CHFSI_CUDA_TRY(cudaEventElapsedTime(&ms[i], t[i], t[i + 1]));
    std::fprintf(stderr,
                 "[chfsi] FP32 start k %d: tridiagonal %.3f ms (%d CTAs, rows %s), "
                 "tridiagonal eigenpairs %.3f ms, W = Q Z %.3f ms\n",
                 k, ms[0], Gc, in_smem ? "shared" : "global", ms[1], ms[2]);
    for (auto& x : t) cudaEventDestroy(x);
  }
}
