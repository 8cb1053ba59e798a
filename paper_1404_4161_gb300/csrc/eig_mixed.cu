// Reduced Hermitian eigensolve of the Rayleigh-Ritz step (Alg. 1,
// G W = W Lambda for the k x k Rayleigh quotient) in mixed precision.
//
// GB300's FP64 pipe makes LAPACK-style k x k eigensolvers slow (about
// 14 ms at k = 320 in FP64).  Here the eigenvectors are obtained by
// iterative refinement on FP64-accurate products -- the tensor-core GEMM
// (8 slices per operand, ~2^-56 of the row and column scales), or FP64
// GEMMs on the CUDA cores for the FP64 engine -- after Ogita and Aishima
// ("Iterative refinement for symmetric eigenvalue decomposition", Japan J.
// Indust. Appl. Math. 35, 2018; part II on clustered eigenvalues, 36, 2019),
// written here for complex Hermitian matrices.  One iteration, for the
// current W:
//     S = W^H G W,  M = W^H W,  R = I - M,  lam_i = Re s_ii / Re m_ii.
//   * Converged when max_{i != j} |s_ij| <= 1e-13 max|lam| (ten times the
//     products' error at k = 1000; stopping right at 1e-12 leaves residuals
//     of a few 1e-12) and max |M - I| <= 1e-13.
//   * "Hard" pairs, |s_ij| > max(tau |lam_i - lam_j|, 1e-12 max|lam|)
//     with tau = 1e-2, are those a first-order update cannot resolve
//     (near-degenerate pairs, or a start far from the eigenvectors).  They
//     are looked for within 16 positions of each other in ascending lam;
//     overlapping hard pairs form clusters of consecutive positions, and
//     each cluster's block of S is diagonalised exactly by cyclic Jacobi
//     sweeps in FP64 (one warp per cluster of at most 32), whose rotation
//     is applied to W's columns.  The next iteration recomputes S and M.
//   * Otherwise the first-order update
//         E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)  (i != j, when that
//                is at most tau in modulus and |lam_j - lam_i| is above
//                1e-9 max|lam|),   E_ij = r_ij / 2 otherwise,
//         W <- W + W E,
//     which roughly squares the error, followed by one Newton-Schulz step
//     W <- W (3I - W^H W)/2 (the update loses orthonormality at second
//     order).
// Start: W = I when G itself has no hard pair more than 16 positions apart
// (the warm Rayleigh quotients of a sequence are nearly diagonal: only
// near-degenerate pairs need the cluster step); otherwise the FP32
// eigenvectors of G from a Householder tridiagonal reduction (eig_trd.cu).
// The eigenvalues returned are the Rayleigh quotients lam_i of the final W.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace {

constexpr int EV_BAND = 16;        // hard pairs are searched this far apart in sorted order
constexpr int EV_CHUNK = 32;       // largest block one warp diagonalises
constexpr int EV_WARPS = 4;        // warps (clusters) per CTA of the cluster kernels
constexpr int EV_ROWS = 64;        // rows (columns) per CTA of the rotation updates
constexpr int EV_SMALL = 8;        // larger clusters on the identity start: FP32 start instead
constexpr int EV_LD = EV_CHUNK + 1;
constexpr double EV_TAU = 1e-2;    // first-order update only where |update| <= tau
constexpr double EV_ETA = 1e-12;   // hard pairs: coupling above this x max |lam|
constexpr double EV_EXIT = 1e-13;  // converged off-diagonal, relative to max |lam|
constexpr double EV_ORTH = 1e-13;  // converged max |W^H W - I|
constexpr double EV_DMIN = 1e-9;   // first-order update only across gaps above this x max |lam|
constexpr int EV_MAX_IT = 12;
constexpr int EV_MAX_CLUSTER_STEPS = 4;

struct EvCtl {
  unsigned long long off_bits;    // max_{i != j} |s_ij| (bits of a non-negative double)
  unsigned long long dm_bits;     // max |M - I|
  unsigned long long gnorm_bits;  // max |lam_i|
  int n_hard;                     // hard pairs (i < j)
  int n_out;                      // ... of which more than EV_BAND positions apart
  int n_clusters;                 // blocks in the cluster list
  int max_cluster;                // largest cluster (before splitting into blocks)
};

__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// lam_i = Re s_ii / Re m_ii; max |lam| and the diagonal part of max |M - I|.
__global__ void __launch_bounds__(256)
ev_diag_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
               double* __restrict__ lam, EvCtl* ctl) {
  double g = 0.0, d = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const double2 s = S[(size_t)i * k + i], m = M[(size_t)i * k + i];
    const double l = s.x / m.x;
    lam[i] = l;
    g = fmax(g, fabs(l));
    d = fmax(d, fmax(fabs(1.0 - m.x), fabs(m.y)));
  }
  g = warp_max(g);
  d = warp_max(d);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&ctl->gnorm_bits, dbits(g));
    atomicMax(&ctl->dm_bits, dbits(d));
  }
}

__global__ void ev_pos_kernel(int k, const int* __restrict__ perm, int* __restrict__ pos) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    pos[perm[p]] = p;
}

// Off-diagonal maxima of S and M, and the hard pairs: reach[p] = the largest
// distance d <= EV_BAND such that the pair at sorted positions (p, p + d)
// is hard; hard pairs further apart are counted in n_out.
__global__ void __launch_bounds__(256)
ev_scan_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
               const double* __restrict__ lam, const int* __restrict__ pos, EvCtl* ctl,
               int* __restrict__ reach) {
  const double floor_ = EV_ETA * __longlong_as_double((long long)ctl->gnorm_bits);
  double off = 0.0, dm = 0.0;
  int nh = 0, no = 0;
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    if (i == j) continue;
    const double2 s = S[t], m = M[t];
    const double a = hypot(s.x, s.y);
    off = fmax(off, a);
    dm = fmax(dm, hypot(m.x, m.y));
    if (i < j && a > fmax(EV_TAU * fabs(lam[i] - lam[j]), floor_)) {
      ++nh;
      const int pi = pos[i], pj = pos[j];
      const int lo = min(pi, pj), d = abs(pi - pj);
      if (d > EV_BAND) ++no;
      else atomicMax(&reach[lo], d);
    }
  }
  off = warp_max(off);
  dm = warp_max(dm);
  nh = warp_sum(nh);
  no = warp_sum(no);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&ctl->off_bits, dbits(off));
    atomicMax(&ctl->dm_bits, dbits(dm));
    if (nh) atomicAdd(&ctl->n_hard, nh);
    if (no) atomicAdd(&ctl->n_out, no);
  }
}

// Cluster list from reach[]: positions p and p + 1 belong to one cluster
// when some hard pair (q, q + d) has q <= p < q + d, i.e. when
// max_{q <= p} (q + reach[q]) > p.  Clusters are split into blocks of at
// most EV_CHUNK consecutive positions: clist[b] = (first position, size),
// blocks of size 1 dropped.  One CTA of 1024 threads, each owning a
// contiguous segment of positions: a block-wide max-scan gives the links,
// a block-wide sum-scan the output slots.
constexpr int EVC_T = 1024;
__global__ void __launch_bounds__(EVC_T)
ev_clusters_kernel(int k, const int* __restrict__ reach, unsigned char* __restrict__ link,
                   EvCtl* ctl, int2* __restrict__ clist) {
  __shared__ int sh[EVC_T];
  const int t = threadIdx.x;
  const int L = (k + EVC_T - 1) / EVC_T;
  const int p0 = min(k, t * L), p1 = min(k, p0 + L);
  // 1. links: exclusive max-scan of the segment maxima of (q + reach[q])
  int m = -1;
  for (int p = p0; p < p1; ++p) m = max(m, p + reach[p]);
  sh[t] = m;
  __syncthreads();
  for (int o = 1; o < EVC_T; o <<= 1) {
    const int v = t >= o ? sh[t - o] : -1;
    __syncthreads();
    sh[t] = max(sh[t], v);
    __syncthreads();
  }
  int run = t > 0 ? sh[t - 1] : -1;
  __syncthreads();
  for (int p = p0; p < p1; ++p) {
    run = max(run, p + reach[p]);
    link[p] = run > p ? 1 : 0;
  }
  __syncthreads();
  // 2. clusters start at p with link[p] and not link[p - 1]; the owner of
  // a start walks to its end and counts its blocks
  int nblk = 0, mx = 0;
  for (int p = p0; p < p1; ++p) {
    if (link[p] && (p == 0 || !link[p - 1])) {
      int e = p;
      while (link[e]) ++e;  // link[k - 1] is 0: the walk stops inside the array
      const int size = e - p + 1;
      mx = max(mx, size);
      nblk += size / EV_CHUNK + (size % EV_CHUNK >= 2 ? 1 : 0);
    }
  }
  sh[t] = nblk;
  __syncthreads();
  for (int o = 1; o < EVC_T; o <<= 1) {
    const int v = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  int slot = sh[t] - nblk;
  const int total = sh[EVC_T - 1];
  for (int p = p0; p < p1; ++p) {
    if (link[p] && (p == 0 || !link[p - 1])) {
      int e = p;
      while (link[e]) ++e;
      for (int a = p; a <= e; a += EV_CHUNK) {
        const int sz = min(EV_CHUNK, e - a + 1);
        if (sz >= 2) clist[slot++] = make_int2(a, sz);
      }
    }
  }
  if (mx) atomicMax(&ctl->max_cluster, mx);
  if (t == 0) ctl->n_clusters = total;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}

// One warp per cluster block: cyclic Jacobi on the block A = S[c, c]
// (positions a0 .. a0 + m - 1 in ascending lam, indices perm[]); the
// accumulated rotation V (m x m, V[p][q] at Vstore[ci][q * EV_CHUNK + p])
// is stored for the updates of W, S and M.
// The rotation of pair (p, q), with a_pq = |a_pq| e^{i phi}, is the
// unitary U = [[cs, sn e^{i phi}], [-sn e^{-i phi}, cs]] where (cs, sn)
// is the real symmetric Schur rotation of [[a_pp, |a_pq|], [|a_pq|, a_qq]]
// (zeta = (a_qq - a_pp) / (2 |a_pq|), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), cs = 1 / sqrt(1 + t^2), sn = t cs); U^H A U has a
// zero (p, q) entry.
__global__ void __launch_bounds__(32 * EV_WARPS)
ev_cluster_jacobi_kernel(int k, const double2* __restrict__ S, const int* __restrict__ perm,
                         const int2* __restrict__ clist, const EvCtl* __restrict__ ctl,
                         double2* __restrict__ Vstore) {
  extern __shared__ double2 ev_sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * EV_WARPS + warp;
  if (ci >= ctl->n_clusters) return;  // whole warps only; no block-wide barrier below
  const int2 cl = clist[ci];
  const int a0 = cl.x, m = cl.y;
  double2* A = ev_sm + (size_t)warp * 2 * EV_CHUNK * EV_LD;  // A[p][q] at A[q * EV_LD + p]
  double2* V = A + EV_CHUNK * EV_LD;
  int* cidx = (int*)(ev_sm + (size_t)EV_WARPS * 2 * EV_CHUNK * EV_LD) + warp * EV_CHUNK;
  if (lane < m) cidx[lane] = perm[a0 + lane];
  __syncwarp();
  for (int q = 0; q < m; ++q) {
    if (lane < m) {
      A[q * EV_LD + lane] = S[(size_t)cidx[q] * k + cidx[lane]];
      V[q * EV_LD + lane] = make_double2(lane == q ? 1.0 : 0.0, 0.0);
    }
  }
  __syncwarp();
  double an = 0.0;
  if (lane < m)
    for (int q = 0; q < m; ++q) {
      const double2 v = A[q * EV_LD + lane];
      an += v.x * v.x + v.y * v.y;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) an += __shfl_xor_sync(0xffffffffu, an, o);
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0;
    if (lane < m)
      for (int q = 0; q < m; ++q)
        if (q != lane) {
          const double2 v = A[q * EV_LD + lane];
          off += v.x * v.x + v.y * v.y;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (off <= 1e-30 * an) break;  // off-diagonal below 1e-15 of the block's norm
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double2 apq = A[q * EV_LD + p];
        const double mag = hypot(apq.x, apq.y);
        if (!(mag > 1e-300)) continue;  // uniform across the warp
        const double app = A[p * EV_LD + p].x, aqq = A[q * EV_LD + q].x;
        const double zeta = (aqq - app) / (2.0 * mag);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        const double2 ph = make_double2(apq.x / mag, apq.y / mag);       // e^{i phi}
        const double2 upq = cscale(ph, sn);                              // U_pq
        const double2 uqp = make_double2(-sn * ph.x, sn * ph.y);         // U_qp = -sn e^{-i phi}
        __syncwarp();
        if (lane < m) {  // columns p, q of A and V: [x y] <- [x y] U
          const double2 x = A[p * EV_LD + lane], y = A[q * EV_LD + lane];
          A[p * EV_LD + lane] = cadd(cscale(x, cs), cmul(y, uqp));
          A[q * EV_LD + lane] = cadd(cmul(x, upq), cscale(y, cs));
          const double2 vx = V[p * EV_LD + lane], vy = V[q * EV_LD + lane];
          V[p * EV_LD + lane] = cadd(cscale(vx, cs), cmul(vy, uqp));
          V[q * EV_LD + lane] = cadd(cmul(vx, upq), cscale(vy, cs));
        }
        __syncwarp();
        if (lane < m) {  // rows p, q of A: [x; y] <- U^H [x; y]
          const double2 x = A[lane * EV_LD + p], y = A[lane * EV_LD + q];
          const double2 cupq = make_double2(upq.x, -upq.y), cuqp = make_double2(uqp.x, -uqp.y);
          A[lane * EV_LD + p] = cadd(cscale(x, cs), cmul(cuqp, y));
          A[lane * EV_LD + q] = cadd(cmul(cupq, x), cscale(y, cs));
        }
        __syncwarp();
        if (lane == 0) {
          A[q * EV_LD + p] = make_double2(0.0, 0.0);
          A[p * EV_LD + q] = make_double2(0.0, 0.0);
          A[p * EV_LD + p].y = 0.0;
          A[q * EV_LD + q].y = 0.0;
        }
        __syncwarp();
      }
    }
  }
  double2* vs = Vstore + (size_t)ci * EV_CHUNK * EV_CHUNK;
  for (int q = 0; q < m; ++q)
    if (lane < m) vs[q * EV_CHUNK + lane] = V[q * EV_LD + lane];
}

// Y[r, c] <- sum_p Y[r, c_p] V[p][q] for Y = W, S, M and the rows r of this
// CTA's slice (blockIdx.y): one warp per cluster block, rows in groups of 32
// staged through shared memory.
__global__ void __launch_bounds__(32 * EV_WARPS)
ev_cluster_cols_kernel(int k, double2* __restrict__ W, double2* __restrict__ S,
                       double2* __restrict__ M, const int* __restrict__ perm,
                       const int2* __restrict__ clist, const EvCtl* __restrict__ ctl,
                       const double2* __restrict__ Vstore) {
  extern __shared__ double2 ev_sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * EV_WARPS + warp;
  if (ci >= ctl->n_clusters) return;
  const int2 cl = clist[ci];
  const int a0 = cl.x, m = cl.y;
  double2* T = ev_sm + (size_t)warp * 2 * EV_CHUNK * EV_LD;  // T[lane][p] at T[lane * EV_LD + p]
  double2* V = T + EV_CHUNK * EV_LD;                         // V[p][q] at V[q * EV_LD + p]
  int* cidx = (int*)(ev_sm + (size_t)EV_WARPS * 2 * EV_CHUNK * EV_LD) + warp * EV_CHUNK;
  const double2* vs = Vstore + (size_t)ci * EV_CHUNK * EV_CHUNK;
  if (lane < m) cidx[lane] = perm[a0 + lane];
  for (int q = 0; q < m; ++q)
    if (lane < m) V[q * EV_LD + lane] = vs[q * EV_CHUNK + lane];
  const int r_begin = blockIdx.y * EV_ROWS, r_end = min(k, r_begin + EV_ROWS);
  for (int mat = 0; mat < 3; ++mat) {
    double2* Y = mat == 0 ? W : (mat == 1 ? S : M);
    for (int r0 = r_begin; r0 < r_end; r0 += 32) {
      const int r = r0 + lane;
      __syncwarp();
      if (r < r_end)
        for (int p = 0; p < m; ++p) T[lane * EV_LD + p] = Y[(size_t)cidx[p] * k + r];
      __syncwarp();
      if (r < r_end)
        for (int q = 0; q < m; ++q) {
          double2 acc = make_double2(0.0, 0.0);
          for (int p = 0; p < m; ++p) acc = cadd(acc, cmul(T[lane * EV_LD + p], V[q * EV_LD + p]));
          Y[(size_t)cidx[q] * k + r] = acc;
        }
    }
  }
}

// Rows of the cluster blocks: Y[c, j] <- (V^H Y[c, :])_j for Y = S and M and
// the columns j of this CTA's slice (blockIdx.y), after ev_cluster_cols
// multiplied their columns: S and M become V^H S V and V^H M V with V
// block-diagonal.  One warp per cluster block, lanes over columns.
__global__ void __launch_bounds__(32 * EV_WARPS)
ev_cluster_rows_kernel(int k, double2* __restrict__ S, double2* __restrict__ M,
                       const int* __restrict__ perm, const int2* __restrict__ clist,
                       const EvCtl* __restrict__ ctl, const double2* __restrict__ Vstore) {
  extern __shared__ double2 ev_sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * EV_WARPS + warp;
  if (ci >= ctl->n_clusters) return;
  const int2 cl = clist[ci];
  const int a0 = cl.x, m = cl.y;
  double2* T = ev_sm + (size_t)warp * 2 * EV_CHUNK * EV_LD;  // T[lane][p] at T[lane * EV_LD + p]
  double2* V = T + EV_CHUNK * EV_LD;                         // V[p][q] at V[q * EV_LD + p]
  int* cidx = (int*)(ev_sm + (size_t)EV_WARPS * 2 * EV_CHUNK * EV_LD) + warp * EV_CHUNK;
  const double2* vs = Vstore + (size_t)ci * EV_CHUNK * EV_CHUNK;
  if (lane < m) cidx[lane] = perm[a0 + lane];
  for (int q = 0; q < m; ++q)
    if (lane < m) V[q * EV_LD + lane] = vs[q * EV_CHUNK + lane];
  __syncwarp();
  const int j_begin = blockIdx.y * EV_ROWS, j_end = min(k, j_begin + EV_ROWS);
  for (int mat = 0; mat < 2; ++mat) {
    double2* Y = mat == 0 ? S : M;
    for (int j0 = j_begin; j0 < j_end; j0 += 32) {
      const int j = j0 + lane;
      __syncwarp();
      if (j < j_end)
        for (int p = 0; p < m; ++p) T[lane * EV_LD + p] = Y[(size_t)j * k + cidx[p]];
      __syncwarp();
      if (j < j_end)
        for (int q = 0; q < m; ++q) {
          double2 acc = make_double2(0.0, 0.0);
          for (int p = 0; p < m; ++p) {
            const double2 v = V[q * EV_LD + p];
            acc = cadd(acc, cmul(make_double2(v.x, -v.y), T[lane * EV_LD + p]));
          }
          Y[(size_t)j * k + cidx[q]] = acc;
        }
    }
  }
}

// lam_i = Re s_ii / Re m_ii (after a cluster step).
__global__ void ev_lam_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
                              double* __restrict__ lam) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    lam[i] = S[(size_t)i * k + i].x / M[(size_t)i * k + i].x;
}

// E of the first-order update (R = I - M): E_ij = (s_ij + lam_j r_ij) /
// (lam_j - lam_i) when that has modulus <= tau and the gap is above
// EV_DMIN max|lam|, else r_ij / 2.  The numerator carries rounding noise of
// order u ||G||; over a gap at that scale the quotient is noise, and
// applying it would undo the exact rotations of a near-degenerate cluster
// (whose pairs are left to the cluster step, or are already converged).
__global__ void oa_e_kernel(int k, const double2* __restrict__ S, const double2* __restrict__ M,
                            const double* __restrict__ lam, const EvCtl* __restrict__ ctl,
                            double2* __restrict__ E) {
  const double dmin = EV_DMIN * __longlong_as_double((long long)ctl->gnorm_bits);
  const size_t total = (size_t)k * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double2 m = M[t];
    const double2 r = make_double2((i == j ? 1.0 : 0.0) - m.x, -m.y);
    double2 e = make_double2(0.5 * r.x, 0.5 * r.y);
    if (i != j) {
      const double d = lam[j] - lam[i];
      const double2 s = S[t];
      const double2 num = make_double2(s.x + lam[j] * r.x, s.y + lam[j] * r.y);
      if (fabs(d) > dmin && hypot(num.x, num.y) <= EV_TAU * fabs(d))
        e = make_double2(num.x / d, num.y / d);
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

unsigned grid_k2(int k) {
  const size_t t = (size_t)k * k;
  return (unsigned)std::min<size_t>((t + 255) / 256, 1024);
}

struct EvHost {
  double off, dm, gnorm;
  int n_hard, n_out, n_clusters, max_cluster;
};

}  // namespace

// Eigenvalues (ascending) into w, eigenvectors into G (k x k, ld k).
void reduced_eigh_mixed(chfsi_ctx* ctx, int k, double2* G, double* w, bool f64_products) {
  cudaStream_t st = ctx->stream;
  const size_t kk = (size_t)k * k;
  double2* W = (double2*)ws_get(ctx, "eig_W", sizeof(double2) * kk);
  double2* W2 = (double2*)ws_get(ctx, "eig_W2", sizeof(double2) * kk);
  double2* GW = (double2*)ws_get(ctx, "eig_GW", sizeof(double2) * kk);
  double2* S = (double2*)ws_get(ctx, "eig_S", sizeof(double2) * kk);
  double2* M = (double2*)ws_get(ctx, "eig_M", sizeof(double2) * kk);
  double2* E = (double2*)ws_get(ctx, "eig_E", sizeof(double2) * kk);
  double* lam = (double*)ws_get(ctx, "eig_lam", sizeof(double) * k);
  int* perm = (int*)ws_get(ctx, "eig_perm", sizeof(int) * k);
  int* pos = (int*)ws_get(ctx, "eig_pos", sizeof(int) * k);
  int* reach = (int*)ws_get(ctx, "eig_reach", sizeof(int) * k);
  unsigned char* link = (unsigned char*)ws_get(ctx, "eig_link", (size_t)k);
  int2* clist = (int2*)ws_get(ctx, "eig_clist", sizeof(int2) * (k / 2 + 1));
  EvCtl* ctl = (EvCtl*)ws_get(ctx, "eig_ctl", sizeof(EvCtl));
  EvCtl* ctl_h = (EvCtl*)pinned_get(ctx, 256);
  const unsigned g1 = (unsigned)std::min(1024, (k + 255) / 256);

  // S, M of the current W, lam, sorted order and the hard-pair analysis.
  auto analyze = [&]() -> EvHost {
    const int slot = kt_begin(st);
    CHFSI_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(EvCtl), st));
    CHFSI_CUDA_TRY(cudaMemsetAsync(reach, 0, sizeof(int) * k, st));
    ev_diag_kernel<<<g1, 256, 0, st>>>(k, S, M, lam, ctl);
    chfsi_check_launch("ev_diag");
    sort_by_value(st, k, lam, perm);
    ev_pos_kernel<<<g1, 256, 0, st>>>(k, perm, pos);
    chfsi_check_launch("ev_pos");
    ev_scan_kernel<<<grid_k2(k), 256, 0, st>>>(k, S, M, lam, pos, ctl, reach);
    chfsi_check_launch("ev_scan");
    ev_clusters_kernel<<<1, EVC_T, 0, st>>>(k, reach, link, ctl, clist);
    chfsi_check_launch("ev_clusters");
    kt_end(st, slot, KT_EIGCTL, 0.0);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(ctl_h, ctl, sizeof(EvCtl), cudaMemcpyDeviceToHost, st));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    EvHost h;
    std::memcpy(&h.off, &ctl_h->off_bits, sizeof(double));
    std::memcpy(&h.dm, &ctl_h->dm_bits, sizeof(double));
    std::memcpy(&h.gnorm, &ctl_h->gnorm_bits, sizeof(double));
    h.n_hard = ctl_h->n_hard;
    h.n_out = ctl_h->n_out;
    h.n_clusters = ctl_h->n_clusters;
    h.max_cluster = ctl_h->max_cluster;
    return h;
  };
  // k x k products: FP64-accurate on the tensor cores (8 slices) or FP64
  // on the CUDA cores.  C = A B + beta C, and C = A^H B.
  auto gnn = [&](const double2* A, const double2* B, double2* C, double beta) {
    if (!f64_products) {
      oz_gemm_nn(ctx, k, k, k, A, k, B, k, C, k, 1.0, beta, 8);
      return;
    }
    EpiNN ep;
    ep.beta = beta;
    ep.P = beta != 0.0 ? C : nullptr;
    ep.ldp = k;
    ep.D = C;
    ep.ldd = k;
    zgemm_nn(st, k, k, k, A, k, B, k, ep);
  };
  auto gcn = [&](const double2* A, const double2* B, double2* C) {
    if (f64_products)
      zgemm_cn(ctx, k, k, k, A, k, B, k, C, k, 1.0, 0.0);
    else
      oz_gemm_cn(ctx, k, k, k, A, k, B, k, C, k, 1.0, 0.0, 8);
  };
  auto products = [&]() {
    gnn(G, W, GW, 0.0);  // G W
    gcn(W, GW, S);       // S = W^H G W
    gcn(W, W, M);        // M = W^H W
  };
  // FP32 eigenvectors of G as the starting W (Householder tridiagonal
  // reduction, tridiagonal eigenpairs, back transformation: eig_trd.cu).
  auto fp32_start = [&]() { trd_eigvecs_f32(ctx, k, G, W, f64_products); };

  bool identity = true;   // W = I (not materialised: S = G, M = I)
  bool tried_fp32 = false;
  bool fresh = false;     // S, M, lam, perm describe the current W
  int cluster_steps = 0;
  double2* Vstore =
      (double2*)ws_get(ctx, "eig_V", sizeof(double2) * (size_t)(k / 2 + 1) * EV_CHUNK * EV_CHUNK);
  const size_t cl_smem =
      sizeof(double2) * EV_WARPS * 2 * EV_CHUNK * EV_LD + sizeof(int) * EV_WARPS * EV_CHUNK;
  static bool cl_attr = false;
  if (!cl_attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(ev_cluster_jacobi_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cl_smem));
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(ev_cluster_cols_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cl_smem));
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(ev_cluster_rows_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cl_smem));
    cl_attr = true;
  }
  for (int it = 0; it < EV_MAX_IT; ++it) {
    if (identity) {
      CHFSI_CUDA_TRY(cudaMemcpyAsync(S, G, sizeof(double2) * kk, cudaMemcpyDeviceToDevice, st));
      shift_identity(st, k, nullptr, 1.0, M);
    } else {
      products();
    }
    const EvHost h = analyze();
    fresh = true;
    if (!std::isfinite(h.off) || !std::isfinite(h.gnorm))
      throw ChfsiError{CHFSI_ENAN, "reduced eigensolve: non-finite Rayleigh quotient"};
    if (h.off <= EV_EXIT * h.gnorm && h.dm <= EV_ORTH) break;
    if (identity && !tried_fp32 && (h.n_out > 0 || h.max_cluster > EV_SMALL)) {
      fp32_start();
      identity = false;
      tried_fp32 = true;
      fresh = false;
      continue;
    }
    if (identity) {
      shift_identity(st, k, nullptr, 1.0, W);
      identity = false;
    }
    fresh = false;
    if (h.n_clusters > 0 && cluster_steps < EV_MAX_CLUSTER_STEPS) {
      // exact rotations of the hard clusters; S and M follow the rotation
      const unsigned nb = (unsigned)((h.n_clusters + EV_WARPS - 1) / EV_WARPS);
      const int slot = kt_begin(st);
      ev_cluster_jacobi_kernel<<<nb, 32 * EV_WARPS, cl_smem, st>>>(k, S, perm, clist, ctl,
                                                                   Vstore);
      chfsi_check_launch("ev_cluster_jacobi");
      const dim3 g2(nb, (unsigned)((k + EV_ROWS - 1) / EV_ROWS));
      ev_cluster_cols_kernel<<<g2, 32 * EV_WARPS, cl_smem, st>>>(k, W, S, M, perm, clist, ctl,
                                                                 Vstore);
      chfsi_check_launch("ev_cluster_cols");
      ev_cluster_rows_kernel<<<g2, 32 * EV_WARPS, cl_smem, st>>>(k, S, M, perm, clist, ctl, Vstore);
      chfsi_check_launch("ev_cluster_rows");
      ev_lam_kernel<<<g1, 256, 0, st>>>(k, S, M, lam);
      chfsi_check_launch("ev_lam");
      kt_end(st, slot, KT_EIGCTL, 0.0);
      ++cluster_steps;
    }
    if (h.off > EV_EXIT * h.gnorm) {
      oa_e_kernel<<<grid_k2(k), 256, 0, st>>>(k, S, M, lam, ctl, E);
      chfsi_check_launch("oa_e");
      CHFSI_CUDA_TRY(cudaMemcpyAsync(W2, W, sizeof(double2) * kk, cudaMemcpyDeviceToDevice, st));
      gnn(W, E, W2, 1.0);  // W + W E
      gcn(W2, W2, M);
    } else {
      // only orthonormality is left
      CHFSI_CUDA_TRY(cudaMemcpyAsync(W2, W, sizeof(double2) * kk, cudaMemcpyDeviceToDevice, st));
    }
    // Newton-Schulz: W <- W2 (3I - W2^H W2) / 2
    ns_kernel<<<grid_k2(k), 256, 0, st>>>(k, M, E);
    chfsi_check_launch("ns");
    gnn(W2, E, W, 0.0);
  }
  if (identity) shift_identity(st, k, nullptr, 1.0, W);
  if (!fresh) {  // the iteration limit was hit after an update: final quotients
    products();
    (void)analyze();
  }
  // ascending order
  gather_values(st, k, lam, perm, w);
  gather_columns(st, k, k, W, k, perm, G, k);
  if (f64_products) {
    CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
    return;
  }
  // the error word of the tensor-core GEMM is only written by its launches
  const int e = oz_check_error(ctx);  // also synchronises
  if (e)
    throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up (code " +
                                         std::to_string(e) + ")"};
}
