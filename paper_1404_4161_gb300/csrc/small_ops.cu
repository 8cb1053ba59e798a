// Loop control of Alg. 1 on the device: locking of converged pairs
// (Alg. 1, out-of-order locking of Sec. 4), the update of the
// filter interval (alpha, gamma; Sec. 3.2 and its footnote), the analytic
// degree rule (Alg. 1, Single Optimization of Sec. 3.2) and the
// stable ascending sort of the columns by degree (Sec. 4), so the filter
// can run on a shrinking suffix of the block.  All of it is O(k) or O(k^2)
// work on at most a few thousand values: one CTA per kernel.
#include "common.cuh"

namespace {

constexpr int NT = 1024;

// Block-wide exclusive scan of one int per thread (NT threads).
__device__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (lane < NT / 32) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;  // inclusive prefix of the warp sums
  }
  __syncthreads();
  const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
  *total = sh[NT / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(NT)
lock_select_kernel(int ka, const double* __restrict__ lam, const double* __restrict__ resid,
                   int n_wanted_left, double tol, double gamma_in, LoopCtl* ctl,
                   int* __restrict__ lock_idx, int* __restrict__ act_idx) {
  __shared__ int sh[32];
  __shared__ double shd[32];
  __shared__ int nf_sh;
  if (threadIdx.x == 0) nf_sh = 0;
  __syncthreads();
  int base_lock = 0, base_act = 0;
  double maxr = 0.0;
  for (int c0 = 0; c0 < ka; c0 += NT) {
    const int j = c0 + threadIdx.x;
    int lk = 0, act = 0;
    if (j < ka) {
      const double r = resid[j];
      if (!isfinite(r) || !isfinite(lam[j])) atomicExch(&nf_sh, 1);
      lk = (j < n_wanted_left && r <= tol) ? 1 : 0;
      act = 1 - lk;
      if (act && j < n_wanted_left) maxr = fmax(maxr, r);
    }
    int tot_l, tot_a;
    const int pl = block_exclusive_scan(lk, sh, &tot_l);
    const int pa = block_exclusive_scan(act, sh, &tot_a);
    if (j < ka) {
      if (lk) lock_idx[base_lock + pl] = j;
      else act_idx[base_act + pa] = j;
    }
    base_lock += tot_l;
    base_act += tot_a;
  }
  // max residual of the wanted, still active pairs
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxr = fmax(maxr, __shfl_xor_sync(0xffffffffu, maxr, o));
  if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = maxr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < NT / 32; ++w) m = fmax(m, shd[w]);
    ctl->n_new_locked = base_lock;
    ctl->k_active = base_act;
    ctl->nonfinite = nf_sh;
    ctl->max_resid_wanted = m;
    ctl->alpha = base_act > 0 ? lam[act_idx[base_act - 1]] : lam[ka - 1];
    ctl->gamma = fmin(gamma_in, lam[0]);
    ctl->deg_max = 0;
  }
}

__device__ int analytic_degree(double ritz, double r, double c, double e, double tol,
                               int deg_min, int deg_max, int deg_extra) {
  const double t = fabs((ritz - c) / e);
  int m = deg_max;
  if (t > 1.0) {
    const double ratio = log(r / tol) / acosh(t);
    const double cm = ceil(ratio) + (double)deg_extra;
    // clamp in double first (ratio may be huge or -inf)
    m = (int)fmin(fmax(cm, (double)deg_min), (double)deg_max);
  }
  return min(max(m, deg_min), deg_max);
}

// Degrees for the k columns idx[j] (or j) of (ritz, resid), then the cap of
// the buffer columns j >= n_wanted at the largest wanted degree and at
// buffer_cap.
__global__ void __launch_bounds__(NT)
degrees_kernel(int k, const double* __restrict__ ritz, const double* __restrict__ resid,
               const int* __restrict__ idx, double c, double e, double tol, int n_wanted,
               int deg_min, int deg_max, int deg_extra, int buffer_cap, int* __restrict__ deg) {
  __shared__ int mx;
  if (threadIdx.x == 0) mx = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += NT) {
    const int s = idx ? idx[j] : j;
    const int m = analytic_degree(ritz[s], resid[s], c, e, tol, deg_min, deg_max, deg_extra);
    deg[j] = m;
    if (j < n_wanted) atomicMax(&mx, m);
  }
  __syncthreads();
  if (n_wanted > 0 && n_wanted < k)
    for (int j = n_wanted + threadIdx.x; j < k; j += NT)
      deg[j] = max(deg_min, min(deg[j], min(mx, buffer_cap)));
}

__global__ void __launch_bounds__(NT)
degree_cap_kernel(int k, int n_wanted, int buffer_cap, int* deg) {
  __shared__ int mx;
  if (threadIdx.x == 0) mx = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < n_wanted && j < k; j += NT) atomicMax(&mx, deg[j]);
  __syncthreads();
  if (n_wanted > 0 && n_wanted < k)
    for (int j = n_wanted + threadIdx.x; j < k; j += NT)
      deg[j] = max(1, min(deg[j], min(mx, buffer_cap)));
}

// Stable ascending sort by degree: rank_j = #{i: m_i < m_j} + #{i < j:
// m_i == m_j}.  perm[rank] = idx[j] (or j), deg_sorted[rank] = m_j.
__global__ void __launch_bounds__(NT)
sort_by_degree_kernel(int k, const int* __restrict__ deg, const int* __restrict__ idx,
                      int* __restrict__ perm, int* __restrict__ deg_sorted) {
  for (int j = threadIdx.x; j < k; j += NT) {
    const int mj = deg[j];
    int rank = 0;
    for (int i = 0; i < k; ++i) {
      const int mi = deg[i];
      rank += (mi < mj) || (mi == mj && i < j);
    }
    perm[rank] = idx ? idx[j] : j;
    deg_sorted[rank] = mj;
  }
}

// Stable ascending sort of doubles: perm[rank] = j.
__global__ void __launch_bounds__(NT)
sort_by_value_kernel(int k, const double* __restrict__ v, int* __restrict__ perm) {
  for (int j = threadIdx.x; j < k; j += NT) {
    const double vj = v[j];
    int rank = 0;
    for (int i = 0; i < k; ++i) {
      const double vi = v[i];
      rank += (vi < vj) || (vi == vj && i < j);
    }
    perm[rank] = j;
  }
}

}  // namespace

void lock_select(cudaStream_t st, int ka, const double* lam, const double* resid,
                 int n_wanted_left, double tol, double gamma_in, LoopCtl* ctl, int* lock_idx,
                 int* act_idx) {
  lock_select_kernel<<<1, NT, 0, st>>>(ka, lam, resid, n_wanted_left, tol, gamma_in, ctl,
                                       lock_idx, act_idx);
  chfsi_check_launch("lock_select");
}

void degrees_analytic(cudaStream_t st, int k, const double* ritz, const double* resid,
                      const int* idx, double c, double e, double tol, int n_wanted,
                      int deg_min, int deg_max, int deg_extra, int* deg_out, int buffer_cap) {
  if (k <= 0) return;
  degrees_kernel<<<1, NT, 0, st>>>(k, ritz, resid, idx, c, e, tol, n_wanted, deg_min,
                                   deg_max, deg_extra, buffer_cap, deg_out);
  chfsi_check_launch("degrees");
}

void degree_cap_buffer(cudaStream_t st, int k, int n_wanted, int* deg, int buffer_cap) {
  if (k <= 0) return;
  degree_cap_kernel<<<1, NT, 0, st>>>(k, n_wanted, buffer_cap, deg);
  chfsi_check_launch("degree_cap");
}

void sort_by_degree(cudaStream_t st, int k, const int* deg, const int* idx_or_null, int* perm,
                    int* deg_sorted) {
  if (k <= 0) return;
  sort_by_degree_kernel<<<1, NT, 0, st>>>(k, deg, idx_or_null, perm, deg_sorted);
  chfsi_check_launch("sort_by_degree");
}

void sort_by_value(cudaStream_t st, int k, const double* val, int* perm) {
  if (k <= 0) return;
  sort_by_value_kernel<<<1, NT, 0, st>>>(k, val, perm);
  chfsi_check_launch("sort_by_value");
}
