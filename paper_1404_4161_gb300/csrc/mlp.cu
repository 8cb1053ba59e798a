// Learned degree predictor: a 5 -> 64 -> 64 -> 1 tanh MLP that maps the
// state of one active column (Ritz value and residual in the filter frame,
// the filter bounds, the sequence index) to a Chebyshev degree.  It stands
// in for the analytic Single Optimization rule of Sec. 3.2 (which stays as
// the fallback); the paper itself has no such network.
//
// Weights: FP32 masters plus FP16 copies; the products use the FP16 values
// of weights and activations with FP32 accumulation.  Training runs the
// forward pass, a per-sample backward pass, a deterministic per-parameter
// reduction over the batch and an Adam step (Kingma and Ba, ICLR 2015),
// all in the kernels below.
#include <cuda_fp16.h>

#include <cstring>

#include "common.cuh"

namespace {

constexpr int F = 5, HD = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HD * F, OFF_W2 = OFF_B1 + HD,
              OFF_B2 = OFF_W2 + HD * HD, OFF_W3 = OFF_B2 + HD, OFF_B3 = OFF_W3 + HD,
              NP = OFF_B3 + 1;
static_assert(NP == CHFSI_MLP_NPARAM, "parameter layout");

constexpr int DEG_LO = 4, DEG_HI = 60;
constexpr float DEG_SCALE = 60.f;

__device__ __forceinline__ float h16(float v) { return __half2float(__float2half_rn(v)); }

// One sample per thread; the FP16 weights sit in shared memory.
template <bool STORE>
__global__ void __launch_bounds__(128)
mlp_fwd_kernel(int B, const float* __restrict__ x, const __half* __restrict__ w16,
               float* __restrict__ y, float* __restrict__ H1, float* __restrict__ H2) {
  __shared__ float w[NP];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __half2float(w16[i]);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float xi[F];
#pragma unroll
  for (int i = 0; i < F; ++i) xi[i] = h16(x[(size_t)b * F + i]);
  float h1[HD];
#pragma unroll
  for (int o = 0; o < HD; ++o) {
    float z = w[OFF_B1 + o];
#pragma unroll
    for (int i = 0; i < F; ++i) z = fmaf(w[OFF_W1 + o * F + i], xi[i], z);
    h1[o] = h16(tanhf(z));
    if (STORE) H1[(size_t)b * HD + o] = h1[o];
  }
  float out = w[OFF_B3];
  for (int o = 0; o < HD; ++o) {
    float z = w[OFF_B2 + o];
#pragma unroll
    for (int i = 0; i < HD; ++i) z = fmaf(w[OFF_W2 + o * HD + i], h1[i], z);
    const float h2 = h16(tanhf(z));
    if (STORE) H2[(size_t)b * HD + o] = h2;
    out = fmaf(w[OFF_W3 + o], h2, out);
  }
  y[b] = out;
}

// Per-sample deltas: d = (y - t)/B, dZ2 = d W3 (1 - h2^2), dZ1 = (dZ2 W2)(1 - h1^2).
__global__ void __launch_bounds__(128)
mlp_delta_kernel(int B, const float* __restrict__ y, const float* __restrict__ t,
                 const __half* __restrict__ w16, const float* __restrict__ H1,
                 const float* __restrict__ H2, float* __restrict__ D, float* __restrict__ DZ1,
                 float* __restrict__ DZ2, float* __restrict__ sq) {
  __shared__ float w[NP];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __half2float(w16[i]);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float r = y[b] - t[b];
  const float d = r / (float)B;
  D[b] = d;
  sq[b] = r * r;
  float dz2[HD];
#pragma unroll
  for (int o = 0; o < HD; ++o) {
    const float h2 = H2[(size_t)b * HD + o];
    dz2[o] = d * w[OFF_W3 + o] * (1.f - h2 * h2);
    DZ2[(size_t)b * HD + o] = dz2[o];
  }
  for (int i = 0; i < HD; ++i) {
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < HD; ++o) s = fmaf(dz2[o], w[OFF_W2 + o * HD + i], s);
    const float h1 = H1[(size_t)b * HD + i];
    DZ1[(size_t)b * HD + i] = s * (1.f - h1 * h1);
  }
}

// Gradient of parameter p as a fixed-order sum over the batch.
__global__ void mlp_grad_kernel(int B, const float* __restrict__ x, const float* __restrict__ H1,
                                const float* __restrict__ H2, const float* __restrict__ D,
                                const float* __restrict__ DZ1, const float* __restrict__ DZ2,
                                float* __restrict__ g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  float s = 0.f;
  if (p < OFF_B1) {
    const int o = (p - OFF_W1) / F, i = (p - OFF_W1) % F;
    for (int b = 0; b < B; ++b) s = fmaf(DZ1[(size_t)b * HD + o], h16(x[(size_t)b * F + i]), s);
  } else if (p < OFF_W2) {
    const int o = p - OFF_B1;
    for (int b = 0; b < B; ++b) s += DZ1[(size_t)b * HD + o];
  } else if (p < OFF_B2) {
    const int o = (p - OFF_W2) / HD, i = (p - OFF_W2) % HD;
    for (int b = 0; b < B; ++b) s = fmaf(DZ2[(size_t)b * HD + o], H1[(size_t)b * HD + i], s);
  } else if (p < OFF_W3) {
    const int o = p - OFF_B2;
    for (int b = 0; b < B; ++b) s += DZ2[(size_t)b * HD + o];
  } else if (p < OFF_B3) {
    const int o = p - OFF_W3;
    for (int b = 0; b < B; ++b) s = fmaf(D[b], H2[(size_t)b * HD + o], s);
  } else {
    for (int b = 0; b < B; ++b) s += D[b];
  }
  g[p] = s;
}

__global__ void mlp_loss_kernel(int B, const float* sq, float* loss) {
  __shared__ float sh[32];
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += sq[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *loss = 0.5f * t / (float)B;
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                float* __restrict__ m, float* __restrict__ v,
                                __half* __restrict__ w16, float lr, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  const float pi = p[i] - lr * mh / (sqrtf(vh) + 1e-8f);
  p[i] = pi;
  w16[i] = __float2half_rn(pi);
}

__global__ void to_half_kernel(const float* p, __half* w16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NP) w16[i] = __float2half_rn(p[i]);
}

// Features of the k active columns idx[j] (the oracle's mlp.features).
__global__ void mlp_features_kernel(int k, const double* ritz, const double* resid,
                                    const int* idx, double c, double e, double gamma, int step,
                                    float* x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int s = idx ? idx[j] : j;
  const double t = (ritz[s] - c) / e;
  const double r = fmax(resid[s], 1e-300);
  float* row = x + (size_t)j * F;
  row[0] = (float)fmin(fmax(t, -8.0), 8.0);
  row[1] = (float)(log10(r) / 10.0);
  row[2] = (float)acosh(fmax(fabs(t), 1.0));
  row[3] = (float)fmin(fmax((gamma - c) / e, -8.0), 8.0);
  row[4] = (float)(min(step, 9) / 10.0);
}

// Degree from the predicted decay ratio (closed form); the analytic rule
// of Sec. 3.2 for a non-finite prediction.
__global__ void mlp_to_degree_kernel(int k, const float* y, const double* ritz,
                                     const double* resid, const int* idx, double c, double e,
                                     double tol, int extra, int a_min, int a_max, int a_extra,
                                     int* deg) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int s = idx ? idx[j] : j;
  const double t = fabs((ritz[s] - c) / e);
  const double r = resid[s];
  const float v = y[j];
  int m;
  if (isfinite(v)) {
    if (t > 1.0) {
      const double yy = fmin(fmax((double)v, 0.02), 1.5);
      const double kan = acosh(fmax(t, 1.0 + 1e-12));
      const double q = ceil(log(fmax(r, tol) / tol) / (kan * yy)) + (double)extra;
      m = (int)fmin(fmax(q, (double)DEG_LO), (double)DEG_HI);
    } else {
      m = DEG_HI;
    }
  } else {  // analytic fallback
    m = a_max;
    if (t > 1.0) {
      const double q = ceil(log(r / tol) / acosh(t)) + (double)a_extra;
      m = (int)fmin(fmax(q, (double)a_min), (double)a_max);
    }
  }
  deg[j] = m;
}

// Trace rows (10 floats): x0..x4, m, r_before, r_after, acosh(max|t|, 1), wanted.
constexpr int TROW = 10;

__global__ void trace_record_kernel(int k, const double* ritz, const double* resid,
                                    const int* idx, const int* deg, double c, double e,
                                    double gamma, int step, int n_wanted, float* rows) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int s = idx ? idx[j] : j;
  const double t = (ritz[s] - c) / e;
  const double r = fmax(resid[s], 1e-300);
  float* row = rows + (size_t)j * TROW;
  row[0] = (float)fmin(fmax(t, -8.0), 8.0);
  row[1] = (float)(log10(r) / 10.0);
  row[2] = (float)acosh(fmax(fabs(t), 1.0));
  row[3] = (float)fmin(fmax((gamma - c) / e, -8.0), 8.0);
  row[4] = (float)(min(step, 9) / 10.0);
  row[5] = (float)deg[j];
  row[6] = (float)r;
  row[7] = __int_as_float(0x7fc00000);  // NaN until the next loop's residual
  row[8] = (float)acosh(fmax(fabs(t), 1.0 + 1e-12));
  row[9] = j < n_wanted ? 1.f : 0.f;
}

__global__ void trace_finish_kernel(int k, const double* resid, float* rows) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) rows[(size_t)j * TROW + 7] = (float)fmax(resid[j], 1e-300);
}

// Compacts complete rows of wanted columns into (x, y), in row order.
__global__ void __launch_bounds__(1024)
trace_dataset_kernel(int nrows, const float* rows, float* x, float* y, int max_rows,
                     int* out_count) {
  __shared__ int warp_sums[32];
  __shared__ int base_sh;
  if (threadIdx.x == 0) base_sh = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nrows; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    int ok = 0;
    if (i < nrows) {
      const float* row = rows + (size_t)i * TROW;
      ok = row[9] > 0.5f && isfinite(row[7]) && row[6] > 0.f && row[5] >= 1.f && row[8] > 0.f;
    }
    // block exclusive scan of ok
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = ok;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
      int s2 = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, s2, o);
        if (lane >= o) s2 += u;
      }
      warp_sums[lane] = s2;
    }
    __syncthreads();
    const int pos = base_sh + (w > 0 ? warp_sums[w - 1] : 0) + v - ok;
    if (ok && pos < max_rows) {
      const float* row = rows + (size_t)i * TROW;
      for (int f = 0; f < F; ++f) x[(size_t)pos * F + f] = row[f];
      const double kre = log((double)row[6] / (double)row[7]) / (double)row[5];
      y[pos] = (float)fmin(fmax(kre / (double)row[8], 0.02), 1.5);
    }
    __syncthreads();
    if (threadIdx.x == 0) base_sh += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_count = min(base_sh, max_rows);
}

}  // namespace

struct MlpState {
  float* trace = nullptr;  // trace rows (TROW floats each)
  int trace_cap = 0, trace_n = 0, pend_base = 0, pend_count = 0;
  float* p = nullptr;   // FP32 master parameters
  float* m = nullptr;   // Adam first moment
  float* v = nullptr;   // Adam second moment
  float* g = nullptr;   // last gradient
  __half* w16 = nullptr;
  int t = 0;
};

void mlp_create(chfsi_ctx* ctx) {
  MlpState* s = new MlpState();
  ctx->mlp = s;
  CHFSI_CUDA_TRY(cudaMalloc(&s->p, sizeof(float) * NP * 4));
  s->m = s->p + NP;
  s->v = s->m + NP;
  s->g = s->v + NP;
  CHFSI_CUDA_TRY(cudaMalloc(&s->w16, sizeof(__half) * NP));
  CHFSI_CUDA_TRY(cudaMemsetAsync(s->p, 0, sizeof(float) * NP * 4, ctx->stream));
  CHFSI_CUDA_TRY(cudaMemsetAsync(s->w16, 0, sizeof(__half) * NP, ctx->stream));
}

void mlp_destroy(chfsi_ctx* ctx) {
  if (!ctx->mlp) return;
  cudaFree(ctx->mlp->p);
  cudaFree(ctx->mlp->w16);
  cudaFree(ctx->mlp->trace);
  delete ctx->mlp;
  ctx->mlp = nullptr;
}

void mlp_set_params(chfsi_ctx* ctx, const float* host) {
  MlpState* s = ctx->mlp;
  CHFSI_CUDA_TRY(cudaMemcpyAsync(s->p, host, sizeof(float) * NP, cudaMemcpyHostToDevice,
                                 ctx->stream));
  CHFSI_CUDA_TRY(cudaMemsetAsync(s->m, 0, sizeof(float) * NP * 3, ctx->stream));
  s->t = 0;
  to_half_kernel<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(s->p, s->w16);
  chfsi_check_launch("mlp to_half");
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
}

void mlp_get_params(chfsi_ctx* ctx, float* host) {
  CHFSI_CUDA_TRY(cudaMemcpyAsync(host, ctx->mlp->p, sizeof(float) * NP, cudaMemcpyDeviceToHost,
                                 ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
}

void mlp_forward(chfsi_ctx* ctx, int B, const float* x, float* y) {
  mlp_fwd_kernel<false><<<(B + 127) / 128, 128, 0, ctx->stream>>>(B, x, ctx->mlp->w16, y,
                                                                  nullptr, nullptr);
  chfsi_check_launch("mlp_fwd");
}

void mlp_train_step(chfsi_ctx* ctx, int B, const float* x, const float* target, float lr,
                    float* grads, float* loss_dev) {
  MlpState* s = ctx->mlp;
  cudaStream_t st = ctx->stream;
  float* scr = (float*)ws_get(ctx, "mlp_scratch", sizeof(float) * (size_t)B * (4 * HD + 3));
  float* H1 = scr;
  float* H2 = H1 + (size_t)B * HD;
  float* DZ1 = H2 + (size_t)B * HD;
  float* DZ2 = DZ1 + (size_t)B * HD;
  float* y = DZ2 + (size_t)B * HD;
  float* D = y + B;
  float* sq = D + B;
  const int nb = (B + 127) / 128;
  mlp_fwd_kernel<true><<<nb, 128, 0, st>>>(B, x, s->w16, y, H1, H2);
  chfsi_check_launch("mlp_fwd_train");
  mlp_delta_kernel<<<nb, 128, 0, st>>>(B, y, target, s->w16, H1, H2, D, DZ1, DZ2, sq);
  chfsi_check_launch("mlp_delta");
  mlp_grad_kernel<<<(NP + 127) / 128, 128, 0, st>>>(B, x, H1, H2, D, DZ1, DZ2, s->g);
  chfsi_check_launch("mlp_grad");
  mlp_loss_kernel<<<1, 1024, 0, st>>>(B, sq, loss_dev);
  chfsi_check_launch("mlp_loss");
  if (grads)
    CHFSI_CUDA_TRY(cudaMemcpyAsync(grads, s->g, sizeof(float) * NP, cudaMemcpyDeviceToDevice, st));
  s->t += 1;
  const float bc1 = 1.f - powf(0.9f, (float)s->t), bc2 = 1.f - powf(0.999f, (float)s->t);
  mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, st>>>(s->p, s->g, s->m, s->v, s->w16, lr, bc1,
                                                      bc2);
  chfsi_check_launch("mlp_adam");
}

void mlp_degrees(chfsi_ctx* ctx, int k, const double* ritz, const double* resid,
                 const int* idx, double c, double e, double gamma, int step, double tol,
                 int* deg_out) {
  if (k <= 0) return;
  float* x = (float*)ws_get(ctx, "mlp_x", sizeof(float) * (size_t)k * (F + 1));
  float* y = x + (size_t)k * F;
  mlp_features_kernel<<<(k + 127) / 128, 128, 0, ctx->stream>>>(k, ritz, resid, idx, c, e,
                                                                  gamma, step, x);
  chfsi_check_launch("mlp_features");
  mlp_forward(ctx, k, x, y);
  const chfsi_opts& o = ctx->opts;
  mlp_to_degree_kernel<<<(k + 127) / 128, 128, 0, ctx->stream>>>(
      k, y, ritz, resid, idx, c, e, tol, o.mlp_extra, o.deg_min, o.deg_max, o.deg_extra, deg_out);
  chfsi_check_launch("mlp_to_degree");
}

void trace_enable(chfsi_ctx* ctx, int cap) {
  MlpState* s = ctx->mlp;
  cudaFree(s->trace);
  s->trace = nullptr;
  s->trace_cap = 0;
  s->trace_n = s->pend_base = s->pend_count = 0;
  if (cap > 0) {
    CHFSI_CUDA_TRY(cudaMalloc(&s->trace, sizeof(float) * TROW * (size_t)cap));
    s->trace_cap = cap;
  }
}

bool trace_on(chfsi_ctx* ctx) { return ctx->mlp && ctx->mlp->trace_cap > 0; }

void trace_record(chfsi_ctx* ctx, int k, const double* ritz, const double* resid,
                  const int* idx, const int* deg, double c, double e, double gamma, int step,
                  int n_wanted) {
  MlpState* s = ctx->mlp;
  s->pend_count = 0;
  if (!trace_on(ctx) || k <= 0 || s->trace_n + k > s->trace_cap) return;
  trace_record_kernel<<<(k + 127) / 128, 128, 0, ctx->stream>>>(
      k, ritz, resid, idx, deg, c, e, gamma, step, n_wanted,
      s->trace + (size_t)s->trace_n * TROW);
  chfsi_check_launch("trace_record");
  s->pend_base = s->trace_n;
  s->pend_count = k;
  s->trace_n += k;
}

void trace_finish(chfsi_ctx* ctx, int k, const double* resid) {
  MlpState* s = ctx->mlp;
  if (!trace_on(ctx) || s->pend_count <= 0) return;
  const int cnt = k < s->pend_count ? k : s->pend_count;
  trace_finish_kernel<<<(cnt + 127) / 128, 128, 0, ctx->stream>>>(
      cnt, resid, s->trace + (size_t)s->pend_base * TROW);
  chfsi_check_launch("trace_finish");
  s->pend_count = 0;
}

void trace_abandon(chfsi_ctx* ctx) {
  if (ctx->mlp) ctx->mlp->pend_count = 0;
}

int trace_dataset(chfsi_ctx* ctx, float* x, float* y, int max_rows) {
  MlpState* s = ctx->mlp;
  if (!trace_on(ctx) || s->trace_n == 0) return 0;
  int* cnt = (int*)ws_get(ctx, "trace_cnt", sizeof(int));
  trace_dataset_kernel<<<1, 1024, 0, ctx->stream>>>(s->trace_n, s->trace, x, y, max_rows, cnt);
  chfsi_check_launch("trace_dataset");
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return *h;
}
