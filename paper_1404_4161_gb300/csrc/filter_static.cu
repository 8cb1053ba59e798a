// FP64 Chebyshev filter that allocates no device memory.
//
// Same arithmetic and kernels as chfsi_filter with CHFSI_PREC_FP64, but
// the three rotating recurrence buffers live in one file-scope device
// array of fixed size instead of a context workspace, so a call needs no
// context and makes no allocation.  Every GPU that loads this library
// holds the array (CHFSI_FILTER_STATIC_MAX_NK complex elements per buffer,
// 12 MiB in all) until the process exits.
//
// The array's name is only a host-side stand-in in host code: its device
// address is looked up once per device with cudaGetSymbolAddress (with
// that device current) on the first call made on that device.
#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) double2 g_filter_scratch[3 * (size_t)CHFSI_FILTER_STATIC_MAX_NK];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.
int scratch_address(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CHFSI_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return CHFSI_ECUDA;
    }
    g_addr[dev] = (double2*)p;
  }
  *out = g_addr[dev];
  return CHFSI_OK;
}

}  // namespace

extern "C" int chfsi_filter_static(const double* H, int n, int k, const double* Y0,
                                   const int* degrees_host, double lam1, double c, double e,
                                   double* Y, void* stream) {
  if (n < 1 || k < 0 || k > n) return CHFSI_EINVAL;
  if (k == 0) return CHFSI_OK;
  if (!H || !Y0 || !Y || !degrees_host || Y0 == Y) return CHFSI_EINVAL;
  if (!(e > 0.0) || lam1 == c) return CHFSI_EINVAL;
  for (int j = 0; j < k; ++j)
    if (degrees_host[j] < 1 || (j > 0 && degrees_host[j] < degrees_host[j - 1]))
      return CHFSI_EINVAL;
  if ((long long)n * (long long)k > (long long)CHFSI_FILTER_STATIC_MAX_NK) return CHFSI_ETOOBIG;
  double2* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != CHFSI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const double2* H2 = reinterpret_cast<const double2*>(H);
  const double2* Y02 = reinterpret_cast<const double2*>(Y0);
  double2* Yout = reinterpret_cast<double2*>(Y);
  const size_t blk = (size_t)n * k;
  // The three buffers are written before they are read at every step, so
  // nothing left by an earlier call needs clearing.
  double2* F[3] = {scratch, scratch + blk, scratch + 2 * blk};
  auto buf = [&](int i) -> const double2* { return i == 0 ? Y02 : F[i % 3]; };
  const int* deg = degrees_host;
  try {
    const int mk = deg[k - 1];
    const double sigma1 = e / (lam1 - c);
    int s = 0;
    while (s < k && deg[s] <= 1) ++s;
    {
      EpiNN ep;
      ep.alpha = sigma1 / e;
      ep.shift = c;
      ep.S = Y02;
      ep.lds = n;
      ep.D = F[1];
      ep.ldd = n;
      ep.F = Yout;
      ep.ldf = n;
      ep.fin_end = s;
      zgemm_nn(st, n, k, n, H2, n, Y02, n, ep);
    }
    double sigma = sigma1;
    for (int i = 1; i < mk; ++i) {
      const double sn = 1.0 / (2.0 / sigma1 - sigma);
      int s_new = s;
      while (s_new < k && deg[s_new] <= i + 1) ++s_new;
      const size_t off = (size_t)s * n;
      EpiNN ep;
      ep.alpha = 2.0 * sn / e;
      ep.shift = c;
      ep.S = buf(i) + off;
      ep.lds = n;
      ep.beta = -sn * sigma;
      ep.P = buf(i - 1) + off;
      ep.ldp = n;
      ep.D = F[(i + 1) % 3] + off;
      ep.ldd = n;
      ep.F = Yout + off;
      ep.ldf = n;
      ep.fin_end = s_new - s;
      zgemm_nn(st, n, k - s, n, H2, n, buf(i) + off, n, ep);
      sigma = sn;
      s = s_new;
    }
  } catch (const ChfsiError& err) {
    return err.code;
  }
  return CHFSI_OK;
}
