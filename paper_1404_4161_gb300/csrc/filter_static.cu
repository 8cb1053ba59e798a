// FP64 Chebyshev filter that allocates no device memory.
//
// Same arithmetic and kernels as chfsi_filter with CHFSI_PREC_FP64 (the
// shared recurrence filter_f64_recurrence), but the three rotating
// recurrence buffers live in one file-scope device array of fixed size
// instead of a context workspace, so a call needs no context and makes no
// allocation.  Every GPU that loads this library holds the array
// (CHFSI_FILTER_STATIC_MAX_NK complex elements per buffer, 12 MiB in all)
// until the process exits.
//
// The array's name is only a host-side stand-in in host code: its device
// address is looked up with cudaGetSymbolAddress, with the device current,
// on the first call made in each CUDA context of a device, and kept for that
// context.  The context is identified by its unique id (cuCtxGetId), so a
// device reset or a released and re-created primary context, after which
// the module is loaded afresh and the array may move, leads to a new lookup
// instead of a stale address.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) double2 g_filter_scratch[3 * (size_t)CHFSI_FILTER_STATIC_MAX_NK];

constexpr int kMaxDevices = 64;
struct ScratchEntry {
  unsigned long long ctx_id = 0;  // 0: no lookup yet
  double2* addr = nullptr;
};
std::mutex g_mu;
ScratchEntry g_entry[kMaxDevices];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique id of the context current on this thread (0 when none is current
// yet or the driver entry points are unavailable).
unsigned long long current_context_id() {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (PfnCtxGetCurrent)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PfnCtxGetId)p;
    (void)cudaGetLastError();
    resolved = true;
  }
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context of the
// current device.
int scratch_address(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return CHFSI_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchEntry& en = g_entry[dev];
  const unsigned long long id = current_context_id();
  if (id == 0 || en.ctx_id != id || !en.addr) {
    void* p = nullptr;  // the lookup also initialises the device's context
    if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return CHFSI_ECUDA;
    }
    en.addr = (double2*)p;
    en.ctx_id = current_context_id();  // 0 keeps the next call looking up again
  }
  *out = en.addr;
  return CHFSI_OK;
}

}  // namespace

extern "C" int chfsi_filter_static(const double* H, int n, int k, const double* Y0,
                                   const int* degrees_host, double lam1, double c, double e,
                                   double* Y, void* stream) {
  try {
    if (n < 1 || k < 0 || k > n) return CHFSI_EINVAL;
    if (k == 0) return CHFSI_OK;
    if (!H || !Y0 || !Y || !degrees_host) return CHFSI_EINVAL;
    // Y may overlap neither Y0 nor H (the filter reads them while it writes Y)
    const size_t yb = sizeof(double2) * (size_t)n * k, hb = sizeof(double2) * (size_t)n * n;
    auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
      const char* pa = (const char*)a;
      const char* pb = (const char*)b;
      return pa < pb + nb && pb < pa + na;
    };
    if (overlap(Y, yb, Y0, yb) || overlap(Y, yb, H, hb)) return CHFSI_EINVAL;
    if (!(e > 0.0) || lam1 == c) return CHFSI_EINVAL;
    for (int j = 0; j < k; ++j)
      if (degrees_host[j] < 1 || (j > 0 && degrees_host[j] < degrees_host[j - 1]))
        return CHFSI_EINVAL;
    if ((long long)n * (long long)k > (long long)CHFSI_FILTER_STATIC_MAX_NK) return CHFSI_ETOOBIG;
    double2* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != CHFSI_OK) return rc;
    const size_t blk = (size_t)n * k;
    // The three buffers are written before they are read at every step, so
    // nothing left by an earlier call needs clearing.
    double2* const F[3] = {scratch, scratch + blk, scratch + 2 * blk};
    filter_f64_recurrence((cudaStream_t)stream, reinterpret_cast<const double2*>(H), n, k,
                          reinterpret_cast<const double2*>(Y0), degrees_host, lam1, c, e,
                          reinterpret_cast<double2*>(Y), F);
  } catch (const ChfsiError& err) {
    return err.code;
  } catch (...) {
    return CHFSI_ECUDA;
  }
  return CHFSI_OK;
}
