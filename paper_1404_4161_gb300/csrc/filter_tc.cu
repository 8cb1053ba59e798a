// Split-precision tensor-core Chebyshev filter (placeholder until the
// tcgen05 kernel lands): reports "not supported" so the solver refuses the
// mixed path rather than falling back.
#include "common.cuh"

struct TcFilterState {};

int tc_filter_supported(chfsi_ctx*) { return 0; }
void tc_filter_prepare(chfsi_ctx*, const double2*, int) {
  throw ChfsiError{CHFSI_ENOTSUP, "tensor-core filter not built"};
}
void tc_filter_run(chfsi_ctx*, const double2*, int, int, const double2*, const int*, double,
                   double, double, double2*) {
  throw ChfsiError{CHFSI_ENOTSUP, "tensor-core filter not built"};
}
void tc_filter_release(chfsi_ctx*) {}
