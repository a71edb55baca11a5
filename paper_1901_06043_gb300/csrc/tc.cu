// Tensor-core (tcgen05) Gram and TTM: not built yet; every plan reports
// "not applicable" so the MIXED path is refused for the modes that need it.
#include "common.cuh"
#include "kernels.h"

namespace tk {

TcGramPlan plan_gram_tc(int64_t, int64_t, int64_t, int) { return TcGramPlan{}; }
cudaError_t launch_gram_tc(const float*, int64_t, int64_t, int64_t, const TcGramPlan&, double*,
                           unsigned*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
int ttm_tc_supported(int64_t, int64_t, int64_t, int64_t) { return 0; }
cudaError_t launch_ttm_tc(const float*, int64_t, int64_t, int64_t, const double*, int64_t, int64_t,
                          int, float*, void*, unsigned*, cudaStream_t) {
  return cudaErrorNotSupported;
}
size_t ttm_tc_scratch_bytes(int64_t, int64_t) { return 0; }

}  // namespace tk
