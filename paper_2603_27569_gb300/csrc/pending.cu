// Entry points whose kernels are not built yet; each reports
// FFT_ERR_NOT_SUPPORTED so a caller never gets a silent fallback.
#include "plan.h"

namespace fftgb {
fft_status_t tc_plan(fft_plan_impl *) { return FFT_ERR_NOT_SUPPORTED; }
fft_status_t tc_exec(fft_plan_impl *, const float2 *, float2 *, int64_t, cudaStream_t) {
  return FFT_ERR_NOT_SUPPORTED;
}
void tc_destroy(fft_plan_impl *) {}
}  // namespace fftgb

extern "C" {
fft_status_t fft_spectral_filter_fused(const void *, const void *, void *, int, int64_t, int,
                                       void *) {
  return FFT_ERR_NOT_SUPPORTED;
}
}
