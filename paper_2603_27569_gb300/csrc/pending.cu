// Entry points whose kernels are not built yet; each reports
// FFT_ERR_NOT_SUPPORTED so a caller never gets a silent fallback.
#include "plan.h"

namespace fftgb {
}  // namespace fftgb

extern "C" {
fft_status_t fft_spectral_filter_fused(const void *, const void *, void *, int, int64_t, int,
                                       void *) {
  return FFT_ERR_NOT_SUPPORTED;
}
}
