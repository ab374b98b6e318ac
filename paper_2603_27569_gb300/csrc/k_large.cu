// Single-CTA Stockham configurations, N = 8192 and 16384 (the in-CTA
// four-step: the last radix-2/4 pass is the N1-point step with the
// W_N^{n1 k2} twiddle, the earlier passes the N2-point sub-transforms).
#include "instantiate.cuh"

FFTGB_STOCKHAM(8192, 16, 1, 0, 16, 16, 16, 2);
FFTGB_STOCKHAM(8192, 32, 1, 2, 32, 16, 16);
FFTGB_STOCKHAM(16384, 16, 1, 0, 16, 16, 16, 4);
FFTGB_STOCKHAM(16384, 32, 1, 2, 32, 32, 16);
