// Single-CTA Stockham configurations, N = 4096.
#include "instantiate.cuh"

FFTGB_STOCKHAM(4096, 16, 1, 2, 16, 16, 16);
FFTGB_STOCKHAM(4096, 8, 1, 0, 8, 8, 8, 8);
FFTGB_STOCKHAM(4096, 32, 2, 0, 32, 32, 4);
