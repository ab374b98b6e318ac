// Single-CTA Stockham configurations, N = 1024 .. 2048.
#include "instantiate.cuh"

FFTGB_STOCKHAM(1024, 16, 4, 0, 16, 16, 4);
FFTGB_STOCKHAM(1024, 8, 2, 0, 8, 8, 8, 2);
FFTGB_STOCKHAM(1024, 32, 8, 0, 32, 32);
FFTGB_STOCKHAM(2048, 16, 2, 0, 16, 16, 8);
FFTGB_STOCKHAM(2048, 8, 1, 0, 8, 8, 8, 4);
