// Column-FFT configurations for the two-phase four-step path (C = 16
// columns per CTA).  Variant 1 = phase 1 (four-step twiddle, transposed
// store); variant 0 = phase 2 (plain, same layout).
#include "instantiate.cuh"

FFTGB_COLUMN(16, 16, 16, 0, 1, 16);
FFTGB_COLUMN(16, 16, 16, 1, 1, 16);
FFTGB_COLUMN(32, 16, 16, 0, 1, 16, 2);
FFTGB_COLUMN(32, 16, 16, 1, 1, 16, 2);
FFTGB_COLUMN(64, 16, 16, 0, 1, 16, 4);
FFTGB_COLUMN(64, 16, 16, 1, 1, 16, 4);
FFTGB_COLUMN(128, 16, 16, 0, 1, 16, 8);
FFTGB_COLUMN(128, 16, 16, 1, 1, 16, 8);
FFTGB_COLUMN(256, 16, 16, 0, 1, 16, 16);
FFTGB_COLUMN(256, 16, 16, 1, 1, 16, 16);
