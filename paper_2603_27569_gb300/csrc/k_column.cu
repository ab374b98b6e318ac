// Column-FFT configurations for the two-phase four-step path and the column
// transforms.  Variant 1 = phase 1 (four-step twiddle, transposed store,
// L <= 256, C = 16 columns per CTA); variant 0 = plain (phase 2, and
// fft_plan_columns).  Lengths beyond 256 take fewer columns per CTA so the
// tile stays small: C = 16 up to L = 512, 8 at 1024 and 2048 (64 KiB and
// 128 KiB; at 1024, 8 columns measured faster than 16: two CTAs per SM), 4 at
// 4096 (32-byte row segments, one sector each).  The 16-column 1024 kernel
// stays registered as a non-default configuration.
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
FFTGB_COLUMN(512, 16, 16, 0, 1, 16, 16, 2);
FFTGB_COLUMN(1024, 16, 16, 0, 0, 16, 16, 4);
FFTGB_COLUMN(1024, 16, 8, 0, 1, 16, 16, 4);
FFTGB_COLUMN(2048, 16, 8, 0, 1, 16, 16, 8);
FFTGB_COLUMN(4096, 16, 4, 0, 1, 16, 16, 16);
