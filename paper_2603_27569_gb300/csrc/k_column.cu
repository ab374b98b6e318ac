// Column-FFT configurations for the two-phase four-step path.  Variant 1 =
// phase 1 (four-step twiddle, transposed store, L <= 256, C = 16 columns per
// CTA); variant 0 = phase 2 (plain, same layout).  Phase-2 lengths beyond 256
// (N > 65536 = 256 x 256) keep the tile at <= 128 KiB by taking fewer columns:
// C = 16 up to L = 1024, 8 at 2048, 4 at 4096 (32-byte row segments, one
// sector each).
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
FFTGB_COLUMN(1024, 16, 16, 0, 1, 16, 16, 4);
FFTGB_COLUMN(2048, 16, 8, 0, 1, 16, 16, 8);
FFTGB_COLUMN(4096, 16, 4, 0, 1, 16, 16, 16);
