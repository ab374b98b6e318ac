// TMA-staged persistent configurations for N = 8192 and 16384.  Ring sizes:
// 16384 keeps 12 (P = 16) or 24 (P = 32) slabs = 96 KiB beside the 128 KiB
// exchange buffer (227 KiB total); 8192 keeps the whole next row.
#include "instantiate.cuh"

FFTGB_STAGED(16384, 16, 12, 0, 16, 16, 16, 4);
FFTGB_STAGED(16384, 32, 24, 0, 32, 32, 16);
FFTGB_STAGED(8192, 16, 16, 0, 16, 16, 16, 2);
FFTGB_STAGED(8192, 32, 32, 0, 32, 16, 16);
