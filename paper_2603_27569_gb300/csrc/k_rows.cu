// Single-CTA Stockham configurations with 64, 128 or 512 threads per CTA (the
// defaults use 256) for N = 256 .. 4096: more or fewer rows per CTA with the
// same radix schedules, as autotuner candidates.  Measured on GB300 (2^25
// points per call): 64 threads (2 rows) fastest at 512, 128 threads at 1024
// (2 rows) and 2048 (1 row) -- the built-in choices there; 256 threads stay
// the built-in at 256 and 4096.
#include "instantiate.cuh"

FFTGB_STOCKHAM(256, 16, 8, 0, 16, 16);
FFTGB_STOCKHAM(256, 16, 32, 0, 16, 16);
FFTGB_STOCKHAM(256, 8, 16, 0, 8, 8, 4);
FFTGB_STOCKHAM(512, 16, 4, 0, 16, 16, 2);
FFTGB_STOCKHAM(512, 16, 16, 0, 16, 16, 2);
FFTGB_STOCKHAM(512, 8, 8, 0, 8, 8, 8);
FFTGB_STOCKHAM(512, 8, 2, 0, 8, 8, 8);
FFTGB_STOCKHAM(1024, 16, 2, 2, 16, 16, 4);
FFTGB_STOCKHAM(1024, 16, 8, 0, 16, 16, 4);
FFTGB_STOCKHAM(1024, 8, 4, 0, 8, 8, 8, 2);
FFTGB_STOCKHAM(2048, 16, 1, 2, 16, 16, 8);
FFTGB_STOCKHAM(2048, 16, 4, 0, 16, 16, 8);
FFTGB_STOCKHAM(2048, 8, 2, 0, 8, 8, 8, 4);
FFTGB_STOCKHAM(4096, 16, 2, 0, 16, 16, 16);
FFTGB_STOCKHAM(256, 16, 4, 0, 16, 16);
FFTGB_STOCKHAM(512, 16, 2, 1, 16, 16, 2);
FFTGB_STOCKHAM(1024, 16, 1, 0, 16, 16, 4);
FFTGB_STOCKHAM(2048, 32, 2, 0, 32, 32, 2);
FFTGB_STOCKHAM(4096, 32, 1, 0, 32, 32, 4);
