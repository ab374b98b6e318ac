// FP16-storage configurations (the FP32 defaults' schedules), N = 256..16384.
#include "instantiate.cuh"

FFTGB_HALF(256, 16, 16, 1, 16, 16);
FFTGB_HALF(512, 16, 2, 1, 16, 16, 2);
FFTGB_HALF(1024, 16, 2, 1, 16, 16, 4);
FFTGB_HALF(2048, 16, 1, 1, 16, 16, 8);
FFTGB_HALF(4096, 16, 1, 0, 16, 16, 16);
FFTGB_HALF(8192, 32, 1, 1, 32, 16, 16);
FFTGB_HALF(16384, 32, 1, 1, 32, 32, 16);
