// Rows of 32768 points on one SM: a radix-2 split into two 16384-point
// transforms, one half parked in tensor memory (tmem2.cuh).  The built-in
// configuration for N = 32768 (twiddle mode 1, like the 16384-point kernel
// whose passes it runs).
#include "instantiate.cuh"

FFTGB_TMEM2(32768, 32, 2, 32, 32, 16);
