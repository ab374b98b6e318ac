// Cluster-split configurations (a row on a 2-CTA cluster, combined through
// distributed shared memory) for N = 8192 and 16384.
#include "instantiate.cuh"

FFTGB_SPLIT2(16384, 16, 0, 16, 16, 16, 2);
FFTGB_SPLIT2(16384, 32, 0, 32, 16, 16);
FFTGB_SPLIT2(8192, 16, 0, 16, 16, 16);
FFTGB_SPLIT2(8192, 32, 0, 32, 32, 4);
