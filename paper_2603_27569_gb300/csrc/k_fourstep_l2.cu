// Single-launch four-step configurations with the intermediate in an L2 ring
// (N = L * L; the column schedules of k_column.cu, C = 16 columns per CTA).
#include "instantiate.cuh"

FFTGB_FOURSTEP_L2(64, 16, 16, 16, 4);
FFTGB_FOURSTEP_L2(128, 16, 16, 16, 8);
FFTGB_FOURSTEP_L2(256, 16, 16, 16, 16);
