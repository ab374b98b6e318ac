// Cluster-split configurations: a row of N points on a cluster of K CTAs,
// each holding an N/K-point part (cluster.cuh).  N = 8192 and 16384 here
// (selectable; the one-CTA kernels are faster at these sizes).
#include "instantiate.cuh"

FFTGB_SPLITK(8192, 2, 16, 0, 16, 16, 16);
FFTGB_SPLITK(16384, 2, 32, 0, 32, 16, 16);
