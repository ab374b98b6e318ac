// Cluster-split configurations beyond one CTA (cluster.cuh), in their own
// translation unit so that the build compiles them in parallel with
// k_cluster.cu.  N = 32768 on 2-CTA clusters is the built-in for that size
// (one HBM pass; 1.19x the two-launch four-step on GB300); N = 65536 on
// 4-CTA clusters (distributed-shared-memory scatter) is selectable but
// slower than the four-step there.
#include "instantiate.cuh"

FFTGB_SPLITK(32768, 2, 32, 2, 32, 32, 16);
FFTGB_SPLITK(65536, 4, 32, 0, 32, 32, 16);
