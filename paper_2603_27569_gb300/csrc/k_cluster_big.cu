// Cluster-split configurations beyond one CTA (cluster.cuh), in their own
// translation unit so that the build compiles them in parallel with
// k_cluster.cu.  Both are selectable (fft_plan_config), not built-ins: on
// GB300 the two-launch four-step with its twiddle grids is ~3 % faster at
// 32768 and 1.5x faster at 65536 (4-CTA clusters, distributed-shared-memory
// scatter).
#include "instantiate.cuh"

FFTGB_SPLITK(32768, 2, 32, 0, 32, 32, 16);
FFTGB_SPLITK(65536, 4, 32, 0, 32, 32, 16);
