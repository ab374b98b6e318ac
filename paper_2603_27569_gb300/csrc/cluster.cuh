// Cluster-split Stockham kernel: one row of N points on a pair of CTAs (a
// thread-block cluster of 2), exchanging through distributed shared memory.
//
// The four-step split with N1 = 2 (paper Sec. IV-B, Eq. 2; Sec. V-D):
//   n = r + 2 n2, k = k2 + (N/2) k1, r, k1 in {0, 1}
//   CTA r:   A_r[k2] = FFT_{N/2} over n2 of x[r + 2 n2]      (registers + smem)
//            B_r[k2] = A_r[k2] W_N^{r k2}                     (the four-step twiddle)
//   combine: X[k2] = B_0[k2] + B_1[k2],  X[k2 + N/2] = B_0[k2] - B_1[k2]
// CTA r combines k2 in [r N/4, (r+1) N/4), reading its own B from shared
// memory and the partner's through the cluster's shared-memory window, and
// stores both halves of X for those k2 (contiguous, coalesced).
//
// Why: a row of 16384 points needs half an SM's register file, so only one
// row fits an SM and its exchange and compute phases cannot overlap.  Split
// across a cluster, each SM hosts two or three half-rows of different rows,
// whose phases interleave as they do for N <= 8192.
#pragma once
#include <cooperative_groups.h>

#include "stockham.cuh"

namespace fftgb {

struct Split2Args {
  const float2 *in;
  float2 *out;
  const float2 *tw;     // pass tables of the N/2-point schedule
  const float2 *tw_n;   // W_N^k, k < N/2
  long long batch;
  float scale;
};

template <int N, int P, int D, class SC, int TWM>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__((N / 2) / P)
split2_kernel(Split2Args a) {
  namespace cg = cooperative_groups;
  constexpr int H = N / 2;
  constexpr int T = H / P;
  static_assert(SC::product() == H, "schedule must multiply to N / 2");
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const long long row = blockIdx.x / 2;
  const bool active = row < a.batch;  // uniform over the cluster
  extern __shared__ __align__(16) float2 smem[];
  const int lt = threadIdx.x;
  float2 v[P];
  const float2 *src = a.in + row * N + r;  // x[r + 2 n2]
  if (active) {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = __ldcs(src + 2 * (lt + m * T));
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
  }
  run_passes<H, P, D, SC, 0, SwizzledRow, TWM>(v, lt, smem, a.tw, SwizzledRow{});
  // v[m] = A_r[lt + m T]
  if (r == 1) {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cmul_dir<D>(v[m], __ldg(a.tw_n + lt + m * T));
  }
  __syncthreads();  // the last exchange has been read out of smem
#pragma unroll
  for (int m = 0; m < P; ++m) smem[lt + m * T] = v[m];  // B_r in natural order
  cl.sync();  // both halves of B are in place
  const float2 *peer = cl.map_shared_rank(smem, 1 - r);
  if (active) {
    float2 *dst = a.out + row * N;
#pragma unroll
    for (int u = 0; u < P / 2; ++u) {
      const int k2 = r * (H / 2) + lt + u * T;
      const float2 own = smem[k2], oth = peer[k2];
      const float2 b0 = r == 0 ? own : oth, b1 = r == 0 ? oth : own;
      __stcs(dst + k2, cscale(cadd(b0, b1), a.scale));
      __stcs(dst + k2 + H, cscale(csub(b0, b1), a.scale));
    }
  }
  cl.sync();  // the partner has finished reading this CTA's shared memory
}

}  // namespace fftgb
