// Cluster-split Stockham kernel: one row of N points on a thread-block
// cluster of K CTAs (K = 2, 4, 8), exchanging through distributed shared
// memory.  One HBM pass per row for N up to K x 16384.
//
// The four-step split with N1 = K (paper Sec. IV-B, Eq. 3; Sec. V-D):
//   n = r + K n2, k = k2 + H k1, H = N / K, r, k1 < K, n2, k2 < H
//   CTA r:   A_r[k2] = FFT_H over n2 of x[r + K n2]        (registers + smem)
//            B_r[k2] = A_r[k2] W_N^{r k2}                   (the four-step twiddle)
//   combine: X[k2 + H k1] = sum_r B_r[k2] W_K^{r k1}        (K-point DFTs)
//
// Per row:
//   1. CTA r reads the contiguous slice x[r H .. (r+1) H) with 16-byte loads
//      and stores each element e into the shared memory of CTA e mod K at
//      position e div K (distributed shared memory), so every CTA ends up
//      with its stride-K subsequence in natural order without strided HBM
//      or L2 reads.
//   2. Each CTA runs the H-point Stockham FFT (stockham.cuh) and multiplies
//      by W_N^{r k2} (table laid out [r - 1][k2]).
//   3. B_r goes back to shared memory; CTA r combines k2 in
//      [r H / K, (r + 1) H / K), reading B_q[k2] from every CTA q, and
//      stores the K outputs k2 + H k1 (coalesced across the warp).
// Clusters are persistent: cluster c handles rows c, c + C, ... (C = the
// clusters launched), and each CTA prefetches its slice of the cluster's
// next row into L2 through the bulk-copy engine.
//
// A cluster barrier before the first row makes sure every CTA has started
// before any remote store.  Three cluster barriers per row keep the
// shared-memory phases apart: after the scatter (every element in place),
// after B is written (the combine may read it), and after the combine (no
// CTA scatters the next row into a buffer another CTA still reads).  Every
// CTA of a cluster runs the same row loop, so all of them reach every
// barrier.
#pragma once
#include <cooperative_groups.h>

#include "stockham.cuh"

namespace fftgb {

struct SplitArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;     // pass tables of the H-point schedule
  const float2 *tw_n;   // W_N^{r k2} at (r - 1) H + k2, 1 <= r < K, k2 < H
  long long batch;
  float scale;          // applied at the final store (1 or 1/N)
};

// Parts of <= 8192 points (<= 256 threads, <= 64 KiB) are bounded to fit two
// CTAs per SM, so that one CTA's exchanges overlap another's compute.
template <int N, int K, int P, int D, class SC, int TWM>
__global__ void __cluster_dims__(K, 1, 1)
    __launch_bounds__((N / K) / P, (N / K) / P <= 256 ? 2 : 1) splitk_kernel(SplitArgs a) {
  namespace cg = cooperative_groups;
  constexpr int H = N / K;
  constexpr int T = H / P;
  static_assert(SC::product() == H, "schedule must multiply to N / K");
  static_assert(K == 2 || K == 4 || K == 8, "cluster of 2, 4 or 8 CTAs");
  static_assert(P % K == 0 && (2 * T) % K == 0, "combine and scatter tile the row");
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const long long c0 = blockIdx.x / K, ncl = gridDim.x / K;
  extern __shared__ __align__(128) float2 smem[];
  const int lt = threadIdx.x;
  // Scatter targets of this thread: pair j = lt + m T holds elements
  // e = r H + 2 j and e + 1; with K | H and K | 2 T they go to CTAs
  // q0 = (2 lt) mod K and q0 + 1, both at position r H / K + (2 lt) div K
  // + m (2 T / K).
  const int q0 = (2 * lt) % K;
  const int base = r * (H / K) + (2 * lt) / K;
  float2 *d0 = cl.map_shared_rank(smem, q0) + base;
  float2 *d1 = cl.map_shared_rank(smem, q0 + 1) + base;
  cl.sync();  // every CTA of the cluster runs before any remote store
  for (long long row = c0; row < a.batch; row += ncl) {
    const long long next = row + ncl;
    const bool first = row == c0;
    if (!first && next < a.batch && lt < 32)
      prefetch_l2_warp(a.in + next * N + (long long)r * H, (long long)H * sizeof(float2), lt);
    float2 v[P];
    if constexpr (K == 2) {
      // x[r + 2 n2] straight from global memory (8-byte loads at a 16-byte
      // stride; the partner CTA reads the other half of each sector)
      const float2 *src = a.in + row * N + r;
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = __ldcs(src + 2 * (lt + m * T));
      if (first && next < a.batch && lt < 32)
        prefetch_l2_warp(a.in + next * N + (long long)r * H, (long long)H * sizeof(float2), lt);
    } else {
      const float4 *src = reinterpret_cast<const float4 *>(a.in + row * N + (long long)r * H);
#pragma unroll
      for (int m = 0; m < P / 2; ++m) {
        const float4 w = __ldcs(src + lt + m * T);
        d0[m * (2 * T / K)] = make_float2(w.x, w.y);
        d1[m * (2 * T / K)] = make_float2(w.z, w.w);
      }
      cl.sync();  // every CTA's subsequence is in place
      if (first && next < a.batch && lt < 32)
        prefetch_l2_warp(a.in + next * N + (long long)r * H, (long long)H * sizeof(float2), lt);
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = smem[lt + m * T];
      __syncthreads();  // pass 0 rewrites the buffer
    }
    run_passes<H, P, D, SC, 0, SwizzledRow, TWM>(v, lt, smem, a.tw, SwizzledRow{});
    // v[m] = A_r[lt + m T]
    if (r > 0) {
      const float2 *w = a.tw_n + (long long)(r - 1) * H;
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = cmul_dir<D>(v[m], __ldg(w + lt + m * T));
    }
    __syncthreads();  // the last exchange has been read out of smem
#pragma unroll
    for (int m = 0; m < P; ++m) smem[lt + m * T] = v[m];  // B_r in natural order
    cl.sync();  // every B_q is in place
    float2 *dst = a.out + row * N;
#pragma unroll
    for (int u = 0; u < P / K; ++u) {
      const int k2 = r * (H / K) + lt + u * T;
      float2 b[K];
#pragma unroll
      for (int q = 0; q < K; ++q) b[q] = *(cl.map_shared_rank(smem, q) + k2);
      Dft<K, D>::run(b);
#pragma unroll
      for (int k1 = 0; k1 < K; ++k1) __stcs(dst + k2 + (long long)k1 * H, cscale(b[k1], a.scale));
    }
    cl.sync();  // no CTA reads this row's B any more
  }
}

}  // namespace fftgb
