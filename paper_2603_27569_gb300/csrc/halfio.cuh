// FP16-storage FFT: complex values stored in HBM as two FP16 halves (4 bytes
// per point), transformed in FP32 in registers and shared memory (paper Sec.
// IX-A mixed-precision future work: half the bytes for SNR-limited radar
// data).  The passes are the single-CTA Stockham passes of stockham.cuh; only
// the first load (FP16 -> FP32) and the last store (FP32 -> FP16, round to
// nearest, overflow to infinity) differ.  The output is scaled (1/N for the
// inverse) before rounding.
#pragma once
#include <cuda_fp16.h>

#include "stockham.cuh"

namespace fftgb {

struct HalfArgs {
  const __half2 *in;
  __half2 *out;
  const float2 *tw;
  long long batch;
  float scale;
};

template <int N, int P, int TB, int D, class SC, int TWM>
__global__ void __launch_bounds__(TB *(N / P))
stockham_half_kernel(HalfArgs args) {
  static_assert(SC::product() == N, "radix schedule must multiply to N");
  constexpr int T = N / P;
  extern __shared__ float2 smem[];
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long row = (long long)blockIdx.x * TB + b;
  const bool active = row < args.batch;
  float2 a[P];
  const __half2 *src = args.in + row * N;
  if (active) {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = __half22float2(__ldcs(src + lt + m * T));
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
  }
  run_passes<N, P, D, SC, 0, SwizzledRow, TWM>(a, lt, buf, args.tw, SwizzledRow{});
  if (active) {
    __half2 *dst = args.out + row * N;
    const float s = args.scale;
#pragma unroll
    for (int m = 0; m < P; ++m)
      __stcs(dst + final_index<N, P, SC>(lt, m), __float22half2_rn(cscale(a[m], s)));
  }
}

}  // namespace fftgb
