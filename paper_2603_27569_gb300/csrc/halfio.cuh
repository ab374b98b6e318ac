// 16-bit-storage FFT: complex values stored in HBM as two FP16 or two BF16
// halves (4 bytes per point), transformed in FP32 in registers and shared
// memory (paper Sec. IX-A mixed-precision future work: half the bytes for
// SNR-limited radar data).  The passes are the single-CTA Stockham passes of
// stockham.cuh; only the first load (16-bit -> FP32, exact) and the last
// store (FP32 -> 16-bit, round to nearest; FP16 overflows to infinity, BF16
// keeps the FP32 range with 8 significant bits) differ.  The output is
// scaled (1/N for the inverse) before rounding.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stockham.cuh"

namespace fftgb {

// The pair type's conversions: S2 = __half2 (FP16) or __nv_bfloat162 (BF16).
__device__ __forceinline__ float2 pair_to_float2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 pair_to_float2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <class S2>
__device__ __forceinline__ S2 float2_to_pair(float2 v);
template <>
__device__ __forceinline__ __half2 float2_to_pair<__half2>(float2 v) { return __float22half2_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat162 float2_to_pair<__nv_bfloat162>(float2 v) {
  return __float22bfloat162_rn(v);
}

struct HalfArgs {
  const void *in;   // __half2 or __nv_bfloat162 pairs, per the kernel's S2
  void *out;
  const float2 *tw;
  long long batch;
  float scale;
};

template <int N, int P, int TB, int D, class SC, int TWM, class S2>
__global__ void __launch_bounds__(TB *(N / P))
stockham_half_kernel(HalfArgs args) {
  static_assert(SC::product() == N, "radix schedule must multiply to N");
  constexpr int T = N / P;
  extern __shared__ __align__(128) float2 smem[];
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long row = (long long)blockIdx.x * TB + b;
  const bool active = row < args.batch;
  float2 a[P];
  const S2 *src = static_cast<const S2 *>(args.in) + row * N;
  if (active) {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = pair_to_float2(__ldcs(src + lt + m * T));
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
  }
  run_passes<N, P, D, SC, 0, SwizzledRow, TWM>(a, lt, buf, args.tw, SwizzledRow{});
  if (active) {
    S2 *dst = static_cast<S2 *>(args.out) + row * N;
    const float s = args.scale;
#pragma unroll
    for (int m = 0; m < P; ++m)
      __stcs(dst + final_index<N, P, SC>(lt, m), float2_to_pair<S2>(cscale(a[m], s)));
  }
}

}  // namespace fftgb
