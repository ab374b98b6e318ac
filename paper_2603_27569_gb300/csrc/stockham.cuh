// Single-CTA Stockham autosort FFT (paper Sec. II-B, V-A, V-B).
//
// One CTA transforms TB independent rows of N points.  Each row is handled by
// T = N / P threads; every thread keeps P complex points in registers.  The
// radix schedule R_0, R_1, ... (product N) is a template pack.  Pass s has
// stride p_s = R_0 ... R_{s-1} and radix r = R_s; butterfly i (0 <= i < N/r)
// reads the points i + j N/r (j < r), multiplies point j by W_{p r}^{j k}
// with k = i mod p (skipped in pass 0, where p = 1), applies DFT_r in
// registers and writes output j to (i - k) r + k + j p.  After the last pass
// the rows are in natural order (no bit reversal, Sec. II-B).
//
// With r < P a thread runs P / r butterflies per pass, i = t + q T, so its
// read set is always {t + m T : m < P} and needs no per-pass reshuffle.
//
// Memory: pass 0 reads straight from global memory into registers and the
// last pass stores straight from registers (the device-memory bypass of
// Sec. V-A); passes exchange through one shared buffer of N points per row,
// laid out by swz<> so that every exchange is free of bank conflicts.  Every
// pass is unrolled with compile-time strides (Sec. V-A).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "butterfly.cuh"

namespace fftgb {

template <int... Rs>
struct Sched {
  static constexpr int npass = sizeof...(Rs);
  static constexpr int radix[npass] = {Rs...};
  __host__ __device__ static constexpr int product() {
    int v = 1;
    for (int i = 0; i < npass; ++i) v *= radix[i];
    return v;
  }
  __host__ __device__ static constexpr int stride(int s) {
    int v = 1;
    for (int i = 0; i < s; ++i) v *= radix[i];
    return v;
  }
  // Offset (in entries) of pass s's twiddle table; pass s holds (r_s - 1) p_s
  // entries laid out [j - 1][k].
  __host__ __device__ static constexpr int tw_offset(int s) {
    int off = 0;
    for (int i = 1; i < s; ++i) off += (radix[i] - 1) * stride(i);
    return off;
  }
  __host__ __device__ static constexpr int tw_total() { return tw_offset(npass); }
  __host__ __device__ static constexpr int max_radix() {
    int v = 1;
    for (int i = 0; i < npass; ++i) v = radix[i] > v ? radix[i] : v;
    return v;
  }
};

// Plain-kernel arguments (passed by value).
struct StockhamArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;     // per-pass twiddle tables of this N
  long long batch;      // rows
  float scale;          // applied at the final store (1 or 1/N)
};

// Twiddle + butterflies of pass S for every butterfly q of this thread.
template <int N, int P, int D, class SC, int S>
__device__ __forceinline__ void pass_compute(float2 (&a)[P], int lt, const float2 *__restrict__ tw) {
  constexpr int r = SC::radix[S];
  constexpr int p = SC::stride(S);
  constexpr int T = N / P;
  constexpr int Q = P / r;
  if constexpr (S > 0) {
    const float2 *tws = tw + SC::tw_offset(S);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = lt + q * T;
      const int k = i & (p - 1);
#pragma unroll
      for (int j = 1; j < r; ++j) {
        float2 w = __ldg(tws + (j - 1) * p + k);
        a[q + j * Q] = cmul_dir<D>(a[q + j * Q], w);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 v[r];
#pragma unroll
    for (int j = 0; j < r; ++j) v[j] = a[q + j * Q];
    Dft<r, D>::run(v);
#pragma unroll
    for (int j = 0; j < r; ++j) a[q + j * Q] = v[j];
  }
}

// Exchange-buffer layouts.  SwizzledRow: one row of N points per buffer,
// laid out by swz<> (plain kernel).  Interleaved<C>: C columns interleaved,
// element (idx, c) at idx * C + c (column kernel); 16 consecutive columns
// make every half-warp access conflict-free without a swizzle.
struct SwizzledRow {
  template <int p, int r>
  __device__ __forceinline__ int at(int idx) const { return swz<p, r>(idx); }
};
template <int C>
struct Interleaved {
  int c;
  template <int p, int r>
  __device__ __forceinline__ int at(int idx) const { return idx * C + c; }
};

// Write pass S's outputs into the exchange buffer.
template <int N, int P, class SC, int S, class LY>
__device__ __forceinline__ void pass_write(const float2 (&a)[P], int lt, float2 *buf, const LY &ly) {
  constexpr int r = SC::radix[S];
  constexpr int p = SC::stride(S);
  constexpr int T = N / P;
  constexpr int Q = P / r;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = lt + q * T;
    const int k = i & (p - 1);
    const int base = (i - k) * r + k;
#pragma unroll
    for (int j = 0; j < r; ++j) buf[ly.template at<p, r>(base + j * p)] = a[q + j * Q];
  }
}

// Read the next pass's points {lt + m T} from the buffer written by pass S.
template <int N, int P, class SC, int S, class LY>
__device__ __forceinline__ void pass_read(float2 (&a)[P], int lt, const float2 *buf, const LY &ly) {
  constexpr int r = SC::radix[S];
  constexpr int p = SC::stride(S);
  constexpr int T = N / P;
#pragma unroll
  for (int m = 0; m < P; ++m) a[m] = buf[ly.template at<p, r>(lt + m * T)];
}

// Passes S .. npass-1.  On entry a[] holds pass S's inputs.  On return a[]
// holds the final outputs of the last pass in its butterfly order.
template <int N, int P, int D, class SC, int S, class LY>
__device__ __forceinline__ void run_passes(float2 (&a)[P], int lt, float2 *buf,
                                           const float2 *__restrict__ tw, const LY &ly) {
  pass_compute<N, P, D, SC, S>(a, lt, tw);
  if constexpr (S + 1 < SC::npass) {
    if constexpr (S > 0) __syncthreads();  // every read of the buffer is done
    pass_write<N, P, SC, S>(a, lt, buf, ly);
    __syncthreads();
    pass_read<N, P, SC, S>(a, lt, buf, ly);
    run_passes<N, P, D, SC, S + 1>(a, lt, buf, tw, ly);
  }
}

// Final-pass output index of register m (after run_passes): the last pass
// has p = N / r, so butterfly i writes j to i + j N / r.
template <int N, int P, class SC>
__device__ __forceinline__ int final_index(int lt, int m) {
  constexpr int r = SC::radix[SC::npass - 1];
  constexpr int Q = P / r;
  constexpr int T = N / P;
  const int q = m % Q, j = m / Q;
  return lt + q * T + j * (N / r);
}

template <int N, int P, int TB, int D, class SC>
__global__ void __launch_bounds__(TB *(N / P))
stockham_kernel(StockhamArgs args) {
  static_assert(SC::product() == N, "radix schedule must multiply to N");
  static_assert(P % SC::max_radix() == 0, "every radix must divide P");
  constexpr int T = N / P;
  extern __shared__ float2 smem[];
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  const long long row = (long long)blockIdx.x * TB + b;
  const bool active = row < args.batch;
  float2 *buf = smem + b * N;
  float2 a[P];
  const float2 *src = args.in + row * N;
  if (active) {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = __ldg(src + lt + m * T);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
  }
  run_passes<N, P, D, SC, 0>(a, lt, buf, args.tw, SwizzledRow{});
  if (active) {
    float2 *dst = args.out + row * N;
    const float s = args.scale;
#pragma unroll
    for (int m = 0; m < P; ++m) dst[final_index<N, P, SC>(lt, m)] = cscale(a[m], s);
  }
}

}  // namespace fftgb
