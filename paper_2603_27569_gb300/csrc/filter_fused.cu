// Fused spectral filter: y = IFFT(FFT(x) * H) in one kernel per row, and its
// backward, for the SAR range-compression layer (paper Sec. II-D; the fused
// FFT -> matched filter -> IFFT pipeline is the paper's future work, Sec. IX-A).
//
// After any forward Stockham transform (stockham.cuh) thread lt holds output
// lt + m T in register m -- exactly the points pass 0 of the next transform
// reads.  So the forward FFT, the multiply by H and the unnormalised inverse
// run back to back on registers with no extra exchange: one HBM read and one
// HBM write per point (plus the optional saved spectrum).
//
//   forward   y = G (F x * H)              (conj_h: * conj(H))
//             X_save = F x                 (optional, for the backward)
//   backward  g_z = G^H g_y = F g_y / N
//             grad_x = F^H (conj(H) * g_z) = G (F g_y * conj(H))
//             grad_H = sum_rows conj(X) * g_z
// The backward accumulates conj(X) * F g_y per CTA in registers (a thread's
// frequencies k = lt + m T are the same for every row it handles), writes
// one partial row per CTA, and a fixed-order pairwise tree over the CTAs
// finishes grad_H (bitwise reproducible for a given GPU).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "plan.h"
#include "stockham.cuh"

namespace fftgb {

enum FilterMode { FM_FWD = 0, FM_BWD = 1 };

struct FilterArgs {
  const float2 *in;       // x (forward) or g_y (backward)
  float2 *out;            // y or grad_x
  const float2 *H;        // [N]
  float2 *x_save;         // forward: F x (nullable)
  const float2 *x_saved;  // backward: F x from the forward
  float2 *partial;        // backward: [gridDim.x][N]
  const float2 *tw;
  long long batch;
  int conj_h;
};

// Register budget: up to 128 per thread (two CTAs per SM for the
// 256/512-thread variants; the 1024-thread N = 16384 variant is held to 64).
// The H and saved-spectrum reads are made to depend on the forward
// transform's result so the compiler cannot hoist them above it.
template <int N, int P, int TB, class SC, int MODE>
__global__ void __launch_bounds__(TB *(N / P), (65536 / (TB * (N / P) * 128)) > 0 ? 65536 / (TB * (N / P) * 128) : 1)
filter_kernel(FilterArgs a) {
  constexpr int T = N / P;
  extern __shared__ float2 smem[];
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long ntiles = (a.batch + TB - 1) / TB;
  const float inv_n = 1.0f / (float)N;
  float2 acc[MODE == FM_BWD ? P : 1];
  if constexpr (MODE == FM_BWD) {
#pragma unroll
    for (int m = 0; m < P; ++m) acc[m] = make_float2(0.f, 0.f);
  }
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row = tile * TB + b;
    const bool active = row < a.batch;
    float2 v[P];
    const float2 *src = a.in + row * N;
    asm volatile("" : "+l"(src));  // no hoisting of the next row's loads into this row
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = active ? __ldcs(src + lt + m * T) : make_float2(0.f, 0.f);
    const float2 *twp = a.tw;
    float2 *bufp = buf;
    int ltp = lt;
    asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
#pragma unroll
    for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
    run_passes<N, P, -1, SC, 0, SwizzledRow, 1>(v, ltp, bufp, twp, SwizzledRow{});
#pragma unroll
    for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
    // v[m] = (F x)[ltp + m T]
    const float2 *Hp = a.H;
    const float2 *xsp = a.x_saved;
    asm volatile("" : "+l"(Hp), "+l"(xsp), "+f"(v[0].x), "+f"(v[P - 1].y));
    if constexpr (MODE == FM_FWD) {
      if (a.x_save && active) {
        float2 *xs = a.x_save + row * N;
#pragma unroll
        for (int m = 0; m < P; ++m) __stcs(xs + ltp + m * T, v[m]);
      }
    } else {
      if (active) {
        const float2 *xs = xsp + row * N;
#pragma unroll
        for (int m = 0; m < P; ++m) {
          const float2 X = __ldcs(xs + ltp + m * T);
          // conj(X) * (F g_y)
          acc[m].x = fmaf(X.x, v[m].x, fmaf(X.y, v[m].y, acc[m].x));
          acc[m].y = fmaf(X.x, v[m].y, fmaf(-X.y, v[m].x, acc[m].y));
        }
      }
    }
    const bool cj = (MODE == FM_BWD) || a.conj_h;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const float2 h = __ldg(Hp + ltp + m * T);
      v[m] = cj ? cmulc(v[m], h) : cmul(v[m], h);
    }
    // A scheduling fence on every data register: nothing of one transform
    // is interleaved with the other.
#pragma unroll
    for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
    __syncthreads();  // the forward's last exchange is read out of the buffer
    // Opaque again: otherwise the inverse's exchange addresses (equal to the
    // forward's) stay live across both transforms and exhaust the registers.
    asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
    run_passes<N, P, +1, SC, 0, SwizzledRow, 1>(v, ltp, bufp, twp, SwizzledRow{});
    if (active) {
      float2 *dst = a.out + row * N;
#pragma unroll
      for (int m = 0; m < P; ++m) __stcs(dst + final_index<N, P, SC>(ltp, m), cscale(v[m], inv_n));
    }
    __syncthreads();  // the next tile rewrites the buffer
  }
  if constexpr (MODE == FM_BWD) {
    // sum the CTA's row slots in slot order, then one partial row per CTA
#pragma unroll
    for (int m = 0; m < P; ++m) buf[lt + m * T] = acc[m];
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      float2 s = smem[k];
      for (int bb = 1; bb < TB; ++bb) s = cadd(s, smem[bb * N + k]);
      a.partial[(size_t)blockIdx.x * N + k] = cscale(s, inv_n);
    }
  }
}

// Pairwise tree over the CTA partials: level h adds row c + h into row c.
__global__ void filter_tree_kernel(float2 *partial, int N, int rows, int h) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y * 2 * h;
  if (k >= N || c + h >= rows) return;
  partial[(size_t)c * N + k] = cadd(partial[(size_t)c * N + k], partial[(size_t)(c + h) * N + k]);
}

__global__ void filter_copy_kernel(const float2 *src, float2 *dst, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) dst[k] = src[k];
}

struct FilterVariant {
  const void *fwd, *bwd;
  int threads, tb;
  size_t smem;
  KernelEntry sched;  // radix schedule (for the twiddle tables)
};

template <int N, int P, int TB, int... Rs>
static FilterVariant make_variant() {
  using SC = Sched<Rs...>;
  FilterVariant v;
  v.fwd = (const void *)&filter_kernel<N, P, TB, SC, FM_FWD>;
  v.bwd = (const void *)&filter_kernel<N, P, TB, SC, FM_BWD>;
  v.threads = TB * (N / P);
  v.tb = TB;
  v.smem = sizeof(float2) * (size_t)N * TB;
  v.sched = KernelEntry{};
  v.sched.npass = SC::npass;
  for (int i = 0; i < SC::npass; ++i) v.sched.radix[i] = SC::radix[i];
  return v;
}

static bool filter_variant(int N, FilterVariant *v) {
  switch (N) {
    case 256: *v = make_variant<256, 16, 16, 16, 16>(); return true;
    case 512: *v = make_variant<512, 16, 8, 16, 16, 2>(); return true;
    case 1024: *v = make_variant<1024, 16, 4, 16, 16, 4>(); return true;
    case 2048: *v = make_variant<2048, 16, 2, 16, 16, 8>(); return true;
    case 4096: *v = make_variant<4096, 16, 1, 16, 16, 16>(); return true;
    case 8192: *v = make_variant<8192, 16, 1, 16, 16, 16, 2>(); return true;
    case 16384: *v = make_variant<16384, 16, 1, 16, 16, 16, 4>(); return true;
  }
  return false;
}

struct FilterState {
  FilterVariant v;
  int grid_bwd = 0;
  float2 *d_partial = nullptr;
};

void filter_destroy(fft_plan_impl *pl) {
  FilterState *f = (FilterState *)pl->filter;
  if (f) cudaFree(f->d_partial);
  delete f;
  pl->filter = nullptr;
}

}  // namespace fftgb

using namespace fftgb;

extern "C" {

fft_status_t fft_filter_plan(fft_plan_t *out, int N, int64_t batch) {
  if (!out) return FFT_ERR_INVALID_VALUE;
  *out = nullptr;
  if (batch < 0 || N < 2 || N > 16384 || (N & (N - 1))) return FFT_ERR_INVALID_SIZE;
  FilterVariant v;
  if (!filter_variant(N, &v)) return FFT_ERR_NOT_SUPPORTED;
  fft_plan_s *h = new (std::nothrow) fft_plan_s;
  FilterState *f = new (std::nothrow) FilterState;
  if (!h || !f) {
    delete h;
    delete f;
    return FFT_ERR_ALLOC;
  }
  fft_plan_impl *pl = &h->impl;
  pl->N = N;
  pl->batch = batch;
  pl->path = FFT_PATH_FILTER;
  pl->filter = f;
  f->v = v;
  cudaGetDevice(&pl->device);
  auto fail = [&](fft_status_t e) {
    filter_destroy(pl);
    if (pl->d_tw) cudaFree(pl->d_tw);
    if (pl->d_status) cudaFree(pl->d_status);
    delete h;
    return e;
  };
  if (cudaMalloc(&pl->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  cudaMemset(pl->d_status, 0, sizeof(int));
  if (v.smem > 48 * 1024) {
    if (cudaFuncSetAttribute(v.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(v.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) !=
            cudaSuccess)
      return fail(FFT_ERR_CUDA);
  }
  int64_t off = 0;
  fft_status_t s = build_twiddles(pl, pass_segments(v.sched, off));
  if (s != FFT_OK) return fail(s);
  int sms = 0, occ = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.bwd, v.threads, v.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_CUDA);
  }
  const int64_t tiles = (batch + v.tb - 1) / v.tb;
  f->grid_bwd = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(occ, 1) * sms));
  if (cudaMalloc(&f->d_partial, sizeof(float2) * (size_t)f->grid_bwd * N) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  pl->scratch_bytes = (int64_t)sizeof(float2) * f->grid_bwd * N;
  *out = h;
  return FFT_OK;
}

static fft_status_t filter_check(fft_plan_t plan, const void *a, const void *b, const void *c) {
  if (!plan || plan->impl.path != FFT_PATH_FILTER) return FFT_ERR_INVALID_VALUE;
  if (!a || !b || !c) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) return FFT_ERR_MISALIGNED;
  return FFT_OK;
}

fft_status_t fft_filter_forward(fft_plan_t plan, const void *x, const void *H, void *y,
                                void *X_save, int conj_h, void *stream) {
  fft_status_t s = filter_check(plan, x, H, y);
  if (s != FFT_OK) return s;
  if ((uintptr_t)X_save & 15) return FFT_ERR_MISALIGNED;
  fft_plan_impl *pl = &plan->impl;
  FilterState *f = (FilterState *)pl->filter;
  if (pl->batch == 0) return FFT_OK;
  FilterArgs a{};
  a.in = (const float2 *)x;
  a.out = (float2 *)y;
  a.H = (const float2 *)H;
  a.x_save = (float2 *)X_save;
  a.tw = pl->d_tw;
  a.batch = pl->batch;
  a.conj_h = conj_h ? 1 : 0;
  const int64_t grid = (pl->batch + f->v.tb - 1) / f->v.tb;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  void *args[] = {&a};
  return cuda_status(cudaLaunchKernel(f->v.fwd, dim3((unsigned)grid), dim3(f->v.threads), args,
                                      f->v.smem, (cudaStream_t)stream));
}

fft_status_t fft_filter_backward(fft_plan_t plan, const void *g_y, const void *H,
                                 const void *X_saved, void *grad_x, void *grad_H, void *stream) {
  fft_status_t s = filter_check(plan, g_y, H, grad_x);
  if (s != FFT_OK) return s;
  if (!X_saved || !grad_H) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)X_saved | (uintptr_t)grad_H) & 15) return FFT_ERR_MISALIGNED;
  fft_plan_impl *pl = &plan->impl;
  FilterState *f = (FilterState *)pl->filter;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = pl->N;
  if (pl->batch == 0) return cuda_status(cudaMemsetAsync(grad_H, 0, sizeof(float2) * N, st));
  FilterArgs a{};
  a.in = (const float2 *)g_y;
  a.out = (float2 *)grad_x;
  a.H = (const float2 *)H;
  a.x_saved = (const float2 *)X_saved;
  a.partial = f->d_partial;
  a.tw = pl->d_tw;
  a.batch = pl->batch;
  a.conj_h = 1;
  void *args[] = {&a};
  if (cudaLaunchKernel(f->v.bwd, dim3(f->grid_bwd), dim3(f->v.threads), args, f->v.smem, st) !=
      cudaSuccess)
    return FFT_ERR_CUDA;
  const unsigned bx = (unsigned)((N + 255) / 256);
  for (int h = 1; h < f->grid_bwd; h *= 2) {
    const unsigned groups = (unsigned)((f->grid_bwd + 2 * h - 1) / (2 * h));
    filter_tree_kernel<<<dim3(bx, groups), 256, 0, st>>>(f->d_partial, N, f->grid_bwd, h);
  }
  filter_copy_kernel<<<bx, 256, 0, st>>>(f->d_partial, (float2 *)grad_H, N);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
