// Fused spectral filter: y = IFFT(FFT(x) * H) in one kernel per row (two
// from N = 8192 on, see variant()), and its backward, for the SAR range-compression layer (paper Sec. II-D; the fused
// FFT -> matched filter -> IFFT pipeline is the paper's future work, Sec. IX-A).
//
// After any forward Stockham transform (stockham.cuh) thread lt holds output
// lt + m T in register m -- exactly the points pass 0 of the next transform
// reads.  So the forward FFT, the multiply by H and the unnormalised inverse
// run back to back on registers with no extra exchange: one HBM read and one
// HBM write per point (plus the optional saved spectrum).
//
//   forward   y = G (F x * H)              (conj_h: * conj(H))       FM_FWD
//             X_save = F x                 (optional, for the backward)
//             (N >= 8192: FM_SPEC into X_save or y, then FM_MULINV)
//   backward  g_z = G^H g_y = F g_y / N                              FM_SPEC
//             grad_H = sum_rows conj(X) * g_z   (fft_filter_grad_h: 32-row
//                      chunks, then a fixed-order pairwise tree)
//             grad_x = F^H (conj(H) * g_z)                           FM_MULINV
// The backward keeps g_z in grad_x's buffer: FM_SPEC writes it there, the
// reduction reads it, and FM_MULINV transforms it in place (a CTA reads its
// whole row before it writes it).  Keeping grad_H's per-frequency sums in
// registers inside one backward kernel instead needs P more complex
// registers per thread; on GB300 that forced 16 points per thread with
// spills, and the three-step backward measured faster at every N.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "plan.h"
#include "stockham.cuh"

extern "C" int64_t fft_filter_grad_h_workspace(int N, int64_t batch);
extern "C" fft_status_t fft_filter_grad_h(const void *X, const void *G, void *grad_H, int N,
                                          int64_t batch, void *work, void *stream);

namespace fftgb {

enum FilterMode { FM_FWD = 0, FM_SPEC = 1, FM_MULINV = 2 };

struct FilterArgs {
  const float2 *in;       // x (FM_FWD), g_y (FM_SPEC) or g_z (FM_MULINV)
  float2 *out;            // y, g_z or grad_x (FM_MULINV: may equal in)
  const float2 *H;        // [N] (FM_FWD, FM_MULINV)
  float2 *x_save;         // FM_FWD: F x (nullable)
  const float2 *tw;
  long long batch;
  int conj_h;             // multiply by conj(H) instead of H
  float scale;            // applied at the final store
};

// Register budget: up to 128 per thread (two CTAs per SM for the 256-thread
// variants).  The H reads are made to depend on the forward transform's
// result so the compiler cannot hoist them above it.
template <int N, int P, int TB, class SC, int MODE>
__global__ void __launch_bounds__(TB *(N / P), (65536 / (TB * (N / P) * 128)) > 0 ? 65536 / (TB * (N / P) * 128) : 1)
filter_kernel(FilterArgs a) {
  constexpr int T = N / P;
  extern __shared__ __align__(128) float2 smem[];
  // Programmatic dependent launch (see stockham_kernel): nothing global
  // before the previous kernel of the stream has completed.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long ntiles = (a.batch + TB - 1) / TB;
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
    if constexpr (MODE != FM_MULINV) {
      run_passes<N, P, -1, SC, 0, SwizzledRow, 1>(v, ltp, bufp, twp, SwizzledRow{});
#pragma unroll
      for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
      // v[m] = (F in)[ltp + m T]
    }
    if constexpr (MODE == FM_SPEC) {
      if (active) {
        float2 *dst = a.out + row * N;
#pragma unroll
        for (int m = 0; m < P; ++m) __stcs(dst + ltp + m * T, cscale(v[m], a.scale));
      }
    } else {
      const float2 *Hp = a.H;
      asm volatile("" : "+l"(Hp), "+f"(v[0].x), "+f"(v[P - 1].y));
      if constexpr (MODE == FM_FWD) {
        if (a.x_save && active) {
          float2 *xs = a.x_save + row * N;
#pragma unroll
          for (int m = 0; m < P; ++m) __stcs(xs + ltp + m * T, v[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < P; ++m) {
        const float2 h = __ldg(Hp + ltp + m * T);
        v[m] = a.conj_h ? cmulc(v[m], h) : cmul(v[m], h);
      }
      // A scheduling fence on every data register: nothing of one transform
      // is interleaved with the other.
#pragma unroll
      for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
      if constexpr (MODE == FM_FWD) __syncthreads();  // the forward's last exchange is read
      // Opaque again: otherwise the inverse's exchange addresses (equal to the
      // forward's) stay live across both transforms and exhaust the registers.
      asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
      run_passes<N, P, +1, SC, 0, SwizzledRow, 1>(v, ltp, bufp, twp, SwizzledRow{});
      if (active) {
        float2 *dst = a.out + row * N;
#pragma unroll
        for (int m = 0; m < P; ++m)
          __stcs(dst + final_index<N, P, SC>(ltp, m), cscale(v[m], a.scale));
      }
    }
    __syncthreads();  // the next tile rewrites the buffer
  }
}

struct FilterKernel {
  const void *fn;
  int threads, tb;
  size_t smem;
};

template <int N, int P, int TB, class SC, int MODE>
static FilterKernel make_kernel() {
  FilterKernel k;
  k.fn = (const void *)&filter_kernel<N, P, TB, SC, MODE>;
  k.threads = TB * (N / P);
  k.tb = TB;
  k.smem = sizeof(float2) * (size_t)N * TB;
  return k;
}

// The kernels of one N share a radix schedule (and its twiddle tables): 32
// points per thread from 8192 on (three passes, like the plain transform's
// built-in), 16 below.  With 32 points both transforms of FM_FWD do not fit
// the register budget (~0.8-1 KiB of spills per thread, written back to
// DRAM), so from 8192 on the forward runs as FM_SPEC into the saved spectrum
// (or into y) and FM_MULINV from there: one more HBM pass, no spills, and
// measured faster.
struct FilterVariant {
  FilterKernel fwd, spec, mulinv;  // fwd.fn == nullptr: the two-kernel forward
  KernelEntry sched;
};

template <int N, int P, int TB, int... Rs>
static FilterVariant variant() {
  using SC = Sched<Rs...>;
  FilterVariant v;
  if constexpr (P < 32) v.fwd = make_kernel<N, P, TB, SC, FM_FWD>();
  else v.fwd = FilterKernel{nullptr, 0, 0, 0};
  v.spec = make_kernel<N, P, TB, SC, FM_SPEC>();
  v.mulinv = make_kernel<N, P, TB, SC, FM_MULINV>();
  v.sched = KernelEntry{};
  v.sched.npass = SC::npass;
  for (int i = 0; i < SC::npass; ++i) v.sched.radix[i] = SC::radix[i];
  return v;
}

static bool filter_variant(int N, FilterVariant *v) {
  switch (N) {
    case 256: *v = variant<256, 16, 16, 16, 16>(); return true;
    case 512: *v = variant<512, 16, 8, 16, 16, 2>(); return true;
    case 1024: *v = variant<1024, 16, 4, 16, 16, 4>(); return true;
    case 2048: *v = variant<2048, 16, 2, 16, 16, 8>(); return true;
    case 4096: *v = variant<4096, 16, 1, 16, 16, 16>(); return true;
    case 8192: *v = variant<8192, 32, 1, 32, 16, 16>(); return true;
    case 16384: *v = variant<16384, 32, 1, 32, 32, 16>(); return true;
  }
  return false;
}

struct FilterState {
  FilterVariant v;
  float2 *d_work = nullptr;  // grad_H reduction workspace (32-row chunk sums)
};

void filter_destroy(fft_plan_impl *pl) {
  FilterState *f = (FilterState *)pl->filter;
  if (f) cudaFree(f->d_work);
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
  for (const FilterKernel *k : {&v.fwd, &v.spec, &v.mulinv}) {
    if (k->fn && k->smem > 48 * 1024 &&
        cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k->smem) !=
            cudaSuccess)
      return fail(FFT_ERR_CUDA);
  }
  int64_t off = 0;
  fft_status_t s = build_twiddles(pl, pass_segments(v.sched, off));
  if (s != FFT_OK) return fail(s);
  const int64_t work = fft_filter_grad_h_workspace(N, batch);
  if (work > 0 && cudaMalloc(&f->d_work, (size_t)work) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  pl->scratch_bytes = work;
  *out = h;
  return FFT_OK;
}

static fft_status_t filter_check(fft_plan_t plan, const void *a, const void *b, const void *c) {
  if (!plan || plan->impl.path != FFT_PATH_FILTER) return FFT_ERR_INVALID_VALUE;
  if (!a || !b || !c) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) return FFT_ERR_MISALIGNED;
  return FFT_OK;
}

static fft_status_t filter_launch(const FilterKernel &k, FilterArgs &a, cudaStream_t st) {
  const int64_t grid = (a.batch + k.tb - 1) / k.tb;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  void *args[] = {&a};
  return cuda_status(launch_pdl(k.fn, dim3((unsigned)grid), dim3(k.threads), k.smem, st, args));
}

fft_status_t fft_filter_forward(fft_plan_t plan, const void *x, const void *H, void *y,
                                void *X_save, int conj_h, void *stream) {
  fft_status_t s = filter_check(plan, x, H, y);
  if (s != FFT_OK) return s;
  if ((uintptr_t)X_save & 15) return FFT_ERR_MISALIGNED;
  fft_plan_impl *pl = &plan->impl;
  FilterState *f = (FilterState *)pl->filter;
  if (pl->batch == 0) return FFT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  FilterArgs a{};
  a.in = (const float2 *)x;
  a.out = (float2 *)y;
  a.H = (const float2 *)H;
  a.x_save = (float2 *)X_save;
  a.tw = pl->d_tw;
  a.batch = pl->batch;
  a.conj_h = conj_h ? 1 : 0;
  a.scale = 1.0f / (float)pl->N;
  if (f->v.fwd.fn) return filter_launch(f->v.fwd, a, st);
  // two kernels: F x into X_save (or y), then y = G (F x * H) from there
  const int64_t bytes = (int64_t)sizeof(float2) * pl->N * pl->batch;
  if (X_save) {
    const char *p = (const char *)X_save;
    for (const void *o : {x, (const void *)y}) {
      const char *q = (const char *)o;
      if (p < q + bytes && q < p + bytes) return FFT_ERR_INVALID_VALUE;
    }
  }
  float2 *spec = X_save ? (float2 *)X_save : (float2 *)y;
  a.out = spec;
  a.x_save = nullptr;
  a.scale = 1.0f;
  if ((s = filter_launch(f->v.spec, a, st)) != FFT_OK) return s;
  a.in = spec;
  a.out = (float2 *)y;
  a.scale = 1.0f / (float)pl->N;
  return filter_launch(f->v.mulinv, a, st);
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
  const int64_t bytes = (int64_t)sizeof(float2) * N * pl->batch;
  {  // grad_x doubles as g_z's buffer, so it may not overlap the other operands
    const char *gx = (const char *)grad_x;
    for (const void *o : {g_y, X_saved}) {
      const char *p = (const char *)o;
      if (p < gx + bytes && gx < p + bytes) return FFT_ERR_INVALID_VALUE;
    }
  }
  FilterArgs a{};
  a.tw = pl->d_tw;
  a.batch = pl->batch;
  // g_z = F g_y / N, into grad_x's buffer
  a.in = (const float2 *)g_y;
  a.out = (float2 *)grad_x;
  a.scale = 1.0f / (float)N;
  if ((s = filter_launch(f->v.spec, a, st)) != FFT_OK) return s;
  // grad_H = sum_rows conj(X) * g_z
  if ((s = fft_filter_grad_h(X_saved, grad_x, grad_H, N, pl->batch, f->d_work, st)) != FFT_OK)
    return s;
  // grad_x = F^H (conj(H) * g_z), in place
  a.in = (const float2 *)grad_x;
  a.out = (float2 *)grad_x;
  a.H = (const float2 *)H;
  a.conj_h = 1;
  a.scale = 1.0f;
  return filter_launch(f->v.mulinv, a, st);
}

}  // extern "C"
