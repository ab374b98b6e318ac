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
//   forward   y = G (F x * H)              (conj_h: * conj(H))       FM_FWD
//             X_save = F x                 (optional, for the backward)
//             (N >= 8192: filter_fwd2_kernel, the two halves as calls)
//   backward  g_z = G^H g_y = F g_y / N                              FM_SPEC
//             grad_H = sum_rows conj(X) * g_z   (fft_filter_grad_h: 32-row
//                      chunks, then a fixed-order pairwise tree)
//             grad_x = F^H (conj(H) * g_z)                           FM_MULINV
//             (N >= 8192: filter_bwd2_kernel, one kernel whose grad_H
//              partial sums live in tensor memory, then the same tree)
// Below 8192 the backward keeps g_z in grad_x's buffer: FM_SPEC writes it
// there, the reduction reads it, and FM_MULINV transforms it in place (a CTA
// reads its whole row before it writes it).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "plan.h"
#include "stockham.cuh"
#include "tmem.cuh"

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
  long long ahead;        // one tile per CTA: resident CTAs (the look-ahead prefetch)
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

// One-kernel forward for 32 points per thread (N >= 8192): the row's first
// half (F x, the optional saved spectrum, the multiply by H) and its second
// half (the inverse) are separately compiled device functions that meet only
// through the exchange buffer, where the first half leaves F x * H in natural
// order.  Inlined into one body, the two transforms' register allocations
// merge and spill (~0.8 KiB per thread); as calls, each half is allocated on
// its own and only pointers cross.  One HBM read and one write per point
// (plus the saved spectrum), the arithmetic of FM_SPEC followed by FM_MULINV.
// Launched with one CTA per row; warp 0 first asks the bulk-copy engine to
// prefetch into L2 the row of the CTA one resident wave later (blockIdx +
// occupancy x SMs), so later waves read their rows from L2.  (Launched as a
// resident grid instead, each CTA prefetches its own next row.)
// Output index of register m after a transform whose last pass is paired (PL:
// registers 2j, 2j + 1 hold adjacent outputs, moved as one 16-byte access) or
// not.
template <int N, int P, class SC, bool PL>
__device__ __forceinline__ int out_index(int lt, int m) {
  if constexpr (PL) return final_index_pair<N, P, SC>(lt, m >> 1) + (m & 1);
  else return final_index<N, P, SC>(lt, m);
}
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int N, int P, class SC>
__device__ __noinline__ void filter_half_fwd(const float2 *src, float2 *xs, const float2 *H,
                                             float2 *buf, const float2 *tw, int lt, int active,
                                             int conj_h) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = active ? __ldcs(src + lt + m * T) : make_float2(0.f, 0.f);
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
  // v[m] = (F x)[out_index(lt, m)]
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2) {
      const int k = out_index<N, P, SC, PL>(lt, m);
      if (active && xs) __stcs(reinterpret_cast<float4 *>(xs + k), pack2(v[m], v[m + 1]));
      const float4 h = __ldg(reinterpret_cast<const float4 *>(H + k));
      v[m] = conj_h ? cmulc(v[m], lo2(h)) : cmul(v[m], lo2(h));
      v[m + 1] = conj_h ? cmulc(v[m + 1], hi2(h)) : cmul(v[m + 1], hi2(h));
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int k = out_index<N, P, SC, PL>(lt, m);
      if (active && xs) __stcs(xs + k, v[m]);
      const float2 h = __ldg(H + k);
      v[m] = conj_h ? cmulc(v[m], h) : cmul(v[m], h);
    }
  }
  __syncthreads();  // every read of the buffer by the transform is done
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2)
      *reinterpret_cast<float4 *>(buf + out_index<N, P, SC, PL>(lt, m)) = pack2(v[m], v[m + 1]);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) buf[out_index<N, P, SC, PL>(lt, m)] = v[m];
  }
}

template <int N, int P, class SC>
__device__ __noinline__ void filter_half_inv(float2 *buf, float2 *dst, const float2 *tw, int lt,
                                             int active, float scale) {
  constexpr int T = N / P;
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = buf[lt + m * T];
  __syncthreads();  // every thread has its inputs: the transform may overwrite the buffer
  constexpr bool PL = pairable<N, P, SC>();
  run_passes<N, P, +1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
  if (active) {
    if constexpr (PL) {
#pragma unroll
      for (int m = 0; m < P; m += 2)
        __stcs(reinterpret_cast<float4 *>(dst + out_index<N, P, SC, PL>(lt, m)),
               pack2(cscale(v[m], scale), cscale(v[m + 1], scale)));
    } else {
#pragma unroll
      for (int m = 0; m < P; ++m) __stcs(dst + out_index<N, P, SC, PL>(lt, m), cscale(v[m], scale));
    }
  }
}

template <int N, int P, int TB, class SC>
__global__ void __launch_bounds__(TB *(N / P), (65536 / (TB * (N / P) * 128)) > 0 ? 65536 / (TB * (N / P) * 128) : 1)
filter_fwd2_kernel(FilterArgs a) {
  constexpr int T = N / P;
  extern __shared__ __align__(128) float2 smem[];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long ntiles = (a.batch + TB - 1) / TB;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // a resident grid prefetches the CTA's own next tile; a grid of one CTA
    // per tile, the tile of the CTA one resident wave later
    const long long next = tile + (gridDim.x >= ntiles ? a.ahead : gridDim.x);
    if (threadIdx.x < 32 && next > tile && next < ntiles) {  // that tile's rows into L2
      const long long rows = a.batch - next * TB < TB ? a.batch - next * TB : TB;
      prefetch_l2_warp(a.in + next * TB * N, rows * N * (long long)sizeof(float2), threadIdx.x);
    }
    const long long row = tile * TB + b;
    const int active = row < a.batch;
    filter_half_fwd<N, P, SC>(a.in + row * N, a.x_save ? a.x_save + row * N : nullptr, a.H, buf,
                              a.tw, lt, active, a.conj_h);
    __syncthreads();  // F x * H is in the buffer
    filter_half_inv<N, P, SC>(buf, a.out + row * N, a.tw, lt, active, a.scale);
    __syncthreads();  // the next tile rewrites the buffer
  }
}

// One-kernel backward for 32 points per thread (N >= 8192), persistent:
// CTA c takes rows c, c + G, c + 2G, ... (G = gridDim.x).  Per row, the first
// half computes g_z = F g_y / N, adds conj(X_saved) * g_z into the CTA's
// grad_H partial sums and leaves conj(H) * g_z in the exchange buffer; the
// second half (filter_half_inv) runs F^H into grad_x.  The partial sums live
// in tensor memory (tcgen05): each thread owns its lane and 64 columns, the
// sums of its 32 frequencies, read and written 8 points at a time; each
// frequency's sum runs over the CTA's rows in row order.  At the end every
// CTA writes its sums as one row of `partial` ([G][N]), and grad_h_tree adds
// the G rows in a fixed pairwise order, so grad_H is bitwise reproducible
// for a given grid.
struct FilterBwdArgs {
  const float2 *gy;   // incoming gradient g_y
  const float2 *xs;   // X_saved = F x
  const float2 *H;
  float2 *gx;         // grad_x
  float2 *partial;    // [gridDim.x][N] per-CTA grad_H sums
  const float2 *tw;
  long long batch;
  float inv_n;
};

template <int N, int P, class SC>
__device__ __noinline__ void filter_half_bwd(const float2 *gy, const float2 *xs, const float2 *H,
                                             float2 *buf, const float2 *tw, int lt, float inv_n,
                                             uint32_t taddr) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  static_assert(P % 8 == 0, "partial sums move 8 points at a time");
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = __ldcs(gy + lt + m * T);
  // this thread's saved-spectrum points into L1 while the transform runs
#pragma unroll
  for (int m = 0; m < P; m += (PL ? 2 : 1))
    asm volatile("prefetch.global.L1 [%0];" ::"l"(xs + out_index<N, P, SC, PL>(lt, m)));
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
  // v[m] = (F g_y)[out_index(lt, m)]; g_z = that / N
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cscale(v[m], inv_n);
  // Chunk c: its sums' tensor-memory read and its X loads are issued
  // together, and chunk c + 1's right after chunk c's store, so the two
  // latencies overlap.
  float r[16];
  float2 x[8];
  // the saved spectrum of registers 8c .. 8c + 7 (adjacent pairs as 16-byte loads)
  auto load_x = [&](int c) {
    if constexpr (PL) {
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const float4 t =
            __ldcs(reinterpret_cast<const float4 *>(xs + out_index<N, P, SC, PL>(lt, 8 * c + q)));
        x[q] = lo2(t);
        x[q + 1] = hi2(t);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = __ldcs(xs + out_index<N, P, SC, PL>(lt, 8 * c + q));
    }
  };
  tmem_ld16(taddr, r);
  load_x(0);
#pragma unroll
  for (int c = 0; c < P / 8; ++c) {
    tmem_wait_ld(r);
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // sum += conj(x) g_z
      const float2 g = v[8 * c + q];
      r[2 * q] = fmaf(x[q].x, g.x, fmaf(x[q].y, g.y, r[2 * q]));
      r[2 * q + 1] = fmaf(x[q].x, g.y, fmaf(-x[q].y, g.x, r[2 * q + 1]));
    }
    tmem_st16(taddr + 16 * c, r);
    if (c + 1 < P / 8) {
      tmem_ld16(taddr + 16 * (c + 1), r);
      load_x(c + 1);
    }
  }
  tmem_wait_st();
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2) {
      const float4 h = __ldg(reinterpret_cast<const float4 *>(H + out_index<N, P, SC, PL>(lt, m)));
      v[m] = cmulc(v[m], lo2(h));
      v[m + 1] = cmulc(v[m + 1], hi2(h));
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cmulc(v[m], __ldg(H + out_index<N, P, SC, PL>(lt, m)));
  }
  __syncthreads();  // every read of the buffer by the transform is done
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2)
      *reinterpret_cast<float4 *>(buf + out_index<N, P, SC, PL>(lt, m)) = pack2(v[m], v[m + 1]);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) buf[out_index<N, P, SC, PL>(lt, m)] = v[m];
  }
}

template <int N, int P, class SC>
__global__ void __launch_bounds__(N / P, (65536 / ((N / P) * 128)) > 0 ? 65536 / ((N / P) * 128) : 1)
filter_bwd2_kernel(FilterBwdArgs a) {
  constexpr int T = N / P;
  constexpr int WARPS = T / 32;
  static_assert(T % 128 == 0, "whole warpgroups cover the tensor-memory lanes");
  constexpr uint32_t NCOL = (WARPS / 4) * 64 < 32 ? 32 : (WARPS / 4) * 64;  // 128 or 256
  extern __shared__ __align__(128) float2 smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + N);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lt = threadIdx.x, warp = lt >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(tslot)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  // lane quarter warp % 4 (the lanes this warp may address), 64 columns per
  // group of four warps
  const uint32_t taddr = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
#pragma unroll
    for (int c = 0; c < P / 8; ++c) tmem_st16(taddr + 16 * c, z);
    tmem_wait_st();
  }
  if (warp == 0 && blockIdx.x < a.batch)  // the first row's saved spectrum into L2
    prefetch_l2_warp(a.xs + (long long)blockIdx.x * N, (long long)sizeof(float2) * N, lt);
  for (long long row = blockIdx.x; row < a.batch; row += gridDim.x) {
    const long long next = row + gridDim.x;
    if (warp == 0 && next < a.batch) {  // the next row's g_y and saved spectrum into L2
      prefetch_l2_warp(a.gy + next * N, (long long)sizeof(float2) * N, lt);
      prefetch_l2_warp(a.xs + next * N, (long long)sizeof(float2) * N, lt);
    }
    filter_half_bwd<N, P, SC>(a.gy + row * N, a.xs + row * N, a.H, smem, a.tw, lt, a.inv_n,
                              taddr);
    __syncthreads();  // conj(H) g_z is in the buffer
    filter_half_inv<N, P, SC>(smem, a.gx + row * N, a.tw, lt, 1, 1.0f);
    __syncthreads();  // the next row rewrites the buffer
  }
  float2 *dst = a.partial + (size_t)blockIdx.x * N;
#pragma unroll
  for (int c = 0; c < P / 8; ++c) {
    float r[16];
    tmem_ld16(taddr + 16 * c, r);
    tmem_wait_ld(r);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[out_index<N, P, SC, pairable<N, P, SC>()>(lt, 8 * c + q)] =
          make_float2(r[2 * q], r[2 * q + 1]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOL));
}

// Fused training step for the masked-energy loss L = sum m |y|^2 (m real,
// one value per point), 32 points per thread, persistent like the backward.
// Per row, four transforms on registers and the exchange buffer:
//   half 1  X = F x; X into tensor memory; X * H into the buffer
//   half 2  y = G (X * H); y stored (optional); L += m |y|^2;
//           g_y = 2 m y into the buffer
//   half 3  g_z = F g_y / N; sum += conj(X) * g_z (the grad_H partial sums,
//           in tensor memory like the backward's); conj(H) * g_z into the buffer
//   half 4  grad_x = F^H (conj(H) * g_z)   (filter_half_inv)
// X never leaves the SM, and neither does g_y: a row reads x and m and writes
// y and grad_x, 28 bytes per point against the 68 of forward, elementwise
// gradient and backward as separate passes.  Tensor memory per CTA: the
// backward's sum columns plus as many for X (256 columns at 8192, two CTAs
// per SM; 512 at 16384, one).
struct FilterStepArgs {
  const float2 *x;
  const float2 *H;
  const float *mask;  // m, [batch][N]
  float2 *y;          // nullable
  float2 *gx;         // grad_x
  float2 *partial;    // [gridDim.x][N] per-CTA grad_H sums
  float *loss_part;   // [gridDim.x] per-CTA loss sums
  const float2 *tw;
  long long batch;
  float inv_n;
};

template <int N, int P, class SC>
__device__ __noinline__ void filter_half_fwd_stash(const float2 *src, const float2 *H, float2 *buf,
                                                   const float2 *tw, int lt, uint32_t taddr_x) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  static_assert(P % 8 == 0, "the spectrum moves to tensor memory 8 points at a time");
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = __ldcs(src + lt + m * T);
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
  // v[m] = X[out_index(lt, m)], the order half 3's transform leaves g_z in
#pragma unroll
  for (int c = 0; c < P / 8; ++c) {
    float r[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      r[2 * q] = v[8 * c + q].x;
      r[2 * q + 1] = v[8 * c + q].y;
    }
    tmem_st16(taddr_x + 16 * c, r);
  }
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2) {
      const float4 h = __ldg(reinterpret_cast<const float4 *>(H + out_index<N, P, SC, PL>(lt, m)));
      v[m] = cmul(v[m], lo2(h));
      v[m + 1] = cmul(v[m + 1], hi2(h));
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cmul(v[m], __ldg(H + out_index<N, P, SC, PL>(lt, m)));
  }
  tmem_wait_st();
  __syncthreads();  // every read of the buffer by the transform is done
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2)
      *reinterpret_cast<float4 *>(buf + out_index<N, P, SC, PL>(lt, m)) = pack2(v[m], v[m + 1]);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) buf[out_index<N, P, SC, PL>(lt, m)] = v[m];
  }
}

// Returns this thread's share of the row's loss.
template <int N, int P, class SC>
__device__ __noinline__ float filter_half_inv_loss(float2 *buf, float2 *y, const float *mask,
                                                   const float2 *tw, int lt, float inv_n) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = buf[lt + m * T];
  __syncthreads();  // every thread has its inputs: the transform may overwrite the buffer
  run_passes<N, P, +1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
  // v[m] * inv_n = y[out_index(lt, m)]
  float loss = 0.f;
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2) {
      const int k = out_index<N, P, SC, PL>(lt, m);
      const float2 a = cscale(v[m], inv_n), b = cscale(v[m + 1], inv_n);
      if (y) __stcs(reinterpret_cast<float4 *>(y + k), pack2(a, b));
      const float2 w = __ldcs(reinterpret_cast<const float2 *>(mask + k));
      loss = fmaf(w.x, fmaf(a.x, a.x, a.y * a.y), loss);
      loss = fmaf(w.y, fmaf(b.x, b.x, b.y * b.y), loss);
      v[m] = cscale(a, 2.f * w.x);
      v[m + 1] = cscale(b, 2.f * w.y);
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int k = out_index<N, P, SC, PL>(lt, m);
      const float2 a = cscale(v[m], inv_n);
      if (y) __stcs(y + k, a);
      const float w = __ldcs(mask + k);
      loss = fmaf(w, fmaf(a.x, a.x, a.y * a.y), loss);
      v[m] = cscale(a, 2.f * w);
    }
  }
  __syncthreads();  // every read of the buffer by the transform is done
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2)
      *reinterpret_cast<float4 *>(buf + out_index<N, P, SC, PL>(lt, m)) = pack2(v[m], v[m + 1]);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) buf[out_index<N, P, SC, PL>(lt, m)] = v[m];
  }
  return loss;
}

template <int N, int P, class SC>
__device__ __noinline__ void filter_half_bwd_buf(float2 *buf, const float2 *H, const float2 *tw,
                                                 int lt, float inv_n, uint32_t taddr,
                                                 uint32_t taddr_x) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = buf[lt + m * T];
  __syncthreads();  // every thread has its inputs: the transform may overwrite the buffer
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1, CtaBarrier, PL>(v, lt, buf, tw, SwizzledRow{});
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cscale(v[m], inv_n);  // g_z
  // chunk c's sums and spectrum are read together, chunk c + 1's right
  // after chunk c's store
  float r[16], xr[16];
  tmem_ld16(taddr, r);
  tmem_ld16(taddr_x, xr);
#pragma unroll
  for (int c = 0; c < P / 8; ++c) {
    tmem_wait_ld(r);
    tmem_wait_ld(xr);
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // sum += conj(X) g_z
      const float2 g = v[8 * c + q];
      const float xx = xr[2 * q], xy = xr[2 * q + 1];
      r[2 * q] = fmaf(xx, g.x, fmaf(xy, g.y, r[2 * q]));
      r[2 * q + 1] = fmaf(xx, g.y, fmaf(-xy, g.x, r[2 * q + 1]));
    }
    tmem_st16(taddr + 16 * c, r);
    if (c + 1 < P / 8) {
      tmem_ld16(taddr + 16 * (c + 1), r);
      tmem_ld16(taddr_x + 16 * (c + 1), xr);
    }
  }
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2) {
      const float4 h = __ldg(reinterpret_cast<const float4 *>(H + out_index<N, P, SC, PL>(lt, m)));
      v[m] = cmulc(v[m], lo2(h));
      v[m + 1] = cmulc(v[m + 1], hi2(h));
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cmulc(v[m], __ldg(H + out_index<N, P, SC, PL>(lt, m)));
  }
  tmem_wait_st();
  __syncthreads();  // every read of the buffer by the transform is done
  if constexpr (PL) {
#pragma unroll
    for (int m = 0; m < P; m += 2)
      *reinterpret_cast<float4 *>(buf + out_index<N, P, SC, PL>(lt, m)) = pack2(v[m], v[m + 1]);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) buf[out_index<N, P, SC, PL>(lt, m)] = v[m];
  }
}

template <int N, int P, class SC>
__global__ void __launch_bounds__(N / P, (65536 / ((N / P) * 128)) > 0 ? 65536 / ((N / P) * 128) : 1)
filter_step_kernel(FilterStepArgs a) {
  constexpr int T = N / P;
  constexpr int WARPS = T / 32;
  static_assert(T % 128 == 0, "whole warpgroups cover the tensor-memory lanes");
  constexpr uint32_t NCOL = (WARPS / 4) * 64;  // the sums; as many again for X
  static_assert(2 * NCOL <= 512, "sums and spectrum fit one SM's tensor memory");
  extern __shared__ __align__(128) float2 smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + N);
  float *red = reinterpret_cast<float *>(smem);  // the loss reduction, after the last row
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lt = threadIdx.x, warp = lt >> 5;
  if (warp == 0) tmem_alloc_warp(tslot, 2 * NCOL);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t taddr = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  const uint32_t taddr_x = taddr + NCOL;
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
#pragma unroll
    for (int c = 0; c < P / 8; ++c) tmem_st16(taddr + 16 * c, z);
    tmem_wait_st();
  }
  float loss = 0.f;
  for (long long row = blockIdx.x; row < a.batch; row += gridDim.x) {
    const long long next = row + gridDim.x;
    if (warp == 0 && next < a.batch) {  // the next row's x and mask into L2
      prefetch_l2_warp(a.x + next * N, (long long)sizeof(float2) * N, lt);
      prefetch_l2_warp(a.mask + next * N, (long long)sizeof(float) * N, lt);
    }
    filter_half_fwd_stash<N, P, SC>(a.x + row * N, a.H, smem, a.tw, lt, taddr_x);
    __syncthreads();  // X * H is in the buffer
    loss += filter_half_inv_loss<N, P, SC>(smem, a.y ? a.y + row * N : nullptr, a.mask + row * N,
                                           a.tw, lt, a.inv_n);
    __syncthreads();  // g_y is in the buffer
    filter_half_bwd_buf<N, P, SC>(smem, a.H, a.tw, lt, a.inv_n, taddr, taddr_x);
    __syncthreads();  // conj(H) g_z is in the buffer
    filter_half_inv<N, P, SC>(smem, a.gx + row * N, a.tw, lt, 1, 1.0f);
    __syncthreads();  // the next row rewrites the buffer
  }
  float2 *dst = a.partial + (size_t)blockIdx.x * N;
#pragma unroll
  for (int c = 0; c < P / 8; ++c) {
    float r[16];
    tmem_ld16(taddr + 16 * c, r);
    tmem_wait_ld(r);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[out_index<N, P, SC, pairable<N, P, SC>()>(lt, 8 * c + q)] =
          make_float2(r[2 * q], r[2 * q + 1]);
  }
  // the CTA's loss: a fixed-order tree over the threads
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if ((lt & 31) == 0) red[warp] = loss;
  tmem_fence_before();
  __syncthreads();
  if (lt == 0) {
    float s = 0.f;
    for (int w = 0; w < WARPS; ++w) s += red[w];
    a.loss_part[blockIdx.x] = s;
  }
  if (warp == 0) tmem_dealloc_warp(tbase, 2 * NCOL);
}

// The training step for 16 points per thread (N <= 4096): TB rows per CTA,
// X and the grad_H sums in tensor memory (32 + 32 columns per thread lane).
// Thread lt holds point lt + m T after every transform, which is what the
// next one reads.  The four transforms inlined into one body spill ~0.5 KiB
// per thread, so, as for 32 points, two separately compiled halves of two
// transforms each meet through the exchange buffer (g_y at lt + m T).  At the
// end the CTA's TB row slots are added in slot order through the buffer, one
// partial row per CTA for the same tree as above.
template <int N, int P, class SC>
__device__ __noinline__ float step_small_front(const float2 *src, int active, const float2 *H,
                                               const float *mk, float2 *yd, float2 *buf,
                                               const float2 *tw, int lt, float inv_n,
                                               uint32_t taddr_x) {
  constexpr int T = N / P;
  static_assert(P == 16, "four 8-column moves of tensor memory per thread");
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = active ? __ldcs(src + lt + m * T) : make_float2(0.f, 0.f);
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1>(v, lt, buf, tw, SwizzledRow{});
  // v[m] = X[lt + m T]: into tensor memory, then X * H
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float r[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      r[2 * q] = v[4 * c + q].x;
      r[2 * q + 1] = v[4 * c + q].y;
    }
    tmem_st8(taddr_x + 8 * c, r);
  }
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cmul(v[m], __ldg(H + lt + m * T));
  tmem_wait_st();
  __syncthreads();  // the forward's last exchange is read
  run_passes<N, P, +1, SC, 0, SwizzledRow, 1>(v, lt, buf, tw, SwizzledRow{});
  // v[m] / N = y[lt + m T]; L += m |y|^2; g_y = 2 m y
  float loss = 0.f;
#pragma unroll
  for (int m = 0; m < P; ++m) {
    const int k = lt + m * T;
    const float2 yv = cscale(v[m], inv_n);
    if (active && yd) __stcs(yd + k, yv);
    const float w = active ? __ldcs(mk + k) : 0.f;
    loss = fmaf(w, fmaf(yv.x, yv.x, yv.y * yv.y), loss);
    v[m] = cscale(yv, 2.f * w);
  }
  __syncthreads();  // the inverse's last exchange is read
#pragma unroll
  for (int m = 0; m < P; ++m) buf[lt + m * T] = v[m];
  return loss;
}

template <int N, int P, class SC>
__device__ __noinline__ void step_small_back(float2 *gd, int active, const float2 *H, float2 *buf,
                                             const float2 *tw, int lt, float inv_n,
                                             uint32_t taddr, uint32_t taddr_x) {
  constexpr int T = N / P;
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = buf[lt + m * T];
  __syncthreads();  // every thread has its g_y: the transform may overwrite the buffer
  run_passes<N, P, -1, SC, 0, SwizzledRow, 1>(v, lt, buf, tw, SwizzledRow{});
  // g_z = v / N; sums += conj(X) g_z, four points (8 columns) at a time
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float r[8], xr[8];
    tmem_ld8(taddr + 8 * c, r);
    tmem_ld8(taddr_x + 8 * c, xr);
    tmem_wait_ld(r);
    tmem_wait_ld(xr);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 g = cscale(v[4 * c + q], inv_n);
      const float xx = xr[2 * q], xy = xr[2 * q + 1];
      r[2 * q] = fmaf(xx, g.x, fmaf(xy, g.y, r[2 * q]));
      r[2 * q + 1] = fmaf(xx, g.y, fmaf(-xy, g.x, r[2 * q + 1]));
      v[4 * c + q] = g;
    }
    tmem_st8(taddr + 8 * c, r);
  }
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cmulc(v[m], __ldg(H + lt + m * T));
  tmem_wait_st();
  __syncthreads();  // the forward's last exchange is read
  run_passes<N, P, +1, SC, 0, SwizzledRow, 1>(v, lt, buf, tw, SwizzledRow{});
  if (active) {
#pragma unroll
    for (int m = 0; m < P; ++m) __stcs(gd + lt + m * T, v[m]);
  }
}

template <int N, int P, int TB, class SC>
__global__ void __launch_bounds__(TB *(N / P), (65536 / (TB * (N / P) * 128)) > 0 ? 65536 / (TB * (N / P) * 128) : 1)
filter_step_small_kernel(FilterStepArgs a) {
  constexpr int T = N / P;
  constexpr int NT = TB * T;
  constexpr int WARPS = NT / 32;
  static_assert(NT % 128 == 0, "whole warpgroups cover the tensor-memory lanes");
  constexpr uint32_t NCOL = (WARPS / 4) * 64 < 32 ? 32 : (WARPS / 4) * 64;
  extern __shared__ __align__(128) float2 smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + TB * N);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = tid / T;
  const int lt = tid - b * T;
  float2 *buf = smem + b * N;
  if (warp == 0) tmem_alloc_warp(tslot, NCOL);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t taddr = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  const uint32_t taddr_x = taddr + 32;
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
    tmem_st16(taddr, z);
    tmem_st16(taddr + 16, z);
    tmem_wait_st();
  }
  float loss = 0.f;
  const long long ntiles = (a.batch + TB - 1) / TB;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    if (warp == 0 && next < ntiles) {  // the next tile's x and mask into L2
      const long long rows = a.batch - next * TB < TB ? a.batch - next * TB : TB;
      prefetch_l2_warp(a.x + next * TB * N, rows * N * (long long)sizeof(float2), tid);
      prefetch_l2_warp(a.mask + next * TB * N, rows * N * (long long)sizeof(float), tid);
    }
    const long long row = tile * TB + b;
    const int active = row < a.batch;
    const long long r0 = active ? row : 0;  // inactive slots compute on zeros, touch nothing
    loss += step_small_front<N, P, SC>(a.x + r0 * N, active, a.H, a.mask + r0 * N,
                                       a.y ? a.y + r0 * N : nullptr, buf, a.tw, lt, a.inv_n,
                                       taddr_x);
    __syncthreads();  // g_y is in the buffer
    step_small_back<N, P, SC>(a.gx + r0 * N, active, a.H, buf, a.tw, lt, a.inv_n, taddr, taddr_x);
    __syncthreads();  // the next tile rewrites the buffer
  }
  // the CTA's grad_H row: its TB row slots added in slot order
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    float r[16];
    tmem_ld16(taddr + 16 * c, r);
    tmem_wait_ld(r);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[lt + (8 * c + q) * T] = make_float2(r[2 * q], r[2 * q + 1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  tmem_fence_before();
  __syncthreads();
  float2 *dst = a.partial + (size_t)blockIdx.x * N;
  for (int k = tid; k < N; k += NT) {
    float2 acc = smem[k];
    for (int t = 1; t < TB; ++t) acc = cadd(acc, smem[t * N + k]);
    dst[k] = acc;
  }
  __syncthreads();  // the slot sums are read: the buffer takes the loss
  float *red = reinterpret_cast<float *>(smem);
  if ((tid & 31) == 0) red[warp] = loss;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < WARPS; ++w) t += red[w];
    a.loss_part[blockIdx.x] = t;
  }
  if (warp == 0) tmem_dealloc_warp(tbase, NCOL);
}

// L = the per-CTA loss sums added in a fixed pairwise order (in FP64).
__global__ void __launch_bounds__(512) loss_tree_kernel(const float *part, int n, float *loss) {
  __shared__ double s[512];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 512) v += (double)part[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = 256; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)s[0];
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
// built-in), 16 below.  With 32 points both transforms inlined into FM_FWD do
// not fit the register budget (~0.8-1 KiB of spills per thread), so from
// 8192 on the forward is filter_fwd2_kernel (the two halves as calls).
struct FilterVariant {
  FilterKernel fwd, spec, mulinv;  // fwd.fn == nullptr: the two-kernel forward
  FilterKernel bwd;                // one-kernel backward (32 points per thread), else nullptr
  FilterKernel step;               // fused training step (32 points per thread), else nullptr
  KernelEntry sched;
};

template <int N, int P, int TB, int... Rs>
static FilterVariant variant() {
  using SC = Sched<Rs...>;
  FilterVariant v;
  if constexpr (P < 32) {
    v.fwd = make_kernel<N, P, TB, SC, FM_FWD>();
  } else {
    v.fwd.fn = (const void *)&filter_fwd2_kernel<N, P, TB, SC>;
    v.fwd.threads = TB * (N / P);
    v.fwd.tb = TB;
    v.fwd.smem = sizeof(float2) * (size_t)N * TB;
    static_assert(P < 32 || TB == 1, "one row per CTA for the persistent backward");
    v.bwd.fn = (const void *)&filter_bwd2_kernel<N, P, SC>;
    v.bwd.threads = N / P;
    v.bwd.tb = 1;
    v.bwd.smem = sizeof(float2) * (size_t)N + 16;  // + the tensor-memory address slot
    v.step.fn = (const void *)&filter_step_kernel<N, P, SC>;
    v.step.threads = N / P;
    v.step.tb = 1;
    v.step.smem = v.bwd.smem;
  }
  if constexpr (P < 32) {
    v.bwd = FilterKernel{nullptr, 0, 0, 0};
    v.step.fn = (const void *)&filter_step_small_kernel<N, P, TB, SC>;
    v.step.threads = TB * (N / P);
    v.step.tb = TB;
    v.step.smem = sizeof(float2) * (size_t)N * TB + 16;  // + the tensor-memory address slot
  }
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
  float2 *d_work = nullptr;  // grad_H workspace: 32-row chunk sums, or one row per CTA of
                             // the one-kernel backward
  int bwd_grid = 0;          // CTAs of the one-kernel backward (resident on the GPU at once)
  int fwd_grid = 0;          // CTAs of the one-kernel forward (32 points per thread)
  int step_grid = 0;         // CTAs of the fused training step (resident at once)
  float *d_loss_part = nullptr;  // per-CTA loss sums of the training step
};

void filter_destroy(fft_plan_impl *pl) {
  FilterState *f = (FilterState *)pl->filter;
  if (f) {
    cudaFree(f->d_work);
    cudaFree(f->d_loss_part);
  }
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
  if (dev_malloc(&pl->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  cudaMemset(pl->d_status, 0, sizeof(int));
  for (const FilterKernel *k : {&v.fwd, &v.spec, &v.mulinv, &v.bwd, &v.step}) {
    if (k->fn && k->smem > 48 * 1024 &&
        cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k->smem) !=
            cudaSuccess)
      return fail(FFT_ERR_CUDA);
  }
  int64_t off = 0;
  fft_status_t s = build_twiddles(pl, pass_segments(v.sched, off));
  if (s != FFT_OK) return fail(s);
  int64_t work = fft_filter_grad_h_workspace(N, batch);
  if (!v.bwd.fn && v.step.fn && batch > 0) {
    // training step of 16-point kernels: resident CTAs as the forward kernel's
    // occupancy allows, capped by tensor memory (64 columns per group of four
    // warps) and by the tiles
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fwd.fn, v.fwd.threads,
                                                      v.fwd.smem) != cudaSuccess ||
        occ < 1)
      return fail(FFT_ERR_CUDA);
    const int tmem_cols = std::max(32, (v.step.threads / 128) * 64);
    const int64_t ntiles = (batch + v.step.tb - 1) / v.step.tb;
    f->step_grid = (int)std::min<int64_t>((int64_t)std::min(occ, 512 / tmem_cols) * sms, ntiles);
    work = std::max<int64_t>(work, (int64_t)f->step_grid * N * (int64_t)sizeof(float2));
    if (dev_malloc(&f->d_loss_part, sizeof(float) * (size_t)f->step_grid) != cudaSuccess) {
      cudaGetLastError();
      return fail(FFT_ERR_ALLOC);
    }
  }
  if (v.bwd.fn && batch > 0) {
    // Resident CTAs per SM: the occupancy query reports one for any kernel
    // that allocates tensor memory, while the hardware co-schedules as many
    // as registers and shared memory allow (measured at 8192: two, 213 vs
    // 270 us).  So take the forward kernel's occupancy (same threads,
    // registers and shared memory) and cap it by the tensor-memory columns:
    // 512 per SM, 64 per group of four warps per CTA.
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fwd.fn, v.fwd.threads,
                                                      v.fwd.smem) != cudaSuccess ||
        occ < 1)
      return fail(FFT_ERR_CUDA);
    f->fwd_grid = (int)std::min<int64_t>((int64_t)occ * sms, batch);
    const int tmem_cols = std::max(32, (v.bwd.threads / 128) * 64);
    f->bwd_grid = (int)std::min<int64_t>((int64_t)std::min(occ, 512 / tmem_cols) * sms, batch);
    // the training step holds twice the columns (the sums and the spectrum)
    f->step_grid =
        (int)std::min<int64_t>((int64_t)std::min(occ, 512 / (2 * tmem_cols)) * sms, batch);
    work = std::max<int64_t>(work, (int64_t)std::max(f->bwd_grid, f->step_grid) * N *
                                       (int64_t)sizeof(float2));
    if (dev_malloc(&f->d_loss_part, sizeof(float) * (size_t)f->step_grid) != cudaSuccess) {
      cudaGetLastError();
      return fail(FFT_ERR_ALLOC);
    }
  }
  if (work > 0 && dev_malloc(&f->d_work, (size_t)work) != cudaSuccess) {
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
  const int64_t bytes = (int64_t)sizeof(float2) * pl->N * pl->batch;
  if (X_save) {  // the saved spectrum may not overlap x or y (header contract)
    const char *p = (const char *)X_save;
    for (const void *o : {x, (const void *)y}) {
      const char *q = (const char *)o;
      if (p < q + bytes && q < p + bytes) return FFT_ERR_INVALID_VALUE;
    }
  }
  if (f->v.fwd.fn && f->fwd_grid > 0) {  // one CTA per row, prefetching a resident wave ahead
    a.ahead = f->fwd_grid;
    return filter_launch(f->v.fwd, a, st);
  }
  if (f->v.fwd.fn) return filter_launch(f->v.fwd, a, st);
  // two kernels: F x into X_save (or y), then y = G (F x * H) from there
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
  if (f->v.bwd.fn) {  // one kernel, then the fixed-order tree over its per-CTA sums
    FilterBwdArgs b{};
    b.gy = (const float2 *)g_y;
    b.xs = (const float2 *)X_saved;
    b.H = (const float2 *)H;
    b.gx = (float2 *)grad_x;
    b.partial = f->d_work;
    b.tw = pl->d_tw;
    b.batch = pl->batch;
    b.inv_n = 1.0f / (float)N;
    void *args[] = {&b};
    if ((s = cuda_status(launch_pdl(f->v.bwd.fn, dim3((unsigned)f->bwd_grid),
                                    dim3(f->v.bwd.threads), f->v.bwd.smem, st, args))) != FFT_OK)
      return s;
    return grad_h_tree(f->d_work, (float2 *)grad_H, N, f->bwd_grid, st);
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

fft_status_t fft_filter_step(fft_plan_t plan, const void *x, const void *H, const float *mask,
                             void *y, void *grad_x, void *grad_H, float *loss, void *stream) {
  fft_status_t s = filter_check(plan, x, H, grad_x);
  if (s != FFT_OK) return s;
  if (!mask || !grad_H || !loss) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)mask | (uintptr_t)y | (uintptr_t)grad_H) & 15 || ((uintptr_t)loss & 3))
    return FFT_ERR_MISALIGNED;
  fft_plan_impl *pl = &plan->impl;
  FilterState *f = (FilterState *)pl->filter;
  if (!f->v.step.fn) return FFT_ERR_NOT_SUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = pl->N;
  if (pl->batch == 0) {
    if ((s = cuda_status(cudaMemsetAsync(grad_H, 0, sizeof(float2) * N, st))) != FFT_OK) return s;
    return cuda_status(cudaMemsetAsync(loss, 0, sizeof(float), st));
  }
  const int64_t bytes = (int64_t)sizeof(float2) * N * pl->batch;
  auto overlap = [](const void *p, int64_t pb, const void *q, int64_t qb) {
    const char *a = (const char *)p, *b = (const char *)q;
    return a < b + qb && b < a + pb;
  };
  // Outputs: y and grad_x may each be x itself (a CTA reads its row before it
  // writes it) but overlap nothing else; the mask, H, grad_H and the loss
  // overlap no output.
  for (const void *o : {(const void *)y, (const void *)grad_x}) {
    if (!o) continue;
    if (o != x && overlap(o, bytes, x, bytes)) return FFT_ERR_INVALID_VALUE;
    if (overlap(o, bytes, mask, bytes / 2) || overlap(o, bytes, H, sizeof(float2) * N) ||
        overlap(o, bytes, grad_H, sizeof(float2) * N) || overlap(o, bytes, loss, sizeof(float)))
      return FFT_ERR_INVALID_VALUE;
  }
  if (y && overlap(y, bytes, grad_x, bytes)) return FFT_ERR_INVALID_VALUE;
  FilterStepArgs a{};
  a.x = (const float2 *)x;
  a.H = (const float2 *)H;
  a.mask = mask;
  a.y = (float2 *)y;
  a.gx = (float2 *)grad_x;
  a.partial = f->d_work;
  a.loss_part = f->d_loss_part;
  a.tw = pl->d_tw;
  a.batch = pl->batch;
  a.inv_n = 1.0f / (float)N;
  void *args[] = {&a};
  if ((s = cuda_status(launch_pdl(f->v.step.fn, dim3((unsigned)f->step_grid),
                                  dim3(f->v.step.threads), f->v.step.smem, st, args))) != FFT_OK)
    return s;
  if ((s = grad_h_tree(f->d_work, (float2 *)grad_H, N, f->step_grid, st)) != FFT_OK) return s;
  loss_tree_kernel<<<1, 512, 0, st>>>(f->d_loss_part, f->step_grid, loss);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
