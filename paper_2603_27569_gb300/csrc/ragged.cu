// Ragged batches: many transforms of mixed lengths and directions in ONE
// persistent launch (paper Sec. II-D: radar workloads are batches of 1-D FFTs
// of 2^10..2^14 points; here a batch may mix them).
//
// Two launches.  Work is cut into units, longest first (LPT order); the
// large rows are claimed through device counters by a persistent grid (one
// CTA per SM, 128 KiB of shared memory), the small units each get a CTA:
//   launch 1, 512-thread CTAs, 32 points per thread (the plain transform's
//   built-in schedules for these sizes; 512 threads leave the 128 registers
//   per thread they need):
//     class A  N = 16384: one row per unit, the whole CTA (barrier: CTA);
//     class B  N = 8192:  one row per unit, each half of the CTA (256
//                         threads, 64 KiB) claims its own units (named
//                         barrier per half);
//   launch 2, one 256-thread CTA (32 KiB) per unit, 16 points per thread
//   (radix-16 passes with a radix-2/4/8 tail):
//     class C  N <= 4096: 4096 points per unit (4096 / N rows of one (N,
//                         direction)), units in longest-first order; a CTA
//                         behaves like one 256-thread CTA of the plain
//                         kernel (a persistent grid of claiming CTAs measured
//                         slower: its CTAs run in lockstep).
// In launch 1 a CTA moves A -> B once, never back, so no class waits for
// another.
//
// The counter reset and the kernel are captured once per (in, out) pair into
// a CUDA graph that each fft_exec replays on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.h"
#include "stockham.cuh"

namespace fftgb {

struct RaggedDesc {
  long long in_off, out_off;  // complex elements from the packed bases
};
struct RaggedUnit {
  int first;  // first descriptor of the unit
  int count;  // rows in the unit
  int log2n;
  int dir;
};

constexpr int kRagMinLog2 = 4, kRagMaxLog2 = 14;
constexpr int kRagSizes = kRagMaxLog2 - kRagMinLog2 + 1;
constexpr size_t kRagSmem = sizeof(float2) * 16384;

struct RaggedArgs {
  const float2 *in;
  float2 *out;
  const RaggedDesc *desc;
  const RaggedUnit *units;
  int nA, nB, nC;     // units per class; class B starts at nA, class C at nA + nB
  unsigned *counters; // [3], zero at launch
  const float2 *tw;   // per-size pass tables, concatenated
  long long tw_off[kRagSizes];
  int unnormalized;   // inverse without 1/N
};

// Radix schedules (P points per thread, twiddle mode TWM).  rag_radices()
// below lists the same schedules for the host's twiddle tables.
template <int N> struct RagSched { static constexpr int P = 16, TWM = 0; };
template <> struct RagSched<16> : RagSched<0> { using T = Sched<16>; };
template <> struct RagSched<32> : RagSched<0> { using T = Sched<16, 2>; };
template <> struct RagSched<64> : RagSched<0> { using T = Sched<16, 4>; };
template <> struct RagSched<128> : RagSched<0> { using T = Sched<16, 8>; };
template <> struct RagSched<256> : RagSched<0> { using T = Sched<16, 16>; };
template <> struct RagSched<512> : RagSched<0> { using T = Sched<16, 16, 2>; };
template <> struct RagSched<1024> : RagSched<0> { using T = Sched<16, 16, 4>; };
template <> struct RagSched<2048> : RagSched<0> { using T = Sched<16, 16, 8>; };
template <> struct RagSched<4096> : RagSched<0> { using T = Sched<16, 16, 16>; };
template <> struct RagSched<8192> {
  using T = Sched<32, 16, 16>;
  static constexpr int P = 32, TWM = 0;
};
template <> struct RagSched<16384> {
  using T = Sched<32, 32, 16>;
  static constexpr int P = 32, TWM = 1;
};

// Radices of the schedule for N = 2^e (host copy of RagSched); returns the
// number of passes.
static int rag_radices(int e, int *rad) {
  if (e == 14) {
    rad[0] = 32, rad[1] = 32, rad[2] = 16;
    return 3;
  }
  if (e == 13) {
    rad[0] = 32, rad[1] = 16, rad[2] = 16;
    return 3;
  }
  int np = 0, rest = 1 << e;
  while (rest > 1) {
    const int rr = rest >= 16 ? 16 : rest;
    rad[np++] = rr;
    rest /= rr;
  }
  return np;
}

// One unit by a group of GT threads (gtid = thread index in the group).
template <int N, int D, int GT, class BR>
__device__ __forceinline__ void rag_unit(const RaggedArgs &a, const RaggedUnit &u, int gtid,
                                         float2 *sm, const BR &br) {
  using SC = typename RagSched<N>::T;
  constexpr int P = RagSched<N>::P;
  constexpr int T = N / P;
  static_assert(GT % T == 0, "group must hold whole rows");
  const int b = gtid / T;
  const int lt = gtid - b * T;
  const bool active = b < u.count;
  float2 v[P];
  RaggedDesc d{0, 0};
  if (active) {
    d = a.desc[u.first + b];
    const float2 *src = a.in + d.in_off;
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = __ldcs(src + lt + m * T);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
  }
  const float2 *tw = a.tw + a.tw_off[ilog2(N) - kRagMinLog2];
  run_passes<N, P, D, SC, 0, SwizzledRow, RagSched<N>::TWM, BR>(v, lt, sm + (size_t)b * N, tw,
                                                                 SwizzledRow{}, br);
  if (active) {
    const float s = (D > 0 && !a.unnormalized) ? 1.0f / (float)N : 1.0f;
    float2 *dst = a.out + d.out_off;
#pragma unroll
    for (int m = 0; m < P; ++m) __stcs(dst + final_index<N, P, SC>(lt, m), cscale(v[m], s));
  }
  br.sync();  // the group's buffer is reused by its next unit
}

// Sizes by class: LARGE (launch 1): 8192 on 256-thread halves, 16384 on the
// 512-thread CTA; otherwise (launch 2) N <= 4096 on 256-thread quarters.
template <int GT, bool LARGE, class BR>
__device__ void rag_dispatch(const RaggedArgs &a, const RaggedUnit &u, int gtid, float2 *sm,
                             const BR &br) {
#define FFTGB_RAG_CASE(L)                                                        \
  case L:                                                                        \
    if (u.dir < 0) rag_unit<(1 << L), -1, GT, BR>(a, u, gtid, sm, br);           \
    else rag_unit<(1 << L), +1, GT, BR>(a, u, gtid, sm, br);                     \
    break;
  if constexpr (!LARGE) {
    switch (u.log2n) {
      FFTGB_RAG_CASE(4)
      FFTGB_RAG_CASE(5)
      FFTGB_RAG_CASE(6)
      FFTGB_RAG_CASE(7)
      FFTGB_RAG_CASE(8)
      FFTGB_RAG_CASE(9)
      FFTGB_RAG_CASE(10)
      FFTGB_RAG_CASE(11)
      FFTGB_RAG_CASE(12)
      default: break;
    }
  } else if constexpr (GT == 256) {
    switch (u.log2n) {
      FFTGB_RAG_CASE(13)
      default: break;
    }
  } else {
    switch (u.log2n) {
      FFTGB_RAG_CASE(14)
      default: break;
    }
  }
#undef FFTGB_RAG_CASE
}

// Launch 1: classes A (whole 512-thread CTA) and B (256-thread halves).
__global__ void __launch_bounds__(512, 1) ragged_large_kernel(RaggedArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ int claim[3];
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) claim[0] = (int)atomicAdd(a.counters + 0, 1u);
    __syncthreads();
    const int u = claim[0];
    __syncthreads();
    if (u >= a.nA) break;
    rag_dispatch<512, true>(a, a.units[u], tid, smem, CtaBarrier{});
  }
  const int h = tid / 256, htid = tid - h * 256;
  const NamedBarrier br{1 + h, 256};
  float2 *sm = smem + (size_t)h * 8192;
  while (true) {
    if (htid == 0) claim[1 + h] = (int)atomicAdd(a.counters + 1, 1u);
    br.sync();
    const int u = claim[1 + h];
    br.sync();
    if (u >= a.nB) break;
    rag_dispatch<256, true>(a, a.units[a.nA + u], htid, sm, br);
  }
}

// Launch 2: class C, one 256-thread CTA (32 KiB) per unit, in the units'
// longest-first order; the hardware scheduler keeps several units per SM
// in flight and staggers their phases.
__global__ void __launch_bounds__(256) ragged_small_kernel(RaggedArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  rag_dispatch<256, false>(a, a.units[a.nA + a.nB + blockIdx.x], threadIdx.x, smem, CtaBarrier{});
}

// FP64-generated pass tables (api.cu).
__global__ void gen_pass_twiddles(float2 *out, int p, int r);

struct RaggedState {
  int count = 0;
  int64_t max_in = 0, max_out = 0;  // elements each packed buffer must hold
  RaggedDesc *d_desc = nullptr;
  RaggedUnit *d_units = nullptr;
  unsigned *d_counters = nullptr;
  float2 *d_tw = nullptr;
  RaggedArgs args{};
  int grid = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void *g_in = nullptr;
  void *g_out = nullptr;
};

static void ragged_free(RaggedState *r) {
  if (!r) return;
  if (r->graph) cudaGraphExecDestroy(r->graph);
  if (r->cap) cudaStreamDestroy(r->cap);
  cudaFree(r->d_desc);
  cudaFree(r->d_units);
  cudaFree(r->d_counters);
  cudaFree(r->d_tw);
  delete r;
}

void ragged_destroy(fft_plan_impl *pl) {
  ragged_free(pl->ragged);
  pl->ragged = nullptr;
}

static fft_status_t capture(RaggedState *r, const float2 *in, float2 *out) {
  if (r->graph) {
    cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
  }
  r->args.in = in;
  r->args.out = out;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return FFT_ERR_CUDA;
  cudaMemsetAsync(r->d_counters, 0, 3 * sizeof(unsigned), r->cap);
  RaggedArgs a = r->args;
  void *args[] = {&a};
  if (a.nA + a.nB > 0)
    cudaLaunchKernel((const void *)ragged_large_kernel, dim3(r->grid), dim3(512), args, kRagSmem,
                     r->cap);
  if (a.nC > 0)
    cudaLaunchKernel((const void *)ragged_small_kernel, dim3((unsigned)a.nC), dim3(256), args,
                     sizeof(float2) * 4096, r->cap);
  if (cudaStreamEndCapture(r->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return FFT_ERR_CUDA;
  }
  cudaError_t e = cudaGraphInstantiate(&r->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    r->graph = nullptr;
    return FFT_ERR_CUDA;
  }
  r->g_in = in;
  r->g_out = out;
  return FFT_OK;
}

fft_status_t ragged_exec(fft_plan_impl *pl, const float2 *in, float2 *out, cudaStream_t st) {
  RaggedState *r = pl->ragged;
  if (!r) return FFT_ERR_INVALID_VALUE;
  if (r->count == 0) return FFT_OK;
  if (r->g_in != in || r->g_out != out || !r->graph) {
    fft_status_t s = capture(r, in, out);
    if (s != FFT_OK) return s;
  }
  return cuda_status(cudaGraphLaunch(r->graph, st));
}

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status_t fft_ragged_plan(fft_plan_t *out, int count, const int *N,
                                        const int *direction, const int64_t *in_offset,
                                        const int64_t *out_offset, int flags) {
  if (!out) return FFT_ERR_INVALID_VALUE;
  *out = nullptr;
  if (count < 0) return FFT_ERR_INVALID_SIZE;
  if (count > 0 && (!N || !direction || !in_offset || !out_offset)) return FFT_ERR_INVALID_VALUE;
  if (flags & ~(FFT_FLAG_UNNORMALIZED_INVERSE | FFT_FLAG_NO_AUTOTUNE_CACHE))
    return FFT_ERR_INVALID_VALUE;
  for (int i = 0; i < count; ++i) {
    const int n = N[i];
    if (n < 2 || n > 16384 || (n & (n - 1))) return FFT_ERR_INVALID_SIZE;
    if (n < (1 << kRagMinLog2)) return FFT_ERR_NOT_SUPPORTED;
    if (direction[i] != FFT_FORWARD && direction[i] != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
    if (in_offset[i] < 0 || out_offset[i] < 0) return FFT_ERR_INVALID_VALUE;
    if ((in_offset[i] & 1) || (out_offset[i] & 1)) return FFT_ERR_MISALIGNED;
  }
  fft_plan_s *h = new (std::nothrow) fft_plan_s;
  RaggedState *r = new (std::nothrow) RaggedState;
  if (!h || !r) {
    delete h;
    delete r;
    return FFT_ERR_ALLOC;
  }
  fft_plan_impl *pl = &h->impl;
  pl->path = FFT_PATH_RAGGED;
  pl->batch = count;
  pl->flags = flags;
  pl->ragged = r;
  r->count = count;
  cudaGetDevice(&pl->device);
  auto fail = [&](fft_status_t e) {
    ragged_free(r);
    pl->ragged = nullptr;
    delete h;
    return e;
  };
  if (cudaMalloc(&pl->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  cudaMemset(pl->d_status, 0, sizeof(int));
  // Order: class A (16384), class B (8192), class C by N descending; within a
  // size, forward before inverse; rows of one (N, direction) keep draw order.
  std::vector<int> idx(count);
  for (int i = 0; i < count; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    if (N[x] != N[y]) return N[x] > N[y];
    return direction[x] < direction[y];
  });
  std::vector<RaggedDesc> desc(count);
  std::vector<RaggedUnit> units;
  int nA = 0, nB = 0, nC = 0;
  for (int i = 0; i < count;) {
    const int n = N[idx[i]], d = direction[idx[i]];
    const int per = n >= 8192 ? 1 : 4096 / n;  // rows per unit
    int j = i;
    while (j < count && j - i < per && N[idx[j]] == n && direction[idx[j]] == d) ++j;
    RaggedUnit u;
    u.first = i;
    u.count = j - i;
    u.log2n = __builtin_ctz((unsigned)n);
    u.dir = d;
    units.push_back(u);
    (n == 16384 ? nA : n == 8192 ? nB : nC)++;
    i = j;
  }
  for (int i = 0; i < count; ++i) {
    desc[i].in_off = in_offset[idx[i]];
    desc[i].out_off = out_offset[idx[i]];
    r->max_in = std::max<int64_t>(r->max_in, in_offset[idx[i]] + N[idx[i]]);
    r->max_out = std::max<int64_t>(r->max_out, out_offset[idx[i]] + N[idx[i]]);
  }
  // Twiddle tables for every size the kernel may meet.
  std::vector<int64_t> tw_off(kRagSizes, 0);
  std::vector<std::pair<int, int>> passes;  // (p, r) in table order
  int64_t total = 0;
  for (int e = kRagMinLog2; e <= kRagMaxLog2; ++e) {
    tw_off[e - kRagMinLog2] = total;
    int rad[8] = {0};
    const int np = rag_radices(e, rad);
    int p = rad[0];
    for (int k = 1; k < np; ++k) {
      passes.push_back({p, rad[k]});
      total += (int64_t)(rad[k] - 1) * p;
      p *= rad[k];
    }
  }
  const size_t ub = sizeof(RaggedUnit) * std::max<size_t>(1, units.size());
  if (cudaMalloc(&r->d_desc, sizeof(RaggedDesc) * std::max(1, count)) != cudaSuccess ||
      cudaMalloc(&r->d_units, ub) != cudaSuccess ||
      cudaMalloc(&r->d_counters, 3 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&r->d_tw, sizeof(float2) * std::max<int64_t>(1, total)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FFT_ERR_ALLOC);
  }
  if (count > 0 &&
      (cudaMemcpy(r->d_desc, desc.data(), sizeof(RaggedDesc) * count, cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemcpy(r->d_units, units.data(), sizeof(RaggedUnit) * units.size(),
                  cudaMemcpyHostToDevice) != cudaSuccess))
    return fail(FFT_ERR_CUDA);
  {
    int64_t off = 0;
    for (auto &pr : passes) {
      const int64_t n = (int64_t)(pr.second - 1) * pr.first;
      gen_pass_twiddles<<<(unsigned)((n + 255) / 256), 256>>>(r->d_tw + off, pr.first, pr.second);
      off += n;
    }
  }
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return fail(FFT_ERR_CUDA);
  if (cudaFuncSetAttribute((const void *)ragged_large_kernel,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRagSmem) !=
      cudaSuccess)
    return fail(FFT_ERR_CUDA);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
  r->grid = std::max(1, std::min<int>(sms, (int)units.size()));
  if (cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FFT_ERR_CUDA);
  RaggedArgs &a = r->args;
  a.desc = r->d_desc;
  a.units = r->d_units;
  a.nA = nA;
  a.nB = nB;
  a.nC = nC;
  a.counters = r->d_counters;
  a.tw = r->d_tw;
  for (int i = 0; i < kRagSizes; ++i) a.tw_off[i] = tw_off[i];
  a.unnormalized = (flags & FFT_FLAG_UNNORMALIZED_INVERSE) ? 1 : 0;
  *out = h;
  return FFT_OK;
}
