// TMA-staged persistent Stockham kernel for long rows (N = 8192, 16384).
//
// At these sizes one row fills half of an SM's register file, so only one
// row per SM can be in flight and its global loads cannot hide behind other
// CTAs.  This kernel hides them inside the CTA instead: the bulk-copy (TMA)
// engine streams the NEXT row of this CTA into shared memory while the
// current row is computed.
//
// The input row is split into P slabs of T = N / P points: slab m holds the
// points {lt + m T : lt < T}, i.e. exactly register m of every thread in
// pass 0 (Sec. V-A's device-memory bypass, re-routed through the TMA).  A
// ring of C slabs (C <= P) sits beside the exchange buffer E.  Slabs 0..C-1
// of the next row are issued into the ring as soon as pass 0 of the current
// row has consumed it; slabs C..P-1 are issued into E as soon as the last
// exchange of the current row has been read out of E.  Each ring slot and E
// complete on their own mbarrier (transaction-count based), once per row, so
// the phase parity of every wait is the row's iteration count & 1.
//
// Every wait is bounded in time (%globaltimer): a wait that runs out makes
// the whole CTA stop (the decision is made CTA-uniform with
// __syncthreads_and), records FFT_ERR_TIMEOUT in the status word, and the
// issuing thread gives the copies it still has in flight a bounded time to
// land before the CTA exits.
#pragma once
#include <stdint.h>

#include "stockham.cuh"

namespace fftgb {

struct StagedArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;
  long long batch;
  float scale;
  int *status;  // device status word (FFT_ERR_TIMEOUT on a wait that ran out)
};

constexpr unsigned long long kWaitNs = 2000000000ull;    // 2 s: a lost copy
constexpr unsigned long long kDrainNs = 200000000ull;    // 0.2 s per barrier on exit

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// True once the phase with parity `parity` has completed; false if it did
// not within limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitNs) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(a, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 1-D bulk copy global -> shared, completing on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a CTA barrier) before its later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory footprint of the staged kernel: exchange buffer + C slabs +
// (C + 1) mbarriers.
template <int N, int P, int C>
__host__ __device__ constexpr size_t staged_smem_bytes() {
  return sizeof(float2) * (size_t)N + sizeof(float2) * (size_t)C * (N / P) + 8 * (C + 1);
}

template <int N, int P, int C, int D, class SC, int TWM>
__global__ void __launch_bounds__(N / P)
staged_kernel(StagedArgs args) {
  static_assert(SC::product() == N, "radix schedule must multiply to N");
  static_assert(P % SC::max_radix() == 0, "every radix must divide P");
  static_assert(C >= 1 && C <= P, "ring holds 1..P slabs");
  constexpr int T = N / P;
  constexpr unsigned kSlab = sizeof(float2) * T;  // bytes per slab
  static_assert(kSlab % 16 == 0, "slab must be a multiple of 16 bytes");
  static_assert((P - C) * T <= N, "the slabs beyond the ring must fit in E");
  extern __shared__ __align__(128) float2 smem[];
  float2 *E = smem;                          // exchange buffer, N points
  float2 *ring = smem + N;                   // C slabs of T points
  uint64_t *bars = reinterpret_cast<uint64_t *>(ring + (size_t)C * T);  // C ring + 1 for E
  uint64_t *barE = bars + C;
  const int lt = threadIdx.x;
  const long long G = gridDim.x;
  const long long first = blockIdx.x;
  if (first >= args.batch) return;
  const long long iters = (args.batch - first + G - 1) / G;  // rows this CTA owns

  if (lt == 0) {
    for (int c = 0; c <= C; ++c) mbar_init(bars + c, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Issue the loads of row `it` (this CTA's it-th row): ring part or E part.
  auto issue_ring = [&](long long it) {
    const float2 *src = args.in + (first + it * G) * (long long)N;
    for (int m = 0; m < C; ++m) {
      mbar_expect_tx(bars + m, kSlab);
      tma_load_1d(ring + (size_t)m * T, src + (size_t)m * T, kSlab, bars + m);
    }
  };
  auto issue_E = [&](long long it) {
    if constexpr (C < P) {
      const float2 *src = args.in + (first + it * G) * (long long)N;
      mbar_expect_tx(barE, kSlab * (P - C));
      for (int m = C; m < P; ++m)
        tma_load_1d(E + (size_t)(m - C) * T, src + (size_t)m * T, kSlab, barE);
    }
  };
  if (lt == 0) {
    issue_ring(0);
    issue_E(0);
  }

  bool ok = true;
  unsigned fail_par = 0;
  for (long long it = 0; it < iters && ok; ++it) {
    const unsigned par = (unsigned)(it & 1);
    fail_par = par;
    const long long row = first + it * G;
    float2 a[P];
    // pass 0 reads: register m <- slab m
#pragma unroll
    for (int m = 0; m < P; ++m) {
      if (m < C) {
        ok = ok && mbar_wait(bars + m, par);
        a[m] = ring[(size_t)m * T + lt];
      } else {
        if (m == C) ok = ok && mbar_wait(barE, par);
        a[m] = E[(size_t)(m - C) * T + lt];
      }
    }
    ok = __syncthreads_and(ok);  // ring and E fully read: free for the next row
    if (!ok) break;
    if (lt == 0 && it + 1 < iters) {
      fence_proxy_async();
      issue_ring(it + 1);
    }
    const float2 *twp = args.tw;
    int ltp = lt;
    asm volatile("" : "+l"(twp), "+r"(ltp));
    run_passes<N, P, D, SC, 0, SwizzledRow, TWM>(a, ltp, E, twp, SwizzledRow{});
    // the last exchange has been read out of E by every thread
    __syncthreads();
    if (lt == 0 && it + 1 < iters) {
      fence_proxy_async();
      issue_E(it + 1);
    }
    float2 *dst = args.out + row * N;
    const float s = args.scale;
#pragma unroll
    for (int m = 0; m < P; ++m) __stcs(dst + final_index<N, P, SC>(ltp, m), cscale(a[m], s));
  }
  if (!ok && lt == 0) {
    if (args.status) atomicCAS(args.status, 0, 6 /* FFT_ERR_TIMEOUT */);
    // The failed row's copies (its ring slots and its E part, phase
    // `fail_par`) may still be in flight: give each a bounded time to land
    // before the CTA's shared memory is released.
    for (int c = 0; c < C; ++c) (void)mbar_wait(bars + c, fail_par, kDrainNs);
    if (C < P) (void)mbar_wait(barE, fail_par, kDrainNs);
  }
}

}  // namespace fftgb
