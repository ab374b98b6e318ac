// One-pass transforms of N = 2 H points (H = 16384: N = 32768) on one SM, one
// half of the row held in tensor memory (paper Sec. IV-D, synthesis rule 3:
// a transform longer than one threadgroup's memory; here the SM's 256 KiB of
// tensor memory holds half the row, so the row crosses HBM once each way
// instead of twice as in the four-step).
//
// A radix-2 decimation-in-frequency step splits the row into two H-point
// transforms (the textbook DIF identity, forward sign; the inverse conjugates
// the roots and scales by 1/N at the store):
//   X[2k]     = sum_n (x[n] + x[n + H]) W_H^{n k}
//   X[2k + 1] = sum_n ((x[n] - x[n + H]) W_N^n) W_H^{n k}     (0 <= n, k < H)
// Thread t of the CTA (T = H / P threads) owns points n = t + m T, m < P, of
// both halves: exactly its pass-0 inputs of the H-point Stockham transform, so
// the split needs no exchange.  Per row, two rounds of one loop body (so the
// transform's code and registers exist once):
//   round 0: the split (first half from registers, loaded during the previous
//            row's epilogue; second half from the exchange buffer, where the
//            bulk-copy engine put it while the previous row stored its
//            outputs) keeps the sums in registers and sends the twiddled
//            differences (W_N^n = W_N^t W_64^m: a per-thread table entry times
//            a compile-time root) to tensor-memory region D; the H-point
//            transform of the sums (the passes of the 16384-point kernel, its
//            exchange buffer and tables) gives X[2k], which goes to region E;
//   round 1: the differences come back from D; their transform gives
//            X[2k + 1]; the epilogue reads X[2k] back from E, stores X[2k],
//            X[2k + 1] as adjacent pairs (16-byte stores) and refills the
//            registers with the next row's first half.
// The second-half copy completes on an mbarrier whose wait is bounded in time
// (%globaltimer, as in the TMA-staged kernel): a wait that runs out stops
// the CTA, records FFT_ERR_TIMEOUT and lets the copy in flight land first.
// Each thread reads and writes only its own tensor-memory lane and columns
// (warp w: lanes 32 (w % 4) .., columns 64 (w / 4) .. in each region), so
// tensor memory needs no barrier; the thread waits for its own stores before
// reading back.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "staged.cuh"
#include "stockham.cuh"
#include "tmem.cuh"

namespace fftgb {

struct Tmem2Args {
  const float2 *in;
  float2 *out;
  const float2 *tw;    // pass tables of the H-point schedule
  const float2 *tw_n;  // W_N^t for the T threads (the split's per-thread root)
  long long batch;
  float scale;         // applied at the final store (1 or 1/N)
  int *status;         // device status word (FFT_ERR_TIMEOUT on a wait that ran out)
  int out32;           // out is 32-byte aligned: the epilogue's 32-byte stores are allowed
};

// One 32-byte streaming store (st.global.v8, sm_100+): p 32-byte aligned.
__device__ __forceinline__ void st_cs_v8(float2 *p, float2 a, float2 b, float2 c, float2 d) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x),
               "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
               : "memory");
}

// Shared memory: the H-point exchange buffer, then the tensor-memory address
// slot and the mbarrier of the second-half copy.
template <int N>
__host__ __device__ constexpr size_t tmem2_smem_bytes() {
  return sizeof(float2) * (size_t)(N / 2) + 16;
}

// cos(k pi / 32), k = 0..16, in FP64 (rounded once to FP32 where used).
struct Cos32d {
  static constexpr double d[17] = {1.0,
                                   0.995184726672196886245,
                                   0.980785280403230449126,
                                   0.956940335732208864936,
                                   0.923879532511286756128,
                                   0.881921264348355029713,
                                   0.831469612302545237079,
                                   0.773010453362736960811,
                                   0.707106781186547524401,
                                   0.634393284163645498215,
                                   0.555570233019602224743,
                                   0.471396736825997648556,
                                   0.382683432365089771728,
                                   0.290284677254462367636,
                                   0.195090322016128267848,
                                   0.098017140329560601994,
                                   0.0};
};

// v * W_64^M (D = -1) or v * conj(W_64^M) (D = +1), 0 <= M < 32.
template <int M, int D>
__device__ __forceinline__ float2 rot64(float2 v) {
  if constexpr (M == 0) {
    return v;
  } else if constexpr (M == 16) {
    return rot90<D>(v);
  } else {
    constexpr double c = M <= 16 ? Cos32d::d[M] : -Cos32d::d[32 - M];
    constexpr double s0 = Cos32d::d[M <= 16 ? 16 - M : M - 16];  // sin(M pi / 32) >= 0
    constexpr float cf = (float)c, sf = (float)(D < 0 ? -s0 : s0);
    // Scalar FMAs with the roots as immediate operands: packed FMAs would
    // take them from register pairs, and the compiler keeps loop-invariant
    // constants live across the whole row loop (31 roots, 62 registers).
    return make_float2(fmaf(v.x, cf, -(v.y * sf)), fmaf(v.x, sf, v.y * cf));
  }
}

// The split for registers M .. E - 1 (one 8-column chunk: E - M = 4): a[m]
// keeps x[n] + x[n + H]; (x[n] - x[n + H]) W_N^n goes to r.
template <int D, int M, int E, int P>
struct Tmem2Split {
  static __device__ __forceinline__ void run(float2 (&a)[P], const float2 (&b)[4], float (&r)[8],
                                             float2 wt) {
    constexpr int q = M & 3;
    const float2 x0 = a[M];
    a[M] = cadd(x0, b[q]);
    const float2 d = cmul_dir<D>(rot64<M, D>(csub(x0, b[q])), wt);
    r[2 * q] = d.x;
    r[2 * q + 1] = d.y;
    if constexpr (M + 1 < E) Tmem2Split<D, M + 1, E, P>::run(a, b, r, wt);
  }
};

template <int N, int P, int D, int C>
__device__ __forceinline__ void tmem2_split_chunk(float2 (&a)[P], const float2 *hi, int lt,
                                                  uint32_t taddr, float2 wt) {
  constexpr int T = N / 2 / P;
  float2 b[4];
  float r[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = hi[lt + (4 * C + q) * T];
  Tmem2Split<D, 4 * C, 4 * C + 4, P>::run(a, b, r, wt);
  tmem_st8(taddr + 8 * C, r);
  if constexpr (4 * C + 4 < P) tmem2_split_chunk<N, P, D, C + 1>(a, hi, lt, taddr, wt);
}

// Round 1's input: registers 8C .. 8C + 7 from tensor memory.
template <int P, int C>
__device__ __forceinline__ void tmem2_load_chunk(float2 (&a)[P], uint32_t taddr) {
  float r[16];
  tmem_ld16(taddr + 16 * C, r);
  tmem_wait_ld(r);
#pragma unroll
  for (int q = 0; q < 8; ++q) a[8 * C + q] = make_float2(r[2 * q], r[2 * q + 1]);
  if constexpr (8 * C + 8 < P) tmem2_load_chunk<P, C + 1>(a, taddr);
}
// Round 0's output: registers 8C .. 8C + 7 to tensor memory.
template <int P, int C>
__device__ __forceinline__ void tmem2_park_chunk(const float2 (&a)[P], uint32_t taddr) {
  float e[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    e[2 * q] = a[8 * C + q].x;
    e[2 * q + 1] = a[8 * C + q].y;
  }
  tmem_st16(taddr + 16 * C, e);
  if constexpr (8 * C + 8 < P) tmem2_park_chunk<P, C + 1>(a, taddr);
}

// The epilogue for one chunk (registers 4C .. 4C + 3 hold X[2k + 1], tensor
// memory the matching X[2k]).
template <int N, int P, class SC, bool PAIR_LAST, bool OUT32, int C>
__device__ __forceinline__ void tmem2_store_chunk(float2 (&a)[P], int lt, uint32_t taddr,
                                                  float2 *dst, const float2 *nsrc, bool load_next,
                                                  float s) {
  constexpr int H = N / 2, T = H / P;
  float r[8];
  tmem_ld8(taddr + 8 * C, r);
  tmem_wait_ld(r);
  if constexpr (PAIR_LAST) {
    // pair (2j, 2j + 1) holds outputs k, k + 1 of the half transforms
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int j = 2 * C + jj;
      const int k = final_index_pair<H, P, SC>(lt, j);
      const float2 e0 = cscale(make_float2(r[4 * jj], r[4 * jj + 1]), s);
      const float2 e1 = cscale(make_float2(r[4 * jj + 2], r[4 * jj + 3]), s);
      const float2 o0 = cscale(a[2 * j], s), o1 = cscale(a[2 * j + 1], s);
      // X[2k .. 2k + 3]: 32 contiguous bytes per thread, so a warp's one
      // 32-byte store fills whole sectors (two 16-byte stores would each
      // write half of every sector they touch)
      if constexpr (OUT32) {
        st_cs_v8(dst + 2 * k, e0, o0, e1, o1);
      } else {
        __stcs(reinterpret_cast<float4 *>(dst + 2 * k), make_float4(e0.x, e0.y, o0.x, o0.y));
        __stcs(reinterpret_cast<float4 *>(dst + 2 * k + 2), make_float4(e1.x, e1.y, o1.x, o1.y));
      }
      if (load_next) {
        a[2 * j] = __ldcs(nsrc + lt + (2 * j) * T);
        a[2 * j + 1] = __ldcs(nsrc + lt + (2 * j + 1) * T);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = 4 * C + q;
      const int k = final_index<H, P, SC>(lt, m);
      const float2 e = cscale(make_float2(r[2 * q], r[2 * q + 1]), s);
      const float2 o = cscale(a[m], s);
      __stcs(reinterpret_cast<float4 *>(dst + 2 * k), make_float4(e.x, e.y, o.x, o.y));
      if (load_next) a[m] = __ldcs(nsrc + lt + m * T);
    }
  }
  if constexpr (4 * C + 4 < P)
    tmem2_store_chunk<N, P, SC, PAIR_LAST, OUT32, C + 1>(a, lt, taddr, dst, nsrc, load_next, s);
}

// Persistent: CTA c takes rows c, c + G, ... (G = gridDim.x, one CTA per SM:
// the H-point exchange buffer and 512 threads of up to 128 registers).
// Warp 0 prefetches the CTA's next row (both halves) into L2 (bulk copy);
// its lanes issue the second-half copy into the exchange buffer, 32 slabs.
template <int N, int P, int D, class SC, int TWM>
__global__ void __launch_bounds__(N / 2 / P, 1) tmem2_kernel(Tmem2Args args) {
  constexpr int H = N / 2, T = H / P;
  static_assert(P == 32 && T % 128 == 0, "whole warpgroups of 32-point threads");
  static_assert(SC::product() == H, "the schedule transforms one half");
  constexpr bool PAIR_LAST = pairable<H, P, SC>();
  constexpr uint32_t REGION = (T / 128) * 64;  // 64 columns (32 points) per thread
  constexpr uint32_t NCOL = 2 * REGION;         // regions D and E
  static_assert(NCOL <= 512, "tensor memory has 512 columns");
  constexpr unsigned kHalf = sizeof(float2) * H, kPiece = kHalf / 32;
  static_assert(kPiece % 16 == 0, "bulk copies move multiples of 16 bytes");
  extern __shared__ __align__(128) float2 smem[];  // tmem2_smem_bytes<N>()
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + H);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + H) + 1;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lt = threadIdx.x, warp = lt >> 5;
  if (warp == 0) tmem_alloc_warp(tslot, NCOL);
  if (lt == 32) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // The second half of row r into the exchange buffer (warp 0; the buffer
  // is free: no thread reads it until the copy's barrier completes).
  auto issue_half = [&](int r) {
    if (warp == 0) {
      if (lt == 0) mbar_expect_tx(bar, kHalf);
      __syncwarp();
      tma_load_1d(reinterpret_cast<char *>(smem) + lt * kPiece,
                  reinterpret_cast<const char *>(args.in + (long long)r * N + H) + lt * kPiece, kPiece,
                  bar);
    }
  };
  const uint32_t tbase = *tslot;
  const uint32_t tD = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  float2 a[P];
  // Row indices fit 32 bits: a row is 256 KiB, so 2^31 rows exceed any memory
  // (the launcher checks batch against INT_MAX).
  const int batch = (int)args.batch;
  int row = blockIdx.x;
  if (row < batch) {
    issue_half(row);
    load_row<H, P>(a, args.in + (long long)row * N, lt);
  }
  bool ok = true;
  unsigned par = 0;  // phase of the copy barrier: one completion per row
  for (; row < batch; row += gridDim.x, par ^= 1u) {
    const int next = row + gridDim.x;
    const bool load_next = next < batch;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      // Opaque per round: keeps the loop-invariant twiddle and buffer
      // addresses and the thread's output indices from being hoisted out of
      // the row loop into registers.
      const float2 *twp = args.tw;
      float2 *bufp = smem;
      int ltp = lt;
      asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
      if (h == 0) {
        ok = __syncthreads_and(mbar_wait(bar, par));  // the second half has landed
        if (!ok) break;
        const float2 wt = __ldg(args.tw_n + ltp);  // read per row: nothing stays live
        tmem2_split_chunk<N, P, D, 0>(a, bufp, ltp, tD, wt);
        tmem_wait_st();
        // the next row into L2 once this row's inputs have landed
        if (load_next && lt < 32)
          prefetch_l2_warp(args.in + (long long)next * N, (long long)N * (long long)sizeof(float2), lt);
        __syncthreads();  // the second half is read: the transform may write the buffer
      } else {
        tmem2_load_chunk<P, 0>(a, tD);
        __syncthreads();  // every thread has read round 0's last exchange
      }
      run_passes_early<H, P, D, SC, 0, TWM, PAIR_LAST>(a, ltp, bufp, twp, NoHook{}, NoTw{});
      if (h == 0) {
        tmem2_park_chunk<P, 0>(a, tD + REGION);
        tmem_wait_st();
      } else {
        // every thread is past round 1's last exchange read: the buffer may
        // take the next row's second half while this row's outputs drain
        __syncthreads();
        if (load_next) {
          fence_proxy_async();
          issue_half(next);
        }
        float2 *dst = args.out + (long long)row * N;
        const float2 *nsrc = args.in + (long long)(load_next ? next : row) * N;
        const float s = args.scale;
        if (args.out32)
          tmem2_store_chunk<N, P, SC, PAIR_LAST, true, 0>(a, ltp, tD + REGION, dst, nsrc, load_next, s);
        else
          tmem2_store_chunk<N, P, SC, PAIR_LAST, false, 0>(a, ltp, tD + REGION, dst, nsrc, load_next, s);
      }
    }
    if (!ok) break;
  }
  if (!ok) {
    if (lt == 0) {
      if (args.status) atomicCAS(args.status, 0, 6 /* FFT_ERR_TIMEOUT */);
      (void)mbar_wait(bar, par, kDrainNs);  // the copy still in flight lands first
    }
  }
  tmem_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc_warp(tbase, NCOL);
}

}  // namespace fftgb
