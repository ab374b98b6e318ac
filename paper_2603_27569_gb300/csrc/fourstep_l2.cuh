// Two-phase four-step with an L2-resident intermediate (paper Sec. IV-B and
// synthesis rule 2 of Sec. IV-D: column FFTs, twiddle, row FFTs, the transpose
// passing through device memory -- here through L2).
//
// N = L * L.  Phase 1 of a row: for each n1, the L-point FFT over n2 of
// x[n1 + L n2], times W_N^{n1 k2}, stored transposed as A[n1][k2]; phase 2:
// for each k2, the L-point FFT over n1 of A[n1][k2], stored at k2 + L k1.
// Both phases are column FFTs of C = 16 adjacent columns (column.cuh).
//
// One persistent launch runs both phases for the whole batch.  Rows are cut
// into chunks; chunk c's intermediate lives in ring slot c mod S, small
// enough to stay in L2.  Work items (phase, chunk, column tile) are claimed
// from a device counter in rounds: round r holds phase-1 tiles of chunk r and
// phase-2 tiles of chunk r - LAG, so a phase-2 tile is claimed LAG rounds
// after the tiles it reads.  A phase-2 tile of chunk c waits until all
// phase-1 tiles of c are done; a phase-1 tile of chunk c waits until all
// phase-2 tiles of chunk c - S (the slot's previous user) are done.  Every
// item waited on was claimed earlier by a running CTA that never waits on a
// later item, so the launch always progresses; each wait is also bounded in
// time and records FFT_ERR_TIMEOUT if it runs out.  Consumed intermediate
// lines are dropped from L2 without write-back (discard.global.L2), so the
// intermediate need not reach HBM.  The counters are cleared by the last CTA
// to finish, so back-to-back launches on one stream need no memset; two
// launches sharing the counters and ring must not run concurrently.
#pragma once
#include <stdint.h>

#include "stockham.cuh"

namespace fftgb {

struct FourstepL2Args {
  const float2 *in;
  float2 *out;
  float2 *ring;            // S slots of chunk_rows * N points
  const float2 *tw;        // pass tables of the L-point schedule
  const float2 *tw_a;      // W_N^{c lt} at lt * L + c (phase-1 twiddle, as column.cuh)
  const float2 *tw_b;      // W_N^{c T m} at m * L + c
  unsigned *counters;      // [0] items claimed, [1] CTAs finished, then nchunks phase-1
                           // done counts and nchunks phase-2 done counts; all zero
                           // between launches (the last CTA to finish clears them)
  int *status;
  long long batch;
  int chunk_rows, nchunks, slots, lag;
  float scale;
};

constexpr unsigned long long kL2WaitNs = 2000000000ull;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long l2_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *cnt >= target (bounded by limit_ns); returns false on
// time-out.
__device__ __forceinline__ bool wait_count(const unsigned *cnt, unsigned target,
                                           unsigned long long limit_ns = kL2WaitNs) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = l2_timer_ns();
  while (true) {
    __nanosleep(256);
    if (ld_acquire(cnt) >= target) return true;
    if (l2_timer_ns() - t0 > limit_ns) return false;
  }
}

// Item w of the schedule: phase, chunk and column tile (chunk out of range:
// an empty slot of the first or last rounds).
struct L2Item {
  bool p1;
  long long chunk, tile;
};

__device__ __forceinline__ L2Item l2_item(long long w, long long TT, int lag) {
  const long long r = w / (2 * TT), off = w - r * 2 * TT;
  L2Item it;
  it.p1 = off < TT;
  it.chunk = it.p1 ? r : r - lag;
  it.tile = it.p1 ? off : off - TT;
  return it;
}

// Register budget 64 per thread (65536 / 64 threads' worth of CTAs per SM).
template <int L, int P, int C, int D, class SC>
__global__ void __launch_bounds__(C *(L / P), 1024 / (C * (L / P)))
fourstep_l2_kernel(FourstepL2Args a) {
  constexpr int N = L * L;
  constexpr int T = L / P;
  constexpr int NT = C * T;
  constexpr int GROUPS = L / C;  // column tiles per row and phase
  static_assert(NT >= 64, "two warps needed (claims and completions)");
  extern __shared__ __align__(128) float2 smem[];
  __shared__ long long s_item[2];
  __shared__ int s_ok;
  const int c = threadIdx.x % C;
  const int lt = threadIdx.x / C;
  const long long TT = (long long)a.chunk_rows * GROUPS;   // tiles per chunk and phase
  const long long total = (long long)(a.nchunks + a.lag) * 2 * TT;
  unsigned *done1 = a.counters + 2;
  unsigned *done2 = a.counters + 2 + a.nchunks;
  // Thread 0 claims items one ahead: the claim for the next item is in flight
  // while the current one is processed (a CTA holding item w and the next
  // claimed item still only ever waits on items below w).
  if (threadIdx.x == 0) s_item[0] = (long long)atomicAdd(a.counters, 1u);
  __syncthreads();
  int cur = 0;
  while (true) {
    const long long w = s_item[cur];
    if (w >= total) break;
    unsigned long long next = 0;
    if (threadIdx.x == 0) next = atomicAdd(a.counters, 1u);
    const L2Item it = l2_item(w, TT, a.lag);
    const bool real = it.chunk >= 0 && it.chunk < a.nchunks;
    if (real) {
      const int rin = (int)(it.tile / GROUPS);                  // row within the chunk
      const int c0 = (int)(it.tile - (long long)rin * GROUPS) * C;
      const long long row = it.chunk * a.chunk_rows + rin;
      float2 *slot = a.ring + ((it.chunk % a.slots) * a.chunk_rows + rin) * (long long)N;
      // dependencies (thread 0 waits, the CTA follows)
      if (threadIdx.x == 0) {
        bool ok = true;
        if (it.p1 && it.chunk >= a.slots)
          ok = wait_count(done2 + (it.chunk - a.slots), (unsigned)TT);
        if (!it.p1) ok = wait_count(done1 + it.chunk, (unsigned)TT);
        if (!ok) atomicCAS(a.status, 0, 6 /* FFT_ERR_TIMEOUT */);
        s_ok = ok;
      }
      __syncthreads();
      if (s_ok && row < a.batch) {
        float2 v[P];
        if (it.p1) {
          // x[row][n1 + L n2], columns n1 = c0 + c
          const float2 *src = a.in + row * N + c0 + c;
#pragma unroll
          for (int m = 0; m < P; ++m) v[m] = __ldcs(src + (long long)(lt + m * T) * L);
        } else {
          // A[n1][k2] of this row, columns k2 = c0 + c (L2 only: the slot is rewritten)
          const float2 *src = slot + c0 + c;
#pragma unroll
          for (int m = 0; m < P; ++m) v[m] = __ldcg(src + (lt + m * T) * L);
        }
        // opaque per item: keeps table addresses and loads inside the loop
        const float2 *twp = a.tw;
        float2 *bufp = smem;
        int ltp = lt, cp = c;
        asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp), "+r"(cp));
        run_passes<L, P, D, SC, 0>(v, ltp, bufp, twp, Interleaved<C>{cp});
        if (it.p1) {
          const int col = c0 + c;  // n1; register m holds k2 = lt + T m
          const float2 wa = __ldg(a.tw_a + lt * L + col);
#pragma unroll
          for (int m = 0; m < P; ++m)
            v[m] = cmul_dir<D>(v[m], cmul(wa, __ldg(a.tw_b + m * L + col)));
          // A[n1][k2] at slot + n1 * L + k2, through a tile padded to C + 1 columns
          constexpr int LD = C + 1;
          __syncthreads();
#pragma unroll
          for (int m = 0; m < P; ++m) smem[final_index<L, P, SC>(lt, m) * LD + c] = v[m];
          __syncthreads();
          float2 *dst = slot + (long long)c0 * L;
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const int e = threadIdx.x + u * NT;
            const int cl = e / L, k = e - cl * L;
            __stcg(dst + e, smem[k * LD + cl]);
          }
        } else {
          // consumed: drop this tile's L row segments (C points = 128 bytes) from L2
          __syncthreads();
          for (int q = threadIdx.x; q < L; q += NT)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(slot + q * L + c0) : "memory");
          float2 *dst = a.out + row * N + c0 + c;
#pragma unroll
          for (int m = 0; m < P; ++m)
            __stcs(dst + (long long)final_index<L, P, SC>(lt, m) * L, cscale(v[m], a.scale));
        }
      }
    }
    if (threadIdx.x == 0) s_item[cur ^ 1] = (long long)next;
    __syncthreads();  // the tile's writes (and the buffer) are done; next item published
    if (real && threadIdx.x == 32) {  // a second warp signals, warp 0 goes on claiming
      __threadfence();
      atomicAdd(it.p1 ? done1 + it.chunk : done2 + it.chunk, 1u);
    }
    cur ^= 1;
  }
  // Every CTA has made its last claim; the last one out clears the counters
  // (after this CTA's last completion signal, by the barrier and the fence).
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_ok = atomicAdd(a.counters + 1, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_ok) {
    __threadfence();
    const int n = 2 + 2 * a.nchunks;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.counters[i] = 0u;
  }
}

}  // namespace fftgb
