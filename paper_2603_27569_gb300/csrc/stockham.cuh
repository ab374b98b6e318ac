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
// read set is always {t + m T : m < P} and needs no per-pass reshuffle.  A
// last pass with two butterflies per thread takes butterflies 2t and 2t + 1
// instead (pairable<>), so its exchange read, twiddle loads and output
// stores are 16-byte accesses.
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
#include "check.cuh"

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
  long long ahead;      // one tile per CTA: resident CTAs (occupancy x SMs); 0: none
};

// The r - 1 twiddles W^{j k}, j = 1 .. r-1, of one butterfly.
//   TWM = 0: every one read from the pass table (row j - 1).
//   TWM = 1: the rows tw_loaded<r> names read, the others derived
//            (derive_twiddles).  This trades r - 3 table reads (L1 traffic)
//            for as many complex multiplies.
template <int r, int p, int TWM>
__device__ __forceinline__ void load_twiddles(float2 (&w)[r], const float2 *__restrict__ tws, int k) {
  const bool ok = FFTGB_OK(k, p, kSiteTwiddle);  // entry k of each table row
#pragma unroll
  for (int j = 1; j < r; ++j)
    if (TWM == 0 || tw_loaded<r>(j)) w[j] = ok ? __ldg(tws + (j - 1) * p + k) : make_float2(1.f, 0.f);
  if constexpr (TWM == 1) derive_twiddles<r>(w);
}

// The twiddles of two butterflies with k0 and k0 + 1 (k0 even): their
// entries of each table row are adjacent, so one 16-byte load gives both.
template <int r, int p, int TWM>
__device__ __forceinline__ void load_twiddles_pair(float2 (&w0)[r], float2 (&w1)[r],
                                                   const float2 *__restrict__ tws, int k0) {
  const bool ok = FFTGB_OK(k0, p, kSiteTwiddle) && FFTGB_OK(k0 + 1, p, kSiteTwiddle);
#pragma unroll
  for (int j = 1; j < r; ++j)
    if (TWM == 0 || tw_loaded<r>(j)) {
      const float4 v = ok ? __ldg(reinterpret_cast<const float4 *>(tws + (j - 1) * p + k0))
                          : make_float4(1.f, 0.f, 1.f, 0.f);
      w0[j] = make_float2(v.x, v.y);
      w1[j] = make_float2(v.z, v.w);
    }
  if constexpr (TWM == 1) {
    derive_twiddles<r>(w0);
    derive_twiddles<r>(w1);
  }
}

// Butterfly of register group q of thread lt in a pass of radix r = P / Q.
// Plain: butterflies lt + q T.  Paired (last pass, Q = 2): butterflies 2 lt
// and 2 lt + 1.  In the last pass (p = N / r) butterfly i reads point
// i + j N / r and writes output i + j N / r, so a paired thread's two points
// (and two outputs) of each j sit side by side: one 16-byte shared load and
// one 16-byte global store instead of two 8-byte ones.
template <int T, int Q, bool PAIRED>
__device__ __forceinline__ int bfly(int lt, int q) {
  if constexpr (PAIRED) {
    static_assert(Q == 2, "paired passes hold two butterflies per thread");
    return 2 * lt + q;
  } else {
    return lt + q * T;
  }
}

// Can schedule SC end in a paired pass?  Two butterflies per thread in the
// last pass, and at least three passes so that the exchange read before it
// uses a layout swz<p, r> with p >= 2, which keeps index pairs (2x, 2x + 1)
// adjacent (the swizzle only permutes bits 1..3).
template <int N, int P, class SC>
__host__ __device__ constexpr bool pairable() {
  return SC::npass >= 3 && P / SC::radix[SC::npass - 1] == 2;
}

// Twiddle + butterflies of pass S for every butterfly q of this thread.
template <int N, int P, int D, class SC, int S, int TWM, bool PAIRED = false>
__device__ __forceinline__ void pass_compute(float2 (&a)[P], int lt, const float2 *__restrict__ tw) {
  constexpr int r = SC::radix[S];
  constexpr int p = SC::stride(S);
  constexpr int T = N / P;
  constexpr int Q = P / r;
  if constexpr (S > 0 && PAIRED) {
    // k of butterflies 2 lt, 2 lt + 1 (p even): 2 lt mod p and one more
    float2 w0[r], w1[r];
    load_twiddles_pair<r, p, TWM>(w0, w1, tw + SC::tw_offset(S), bfly<T, Q, true>(lt, 0) & (p - 1));
#pragma unroll
    for (int j = 1; j < r; ++j) {
      a[j * Q] = cmul_dir<D>(a[j * Q], w0[j]);
      a[1 + j * Q] = cmul_dir<D>(a[1 + j * Q], w1[j]);
    }
  } else if constexpr (S > 0) {
    const float2 *tws = tw + SC::tw_offset(S);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = bfly<T, Q, PAIRED>(lt, q);
      const int k = i & (p - 1);
      float2 w[r];
      load_twiddles<r, p, TWM>(w, tws, k);
#pragma unroll
      for (int j = 1; j < r; ++j) a[q + j * Q] = cmul_dir<D>(a[q + j * Q], w[j]);
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
  static constexpr int width = 1;  // buffer slots per logical index
  template <int p, int r>
  __device__ __forceinline__ int at(int idx) const { return swz<p, r>(idx); }
};
template <int C>
struct Interleaved {
  static constexpr int width = C;
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
    for (int j = 0; j < r; ++j) {
      const int at = ly.template at<p, r>(base + j * p);
      if (FFTGB_OK(base + j * p, N, kSiteXchgWrite) && FFTGB_OK(at, N * LY::width, kSiteXchgWrite))
        buf[at] = a[q + j * Q];
    }
  }
}

// Read the next pass's points {lt + m T} from the buffer written by pass S
// (PAIRED: the points of the next pass's paired butterflies, register
// q + 2 j = point j of butterfly bfly(lt, q), as 16-byte pairs).
template <int N, int P, class SC, int S, class LY, bool PAIRED = false>
__device__ __forceinline__ void pass_read(float2 (&a)[P], int lt, const float2 *buf, const LY &ly) {
  constexpr int r = SC::radix[S];
  constexpr int p = SC::stride(S);
  constexpr int T = N / P;
  if constexpr (PAIRED) {
    static_assert(p >= 2, "paired reads need a layout that keeps pairs adjacent");
    constexpr int rn = SC::radix[S + 1];
    const int i0 = bfly<T, P / rn, true>(lt, 0);
#pragma unroll
    for (int j = 0; j < P / 2; ++j) {
      const int at = ly.template at<p, r>(i0 + j * (N / rn));
      const float4 v = FFTGB_OK(i0 + 1 + j * (N / rn), N, kSiteXchgRead) &&
                               FFTGB_OK(at + 1, N * LY::width, kSiteXchgRead)
                           ? *reinterpret_cast<const float4 *>(buf + at)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      a[2 * j] = make_float2(v.x, v.y);
      a[2 * j + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int at = ly.template at<p, r>(lt + m * T);
      a[m] = FFTGB_OK(lt + m * T, N, kSiteXchgRead) && FFTGB_OK(at, N * LY::width, kSiteXchgRead)
                 ? buf[at]
                 : make_float2(0.f, 0.f);
    }
  }
}

// Passes S .. npass-1.  On entry a[] holds pass S's inputs.  On return a[]
// holds the final outputs of the last pass in its butterfly order.
// Barrier policies for the exchanges: the whole CTA, or a named barrier
// (`bar.sync id, count`) shared by a group of warps working on its own rows.
struct CtaBarrier {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct NamedBarrier {
  int id, count;  // id 1..15; count a multiple of 32
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
  }
};

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// PAIR_LAST: the last pass runs paired butterflies (its outputs leave as
// 16-byte pairs, see final_index_pair).  hk() runs once, after the barrier
// that follows pass 0's exchange write: by then every thread has consumed
// its pass-0 loads.
template <int N, int P, int D, class SC, int S, class LY, int TWM = 0, class BR = CtaBarrier,
          bool PAIR_LAST = false, class HK = NoHook>
__device__ __forceinline__ void run_passes(float2 (&a)[P], int lt, float2 *buf,
                                           const float2 *__restrict__ tw, const LY &ly,
                                           const BR &br = BR{}, const HK &hk = HK{}) {
  constexpr bool PAIRED_HERE = PAIR_LAST && S + 1 == SC::npass;
  pass_compute<N, P, D, SC, S, TWM, PAIRED_HERE>(a, lt, tw);
  if constexpr (S + 1 < SC::npass) {
    if constexpr (S > 0) br.sync();  // every read of the buffer is done
    pass_write<N, P, SC, S>(a, lt, buf, ly);
    br.sync();
    if constexpr (S == 0) hk();
    pass_read<N, P, SC, S, LY, PAIR_LAST && S + 2 == SC::npass>(a, lt, buf, ly);
    run_passes<N, P, D, SC, S + 1, LY, TWM, BR, PAIR_LAST>(a, lt, buf, tw, ly, br);
  }
}

// Twiddle-table rows of pass S for this thread's butterflies, read ahead:
// run_passes_early issues these loads before the barrier that precedes the
// pass's exchange read, so their latency overlaps the barrier wait (the
// rows do not depend on the exchanged data).  Only the rows the twiddle mode
// reads are filled; pass_apply derives the rest.
template <int N, int P, class SC, int S, int TWM, bool PAIRED>
struct PassTw {
  static constexpr int r = SC::radix[S];
  static constexpr int p = SC::stride(S);
  static constexpr int T = N / P;
  static constexpr int Q = P / r;
  float2 w[Q][r];
  __device__ __forceinline__ void load(int lt, const float2 *__restrict__ tw) {
    const float2 *tws = tw + SC::tw_offset(S);
    if constexpr (PAIRED) {
      const int k0 = bfly<T, Q, true>(lt, 0) & (p - 1);
      const bool ok = FFTGB_OK(k0, p, kSiteTwiddle) && FFTGB_OK(k0 + 1, p, kSiteTwiddle);
#pragma unroll
      for (int j = 1; j < r; ++j)
        if (TWM == 0 || tw_loaded<r>(j)) {
          const float4 v = ok ? __ldg(reinterpret_cast<const float4 *>(tws + (j - 1) * p + k0))
                              : make_float4(1.f, 0.f, 1.f, 0.f);
          w[0][j] = make_float2(v.x, v.y);
          w[1][j] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = bfly<T, Q, false>(lt, q) & (p - 1);
        const bool ok = FFTGB_OK(k, p, kSiteTwiddle);
#pragma unroll
        for (int j = 1; j < r; ++j)
          if (TWM == 0 || tw_loaded<r>(j))
            w[q][j] = ok ? __ldg(tws + (j - 1) * p + k) : make_float2(1.f, 0.f);
      }
    }
  }
};
struct NoTw {};

// Pass S from read-ahead twiddle rows (S > 0) or none (S = 0): the same
// twiddle multiplies and butterflies as pass_compute.
template <int N, int P, int D, class SC, int S, int TWM, class PT>
__device__ __forceinline__ void pass_apply(float2 (&a)[P], const PT &t) {
  constexpr int r = SC::radix[S];
  constexpr int Q = P / r;
  if constexpr (S > 0) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2 w[r];
#pragma unroll
      for (int j = 1; j < r; ++j)
        if (TWM == 0 || tw_loaded<r>(j)) w[j] = t.w[q][j];
      if constexpr (TWM == 1) derive_twiddles<r>(w);
#pragma unroll
      for (int j = 1; j < r; ++j) a[q + j * Q] = cmul_dir<D>(a[q + j * Q], w[j]);
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

// A warp-wide barrier: for thread groups that lie inside one warp.
struct WarpBarrier {
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// run_passes for one row per thread group with the swizzled row layout,
// reading each pass's twiddle rows ahead of its exchange barrier (PassTw).
// hk() as in run_passes; br: the group's barrier (the whole CTA by default).
template <int N, int P, int D, class SC, int S, int TWM, bool PAIR_LAST, class HK, class PT,
          class BR = CtaBarrier>
__device__ __forceinline__ void run_passes_early(float2 (&a)[P], int lt, float2 *buf,
                                                 const float2 *__restrict__ tw, const HK &hk,
                                                 const PT &pre, const BR &br = BR{}) {
  pass_apply<N, P, D, SC, S, TWM>(a, pre);
  if constexpr (S + 1 < SC::npass) {
    constexpr bool PN = PAIR_LAST && S + 2 == SC::npass;
    if constexpr (S > 0) br.sync();  // every read of the buffer is done
    pass_write<N, P, SC, S>(a, lt, buf, SwizzledRow{});
    PassTw<N, P, SC, S + 1, TWM, PN> next;
    next.load(lt, tw);
    br.sync();
    if constexpr (S == 0) hk();
    pass_read<N, P, SC, S, SwizzledRow, PN>(a, lt, buf, SwizzledRow{});
    run_passes_early<N, P, D, SC, S + 1, TWM, PAIR_LAST>(a, lt, buf, tw, hk, next, br);
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

// Paired last pass: register pair (2 j, 2 j + 1) holds outputs i0 + j N / r
// and i0 + 1 + j N / r (i0 = bfly(lt, 0)), adjacent in the output row.
template <int N, int P, class SC>
__device__ __forceinline__ int final_index_pair(int lt, int j) {
  constexpr int r = SC::radix[SC::npass - 1];
  constexpr int T = N / P;
  return bfly<T, P / r, true>(lt, 0) + j * (N / r);
}

// L2 prefetch of `bytes` (a multiple of 16) starting at p, issued by the 32
// lanes of one warp, each for its slice, through the bulk-copy (TMA) engine.
__device__ __forceinline__ void prefetch_l2_warp(const void *p, long long bytes, int lane) {
  const long long chunk = (((bytes + 31) / 32) + 15) & ~15ll;
  const long long off = lane * chunk;
  if (off < bytes) {
    const long long n = bytes - off < chunk ? bytes - off : chunk;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                 :: "l"((const char *)p + off), "r"((unsigned)n) : "memory");
  }
}

// Row loads of pass 0: thread lt of row `row` takes the points lt + m T.
template <int N, int P>
__device__ __forceinline__ void load_row(float2 (&a)[P], const float2 *src, int lt) {
  constexpr int T = N / P;
#pragma unroll
  for (int m = 0; m < P; ++m)
    a[m] = FFTGB_OK(lt + m * T, N, kSiteLoadIdx) ? __ldcs(src + lt + m * T) : make_float2(0.f, 0.f);
}

// Persistent over tiles of TB rows: CTA c handles tiles c, c + G, c + 2G, ...
// (G = gridDim.x; a grid of one CTA per tile runs the loop once).  Warp 0
// asks the bulk-copy engine to prefetch the CTA's NEXT tile into L2, so HBM
// streams the next rows while this tile computes.
//
// Epilogue: the output held in register m (or register pair 2j, 2j + 1) is
// stored, and the register is at once refilled with the next tile's input
// point m.  The next tile's loads (from L2, prefetched) are then in flight
// while this tile's stores drain, instead of being issued after them: the
// SM's read and write paths to L2 work at the same time.  The buffer is
// rewritten only after the end-of-tile barrier, so nothing else changes.
template <int N, int P, int TB, int D, class SC, int TWM>
__global__ void __launch_bounds__(TB *(N / P))
stockham_kernel(StockhamArgs args) {
  constexpr bool PAIR_LAST = pairable<N, P, SC>();
  static_assert(SC::product() == N, "radix schedule must multiply to N");
  static_assert(P % SC::max_radix() == 0, "every radix must divide P");
  constexpr int T = N / P;
  extern __shared__ __align__(128) float2 smem[];
  // Launched with programmatic stream serialization: this grid's CTAs may
  // become resident while the previous kernel of the stream is finishing;
  // nothing global is touched before that kernel has completed and its
  // writes are visible.  Then the next kernel's CTAs may launch as this
  // grid's CTAs retire.  (Without the launch attribute both are no-ops.)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int b = threadIdx.x / T;
  const int lt = threadIdx.x - b * T;
  float2 *buf = smem + b * N;
  const long long ntiles = (args.batch + TB - 1) / TB;
  long long tile = blockIdx.x;
  // One tile per CTA: first have the tile of the CTA one resident wave later
  // prefetched into L2, so that CTA reads its rows from L2 instead of HBM.
  if (args.ahead > 0 && gridDim.x >= ntiles && threadIdx.x < 32) {
    const long long t2 = tile + args.ahead;
    if (t2 < ntiles) {
      const long long rows = args.batch - t2 * TB < TB ? args.batch - t2 * TB : TB;
      prefetch_l2_warp(args.in + t2 * TB * N, rows * N * (long long)sizeof(float2), threadIdx.x);
    }
  }
  float2 a[P];
  // Rows past the batch exist only in the last tile (all later tiles of
  // this CTA would be past it too), so an inactive row ends the loop.
  if (tile < ntiles && tile * TB + b < args.batch &&
      FFTGB_OK(tile * TB + b, args.batch, kSiteLoadRow)) {
    load_row<N, P>(a, args.in + (tile * TB + b) * N, lt);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
  }
  for (; tile < ntiles; tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    auto prefetch_next = [&]() {
      if (next < ntiles && threadIdx.x < 32) {
        const long long rows = args.batch - next * TB < TB ? args.batch - next * TB : TB;
        prefetch_l2_warp(args.in + next * TB * N, rows * N * (long long)sizeof(float2),
                         threadIdx.x);
      }
    };
    // The first tile's own loads come from HBM: its prefetch of the next
    // tile waits until they have landed (after the first exchange).  Later
    // tiles were prefetched into L2 and prefetch theirs at once, which
    // gives the next tile the whole tile time to arrive.
    const bool first = tile == (long long)blockIdx.x;
    if (SC::npass == 1 || !first) prefetch_next();
    const long long row = tile * TB + b;
    const bool active = row < args.batch;
    const long long nrow = next * TB + b;
    const bool load_next = next < ntiles && nrow < args.batch;
    // Opaque per tile: keeps the compiler from hoisting the loop-invariant
    // twiddle reads and exchange addresses out of the tile loop into
    // (occupancy-costly) registers.
    const float2 *twp = args.tw;
    float2 *bufp = buf;
    int ltp = lt;
    asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
    run_passes_early<N, P, D, SC, 0, TWM, PAIR_LAST>(
        a, ltp, bufp, twp,
        [&]() {
          if (first) prefetch_next();
        },
        NoTw{});
    if (active && FFTGB_OK(row, args.batch, kSiteStoreRow) &&
        (!load_next || FFTGB_OK(nrow, args.batch, kSiteLoadRow))) {
      float2 *dst = args.out + row * N;
      const float2 *nsrc = args.in + (load_next ? nrow : row) * N;
      const float s = args.scale;
      if constexpr (PAIR_LAST) {
#pragma unroll
        for (int j = 0; j < P / 2; ++j) {
          const float2 u = cscale(a[2 * j], s), v = cscale(a[2 * j + 1], s);
          const int k = final_index_pair<N, P, SC>(ltp, j);
          if (FFTGB_OK(k, N, kSiteStoreIdx) && FFTGB_OK(k + 1, N, kSiteStoreIdx))
            __stcs(reinterpret_cast<float4 *>(dst + k), make_float4(u.x, u.y, v.x, v.y));
          if (load_next) {
            a[2 * j] = __ldcs(nsrc + lt + (2 * j) * T);
            a[2 * j + 1] = __ldcs(nsrc + lt + (2 * j + 1) * T);
          }
        }
      } else {
#pragma unroll
        for (int m = 0; m < P; ++m) {
          const int k = final_index<N, P, SC>(ltp, m);
          if (FFTGB_OK(k, N, kSiteStoreIdx)) __stcs(dst + k, cscale(a[m], s));
          if (load_next) a[m] = __ldcs(nsrc + lt + m * T);
        }
      }
    }
    if (next < ntiles) __syncthreads();  // the next tile rewrites the buffer
  }
}

}  // namespace fftgb
