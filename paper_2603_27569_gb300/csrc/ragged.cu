// Ragged batches: many transforms of mixed lengths and directions in ONE
// persistent launch (paper Sec. II-D: radar workloads are batches of 1-D FFTs
// of 2^10..2^14 points; here a batch may mix them).
//
// One kernel, one 512-thread CTA per SM, persistent, in two phases.  Phase
// 1: the whole CTA is one worker that takes 16384-point rows (512 threads x
// 32 points).  Once no row of 16384 is left, the CTA splits for good into
// two independent 256-thread workers (64 KiB of shared memory each) that
// take the other classes, like two CTAs of the plain kernel.  A worker's
// unit fills it: W P / N rows of one (N, direction), N / P threads each (W =
// 512 or 256 threads; one row of 8192, ..., 256 rows of 16 points).  Units
// are listed longest N first (LPT order) and claimed through one device
// counter per phase; a worker claims the unit after next while it works, so
// at the end of a unit each thread stores its outputs and, register by
// register, loads its inputs of the next unit of the same class in the same
// loop (the next unit's loads overlap this unit's stores; warp 0 of the
// worker asks the bulk-copy engine to prefetch the next unit's rows into L2
// after its first exchange).  The rows of a unit are independent: each row
// group synchronises on its own barrier (a named barrier `bar.sync id,
// count` for 64..512 threads, the warp for rows that fit in one), so groups
// drift apart inside a unit and meet only at the unit boundary.
//
// Every class (N) has a few compiled routines (points per thread, radix
// schedule, twiddle mode; FFTGB_RAG_ROUTINES).  Which one a class uses is
// the built-in choice, or the autotuner's (FFT_FLAG_RAGGED_AUTOTUNE): it
// times every routine of every class of the batch on that class's rows and
// keeps the fastest in a process-wide cache that later ragged plans use.
//
// The kernel is captured once per (in, out) pair into a CUDA graph that each
// fft_exec replays on the caller's stream; the graph holds that one kernel
// node (the last CTA of a launch resets the claim counters itself).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "plan.h"
#include "stockham.cuh"

namespace fftgb {

struct RaggedDesc {
  long long in_off, out_off;  // complex elements from the packed bases
};
struct RaggedUnit {
  int first;       // first descriptor of the unit
  int count;       // rows in the unit (at most the routine's rows per unit)
  int routine;     // index of the compiled routine (FFTGB_RAG_ROUTINES)
  int dir;         // -1 forward, +1 inverse
  long long in0;   // input offset of the unit's first row (its L2 prefetch)
};

// The compiled routines: (index, N, points per thread P, twiddle mode,
// radix schedule).  A unit of routine r has 512 threads: 512 P / N rows of
// N / P threads.  Each class lists its built-in routine first.
#define FFTGB_RAG_ROUTINES(X)            \
  X(0, 16384, 32, 1, 32, 32, 16)         \
  X(1, 16384, 32, 0, 32, 32, 16)         \
  X(2, 8192, 32, 1, 32, 16, 16)          \
  X(3, 8192, 32, 0, 32, 16, 16)          \
  X(4, 4096, 16, 1, 16, 16, 16)          \
  X(5, 4096, 32, 1, 16, 16, 16)          \
  X(6, 2048, 16, 1, 16, 16, 8)           \
  X(7, 2048, 32, 1, 16, 16, 8)           \
  X(8, 1024, 16, 1, 16, 16, 4)           \
  X(9, 1024, 32, 1, 32, 32)              \
  X(10, 512, 16, 1, 16, 16, 2)           \
  X(11, 512, 32, 1, 32, 16)              \
  X(12, 256, 16, 0, 16, 16)              \
  X(13, 256, 32, 0, 16, 16)              \
  X(14, 128, 16, 0, 16, 8)               \
  X(15, 64, 16, 0, 16, 4)                \
  X(16, 32, 16, 0, 16, 2)                \
  X(17, 16, 16, 0, 16)
constexpr int kRagRoutines = 18;
constexpr int kRagThreads = 512;
constexpr int kRagMinLog2 = 4, kRagMaxLog2 = 14;
constexpr size_t kRagSmem = sizeof(float2) * 16384;  // one unit of 32 points per thread

struct RagRoutine {
  int N, P, twm, npass, radix[4];
};
#define FFTGB_RAG_HOST(I, N, P, TWM, ...) {N, P, TWM, 0, {__VA_ARGS__}},
static const RagRoutine kRagTable[kRagRoutines] = {FFTGB_RAG_ROUTINES(FFTGB_RAG_HOST)};
#undef FFTGB_RAG_HOST

static int rag_npass(const RagRoutine &r) {
  int n = 0;
  while (n < 4 && r.radix[n] > 0) ++n;
  return n;
}
// Threads of the worker that runs a routine's units: the whole CTA for
// 16384-point rows, a 256-thread half for every other class.
static int rag_worker(const RagRoutine &r) { return r.N == 16384 ? kRagThreads : 256; }
static int rag_rows_per_unit(const RagRoutine &r) { return rag_worker(r) * r.P / r.N; }

struct RaggedArgs {
  const float2 *in;
  float2 *out;
  const RaggedDesc *desc;
  const RaggedUnit *units;
  int nunits;
  int nA;             // units [0, nA): 16384-point rows (phase 1); the rest: phase 2
  unsigned *counter;  // [3]: phase-2 claims, CTAs finished, spare; zero at launch,
                      // and zero again when the last CTA leaves
  const float2 *tw;   // per-routine pass tables, concatenated
  long long tw_off[kRagRoutines];
  int unnormalized;   // inverse without 1/N
};

// Transform length of routine r.
__device__ __forceinline__ int rag_N(int r) {
#define FFTGB_RAG_N(I, NN, ...) \
  case I:                       \
    return NN;
  switch (r) { FFTGB_RAG_ROUTINES(FFTGB_RAG_N) default: return 16; }
#undef FFTGB_RAG_N
}

// The units a worker takes.  Static (phase 1, rows of 16384, all of equal
// cost): unit first + k * stride at iteration k, no atomics.  Claimed
// (phase 2): the worker's claim k sits in slot k % 3 of a ring in shared
// memory.  Claim i + 1 was written (by the worker's first thread) before the
// barrier that ended iteration i - 1; slot (i + 2) % 3 held claim i - 1,
// which every thread of the worker read before that same barrier, so it may
// be refilled during iteration i.  The atomic is issued at the start of the
// iteration and its result stored into the slot only at the end, so its
// latency hides behind the unit's work.  Claims of a phase are unit indices
// base + counter.
struct RagClaims {
  int *slot;          // shared memory, 3 entries (claimed mode)
  int base, limit;    // the phase's units are [base, limit)
  unsigned *counter;  // the phase's counter; nullptr: static mode
  bool leader;        // the worker's first thread
  int first, stride;  // static mode
  __device__ __forceinline__ int next(int i) const {
    return counter ? slot[(i + 1) % 3] : first + (i + 1) * stride;
  }
  __device__ __forceinline__ int take() const {
    return (counter && leader) ? base + (int)atomicAdd(counter, 1u) : 0;
  }
  __device__ __forceinline__ void put(int i, int c) const {
    if (counter && leader) slot[(i + 2) % 3] = c;
  }
};

// L1 prefetch of one 32-byte-aligned line (a unit or descriptor entry read
// later, after the passes, so that nothing about the next unit stays in
// registers while they run).
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Hook after the first exchange of a unit: the descriptor entry of this
// thread's row of the next unit into L1, and that unit's rows into L2
// through the bulk-copy engine (warp 0 of the worker).  `row0`: the next
// unit's first row, read at the start of the unit (static mode, one row per
// unit); otherwise lane b reads row b's address here (units of up to 32
// rows; longer units of short rows are not prefetched).
struct RagHook {
  const RaggedArgs *A;
  int un, limit, g, wtid;
  const float2 *row0;
  unsigned bytes;
  __device__ __forceinline__ void operator()() const {
    if (un >= limit) return;
    if (row0) {
      if (wtid == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row0), "r"(bytes)
                     : "memory");
      return;
    }
    const RaggedUnit nu = A->units[un];
    if (g < nu.count) prefetch_l1(A->desc + nu.first + g);
    if (nu.count == 1) {  // one row: its offset is in the unit entry
      if (wtid == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A->in + nu.in0),
                     "r"((unsigned)(sizeof(float2) * rag_N(nu.routine)))
                     : "memory");
    } else if (wtid < 32 && nu.count <= 32 && wtid < nu.count) {
      const float2 *row = A->in + A->desc[nu.first + wtid].in_off;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row),
                   "r"((unsigned)(sizeof(float2) * rag_N(nu.routine)))
                   : "memory");
    }
  }
};

// The barrier a worker of W threads ends each unit with: the CTA for W =
// 512, named barrier 9 + worker for a 256-thread half.
template <int W>
__device__ __forceinline__ void rag_worker_sync(int wid) {
  if constexpr (W == kRagThreads) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(9 + wid), "r"(W) : "memory");
}

// All consecutive units of one routine (N, P, TWM, SC) and direction D that
// worker `wid` (W threads, thread wtid) claims, starting with unit u
// (iteration i of its claim sequence): the persistent loop of the plain
// Stockham kernel, with units instead of tiles.  Each unit: the passes, then
// an epilogue that stores the outputs and, when the next claimed unit has
// the same routine and direction, refills each register with that unit's
// input at once.  Returns the first claimed unit of another class (or one
// past the phase's units); `i` advances with the claims.
template <int W, int N, int P, int D, int TWM, class SC>
__device__ __forceinline__ int rag_class(const RaggedArgs &A, float2 *smem, const RagClaims &cl,
                                         int u, int &i, int routine, int wid, int wtid) {
  constexpr int T = N / P;
  constexpr bool PL = pairable<N, P, SC>();
  static_assert(W % T == 0, "rows tile the worker");
  const int g = wtid / T, lt = wtid - g * T;
  float2 a[P];
  {
    const RaggedUnit cu = A.units[u];
    if (g < cu.count) {
      const float2 *src = A.in + A.desc[cu.first + g].in_off;
#pragma unroll
      for (int m = 0; m < P; ++m) a[m] = __ldcs(src + lt + m * T);
    } else {
#pragma unroll
      for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
    }
  }
  while (true) {
    const int un = cl.next(i);
    const int claim = cl.take();
    if (un < cl.limit) prefetch_l1(A.units + un);
    const float2 *row0 = nullptr;  // static mode: the next unit's one row
    if (!cl.counter && wtid == 0 && un < cl.limit) row0 = A.in + A.units[un].in0;
    // Opaque per unit: keeps the table and buffer addresses from being
    // hoisted out of the loop into registers (as in the plain kernel).
    const float2 *twp = A.tw + A.tw_off[routine];
    float2 *bufp = smem + (size_t)g * N;
    int ltp = lt;
    asm volatile("" : "+l"(twp), "+l"(bufp), "+r"(ltp));
    const RagHook hk{&A, un, cl.limit, g, wtid, row0, (unsigned)(sizeof(float2) * N)};
    if constexpr (T == kRagThreads) {
      run_passes_early<N, P, D, SC, 0, TWM, PL>(a, ltp, bufp, twp, hk, NoTw{}, CtaBarrier{});
    } else if constexpr (T >= 64) {
      run_passes_early<N, P, D, SC, 0, TWM, PL>(a, ltp, bufp, twp, hk, NoTw{},
                                                NamedBarrier{1 + wid * 4 + g, T});
    } else {
      run_passes_early<N, P, D, SC, 0, TWM, PL>(a, ltp, bufp, twp, hk, NoTw{}, WarpBarrier{});
    }
    if constexpr (SC::npass == 1) hk();  // no exchange: no hook ran
    // The current and the next unit's descriptors (L1 hits by now).
    const RaggedUnit cu = A.units[u];
    RaggedUnit nu{0, 0, -1, 0};
    if (un < cl.limit) nu = A.units[un];
    const bool active = g < cu.count;
    const bool same = nu.routine == routine && nu.dir == D;
    const bool load_next = same && g < nu.count;
    float2 *dst = A.out + (active ? A.desc[cu.first + g].out_off : 0);
    const float2 *nsrc = A.in + (load_next ? A.desc[nu.first + g].in_off : 0);
    const float s = (D > 0 && !A.unnormalized) ? 1.0f / (float)N : 1.0f;
    if constexpr (PL) {
#pragma unroll
      for (int j = 0; j < P / 2; ++j) {
        if (active) {
          const float2 x = cscale(a[2 * j], s), y = cscale(a[2 * j + 1], s);
          __stcs(reinterpret_cast<float4 *>(dst + final_index_pair<N, P, SC>(ltp, j)),
                 make_float4(x.x, x.y, y.x, y.y));
        }
        if (load_next) {
          a[2 * j] = __ldcs(nsrc + lt + (2 * j) * T);
          a[2 * j + 1] = __ldcs(nsrc + lt + (2 * j + 1) * T);
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < P; ++m) {
        if (active) __stcs(dst + final_index<N, P, SC>(ltp, m), cscale(a[m], s));
        if (load_next) a[m] = __ldcs(nsrc + lt + m * T);
      }
    }
    if (same && !load_next) {
#pragma unroll
      for (int m = 0; m < P; ++m) a[m] = make_float2(0.f, 0.f);
    }
    cl.put(i, claim);
    rag_worker_sync<W>(wid);  // the unit's buffers are free; claim i + 2 is visible
    ++i;
    u = un;
    if (!same) return u;
  }
}

__global__ void __launch_bounds__(kRagThreads, 1) ragged_kernel(RaggedArgs A) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ int ring[2][3];
  const int tid = threadIdx.x;
  // Phase 1: the whole CTA on rows of 16384.
  if (A.nA > 0) {
    const RagClaims cl{nullptr, 0, A.nA, nullptr, tid == 0, (int)blockIdx.x, (int)gridDim.x};
    int u = blockIdx.x, i = 0;
    while (u < A.nA) {
      const RaggedUnit cu = A.units[u];
      switch (cu.routine * 2 + (cu.dir > 0 ? 1 : 0)) {
#define FFTGB_RAG_CASE(I, N, P, TWM, ...)                                                  \
  case 2 * I:                                                                           \
    if constexpr (N == 16384)                                                           \
      u = rag_class<kRagThreads, N, P, -1, TWM, Sched<__VA_ARGS__>>(A, smem, cl, u, i, I, 0, tid); \
    else                                                                                \
      u = A.nA;                                                                         \
    break;                                                                              \
  case 2 * I + 1:                                                                       \
    if constexpr (N == 16384)                                                           \
      u = rag_class<kRagThreads, N, P, +1, TWM, Sched<__VA_ARGS__>>(A, smem, cl, u, i, I, 0, tid); \
    else                                                                                \
      u = A.nA;                                                                         \
    break;
        FFTGB_RAG_ROUTINES(FFTGB_RAG_CASE)
#undef FFTGB_RAG_CASE
        default:
          u = A.nA;  // unreachable: every unit names a compiled routine
      }
    }
    __syncthreads();  // phase 1 done in this CTA: the halves may split
  }
  // Phase 2: two independent 256-thread workers on the other classes.
  const int wid = tid / 256, wtid = tid - wid * 256;
  float2 *wsm = smem + (size_t)wid * 8192;
  if (wtid == 0) {
    ring[wid][0] = A.nA + (int)atomicAdd(A.counter, 1u);
    ring[wid][1] = A.nA + (int)atomicAdd(A.counter, 1u);
  }
  rag_worker_sync<256>(wid);
  const RagClaims cl{ring[wid], A.nA, A.nunits, A.counter, wtid == 0, 0, 0};
  int u = ring[wid][0], i = 0;
  while (u < A.nunits) {
    const RaggedUnit cu = A.units[u];
    switch (cu.routine * 2 + (cu.dir > 0 ? 1 : 0)) {
#define FFTGB_RAG_CASE(I, N, P, TWM, ...)                                                  \
  case 2 * I:                                                                           \
    if constexpr (N != 16384)                                                           \
      u = rag_class<256, N, P, -1, TWM, Sched<__VA_ARGS__>>(A, wsm, cl, u, i, I, wid, wtid); \
    else                                                                                \
      u = A.nunits;                                                                     \
    break;                                                                              \
  case 2 * I + 1:                                                                       \
    if constexpr (N != 16384)                                                           \
      u = rag_class<256, N, P, +1, TWM, Sched<__VA_ARGS__>>(A, wsm, cl, u, i, I, wid, wtid); \
    else                                                                                \
      u = A.nunits;                                                                     \
    break;
      FFTGB_RAG_ROUTINES(FFTGB_RAG_CASE)
#undef FFTGB_RAG_CASE
      default:
        u = A.nunits;  // unreachable: every unit names a compiled routine
    }
  }
  // The last CTA to leave puts the counters back to zero for the next
  // launch: every claim of this launch has been made by then (a worker
  // stops only after a claim past the end), so nothing reads them again.
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(A.counter + 1, 1u) == gridDim.x - 1) {
      A.counter[0] = 0;
      A.counter[1] = 0;
      __threadfence();
    }
  }
}

// FP64-generated pass tables (api.cu).
__global__ void gen_pass_twiddles(float2 *out, int p, int r);

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

// Autotuned routine per class (log2 N, direction), process-wide.
std::mutex g_rag_mu;
std::map<std::pair<int, int>, int> g_rag_choice;

int default_routine(int log2n) {
  for (int i = 0; i < kRagRoutines; ++i)
    if (kRagTable[i].N == (1 << log2n)) return i;  // first listed: built-in
  return -1;
}

}  // namespace

struct RaggedState {
  int count = 0;
  int64_t max_in = 0, max_out = 0;  // elements each packed buffer must hold
  RaggedDesc *d_desc = nullptr;
  RaggedUnit *d_units = nullptr;
  unsigned *d_counter = nullptr;  // [2]
  float2 *d_tw = nullptr;
  RaggedArgs args{};
  int grid = 0;
  int routine_of[kRagMaxLog2 + 1][2];  // chosen routine per (log2 N, direction), -1: absent
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
  cudaFree(r->d_counter);
  cudaFree(r->d_tw);
  delete r;
}

void ragged_destroy(fft_plan_impl *pl) {
  ragged_free(pl->ragged);
  pl->ragged = nullptr;
}

static fft_status_t launch_ragged(const RaggedArgs &args, int grid, cudaStream_t st) {
  RaggedArgs a = args;
  void *p[] = {&a};
  return cuda_status(cudaLaunchKernel((const void *)ragged_kernel, dim3(grid), dim3(kRagThreads),
                                      p, kRagSmem, st));
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
  const fft_status_t e2 = launch_ragged(r->args, r->grid, r->cap);
  const cudaError_t e3 = cudaStreamEndCapture(r->cap, &g);
  if (e2 != FFT_OK || e3 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return FFT_ERR_CUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&r->graph, g, 0);
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

// Units of the rows idx[i0 .. i1) (one class, in order) with routine `rt`.
static void cut_units(std::vector<RaggedUnit> &units, int i0, int i1, int rt, int dir) {
  const int per = rag_rows_per_unit(kRagTable[rt]);
  for (int i = i0; i < i1; i += per) {
    RaggedUnit u;
    u.first = i;
    u.count = std::min(per, i1 - i);
    u.routine = rt;
    u.dir = dir;
    u.in0 = 0;
    units.push_back(u);
  }
}

// Pass tables of every routine, concatenated; offsets per routine.
static fft_status_t build_tables(RaggedState *r) {
  std::vector<std::pair<int, int>> passes;  // (p, r) in table order
  int64_t total = 0;
  for (int i = 0; i < kRagRoutines; ++i) {
    const RagRoutine &rt = kRagTable[i];
    r->args.tw_off[i] = total;
    const int np = rag_npass(rt);
    int p = rt.radix[0];
    for (int k = 1; k < np; ++k) {
      passes.push_back({p, rt.radix[k]});
      total += (int64_t)(rt.radix[k] - 1) * p;
      p *= rt.radix[k];
    }
  }
  if (dev_malloc(&r->d_tw, sizeof(float2) * std::max<int64_t>(1, total)) != cudaSuccess)
    return FFT_ERR_ALLOC;
  int64_t off = 0;
  for (auto &pr : passes) {
    const int64_t n = (int64_t)(pr.second - 1) * pr.first;
    float2 *dst = r->d_tw + off;
    int p = pr.first, rr = pr.second;
    void *args[] = {&dst, &p, &rr};
    if (cudaLaunchKernel((const void *)gen_pass_twiddles, dim3((unsigned)((n + 255) / 256)),
                         dim3(256), args, 0, nullptr) != cudaSuccess)
      return FFT_ERR_CUDA;
    off += n;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

// Time each routine of class (log2n, dir) on `rows` rows of that class packed
// contiguously in scratch buffers; returns the fastest routine.
static int tune_class(RaggedState *r, int log2n, int dir, int rows) {
  const int N = 1 << log2n;
  std::vector<int> cands;
  for (int i = 0; i < kRagRoutines; ++i)
    if (kRagTable[i].N == N) cands.push_back(i);
  if (cands.size() < 2) return cands.empty() ? -1 : cands[0];
  float2 *x = nullptr, *y = nullptr;
  RaggedDesc *dd = nullptr;
  RaggedUnit *du = nullptr;
  unsigned *cnt = nullptr;
  const size_t pts = (size_t)rows * N;
  int best = cands[0];
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (dev_malloc(&x, pts * sizeof(float2)) != cudaSuccess ||
      dev_malloc(&y, pts * sizeof(float2)) != cudaSuccess ||
      dev_malloc(&dd, rows * sizeof(RaggedDesc)) != cudaSuccess ||
      dev_malloc(&du, (rows + 1) * sizeof(RaggedUnit)) != cudaSuccess ||
      dev_malloc(&cnt, 3 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(cnt, 0, 3 * sizeof(unsigned)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    goto done;
  {
    std::vector<RaggedDesc> desc(rows);
    for (int i = 0; i < rows; ++i) desc[i].in_off = desc[i].out_off = (long long)i * N;
    if (cudaMemcpy(dd, desc.data(), rows * sizeof(RaggedDesc), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(x, 0, pts * sizeof(float2)) != cudaSuccess)
      goto done;
    for (int c : cands) {
      std::vector<RaggedUnit> units;
      cut_units(units, 0, rows, c, dir);
      for (auto &un : units) un.in0 = (long long)un.first * N;
      if (cudaMemcpy(du, units.data(), units.size() * sizeof(RaggedUnit),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        goto done;
      RaggedArgs a = r->args;
      a.in = x;
      a.out = y;
      a.desc = dd;
      a.units = du;
      a.nunits = (int)units.size();
      a.nA = N == 16384 ? a.nunits : 0;
      a.counter = cnt;
      const int grid = std::max(1, std::min<int>(r->grid, a.nunits));
      float ms_tot = 0.f;
      const int reps = 5;
      for (int rep = 0; rep < reps + 2; ++rep) {
        if (rep >= 2) cudaEventRecord(e0);
        if (launch_ragged(a, grid, nullptr) != FFT_OK) goto done;
        if (rep >= 2) {
          cudaEventRecord(e1);
          if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          ms_tot += ms;
        }
      }
      if (ms_tot < best_ms) {
        best_ms = ms_tot;
        best = c;
      }
    }
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  cudaFree(dd);
  cudaFree(du);
  cudaFree(cnt);
  return best;
}

int ragged_class_routine(const fft_plan_impl *pl, int N, int dir) {
  const RaggedState *r = pl->ragged;
  if (!r || N < 16 || N > 16384 || (N & (N - 1))) return -1;
  return r->routine_of[__builtin_ctz((unsigned)N)][dir > 0 ? 1 : 0];
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
  if (flags & ~(FFT_FLAG_UNNORMALIZED_INVERSE | FFT_FLAG_NO_AUTOTUNE_CACHE |
                FFT_FLAG_RAGGED_AUTOTUNE))
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
  for (auto &row : r->routine_of) row[0] = row[1] = -1;
  cudaGetDevice(&pl->device);
  auto fail = [&](fft_status_t e) {
    ragged_free(r);
    pl->ragged = nullptr;
    if (pl->d_status) cudaFree(pl->d_status);
    delete h;
    return e;
  };
  if (dev_malloc(&pl->d_status, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_ALLOC);
  if (cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_CUDA);
  if (cudaFuncSetAttribute((const void *)ragged_kernel,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRagSmem) !=
      cudaSuccess)
    return fail(FFT_ERR_CUDA);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess)
    return fail(FFT_ERR_CUDA);
  r->grid = std::max(1, sms);
  fft_status_t st = build_tables(r);
  if (st != FFT_OK) return fail(st);
  r->args.tw = r->d_tw;  // the autotuner's launches below read these tables
  r->args.unnormalized = (flags & FFT_FLAG_UNNORMALIZED_INVERSE) ? 1 : 0;
  // Order: N descending (LPT); within a size, forward before inverse; rows
  // of one (N, direction) keep their order in the caller's list.
  std::vector<int> idx(count);
  for (int i = 0; i < count; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    if (N[x] != N[y]) return N[x] > N[y];
    return direction[x] < direction[y];
  });
  // Routine per class: the autotuner's (timed now if asked), the cache's,
  // or the built-in one.
  std::vector<std::pair<int, int>> cls;  // (start index, end index) of each class
  for (int i = 0; i < count;) {
    int j = i;
    while (j < count && N[idx[j]] == N[idx[i]] && direction[idx[j]] == direction[idx[i]]) ++j;
    cls.push_back({i, j});
    i = j;
  }
  const bool tune = (flags & FFT_FLAG_RAGGED_AUTOTUNE) != 0;
  const bool use_cache = !(flags & FFT_FLAG_NO_AUTOTUNE_CACHE);
  for (auto &c : cls) {
    const int e = __builtin_ctz((unsigned)N[idx[c.first]]);
    const int d = direction[idx[c.first]];
    int rt = default_routine(e);
    if (tune) {
      const int t = tune_class(r, e, d, std::min(c.second - c.first, 1 << (24 - e)));
      if (t >= 0) {
        rt = t;
        std::lock_guard<std::mutex> lk(g_rag_mu);
        g_rag_choice[{e, d}] = t;
      }
    } else if (use_cache) {
      std::lock_guard<std::mutex> lk(g_rag_mu);
      auto it = g_rag_choice.find({e, d});
      if (it != g_rag_choice.end()) rt = it->second;
    }
    r->routine_of[e][d > 0 ? 1 : 0] = rt;
  }
  std::vector<RaggedDesc> desc(count);
  std::vector<RaggedUnit> units;
  for (auto &c : cls) {
    const int e = __builtin_ctz((unsigned)N[idx[c.first]]);
    const int d = direction[idx[c.first]];
    cut_units(units, c.first, c.second, r->routine_of[e][d > 0 ? 1 : 0], d);
  }
  for (auto &un : units) un.in0 = in_offset[idx[un.first]];
  for (int i = 0; i < count; ++i) {
    desc[i].in_off = in_offset[idx[i]];
    desc[i].out_off = out_offset[idx[i]];
    r->max_in = std::max<int64_t>(r->max_in, in_offset[idx[i]] + N[idx[i]]);
    r->max_out = std::max<int64_t>(r->max_out, out_offset[idx[i]] + N[idx[i]]);
  }
  const size_t ub = sizeof(RaggedUnit) * std::max<size_t>(1, units.size());
  if (dev_malloc(&r->d_desc, sizeof(RaggedDesc) * std::max(1, count)) != cudaSuccess ||
      dev_malloc(&r->d_units, ub) != cudaSuccess ||
      dev_malloc(&r->d_counter, 3 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(r->d_counter, 0, 3 * sizeof(unsigned)) != cudaSuccess)
    return fail(FFT_ERR_ALLOC);
  if (count > 0 &&
      (cudaMemcpy(r->d_desc, desc.data(), sizeof(RaggedDesc) * count, cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemcpy(r->d_units, units.data(), sizeof(RaggedUnit) * units.size(),
                  cudaMemcpyHostToDevice) != cudaSuccess))
    return fail(FFT_ERR_CUDA);
  r->grid = std::max(1, std::min<int>(sms, (int)units.size()));
  pl->grid_ctas = r->grid;
  if (cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FFT_ERR_CUDA);
  RaggedArgs &a = r->args;
  a.desc = r->d_desc;
  a.units = r->d_units;
  a.nunits = (int)units.size();
  a.nA = 0;
  while (a.nA < a.nunits && kRagTable[units[a.nA].routine].N == 16384) ++a.nA;
  a.counter = r->d_counter;
  a.tw = r->d_tw;
  *out = h;
  return FFT_OK;
}

// Routine of class N described by `c` (P, radix schedule, twiddle mode).
static int find_routine(int N, const fft_config_t *c) {
  for (int i = 0; i < kRagRoutines; ++i) {
    const RagRoutine &t = kRagTable[i];
    if (t.N != N || t.P != c->points_per_thread || t.twm != c->twiddle_mode ||
        rag_npass(t) != c->num_passes)
      continue;
    bool same = true;
    for (int k = 0; k < c->num_passes; ++k) same = same && t.radix[k] == c->radix[k];
    if (same) return i;
  }
  return -1;
}

static void routine_config(int rt, fft_config_t *config) {
  const RagRoutine &t = kRagTable[rt];
  memset(config, 0, sizeof(*config));
  config->path = FFT_PATH_RAGGED;
  config->points_per_thread = t.P;
  config->transforms_per_cta = rag_rows_per_unit(t);
  config->threads_per_cta = rag_worker(t);  // the worker: whole CTA or a half
  config->num_passes = rag_npass(t);
  for (int i = 0; i < config->num_passes; ++i) config->radix[i] = t.radix[i];
  config->twiddle_mode = t.twm;
  config->ctas_per_sm = 1;
}

namespace fftgb {
void ragged_clear_choices() {
  std::lock_guard<std::mutex> lk(g_rag_mu);
  g_rag_choice.clear();
}
}  // namespace fftgb

extern "C" int fft_ragged_list_configs(int N, fft_config_t *out, int capacity) {
  int n = 0;
  for (int i = 0; i < kRagRoutines; ++i) {
    if (kRagTable[i].N != N) continue;
    if (out && n < capacity) routine_config(i, out + n);
    ++n;
  }
  return n;
}

extern "C" fft_status_t fft_ragged_choose(int N, int direction, const fft_config_t *config) {
  if (!config || (direction != FFT_FORWARD && direction != FFT_INVERSE))
    return FFT_ERR_INVALID_VALUE;
  if (N < 16 || N > 16384 || (N & (N - 1))) return FFT_ERR_INVALID_SIZE;
  const int rt = find_routine(N, config);
  if (rt < 0) return FFT_ERR_NOT_SUPPORTED;
  std::lock_guard<std::mutex> lk(g_rag_mu);
  g_rag_choice[{__builtin_ctz((unsigned)N), direction}] = rt;
  return FFT_OK;
}

extern "C" fft_status_t fft_ragged_class_config(fft_plan_t plan, int N, int direction,
                                                fft_config_t *config) {
  if (!plan || !config || plan->impl.path != FFT_PATH_RAGGED) return FFT_ERR_INVALID_VALUE;
  if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
  const int rt = ragged_class_routine(&plan->impl, N, direction);
  if (rt < 0) return FFT_ERR_INVALID_VALUE;
  routine_config(rt, config);
  return FFT_OK;
}
