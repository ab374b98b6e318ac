// C ABI of libfftgb: planning, twiddle generation and execution.
//
// Planning follows the synthesis rules of the paper (Sec. IV-D) re-derived
// for GB300: a transform whose N points fit one CTA's shared memory (every N
// up to 16384 = 128 KiB, within the 227 KiB a CTA may use) runs as a
// single-CTA Stockham kernel; the two-phase four-step path (Sec. IV-B, Eq. 3)
// splits N = N1 N2 into column FFTs plus twiddle, then row FFTs, through a
// device intermediate; cluster-split rows (cluster.cuh, the four-step with
// N1 = K in one HBM pass) are selectable configurations.  The autotuner's
// cache may override the choice per (N, direction, precision) for
// N <= 16384.
//
// Twiddle tables (Sec. V-A/V-B compute them with a sincos chain; here they are
// precomputed once per plan): every entry W_M^e = exp(-2 pi i e / M) is
// formed on the GPU in FP64 with sincospi(-2 e / M) from the exact integer e,
// then rounded to nearest FP32.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "column.cuh"
#include "fourstep_l2.cuh"
#include "cluster.cuh"
#include "halfio.cuh"
#include "staged.cuh"
#include "tmem2.cuh"
#include "plan.h"

namespace fftgb {

// ---------------------------------------------------------------------------
// Registry
// ---------------------------------------------------------------------------
static std::vector<KernelEntry> &registry_storage() {
  static std::vector<KernelEntry> v;
  return v;
}
void register_kernel(const KernelEntry &e) { registry_storage().push_back(e); }
const std::vector<KernelEntry> &kernel_registry() { return registry_storage(); }

const KernelEntry *find_stockham(int N, int P, int TB, const int *radix, int npass, int twm) {
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_STOCKHAM || e.N != N || e.P != P || e.TB != TB || e.npass != npass ||
        e.twm != twm)
      continue;
    bool same = true;
    for (int i = 0; i < npass; ++i) same = same && e.radix[i] == radix[i];
    if (same) return &e;
  }
  return nullptr;
}

const KernelEntry *find_staged(int N, int P, int C, const int *radix, int npass, int twm) {
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_STAGED || e.N != N || e.P != P || e.slabs != C || e.npass != npass ||
        e.twm != twm)
      continue;
    bool same = true;
    for (int i = 0; i < npass; ++i) same = same && e.radix[i] == radix[i];
    if (same) return &e;
  }
  return nullptr;
}

const KernelEntry *find_split(int N, int K, int P, const int *radix, int npass, int twm) {
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_SPLIT || e.N != N || e.split != K || e.P != P || e.npass != npass ||
        e.twm != twm)
      continue;
    bool same = true;
    for (int i = 0; i < npass; ++i) same = same && e.radix[i] == radix[i];
    if (same) return &e;
  }
  return nullptr;
}

const KernelEntry *find_tmem2(int N, int P, const int *radix, int npass, int twm) {
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_TMEM2 || e.N != N || e.P != P || e.npass != npass || e.twm != twm)
      continue;
    bool same = true;
    for (int i = 0; i < npass; ++i) same = same && e.radix[i] == radix[i];
    if (same) return &e;
  }
  return nullptr;
}

const KernelEntry *default_stockham(int N) {
  const KernelEntry *any = nullptr;
  for (const auto &e : kernel_registry()) {
    if ((e.kind != KIND_STOCKHAM && e.kind != KIND_STAGED && e.kind != KIND_SPLIT) || e.N != N)
      continue;
    if (e.is_default) return &e;
    if (!any && e.kind == KIND_STOCKHAM) any = &e;
  }
  return any;
}

// Column transforms: the longest length (n1 = 4096 rows after a 512-point
// phase 1) and the scratch one pass of a long-column plan may hold (at least
// one matrix).
constexpr int kMaxColumnLength = 1 << 21;
constexpr int64_t kColumnScratchBytes = 1ll << 30;

const KernelEntry *default_column(int L, int variant) {
  for (const auto &e : kernel_registry())
    if (e.kind == KIND_COLUMN && e.N == L && e.variant == variant && e.is_default) return &e;
  return nullptr;
}

fft_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA; }

#define FFTGB_CUDA(call)                                  \
  do {                                                    \
    cudaError_t err__ = (call);                           \
    if (err__ != cudaSuccess) return FFT_ERR_CUDA;        \
  } while (0)

fft_status_t ensure_smem_attr(const KernelEntry *k) {
  if (k->smem > 48 * 1024) {
    for (int d = 0; d < 2; ++d)
      FFTGB_CUDA(cudaFuncSetAttribute(k->fn[d], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)k->smem));
  }
  return FFT_OK;
}

// ---------------------------------------------------------------------------
// Twiddle generation (FP64 on the GPU, rounded to FP32)
// ---------------------------------------------------------------------------
// Pass table: entry (j - 1) * p + k = W_{p r}^{j k}, 1 <= j < r, 0 <= k < p.
__global__ void gen_pass_twiddles(float2 *out, int p, int r) {
  const int64_t total = (int64_t)(r - 1) * p;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t j = idx / p + 1, k = idx % p;
  const int64_t M = (int64_t)p * r;
  const int64_t e = (j * k) % M;
  double s, c;
  sincospi(-2.0 * (double)e / (double)M, &s, &c);
  out[idx] = make_float2(__double2float_rn(c), __double2float_rn(s));
}

// Full table: entry e = W_M^e, 0 <= e < count (count <= M).
__global__ void gen_full_twiddles(float2 *out, int64_t M, int64_t count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double s, c;
  sincospi(-2.0 * (double)e / (double)M, &s, &c);
  out[e] = make_float2(__double2float_rn(c), __double2float_rn(s));
}

// Grid: entry i * cols + c = W_M^{(i step c) mod M}, i * cols + c < count.
__global__ void gen_grid_twiddles(float2 *out, int64_t cols, int64_t step, int64_t M,
                                  int64_t count) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int64_t i = idx / cols, c = idx % cols;
  const int64_t e = ((i * step) % M) * c % M;
  double s, co;
  sincospi(-2.0 * (double)e / (double)M, &s, &co);
  out[idx] = make_float2(__double2float_rn(co), __double2float_rn(s));
}

std::vector<TwSeg> pass_segments(const KernelEntry &k, int64_t &offset) {
  std::vector<TwSeg> segs;
  int p = k.radix[0];
  for (int s = 1; s < k.npass; ++s) {
    TwSeg g;
    g.offset = offset;
    g.count = (int64_t)(k.radix[s] - 1) * p;
    g.kind = 0;
    g.p = p;
    g.r = k.radix[s];
    g.M = (int64_t)p * k.radix[s];
    offset += g.count;
    segs.push_back(g);
    p *= k.radix[s];
  }
  return segs;
}

fft_status_t build_twiddles(fft_plan_impl *pl, const std::vector<TwSeg> &segs) {
  int64_t total = 0;
  for (const auto &g : segs) total = std::max(total, g.offset + g.count);
  pl->tw_segs = segs;
  pl->tw_count = total;
  if (total == 0) return FFT_OK;
  if (dev_malloc(&pl->d_tw, sizeof(float2) * (size_t)total) != cudaSuccess) {
    cudaGetLastError();
    return FFT_ERR_ALLOC;
  }
  for (const auto &g : segs) {
    if (g.count == 0) continue;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.count + threads - 1) / threads);
    if (g.kind == 0)
      gen_pass_twiddles<<<blocks, threads>>>(pl->d_tw + g.offset, g.p, g.r);
    else if (g.kind == 2)
      gen_grid_twiddles<<<blocks, threads>>>(pl->d_tw + g.offset, g.p, g.step, g.M, g.count);
    else
      gen_full_twiddles<<<blocks, threads>>>(pl->d_tw + g.offset, g.M, g.count);
    FFTGB_CUDA(cudaGetLastError());
  }
  FFTGB_CUDA(cudaDeviceSynchronize());
  return FFT_OK;
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
int64_t persistent_grid(const KernelEntry *k, int per_sm) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->fn[0], k->threads, k->smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (occ < 1) occ = 1;
  const int use = (per_sm < 0 || per_sm > occ) ? occ : per_sm;
  return (int64_t)use * sms;
}

// Programmatic stream serialization: the kernel waits (griddepcontrol.wait)
// for the previous kernel of the stream before any global access, so it may
// be launched while that kernel's last CTAs are still running.
cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       void **args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

fft_status_t launch_stockham(const KernelEntry *k, int dir, const float2 *in, float2 *out,
                             const float2 *tw, int64_t rows, float scale, int64_t grid_cap,
                             int64_t ahead, cudaStream_t st) {
  if (rows <= 0) return FFT_OK;
  StockhamArgs a;
  a.in = in;
  a.out = out;
  a.tw = tw;
  a.batch = rows;
  a.scale = scale;
  int64_t grid = (rows + k->TB - 1) / k->TB;
  a.ahead = grid_cap > 0 && grid > grid_cap ? 0 : ahead;  // one tile per CTA only
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  void *args[] = {&a};
  FFTGB_CUDA(launch_pdl(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads), k->smem,
                        st, args));
  return FFT_OK;
}

static fft_status_t launch_staged(const KernelEntry *k, int dir, const float2 *in, float2 *out,
                                  const float2 *tw, int64_t rows, float scale, int64_t grid,
                                  int *status, cudaStream_t st) {
  if (rows <= 0) return FFT_OK;
  StagedArgs a;
  a.in = in;
  a.out = out;
  a.tw = tw;
  a.batch = rows;
  a.scale = scale;
  a.status = status;
  if (grid <= 0 || grid > rows) grid = rows;
  void *args[] = {&a};
  FFTGB_CUDA(cudaLaunchKernel(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads),
                              args, k->smem, st));
  return FFT_OK;
}

// Clusters of K CTAs that can be resident at once (0 if the query fails).
static int64_t resident_clusters(const KernelEntry *k) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)k->split;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)k->split);
  cfg.blockDim = dim3((unsigned)k->threads);
  cfg.dynamicSmemBytes = k->smem;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k->fn[0], &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

static fft_status_t launch_split(const KernelEntry *k, int dir, const float2 *in, float2 *out,
                                 const float2 *tw, const float2 *tw_n, int64_t rows,
                                 float scale, int64_t clusters, cudaStream_t st) {
  if (rows <= 0) return FFT_OK;
  SplitArgs a;
  a.in = in;
  a.out = out;
  a.tw = tw;
  a.tw_n = tw_n;
  a.batch = rows;
  a.scale = scale;
  const int64_t grid = (int64_t)k->split * (clusters > 0 && clusters < rows ? clusters : rows);
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  void *args[] = {&a};
  FFTGB_CUDA(cudaLaunchKernel(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads),
                              args, k->smem, st));
  return FFT_OK;
}

static fft_status_t launch_tmem2(const KernelEntry *k, int dir, const float2 *in, float2 *out,
                                 const float2 *tw, const float2 *tw_n, int64_t rows, float scale,
                                 int64_t grid_cap, int *status, cudaStream_t st) {
  if (rows <= 0) return FFT_OK;
  Tmem2Args a;
  a.in = in;
  a.out = out;
  a.tw = tw;
  a.tw_n = tw_n;
  a.batch = rows;
  a.scale = scale;
  a.status = status;
  a.out32 = ((uintptr_t)out & 31) == 0;
  if (rows > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;  // the kernel indexes rows in 32 bits
  const int64_t grid = grid_cap > 0 && grid_cap < rows ? grid_cap : rows;
  void *args[] = {&a};
  FFTGB_CUDA(launch_pdl(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads), k->smem,
                        st, args));
  return FFT_OK;
}

fft_status_t launch_column(const KernelEntry *k, int dir, const ColumnArgs &ca,
                           cudaStream_t st) {
  const int64_t grid = ca.nmat * (ca.ncols / k->TB);
  if (grid <= 0) return FFT_OK;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  ColumnArgs a = ca;
  void *args[] = {&a};
  // Programmatic dependent launch up to 2048-point columns (the kernels that
  // carry the griddepcontrol instructions); the 4096-point column kernels (one
  // CTA of 128 KiB per SM) measured 1-4 % slower with it.
  if (k->N <= 2048) {
    FFTGB_CUDA(launch_pdl(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads),
                          k->smem, st, args));
  } else {
    FFTGB_CUDA(cudaLaunchKernel(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads),
                                args, k->smem, st));
  }
  return FFT_OK;
}

// Single-launch four-step (fourstep_l2.cuh).  Batches whose work-item count
// would pass 2^30 run as several launches of whole chunks.
static fft_status_t launch_fourstep_l2(fft_plan_impl *pl, const float2 *in, float2 *out,
                                       int64_t rows, cudaStream_t st) {
  const KernelEntry *k = pl->k_l2;
  const int64_t R = pl->l2_rows;
  const int64_t tiles_per_row = pl->n1 / k->TB;
  const int64_t max_chunks = std::max<int64_t>(1, (1ll << 29) / (R * tiles_per_row)) - pl->l2_lag;
  if (max_chunks < 1) return FFT_ERR_INVALID_SIZE;
  for (int64_t r0 = 0; r0 < rows; r0 += max_chunks * R) {
    const int64_t nr = std::min(max_chunks * R, rows - r0);
    FourstepL2Args a;
    a.in = in + r0 * pl->N;
    a.out = out + r0 * pl->N;
    a.ring = pl->d_scratch;
    a.tw = pl->d_tw + pl->tw_col1;
    a.tw_a = pl->d_tw + pl->tw_big;
    a.tw_b = pl->d_tw + pl->tw_big2;
    a.counters = pl->d_l2cnt;
    a.status = pl->d_status;
    a.batch = nr;
    a.chunk_rows = (int)R;
    a.nchunks = (int)((nr + R - 1) / R);
    a.slots = std::min(pl->l2_slots, a.nchunks);
    a.lag = pl->l2_lag;
    a.scale = pl->scale;
    const int64_t items = (int64_t)(a.nchunks + a.lag) * 2 * R * tiles_per_row;
    const int64_t grid = std::min(pl->l2_grid, items);
    void *args[] = {&a};
    FFTGB_CUDA(cudaLaunchKernel(k->fn[pl->direction > 0 ? 1 : 0], dim3((unsigned)grid),
                                dim3(k->threads), args, k->smem, st));
  }
  return FFT_OK;
}

fft_status_t exec_rows(fft_plan_impl *pl, const float2 *in, float2 *out, int64_t rows,
                       cudaStream_t st) {
  if (rows <= 0) return FFT_OK;
  if (pl->path == FFT_PATH_TMEM_HALVES) {
    return launch_tmem2(pl->k_single, pl->direction, in, out, pl->d_tw + pl->tw_single,
                        pl->d_tw + pl->tw_big, rows, pl->scale, pl->grid_ctas, pl->d_status,
                        st);
  }
  if (pl->path == FFT_PATH_SINGLE_CTA && pl->k_single->kind == KIND_SPLIT) {
    return launch_split(pl->k_single, pl->direction, in, out, pl->d_tw + pl->tw_single,
                        pl->d_tw + pl->tw_big, rows, pl->scale, pl->grid_ctas / pl->k_single->split,
                        st);
  }
  if (pl->path == FFT_PATH_SINGLE_CTA && pl->k_single->kind == KIND_HALFIO) {
    HalfArgs a;
    a.in = in;    // FP16 or BF16 pairs, per the kernel's variant
    a.out = out;
    a.tw = pl->d_tw + pl->tw_single;
    a.batch = rows;
    a.scale = pl->scale;
    const int64_t grid = (rows + pl->k_single->TB - 1) / pl->k_single->TB;
    if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
    void *args[] = {&a};
    FFTGB_CUDA(cudaLaunchKernel(pl->k_single->fn[pl->direction > 0 ? 1 : 0], dim3((unsigned)grid),
                                dim3(pl->k_single->threads), args, pl->k_single->smem, st));
    return FFT_OK;
  }
  if (pl->path == FFT_PATH_SINGLE_CTA && pl->k_single->kind == KIND_STAGED) {
    return launch_staged(pl->k_single, pl->direction, in, out, pl->d_tw + pl->tw_single, rows,
                         pl->scale, pl->grid_ctas, pl->d_status, st);
  }
  if (pl->path == FFT_PATH_SINGLE_CTA) {
    return launch_stockham(pl->k_single, pl->direction, in, out, pl->d_tw + pl->tw_single, rows,
                           pl->scale, pl->grid_ctas, pl->resident_ctas, st);
  }
  if (pl->path == FFT_PATH_FOURSTEP && pl->k_l2) return launch_fourstep_l2(pl, in, out, rows, st);
  if (pl->path == FFT_PATH_FOURSTEP) {
    ColumnArgs c1{};
    c1.in = in;
    c1.out = pl->d_scratch;
    c1.tw = pl->d_tw + pl->tw_col1;
    c1.tw_a = pl->d_tw + pl->tw_big;
    c1.tw_b = pl->d_tw + pl->tw_big2;
    c1.nmat = rows;
    c1.in_mat_stride = pl->N;
    c1.out_mat_stride = pl->N;
    c1.in_row_stride = pl->n1;
    c1.out_row_stride = 0;
    c1.ncols = pl->n1;
    c1.ntot = pl->N;
    c1.scale = 1.f;
    c1.in_extent = c1.out_extent = rows * pl->N;
    fft_status_t s = launch_column(pl->k_col1, pl->direction, c1, st);
    if (s != FFT_OK) return s;
    ColumnArgs c2{};
    c2.in = pl->d_scratch;
    c2.out = out;
    c2.tw = pl->d_tw + pl->tw_col2;
    c2.tw_a = c2.tw_b = nullptr;
    c2.nmat = rows;
    c2.in_mat_stride = pl->N;
    c2.out_mat_stride = pl->N;
    c2.in_row_stride = pl->n2;
    c2.out_row_stride = pl->n2;
    c2.ncols = pl->n2;
    c2.ntot = pl->N;
    c2.scale = pl->scale;
    c2.in_extent = c2.out_extent = rows * pl->N;
    return launch_column(pl->k_col2, pl->direction, c2, st);
  }
  if (pl->path == FFT_PATH_TENSORCORE) return tc_exec(pl, in, out, rows, st);
  return FFT_ERR_INVALID_VALUE;
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Bytes per stored point: 8 (complex64), 4 for FP16 storage.
static int64_t elem_bytes(const fft_plan_impl *pl) {
  return (pl->precision == FFT_PREC_FP16_STORAGE || pl->precision == FFT_PREC_BF16_STORAGE)
             ? 4
             : (int64_t)sizeof(float2);
}

// Largest N: single CTA (the whole row in registers + shared memory), and
// overall (two-phase four-step: phase 1 <= 256 points, phase 2 <= 4096).
constexpr int kMaxSingleN = 16384;
constexpr int kMaxN = 1 << 20;

// Built-in launch shape of the single-CTA path: one CTA per tile, measured
// faster than the persistent shape for every N up to 8192 on GB300; at
// N = 16384 (one row per SM) the persistent shape with L2 prefetch of the
// next row is faster (~134 against ~150 µs per 2^25 points).
constexpr int kDefaultCtasPerSm = 0;
static int default_ctas_per_sm(int N) { return N >= 16384 ? -1 : kDefaultCtasPerSm; }

// Four-step split N = n1 * n2: n2 (phase 1) a length with a twiddle +
// transposed-store column kernel (16..512), n1 (phase 2) a length with a
// plain column kernel (16..4096).
static bool fourstep_split(int N, int want_n1, int *n1, int *n2) {
  auto ok = [&](int a) {
    const int b = N / a;
    return a >= 16 && b >= 16 && default_column(b, 1) && default_column(a, 0);
  };
  if (want_n1 > 0) {
    if (N % want_n1 || !ok(want_n1)) return false;
    *n1 = want_n1;
    *n2 = N / want_n1;
    return true;
  }
  // Prefer n2 >= n1 (longer first-phase transforms), as square as possible,
  // with phase 1 at most 256 points up to N = 2^17 and 512 beyond, where the
  // 512-point phase 1 costs less than a phase 2 of 2048 or 4096 points
  // (measured over 2^25 points: 2^17 512 x 256 181 us against 256 x 512
  // 190 us; 2^20 2048 x 512 256 us against 4096 x 256 277 us).
  const int cap = N >= (1 << 18) ? 512 : 256;
  int best = 0;
  for (int a = 16; a <= 4096 && a <= N; a *= 2)
    if (N % a == 0 && ok(a) && a <= N / a && N / a <= cap) best = a;
  for (int a = 16; !best && a <= 4096 && a <= N; a *= 2)
    if (N % a == 0 && ok(a) && N / a <= cap) best = a;
  if (!best) return false;
  *n1 = best;
  *n2 = N / best;
  return true;
}

// Largest chunk of the single-launch four-step (rows per chunk).
constexpr int kMaxL2Rows = 4096;

// Ring geometry of the single-launch four-step.  Claims run one item ahead
// of the work, so up to F = 2 * grid items are claimed but unfinished.  A
// phase-2 tile of chunk c is claimed l2_lag rounds after chunk c's phase-1
// tiles, and a phase-1 tile of chunk c reuses the slot of chunk c - slots,
// whose phase-2 tiles were claimed slots - lag rounds earlier; both distances
// are F items plus a round of margin, so neither wait normally spins.
// Deadlock freedom needs slots > lag.
static void l2_geometry(fft_plan_impl *pl) {
  const int64_t round = 2 * (int64_t)pl->l2_rows * (pl->n1 / pl->k_l2->TB);
  const int64_t f = 2 * std::max<int64_t>(1, pl->l2_grid);
  const int d = (int)((f + round - 1) / round) + 1;
  pl->l2_lag = d;
  pl->l2_slots = 2 * d;
}

static fft_status_t plan_fourstep(fft_plan_impl *pl, int want_n1, int l2_rows) {
  int n1, n2;
  if (!fourstep_split(pl->N, want_n1, &n1, &n2)) return FFT_ERR_NOT_SUPPORTED;
  if (l2_rows < 0 || l2_rows > kMaxL2Rows) return FFT_ERR_INVALID_VALUE;
  pl->path = FFT_PATH_FOURSTEP;
  pl->n1 = n1;
  pl->n2 = n2;
  int64_t off = 0;
  std::vector<TwSeg> segs;
  fft_status_t s = FFT_OK;
  if (l2_rows > 0) {
    if (n1 != n2) return FFT_ERR_NOT_SUPPORTED;
    for (const auto &e : kernel_registry())
      if (e.kind == KIND_FOURSTEP_L2 && e.N == n1) pl->k_l2 = &e;
    if (!pl->k_l2) return FFT_ERR_NOT_SUPPORTED;
    s = ensure_smem_attr(pl->k_l2);
    if (s != FFT_OK) return s;
    pl->l2_rows = l2_rows;
    pl->l2_grid = persistent_grid(pl->k_l2, -1);
    if (pl->l2_grid <= 0) return FFT_ERR_CUDA;
    l2_geometry(pl);
    pl->tw_col1 = pl->tw_col2 = off;
    auto a = pass_segments(*pl->k_l2, off);
    segs.insert(segs.end(), a.begin(), a.end());
  } else {
    pl->k_col1 = default_column(n2, 1);
    pl->k_col2 = default_column(n1, 0);
    s = ensure_smem_attr(pl->k_col1);
    if (s == FFT_OK) s = ensure_smem_attr(pl->k_col2);
    if (s != FFT_OK) return s;
    pl->tw_col1 = off;
    auto a = pass_segments(*pl->k_col1, off);
    segs.insert(segs.end(), a.begin(), a.end());
    pl->tw_col2 = off;
    auto b = pass_segments(*pl->k_col2, off);
    segs.insert(segs.end(), b.begin(), b.end());
  }
  pl->tw_big = off;
  {  // phase-1 twiddle: W_N^{c lt} [lt][c] and W_N^{c T m} [m][c] (column.cuh)
    const int P1 = pl->k_l2 ? pl->k_l2->P : pl->k_col1->P, T1 = n2 / P1;
    TwSeg ga;
    ga.offset = off;
    ga.kind = 2;
    ga.p = n1;
    ga.r = 0;
    ga.step = 1;
    ga.M = pl->N;
    ga.count = (int64_t)T1 * n1;
    off += ga.count;
    segs.push_back(ga);
    TwSeg gb = ga;
    gb.offset = off;
    gb.step = T1;
    gb.count = (int64_t)P1 * n1;
    pl->tw_big2 = off;
    off += gb.count;
    segs.push_back(gb);
  }
  s = build_twiddles(pl, segs);
  if (s != FFT_OK) return s;
  if (pl->k_l2) {
    // ring slots (no more than the batch has chunks) + the launch counters
    const int64_t nch = (pl->batch + l2_rows - 1) / l2_rows;
    const int64_t slots = std::min<int64_t>(pl->l2_slots, nch);
    pl->scratch_bytes = (int64_t)sizeof(float2) * pl->N * l2_rows * slots;
    const int64_t ncnt = 2 + 2 * std::max<int64_t>(nch, 1);
    if (dev_malloc(&pl->d_l2cnt, sizeof(unsigned) * (size_t)ncnt) != cudaSuccess) {
      cudaGetLastError();
      return FFT_ERR_ALLOC;
    }
    if (cudaMemset(pl->d_l2cnt, 0, sizeof(unsigned) * (size_t)ncnt) != cudaSuccess)
      return FFT_ERR_CUDA;
  } else {
    pl->scratch_bytes = (int64_t)sizeof(float2) * pl->N * pl->batch;
  }
  if (pl->scratch_bytes > 0) {
    if (dev_malloc(&pl->d_scratch, (size_t)pl->scratch_bytes) != cudaSuccess) {
      cudaGetLastError();
      return FFT_ERR_ALLOC;
    }
  }
  return FFT_OK;
}

static fft_status_t plan_single(fft_plan_impl *pl, const KernelEntry *k, int ctas_per_sm) {
  if (!k) return FFT_ERR_NOT_SUPPORTED;
  pl->path = k->kind == KIND_TMEM2 ? FFT_PATH_TMEM_HALVES : FFT_PATH_SINGLE_CTA;
  pl->k_single = k;
  fft_status_t s = ensure_smem_attr(k);
  if (s != FFT_OK) return s;
  if (k->kind == KIND_STAGED || k->kind == KIND_TMEM2) ctas_per_sm = 1;  // one per SM by design
  pl->ctas_per_sm = k->kind == KIND_SPLIT ? -1 : ctas_per_sm;
  // One-tile-per-CTA plain kernels from 4096 points on prefetch one resident
  // wave ahead (measured back to back: 8192 94.6 -> 89.8 us, 4096 -1.5 %);
  // the shorter rows are HBM-bound already and measured 3-5 % slower with it.
  pl->resident_ctas = k->kind == KIND_STOCKHAM && ctas_per_sm == 0 && k->N >= 4096
                          ? persistent_grid(k, -1)
                          : 0;
  pl->grid_ctas = k->kind == KIND_SPLIT ? k->split * resident_clusters(k)  // persistent clusters
                  : ctas_per_sm != 0   ? persistent_grid(k, ctas_per_sm)
                                       : 0;
  int64_t off = 0;
  pl->tw_single = 0;
  auto segs = pass_segments(*k, off);
  if (k->kind == KIND_TMEM2) {  // + W_N^t, t < threads, the split's per-thread root
    TwSeg g;
    g.offset = off;
    g.count = k->threads;
    g.kind = 1;
    g.p = g.r = 0;
    g.M = pl->N;
    pl->tw_big = off;
    segs.push_back(g);
  }
  if (k->kind == KIND_SPLIT) {  // + W_N^{r k2} at (r - 1) H + k2 for the cluster combine
    TwSeg g;
    g.offset = off;
    g.p = pl->N / k->split;
    g.r = k->split;
    g.count = (int64_t)(g.r - 1) * g.p;
    g.kind = 0;
    g.M = pl->N;
    pl->tw_big = off;
    segs.push_back(g);
  }
  return build_twiddles(pl, segs);
}

// Columns longer than 4096 (L = n1 n2, column.cuh): per chunk of matrices,
// phase 1 (n2-point columns of the n1 sub-matrices, twiddled) into the
// compact scratch [row n1 + n1_count k2][col], then phase 2 (n1-point columns
// of the n2 sub-matrices) into the caller's layout at rows k2 + n2 k1.
static fft_status_t exec_long_columns(fft_plan_impl *pl, const float2 *in, float2 *out,
                                      cudaStream_t st) {
  const int64_t L = pl->N, n1 = pl->n1, n2 = pl->n2, nc = pl->col_ncols;
  const int64_t rs = pl->col_row_stride, ms = pl->col_mat_stride;
  for (int64_t m0 = 0; m0 < pl->col_nmat; m0 += pl->col_chunk) {
    const int64_t nm = std::min(pl->col_chunk, pl->col_nmat - m0);
    const int64_t user_extent = (nm - 1) * ms + (L - 1) * rs + nc;  // elements of this chunk
    ColumnArgs c1{};
    c1.in = in + m0 * ms;
    c1.out = pl->d_scratch;
    c1.tw = pl->d_tw + pl->tw_col1;
    c1.tw_a = pl->d_tw + pl->tw_big;
    c1.nmat = nm * n1;
    c1.nsub = (int)n1;
    c1.in_mat_stride = ms;
    c1.in_sub_stride = rs;
    c1.in_row_stride = (int)(n1 * rs);
    c1.out_mat_stride = L * nc;
    c1.out_sub_stride = nc;
    c1.out_row_stride = (int)(n1 * nc);
    c1.ncols = (int)nc;
    c1.ntot = (int)L;
    c1.scale = 1.0f;
    c1.in_extent = user_extent;
    c1.out_extent = nm * L * nc;
    fft_status_t s = launch_column(pl->k_col1, pl->direction, c1, st);
    if (s != FFT_OK) return s;
    ColumnArgs c2{};
    c2.in = pl->d_scratch;
    c2.out = out + m0 * ms;
    c2.tw = pl->d_tw + pl->tw_col2;
    c2.nmat = nm * n2;
    c2.nsub = (int)n2;
    c2.in_mat_stride = L * nc;
    c2.in_sub_stride = n1 * nc;
    c2.in_row_stride = (int)nc;
    c2.out_mat_stride = ms;
    c2.out_sub_stride = rs;
    c2.out_row_stride = (int)(n2 * rs);
    c2.ncols = (int)nc;
    c2.ntot = (int)L;
    c2.scale = pl->scale;
    c2.in_extent = nm * L * nc;
    c2.out_extent = user_extent;
    s = launch_column(pl->k_col2, pl->direction, c2, st);
    if (s != FFT_OK) return s;
  }
  return FFT_OK;
}

static void free_plan(fft_plan_impl *pl) {
  if (!pl) return;
  if (pl->ragged) ragged_destroy(pl);
  if (pl->filter) filter_destroy(pl);
  if (pl->tc) tc_destroy(pl);
  if (pl->d_tw) cudaFree(pl->d_tw);
  if (pl->d_scratch) cudaFree(pl->d_scratch);
  if (pl->d_l2cnt) cudaFree(pl->d_l2cnt);
  if (pl->d_status) cudaFree(pl->d_status);
  if (pl->d_stage) cudaFree(pl->d_stage);
  if (pl->s_h2d) cudaStreamDestroy(pl->s_h2d);
  if (pl->s_d2h) cudaStreamDestroy(pl->s_d2h);
}

}  // namespace fftgb

using namespace fftgb;

extern "C" {

const char *fft_status_string(fft_status_t s) {
  switch (s) {
    case FFT_OK: return "FFT_OK";
    case FFT_ERR_INVALID_SIZE: return "FFT_ERR_INVALID_SIZE";
    case FFT_ERR_INVALID_VALUE: return "FFT_ERR_INVALID_VALUE";
    case FFT_ERR_MISALIGNED: return "FFT_ERR_MISALIGNED";
    case FFT_ERR_ALLOC: return "FFT_ERR_ALLOC";
    case FFT_ERR_CUDA: return "FFT_ERR_CUDA";
    case FFT_ERR_TIMEOUT: return "FFT_ERR_TIMEOUT";
    case FFT_ERR_NOT_SUPPORTED: return "FFT_ERR_NOT_SUPPORTED";
  }
  return "FFT_ERR_UNKNOWN";
}

static fft_status_t plan_common(fft_plan_t *out, int N, int64_t batch, int direction,
                                int precision, int flags, const fft_config_t *cfg) {
  if (!out) return FFT_ERR_INVALID_VALUE;
  *out = nullptr;
  if (!is_pow2(N) || N < 2 || N > kMaxN || batch < 0) return FFT_ERR_INVALID_SIZE;
  if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
  if (precision < FFT_PREC_FP32 || precision > FFT_PREC_BF16_STORAGE) return FFT_ERR_INVALID_VALUE;
  if (flags & ~(FFT_FLAG_UNNORMALIZED_INVERSE | FFT_FLAG_FORCE_SINGLE_CTA |
                FFT_FLAG_FORCE_FOURSTEP | FFT_FLAG_NO_AUTOTUNE_CACHE | FFT_FLAG_ADJOINT))
    return FFT_ERR_INVALID_VALUE;
  if ((flags & FFT_FLAG_FORCE_SINGLE_CTA) && (flags & FFT_FLAG_FORCE_FOURSTEP))
    return FFT_ERR_INVALID_VALUE;
  if (cfg && (cfg->l2_chunk_rows < 0 || cfg->l2_chunk_rows > kMaxL2Rows ||
              (cfg->l2_chunk_rows > 0 && cfg->path != FFT_PATH_FOURSTEP)))
    return FFT_ERR_INVALID_VALUE;
  // Beyond one CTA's reach (N > 16384): a built-in one-pass configuration
  // where one exists and was measured faster (a row on one SM with half of
  // it in tensor memory, or on a cluster of CTAs), else the two-phase
  // four-step (synthesis rule 3 of Sec. IV-D, one level: N = n1 * n2,
  // n2 <= 256, n1 <= 4096).
  const KernelEntry *big_default = nullptr;
  if (N > kMaxSingleN) {
    if (precision != FFT_PREC_FP32 || (flags & FFT_FLAG_FORCE_SINGLE_CTA))
      return FFT_ERR_NOT_SUPPORTED;
    const bool split = cfg && ((cfg->path == FFT_PATH_SINGLE_CTA && cfg->cluster_split > 0) ||
                               cfg->path == FFT_PATH_TMEM_HALVES);
    if (cfg && cfg->path != FFT_PATH_FOURSTEP && !split) return FFT_ERR_NOT_SUPPORTED;
    if (!cfg && !(flags & FFT_FLAG_FORCE_FOURSTEP)) {
      for (const auto &e : kernel_registry())
        if ((e.kind == KIND_SPLIT || e.kind == KIND_TMEM2) && e.N == N && e.is_default)
          big_default = &e;
    }
    if (!split && !big_default) flags |= FFT_FLAG_FORCE_FOURSTEP;
  }
  fft_plan_s *h = new (std::nothrow) fft_plan_s;
  if (!h) return FFT_ERR_ALLOC;
  fft_plan_impl *pl = &h->impl;
  pl->N = N;
  pl->batch = batch;
  pl->precision = precision;
  pl->flags = flags;
  {
    // Kernel direction and output scale.  The adjoint of F is F^H (sign +1,
    // scale 1); the adjoint of G = F^H / N is F / N (sign -1, scale 1/N).
    const bool scaled_inverse = !(flags & FFT_FLAG_UNNORMALIZED_INVERSE);
    if (flags & FFT_FLAG_ADJOINT) {
      pl->direction = -direction;
      pl->scale = (direction == FFT_INVERSE && scaled_inverse) ? 1.0f / (float)N : 1.0f;
    } else {
      pl->direction = direction;
      pl->scale = (direction == FFT_INVERSE && scaled_inverse) ? 1.0f / (float)N : 1.0f;
    }
  }
  cudaGetDevice(&pl->device);
  fft_status_t s = FFT_OK;
  if (dev_malloc(&pl->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    s = FFT_ERR_ALLOC;
  } else if (cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) {
    s = FFT_ERR_CUDA;
  }
  if (s == FFT_OK) {
    if (cfg) {
      if (cfg->path == FFT_PATH_FOURSTEP) {
        s = plan_fourstep(pl, cfg->n1, cfg->l2_chunk_rows);
      } else if (cfg->path == FFT_PATH_TMEM_HALVES) {
        const KernelEntry *k = find_tmem2(N, cfg->points_per_thread, cfg->radix,
                                          cfg->num_passes, cfg->twiddle_mode);
        s = k ? plan_single(pl, k, -1) : FFT_ERR_NOT_SUPPORTED;
      } else if (cfg->path == FFT_PATH_SINGLE_CTA) {
        const KernelEntry *k =
            cfg->cluster_split > 0
                ? find_split(N, cfg->cluster_split, cfg->points_per_thread, cfg->radix,
                             cfg->num_passes, cfg->twiddle_mode)
            : cfg->tma_slabs > 0
                ? find_staged(N, cfg->points_per_thread, cfg->tma_slabs, cfg->radix,
                              cfg->num_passes, cfg->twiddle_mode)
                : find_stockham(N, cfg->points_per_thread, cfg->transforms_per_cta, cfg->radix,
                                cfg->num_passes, cfg->twiddle_mode);
        s = k ? plan_single(pl, k, cfg->ctas_per_sm) : FFT_ERR_NOT_SUPPORTED;
      } else {
        s = FFT_ERR_INVALID_VALUE;
      }
    } else if (precision == FFT_PREC_FP16_STORAGE || precision == FFT_PREC_BF16_STORAGE) {
      const int variant = precision == FFT_PREC_BF16_STORAGE ? 1 : 0;
      const KernelEntry *k = nullptr;
      for (const auto &e : kernel_registry())
        if (e.kind == KIND_HALFIO && e.N == N && e.variant == variant) k = &e;
      s = k ? plan_single(pl, k, 0) : FFT_ERR_NOT_SUPPORTED;
    } else if (precision != FFT_PREC_FP32) {
      s = tc_plan(pl);
    } else if (big_default) {
      s = plan_single(pl, big_default, -1);
    } else if (flags & FFT_FLAG_FORCE_FOURSTEP) {
      s = plan_fourstep(pl, 0, 0);
    } else if (flags & FFT_FLAG_FORCE_SINGLE_CTA) {
      s = plan_single(pl, default_stockham(N), default_ctas_per_sm(N));
    } else {
      TuneChoice tc;
      bool have = !(flags & FFT_FLAG_NO_AUTOTUNE_CACHE) &&
                  tune_lookup(N, pl->direction, precision, &tc);
      if (have && tc.path == FFT_PATH_FOURSTEP) {
        s = plan_fourstep(pl, tc.n1, tc.l2rows);
        if (s == FFT_ERR_NOT_SUPPORTED) have = false;
      } else if (have) {
        const KernelEntry *k =
            tc.split > 0   ? find_split(N, tc.split, tc.P, tc.radix, tc.npass, tc.twm)
            : tc.slabs > 0 ? find_staged(N, tc.P, tc.slabs, tc.radix, tc.npass, tc.twm)
                           : find_stockham(N, tc.P, tc.TB, tc.radix, tc.npass, tc.twm);
        if (k) s = plan_single(pl, k, tc.ctas_per_sm);
        else have = false;
      }
      if (!have) s = plan_single(pl, default_stockham(N), default_ctas_per_sm(N));
    }
  }
  if (s != FFT_OK) {
    free_plan(pl);
    delete h;
    return s;
  }
  *out = h;
  return FFT_OK;
}

fft_status_t fft_plan_ex(fft_plan_t *out, int N, int64_t batch, int direction, int precision,
                         int flags) {
  return plan_common(out, N, batch, direction, precision, flags, nullptr);
}

fft_status_t fft_plan(fft_plan_t *out, int N, int64_t batch, int direction) {
  return plan_common(out, N, batch, direction, FFT_PREC_FP32, 0, nullptr);
}

fft_status_t fft_plan_config(fft_plan_t *out, int N, int64_t batch, int direction, int flags,
                             const fft_config_t *config) {
  if (out) *out = nullptr;
  if (!config) return FFT_ERR_INVALID_VALUE;
  if (flags & (FFT_FLAG_FORCE_SINGLE_CTA | FFT_FLAG_FORCE_FOURSTEP)) return FFT_ERR_INVALID_VALUE;
  return plan_common(out, N, batch, direction, FFT_PREC_FP32, flags, config);
}

int fft_list_configs(int N, fft_config_t *out, int capacity) {
  int n = 0;
  auto emit = [&](const fft_config_t &c) {
    if (out && n < capacity) out[n] = c;
    ++n;
  };
  if (!is_pow2(N) || N < 2 || N > kMaxN) return 0;
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_STOCKHAM || e.N != N) continue;
    for (int shape : {0, -1}) {
      fft_config_t c;
      memset(&c, 0, sizeof(c));
      c.path = FFT_PATH_SINGLE_CTA;
      c.points_per_thread = e.P;
      c.transforms_per_cta = e.TB;
      c.threads_per_cta = e.threads;
      c.num_passes = e.npass;
      for (int i = 0; i < 8; ++i) c.radix[i] = e.radix[i];
      c.twiddle_mode = e.twm;
      c.ctas_per_sm = shape;
      emit(c);
    }
  }
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_SPLIT || e.N != N) continue;
    fft_config_t c;
    memset(&c, 0, sizeof(c));
    c.path = FFT_PATH_SINGLE_CTA;
    c.points_per_thread = e.P;
    c.transforms_per_cta = 1;
    c.threads_per_cta = e.threads;
    c.num_passes = e.npass;
    for (int i = 0; i < 8; ++i) c.radix[i] = e.radix[i];
    c.twiddle_mode = e.twm;
    c.cluster_split = e.split;
    c.ctas_per_sm = -1;
    emit(c);
  }
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_TMEM2 || e.N != N) continue;
    fft_config_t c;
    memset(&c, 0, sizeof(c));
    c.path = FFT_PATH_TMEM_HALVES;
    c.points_per_thread = e.P;
    c.transforms_per_cta = 1;
    c.threads_per_cta = e.threads;
    c.num_passes = e.npass;
    for (int i = 0; i < 8; ++i) c.radix[i] = e.radix[i];
    c.twiddle_mode = e.twm;
    c.ctas_per_sm = 1;
    emit(c);
  }
  for (const auto &e : kernel_registry()) {
    if (e.kind != KIND_STAGED || e.N != N) continue;
    fft_config_t c;
    memset(&c, 0, sizeof(c));
    c.path = FFT_PATH_SINGLE_CTA;
    c.points_per_thread = e.P;
    c.transforms_per_cta = 1;
    c.threads_per_cta = e.threads;
    c.num_passes = e.npass;
    for (int i = 0; i < 8; ++i) c.radix[i] = e.radix[i];
    c.twiddle_mode = e.twm;
    c.ctas_per_sm = 1;
    c.tma_slabs = e.slabs;
    emit(c);
  }
  for (int a = 16; a <= 4096 && a <= N; a *= 2) {
    int n1, n2;
    if (N % a || !fourstep_split(N, a, &n1, &n2)) continue;
    const KernelEntry *k = default_column(n2, 1);
    fft_config_t c;
    memset(&c, 0, sizeof(c));
    c.path = FFT_PATH_FOURSTEP;
    c.points_per_thread = k->P;
    c.transforms_per_cta = k->TB;
    c.threads_per_cta = k->threads;
    c.num_passes = k->npass;
    for (int i = 0; i < 8; ++i) c.radix[i] = k->radix[i];
    c.n1 = n1;
    emit(c);
    if (n1 != n2) continue;
    for (const auto &e : kernel_registry()) {
      if (e.kind != KIND_FOURSTEP_L2 || e.N != n1) continue;
      for (int rows : {8, 16, 32, 64}) {
        fft_config_t d;
        memset(&d, 0, sizeof(d));
        d.path = FFT_PATH_FOURSTEP;
        d.points_per_thread = e.P;
        d.transforms_per_cta = e.TB;
        d.threads_per_cta = e.threads;
        d.num_passes = e.npass;
        for (int i = 0; i < 8; ++i) d.radix[i] = e.radix[i];
        d.n1 = n1;
        d.ctas_per_sm = -1;
        d.l2_chunk_rows = rows;
        emit(d);
      }
    }
  }
  return n;
}

static fft_status_t check_buffers(const void *in, const void *out, int64_t bytes) {
  if (!in || !out) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
  if (in != out) {
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return FFT_ERR_INVALID_VALUE;
  }
  return FFT_OK;
}

fft_status_t fft_exec(fft_plan_t plan, const void *in, void *out, void *stream) {
  if (!plan) return FFT_ERR_INVALID_VALUE;
  fft_plan_impl *pl = &plan->impl;
  if (pl->path == FFT_PATH_RAGGED) {
    if (!in || !out) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
    return ragged_exec(pl, (const float2 *)in, (float2 *)out, (cudaStream_t)stream);
  }
  if (pl->path == FFT_PATH_FILTER) return FFT_ERR_INVALID_VALUE;  // use fft_filter_forward
  if (pl->path == FFT_PATH_COLUMNS) {
    if (pl->batch == 0) return FFT_OK;
    if (!in || !out) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return FFT_ERR_MISALIGNED;
    const int64_t extent = (int64_t)sizeof(float2) *
                           ((pl->col_nmat - 1) * pl->col_mat_stride +
                            (int64_t)(pl->N - 1) * pl->col_row_stride + pl->col_ncols);
    if (in != out) {
      const char *a = (const char *)in, *b = (const char *)out;
      if (a < b + extent && b < a + extent) return FFT_ERR_INVALID_VALUE;
    }
    if (pl->k_col1) return exec_long_columns(pl, (const float2 *)in, (float2 *)out,
                                             (cudaStream_t)stream);
    ColumnArgs c{};
    c.in = (const float2 *)in;
    c.out = (float2 *)out;
    c.tw = pl->d_tw + pl->tw_col2;
    c.tw_a = c.tw_b = nullptr;
    c.nmat = pl->col_nmat;
    c.in_mat_stride = pl->col_mat_stride;
    c.out_mat_stride = pl->col_mat_stride;
    c.in_row_stride = (int)pl->col_row_stride;
    c.out_row_stride = (int)pl->col_row_stride;
    c.ncols = (int)pl->col_ncols;
    c.ntot = 0;  // no four-step twiddle on this path
    c.scale = pl->scale;
    c.in_extent = c.out_extent = extent / (int64_t)sizeof(float2);
    return launch_column(pl->k_col2, pl->direction, c, (cudaStream_t)stream);
  }
  if (pl->batch == 0) return FFT_OK;
  fft_status_t s = check_buffers(in, out, elem_bytes(pl) * pl->N * pl->batch);
  if (s != FFT_OK) return s;
  return exec_rows(pl, (const float2 *)in, (float2 *)out, pl->batch, (cudaStream_t)stream);
}

fft_status_t fft_exec_host(fft_plan_t plan, const void *host_in, void *host_out, void *stream) {
  if (!plan) return FFT_ERR_INVALID_VALUE;
  fft_plan_impl *pl = &plan->impl;
  if (pl->path == FFT_PATH_RAGGED || pl->path == FFT_PATH_FILTER || pl->path == FFT_PATH_COLUMNS)
    return FFT_ERR_NOT_SUPPORTED;
  if (pl->batch == 0) return FFT_OK;
  if (!host_in || !host_out) return FFT_ERR_INVALID_VALUE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t row_bytes = elem_bytes(pl) * pl->N;
  // Chunks of about 32 MiB; two input and two output staging slots.
  if (!pl->d_stage) {
    int64_t rows = std::max<int64_t>(1, (32ll << 20) / row_bytes);
    rows = std::min(rows, pl->batch);
    if (dev_malloc(&pl->d_stage, (size_t)(4 * rows * row_bytes)) != cudaSuccess) {
      cudaGetLastError();
      return FFT_ERR_ALLOC;
    }
    pl->stage_rows = rows;
    FFTGB_CUDA(cudaStreamCreateWithFlags(&pl->s_h2d, cudaStreamNonBlocking));
    FFTGB_CUDA(cudaStreamCreateWithFlags(&pl->s_d2h, cudaStreamNonBlocking));
  }
  const int64_t R = pl->stage_rows;
  const int64_t nchunk = (pl->batch + R - 1) / R;
  char *stage = (char *)pl->d_stage;
  float2 *slot_in[2] = {(float2 *)stage, (float2 *)(stage + R * row_bytes)};
  float2 *slot_out[2] = {(float2 *)(stage + 2 * R * row_bytes),
                         (float2 *)(stage + 3 * R * row_bytes)};
  cudaEvent_t ev_start, ev_in[2], ev_done[2], ev_out[2];
  FFTGB_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) {
    FFTGB_CUDA(cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming));
    FFTGB_CUDA(cudaEventCreateWithFlags(&ev_done[i], cudaEventDisableTiming));
    FFTGB_CUDA(cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming));
  }
  fft_status_t s = FFT_OK;
  cudaError_t e = cudaEventRecord(ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->s_h2d, ev_start, 0);
  const char *hin = (const char *)host_in;
  char *hout = (char *)host_out;
  for (int64_t c = 0; c < nchunk && e == cudaSuccess && s == FFT_OK; ++c) {
    const int slot = (int)(c & 1);
    const int64_t r0 = c * R, rows = std::min(R, pl->batch - r0);
    const size_t bytes = (size_t)(rows * row_bytes);
    if (c >= 2) {  // slot reuse: compute(c-2) read slot_in, D2H(c-2) read slot_out
      e = cudaStreamWaitEvent(pl->s_h2d, ev_done[slot], 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_out[slot], 0);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(slot_in[slot], hin + r0 * row_bytes, bytes, cudaMemcpyHostToDevice,
                          pl->s_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[slot], pl->s_h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in[slot], 0);
    if (e != cudaSuccess) break;
    s = exec_rows(pl, slot_in[slot], slot_out[slot], rows, st);
    if (s != FFT_OK) break;
    e = cudaEventRecord(ev_done[slot], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->s_d2h, ev_done[slot], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hout + r0 * row_bytes, slot_out[slot], bytes, cudaMemcpyDeviceToHost,
                          pl->s_d2h);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[slot], pl->s_d2h);
  }
  if (e == cudaSuccess && s == FFT_OK) e = cudaStreamSynchronize(pl->s_d2h);
  if (e == cudaSuccess && s == FFT_OK) e = cudaStreamSynchronize(st);
  cudaEventDestroy(ev_start);
  for (int i = 0; i < 2; ++i) {
    cudaEventDestroy(ev_in[i]);
    cudaEventDestroy(ev_done[i]);
    cudaEventDestroy(ev_out[i]);
  }
  if (s != FFT_OK) return s;
  return cuda_status(e);
}

fft_status_t fft_destroy(fft_plan_t plan) {
  if (!plan) return FFT_OK;
  free_plan(&plan->impl);
  delete plan;
  return FFT_OK;
}

fft_status_t fft_plan_columns(fft_plan_t *out, int L, int64_t ncols, int64_t nmat,
                              int64_t row_stride, int64_t mat_stride, int direction,
                              int flags) {
  if (!out) return FFT_ERR_INVALID_VALUE;
  *out = nullptr;
  if (!is_pow2(L) || L < 16 || L > kMaxColumnLength) return FFT_ERR_INVALID_SIZE;
  if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
  const int route = flags & (FFT_FLAG_FORCE_SINGLE_CTA | FFT_FLAG_FORCE_FOURSTEP);
  if (flags & ~(FFT_FLAG_UNNORMALIZED_INVERSE | route)) return FFT_ERR_INVALID_VALUE;
  if (route == (FFT_FLAG_FORCE_SINGLE_CTA | FFT_FLAG_FORCE_FOURSTEP)) return FFT_ERR_INVALID_VALUE;
  if (route == FFT_FLAG_FORCE_SINGLE_CTA && L > 4096) return FFT_ERR_NOT_SUPPORTED;
  if (route == FFT_FLAG_FORCE_FOURSTEP && L < 2048) return FFT_ERR_NOT_SUPPORTED;
  // Two launches (L = n1 n2, phase 1 of length n2 = min(512, 2^ceil(log2 L /
  // 2)), phase 2 of length n1 <= 4096) beyond one CTA's column, on request
  // from L = 2048, and by default at 4096 when ncols fills 16-column tiles:
  // the 4-column single-launch tile measured 188 us over 2^25 points against
  // 165 us for the two 64-point launches (at 2048 one launch stays ahead,
  // 138 us against 165 us).
  const bool two = L > 4096 || route == FFT_FLAG_FORCE_FOURSTEP ||
                   (L == 4096 && route == 0 && ncols > 0 && ncols % 16 == 0);
  int n1 = L, n2 = 1;
  if (two) {
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    n2 = std::min(512, 1 << ((lg + 1) / 2));
    n1 = L / n2;
  }
  const KernelEntry *k = default_column(n1, 0);
  const KernelEntry *k1 = n2 > 1 ? default_column(n2, 2) : nullptr;
  if (!k || (n2 > 1 && !k1)) return FFT_ERR_NOT_SUPPORTED;
  const int tile = k1 ? std::max(k->TB, k1->TB) : k->TB;
  if (ncols < 0 || nmat < 0) return FFT_ERR_INVALID_SIZE;
  if (ncols % tile != 0 || ncols > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  if (row_stride < ncols || row_stride > 0x7fffffffLL) return FFT_ERR_INVALID_VALUE;
  if (nmat > 1 && mat_stride < (int64_t)(L - 1) * row_stride + ncols) return FFT_ERR_INVALID_VALUE;
  if (mat_stride < 0) return FFT_ERR_INVALID_VALUE;
  if (nmat * (ncols / k->TB) > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  // The long path's row strides (n1 or n2 rows apart) and grids stay 32-bit.
  int64_t chunk = 0;
  if (k1) {
    if ((int64_t)n1 * std::max(row_stride, ncols) > 0x7fffffffLL ||
        (int64_t)n2 * row_stride > 0x7fffffffLL)
      return FFT_ERR_INVALID_SIZE;
    if (nmat * n1 * (ncols / k1->TB) > 0x7fffffffLL || nmat * n2 * (ncols / k->TB) > 0x7fffffffLL)
      return FFT_ERR_INVALID_SIZE;
    const int64_t mat_bytes = (int64_t)sizeof(float2) * L * ncols;
    if (nmat > 0)
      chunk = std::max<int64_t>(
          1, std::min<int64_t>(nmat, kColumnScratchBytes / std::max<int64_t>(1, mat_bytes)));
  }
  fft_plan_s *h = new (std::nothrow) fft_plan_s;
  if (!h) return FFT_ERR_ALLOC;
  fft_plan_impl *pl = &h->impl;
  pl->N = L;
  pl->batch = nmat * ncols;
  pl->direction = direction;
  pl->flags = flags;
  pl->scale = (direction == FFT_INVERSE && !(flags & FFT_FLAG_UNNORMALIZED_INVERSE))
                  ? 1.0f / (float)L
                  : 1.0f;
  pl->path = FFT_PATH_COLUMNS;
  pl->k_col2 = k;
  pl->k_col1 = k1;
  pl->n1 = k1 ? n1 : 0;
  pl->n2 = k1 ? n2 : 0;
  pl->col_ncols = ncols;
  pl->col_nmat = nmat;
  pl->col_row_stride = row_stride;
  pl->col_mat_stride = mat_stride;
  pl->col_chunk = chunk;
  cudaGetDevice(&pl->device);
  fft_status_t s = FFT_OK;
  if (dev_malloc(&pl->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    s = FFT_ERR_ALLOC;
  } else if (cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) {
    s = FFT_ERR_CUDA;
  }
  if (s == FFT_OK) s = ensure_smem_attr(k);
  if (s == FFT_OK && k1) s = ensure_smem_attr(k1);
  if (s == FFT_OK && k1 && chunk > 0 && ncols > 0) {
    pl->scratch_bytes = (int64_t)sizeof(float2) * L * ncols * chunk;
    if (dev_malloc(&pl->d_scratch, (size_t)pl->scratch_bytes) != cudaSuccess) {
      cudaGetLastError();
      s = FFT_ERR_ALLOC;
    }
  }
  if (s == FFT_OK) {
    int64_t off = 0;
    pl->tw_col2 = 0;
    std::vector<TwSeg> segs = pass_segments(*k, off);
    if (k1) {
      pl->tw_col1 = off;
      auto a = pass_segments(*k1, off);
      segs.insert(segs.end(), a.begin(), a.end());
      TwSeg g;  // W_L^{j k} at j * n2 + k, j < n1, k < n2
      g.offset = off;
      g.kind = 2;
      g.p = n2;
      g.r = 0;
      g.step = 1;
      g.M = L;
      g.count = L;
      pl->tw_big = off;
      off += g.count;
      segs.push_back(g);
    }
    s = build_twiddles(pl, segs);
  }
  if (s != FFT_OK) {
    free_plan(pl);
    delete h;
    return s;
  }
  *out = h;
  return FFT_OK;
}

fft_status_t fft_plan_info(fft_plan_t plan, fft_plan_info_t *info) {
  if (!plan || !info) return FFT_ERR_INVALID_VALUE;
  const fft_plan_impl *pl = &plan->impl;
  memset(info, 0, sizeof(*info));
  info->N = pl->N;
  info->batch = pl->batch;
  info->direction = pl->path == FFT_PATH_RAGGED ? 0 : pl->direction;
  info->precision = pl->precision;
  info->path = pl->path;
  info->scratch_bytes = pl->scratch_bytes;
  const bool one = pl->path == FFT_PATH_SINGLE_CTA || pl->path == FFT_PATH_TMEM_HALVES;
  const KernelEntry *k = one                             ? pl->k_single
                         : pl->path == FFT_PATH_FOURSTEP ? (pl->k_l2 ? pl->k_l2 : pl->k_col1)
                         : pl->path == FFT_PATH_COLUMNS  ? pl->k_col2
                                                         : nullptr;
  if (k) {
    info->points_per_thread = k->P;
    info->transforms_per_cta = k->TB;
    info->threads_per_cta = k->threads;
    info->num_passes = k->npass;
    for (int i = 0; i < 8; ++i) info->radix[i] = k->radix[i];
  }
  info->n1 = pl->n1;
  info->n2 = pl->n2;
  info->twiddle_mode = one ? pl->k_single->twm : 0;
  info->grid_ctas = (int)pl->grid_ctas;
  info->tma_slabs = pl->path == FFT_PATH_SINGLE_CTA ? pl->k_single->slabs : 0;
  info->cluster_split = pl->path == FFT_PATH_SINGLE_CTA ? pl->k_single->split : 0;
  info->l2_chunk_rows = pl->l2_rows;
  if (pl->k_l2) info->grid_ctas = (int)pl->l2_grid;
  if (pl->path == FFT_PATH_RAGGED) info->threads_per_cta = 512;  // one persistent launch
  return FFT_OK;
}

fft_status_t fft_last_device_status(fft_plan_t plan) {
  if (!plan) return FFT_ERR_INVALID_VALUE;
  fft_plan_impl *pl = &plan->impl;
  if (cudaDeviceSynchronize() != cudaSuccess) return FFT_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FFT_ERR_CUDA;
  if (cudaMemset(pl->d_status, 0, sizeof(int)) != cudaSuccess) return FFT_ERR_CUDA;
  return (fft_status_t)v;
}

fft_status_t fft_twiddle_table(fft_plan_t plan, void *host_out, int64_t capacity, int64_t *count) {
  if (!plan || !count) return FFT_ERR_INVALID_VALUE;
  const fft_plan_impl *pl = &plan->impl;
  *count = pl->tw_count;
  if (host_out && pl->tw_count > 0 && capacity > 0) {
    const int64_t n = std::min(capacity, pl->tw_count);
    if (cudaMemcpy(host_out, pl->d_tw, sizeof(float2) * (size_t)n, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return FFT_ERR_CUDA;
  }
  return FFT_OK;
}

fft_status_t fft_twiddle_index(fft_plan_t plan, int64_t pos, int64_t *M, int64_t *e) {
  if (!plan || !M || !e) return FFT_ERR_INVALID_VALUE;
  for (const auto &g : plan->impl.tw_segs) {
    if (pos < g.offset || pos >= g.offset + g.count) continue;
    const int64_t local = pos - g.offset;
    if (g.kind == 0) {
      const int64_t j = local / g.p + 1, k = local % g.p;
      *M = g.M;
      *e = j * k;
    } else if (g.kind == 2) {
      const int64_t i = local / g.p, c = local % g.p;
      *M = g.M;
      *e = ((i * g.step) % g.M) * c % g.M;
    } else {
      *M = g.M;
      *e = local;
    }
    return FFT_OK;
  }
  return FFT_ERR_INVALID_VALUE;
}

}  // extern "C"
