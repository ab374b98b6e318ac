// Internal plan representation shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fftgb.h"
#include "registry.h"

namespace fftgb {

// One segment of a plan's twiddle allocation.
struct TwSeg {
  int64_t offset;  // first entry
  int64_t count;   // entries
  int kind;        // 0: per-pass table W_{p r}^{j k} laid out [j-1][k]; 1: W_M^e, e < M;
                   // 2: grid W_M^{(i step c) mod M} at i * p + c, c < p (p columns)
  int p, r;        // kind 0 (kind 2: p = columns)
  int64_t M;       // kinds 1 and 2 (and p*r for kind 0)
  int64_t step = 0;  // kind 2
};

struct RaggedState;  // ragged.cu

struct fft_plan_impl {
  int N = 0;
  int64_t batch = 0;
  int direction = -1;
  int precision = FFT_PREC_FP32;
  int flags = 0;
  int path = 0;
  float scale = 1.f;
  int device = 0;
  // single-CTA path
  const KernelEntry *k_single = nullptr;
  int ctas_per_sm = 0;    // 0: one CTA per tile; > 0 persistent grid
  int64_t grid_ctas = 0;  // persistent grid size (0 = one CTA per tile)
  // four-step path: phase-1 and phase-2 column kernels, split N = n1 * n2
  const KernelEntry *k_col1 = nullptr, *k_col2 = nullptr;
  int n1 = 0, n2 = 0;
  // column path (fft_plan_columns): transforms down the columns of strided
  // matrices, element (mat, row, col) at mat * col_mat_stride + row *
  // col_row_stride + col
  int64_t col_ncols = 0, col_nmat = 0, col_row_stride = 0, col_mat_stride = 0;
  // columns longer than 4096: matrices per pass through the scratch
  int64_t col_chunk = 0;
  // four-step in one launch with the intermediate in an L2 ring (n1 == n2):
  // chunks of l2_rows rows, l2_slots ring slots, phase 2 of a chunk claimed
  // l2_lag rounds after its phase 1; d_l2cnt = the launch's work counters
  const KernelEntry *k_l2 = nullptr;
  int l2_rows = 0, l2_lag = 0, l2_slots = 0;
  int64_t l2_grid = 0;
  unsigned *d_l2cnt = nullptr;
  // twiddles
  float2 *d_tw = nullptr;
  int64_t tw_count = 0;
  std::vector<TwSeg> tw_segs;
  int64_t tw_single = 0, tw_col1 = 0, tw_col2 = 0, tw_big = 0;  // offsets
  int64_t tw_big2 = 0;  // four-step phase 1: W_N^{c T m} grid (tw_big: W_N^{c lt})
  // scratch (four-step intermediate)
  float2 *d_scratch = nullptr;
  int64_t scratch_bytes = 0;
  // one-tile-per-CTA plain kernels: CTAs resident at once (the look-ahead prefetch)
  int64_t resident_ctas = 0;
  // device status word (bounded waits report here)
  int *d_status = nullptr;
  // host-buffer exec staging
  float2 *d_stage = nullptr;
  int64_t stage_rows = 0;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  // tensor-core path
  void *tc = nullptr;
  // ragged path
  RaggedState *ragged = nullptr;
  // fused spectral-filter path
  void *filter = nullptr;
};

// Every device allocation of the library (debug.cu): cudaMalloc, or the
// failure that fft_debug_fail_alloc armed.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

// Helpers implemented in api.cu, shared with the other units.
fft_status_t cuda_status(cudaError_t e);
// Launch with programmatic stream serialization: the kernel must begin with
// griddepcontrol.wait (no global access before the previous kernel of the
// stream has completed), and may then let the next one launch early.
cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       void **args);
// One column-kernel launch (column.cuh) with the library's launch policy:
// programmatic dependent launch for columns up to 2048 points.
struct ColumnArgs;
fft_status_t launch_column(const KernelEntry *k, int dir, const ColumnArgs &ca, cudaStream_t st);
fft_status_t build_twiddles(fft_plan_impl *pl, const std::vector<TwSeg> &segs);
std::vector<TwSeg> pass_segments(const KernelEntry &k, int64_t &offset);
const KernelEntry *find_stockham(int N, int P, int TB, const int *radix, int npass, int twm);
const KernelEntry *find_split(int N, int K, int P, const int *radix, int npass, int twm);
const KernelEntry *default_stockham(int N);
const KernelEntry *default_column(int L, int variant);
fft_status_t launch_stockham(const KernelEntry *k, int dir, const float2 *in, float2 *out,
                             const float2 *tw, int64_t rows, float scale, int64_t grid_cap,
                             int64_t ahead, cudaStream_t st);
// Persistent grid for kernel k with `per_sm` CTAs per SM (-1: occupancy).
int64_t persistent_grid(const KernelEntry *k, int per_sm);
fft_status_t exec_rows(fft_plan_impl *pl, const float2 *in, float2 *out, int64_t rows,
                       cudaStream_t st);
fft_status_t ensure_smem_attr(const KernelEntry *k);

// Autotuner cache lookup (autotune.cu).  Returns true and fills the choice if
// the process-wide cache holds one for this key.
struct TuneChoice {
  int path;                 // FFT_PATH_SINGLE_CTA or FFT_PATH_FOURSTEP
  int P, TB, npass;
  int radix[8];
  int n1;                   // four-step split (n1)
  int twm;                  // twiddle mode
  int ctas_per_sm;          // 0 / -1 / k (see fft_config_t)
  int slabs;                // TMA-staged ring size (0: direct loads)
  int split;                // 2: cluster-split kernel
  int l2rows;               // four-step in one launch, chunks of this many rows
};
bool tune_lookup(int N, int direction, int precision, TuneChoice *out);

// Tensor-core path (tc.cu)
fft_status_t tc_plan(fft_plan_impl *pl);
fft_status_t tc_exec(fft_plan_impl *pl, const float2 *in, float2 *out, int64_t rows,
                     cudaStream_t st);
void tc_destroy(fft_plan_impl *pl);

// Fused spectral filter (filter_fused.cu)
void filter_destroy(fft_plan_impl *pl);

// Ragged path (ragged.cu)
fft_status_t ragged_exec(fft_plan_impl *pl, const float2 *in, float2 *out, cudaStream_t st);
void ragged_destroy(fft_plan_impl *pl);
void ragged_clear_choices();  // forget the ragged autotuner's choices
// grad_H = fixed-order pairwise sum of the nchunk rows of partial (spectral.cu)
fft_status_t grad_h_tree(float2 *partial, float2 *grad_H, int N, int64_t nchunk,
                         cudaStream_t st);

}  // namespace fftgb

struct fft_plan_s {
  fftgb::fft_plan_impl impl;
};
