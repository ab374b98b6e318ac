// fft_fourstep_noalloc: the two-phase four-step transform for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc: code that must not allocate once it
// is running (a real-time radar chain whose memory is fixed at start-up),
// code that owns the device heap through its own allocator, or code called
// from contexts where an allocation would stall or break a captured
// sequence.  The regular four-step path needs a device intermediate the size
// of the batch, which its plan allocates; this entry point instead keeps the
// intermediate in a fixed, file-scope device array, and its twiddle tables in
// another one, so a call allocates nothing.
//
// Both arrays are reserved on every GPU that loads the library and stay there
// until the process exits (16 MiB of scratch + 512 KiB of tables).  The
// first call on a device sets that device up (resolves the arrays'
// addresses, fills the twiddle tables, synchronises the device); make that
// first call outside any stream capture.  Every call shares the one scratch
// array, so calls whose work overlaps on the GPU (for instance on two
// streams) race; the intermediate is fully rewritten by phase 1 before
// phase 2 reads it, so nothing needs clearing between calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "column.cuh"
#include "plan.h"

namespace fftgb {

// Twiddle generators of the regular planner (api.cu), reused unchanged.
__global__ void gen_pass_twiddles(float2 *out, int p, int r);
__global__ void gen_grid_twiddles(float2 *out, int64_t cols, int64_t step, int64_t M,
                                  int64_t count);

namespace {

constexpr int64_t kScratchPoints = FFT_NOALLOC_MAX_POINTS;  // 2^21 complex = 16 MiB
constexpr int64_t kTwEntries = 1 << 16;                     // 512 KiB of tables
constexpr int kMinLog2 = 8, kMaxLog2 = 14;                  // N = 256 .. 16384
constexpr int kSizes = kMaxLog2 - kMinLog2 + 1;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_scratch[kScratchPoints];
static __device__ __align__(256) float2 g_tw[kTwEntries];

struct SizeSetup {
  int n1 = 0, n2 = 0;
  const KernelEntry *k1 = nullptr, *k2 = nullptr;  // phase-1 / phase-2 column kernels
  int64_t tw1 = 0, tw2 = 0, twa = 0, twb = 0;      // offsets into g_tw
};

struct DeviceSetup {
  bool ready = false;
  float2 *scratch = nullptr;  // device address of g_scratch on this device
  float2 *tw = nullptr;       // device address of g_tw on this device
  SizeSetup size[kSizes];
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

// Same split rule as the regular planner: n1 <= n2, both column lengths.
bool split(int N, int *n1, int *n2) {
  int best = 0;
  for (int a = 16; a <= 256; a *= 2) {
    const int b = N / a;
    if (N % a || b < 16 || b > 256 || a > b) continue;
    if (!default_column(b, 1) || !default_column(a, 0)) continue;
    best = a;
  }
  if (!best) return false;
  *n1 = best;
  *n2 = N / best;
  return true;
}

// Per-pass tables of column kernel k written from `off` on; returns the end.
int64_t fill_pass_tables(const KernelEntry *k, float2 *tw, int64_t off) {
  int p = k->radix[0];
  for (int s = 1; s < k->npass; ++s) {
    const int r = k->radix[s];
    const int64_t n = (int64_t)(r - 1) * p;
    gen_pass_twiddles<<<(unsigned)((n + 255) / 256), 256>>>(tw + off, p, r);
    off += n;
    p *= r;
  }
  return off;
}

fft_status_t setup_device(int dev, DeviceSetup **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup &d = g_dev[dev];
  if (!d.ready) {
    // Host code may not take the arrays' addresses directly: resolve the
    // device addresses with the runtime, for the current device.
    if (cudaGetSymbolAddress((void **)&d.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void **)&d.tw, g_tw) != cudaSuccess) {
      cudaGetLastError();
      return FFT_ERR_CUDA;
    }
    int64_t off = 0;
    for (int e = kMinLog2; e <= kMaxLog2; ++e) {
      SizeSetup &z = d.size[e - kMinLog2];
      const int N = 1 << e;
      if (!split(N, &z.n1, &z.n2)) return FFT_ERR_NOT_SUPPORTED;
      z.k1 = default_column(z.n2, 1);
      z.k2 = default_column(z.n1, 0);
      z.tw1 = off;
      off = fill_pass_tables(z.k1, d.tw, off);
      z.tw2 = off;
      off = fill_pass_tables(z.k2, d.tw, off);
      // phase-1 twiddle grids W_N^{c lt} [lt][c] and W_N^{c T m} [m][c]
      const int T1 = z.n2 / z.k1->P;
      const int64_t na = (int64_t)T1 * z.n1, nb = (int64_t)z.k1->P * z.n1;
      if (off + na + nb > kTwEntries) return FFT_ERR_NOT_SUPPORTED;
      z.twa = off;
      gen_grid_twiddles<<<(unsigned)((na + 255) / 256), 256>>>(d.tw + off, z.n1, 1, N, na);
      off += na;
      z.twb = off;
      gen_grid_twiddles<<<(unsigned)((nb + 255) / 256), 256>>>(d.tw + off, z.n1, T1, N, nb);
      off += nb;
    }
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return FFT_ERR_CUDA;
    d.ready = true;
  }
  *out = &d;
  return FFT_OK;
}

fft_status_t launch(const KernelEntry *k, int dir, const ColumnArgs &ca, cudaStream_t st) {
  const int64_t grid = ca.nmat * (ca.ncols / k->TB);
  if (grid <= 0) return FFT_OK;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  ColumnArgs a = ca;
  void *args[] = {&a};
  return cudaLaunchKernel(k->fn[dir > 0 ? 1 : 0], dim3((unsigned)grid), dim3(k->threads), args,
                          k->smem, st) == cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace
}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status_t fft_fourstep_noalloc(const void *in, void *out, int N, int64_t batch,
                                             int direction, void *stream) {
  if (N < (1 << kMinLog2) || N > (1 << kMaxLog2) || (N & (N - 1)) || batch < 0)
    return FFT_ERR_INVALID_SIZE;
  if (batch > kScratchPoints / N) return FFT_ERR_INVALID_SIZE;  // beyond the fixed scratch
  if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
  if (!in || !out) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)in | (uintptr_t)out) & 15) return FFT_ERR_MISALIGNED;
  const int64_t bytes = (int64_t)sizeof(float2) * N * batch;
  if (in != out) {
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return FFT_ERR_INVALID_VALUE;
  }
  if (batch == 0) return FFT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FFT_ERR_CUDA;
  DeviceSetup *d = nullptr;
  fft_status_t s = setup_device(dev, &d);
  if (s != FFT_OK) return s;
  const SizeSetup &z = d->size[__builtin_ctz((unsigned)N) - kMinLog2];
  cudaStream_t st = (cudaStream_t)stream;
  ColumnArgs c1{};
  c1.in = (const float2 *)in;
  c1.out = d->scratch;
  c1.tw = d->tw + z.tw1;
  c1.tw_a = d->tw + z.twa;
  c1.tw_b = d->tw + z.twb;
  c1.nmat = batch;
  c1.in_mat_stride = N;
  c1.out_mat_stride = N;
  c1.in_row_stride = z.n1;
  c1.ncols = z.n1;
  c1.ntot = N;
  c1.scale = 1.f;
  s = launch(z.k1, direction, c1, st);
  if (s != FFT_OK) return s;
  ColumnArgs c2{};
  c2.in = d->scratch;
  c2.out = (float2 *)out;
  c2.tw = d->tw + z.tw2;
  c2.nmat = batch;
  c2.in_mat_stride = N;
  c2.out_mat_stride = N;
  c2.in_row_stride = z.n2;
  c2.out_row_stride = z.n2;
  c2.ncols = z.n2;
  c2.ntot = N;
  c2.scale = direction == FFT_INVERSE ? 1.0f / (float)N : 1.0f;
  return launch(z.k2, direction, c2, st);
}
