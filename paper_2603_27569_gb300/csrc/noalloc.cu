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
// first call outside any stream capture.  The set-up is tied to the device's
// current context: after cudaDeviceReset (which reloads the module and so
// zeroes both arrays) the next call sets the device up again.  Every call
// shares the one scratch array, so calls whose work overlaps on the GPU (for
// instance on two streams) race; the intermediate is fully rewritten by
// phase 1 before phase 2 reads it, so nothing needs clearing between calls.
#include <cuda.h>  // CUcontext / CUresult for two driver entry points (not linked)
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
  unsigned long long ctx_id = 0;  // context the tables were filled in (0: unknown)
  float2 *scratch = nullptr;      // device address of g_scratch on this device
  float2 *tw = nullptr;           // device address of g_tw on this device
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

// Entries of the per-pass tables of column kernel k.
int64_t pass_table_entries(const KernelEntry *k) {
  int64_t n = 0;
  int p = k->radix[0];
  for (int s = 1; s < k->npass; ++s) {
    n += (int64_t)(k->radix[s] - 1) * p;
    p *= k->radix[s];
  }
  return n;
}

// One generator launch; its status is checked here (cudaLaunchKernel returns
// it directly), not read back from the thread's shared last-error slot.
cudaError_t launch_gen(const void *fn, int64_t n, void **args) {
  return cudaLaunchKernel(fn, dim3((unsigned)((n + 255) / 256)), dim3(256), args, 0, nullptr);
}

// Per-pass tables of column kernel k written from `off` on; returns the end.
cudaError_t fill_pass_tables(const KernelEntry *k, float2 *tw, int64_t &off) {
  int p = k->radix[0];
  for (int s = 1; s < k->npass; ++s) {
    int r = k->radix[s];
    const int64_t n = (int64_t)(r - 1) * p;
    float2 *dst = tw + off;
    void *args[] = {&dst, &p, &r};
    const cudaError_t e = launch_gen((const void *)&gen_pass_twiddles, n, args);
    if (e != cudaSuccess) return e;
    off += n;
    p *= r;
  }
  return cudaSuccess;
}

// Process-unique id of the calling thread's current context (cuCtxGetId),
// through driver entry points the runtime hands out; false if unavailable.
bool current_context_id(unsigned long long *id) {
  typedef CUresult (*GetCurrent)(CUcontext *);
  typedef CUresult (*GetId)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  });
  CUcontext ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

fft_status_t setup_device(int dev, DeviceSetup **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup &d = g_dev[dev];
  // Host code may not take the arrays' addresses directly: resolve the
  // device addresses with the runtime, for the current device (this also
  // makes the device's context current).  A failure is returned as
  // FFT_ERR_CUDA; the runtime's last-error slot keeps it, as for any failed
  // runtime call, and nothing of the caller's is cleared.
  float2 *scratch = nullptr, *tw = nullptr;
  if (cudaGetSymbolAddress((void **)&scratch, g_scratch) != cudaSuccess ||
      cudaGetSymbolAddress((void **)&tw, g_tw) != cudaSuccess)
    return FFT_ERR_CUDA;
  unsigned long long ctx = 0;
  const bool have_ctx = current_context_id(&ctx);
  if (d.ready && d.scratch == scratch && d.tw == tw && (!have_ctx || d.ctx_id == ctx)) {
    *out = &d;
    return FFT_OK;
  }
  d.ready = false;
  d.scratch = scratch;
  d.tw = tw;
  // Lay out every size's tables first and check the total against the
  // array before anything is written.
  int64_t off = 0;
  for (int e = kMinLog2; e <= kMaxLog2; ++e) {
    SizeSetup &z = d.size[e - kMinLog2];
    const int N = 1 << e;
    if (!split(N, &z.n1, &z.n2)) return FFT_ERR_NOT_SUPPORTED;
    z.k1 = default_column(z.n2, 1);
    z.k2 = default_column(z.n1, 0);
    const int T1 = z.n2 / z.k1->P;
    z.tw1 = off;
    off += pass_table_entries(z.k1);
    z.tw2 = off;
    off += pass_table_entries(z.k2);
    z.twa = off;  // phase-1 twiddle grid W_N^{c lt}, [lt][c]
    off += (int64_t)T1 * z.n1;
    z.twb = off;  // phase-1 twiddle grid W_N^{c T m}, [m][c]
    off += (int64_t)z.k1->P * z.n1;
  }
  if (off > kTwEntries) return FFT_ERR_NOT_SUPPORTED;
  for (int e = kMinLog2; e <= kMaxLog2; ++e) {
    SizeSetup &z = d.size[e - kMinLog2];
    if (ensure_smem_attr(z.k1) != FFT_OK || ensure_smem_attr(z.k2) != FFT_OK)
      return FFT_ERR_CUDA;
    int64_t o = z.tw1;
    if (fill_pass_tables(z.k1, tw, o) != cudaSuccess) return FFT_ERR_CUDA;
    o = z.tw2;
    if (fill_pass_tables(z.k2, tw, o) != cudaSuccess) return FFT_ERR_CUDA;
    int64_t cols = z.n1, step = 1, M = 1 << e;
    int64_t na = (int64_t)(z.n2 / z.k1->P) * z.n1, nb = (int64_t)z.k1->P * z.n1;
    float2 *dst = tw + z.twa;
    void *aa[] = {&dst, &cols, &step, &M, &na};
    if (launch_gen((const void *)&gen_grid_twiddles, na, aa) != cudaSuccess) return FFT_ERR_CUDA;
    float2 *dstb = tw + z.twb;
    int64_t stepb = z.n2 / z.k1->P;
    void *ab[] = {&dstb, &cols, &stepb, &M, &nb};
    if (launch_gen((const void *)&gen_grid_twiddles, nb, ab) != cudaSuccess) return FFT_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return FFT_ERR_CUDA;
  d.ctx_id = have_ctx ? ctx : 0;
  d.ready = true;
  *out = &d;
  return FFT_OK;
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
  c1.in_extent = c1.out_extent = (long long)batch * N;
  s = launch_column(z.k1, direction, c1, st);
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
  c2.in_extent = c2.out_extent = (long long)batch * N;
  return launch_column(z.k2, direction, c2, st);
}
