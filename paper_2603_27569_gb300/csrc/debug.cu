// Failure injection for the library's own tests (no GPU fault, trap or hang):
//
//   fft_debug_fail_alloc(after): the next `after` device allocations succeed
//   and the one after them fails as cudaMalloc would (no memory taken), so a
//   test can walk every allocation of a plan's creation and check that each
//   failure comes back as FFT_ERR_ALLOC with nothing leaked.
//
//   fft_debug_bounded_wait(kind, limit_us): runs one of the bounded device
//   waits the kernels use, on something that never arrives (an mbarrier with
//   no arrival, a counter nobody increments), with a short limit; the waiting
//   thread gives up, records FFT_ERR_TIMEOUT in a device status word and
//   returns, and the host reads that word: the error path of a lost bulk copy
//   or a stalled producer, exercised without one.
//
//   Debug build (FFTGB_BOUNDS_CHECK, check.cuh): fft_debug_bounds_status()
//   reports the first failed bounds check of any unit (0: none) and clears
//   them; fft_debug_bounds_selftest() fails one check on purpose (the access
//   it guards is skipped) to show the checks are live.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "fourstep_l2.cuh"
#include "plan.h"
#include "staged.cuh"

namespace fftgb {

static std::atomic<int> g_fail_after{-1};  // -1: disarmed

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
  int n = g_fail_after.load();
  while (n >= 0) {
    if (g_fail_after.compare_exchange_weak(n, n - 1)) {
      if (n == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;  // the armed failure (no sticky error is left)
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

// kind 0: the mbarrier wait of the bulk-copy kernels (mbar_wait), on a
// barrier initialised for one arrival that never comes.  kind 1: the counter
// wait of the single-launch four-step (wait_count), on a zeroed counter.
__global__ void debug_wait_kernel(int kind, unsigned long long limit_ns, unsigned *counter,
                                  int *status) {
  __shared__ __align__(8) uint64_t bar;
  bool ok;
  if (kind == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok = mbar_wait(&bar, 0, limit_ns);
  } else {
    ok = wait_count(counter, 1u, limit_ns);
  }
  *status = ok ? 0 : 6 /* FFT_ERR_TIMEOUT */;
}

#ifdef FFTGB_BOUNDS_CHECK
// The per-unit error-word readers (check.cuh), registered at load time.
static std::vector<int (*)()> &bounds_readers() {
  static std::vector<int (*)()> v;
  return v;
}
void register_bounds_reader(int (*read_and_clear)()) { bounds_readers().push_back(read_and_clear); }

__global__ void debug_bounds_selftest_kernel(int n) {
  (void)FFTGB_OK(n, n, kSiteSelfTest);  // one past the end: recorded, nothing accessed
}
#endif

}  // namespace fftgb

using namespace fftgb;

extern "C" {

int fft_debug_bounds_status(void) {
#ifdef FFTGB_BOUNDS_CHECK
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  int first = 0;
  for (auto read : bounds_readers()) {
    const int v = read();
    if (v < 0) return -2;
    if (v != 0 && first == 0) first = v;
  }
  return first;
#else
  return -1;
#endif
}

fft_status_t fft_debug_bounds_selftest(void *stream) {
#ifdef FFTGB_BOUNDS_CHECK
  cudaStream_t st = (cudaStream_t)stream;
  debug_bounds_selftest_kernel<<<1, 1, 0, st>>>(4);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return FFT_ERR_CUDA;
  return FFT_OK;
#else
  (void)stream;
  return FFT_ERR_NOT_SUPPORTED;
#endif
}

void fft_debug_fail_alloc(int after) { g_fail_after.store(after < 0 ? -1 : after); }

fft_status_t fft_debug_bounded_wait(int kind, int limit_us, void *stream) {
  if ((kind != 0 && kind != 1) || limit_us <= 0 || limit_us > 1000000)
    return FFT_ERR_INVALID_VALUE;
  cudaStream_t st = (cudaStream_t)stream;
  int *d = nullptr;  // [0] status, [1] the counter nobody increments
  if (dev_malloc(&d, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return FFT_ERR_ALLOC;
  }
  fft_status_t s = FFT_OK;
  int h = -1;
  if (cudaMemsetAsync(d, 0, 2 * sizeof(int), st) != cudaSuccess) s = FFT_ERR_CUDA;
  if (s == FFT_OK) {
    debug_wait_kernel<<<1, 1, 0, st>>>(kind, 1000ull * (unsigned long long)limit_us,
                                       reinterpret_cast<unsigned *>(d + 1), d);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = FFT_ERR_CUDA;
  }
  cudaFree(d);
  return s != FFT_OK ? s : (fft_status_t)h;
}

}  // extern "C"
