// Bounds checks of the debug build (compiled with FFTGB_BOUNDS_CHECK; the
// product build compiles every check to `true`).  A check that fails records
// its site number in this translation unit's error word (the first failure
// wins) and the access it guards is skipped, so a wrong index is reported
// instead of faulting; nothing traps.  Each unit keeps its own word (no
// relocatable device code) and registers a host reader that
// fft_debug_bounds_status() polls.
#pragma once
#include <cuda_runtime.h>

namespace fftgb {

#ifdef FFTGB_BOUNDS_CHECK
void register_bounds_reader(int (*read_and_clear)());
static __device__ int g_bounds_site;  // this unit's first failing site (0: none)
static int read_bounds_site() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_site, sizeof(int)) != cudaSuccess) return -1;
  if (v != 0) cudaMemcpyToSymbol(g_bounds_site, &z, sizeof(int));
  return v;
}
static const bool g_bounds_reader = (register_bounds_reader(&read_bounds_site), true);
__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_bounds_site, 0, site);
  return false;
}
#define FFTGB_OK(i, n, site) ::fftgb::in_bounds((long long)(i), (long long)(n), (site))
#else
#define FFTGB_OK(i, n, site) true
#endif

// Site numbers (reported by fft_debug_bounds_status).
enum BoundsSite {
  kSiteLoadIdx = 1,     // pass-0 load: index in the row
  kSiteLoadRow = 2,     // pass-0 load: row in the batch
  kSiteStoreIdx = 3,    // final store: index in the row
  kSiteStoreRow = 4,    // final store: row in the batch
  kSiteTwiddle = 5,     // pass-table entry
  kSiteXchgWrite = 6,   // exchange write: logical index, then buffer slot
  kSiteXchgRead = 7,    // exchange read: logical index, then buffer slot
  kSiteColLoad = 8,     // column kernel: global load (offset in the input extent)
  kSiteColStore = 9,    // column kernel: global store (offset in the output extent)
  kSiteColTwiddle = 10, // column kernel: per-sub-matrix twiddle entry
  kSiteSelfTest = 99,   // fft_debug_bounds_selftest
};

}  // namespace fftgb
