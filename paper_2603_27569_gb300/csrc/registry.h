// Kernel registry: every compiled kernel configuration registers itself here
// at library load, so the planner and the autotuner can enumerate them.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

namespace fftgb {

enum KernelKind {
  KIND_STOCKHAM = 1,
  KIND_COLUMN = 2,
  KIND_STAGED = 3,
  KIND_SPLIT = 4,       // a row on a cluster of `split` CTAs (cluster.cuh)
  KIND_HALFIO = 5,      // FP16 storage, FP32 arithmetic
  KIND_FOURSTEP_L2 = 6, // both four-step phases in one persistent launch (N = L * L)
  KIND_TMEM2 = 7        // N = 2 H on one SM, one half in tensor memory (tmem2.cuh)
};

struct KernelEntry {
  int kind;
  int N;          // transform length (L for column and L2 four-step kernels; the full N for split)
  int P;          // complex points per thread
  int TB;         // rows per CTA (single-CTA) / columns per CTA (column)
  int threads;    // threads per CTA
  size_t smem;    // dynamic shared memory bytes
  int npass;
  int radix[8];   // (split: the schedule of the N/K-point part)
  int tw_total;   // entries of the per-pass twiddle tables
  int is_default; // the built-in choice for this (kind, N, variant)
  int variant;    // column kernels: 0 plain, 1 twiddle + transposed store;
                  // 16-bit storage: 0 FP16 pairs, 1 BF16 pairs
  int twm;        // twiddle mode: 0 all from tables, 1 rows 1/4(/16) + products
  int slabs;      // staged kernels: slabs held in the TMA ring (0 otherwise)
  int split;      // cluster kernels: CTAs per row, K (0 otherwise)
  const void *fn[2];  // [0] forward (D = -1), [1] inverse (D = +1)
};

void register_kernel(const KernelEntry &e);
const std::vector<KernelEntry> &kernel_registry();

struct Registrar {
  explicit Registrar(const KernelEntry &e) { register_kernel(e); }
};

}  // namespace fftgb
