// Column-FFT configurations for the two-phase four-step path and the column
// transforms.  Variant 1 = phase 1 (four-step twiddle, transposed store,
// L <= 256, C = 16 columns per CTA); variant 0 = plain (phase 2, and
// fft_plan_columns).  Lengths beyond 256 take fewer columns per CTA so the
// tile stays small: C = 16 up to L = 512, 8 at 1024 and 2048 (64 KiB and
// 128 KiB; at 1024, 8 columns measured faster than 16: two CTAs per SM), 4 at
// 4096 (32-byte row segments, one sector each).  The 16-column 1024 kernel
// stays registered as a non-default configuration.  Variant 2 = phase 1 of a
// column longer than 4096 (per-sub-matrix twiddle, plain store), at the
// lengths L2 that such a column's split uses (64 to 512).
#include "instantiate.cuh"

namespace fftgb {
// Variant 2 (TWM 2, plain store): an unpadded C-column tile.
template <int L, int P, int C, class SC>
inline KernelEntry long_column_entry() {
  KernelEntry e{};
  e.kind = KIND_COLUMN;
  e.N = L;
  e.P = P;
  e.TB = C;
  e.threads = C * (L / P);
  e.smem = sizeof(float2) * (size_t)L * C;
  fill_radix<SC>(e);
  e.is_default = 1;
  e.variant = 2;
  e.fn[0] = (const void *)&column_kernel<L, P, C, -1, SC, 2, false>;
  e.fn[1] = (const void *)&column_kernel<L, P, C, +1, SC, 2, false>;
  return e;
}
}  // namespace fftgb
#define FFTGB_LONG_COLUMN(L, P, C, ...)                                      \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::long_column_entry<L, P, C, ::fftgb::Sched<__VA_ARGS__>>())

FFTGB_COLUMN(16, 16, 16, 0, 1, 16);
FFTGB_COLUMN(16, 16, 16, 1, 1, 16);
FFTGB_COLUMN(32, 16, 16, 0, 1, 16, 2);
FFTGB_COLUMN(32, 16, 16, 1, 1, 16, 2);
FFTGB_COLUMN(64, 16, 16, 0, 1, 16, 4);
FFTGB_COLUMN(64, 16, 16, 1, 1, 16, 4);
FFTGB_COLUMN(128, 16, 16, 0, 1, 16, 8);
FFTGB_COLUMN(128, 16, 16, 1, 1, 16, 8);
FFTGB_COLUMN(256, 16, 16, 0, 1, 16, 16);
FFTGB_COLUMN(256, 16, 16, 1, 1, 16, 16);
FFTGB_COLUMN(512, 16, 16, 0, 1, 16, 16, 2);
FFTGB_COLUMN(512, 16, 16, 1, 1, 16, 16, 2);
FFTGB_COLUMN(1024, 16, 16, 0, 0, 16, 16, 4);
FFTGB_COLUMN(1024, 16, 8, 0, 1, 16, 16, 4);
FFTGB_COLUMN(2048, 16, 8, 0, 1, 16, 16, 8);
FFTGB_COLUMN(4096, 16, 4, 0, 1, 16, 16, 16);
FFTGB_LONG_COLUMN(64, 16, 16, 16, 4);
FFTGB_LONG_COLUMN(128, 16, 16, 16, 8);
FFTGB_LONG_COLUMN(256, 16, 16, 16, 16);
FFTGB_LONG_COLUMN(512, 16, 16, 16, 16, 2);
