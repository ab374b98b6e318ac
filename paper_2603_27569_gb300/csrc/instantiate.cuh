// Helpers that instantiate a kernel configuration and register it.
#pragma once
#include <type_traits>

#include "cluster.cuh"
#include "column.cuh"
#include "fourstep_l2.cuh"
#include "halfio.cuh"
#include "registry.h"
#include "staged.cuh"
#include "stockham.cuh"
#include "tmem2.cuh"

namespace fftgb {

template <class SC>
inline void fill_radix(KernelEntry &e) {
  e.npass = SC::npass;
  for (int i = 0; i < 8; ++i) e.radix[i] = i < SC::npass ? SC::radix[i] : 0;
  e.tw_total = SC::tw_total();
}

template <int N, int P, int TB, int TWM, int DEF, class SC>
inline KernelEntry stockham_entry() {
  KernelEntry e{};
  e.kind = KIND_STOCKHAM;
  e.N = N;
  e.P = P;
  e.TB = TB;
  e.threads = TB * (N / P);
  e.smem = sizeof(float2) * (size_t)TB * N;
  fill_radix<SC>(e);
  e.is_default = DEF;
  e.variant = 0;
  e.twm = TWM;
  e.fn[0] = (const void *)&stockham_kernel<N, P, TB, -1, SC, TWM>;
  e.fn[1] = (const void *)&stockham_kernel<N, P, TB, +1, SC, TWM>;
  return e;
}

template <int N, int P, int C, int TWM, int DEF, class SC>
inline KernelEntry staged_entry() {
  KernelEntry e{};
  e.kind = KIND_STAGED;
  e.N = N;
  e.P = P;
  e.TB = 1;
  e.threads = N / P;
  e.smem = staged_smem_bytes<N, P, C>();
  fill_radix<SC>(e);
  e.is_default = DEF;
  e.variant = 0;
  e.twm = TWM;
  e.slabs = C;
  e.fn[0] = (const void *)&staged_kernel<N, P, C, -1, SC, TWM>;
  e.fn[1] = (const void *)&staged_kernel<N, P, C, +1, SC, TWM>;
  return e;
}

template <int N, int K, int P, int TWM, int DEF, class SC>
inline KernelEntry splitk_entry() {
  KernelEntry e{};
  e.kind = KIND_SPLIT;
  e.N = N;
  e.P = P;
  e.TB = 1;
  e.threads = (N / K) / P;
  e.smem = sizeof(float2) * (size_t)(N / K);
  fill_radix<SC>(e);
  e.is_default = DEF;
  e.twm = TWM;
  e.split = K;
  e.fn[0] = (const void *)&splitk_kernel<N, K, P, -1, SC, TWM>;
  e.fn[1] = (const void *)&splitk_kernel<N, K, P, +1, SC, TWM>;
  return e;
}

template <int N, int P, int TWM, int DEF, class SC>
inline KernelEntry tmem2_entry() {
  KernelEntry e{};
  e.kind = KIND_TMEM2;
  e.N = N;
  e.P = P;
  e.TB = 1;
  e.threads = (N / 2) / P;
  e.smem = tmem2_smem_bytes<N>();
  fill_radix<SC>(e);
  e.is_default = DEF;
  e.twm = TWM;
  e.fn[0] = (const void *)&tmem2_kernel<N, P, -1, SC, TWM>;
  e.fn[1] = (const void *)&tmem2_kernel<N, P, +1, SC, TWM>;
  return e;
}

template <int N, int P, int TB, int TWM, class SC, class S2>
inline KernelEntry half_entry() {
  KernelEntry e{};
  e.kind = KIND_HALFIO;
  e.N = N;
  e.P = P;
  e.TB = TB;
  e.threads = TB * (N / P);
  e.smem = sizeof(float2) * (size_t)TB * N;
  fill_radix<SC>(e);
  e.is_default = 1;
  e.twm = TWM;
  e.variant = std::is_same<S2, __nv_bfloat162>::value ? 1 : 0;  // 0 FP16, 1 BF16 pairs
  e.fn[0] = (const void *)&stockham_half_kernel<N, P, TB, -1, SC, TWM, S2>;
  e.fn[1] = (const void *)&stockham_half_kernel<N, P, TB, +1, SC, TWM, S2>;
  return e;
}

template <int L, int P, int C, int VAR, int DEF, class SC>
inline KernelEntry column_entry() {
  KernelEntry e{};
  e.kind = KIND_COLUMN;
  e.N = L;
  e.P = P;
  e.TB = C;
  e.threads = C * (L / P);
  e.smem = sizeof(float2) * (size_t)L * (VAR ? C + 1 : C);
  fill_radix<SC>(e);
  e.is_default = DEF;
  e.variant = VAR;
  e.fn[0] = (const void *)&column_kernel<L, P, C, -1, SC, VAR != 0, VAR != 0>;
  e.fn[1] = (const void *)&column_kernel<L, P, C, +1, SC, VAR != 0, VAR != 0>;
  return e;
}

template <int L, int P, int C, class SC>
inline KernelEntry fourstep_l2_entry() {
  KernelEntry e{};
  e.kind = KIND_FOURSTEP_L2;
  e.N = L;
  e.P = P;
  e.TB = C;
  e.threads = C * (L / P);
  e.smem = sizeof(float2) * (size_t)L * (C + 1);
  fill_radix<SC>(e);
  e.is_default = 0;
  e.variant = 0;
  e.fn[0] = (const void *)&fourstep_l2_kernel<L, P, C, -1, SC>;
  e.fn[1] = (const void *)&fourstep_l2_kernel<L, P, C, +1, SC>;
  return e;
}

}  // namespace fftgb

#define FFTGB_CAT2(a, b) a##b
#define FFTGB_CAT(a, b) FFTGB_CAT2(a, b)
// FFTGB_STOCKHAM(N, P, TB, is_default, radices...): registers the kernel in
// both twiddle modes; `is_default` marks which mode (1 or 2 = TWM + 1) is the
// built-in choice (0: neither).
#define FFTGB_STOCKHAM(N, P, TB, DEF, ...)                                   \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::stockham_entry<N, P, TB, 0, DEF == 1, ::fftgb::Sched<__VA_ARGS__>>()); \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::stockham_entry<N, P, TB, 1, DEF == 2, ::fftgb::Sched<__VA_ARGS__>>())
// FFTGB_STAGED(N, P, C, is_default, radices...): TMA-staged kernel with a
// ring of C slabs, both twiddle modes (is_default as for FFTGB_STOCKHAM).
#define FFTGB_STAGED(N, P, C, DEF, ...)                                      \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::staged_entry<N, P, C, 0, DEF == 1, ::fftgb::Sched<__VA_ARGS__>>()); \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::staged_entry<N, P, C, 1, DEF == 2, ::fftgb::Sched<__VA_ARGS__>>())
// FFTGB_SPLITK(N, K, P, is_default, radices of N/K...): a row on a cluster
// of K CTAs, both twiddle modes (is_default as for FFTGB_STOCKHAM).
#define FFTGB_SPLITK(N, K, P, DEF, ...)                                      \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::splitk_entry<N, K, P, 0, DEF == 1, ::fftgb::Sched<__VA_ARGS__>>()); \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::splitk_entry<N, K, P, 1, DEF == 2, ::fftgb::Sched<__VA_ARGS__>>())
// FFTGB_TMEM2(N, P, is_default, radices of N/2...): a row of N points on one
// SM with one half in tensor memory, both twiddle modes (is_default as for
// FFTGB_STOCKHAM).
#define FFTGB_TMEM2(N, P, DEF, ...)                                          \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::tmem2_entry<N, P, 0, DEF == 1, ::fftgb::Sched<__VA_ARGS__>>()); \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::tmem2_entry<N, P, 1, DEF == 2, ::fftgb::Sched<__VA_ARGS__>>())
// FFTGB_HALF(N, P, TB, twiddle mode, radices...): 16-bit-storage kernels,
// FP16 pairs (variant 0) and BF16 pairs (variant 1).
#define FFTGB_HALF(N, P, TB, TWM, ...)                                       \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::half_entry<N, P, TB, TWM, ::fftgb::Sched<__VA_ARGS__>, __half2>()); \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::half_entry<N, P, TB, TWM, ::fftgb::Sched<__VA_ARGS__>, __nv_bfloat162>())
// FFTGB_COLUMN(L, P, C, variant, is_default, radices...)
#define FFTGB_COLUMN(L, P, C, VAR, DEF, ...)                                 \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::column_entry<L, P, C, VAR, DEF, ::fftgb::Sched<__VA_ARGS__>>())
// FFTGB_FOURSTEP_L2(L, P, C, radices of L...): N = L * L in one launch.
#define FFTGB_FOURSTEP_L2(L, P, C, ...)                                      \
  static ::fftgb::Registrar FFTGB_CAT(fftgb_reg_, __COUNTER__)(              \
      ::fftgb::fourstep_l2_entry<L, P, C, ::fftgb::Sched<__VA_ARGS__>>())
