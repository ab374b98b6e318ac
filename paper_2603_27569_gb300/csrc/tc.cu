// Split-precision tensor-core FFT on the fifth-generation tensor cores
// (tcgen05): radix-16 DFT blocks as dense FP16/BF16 contractions with FP32
// accumulation (paper Sec. V-C, Eq. 5-6, where the Apple kernel maps DFT_8
// onto 8x8 matrix units; here DFT_16 maps onto a 128 x 32 x 32 tcgen05.mma,
// the tcFFT idea of Sec. VIII).
//
// One radix-16 Stockham stage over 128 butterflies is the real product
//     D (128 x 32) = A (128 x 32) . G^T,
// row m of A = the 16 twiddled inputs of one butterfly, interleaved
// [Re x(0), Im x(0), Re x(1), ...]; G (32 x 32) the real form of F =
// (W_16^{jk}) (conjugated for the inverse) with the same interleaving; row m
// of D = the butterfly's 16 outputs.  Both operands are split into a high
// and a low 16-bit part, v = hi + lo with hi = round16(v), lo = round16(v -
// hi), and D = Ahi.Ghi^T + Ahi.Glo^T + Alo.Ghi^T is accumulated in FP32 in
// tensor memory (lo.lo, ~2^-22 relative, is dropped): ~22-bit (FP16) or
// ~16-bit (BF16) operands.
//
// Data path per stage: A (hi and lo planes) and G sit in shared memory in the
// K-major, unswizzled canonical layout (core matrices of 8 rows x 16 bytes;
// K-adjacent core matrices LBO bytes apart, 8-row groups SBO bytes apart);
// one thread issues 6 tcgen05.mma per 128-row tile into TMEM and commits to
// an mbarrier; every thread then reads its TMEM lane (tcgen05.ld 32x32b) --
// one butterfly's 16 outputs -- multiplies each output by the next stage's
// FP32 twiddle, splits it and stores it straight into the next stage's A
// (that store is the Stockham exchange; the tensor core reads the operand).
// Which A row holds which butterfly is a per-stage bit permutation of the
// butterfly index, and LBO/SBO are padded (144/576 or 144/592 bytes), chosen
// by exhaustive search on a model of the bank mapping so that every
// exchange store is conflict-free, the first stage's row stores take the
// minimum wavefronts and the global loads/stores touch the minimum sectors.
// N = 4096 uses the unpadded 128/512 layout instead: 36 KiB per CTA fits six
// CTAs per SM (five with padding), which measured faster than the
// conflict-free stores (at N = 256 the same change measured 15 % slower).
// N = 16384 = 16^3 * 4 ends with a radix-4 pass in registers: each thread's
// four TMEM tiles hold the four butterflies that feed one radix-4 butterfly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "plan.h"
#include "staged.cuh"
#include "stockham.cuh"

namespace fftgb {

struct TcArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;       // N = 16384: the radix-4 tail's table (stride 4096, radix 4)
  const float2 *twx;      // exchange twiddle factors: W_256^{j2 j} [j][j2], W_4096^{j2 k} [j2][k]
  const uint4 *bimg;      // this direction's G image: hi plane, lo plane (2 KiB each)
  int *status;            // FFT_ERR_TIMEOUT if an MMA completion wait ran out
  long long batch;
  long long ahead;        // one-group-per-CTA grids: resident CTAs (occupancy x SMs)
  float scale;
};

// Per-size plan: NW warps per CTA, MINB CTAs per SM the register budget is
// sized for, PERSIST: a resident grid walks the row groups (otherwise one
// group per CTA, which measured faster where several CTAs share an SM: their
// phases stay staggered).
// Row permutations rho_s are nibble-packed: nibble b = the
// bit of the packed butterfly index (row-in-CTA << log2 NB | butterfly) that
// becomes bit b of the A row at stage s.
template <int N>
struct TcCfg;
template <>
struct TcCfg<256> {
  static constexpr int S = 2, TAIL = 0, TB = 16, NW = 4, LBO = 144, SBO = 576, MINB = 5;
  static constexpr bool PERSIST = false;
  static constexpr unsigned long long R0 = 0x45763021ull, R1 = 0x73526140ull, R2 = 0;
};
template <>
struct TcCfg<4096> {
  static constexpr int S = 3, TAIL = 0, TB = 1, NW = 4, LBO = 128, SBO = 512, MINB = 6;
  static constexpr bool PERSIST = false;
  static constexpr unsigned long long R0 = 0x76354210ull, R1 = 0x73210654ull, R2 = 0x76543102ull;
};
template <>
struct TcCfg<16384> {
  static constexpr int S = 3, TAIL = 4, TB = 1, NW = 16, LBO = 144, SBO = 592, MINB = 1;
  static constexpr bool PERSIST = true;
  static constexpr unsigned long long R0 = 0x8539064712ull, R1 = 0x4130576289ull,
                                      R2 = 0x9876543210ull;
};

template <class C>
__host__ __device__ constexpr unsigned long long tc_rcode(int s) {
  return s == 0 ? C::R0 : s == 1 ? C::R1 : C::R2;
}

// v (packed butterfly index) -> row; and back.
template <unsigned long long R, int NBITS>
__host__ __device__ constexpr int tc_row(int v) {
  int m = 0;
  for (int b = 0; b < NBITS; ++b) m |= ((v >> (int)((R >> (4 * b)) & 15)) & 1) << b;
  return m;
}
template <unsigned long long R, int NBITS>
__host__ __device__ constexpr int tc_unrow(int m) {
  int v = 0;
  for (int b = 0; b < NBITS; ++b) v |= ((m >> b) & 1) << (int)((R >> (4 * b)) & 15);
  return v;
}
// Byte offset of row m's first core-matrix row (the K-slot terms are added).
template <int SBO>
__host__ __device__ constexpr int tc_rowoff(int m) {
  return (m >> 3) * SBO + (m & 7) * 16;
}

// 16-bit split of (v0, v1): hi = round(v), lo = round(v - hi), packed two per u32.
template <int PREC>
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  if constexpr (PREC == FFT_PREC_FP16X2) {
    const __half2 H = __floats2half2_rn(v0, v1);
    const float2 h = __half22float2(H);
    const __half2 L = __floats2half2_rn(v0 - h.x, v1 - h.y);
    hi = *reinterpret_cast<const uint32_t *>(&H);
    lo = *reinterpret_cast<const uint32_t *>(&L);
  } else {
    const __nv_bfloat162 H = __floats2bfloat162_rn(v0, v1);
    const float2 h = __bfloat1622float2(H);
    const __nv_bfloat162 L = __floats2bfloat162_rn(v0 - h.x, v1 - h.y);
    hi = *reinterpret_cast<const uint32_t *>(&H);
    lo = *reinterpret_cast<const uint32_t *>(&L);
  }
}

// Shared-memory matrix descriptor: K-major, no swizzle (layout type 0),
// descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B FP16 or BF16,
// both K-major, N = 32, M = 128.
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (PREC == FFT_PREC_BF16X2 ? ((1u << 7) | (1u << 10)) : 0u) |
         ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
// 8 consecutive FP32 columns.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Exchange after TC stage s (stride p = 16^s): this thread's butterfly (row
// m, outputs in r) writes output j, times the stage-(s+1) twiddle, into the
// stage-(s+1) A planes.  With butterfly i = p u + k the output lands at
// position p (16 u + j) + k = base | j p (disjoint bits, j p < N / 16), so
// its row is row(base) | row(j p) and its byte offset is the thread's
// offset plus a compile-time constant per j.
template <int N, int D, int PREC, int s>
__device__ __forceinline__ void tc_exchange(const uint32_t (&r)[32], int m, uint8_t *Ahi,
                                            uint8_t *Alo, const float2 *__restrict__ twx) {
  using C = TcCfg<N>;
  constexpr int NB = N / 16, IB = ilog2(NB), NBITS = ilog2(C::TB * NB);
  constexpr int p = s == 0 ? 1 : s == 1 ? 16 : 256, LP = 4 * s;
  constexpr unsigned long long RS = tc_rcode<C>(s), RN = tc_rcode<C>(s + 1);
  static_assert(16 * p <= NB, "j p must stay below the butterfly count");
  const int v = tc_unrow<RS, NBITS>(m);
  const int b = v >> IB, i = v & (NB - 1);
  const int k = i & (p - 1), u = i >> LP;
  const int base = (u << (LP + 4)) | k;       // position of output j = 0
  const int j2 = base >> IB;                  // the next stage's point index
  const int m2 = tc_row<RN, NBITS>((b << IB) | (base & (NB - 1)));
  const int off = tc_rowoff<C::SBO>(m2) + (j2 >> 2) * C::LBO + (j2 & 3) * 4;
  // The next pass's twiddle W_{256 p}^{j2 (j p + k)} of this row's output j
  // is W_256^{j2 j} (times W_4096^{j2 k} after stage 1, where p = 16; k = 0
  // after stage 0): two 16 x 16 tables of 2 KiB that stay in L1.  A warp's
  // j2 values lie in 0..15, so each j reads one 128-byte line.
  const float2 *tj = twx + j2;
  float2 aw = make_float2(1.f, 0.f);
  if constexpr (s > 0) aw = __ldg(twx + 256 + j2 * 16 + k);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float2 x = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
    float2 w = __ldg(tj + 16 * j);
    if constexpr (s > 0) w = cmul(aw, w);
    x = cmul_dir<D>(x, w);
    uint32_t hi, lo;
    split2<PREC>(x.x, x.y, hi, lo);
    const int oj = off + tc_rowoff<C::SBO>(tc_row<RN, NBITS>(j * p));
    *reinterpret_cast<uint32_t *>(Ahi + oj) = hi;
    *reinterpret_cast<uint32_t *>(Alo + oj) = lo;
  }
}

// Shared-memory layout of the kernel: A hi and lo planes, the G image, the
// MMA-completion mbarrier and the TMEM address slot.
template <int N>
struct TcSmem {
  static constexpr int PLANE = (TcCfg<N>::TB * (N / 16) / 8) * TcCfg<N>::SBO;
  static constexpr int B = 2 * PLANE, BAR = B + 4096, TOTAL = BAR + 16;
  static_assert(B % 1024 == 0, "operand alignment");
};

// A CTA transforms groups of TB rows: one group, or (PERSIST) every
// gridDim.x-th group from blockIdx.x.  A one-group CTA first has the group
// one resident wave ahead (blockIdx.x + occupancy x SMs) prefetched into L2,
// so the CTA that starts when this wave retires reads its rows from L2.
template <int N, int D, int PREC>
__global__ void __launch_bounds__(TcCfg<N>::NW * 32, TcCfg<N>::MINB)
tc_kernel(TcArgs a) {
  using C = TcCfg<N>;
  using L = TcSmem<N>;
  constexpr int NW = C::NW;
  constexpr int NB = N / 16, IB = ilog2(NB), ROWS = C::TB * NB, NBITS = ilog2(ROWS);
  constexpr int TM = ROWS / 128, NT = NW * 32, TPT = TM * 4 / NW;
  constexpr uint32_t NCOL = TM * 32 <= 32 ? 32 : TM * 32;  // power of two for TM in {1, 2, 8}
  static_assert(TM * 4 % NW == 0 && NW % 4 == 0, "warps must cover the TMEM lanes");
  static_assert(ROWS % NT == 0, "loader threads must cover the rows");
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t *Ahi = sm, *Alo = sm + L::PLANE, *Bs = sm + L::B;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + L::BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ngroups = (a.batch + C::TB - 1) / C::TB;

  for (int e = tid; e < 256; e += NT) reinterpret_cast<uint4 *>(Bs)[e] = __ldg(a.bimg + e);
  if (tid == 0) {
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const int q4 = warp & 3, g4 = warp >> 2;
  bool ok = true;
  unsigned mph = 0;  // completed phases of the MMA mbarrier
  for (long long grp = blockIdx.x; grp < ngroups; grp += C::PERSIST ? gridDim.x : ngroups) {
    const long long row0 = grp * C::TB;
    if (!C::PERSIST && warp == 0 && grp + a.ahead < ngroups) {
      // the group that the CTA one resident wave later will load, into L2
      const long long nxt = grp + a.ahead;
      const long long rows = min((long long)C::TB, a.batch - nxt * C::TB);
      prefetch_l2_warp(a.in + nxt * C::TB * N, rows * N * (long long)sizeof(float2), lane);
    }
    if (C::PERSIST && warp == 0 && grp + gridDim.x < ngroups) {
      // the next group's rows into L2 while this one runs (bulk prefetch)
      const long long nxt = grp + gridDim.x;
      const long long rows = min((long long)C::TB, a.batch - nxt * C::TB);
      prefetch_l2_warp(a.in + nxt * C::TB * N, rows * N * (long long)sizeof(float2), lane);
    }
    // Stage 0 operand: lanes take consecutive butterflies and each writes its
    // butterfly's whole row (four 16-byte chunks per plane).
#pragma unroll
    for (int q = 0; q < ROWS / NT; ++q) {
      const int v = tid + NT * q;
      const int b = v >> IB, i = v & (NB - 1);
      const long long grow = row0 + b;
      const bool active = grow < a.batch;
      const float2 *src = a.in + grow * N + i;
      float2 x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = active ? __ldcs(src + j * NB) : make_float2(0.f, 0.f);
      const int ro = tc_rowoff<C::SBO>(tc_row<C::R0, NBITS>(v));
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint4 h, l;
        split2<PREC>(x[4 * c + 0].x, x[4 * c + 0].y, h.x, l.x);
        split2<PREC>(x[4 * c + 1].x, x[4 * c + 1].y, h.y, l.y);
        split2<PREC>(x[4 * c + 2].x, x[4 * c + 2].y, h.z, l.z);
        split2<PREC>(x[4 * c + 3].x, x[4 * c + 3].y, h.w, l.w);
        *reinterpret_cast<uint4 *>(Ahi + ro + c * C::LBO) = h;
        *reinterpret_cast<uint4 *>(Alo + ro + c * C::LBO) = l;
      }
    }
    fence_proxy_async();  // A for the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
#pragma unroll
    for (int s = 0; s < C::S; ++s) {
      if (tid == 0) {
        // A descriptor holds the operand's shared-memory address / 16 in its
        // low 14 bits (addresses < 256 KiB), so the descriptor of base + off
        // is the base descriptor + off / 16: one 64-bit add per operand, the
        // offsets compile-time constants (all offsets are multiples of 16).
        const uint32_t idesc = tc_idesc<PREC>();
        const uint64_t dA = tc_desc(smem_u32(Ahi), C::LBO, C::SBO);
        const uint64_t dB = tc_desc(smem_u32(Bs), 128, 512);
        constexpr uint32_t kLo = (uint32_t)L::PLANE / 16;  // Alo - Ahi
        static_assert(L::PLANE % 16 == 0 && 16 * C::SBO % 16 == 0, "16-byte operand offsets");
#pragma unroll
        for (int t = 0; t < TM; ++t) {
          const uint32_t d = tbase + 32 * t;
          const uint32_t arow = 16 * t * C::SBO / 16;
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t A = dA + (pr == 2 ? kLo : 0u) + arow + kk * 2 * C::LBO / 16;
              const uint64_t B = dB + (pr == 1 ? 2048u / 16 : 0u) + kk * 256 / 16;
              tc_mma(d, A, B, idesc, (pr | kk) ? 1u : 0u);
            }
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar))
            : "memory");
      }
      ok = __syncthreads_and(ok && mbar_wait(mbar, mph & 1));
      if (!ok) break;
      ++mph;
      tc_fence_after();
      if (s + 1 < C::S) {
#pragma unroll 1
        for (int t = 0; t < TPT; ++t) {
          const int tile = g4 + (NW / 4) * t;
          const int m = 128 * tile + 32 * q4 + lane;
          uint32_t r[32];
          tc_ld32(tbase + ((uint32_t)(32 * q4) << 16) + 32 * tile, r);
          tc_wait_ld();
          if (s == 0) tc_exchange<N, D, PREC, 0>(r, m, Ahi, Alo, a.twx);
          else tc_exchange<N, D, PREC, (C::S > 2 ? 1 : 0)>(r, m, Ahi, Alo, a.twx);
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
      } else if constexpr (C::TAIL == 0) {
        // last stage: butterfly i (< N / 16 = its stride) writes outputs i + j N/16
        constexpr unsigned long long RL = tc_rcode<C>(C::S - 1);
#pragma unroll 1
        for (int t = 0; t < TPT; ++t) {
          const int tile = g4 + (NW / 4) * t;
          const int m = 128 * tile + 32 * q4 + lane;
          uint32_t r[32];
          tc_ld32(tbase + ((uint32_t)(32 * q4) << 16) + 32 * tile, r);
          tc_wait_ld();
          const int v = tc_unrow<RL, NBITS>(m);
          const int b = v >> IB, i = v & (NB - 1);
          const long long grow = row0 + b;
          if (grow < a.batch) {
            float2 *dst = a.out + grow * N + i;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              __stcs(dst + j * NB, cscale(make_float2(__uint_as_float(r[2 * j]),
                                                      __uint_as_float(r[2 * j + 1])),
                                          a.scale));
          }
        }
      } else {
        // radix-4 tail (stride 4096): tiles g + 2v (v = 0..3, g = g4 & 1)
        // hold butterflies k + 256 v of the last TC stage (identity rows),
        // whose outputs j are the four points of radix-4 butterfly 256 j + k.
        // The warps that share a lane quarter split the tile parities g and,
        // with 16 warps, the four column chunks jc (two each).
        static_assert(N == 16384 && ((NW == 8 && TPT == 4) || (NW == 16 && TPT == 2)),
                      "tail mapping");
        constexpr int NJC = 4 / (NW / 8);
        const int g = g4 & 1, jc0 = (g4 >> 1) * NJC;
        const int k = 128 * g + 32 * q4 + lane;
        const float2 *tw3 = a.tw;  // W_16384^{v it}: entry (v - 1) * 4096 + it
#pragma unroll 1
        for (int jc = jc0; jc < jc0 + NJC; ++jc) {
          uint32_t r[4][8];
#pragma unroll
          for (int v = 0; v < 4; ++v)
            tc_ld8(tbase + ((uint32_t)(32 * q4) << 16) + 32 * (g + 2 * v) + 8 * jc, r[v]);
          tc_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int it = 256 * (4 * jc + jj) + k;
            float2 w[4];
#pragma unroll
            for (int v = 0; v < 4; ++v)
              w[v] = make_float2(__uint_as_float(r[v][2 * jj]), __uint_as_float(r[v][2 * jj + 1]));
#pragma unroll
            for (int v = 1; v < 4; ++v)
              w[v] = cmul_dir<D>(w[v], __ldg(tw3 + (v - 1) * 4096 + it));
            Dft<4, D>::run(w);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              __stcs(a.out + row0 * N + it + 4096 * v, cscale(w[v], a.scale));
          }
        }
      }
    }
    if (!ok) break;
    // (the next group's first MMA is issued after its stage-0 barrier, which
    // every thread reaches after its last TMEM read of this group)
  }
  if (!ok && tid == 0) atomicCAS(a.status, 0, 6 /* FFT_ERR_TIMEOUT */);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOL));
}

// G images for both directions, from the FP64 DFT-16 matrix: img[dir][plane]
// = 32 x 32 16-bit values G[n][k] (n = 2 jo + re/im of the output, k = 2 ji +
// re/im of the input) in the K-major layout with LBO 128, SBO 512.
template <int PREC>
__global__ void tc_gen_bimg(uint16_t *img) {
  const int n = threadIdx.x >> 5, k = threadIdx.x & 31;  // 1024 threads
  for (int dir = 0; dir < 2; ++dir) {
    const int jo = n >> 1, ji = k >> 1;
    double sn, cs;
    sincospi((dir ? 2.0 : -2.0) * (double)((jo * ji) % 16) / 16.0, &sn, &cs);
    // out_re = Fr x_re - Fi x_im ; out_im = Fi x_re + Fr x_im
    const double gv = (n & 1) == 0 ? ((k & 1) == 0 ? cs : -sn) : ((k & 1) == 0 ? sn : cs);
    uint16_t h, l;
    if (PREC == FFT_PREC_FP16X2) {
      const __half a = __double2half(gv);
      const __half b = __double2half(gv - (double)__half2float(a));
      h = *reinterpret_cast<const uint16_t *>(&a);
      l = *reinterpret_cast<const uint16_t *>(&b);
    } else {
      const __nv_bfloat16 a = __double2bfloat16(gv);
      const __nv_bfloat16 b = __double2bfloat16(gv - (double)__bfloat162float(a));
      h = *reinterpret_cast<const uint16_t *>(&a);
      l = *reinterpret_cast<const uint16_t *>(&b);
    }
    const int off = ((n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
    img[dir * 2048 + off] = h;
    img[dir * 2048 + 1024 + off] = l;
  }
}

// Exchange twiddle factors, forward sign (the kernels conjugate for the
// inverse), each from its exact integer exponent in FP64, rounded to FP32:
// out[16 j + j2] = W_256^{j2 j} and out[256 + 16 j2 + k] = W_4096^{j2 k}
// (j, j2, k < 16).  The twiddle W_{256 p}^{j2 (j p + k)} that output j of a
// butterfly (offset k < p in its stride-p group) takes into the next stage
// is their product: p = 1 (k = 0) after stage 0, p = 16 after stage 1.
constexpr int kTcTwx = 512;
__global__ void tc_gen_twx(float2 *out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kTcTwx) return;
  long long M, e;
  if (idx < 256) {
    M = 256;
    e = (long long)((idx >> 4) * (idx & 15)) % M;
  } else {
    M = 4096;
    e = (long long)(((idx - 256) >> 4) * (idx & 15)) % M;
  }
  double sn, cs;
  sincospi(-2.0 * (double)e / (double)M, &sn, &cs);
  out[idx] = make_float2(__double2float_rn(cs), __double2float_rn(sn));
}

struct TcState {
  uint16_t *d_bimg = nullptr;  // G images, both directions (8 KiB)
  float2 *d_twx = nullptr;     // exchange twiddle factors (kTcTwx entries)
  const void *fn = nullptr;
  int threads = 0, tb = 0;
  size_t smem = 0;
  bool persist = false;
  int64_t grid_cap = 0;  // CTAs per launch: occupancy x SMs when persistent
  int64_t resident = 0;  // occupancy x SMs
};

template <int N, int PREC>
static void pick(TcState *st, int dir) {
  st->fn = dir < 0 ? (const void *)&tc_kernel<N, -1, PREC> : (const void *)&tc_kernel<N, +1, PREC>;
  st->threads = TcCfg<N>::NW * 32;
  st->tb = TcCfg<N>::TB;
  st->smem = (size_t)TcSmem<N>::TOTAL;
  st->persist = TcCfg<N>::PERSIST;
}

template <int PREC>
static bool pick_prec(TcState *st, int N, int dir) {
  switch (N) {
    case 256: pick<256, PREC>(st, dir); return true;
    case 4096: pick<4096, PREC>(st, dir); return true;
    case 16384: pick<16384, PREC>(st, dir); return true;
  }
  return false;
}

fft_status_t tc_plan(fft_plan_impl *pl) {
  TcState *st = new (std::nothrow) TcState;
  if (!st) return FFT_ERR_ALLOC;
  pl->tc = st;
  const bool ok = pl->precision == FFT_PREC_FP16X2
                      ? pick_prec<FFT_PREC_FP16X2>(st, pl->N, pl->direction)
                      : pick_prec<FFT_PREC_BF16X2>(st, pl->N, pl->direction);
  if (!ok) return FFT_ERR_NOT_SUPPORTED;
  if (cudaFuncSetAttribute(st->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem) !=
      cudaSuccess)
    return FFT_ERR_CUDA;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, st->fn, st->threads, st->smem) !=
          cudaSuccess || occ < 1)
    return FFT_ERR_CUDA;
  st->grid_cap = st->persist ? (int64_t)occ * sms : 0x7fffffffLL;
  st->resident = (int64_t)occ * sms;
  // The TC stages take their twiddles from the factor tables (d_twx); only
  // N = 16384's radix-4 tail (stride 4096) reads a pass table.
  std::vector<TwSeg> segs;
  if (pl->N == 16384) {
    TwSeg g;
    g.offset = 0;
    g.count = 3 * 4096;
    g.kind = 0;
    g.p = 4096;
    g.r = 4;
    g.M = 16384;
    segs.push_back(g);
  }
  fft_status_t s = build_twiddles(pl, segs);
  if (s != FFT_OK) return s;
  if (dev_malloc(&st->d_bimg, 2 * 4096) != cudaSuccess ||
      dev_malloc(&st->d_twx, sizeof(float2) * (size_t)kTcTwx) != cudaSuccess) {
    cudaGetLastError();
    return FFT_ERR_ALLOC;
  }
  if (pl->precision == FFT_PREC_FP16X2) tc_gen_bimg<FFT_PREC_FP16X2><<<1, 1024>>>(st->d_bimg);
  else tc_gen_bimg<FFT_PREC_BF16X2><<<1, 1024>>>(st->d_bimg);
  tc_gen_twx<<<(kTcTwx + 255) / 256, 256>>>(st->d_twx);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return FFT_ERR_CUDA;
  pl->path = FFT_PATH_TENSORCORE;
  return FFT_OK;
}

fft_status_t tc_exec(fft_plan_impl *pl, const float2 *in, float2 *out, int64_t rows,
                     cudaStream_t stream) {
  TcState *st = (TcState *)pl->tc;
  if (!st || !st->fn) return FFT_ERR_INVALID_VALUE;
  if (rows <= 0) return FFT_OK;
  TcArgs a;
  a.in = in;
  a.out = out;
  a.tw = pl->d_tw;
  a.bimg = reinterpret_cast<const uint4 *>(st->d_bimg + (pl->direction > 0 ? 2048 : 0));
  a.twx = st->d_twx;
  a.status = pl->d_status;
  a.batch = rows;
  a.ahead = st->resident;
  a.scale = pl->scale;
  const int64_t groups = (rows + st->tb - 1) / st->tb;
  if (!st->persist && groups > st->grid_cap) return FFT_ERR_INVALID_SIZE;
  const int64_t grid = std::min<int64_t>(groups, st->grid_cap);
  void *args[] = {&a};
  return cuda_status(
      cudaLaunchKernel(st->fn, dim3((unsigned)grid), dim3(st->threads), args, st->smem, stream));
}

void tc_destroy(fft_plan_impl *pl) {
  TcState *st = (TcState *)pl->tc;
  if (st) {
    cudaFree(st->d_bimg);
    cudaFree(st->d_twx);
  }
  delete st;
  pl->tc = nullptr;
}

}  // namespace fftgb
