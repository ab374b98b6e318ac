// Split-precision tensor-core FFT: radix-16 DFT blocks as dense FP16/BF16
// contractions with FP32 accumulation (paper Sec. V-C, Eq. 5-6, where the
// Apple kernel maps DFT_8 onto 8x8 matrix units; here DFT_16 maps onto the
// m16n8k16 tensor-core shape, the tcFFT idea of Sec. VIII).
//
// One radix-16 Stockham stage over 16 butterflies is the real product
//     D (16 x 32) = X^T (16 x 32) . G^T (32 x 32),
// row b of X^T = [Re x_b(0..15), Im x_b(0..15)] (the twiddled inputs of
// butterfly b), G = [[Fr, -Fi], [Fi, Fr]] with F = (W_16^{jk}) (conjugated for
// the inverse), row b of D = [Re X_b(0..15), Im X_b(0..15)].  Both operands
// are split into a high and a low 16-bit part, v = hi + lo with
// hi = round16(v), lo = round16(v - hi), and the product is accumulated in
// FP32 as hi.hi + hi.lo + lo.hi (lo.lo, ~2^-22 relative, is dropped).  The
// split doubles the operand precision to ~22 bits (FP16) / ~16 bits (BF16).
//
// Mapping: a warp owns groups of 16 butterflies; lane (g = lane / 4,
// t = lane % 4) owns butterflies g and g + 8 of the group and their points
// {2t, 2t+1, 2t+8, 2t+9} -- exactly the A-fragment (row g / g+8, columns
// 2t.., 2t+8..) and accumulator (row g / g+8, columns 2t..) positions of
// mma.m16n8k16, so no shuffles are needed.  Stages exchange through shared
// memory like the FP32 Stockham passes; twiddles between stages are FP32
// from the FP64-generated pass tables; N = 16384's radix-4 tail runs on the
// CUDA cores.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "plan.h"
#include "stockham.cuh"

namespace fftgb {

struct TcArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;        // pass tables of the radix schedule (16,16[,16][,4])
  const uint32_t *frag;    // B fragments: [hi/lo][kt 2][nt 4][lane 32][2] u32
  long long batch;
  float scale;
};

// 16-bit split of v: hi = round(v), lo = round(v - hi), packed two per u32.
template <int PREC>
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  if constexpr (PREC == FFT_PREC_FP16X2) {
    __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
    __half l0 = __float2half_rn(v0 - __half2float(h0));
    __half l1 = __float2half_rn(v1 - __half2float(h1));
    __half2 H = __halves2half2(h0, h1), L = __halves2half2(l0, l1);
    hi = *reinterpret_cast<uint32_t *>(&H);
    lo = *reinterpret_cast<uint32_t *>(&L);
  } else {
    __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
    __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    __nv_bfloat162 H = __halves2bfloat162(h0, h1), L = __halves2bfloat162(l0, l1);
    hi = *reinterpret_cast<uint32_t *>(&H);
    lo = *reinterpret_cast<uint32_t *>(&L);
  }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  if constexpr (PREC == FFT_PREC_FP16X2) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// DFT_16 of the lane's two butterflies on the tensor cores.  x[r][c]: row
// r (0: butterfly g, 1: g + 8), point c (0..3 -> 2t, 2t+1, 2t+8, 2t+9);
// replaced by the outputs at the same (row, index) positions.
template <int PREC>
__device__ __forceinline__ void tc_dft16(float2 (&x)[2][4], const uint32_t *__restrict__ fr,
                                         int lane) {
  uint32_t ah[2][4], al[2][4];  // [kt: 0 = real parts, 1 = imaginary parts][a-reg]
#pragma unroll
  for (int kt = 0; kt < 2; ++kt) {
    auto comp = [&](const float2 &v) { return kt == 0 ? v.x : v.y; };
    split2<PREC>(comp(x[0][0]), comp(x[0][1]), ah[kt][0], al[kt][0]);  // row g,   cols 2t..
    split2<PREC>(comp(x[1][0]), comp(x[1][1]), ah[kt][1], al[kt][1]);  // row g+8, cols 2t..
    split2<PREC>(comp(x[0][2]), comp(x[0][3]), ah[kt][2], al[kt][2]);  // row g,   cols 2t+8..
    split2<PREC>(comp(x[1][2]), comp(x[1][3]), ah[kt][3], al[kt][3]);  // row g+8, cols 2t+8..
  }
  float acc[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[nt][r] = 0.f;
#pragma unroll
  for (int kt = 0; kt < 2; ++kt) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const uint2 bh = *reinterpret_cast<const uint2 *>(fr + (((0 * 2 + kt) * 4 + nt) * 32 + lane) * 2);
      const uint2 bl = *reinterpret_cast<const uint2 *>(fr + (((1 * 2 + kt) * 4 + nt) * 32 + lane) * 2);
      mma16816<PREC>(acc[nt], ah[kt], bh.x, bh.y);
      mma16816<PREC>(acc[nt], ah[kt], bl.x, bl.y);
      mma16816<PREC>(acc[nt], al[kt], bh.x, bh.y);
    }
  }
  // accumulator (row g / g+8, cols nt*8 + 2t + {0,1}); cols 0..15 real, 16..31 imag
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    x[r][0] = make_float2(acc[0][2 * r + 0], acc[2][2 * r + 0]);
    x[r][1] = make_float2(acc[0][2 * r + 1], acc[2][2 * r + 1]);
    x[r][2] = make_float2(acc[1][2 * r + 0], acc[3][2 * r + 0]);
    x[r][3] = make_float2(acc[1][2 * r + 1], acc[3][2 * r + 1]);
  }
}

__device__ __forceinline__ int tc_point(int t, int c) { return 2 * t + (c & 1) + (c >> 1) * 8; }

// Shared-memory layout of the exchange after TC stage e: bit b (b < 4) of a
// position is XOR-ed with bit src[e][b] (>= 4, or none), a permutation within
// each 16-point block.  The source bits were chosen (by exhaustive search on a
// model of the lane -> (butterfly, point) map) so that the half-warp accesses
// of the writing stage and of the reading stage (TC gather or radix-4 tail)
// hit at most 2 accesses per bank pair; the direct layout gives 4.
__host__ __device__ constexpr int tc_src(int N, int e, int b) {
  // rows: exchange e; columns: target bit b = 0..3
  return N == 256     ? (e == 0 ? (b == 0 ? 4 : b == 1 ? -1 : b == 2 ? 6 : 5) : -1)
         : N == 4096  ? (e == 0   ? (b == 0 ? 4 : b == 1 ? -1 : b == 2 ? 9 : 5)
                         : e == 1 ? (b == 2 ? 5 : b == 3 ? 9 : -1)
                                  : -1)
         : N == 16384 ? (e == 0   ? (b == 0 ? 4 : b == 1 ? -1 : b == 2 ? 11 : 5)
                         : e == 1 ? (b == 2 ? 5 : b == 3 ? 11 : -1)
                         : e == 2 ? (b == 2 ? 9 : b == 3 ? 10 : -1)
                                  : -1)
                      : -1;
}

template <int N>
__device__ __forceinline__ int tc_swz(int pos, int e) {
  int a = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int sb = tc_src(N, e, b);
    if (sb >= 0) a |= ((pos >> sb) & 1) << b;
  }
  return pos ^ a;
}

// N = 16^S (S TC stages) or 16^S * 4 (radix-4 tail).  WPR warps per row, TB
// rows per CTA, G groups of 16 butterflies per warp per stage.
template <int N, int D, int PREC, int S, int TAIL, int WPR, int TB, int G>
__global__ void __launch_bounds__(TB *WPR * 32)
tc_kernel(TcArgs a) {
  constexpr int NB = N / 16;          // butterflies per TC stage
  static_assert(NB == WPR * G * 16, "groups must cover the stage");
  constexpr int RT = WPR * 32;        // threads per row
  extern __shared__ __align__(16) float2 smem[];
  __shared__ uint32_t fr[2 * 2 * 4 * 32 * 2];  // this direction's B fragments
  for (int i = threadIdx.x; i < 2 * 2 * 4 * 32 * 2; i += blockDim.x) fr[i] = __ldg(a.frag + i);
  const int rb = threadIdx.x / RT;     // row slot in the CTA
  const int rt = threadIdx.x - rb * RT;
  const int warp = rt / 32, lane = rt & 31;
  const int g = lane >> 2, t = lane & 3;
  float2 *buf = smem + (size_t)rb * N;
  const long long row = (long long)blockIdx.x * TB + rb;
  const bool active = row < a.batch;
  const float2 *src = a.in + row * N;
  float2 x[G][2][4];
  __syncthreads();  // fragments staged
  const float2 *tw = a.tw;
  int p = 1;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    // gather: butterfly i = i0 + g + 8 r, point j = tc_point(t, c): input i + j NB
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int i0 = (warp * G + q) * 16;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int idx = i0 + g + 8 * r + tc_point(t, c) * NB;
          if (s == 0) x[q][r][c] = active ? __ldcs(src + idx) : make_float2(0.f, 0.f);
          else x[q][r][c] = buf[tc_swz<N>(idx, s - 1)];
        }
    }
    if (s > 0) __syncthreads();  // every read of the buffer is done
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int i0 = (warp * G + q) * 16;
      if (s > 0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int k = (i0 + g + 8 * r) & (p - 1);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = tc_point(t, c);
            if (j) x[q][r][c] = cmul_dir<D>(x[q][r][c], __ldg(tw + (j - 1) * p + k));
          }
        }
      }
      tc_dft16<PREC>(x[q], fr, lane);
      const bool last = (s == S - 1) && !TAIL;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i = i0 + g + 8 * r;
        const int k = i & (p - 1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int pos = (i - k) * 16 + k + tc_point(t, c) * p;
          if (last) {
            if (active) __stcs(a.out + row * N + pos, cscale(x[q][r][c], a.scale));
          } else {
            buf[tc_swz<N>(pos, s)] = x[q][r][c];
          }
        }
      }
    }
    if (s > 0) tw += 15 * p;
    p *= 16;
    if (s + 1 < S || TAIL) __syncthreads();
  }
  if constexpr (TAIL == 4) {
    // radix-4 pass on the CUDA cores: p = N / 4, butterfly i reads i + j N/4
    constexpr int Q = (N / 4) / RT;  // butterflies per thread
    float2 v[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[q][j] = buf[tc_swz<N>(rt + q * RT + j * (N / 4), S - 1)];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = rt + q * RT;  // i = k since i < p
#pragma unroll
      for (int j = 1; j < 4; ++j) v[q][j] = cmul_dir<D>(v[q][j], __ldg(tw + (j - 1) * p + k));
      float2 w[4] = {v[q][0], v[q][1], v[q][2], v[q][3]};
      Dft<4, D>::run(w);
      if (active)
#pragma unroll
        for (int j = 0; j < 4; ++j) __stcs(a.out + row * N + k + j * (N / 4), cscale(w[j], a.scale));
    }
  }
}

// B fragments of G^T for both directions, from the FP64 DFT-16 matrix:
// frag[dir][hl][kt][nt][lane][e], e = 0..3 halves (2 u32): rows k of G^T are
// kt*16 + 2t + {0,1} (e = 0,1) and + 8 (e = 2,3), column n = nt*8 + g.
template <int PREC>
__global__ void tc_gen_fragments(uint32_t *frag) {
  const int lane = threadIdx.x & 31;
  const int nt = (threadIdx.x >> 5) & 3;
  const int kt = (threadIdx.x >> 7) & 1;
  const int dir = (threadIdx.x >> 8) & 1;  // 0: forward, 1: inverse
  const int g = lane >> 2, t = lane & 3;
  const int col = nt * 8 + g;              // output component: < 16 real, else imag
  float hv[4], lv[4];
  for (int e = 0; e < 4; ++e) {
    const int comp = kt * 16 + 2 * t + (e & 1) + (e >> 1) * 8;  // input component
    const int n = comp & 15, k = col & 15;
    // W_16^{kn} with the sign of the direction, FP64
    double s, c;
    sincospi((dir ? 2.0 : -2.0) * (double)((k * n) % 16) / 16.0, &s, &c);
    // G[col][comp]: [[Fr, -Fi], [Fi, Fr]]
    double v;
    if (col < 16) v = (comp < 16) ? c : -s;
    else v = (comp < 16) ? s : c;
    if (PREC == FFT_PREC_FP16X2) {
      __half h = __double2half(v);
      hv[e] = __half2float(h);
      lv[e] = (float)(v - (double)hv[e]);
    } else {
      __nv_bfloat16 h = __double2bfloat16(v);
      hv[e] = __bfloat162float(h);
      lv[e] = (float)(v - (double)hv[e]);
    }
  }
  for (int hl = 0; hl < 2; ++hl) {
    const float *src = hl ? lv : hv;
    uint32_t u0, u1, dummy;
    split2<PREC>(src[0], src[1], u0, dummy);
    split2<PREC>(src[2], src[3], u1, dummy);
    uint32_t *dst = frag + (size_t)dir * 2048 + (((hl * 2 + kt) * 4 + nt) * 32 + lane) * 2;
    dst[0] = u0;
    dst[1] = u1;
  }
}

struct TcState {
  uint32_t *d_frag = nullptr;
  const void *fn = nullptr;
  int threads = 0, tb = 0;
  size_t smem = 0;
};

template <int N, int PREC, int S, int TAIL, int WPR, int TB, int G>
static void pick(TcState *st, int dir) {
  st->fn = dir < 0 ? (const void *)&tc_kernel<N, -1, PREC, S, TAIL, WPR, TB, G>
                   : (const void *)&tc_kernel<N, +1, PREC, S, TAIL, WPR, TB, G>;
  st->threads = TB * WPR * 32;
  st->tb = TB;
  st->smem = sizeof(float2) * (size_t)N * TB;
}

template <int PREC>
static bool pick_prec(TcState *st, int N, int dir) {
  switch (N) {
    case 256: pick<256, PREC, 2, 0, 1, 8, 1>(st, dir); return true;
    case 4096: pick<4096, PREC, 3, 0, 16, 1, 1>(st, dir); return true;
    case 16384: pick<16384, PREC, 3, 4, 16, 1, 4>(st, dir); return true;
  }
  return false;
}

fft_status_t tc_plan(fft_plan_impl *pl) {
  TcState *st = new (std::nothrow) TcState;
  if (!st) return FFT_ERR_ALLOC;
  pl->tc = st;
  const bool ok = pl->precision == FFT_PREC_FP16X2 ? pick_prec<FFT_PREC_FP16X2>(st, pl->N, pl->direction)
                                                  : pick_prec<FFT_PREC_BF16X2>(st, pl->N, pl->direction);
  if (!ok) return FFT_ERR_NOT_SUPPORTED;
  if (st->smem > 48 * 1024 &&
      cudaFuncSetAttribute(st->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem) !=
          cudaSuccess)
    return FFT_ERR_CUDA;
  // twiddle tables: schedule 16, 16[, 16][, 4]
  KernelEntry k{};
  k.npass = pl->N == 256 ? 2 : pl->N == 4096 ? 3 : 4;
  for (int i = 0; i < 3; ++i) k.radix[i] = 16;
  if (pl->N == 16384) k.radix[3] = 4;
  int64_t off = 0;
  fft_status_t s = build_twiddles(pl, pass_segments(k, off));
  if (s != FFT_OK) return s;
  if (cudaMalloc(&st->d_frag, 2 * 2048 * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return FFT_ERR_ALLOC;
  }
  if (pl->precision == FFT_PREC_FP16X2) tc_gen_fragments<FFT_PREC_FP16X2><<<1, 512>>>(st->d_frag);
  else tc_gen_fragments<FFT_PREC_BF16X2><<<1, 512>>>(st->d_frag);
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
  a.frag = st->d_frag + (pl->direction > 0 ? 2048 : 0);
  a.batch = rows;
  a.scale = pl->scale;
  const int64_t grid = (rows + st->tb - 1) / st->tb;
  if (grid > 0x7fffffffLL) return FFT_ERR_INVALID_SIZE;
  void *args[] = {&a};
  return cuda_status(
      cudaLaunchKernel(st->fn, dim3((unsigned)grid), dim3(st->threads), args, st->smem, stream));
}

void tc_destroy(fft_plan_impl *pl) {
  TcState *st = (TcState *)pl->tc;
  if (st) cudaFree(st->d_frag);
  delete st;
  pl->tc = nullptr;
}

}  // namespace fftgb
