// Spectral-filter kernels for the differentiable SAR range-compression layer
// (paper Sec. II-D: range compression is a batched FFT, a pointwise
// multiplication by the matched filter and an inverse FFT).
//
//   forward   z = FFT(x) * H,  y = IFFT(z)
//   backward  g_z = G^H g_y = (1/N) FFT(g_y)      (adjoint of the inverse)
//             grad_H = sum_rows conj(FFT(x)) * g_z
//             grad_x = F^H (conj(H) * g_z)         (adjoint of the forward)
//
// The transforms are the library's plans; this unit holds the pointwise
// multiply and the batch reduction for grad_H.
#include <cuda_runtime.h>
#include <stdint.h>

#include "butterfly.cuh"
#include "plan.h"

namespace fftgb {

// Z = X * H (or X * conj H), times scale; two complex points per thread.
template <bool CONJ>
__global__ void filter_apply_kernel(const float4 *__restrict__ X, const float4 *__restrict__ H,
                                    float4 *Z, int halfN, int64_t total_half, float scale) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_half; i += stride) {
    const int k = (int)(i % halfN);
    float4 x = __ldg(X + i);
    float4 h = __ldg(H + k);
    float2 a = make_float2(x.x, x.y), b = make_float2(x.z, x.w);
    float2 ha = make_float2(h.x, h.y), hb = make_float2(h.z, h.w);
    a = CONJ ? cmulc(a, ha) : cmul(a, ha);
    b = CONJ ? cmulc(b, hb) : cmul(b, hb);
    Z[i] = make_float4(a.x * scale, a.y * scale, b.x * scale, b.y * scale);
  }
}

// Stage 1: partial[c][k] = sum over the rows of chunk c, in row order, of
// conj(X[b][k]) * G[b][k].  Stage 2: grad_H[k] = pairwise sum over chunks.
constexpr int kRowsPerChunk = 32;

__global__ void grad_h_partial_kernel(const float2 *__restrict__ X, const float2 *__restrict__ G,
                                      float2 *partial, int N, int64_t batch) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (k >= N) return;
  const int64_t b0 = c * kRowsPerChunk;
  const int rows = (int)(batch - b0 < kRowsPerChunk ? batch - b0 : kRowsPerChunk);
  // Unrolled over the chunk with predicated loads, so all of a thread's
  // loads are in flight at once; the sum still runs in row order.
  float2 xs[kRowsPerChunk], gs[kRowsPerChunk];
#pragma unroll
  for (int i = 0; i < kRowsPerChunk; ++i) {
    const bool on = i < rows;
    xs[i] = on ? __ldcs(X + (b0 + i) * N + k) : make_float2(0.f, 0.f);
    gs[i] = on ? __ldcs(G + (b0 + i) * N + k) : make_float2(0.f, 0.f);
  }
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < kRowsPerChunk; ++i) {
    // conj(x) * g (zero for rows past the batch)
    acc.x = fmaf(xs[i].x, gs[i].x, fmaf(xs[i].y, gs[i].y, acc.x));
    acc.y = fmaf(xs[i].x, gs[i].y, fmaf(-xs[i].y, gs[i].x, acc.y));
  }
  partial[c * N + k] = acc;
}

// Pairwise tree over chunks: level by level, partial[c] += partial[c + h].
__global__ void grad_h_tree_kernel(float2 *partial, int N, int64_t nchunk, int64_t h) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = (int64_t)blockIdx.y * 2 * h;
  if (k >= N || c + h >= nchunk) return;
  float2 a = partial[c * N + k], b = partial[(c + h) * N + k];
  partial[c * N + k] = make_float2(a.x + b.x, a.y + b.y);
}

// The same pairwise tree in one launch.  A CTA owns kTreeCols frequencies.
// Each thread loads aligned blocks of kTreeBlk consecutive chunks of one
// frequency (all of a block's loads in flight together) and runs the tree's
// first levels (h = 1, 2, 4) inside the block in registers; the block sums go
// to shared memory, where the remaining levels run over blocks.  Levels h <
// kTreeBlk only pair chunks inside an aligned block, and level kTreeBlk * hb
// pairs block b with block b + hb exactly when chunk 8 (b + hb) exists, so
// the additions and their order are those of grad_h_tree_kernel and the
// result is identical.  Used while the block sums fit the shared memory
// (kTreeMaxChunks).
constexpr int kTreeCols = 16;
constexpr int kTreeThreads = 256;
constexpr int kTreeBlk = 8;
constexpr int64_t kTreeMaxChunks = 4096;  // 512 blocks x 16 x 8 B = 64 KiB

__global__ void __launch_bounds__(kTreeThreads) grad_h_tree_smem_kernel(const float2 *partial,
                                                                       float2 *out, int N,
                                                                       int nchunk) {
  extern __shared__ float2 tree[];  // [nblk][kTreeCols] block sums
  const int k0 = blockIdx.x * kTreeCols;
  const int f = threadIdx.x % kTreeCols, lane = threadIdx.x / kTreeCols;
  constexpr int kLanes = kTreeThreads / kTreeCols;
  const bool on = k0 + f < N;
  const int nblk = (nchunk + kTreeBlk - 1) / kTreeBlk;
  for (int bl = lane; bl < nblk; bl += kLanes) {
    const int c0 = bl * kTreeBlk;
    float2 v[kTreeBlk];
#pragma unroll
    for (int i = 0; i < kTreeBlk; ++i)
      v[i] = on && c0 + i < nchunk ? __ldcs(partial + (int64_t)(c0 + i) * N + k0 + f)
                                   : make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 1; h < kTreeBlk; h *= 2) {
#pragma unroll
      for (int i = 0; i + h < kTreeBlk; i += 2 * h)
        if (c0 + i + h < nchunk) v[i] = make_float2(v[i].x + v[i + h].x, v[i].y + v[i + h].y);
    }
    tree[bl * kTreeCols + f] = v[0];
  }
  __syncthreads();
  for (int h = 1; h < nblk; h *= 2) {
    for (int b = 2 * h * lane; b + h < nblk; b += 2 * h * kLanes) {
      const float2 a = tree[b * kTreeCols + f], c = tree[(b + h) * kTreeCols + f];
      tree[b * kTreeCols + f] = make_float2(a.x + c.x, a.y + c.y);
    }
    __syncthreads();
  }
  if (lane == 0 && on) out[k0 + f] = tree[f];
}

__global__ void copy_row_kernel(const float2 *src, float2 *dst, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) dst[k] = src[k];
}

static bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// grad_H[k] = fixed-order pairwise sum over the nchunk rows of partial
// ([nchunk][N], overwritten): one launch while the rows fit shared memory,
// else level by level.
fft_status_t grad_h_tree(float2 *partial, float2 *grad_H, int N, int64_t nchunk,
                         cudaStream_t st) {
  const int threads = 256;
  const unsigned bx = (unsigned)((N + threads - 1) / threads);
  if (nchunk <= kTreeMaxChunks) {
    const size_t smem =
        sizeof(float2) * (size_t)((nchunk + kTreeBlk - 1) / kTreeBlk) * kTreeCols;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(grad_h_tree_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return FFT_ERR_CUDA;
    grad_h_tree_smem_kernel<<<(unsigned)((N + kTreeCols - 1) / kTreeCols), kTreeThreads, smem, st>>>(
        partial, grad_H, N, (int)nchunk);
    return cuda_status(cudaGetLastError());
  }
  if (nchunk > 65535 * 2) return FFT_ERR_INVALID_SIZE;
  for (int64_t h = 1; h < nchunk; h *= 2) {
    const int64_t groups = (nchunk + 2 * h - 1) / (2 * h);
    grad_h_tree_kernel<<<dim3(bx, (unsigned)groups), threads, 0, st>>>(partial, N, nchunk, h);
  }
  copy_row_kernel<<<bx, threads, 0, st>>>(partial, grad_H, N);
  return cuda_status(cudaGetLastError());
}

}  // namespace fftgb

using namespace fftgb;

extern "C" {

fft_status_t fft_filter_apply(const void *X, const void *H, void *Z, int N, int64_t batch,
                              int conj_h, float scale, void *stream) {
  if (!pow2(N) || N < 2 || N > (1 << 30) || batch < 0) return FFT_ERR_INVALID_SIZE;
  if (!X || !H || !Z) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)X | (uintptr_t)H | (uintptr_t)Z) & 15) return FFT_ERR_MISALIGNED;
  if (batch == 0) return FFT_OK;
  const int64_t total_half = (int64_t)N / 2 * batch;
  const int threads = 256;
  int64_t blocks = (total_half + threads - 1) / threads;
  blocks = blocks > 152 * 64 ? 152 * 64 : blocks;
  cudaStream_t st = (cudaStream_t)stream;
  if (conj_h)
    filter_apply_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(
        (const float4 *)X, (const float4 *)H, (float4 *)Z, N / 2, total_half, scale);
  else
    filter_apply_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(
        (const float4 *)X, (const float4 *)H, (float4 *)Z, N / 2, total_half, scale);
  return cuda_status(cudaGetLastError());
}

int64_t fft_filter_grad_h_workspace(int N, int64_t batch) {
  if (N <= 0 || batch <= 0) return 0;
  const int64_t nchunk = (batch + kRowsPerChunk - 1) / kRowsPerChunk;
  return nchunk * N * (int64_t)sizeof(float2);
}

fft_status_t fft_filter_grad_h(const void *X, const void *G, void *grad_H, int N, int64_t batch,
                               void *work, void *stream) {
  if (!pow2(N) || N < 2 || N > (1 << 30) || batch < 0) return FFT_ERR_INVALID_SIZE;
  if (!X || !G || !grad_H || (batch > 0 && !work)) return FFT_ERR_INVALID_VALUE;
  if (((uintptr_t)X | (uintptr_t)G | (uintptr_t)grad_H | (uintptr_t)work) & 7)
    return FFT_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  const unsigned bx = (unsigned)((N + threads - 1) / threads);
  if (batch == 0) {
    return cuda_status(cudaMemsetAsync(grad_H, 0, sizeof(float2) * (size_t)N, st));
  }
  const int64_t nchunk = (batch + kRowsPerChunk - 1) / kRowsPerChunk;
  if (nchunk > 65535) return FFT_ERR_INVALID_SIZE;
  float2 *part = (float2 *)work;
  grad_h_partial_kernel<<<dim3(bx, (unsigned)nchunk), threads, 0, st>>>(
      (const float2 *)X, (const float2 *)G, part, N, batch);
  return grad_h_tree(part, (float2 *)grad_H, N, nchunk, st);
}

}  // extern "C"
