// Column FFTs: batched length-L transforms down the columns of a row-major
// matrix, C adjacent columns per CTA.  This is the building block of the
// two-phase four-step path (paper Sec. IV-B, Eq. 3 and Sec. V-D):
//
//   N = N1 N2, input index n = n1 + N1 n2, output index k = k2 + N2 k1.
//   phase 1: for every n1, the N2-point FFT over n2 of x[n1 + N1 n2], times
//            the four-step twiddle W_N^{n1 k2}, stored as A[n1][k2];
//   phase 2: for every k2, the N1-point FFT over n1 of A[n1][k2], stored at
//            X[k2 + N2 k1].
//
// Both phases read C consecutive columns of every row, so each warp load
// covers whole row segments (128 bytes at C = 16; 32 bytes, one sector, at
// the narrowest C = 4).  In shared memory element (row, c) of the tile sits
// at row * C + c: with C = 16 a half-warp always touches 16 consecutive
// columns, so every exchange is free of bank conflicts without a swizzle.
// Phase 1 stores its result transposed (column-major) through a padded
// shared tile so that the global store is coalesced as well.
//
// Phase-1 twiddle W_N^{c k} for column c and output k: register m of thread
// lt holds k = lt + T m (T = L / P), so W_N^{c k} = W_N^{c lt} W_N^{c T m},
// the product of two exact table entries from grids laid out [lt][c] and
// [m][c]: a warp's loads read C consecutive columns (whole sectors) instead
// of gathering one sector per element from a table of all N powers.
//
// Columns longer than one CTA holds (L = L1 L2 > 4096) run the same two
// phases down the column instead of along a row: input row n = n1 + L1 n2,
// output row k = k2 + L2 k1.  Phase 1 is an L2-point column FFT of each of the
// L1 sub-matrices n1 (rows n1, n1 + L1, ...), times W_L^{n1 k2}, the twiddle
// now indexed by the sub-matrix rather than the column (TWM == 2; a table
// laid out [n1][k2] of exact powers, one contiguous slice per CTA); phase 2
// is an L1-point column FFT of each of the L2 sub-matrices k2 of the phase-1
// result, stored to rows k2 + L2 k1.  A launch therefore covers nmat matrices
// of nsub sub-matrices each, sub-matrix j of matrix m starting at
// m * mat_stride + j * sub_stride.
#pragma once
#include "stockham.cuh"

namespace fftgb {

struct ColumnArgs {
  const float2 *in;
  float2 *out;
  const float2 *tw;      // per-pass tables of the length-L transform
  const float2 *tw_a;    // TWM 1: W_Ntot^{c lt} at lt * ncols + c; TWM 2:
                         // W_Ntot^{j k} at j * L + k for sub-matrix j; else null
  const float2 *tw_b;    // TWM 1: W_Ntot^{c T m} at m * ncols + c
  long long nmat;        // number of matrices times nsub
  long long in_mat_stride, out_mat_stride;  // elements between matrices
  long long in_sub_stride, out_sub_stride;  // elements between sub-matrices
  int nsub;              // sub-matrices per matrix (0 and 1: one)
  long long in_extent, out_extent;  // elements reachable from in / out (bounds-check build)
  int in_row_stride;     // elements between consecutive rows of the input
  int out_row_stride;    // elements between rows of a non-transposed output
  int ncols;             // columns per matrix (multiple of C)
  int ntot;              // L * ncols, the size of the four-step twiddle
  float scale;
};

// TWM: 0 no twiddle, 1 the row four-step's per-column twiddle (with a
// transposed store), 2 the per-sub-matrix twiddle of a long column.
template <int L, int P, int C, int D, class SC, int TWM, bool TRANSPOSED>
__global__ void __launch_bounds__(C *(L / P))
column_kernel(ColumnArgs args) {
  static_assert(SC::product() == L, "radix schedule must multiply to L");
  static_assert(P % SC::max_radix() == 0, "every radix must divide P");
  constexpr int T = L / P;
  constexpr int NT = C * T;
  extern __shared__ __align__(128) float2 smem[];
  // Programmatic dependent launch (see stockham_kernel) up to 2048-point
  // columns: phase 2 may become resident while phase 1 finishes, but reads
  // nothing before it completed.  The 4096-point kernels (one 128 KiB CTA
  // per SM, many waves) are launched plainly and carry neither instruction.
  if constexpr (L <= 2048) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  }
  const int c = threadIdx.x % C;
  const int lt = threadIdx.x / C;
  const int tiles_per_mat = args.ncols / C;
  const long long tile_mat = blockIdx.x / tiles_per_mat;
  const int c0 = (int)(blockIdx.x - tile_mat * tiles_per_mat) * C;
  long long mat = tile_mat, sub = 0;
  if (args.nsub > 1) {
    mat = tile_mat / args.nsub;
    sub = tile_mat - mat * args.nsub;
  }
  float2 a[P];
  {
    const long long base = mat * args.in_mat_stride + sub * args.in_sub_stride + c0 + c;
    const float2 *src = args.in + base;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const long long off = (long long)(lt + m * T) * args.in_row_stride;
      a[m] = FFTGB_OK(base + off, args.in_extent, kSiteColLoad) ? __ldg(src + off)
                                                               : make_float2(0.f, 0.f);
    }
  }
  run_passes<L, P, D, SC, 0>(a, lt, smem, args.tw, Interleaved<C>{c});
  // a[m] now holds output index final_index(lt, m) of column c0 + c.
  if constexpr (TWM == 1) {
    const int col = c0 + c;
    const float2 wa = __ldg(args.tw_a + (long long)lt * args.ncols + col);
#pragma unroll
    for (int m = 0; m < P; ++m) {  // final_index(lt, m) = lt + T m
      const float2 w = cmul(wa, __ldg(args.tw_b + (long long)m * args.ncols + col));
      a[m] = cmul_dir<D>(a[m], w);
    }
  } else if constexpr (TWM == 2) {
    // W_L^{sub k}: the CTA reads one contiguous row of L entries, a warp at
    // most two adjacent entries per load (all C columns share k).
    const float2 *tw = args.tw_a + sub * L;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int k = final_index<L, P, SC>(lt, m);
      if (FFTGB_OK(sub * L + k, (long long)(args.nsub > 1 ? args.nsub : 1) * L, kSiteColTwiddle))
        a[m] = cmul_dir<D>(a[m], __ldg(tw + k));
    }
  }
  if constexpr (TRANSPOSED) {
    // out[col * L + k]: stage through a tile padded to C + 1 columns.
    constexpr int LD = C + 1;
    __syncthreads();
#pragma unroll
    for (int m = 0; m < P; ++m) smem[final_index<L, P, SC>(lt, m) * LD + c] = a[m];
    __syncthreads();
    const long long base = mat * args.out_mat_stride + (long long)c0 * L;
    float2 *dst = args.out + base;
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int e = threadIdx.x + u * NT;  // e = col_local * L + k
      const int cl = e / L, k = e - cl * L;
      if (FFTGB_OK(base + e, args.out_extent, kSiteColStore))
        dst[e] = cscale(smem[k * LD + cl], args.scale);
    }
  } else {
    const long long base = mat * args.out_mat_stride + sub * args.out_sub_stride + c0 + c;
    float2 *dst = args.out + base;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const long long off = (long long)final_index<L, P, SC>(lt, m) * args.out_row_stride;
      if (FFTGB_OK(base + off, args.out_extent, kSiteColStore)) dst[off] = cscale(a[m], args.scale);
    }
  }
}

}  // namespace fftgb
