// Register-resident DFT butterflies for the Stockham passes.
//
// DFT_R on R complex values held in registers, DIT, natural order in and out.
//   R = 2, 4     written out directly;
//   R = 8        split-radix DIT (paper Sec. V-B): radix-2 combination of the
//                even and odd DFT_4, the odd half rotated by W_8^k;
//   R = 16, 32   the same radix-2 DIT step applied to two DFT_8 / DFT_16.
// D is the sign of the exponent: D = -1 forward (W = e^{-2 pi i/R}), D = +1
// inverse.  Multiplications by the constant roots W_R^k use exact special
// cases for k*8/R integral (1, -i, W_8) and two FMUL + two FFMA otherwise.
// Inside the radix-2 combine steps the rotation is fused into the butterfly
// (e +- o w) in the tangent form: with w = c + i s and g the larger of |c|
// and |s|, o w = g u where u = o rotated by the ratio of the smaller to g
// (|ratio| <= 1), so the pair costs 2 FFMA for u and 4 FFMA for e +- g u:
// six instructions instead of eight (four for o w, four for the add and
// the subtract).  On sm_100 and later the two components of every complex
// add, FMA and product issue as one packed FP32x2 instruction (FADD2, FFMA2,
// FMUL2) with the scalar forms' roundings, so results are bit-identical and
// the six FMAs of a rotated butterfly pair are three instructions.
// Twiddle mode 1 helpers (tw_loaded, cmul_pm, derive_twiddles) form a pass's
// twiddle powers from the few table rows it reads.
#pragma once
#include <cuda_runtime.h>

namespace fftgb {

// Complex add and subtract.  On sm_100 and later one packed FP32x2 add
// (FADD2) does both components: round-to-nearest like two scalar adds, so
// bit-identical results in half the issue slots.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fmul2_rn(a, make_float2(s, s));
#else
  return make_float2(a.x * s, a.y * s);
#endif
}

// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  const float2 t = __fmul2_rn(make_float2(a.y, a.y), make_float2(w.y, w.x));
  return __ffma2_rn(make_float2(a.x, a.x), w, make_float2(-t.x, t.y));
#else
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
#endif
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  const float2 t = __fmul2_rn(make_float2(a.y, a.x), make_float2(w.y, w.y));
  return __ffma2_rn(make_float2(a.x, a.y), make_float2(w.x, w.x), make_float2(t.x, -t.y));
#else
  return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
#endif
}
// a * w (D = -1) or a * conj(w) (D = +1): tables hold forward roots.
template <int D>
__device__ __forceinline__ float2 cmul_dir(float2 a, float2 w) {
  if constexpr (D < 0) return cmul(a, w);
  else return cmulc(a, w);
}
// a * (D i): multiplication by W_4 (forward: -i, inverse: +i)
template <int D>
__device__ __forceinline__ float2 rot90(float2 a) {
  if constexpr (D < 0) return make_float2(a.y, -a.x);
  else return make_float2(-a.y, a.x);
}

// cos(j pi / 16), j = 0..8, in FP32 and in FP64 (the FP64 copy forms the
// tangent-form ratios before their single rounding to FP32)
struct Cos16d {
  static constexpr double d[9] = {1.0,
                                  0.98078528040323044913,
                                  0.92387953251128675613,
                                  0.83146961230254523708,
                                  0.70710678118654752440,
                                  0.55557023301960222474,
                                  0.38268343236508977173,
                                  0.19509032201612826785,
                                  0.0};
};
struct Cos16 {
  static constexpr float c[9] = {1.0f,
                                 0.98078528040323044913f,
                                 0.92387953251128675613f,
                                 0.83146961230254523708f,
                                 0.70710678118654752440f,
                                 0.55557023301960222474f,
                                 0.38268343236508977173f,
                                 0.19509032201612826785f,
                                 0.0f};
};

// v * exp(D * 2 pi i * m / 32) for a compile-time m in [0, 32).
template <int M, int D>
__device__ __forceinline__ float2 rot32(float2 v) {
  constexpr int m = ((M % 32) + 32) % 32;
  constexpr int q = m / 8, r = m % 8;
  // cos and sin of the angle 2 pi m / 32 = m pi / 16 (before the sign D)
  constexpr float c = (q == 0) ? Cos16::c[r] : (q == 1) ? -Cos16::c[8 - r]
                    : (q == 2) ? -Cos16::c[r] : Cos16::c[8 - r];
  constexpr float s0 = (q == 0) ? Cos16::c[8 - r] : (q == 1) ? Cos16::c[r]
                     : (q == 2) ? -Cos16::c[8 - r] : -Cos16::c[r];
  constexpr float s = (D < 0) ? -s0 : s0;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 8) {
    return rot90<D>(v);
  } else if constexpr (m == 16) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 24) {
    return rot90<-D>(v);
  } else if constexpr (m % 4 == 0) {
    // odd multiples of pi/4: |c| = |s| = sqrt(1/2)
    constexpr float h = Cos16::c[4];
    constexpr float sc = (c > 0.f) ? 1.f : -1.f, ss = (s > 0.f) ? 1.f : -1.f;
    // (x + i y)(sc + i ss) h = h (sc x - ss y) + i h (ss x + sc y)
    float re = (sc > 0.f ? v.x : -v.x) - (ss > 0.f ? v.y : -v.y);
    float im = (ss > 0.f ? v.x : -v.x) + (sc > 0.f ? v.y : -v.y);
    return make_float2(re * h, im * h);
  } else {
    return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
  }
}

template <int R, int D>
struct Dft;

template <int D>
struct Dft<1, D> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

template <int D>
struct Dft<2, D> {
  static __device__ __forceinline__ void run(float2 (&a)[2]) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <int D>
struct Dft<4, D> {
  static __device__ __forceinline__ void run(float2 (&a)[4]) {
    float2 t0 = cadd(a[0], a[2]);
    float2 t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]);
    float2 t3 = rot90<D>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

// lo = e + o w, hi = e - o w for the constant root w = exp(D 2 pi i M / 32).
// Multiples of pi/2 are exact swaps and sign changes; every other root uses
// the tangent form (header): |c| >= |s|: o w = c (o.x - o.y q, o.y + o.x q),
// q = s / c; |s| > |c|: o w = s (o.x q - o.y, o.y q + o.x), q = c / s.
template <int M, int D>
__device__ __forceinline__ void bfly_rot32(float2 e, float2 o, float2 &lo, float2 &hi) {
  constexpr int m = ((M % 32) + 32) % 32;
  if constexpr (m % 8 == 0) {
    const float2 t = rot32<m, D>(o);
    lo = cadd(e, t);
    hi = csub(e, t);
  } else {
    constexpr int q4 = m / 8, r = m % 8;
    // cos and sin of m pi / 16 by quadrant (as in rot32), in FP64
    constexpr double c = (q4 == 0) ? Cos16d::d[r] : (q4 == 1) ? -Cos16d::d[8 - r]
                       : (q4 == 2) ? -Cos16d::d[r] : Cos16d::d[8 - r];
    constexpr double s0 = (q4 == 0) ? Cos16d::d[8 - r] : (q4 == 1) ? Cos16d::d[r]
                        : (q4 == 2) ? -Cos16d::d[8 - r] : -Cos16d::d[r];
    constexpr double s = (D < 0) ? -s0 : s0;
    constexpr bool cbig = (c < 0 ? -c : c) >= (s < 0 ? -s : s);
    constexpr float q = cbig ? (float)(s / c) : (float)(c / s);
    constexpr float g = cbig ? (float)c : (float)s;
    float2 u;
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (cbig) {
      u = __ffma2_rn(make_float2(-o.y, o.x), make_float2(q, q), o);
    } else {
      u = __ffma2_rn(o, make_float2(q, q), make_float2(-o.y, o.x));
    }
#else
    if constexpr (cbig) {
      u = make_float2(fmaf(-o.y, q, o.x), fmaf(o.x, q, o.y));
    } else {
      u = make_float2(fmaf(o.x, q, -o.y), fmaf(o.y, q, o.x));
    }
#endif
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    // e +- g u as two packed FP32x2 FMAs (the same roundings as four scalar ones)
    lo = __ffma2_rn(u, make_float2(g, g), e);
    hi = __ffma2_rn(u, make_float2(-g, -g), e);
#else
    lo = make_float2(fmaf(u.x, g, e.x), fmaf(u.y, g, e.y));
    hi = make_float2(fmaf(u.x, -g, e.x), fmaf(u.y, -g, e.y));
#endif
  }
}

// Radix-2 DIT step: DFT_R from DFT_{R/2} of the even and odd samples.
template <int R, int D, int K>
struct Combine {
  static_assert(32 % R == 0, "constant roots only for R | 32");
  static __device__ __forceinline__ void run(float2 (&a)[R], const float2 (&e)[R / 2],
                                             const float2 (&o)[R / 2]) {
    bfly_rot32<K * (32 / R), D>(e[K], o[K], a[K], a[K + R / 2]);
    if constexpr (K + 1 < R / 2) Combine<R, D, K + 1>::run(a, e, o);
  }
};

template <int R, int D>
struct Dft {
  static_assert(R == 8 || R == 16 || R == 32, "unsupported radix");
  static __device__ __forceinline__ void run(float2 (&a)[R]) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = a[2 * i];
      o[i] = a[2 * i + 1];
    }
    Dft<R / 2, D>::run(e);
    Dft<R / 2, D>::run(o);
    Combine<R, D, 0>::run(a, e, o);
  }
};

// Is row j of a pass table loaded (twiddle mode 1) rather than derived?
template <int r>
__host__ __device__ constexpr bool tw_loaded(int j) {
  return j == 1 || (r == 4 && j == 2) || (r >= 8 && j == 4) || (r == 32 && j == 16);
}

// a b and a conj(b) with their shared products formed once: 2 FMUL + 4 FFMA
// for the two, against 2 x (FMUL + FFMA) x 2 for two separate products.
__device__ __forceinline__ void cmul_pm(float2 a, float2 b, float2 &plus, float2 &minus) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  const float2 tu = __fmul2_rn(make_float2(a.y, a.x), make_float2(b.y, b.y));
  const float2 ab = make_float2(a.x, a.y), bb = make_float2(b.x, b.x);
  plus = __ffma2_rn(ab, bb, make_float2(-tu.x, tu.y));
  minus = __ffma2_rn(ab, bb, make_float2(tu.x, -tu.y));
#else
  const float t = a.y * b.y, u = a.x * b.y;
  plus = make_float2(fmaf(a.x, b.x, -t), fmaf(a.y, b.x, u));
  minus = make_float2(fmaf(a.x, b.x, t), fmaf(a.y, b.x, -u));
#endif
}

// Twiddle mode 1: form the rows that are not read as products of rows
// already formed, W^{(c +- d) k} = W^{c k} W^{+-d k}, the two signs of one
// (c, d) together (cmul_pm), from rows 1, 4 (and 2 for r = 4, 16 for
// r = 32); product depth <= 3.
template <int r>
__device__ __forceinline__ void derive_twiddles(float2 (&w)[r]) {
  if constexpr (r == 4) {
    w[3] = cmul(w[2], w[1]);
  } else if constexpr (r == 8) {
    w[2] = cmul(w[1], w[1]);
    cmul_pm(w[4], w[1], w[5], w[3]);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
  } else if constexpr (r == 16) {
    w[2] = cmul(w[1], w[1]);
    w[8] = cmul(w[4], w[4]);
    cmul_pm(w[4], w[1], w[5], w[3]);
    cmul_pm(w[8], w[1], w[9], w[7]);
    cmul_pm(w[8], w[2], w[10], w[6]);
    w[12] = cmul(w[8], w[4]);
    cmul_pm(w[12], w[1], w[13], w[11]);
    w[14] = cmul(w[12], w[2]);
    w[15] = cmul(w[12], w[3]);
  } else if constexpr (r == 32) {
    w[2] = cmul(w[1], w[1]);
    w[8] = cmul(w[4], w[4]);
    cmul_pm(w[16], w[4], w[20], w[12]);
    w[24] = cmul(w[16], w[8]);
    w[28] = cmul(w[16], w[12]);
    cmul_pm(w[4], w[1], w[5], w[3]);
    cmul_pm(w[8], w[1], w[9], w[7]);
    cmul_pm(w[12], w[1], w[13], w[11]);
    cmul_pm(w[16], w[1], w[17], w[15]);
    cmul_pm(w[20], w[1], w[21], w[19]);
    cmul_pm(w[24], w[1], w[25], w[23]);
    cmul_pm(w[28], w[1], w[29], w[27]);
    cmul_pm(w[8], w[2], w[10], w[6]);
    cmul_pm(w[16], w[2], w[18], w[14]);
    cmul_pm(w[24], w[2], w[26], w[22]);
    w[30] = cmul(w[28], w[2]);
    w[31] = cmul(w[28], w[3]);
  } else {
    static_assert(r == 2, "twiddle mode 1 for radix 2, 4, 8, 16, 32");
  }
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Exchange-buffer layout of one Stockham exchange, chosen by the writing pass
// (stride p, radix r).  For p >= 16 a warp's writes are runs of 16 consecutive
// elements and the identity layout is conflict-free.  For p < 16 a half-warp
// writes at stride p*r; XOR-ing the index bits that carry the lane's high
// bits (bit log2(p*r) upward) into bits [log2 p, 4) makes the 16 targets of a
// half-warp land in 16 distinct 8-byte bank pairs, while a 16-aligned run of
// consecutive indices (the next pass's read) stays a permutation of its block.
template <int p, int r>
__device__ __forceinline__ int swz(int idx) {
  if constexpr (p >= 16) {
    return idx;
  } else {
    constexpr int sh = ilog2(p * r);
    constexpr int mask = 16 / p - 1;
    constexpr int tsh = ilog2(p);
    return idx ^ (((idx >> sh) & mask) << tsh);
  }
}

}  // namespace fftgb
