// Arithmetic policies of the fused apply kernel.
//
//  ArF64    IEEE FP64 on the FP64 pipe: every multiply-add is one DFMA.
//  ArF32x2  FP64-accurate float-float arithmetic on the FP32 pipe (GB300's FP64 pipe delivers
//           ~1.2 TFLOP/s against ~75 TFLOP/s FP32).  A value is the unevaluated sum h + l of two
//           floats (|l| <= ulp(h)).  Two accumulation schemes:
//
//   * anchored dot products (amad*, dot3), used wherever a bound B >= sum_i |a_i x_i| of the sum
//     is known before it starts (a 1D contraction: max_i |x_i| times the 1D table's largest
//     absolute row or column sum; a row of the pointwise D: the exact sum of |a_i| |x_i|).  The
//     high accumulator starts at the anchor sigma = 2^ceil(log2(2 (1 + 2^-9) B)), so it stays
//     within [sigma/2, 3 sigma/2]; then per term
//         t = fma(ah, xh, A);  z = t - A;  r = fma(ah, xh, -z);  L += r;  L += ah xl + al xh
//     z is exact (t and A are multiples of 2^-24 sigma and differ by less than 2^23 of them), so
//     A - sigma is exactly the sum of the parts of the products above that grid, and r, the rest
//     of each product, is rounded once to float -- an error below 2^-48 sigma.  Six FP32
//     instructions per term; the error of the sum is a small multiple of 2^-48 sigma.
//   * compensated dot products (mad*), for sums whose bound is not known in advance (the
//     transposed z contraction at Q > 6, whose inputs are produced on the fly; the mass
//     pointwise product): Dekker's exact product by FMA plus Knuth's TwoSum, twelve
//     instructions per term.
//
//  The primitives (fe_f2.h) are __host__ __device__ with explicit rounding, so the same
//  error-free steps also run in the CPU unit test of that header.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include "fe_f2.h"

namespace fe {

// ---------------------------------------------------------------------------- tables
// 1D basis tables passed by value in the kernel parameter space (constant bank), so that
// fully unrolled contractions read them as immediate constant operands.
template <int D, int Q>
struct TabF64 {
  double B[Q * D];
  double G[Q * D];
};

// Tables with their even-odd halves (FP64, or FP32 for the FP32 policy).  The 1D tables are symmetric under reversal of both
// indices (GLL nodes and Gauss points are symmetric about the element centre):
// B[Q-1-q][D-1-d] = B[q][d] and G[Q-1-q][D-1-d] = -G[q][d].  So a contraction out = M x of a
// line splits into half-size sums over x's even and odd parts
// (ue[i] = x[i] + x[N-1-i], uo[i] = x[i] - x[N-1-i]; ue takes the middle entry of an odd line):
// out[o] = S[o] + Dd[o], out[NO-1-o] = S[o] - Dd[o] (and out[mid] = S[mid]), with
// S[o] = sum_i (M[o][i] + M[NO-1-o][i]) / 2 u_S[i], Dd[o] = sum_i (M[o][i] - M[NO-1-o][i]) / 2 u_D[i],
// where u_S, u_D = ue, uo for the symmetric B and uo, ue for the antisymmetric G.  Forward
// tables are [output q][input d], transposed ones [output d][input q].
template <class R, int D, int Q>
struct TabEO {
  static constexpr int DE = (D + 1) / 2, DH = D / 2, QE = (Q + 1) / 2, QH = Q / 2;
  R B[Q * D];
  R G[Q * D];
  R bS[QE][DE], bD[QH][DH];    // B forward:  S on ue, Dd on uo
  R gS[QE][DH], gD[QH][DE];    // G forward:  S on uo, Dd on ue
  R btS[DE][QE], btD[DH][QH];  // B^T:        S on ue, Dd on uo (over q)
  R gtS[DE][QH], gtD[DH][QE];  // G^T:        S on uo, Dd on ue (over q)
};
template <int D, int Q>
using TabF64EO = TabEO<double, D, Q>;
template <int D, int Q>
using TabF32EO = TabEO<float, D, Q>;

// Float-float tables; rB/rG = max_q sum_d |.| (forward contractions), cB/cG = max_d sum_q |.|
// (transposed contractions), each rounded up.
template <int D, int Q>
struct TabF32x2 {
  float Bh[Q * D], Bl[Q * D];
  float Gh[Q * D], Gl[Q * D];
  float rB, rG, cB, cG;
};

// ---------------------------------------------------------------------------- policies
struct ArF64 {
  static constexpr bool kAnchored = false;
  static constexpr bool kScaled = false;  // inputs converted as they are gathered
  static constexpr bool kPrefetchQd = false;  // FP64-pipe bound: nothing to hide
  using QdT = double;
  using T = double;
  using Acc = double;
  using Sig = float;  // unused
  template <int D, int Q>
  using Tab = TabF64EO<D, Q>;
  // contractions by even-odd halves (fe_apply_eo.cuh): fewer FP64-pipe instructions
  static constexpr bool kEvenOdd = true;

  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T from_vec(double v) { return v; }
  static __device__ __forceinline__ T load_qd(const double* p) { return __ldcs(p); }
  // compensated / plain accumulation
  template <int D, int Q>
  static __device__ __forceinline__ void madB(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fma(t.B[q * D + d], x, acc);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madG(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fma(t.G[q * D + d], x, acc);
  }
  static __device__ __forceinline__ void mad(T& acc, T a, T x) { acc = fma(a, x, acc); }
  static __device__ __forceinline__ T mul(T a, T x) { return a * x; }
  static __device__ __forceinline__ T norm(T a) { return a; }
  // anchored accumulation degenerates to plain FMA in FP64
  static __device__ __forceinline__ float amax(float m, T) { return m; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigB(const Tab<D, Q>&, float, bool) { return 0.f; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigG(const Tab<D, Q>&, float, bool) { return 0.f; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigGB(const Tab<D, Q>&, float, float, bool) {
    return 0.f;
  }
  static __device__ __forceinline__ Acc begin(Sig) { return 0.0; }
  template <int D, int Q>
  static __device__ __forceinline__ void amadB(Acc& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fma(t.B[q * D + d], x, acc);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void amadG(Acc& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fma(t.G[q * D + d], x, acc);
  }
  static __device__ __forceinline__ T end(Acc a, Sig) { return a; }
  // a0 x0 + a1 x1 + a2 x2 (one row of the pointwise D)
  static __device__ __forceinline__ T dot3(T a0, T x0, T a1, T x1, T a2, T x2) {
    return fma(a2, x2, fma(a1, x1, a0 * x0));
  }
  // FP64 value of a result (no scaling in this policy)
  static __device__ __forceinline__ double widen(T v, int) { return v; }
  // accumulation of the fused x . (A x): FP64
  using DotAcc = double;
  static __device__ __forceinline__ DotAcc dot_zero() { return 0.0; }
  static __device__ __forceinline__ void dot_acc(DotAcc& a, double x, double v) { a = fma(x, v, a); }
  static __device__ __forceinline__ double dot_value(DotAcc a) { return a; }
};

// ANCHORED: anchored dot products (else every sum is compensated); LAZY: anchored results are
// left unnormalised.  The launcher picks the combination per order from the measured error.
template <bool ANCHORED, bool LAZY>
struct ArF32x2T {
  static constexpr bool kAnchored = ANCHORED;
  // Inputs are gathered as FP64 and converted with a power-of-two scale per thread block (its
  // largest input in [1, 2)); the quadrature data carry a power-of-two scale per element (the
  // element's largest entry in [1, 2)); results are widened with both scales undone.  So the
  // arithmetic is FP64-accurate for inputs anywhere in the FP64 range, not only the float range.
  static constexpr bool kScaled = true;
  // compensated orders: even-odd contractions with TwoSum splits and joins (fe_apply_eo.cuh);
  // anchored orders keep the direct contractions, whose anchors need a-priori bounds
  static constexpr bool kEvenOdd = !ANCHORED;
  static constexpr bool kPrefetchQd = true;  // bulk L2 prefetch of the block's quadrature data
  using QdT = double;  // 8-byte (hi, lo) float pairs
  using T = f2;
  using Acc = Anch;
  using Sig = float;
  template <int D, int Q>
  using Tab = typename std::conditional<ANCHORED, TabF32x2<D, Q>, TabEO<f2, D, Q>>::type;

  static __device__ __forceinline__ T zero() { return f2{0.0f, 0.0f}; }
  static __device__ __forceinline__ T from_vec(double v) { return f2_from_f64(v); }
  // v * 2^off as a pair (off from the block's largest input exponent)
  static __device__ __forceinline__ T from_raw(double v, int off) {
    return f2_from_f64_scaled(v, off);
  }
  // quadrature data is stored pre-split: the 8 bytes of each entry hold (h, l)
  static __device__ __forceinline__ T load_qd(const double* p) {
    const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
    return f2{v.x, v.y};
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madB(T& acc, const TabF32x2<D, Q>& t, int q, int d, T x) {
    f2_mad(acc, t.Bh[q * D + d], t.Bl[q * D + d], x);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madG(T& acc, const TabF32x2<D, Q>& t, int q, int d, T x) {
    f2_mad(acc, t.Gh[q * D + d], t.Gl[q * D + d], x);
  }
  static __device__ __forceinline__ void mad(T& acc, T a, T x) { f2_mad(acc, a.h, a.l, x); }
  static __device__ __forceinline__ T mul(T a, T x) {
    T r = zero();
    f2_mad(r, a.h, a.l, x);
    return r;
  }
  static __device__ __forceinline__ T norm(T a) { return f2_norm(a); }
  static __device__ __forceinline__ float amax(float m, T x) { return fmaxf(m, fabsf(x.h)); }
  // anchors: forward (row sums) or transposed (column sums) use of the table
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigB(const TabF32x2<D, Q>& t, float m, bool transposed) {
    return anchor_of(f_mul(transposed ? t.cB : t.rB, m));
  }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigG(const TabF32x2<D, Q>& t, float m, bool transposed) {
    return anchor_of(f_mul(transposed ? t.cG : t.rG, m));
  }
  // bound of G.a + B.b with max |a| = mg, max |b| = mb
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigGB(const TabF32x2<D, Q>& t, float mg, float mb,
                                             bool transposed) {
    return anchor_of(f_fma(transposed ? t.cG : t.rG, mg, f_mul(transposed ? t.cB : t.rB, mb)));
  }
  static __device__ __forceinline__ Acc begin(Sig s) {
    return ANCHORED ? anch_begin(s) : Anch{0.0f, 0.0f};
  }
  template <int D, int Q>
  static __device__ __forceinline__ void amadB(Acc& acc, const TabF32x2<D, Q>& t, int q, int d, T x) {
    amad(acc, t.Bh[q * D + d], t.Bl[q * D + d], x);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void amadG(Acc& acc, const TabF32x2<D, Q>& t, int q, int d, T x) {
    amad(acc, t.Gh[q * D + d], t.Gl[q * D + d], x);
  }
  static __device__ __forceinline__ void amad(Acc& acc, float ah, float al, T x) {
    if constexpr (ANCHORED) {
      anch_mad(acc, ah, al, x);
    } else {  // compensated, the Anch pair used as (h, l)
      f2 c{acc.A, acc.L};
      f2_mad(c, ah, al, x);
      acc = Anch{c.h, c.l};
    }
  }
  static __device__ __forceinline__ T end(Acc a, Sig s) {
    if constexpr (!ANCHORED) return f2_norm(f2{a.A, a.L});
    if constexpr (LAZY) return anch_end_lazy(a, s);
    return anch_end(a, s);
  }
  // a0 x0 + a1 x1 + a2 x2, anchored with the exact bound sum |a_i.h x_i.h| of this point
  static __device__ __forceinline__ T dot3(T a0, T x0, T a1, T x1, T a2, T x2) {
    if constexpr (!ANCHORED) {
      f2 c{0.0f, 0.0f};
      f2_mad(c, a0.h, a0.l, x0);
      f2_mad(c, a1.h, a1.l, x1);
      f2_mad(c, a2.h, a2.l, x2);
      return f2_norm(c);
    }
    const float b = f_fma(fabsf(a2.h), fabsf(x2.h),
                          f_fma(fabsf(a1.h), fabsf(x1.h), f_mul(fabsf(a0.h), fabsf(x0.h))));
    const float sg = anchor_of(b);
    Anch acc = anch_begin(sg);
    anch_mad(acc, a0.h, a0.l, x0);
    anch_mad(acc, a1.h, a1.l, x1);
    anch_mad(acc, a2.h, a2.l, x2);
    return end(acc, sg);
  }
  // FP64 value of a result times 2^off: both words widened exactly by integer manipulation
  // (no FP64-pipe conversion), then one exact FP64 add (h + l needs at most 49 bits)
  static __device__ __forceinline__ double widen(T v, int off) {
    return f64_from_f32_scaled(v.h, off) + f64_from_f32_scaled(v.l, off);
  }
  // accumulation of the fused x . (A x): FP64, on the FP64 inputs and the widened results
  using DotAcc = double;
  static __device__ __forceinline__ DotAcc dot_zero() { return 0.0; }
  static __device__ __forceinline__ void dot_acc(DotAcc& a, double x, double v) { a = fma(x, v, a); }
  static __device__ __forceinline__ double dot_value(DotAcc a) { return a; }
};

using ArF32x2 = ArF32x2T<true, false>;

// Plain FP32 (the inner solves of mixed-precision iterative refinement): FP32 quadrature data
// (half the bytes), FP32 FMAs; FP64 vectors in and out, converted by integer manipulation.
struct ArF32 {
  static constexpr bool kAnchored = false;
  static constexpr bool kScaled = false;
  static constexpr bool kEvenOdd = true;  // even-odd contractions (fe_apply_eo.cuh)
  static constexpr bool kPrefetchQd = true;  // bulk L2 prefetch of the block's quadrature data
  using QdT = float;
  using T = float;
  using Acc = float;
  using Sig = float;
  template <int D, int Q>
  using Tab = TabF32EO<D, Q>;

  static __device__ __forceinline__ T zero() { return 0.0f; }
  static __device__ __forceinline__ T from_vec(double v) { return f2_from_f64(v).h; }
  static __device__ __forceinline__ T from_vec(float v) { return v; }
  static __device__ __forceinline__ T load_qd(const float* p) { return __ldcs(p); }
  template <int D, int Q>
  static __device__ __forceinline__ void madB(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fmaf(t.B[q * D + d], x, acc);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madG(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fmaf(t.G[q * D + d], x, acc);
  }
  static __device__ __forceinline__ void mad(T& acc, T a, T x) { acc = fmaf(a, x, acc); }
  static __device__ __forceinline__ T mul(T a, T x) { return a * x; }
  static __device__ __forceinline__ T norm(T a) { return a; }
  static __device__ __forceinline__ float amax(float m, T) { return m; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigB(const Tab<D, Q>&, float, bool) { return 0.f; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigG(const Tab<D, Q>&, float, bool) { return 0.f; }
  template <int D, int Q>
  static __device__ __forceinline__ Sig sigGB(const Tab<D, Q>&, float, float, bool) {
    return 0.f;
  }
  static __device__ __forceinline__ Acc begin(Sig) { return 0.0f; }
  template <int D, int Q>
  static __device__ __forceinline__ void amadB(Acc& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fmaf(t.B[q * D + d], x, acc);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void amadG(Acc& acc, const Tab<D, Q>& t, int q, int d, T x) {
    acc = fmaf(t.G[q * D + d], x, acc);
  }
  static __device__ __forceinline__ T end(Acc a, Sig) { return a; }
  static __device__ __forceinline__ T dot3(T a0, T x0, T a1, T x1, T a2, T x2) {
    return fmaf(a2, x2, fmaf(a1, x1, a0 * x0));
  }
  // FP64 value of a result times 2^off (the FP32 data's shift undone), exact
  static __device__ __forceinline__ double widen(T v, int off) { return f64_from_f32_scaled(v, off); }
  static __device__ __forceinline__ void scatter(float* y, T v) { atomicAdd(y, v); }
  // accumulation of the fused x . (A x): FP32 (the inner solves need no more)
  using DotAcc = float;
  static __device__ __forceinline__ DotAcc dot_zero() { return 0.0f; }
  static __device__ __forceinline__ void dot_acc(DotAcc& a, double x, double v) {
    a = fmaf(f2_from_f64(x).h, f2_from_f64(v).h, a);
  }
  static __device__ __forceinline__ void dot_acc(DotAcc& a, float x, T v) { a = fmaf(x, v, a); }
  static __device__ __forceinline__ double dot_value(DotAcc a) { return f64_from_f32(a); }
};

}  // namespace fe
