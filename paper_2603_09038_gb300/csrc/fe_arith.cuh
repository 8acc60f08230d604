// Arithmetic policies of the fused apply kernel.
//
//  ArF64    IEEE FP64 on the FP64 pipe: every multiply-add is one DFMA.
//  ArF32x2  FP64-accurate float-float arithmetic on the FP32 pipe (GB300's FP64 pipe delivers
//           ~1.2 TFLOP/s against ~75 TFLOP/s FP32).  A value is the unevaluated sum h + l of two
//           floats.  Products use Dekker's error-free product (via FMA: p = fl(a*b),
//           e = fma(a, b, -p) is exact); sums use Knuth's TwoSum (s = fl(a+b),
//           err = (a - (s - bb)) + (b - bb), bb = s - a, exact).  Accumulators carry their
//           rounding errors in the low word and are renormalised once per output.  The
//           relative error of a length-n dot product is O(n * 2^-47) of sum |a_i b_i|, i.e. FP64
//           class.  Intrinsics with explicit rounding (__fmul_rn, __fadd_rn, ...) keep the
//           compiler from contracting the error-free steps into FMAs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fe {

// 1D basis tables passed by value in the kernel parameter space (constant bank), so that
// fully unrolled contractions read them as immediate constant operands.
template <int D, int Q>
struct TabF64 {
  double B[Q * D];
  double G[Q * D];
};

template <int D, int Q>
struct TabF32x2 {
  float Bh[Q * D], Bl[Q * D];
  float Gh[Q * D], Gl[Q * D];
};

struct f2 {
  float h, l;
};

// ---------------------------------------------------------------------------------------------
struct ArF64 {
  using T = double;
  template <int D, int Q>
  using Tab = TabF64<D, Q>;

  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T from_f64(double v) { return v; }
  static __device__ __forceinline__ T load_qd(const double* p) { return __ldcs(p); }
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
  static __device__ __forceinline__ void scatter(double* y, T v) { atomicAdd(y, v); }
};

// ---------------------------------------------------------------------------------------------
// float-float helpers

// acc += a * x with a = (ah, al) and x = (x.h, x.l); acc stays unnormalised (h, l).
static __device__ __forceinline__ void f2_mad(f2& acc, float ah, float al, f2 x) {
  const float p = __fmul_rn(ah, x.h);
  float e = __fmaf_rn(ah, x.h, -p);          // exact low part of ah * x.h
  e = __fmaf_rn(ah, x.l, e);
  e = __fmaf_rn(al, x.h, e);
  const float s = __fadd_rn(acc.h, p);       // TwoSum(acc.h, p)
  const float bb = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, err));
}

// Normalised (h, l) with h = fl(h + l) (TwoSum, valid for any ordering of magnitudes).
static __device__ __forceinline__ f2 f2_norm(f2 a) {
  const float s = __fadd_rn(a.h, a.l);
  const float bb = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(a.l, bb));
  return f2{s, err};
}

// Splits an FP64 value into floats without touching the FP64 pipe: h = v truncated to 24
// significant bits (exact), l = the next 23 bits of the remainder (exact), by integer
// manipulation of the IEEE encodings.  Valid for 2^-80 < |v| < 2^127; smaller magnitudes fall
// back to a plain conversion (their relative accuracy is irrelevant for O(1) data), larger
// ones overflow to +-inf.
static __device__ __forceinline__ f2 f2_from_f64(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int sign = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7FFu);  // biased double exponent
  const int fexp = ex - 896;                  // biased float exponent (1023 - 127)
  if (fexp <= 0 || fexp >= 255 || ex < 943) return f2{__double2float_rn(v), 0.0f};
  const unsigned int mant = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const float h = __uint_as_float(sign | ((unsigned int)fexp << 23) | mant);
  // remaining 29 significand bits: keep the top 23, an exact integer r < 2^23, scaled by
  // 2^(ex - 1075 + 6) (float exponent field ex - 942 >= 1 for ex >= 943)
  const unsigned int rem = (lw & 0x1FFFFFFFu) >> 6;
  const float r = __fsub_rn(__uint_as_float(0x4B000000u | rem), 8388608.0f);
  const float l = __fmul_rn(r, __uint_as_float((unsigned int)(ex - 942) << 23));
  return f2{h, __uint_as_float(__float_as_uint(l) | sign)};
}

// ---------------------------------------------------------------------------------------------
struct ArF32x2 {
  using T = f2;
  template <int D, int Q>
  using Tab = TabF32x2<D, Q>;

  static __device__ __forceinline__ T zero() { return f2{0.0f, 0.0f}; }
  static __device__ __forceinline__ T from_f64(double v) { return f2_from_f64(v); }
  // quadrature data is stored pre-split: the 8 bytes of each entry hold (h, l)
  static __device__ __forceinline__ T load_qd(const double* p) {
    const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
    return f2{v.x, v.y};
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madB(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    f2_mad(acc, t.Bh[q * D + d], t.Bl[q * D + d], x);
  }
  template <int D, int Q>
  static __device__ __forceinline__ void madG(T& acc, const Tab<D, Q>& t, int q, int d, T x) {
    f2_mad(acc, t.Gh[q * D + d], t.Gl[q * D + d], x);
  }
  static __device__ __forceinline__ void mad(T& acc, T a, T x) { f2_mad(acc, a.h, a.l, x); }
  static __device__ __forceinline__ T mul(T a, T x) {
    T r = zero();
    f2_mad(r, a.h, a.l, x);
    return r;
  }
  static __device__ __forceinline__ T norm(T a) { return f2_norm(a); }
  static __device__ __forceinline__ void scatter(double* y, T v) {
    atomicAdd(y, (double)v.h + (double)v.l);
  }
};

}  // namespace fe
