// Float-float ("double-FP32") primitives of the apply kernels: error-free transformations
// written once for device and host.  On the device they use the explicit-rounding intrinsics
// (which the compiler never contracts into FMAs); on the host plain float arithmetic, which the
// CPU unit test compiles with -ffp-contract=off, so both sides perform the same IEEE steps.
// See fe_arith.cuh for the accumulation schemes built from them.
#pragma once

#include <stdint.h>

#include <cmath>
#include <cstring>

#if defined(__CUDACC__)
#define FE_HD __host__ __device__ __forceinline__
#else
#define FE_HD inline
#endif

namespace fe {

// ---------------------------------------------------------------------------- primitives
FE_HD float f_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
FE_HD float f_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
FE_HD float f_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
FE_HD float f_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
FE_HD uint32_t f_bits(float a) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(a);
#else
  uint32_t u;
  std::memcpy(&u, &a, 4);
  return u;
#endif
}
FE_HD float f_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float a;
  std::memcpy(&a, &u, 4);
  return a;
#endif
}

struct f2 {
  float h, l;
};

// a + b as a normalised pair (Knuth's TwoSum, any ordering of magnitudes).
FE_HD f2 two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float bb = f_sub(s, a);
  const float err = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
  return f2{s, err};
}

// acc += a * x (compensated: exact product, TwoSum on the high words); acc unnormalised.
FE_HD void f2_mad(f2& acc, float ah, float al, f2 x) {
  const float p = f_mul(ah, x.h);
  float e = f_fma(ah, x.h, -p);
  e = f_fma(ah, x.l, e);
  e = f_fma(al, x.h, e);
  const f2 s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = f_add(acc.l, f_add(e, s.l));
}

FE_HD f2 f2_norm(f2 a) { return two_sum(a.h, a.l); }

// Anchor of a dot product whose terms satisfy sum |a_i x_i| <= b: the smallest power of two
// sigma >= 2 (1 + 2^-9) b (0 for b = 0).  Every partial sum A = sigma + sum z_i then stays in
// [sigma/2, 3 sigma/2], where floats are multiples of 2^-24 sigma, and each step t - A is below
// 2^23 of those units: exact.
FE_HD float anchor_of(float b) {
  const uint32_t u = f_bits(f_mul(2.00390625f, b));
  return f_from_bits((u + 0x007FFFFFu) & 0x7F800000u);
}

struct Anch {
  float A, L;  // value = (A - sigma) + L
};

FE_HD Anch anch_begin(float sigma) { return Anch{sigma, 0.0f}; }

// acc += a * x, anchored (requires the a-priori bound behind sigma).
FE_HD void anch_mad(Anch& acc, float ah, float al, f2 x) {
  const float t = f_fma(ah, x.h, acc.A);
  const float z = f_sub(t, acc.A);
  const float r = f_fma(ah, x.h, -z);
  acc.L = f_add(acc.L, r);
  acc.L = f_fma(ah, x.l, acc.L);
  acc.L = f_fma(al, x.h, acc.L);
  acc.A = t;
}

// Result of an anchored sum: (A - sigma) exactly, plus the low word, normalised by TwoSum.
FE_HD f2 anch_end(Anch acc, float sigma) { return two_sum(f_sub(acc.A, sigma), acc.L); }

// The same without normalisation: the next stage uses the high word for its exact products
// and the low word only in first-order correction terms, so an unnormalised pair costs
// accuracy only through slightly larger bounds (used where the error budget allows).
FE_HD f2 anch_end_lazy(Anch acc, float sigma) { return f2{f_sub(acc.A, sigma), acc.L}; }

// Splits an FP64 value into floats without the FP64 pipe: h = v truncated to 24 significant
// bits (exact), l = the next 23 bits of the remainder (exact), by integer manipulation of the
// IEEE encodings.  Valid for 2^-80 < |v| < 2^127; other magnitudes fall back to a plain
// conversion (relative accuracy of such tiny values is irrelevant for O(1) data).
FE_HD f2 f2_from_f64(double v) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7FFu);  // biased double exponent
  const int fexp = ex - 896;                  // biased float exponent (1023 - 127)
  if (fexp <= 0 || fexp >= 255 || ex < 943) return f2{(float)v, 0.0f};
  const uint32_t mant = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const float h = f_from_bits(sign | ((uint32_t)fexp << 23) | mant);
  // remaining 29 significand bits: keep the top 23, an exact integer r < 2^23, scaled by
  // 2^(ex - 1075 + 6) (float exponent field ex - 942 >= 1 for ex >= 943)
  const uint32_t rem = (lw & 0x1FFFFFFFu) >> 6;
  const float r = f_sub(f_from_bits(0x4B000000u | rem), 8388608.0f);
  const float l = f_mul(r, f_from_bits((uint32_t)(ex - 942) << 23));
  return f2{h, f_from_bits(f_bits(l) | sign)};
}

// Biased FP64 exponent field of v (0 for zero and subnormals, 2047 for inf / NaN).
FE_HD int f64_exponent(double v) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return (int)((b >> 52) & 0x7FFu);
}

// Split of v * 2^off into floats, by integer manipulation of the encodings like f2_from_f64.
// The apply kernels call it with off = 1023 - (the largest biased exponent of a block's
// inputs), so that the block's largest input lands in [1, 2) and the whole FP64 exponent range
// maps into the float range.  Scaled values below 2^-126 (relative 2^-126 to the block's
// largest) become zero, those below 2^-80 keep a high word only; FP64 zeros and subnormals
// become zero; inf / NaN stay inf / NaN.
FE_HD f2 f2_from_f64_scaled(double v, int off) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7FFu);
  if (ex == 0x7FF) {  // inf or NaN
    const uint32_t nan = ((hw & 0xFFFFFu) | lw) ? 0x00400000u : 0u;
    return f2{f_from_bits(sign | 0x7F800000u | nan), 0.0f};
  }
  const int es = ex + off;     // biased FP64 exponent of the scaled value
  const int fexp = es - 896;   // its biased float exponent
  if (ex == 0 || fexp <= 0) return f2{f_from_bits(sign), 0.0f};
  if (fexp >= 255) return f2{f_from_bits(sign | 0x7F800000u), 0.0f};
  const uint32_t mant = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const float h = f_from_bits(sign | ((uint32_t)fexp << 23) | mant);
  if (es < 943) return f2{h, 0.0f};
  const uint32_t rem = (lw & 0x1FFFFFFFu) >> 6;
  const float r = f_sub(f_from_bits(0x4B000000u | rem), 8388608.0f);
  const float l = f_mul(r, f_from_bits((uint32_t)(es - 942) << 23));
  return f2{h, f_from_bits(f_bits(l) | sign)};
}

// Exact widening of a float times 2^off to a double by integer manipulation (no FP64-pipe
// conversion): zero and float subnormals map to a signed zero, inf / NaN to inf / NaN, results
// below the FP64 normal range to zero and above it to inf.
FE_HD double f64_from_f32_scaled(float a, int off) {
  const uint32_t u = f_bits(a);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const int e = (int)((u >> 23) & 0xFFu);
  uint64_t bits;
  if (e == 0) {
    bits = sign;
  } else if (e == 0xFF) {
    bits = sign | ((uint64_t)0x7FF << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  } else {
    const int ed = e + 896 + off;
    if (ed <= 0)
      bits = sign;
    else if (ed >= 0x7FF)
      bits = sign | ((uint64_t)0x7FF << 52);
    else
      bits = sign | ((uint64_t)ed << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  }
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}

// Exact widening of a float to a double by integer manipulation (no FP64-pipe conversion):
// normal floats only; zero and subnormals map to a signed zero, inf/NaN to inf/NaN.
FE_HD double f64_from_f32(float a) {
  const uint32_t u = f_bits(a);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu;
  uint64_t bits;
  if (e == 0)
    bits = sign;
  else if (e == 0xFFu)
    bits = sign | ((uint64_t)0x7FF << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  else
    bits = sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}

}  // namespace fe
