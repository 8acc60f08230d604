"""CPU unit test of the float-float primitives of the apply kernels (csrc/fe_f2.h).

The header is compiled for the host with g++ (-ffp-contract=off, IEEE single precision with
round-to-nearest: the same steps the device performs with explicit-rounding intrinsics) and
checked against long double references: exact splitting of doubles, exact TwoSum, and the
error bounds of the anchored and compensated dot products, including heavy cancellation.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_09038_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <random>
#include <cmath>
#include "fe_f2.h"
using namespace fe;
typedef long double LD;
static LD val(f2 a) { return (LD)a.h + (LD)a.l; }
int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  // 1. splitting of doubles: h + l reproduces v to 2^-46 relative, h is v truncated
  double worst_split = 0;
  for (int i = 0; i < 200000; ++i) {
    double v = U(rng) * std::ldexp(1.0, (int)(rng() % 120) - 60);
    f2 s = f2_from_f64(v);
    double rel = std::fabs((double)(((LD)s.h + (LD)s.l) - (LD)v)) / std::fabs(v);
    if (rel > worst_split) worst_split = rel;
    if (std::fabs((double)s.h) > std::fabs(v)) { std::printf("FAIL trunc\n"); return 1; }
  }
  // 2. TwoSum is exact
  for (int i = 0; i < 200000; ++i) {
    float a = (float)(U(rng) * std::ldexp(1.0, (int)(rng() % 40) - 20));
    float b = (float)(U(rng) * std::ldexp(1.0, (int)(rng() % 40) - 20));
    f2 s = two_sum(a, b);
    if ((LD)s.h + (LD)s.l != (LD)a + (LD)b) { std::printf("FAIL twosum\n"); return 1; }
  }
  // 3. dot products of length n <= 10 with float-float tables and inputs, incl. cancellation
  double worst_anch = 0, worst_comp = 0;
  for (int it = 0; it < 100000; ++it) {
    int n = 1 + (int)(rng() % 10);
    f2 a[10], x[10];
    LD exact = 0, absum = 0, rowsum = 0;
    float m = 0;
    for (int i = 0; i < n; ++i) {
      double av = U(rng) * 3.0, xv = U(rng) * std::ldexp(1.0, (int)(rng() % 8) - 4);
      a[i] = f2_from_f64(av);
      x[i] = f2_from_f64(xv);
      if (it % 3 == 0 && i == n - 1) {   // force near-cancellation of the exact sum
        LD partial = 0;
        for (int k = 0; k < i; ++k) partial += val(a[k]) * val(x[k]);
        x[i] = f2_from_f64((double)(-partial / val(a[i])));
      }
      exact += val(a[i]) * val(x[i]);
      absum += std::fabs((double)(val(a[i]) * val(x[i])));
      rowsum += std::fabs(a[i].h);
      m = std::fmax(m, std::fabs(x[i].h));
    }
    float sigma = anchor_of((float)(rowsum * (1 + 1e-6)) * m);
    Anch acc = anch_begin(sigma);
    for (int i = 0; i < n; ++i) anch_mad(acc, a[i].h, a[i].l, x[i]);
    f2 r = anch_end(acc, sigma);
    double ea = (double)std::fabs(val(r) - exact) / (double)(sigma > 0 ? sigma : 1);
    if (ea > worst_anch) worst_anch = ea;
    f2 c{0.f, 0.f};
    for (int i = 0; i < n; ++i) f2_mad(c, a[i].h, a[i].l, x[i]);
    c = f2_norm(c);
    double ec = absum > 0 ? (double)(std::fabs(val(c) - exact) / absum) : 0.0;
    if (ec > worst_comp) worst_comp = ec;
  }
  // 4. scaled split of doubles anywhere in the FP64 range: v 2^off with off = 1023 - e_max
  //    (e_max the biased exponent of a block maximum at or above |v|) reproduces v 2^off to
  //    2^-46 relative down to 2^-80 below the block maximum, and to 2^-104 of the block scale
  //    below that (the high word alone); widening back by -off is exact
  double worst_scaled = 0;
  int bad_widen = 0;
  for (int i = 0; i < 200000; ++i) {
    // block scale 2^eb, kept 2^120 above the FP64 subnormals (flushed to zero by design)
    const int eb = (int)(rng() % 1800) - 900;
    const double vmax = std::ldexp(1.0 + 0.5 * std::fabs(U(rng)), eb);
    const double v = U(rng) * vmax * std::ldexp(1.0, -(int)(rng() % 70));
    const int off = 1023 - f64_exponent(vmax);
    f2 s = f2_from_f64_scaled(v, off);
    const LD target = std::ldexp((LD)v, off);
    if (v != 0.0) {  // relative to the value, or to 2^-58 of the block scale below that
      const LD den = std::fmax(std::fabs(target), std::ldexp((LD)1, -58));
      double rel = (double)(std::fabs(((LD)s.h + (LD)s.l) - target) / den);
      if (rel > worst_scaled) worst_scaled = rel;
    }
    const double back = f64_from_f32_scaled(s.h, -off) + f64_from_f32_scaled(s.l, -off);
    if ((LD)back != std::ldexp((LD)s.h + (LD)s.l, -off)) ++bad_widen;
  }
  // 5. special values: zero and FP64 subnormals give zero; inf and NaN survive; values far
  //    below the block maximum flush to zero
  int bad_special = 0;
  if (f2_from_f64_scaled(0.0, 5).h != 0.0f) ++bad_special;
  if (f2_from_f64_scaled(4.9e-324, 1000).h != 0.0f) ++bad_special;
  if (!std::isinf(f2_from_f64_scaled(INFINITY, -1024).h)) ++bad_special;
  if (!std::isnan(f2_from_f64_scaled(NAN, -1024).h)) ++bad_special;
  if (f2_from_f64_scaled(std::ldexp(1.0, -200), 0).h != 0.0f) ++bad_special;
  if (!std::isinf(f64_from_f32_scaled(1.0f, 2000))) ++bad_special;
  if (f64_from_f32_scaled(1.0f, -2000) != 0.0) ++bad_special;
  std::printf("%.6e %.6e %.6e %.6e %d %d\n", worst_split, worst_anch, worst_comp, worst_scaled,
              bad_widen, bad_special);
  return 0;
}
'''


@pytest.fixture(scope="module")
def results():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    open(src, "w").write(HARNESS)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, src, "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    shutil.rmtree(d)
    return [float(v) for v in out]


def test_split_reproduces_doubles_to_2_pow_minus_46(results):
    assert results[0] <= 2.0 ** -46


def test_anchored_dot_error_is_below_n_2_pow_minus_46_of_the_anchor(results):
    # every term adds at most three roundings of the low word (|L| < n 2^-23 sigma) and one of
    # its residual r: about 2^-46 sigma per term; n <= 10 here
    assert results[1] <= 10 * 2.0 ** -46


def test_compensated_dot_error_is_below_n_2_pow_minus_46_of_the_absolute_sum(results):
    # roundings of the low word relative to the largest partial sum, n <= 10 terms
    assert results[2] <= 10 * 2.0 ** -46


def test_scaled_split_covers_the_fp64_range(results):
    # block scales from 2^-900 to 2^900, values down to 2^-70 below the block maximum
    assert results[3] <= 2.0 ** -46


def test_scaled_widening_is_exact_and_special_values_hold(results):
    assert results[4] == 0 and results[5] == 0
