// Host harness for the double-float arithmetic of csrc/dfloat.cuh (the
// FP32-mixed CG scalars).  Each operation is compared with long double on
// seeded random operands over twelve decades; the largest errors are
// printed as "name value" lines for tests/test_dfloat.py to judge.
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_1711_08013_gb300/csrc/dfloat.cuh"

using osqpgb::ff;

static long double val(ff x) { return (long double)x.h + (long double)x.l; }

int main() {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0), E(-6.0, 6.0);
  auto draw = [&]() { return U(g) * std::pow(10.0, E(g)); };
  long double two_sum_err = 0, fast_err = 0, mul_rel = 0, div_rel = 0, sub_abs = 0, den_rel = 0;
  long double den_rel_fp32 = 0;
  for (int i = 0; i < 200000; ++i) {
    const double a = draw(), b = draw();
    const float fa = (float)a, fb = (float)b;
    // TwoSum is exact for any pair; FastTwoSum when |a| ≥ |b|
    const ff s = osqpgb::ff_two_sum(fa, fb);
    two_sum_err = std::fmax(two_sum_err, fabsl(val(s) - ((long double)fa + fb)));
    const float big = std::fabs(fa) >= std::fabs(fb) ? fa : fb, small = big == fa ? fb : fa;
    const ff fs = osqpgb::ff_fast_two_sum(big, small);
    fast_err = std::fmax(fast_err, fabsl(val(fs) - ((long double)big + small)));
    const ff x = osqpgb::ff_of(a), y = osqpgb::ff_of(b);
    const long double X = val(x), Y = val(y);
    mul_rel = std::fmax(mul_rel, fabsl((val(osqpgb::ff_mul(x, y)) - X * Y) / (X * Y)));
    div_rel = std::fmax(div_rel, fabsl((val(osqpgb::ff_div(x, y)) - X / Y) / (X / Y)));
    // subtraction: error relative to the larger operand (cancellation included)
    const ff z = osqpgb::ff_of(a * (1.0 + 1e-6 * U(g)));
    const long double Z = val(z);
    sub_abs = std::fmax(sub_abs, fabsl(val(osqpgb::ff_sub(x, z)) - (X - Z)) / fmaxl(fabsl(X), fabsl(Z)));
    // the Chronopoulos–Gear denominator δ − β·c with δ within 1e-4 of β·c
    const double beta = 0.5 + 0.5 * std::fabs(U(g)), c = std::fabs(draw()) + 1e-3;
    const double delta = beta * c * (1.0 + 1e-4 * (1.5 + U(g)));
    const ff fd = osqpgb::ff_of(delta), fbeta = osqpgb::ff_of(beta), fc = osqpgb::ff_of(c);
    const long double exact = val(fd) - val(fbeta) * val(fc);
    const ff den = osqpgb::ff_sub(fd, osqpgb::ff_mul(fbeta, fc));
    den_rel = std::fmax(den_rel, fabsl((val(den) - exact) / exact));
    // the same in plain FP32, for contrast
    const float d32 = (float)delta - (float)beta * (float)c;
    den_rel_fp32 = std::fmax(den_rel_fp32, fabsl(((long double)d32 - exact) / exact));
  }
  std::printf("two_sum_err %.6Le\n", two_sum_err);
  std::printf("fast_two_sum_err %.6Le\n", fast_err);
  std::printf("mul_rel %.6Le\n", mul_rel);
  std::printf("div_rel %.6Le\n", div_rel);
  std::printf("sub_rel_to_operand %.6Le\n", sub_abs);
  std::printf("cg_denominator_rel %.6Le\n", den_rel);
  std::printf("cg_denominator_rel_fp32 %.6Le\n", den_rel_fp32);
  return 0;
}
