// Double-float arithmetic: a value held as the unevaluated sum h + l of two
// floats with |l| ≤ ulp(h)/2, about 48 significant bits from FP32
// instructions alone.  The FP32-mixed PCG runs its scalar recurrence in it
// (every thread, no FP64 instruction).
//
// The error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum
// and the product error taken exactly by one fused multiply-add; ff_div is
// the FP32 quotient corrected once by the remainder (Dekker's division
// step).  Every operation is an explicitly rounded FP32 operation: on the
// device the _rn intrinsics, on the host (tests) single-precision operations
// whose results pass through volatile stores, so that no compiler contracts
// or reorders them.  The header has no CUDA dependency outside those guards.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define OSQPGB_DF __host__ __device__ __forceinline__
#else
#define OSQPGB_DF inline
#endif

namespace osqpgb {

struct ff {
  float h, l;
};

OSQPGB_DF float df_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
OSQPGB_DF float df_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  volatile float r = a - b;
  return r;
#endif
}
OSQPGB_DF float df_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
OSQPGB_DF float df_div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  volatile float r = a / b;
  return r;
#endif
}
OSQPGB_DF float df_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  volatile float r = fmaf(a, b, c);
  return r;
#endif
}

// a + b exactly as (sum, error), for |a| ≥ |b|
OSQPGB_DF ff ff_fast_two_sum(float a, float b) {
  const float s = df_add(a, b);
  return {s, df_sub(b, df_sub(s, a))};
}
// a + b exactly as (sum, error), any magnitudes
OSQPGB_DF ff ff_two_sum(float a, float b) {
  const float s = df_add(a, b);
  const float bb = df_sub(s, a);
  return {s, df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb))};
}
// x − y; the closing TwoSum keeps the low part when the high parts cancel
OSQPGB_DF ff ff_sub(ff x, ff y) {
  const ff s = ff_two_sum(x.h, -y.h);
  return ff_two_sum(s.h, df_add(s.l, df_sub(x.l, y.l)));
}
OSQPGB_DF ff ff_mul(ff x, ff y) {
  const float p = df_mul(x.h, y.h);
  float e = df_fma(x.h, y.h, -p);
  e = df_fma(x.h, y.l, e);
  e = df_fma(x.l, y.h, e);
  return ff_fast_two_sum(p, e);
}
// x / y: the FP32 quotient, then one correction from the remainder x − q·y
OSQPGB_DF ff ff_div(ff x, ff y) {
  const float q = df_div(x.h, y.h);
  const ff r = ff_sub(x, ff_mul(y, ff{q, 0.0f}));
  return ff_fast_two_sum(q, df_div(r.h, y.h));
}
// the pair nearest to a double
OSQPGB_DF ff ff_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

}  // namespace osqpgb
