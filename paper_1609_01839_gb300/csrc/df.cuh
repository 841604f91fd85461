// Double-float arithmetic: a value is hi + lo with two FP32 numbers
// (|lo| <= ulp(hi)/2), carried with error-free transformations (Knuth's
// two-sum, FMA-based two-product; Dekker / Shewchuk).  About 48 significant
// bits using only FP32 instructions, which matters on a part whose FP64
// pipeline is slow.
#pragma once
#include "common.cuh"

namespace gfd {

struct df {
  float hi, lo;
};

GFD_D df df_make(float a) { return df{a, 0.0f}; }

GFD_D df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df{s, e};
}

GFD_D df quick_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = a + b;
  return df{s, b - (s - a)};
}

GFD_D df two_prod(float a, float b) {
  const float p = a * b;
  return df{p, fmaf(a, b, -p)};
}

GFD_D df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

GFD_D df df_neg(df a) { return df{-a.hi, -a.lo}; }
GFD_D df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

GFD_D df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}

GFD_D df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// 1/a: FP32 reciprocal refined by one double-float Newton step.
GFD_D df df_rcp(df a) {
  const float r = 1.0f / a.hi;
  // e = 1 - a*r (in double-float), result r + r*e
  const df ar = df_mul_f(a, r);
  const df e = df_sub(df_make(1.0f), ar);
  return df_add(df_make(r), df_mul_f(e, r));
}

GFD_D double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
GFD_D df df_from_double(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}

}  // namespace gfd
