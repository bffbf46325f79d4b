// Error-free float32 transformations for float64-accurate residual sums
// (Knuth's TwoSum; Dekker's TwoProd through fma).
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Knuth's TwoSum: s + e == a + b exactly (no branch, any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// sum_a a_ba (kap x_b - x_a) for one component with float32 error-free
// transformations: the difference of the hi parts exactly (TwoSum), its product
// with a_hi exactly (Dekker's TwoProd via fma), the running sum exactly
// (TwoSum), and the terms of order 2^-24 (a_hi * diff error, a_lo * diff,
// a_hi * lo-part difference) in plain float32.  Error ~2^-47 of sum |terms|.
struct DFAcc {
  float sh = 0.f, sl = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float ahi, float alo, float kxbh, float xah, float kxbl, float xal) {
    float d, de;
    two_sum(kxbh, -xah, d, de);
    const float p = ahi * d;
    const float pe = fmaf(ahi, d, -p);
    float t, te;
    two_sum(sh, p, t, te);
    sh = t;
    sl += te;
    c += pe + fmaf(ahi, de, fmaf(alo, d, ahi * (kxbl - xal)));
  }
  __device__ __forceinline__ double value() const { return (double)sh + ((double)sl + (double)c); }
};

}  // namespace sph

namespace sph {

// Double-float numbers x = hi + lo (|lo| <= ulp(hi) / 2), about 48 significant
// bits from float32 operations only: the arithmetic of the operator set-up,
// where float64 would run at a small fraction of the float32 rate.  Operations
// follow Dekker (1971) and Knuth's TwoSum; each has a relative error of a few
// 2^-47 (the sums without cancellation between their high parts, as used here).
struct dfl {
  float hi, lo;
};

// s + e == a + b for |a| >= |b| (Dekker's Fast2Sum)
__device__ __forceinline__ dfl df_quick(float a, float b) {
  const float s = a + b;
  return dfl{s, b - (s - a)};
}
__device__ __forceinline__ dfl df_exact_sum(float a, float b) {
  float s, e;
  two_sum(a, b, s, e);
  return dfl{s, e};
}
__device__ __forceinline__ dfl df_exact_prod(float a, float b) {
  const float p = a * b;
  return dfl{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_quick(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return df_quick(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
// sqrt(a) for a > 0: float32 root, then one Newton correction from the exact
// residual a - y^2
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  const float y = sqrtf(a.hi);
  if (y == 0.f) return dfl{0.f, 0.f};
  const dfl y2 = df_exact_prod(y, y);
  const float r = ((a.hi - y2.hi) - y2.lo) + a.lo;
  return df_quick(y, r * (0.5f / y));
}
// 1 / a for a != 0: float32 reciprocal, then one Newton correction (the residual
// 1 - a_hi y of a correctly rounded reciprocal is exact in float32)
__device__ __forceinline__ dfl df_rcp(dfl a) {
  const float y = __frcp_rn(a.hi);
  const float r = fmaf(-a.lo, y, fmaf(-a.hi, y, 1.f));
  return df_quick(y, y * r);
}
__device__ __forceinline__ dfl df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return dfl{hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace sph
