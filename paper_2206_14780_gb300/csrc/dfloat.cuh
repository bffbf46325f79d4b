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
