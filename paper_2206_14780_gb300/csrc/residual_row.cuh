// One row of the float64-accurate residual's operator sum, shared by the
// single-scene and batched residual kernels: sum over the row's stored entries
// of a_ba (kap x_b - x_a) per component, with a = hi + lo, in double-float
// arithmetic (DFAcc).  Two forms of x:
//   X2 = true:  x = hi + lo interleaved, x2[2 t] = hi, x2[2 t + 1] = lo, so the
//               two gathers of an entry read one 32-byte sector;
//   X2 = false: a float32 vector d (one gather per entry), for the residual
//               update r64 -= A d after a refinement pass.
// In both, a_ba (kap x_b - x_a) is formed exactly (TwoSum) before the products.
//
// Entries are taken in groups of kResU, software-pipelined as the solver's
// apply is: the next group's coefficient loads are issued before the current
// group's error-free sums, so the coefficient stream stays in flight across
// the long dependent arithmetic.  The loop runs to the slice width (uniform over
// the warp); a slot past the row's count reads the row itself with a zero
// coefficient, which adds exactly nothing.
#pragma once

#include "apply.cuh"
#include "dfloat.cuh"

namespace sph {

constexpr int kResU = 4;

template <bool X2>
__device__ __forceinline__ void residual_row(const OpView& op, const float* __restrict__ op_lo,
                                             const float4* __restrict__ x, int64_t sl, int lane, float kap,
                                             float4& xb, DFAcc& a0, DFAcc& a1, DFAcc& a2) {
  const int64_t s = sl * kSlice + lane;
  const float4 bh = X2 ? x[2 * s] : x[s];
  const float4 bl = X2 ? x[2 * s + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  xb = bh;
  const int c = op.cnt[s];
  const int64_t o0 = op.off[sl];
  const int w = (int)((op.off[sl + 1] - o0) / kSlice);
  const int2* __restrict__ p = op.ih + o0 + lane;
  const float* __restrict__ q = op_lo + o0 + lane;
  const float kbh0 = kap * bh.x, kbh1 = kap * bh.y, kbh2 = kap * bh.z;
  const float kbl0 = kap * bl.x, kbl1 = kap * bl.y, kbl2 = kap * bl.z;
  int2 ih[kResU];
  float lo[kResU];
#pragma unroll
  for (int u = 0; u < kResU; ++u) {
    const bool ok = u < c;
    ih[u] = ok ? __ldcs(p + (int64_t)u * kSlice) : make_int2((int)s, 0);
    lo[u] = ok ? __ldcs(q + (int64_t)u * kSlice) : 0.f;
  }
  for (int j0 = 0; j0 < w; j0 += kResU) {
    float4 ah[kResU], al[kResU];
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      if (X2) {
        ah[u] = __ldg(x + 2 * (int64_t)ih[u].x);
        al[u] = __ldg(x + 2 * (int64_t)ih[u].x + 1);
      } else {
        ah[u] = __ldg(x + ih[u].x);
      }
    }
    int2 ihn[kResU];
    float lon[kResU];
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      const int j = j0 + kResU + u;
      const bool ok = j < c;
      ihn[u] = ok ? __ldcs(p + (int64_t)j * kSlice) : make_int2((int)s, 0);
      lon[u] = ok ? __ldcs(q + (int64_t)j * kSlice) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      const float ahi = __int_as_float(ih[u].y);
      a0.add(ahi, lo[u], kbh0, ah[u].x, kbl0, X2 ? al[u].x : 0.f);
      a1.add(ahi, lo[u], kbh1, ah[u].y, kbl1, X2 ? al[u].y : 0.f);
      a2.add(ahi, lo[u], kbh2, ah[u].z, kbl2, X2 ? al[u].z : 0.f);
    }
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      ih[u] = ihn[u];
      lo[u] = lon[u];
    }
  }
}

__device__ __forceinline__ void residual_row_df(const OpView& op, const float* __restrict__ op_lo,
                                                const float4* __restrict__ x2, int64_t sl, int lane, float kap,
                                                DFAcc& a0, DFAcc& a1, DFAcc& a2) {
  float4 xb;
  residual_row<true>(op, op_lo, x2, sl, lane, kap, xb, a0, a1, a2);
}

__device__ __forceinline__ void residual_row_f32x(const OpView& op, const float* __restrict__ op_lo,
                                                  const float4* __restrict__ d, int64_t sl, int lane, float kap,
                                                  float4& db, DFAcc& a0, DFAcc& a1, DFAcc& a2) {
  residual_row<false>(op, op_lo, d, sl, lane, kap, db, a0, a1, a2);
}

}  // namespace sph
