// One row of the float64-accurate residual's operator sum, shared by the
// single-scene and batched residual kernels: sum over the row's stored entries
// of a_ba (kap x_b - x_a) per component, with a = hi + lo and x = hi + lo, in
// double-float arithmetic (DFAcc).  x is interleaved: x2[2 t] = hi, x2[2 t + 1]
// = lo, so one gather reads both halves from the same 32-byte sector.
//
// Entries are taken in groups of kResU: the group's coefficient loads, then its
// gathers of xh and xl, then the error-free sums, so each thread keeps kResU
// gathers in flight.  A slot past the row's count reads the row itself with a
// zero coefficient, which adds exactly nothing.
#pragma once

#include "apply.cuh"
#include "dfloat.cuh"

namespace sph {

constexpr int kResU = 4;

__device__ __forceinline__ void residual_row_df(const OpView& op, const float* __restrict__ op_lo,
                                                const float4* __restrict__ x2, int64_t sl, int lane, float kap,
                                                DFAcc& a0, DFAcc& a1, DFAcc& a2) {
  const int64_t s = sl * kSlice + lane;
  const float4 bh = x2[2 * s], bl = x2[2 * s + 1];
  const int c = op.cnt[s];
  const float kbh0 = kap * bh.x, kbh1 = kap * bh.y, kbh2 = kap * bh.z;
  const float kbl0 = kap * bl.x, kbl1 = kap * bl.y, kbl2 = kap * bl.z;
  const int64_t base = op.off[sl] + lane;
  for (int j0 = 0; j0 < c; j0 += kResU) {
    int2 ih[kResU];
    float lo[kResU];
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      const bool ok = j0 + u < c;
      const int64_t e = base + (int64_t)(j0 + u) * kSlice;
      ih[u] = ok ? __ldcs(op.ih + e) : make_int2((int)s, 0);
      lo[u] = ok ? __ldcs(op_lo + e) : 0.f;
    }
    float4 ah[kResU], al[kResU];
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      ah[u] = __ldg(x2 + 2 * (int64_t)ih[u].x);
      al[u] = __ldg(x2 + 2 * (int64_t)ih[u].x + 1);
    }
#pragma unroll
    for (int u = 0; u < kResU; ++u) {
      const float ahi = __int_as_float(ih[u].y);
      a0.add(ahi, lo[u], kbh0, ah[u].x, kbl0, al[u].x);
      a1.add(ahi, lo[u], kbh1, ah[u].y, kbl1, al[u].y);
      a2.add(ahi, lo[u], kbh2, ah[u].z, kbl2, al[u].z);
    }
  }
}

}  // namespace sph
