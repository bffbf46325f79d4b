// One row of y = A v (or D^-1 A v) over the operator's SELL-32 storage.
//
// Storage: entry j of row s sits at off[s/32] + 32 j + s%32 as an int2
// (x = neighbour row, y = the float32 coefficient's bits), so a warp reading
// entry j of its 32 rows loads 256 consecutive bytes with one instruction.
// The stream is read once per apply: it is loaded with the evict-first hint
// (ld.global.cs) so L1/L2 keep the gathered neighbour vectors instead.
//
// The loop runs to the slice width (uniform across the warp) in groups of U
// entries: U coefficient loads, then U neighbour gathers, then the FMAs, so a
// warp keeps U independent memory requests in flight instead of walking one
// dependent load chain per neighbour.  Entries past a row's own count read the
// row itself with a zero coefficient.
#pragma once

#include "sph_internal.cuh"

namespace sph {

enum : uint8_t { KIND_FLUID = 0, KIND_SHEPARD = 1, KIND_IDENTITY = 2 };

struct OpView {
  const int64_t* off;    // [nslices + 1]
  const int32_t* cnt;    // [n_pad]
  const int2* ih;        // [op_nnz_pad] (row, coefficient bits)
  const uint8_t* kind;   // [n_pad]
  const float* invD;     // [n_pad]
  int64_t nslices;
  int64_t n_pad;
  // per-slice neighbour unions (apply form 5; null until built)
  const int2* loc;       // [op_nnz_pad] (position in the slice's union, coefficient bits)
  const int32_t* uni;    // [op_nnz_pad] the slice's distinct neighbour rows at its offset
  const int32_t* unum;   // [nslices] union size, -1: use ih
  // balanced slice ranges: warp w of a grid of wpart_nw warps takes the
  // contiguous slices [wpart[w], wpart[w + 1]), cut so that every warp streams
  // about the same bytes (null, or another warp count: grid-stride instead).
  // The float64 residual kernels use them; the apply stays grid-stride.
  const int32_t* wpart;  // [wpart_nw + 1]
  int64_t wpart_nw;
};

// The slices warp gw of nw takes: [first, end) in steps of step.
struct SliceRange {
  int64_t first, end, step;
};
__device__ __forceinline__ SliceRange warp_slices(const OpView& op, int64_t gw, int64_t nw) {
  if (op.wpart != nullptr && op.wpart_nw == nw) return SliceRange{op.wpart[gw], op.wpart[gw + 1], 1};
  return SliceRange{gw, op.nslices, nw};
}

// Fluid rows: v_b + sum a (v_b - v_a); Shepard rows: v_b + sum a v_a; identity
// rows: v_b; with Jacobi each row times its invD (1/D on fluid rows, 1 on wall
// rows, times the row scale when one is set).
//
// PF = false: each group of U entries issues its U coefficient loads, then its U
// gathers, then the FMAs.  PF = true: the coefficient loads of the next group
// are issued before the current group's FMAs (software pipelining).  Which of
// the four (U, PF) forms runs fastest depends on the registers the surrounding
// kernel needs, so the solver times them on the actual operator (autotune.cu).
template <int U, bool PF, bool JACOBI>
__device__ __forceinline__ float4 apply_row(const OpView& op, const float4* __restrict__ v, int64_t sl, int lane,
                                            float4& vb_out) {
  const int64_t s = sl * kSlice + lane;
  const int c = op.cnt[s];
  const uint8_t kd = op.kind[s];
  const float4 vb = v[s];
  vb_out = vb;
  const float kap = (kd == KIND_FLUID) ? 1.f : 0.f;
  const int64_t o0 = op.off[sl];
  const int w = (int)((op.off[sl + 1] - o0) / kSlice);
  const int2* __restrict__ p = op.ih + o0 + lane;
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (!PF) {
    for (int j0 = 0; j0 < w; j0 += U) {
      int2 e[U];
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = (j0 + u < c) ? __ldcs(p + (int64_t)(j0 + u) * kSlice) : make_int2((int)s, 0);
      float4 va[U];
#pragma unroll
      for (int u = 0; u < U; ++u) va[u] = __ldg(v + e[u].x);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float a = __int_as_float(e[u].y);
        ax = fmaf(a, fmaf(kap, vb.x, -va[u].x), ax);
        ay = fmaf(a, fmaf(kap, vb.y, -va[u].y), ay);
        az = fmaf(a, fmaf(kap, vb.z, -va[u].z), az);
      }
    }
  } else {
    int2 e[U];
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = (u < c) ? __ldcs(p + (int64_t)u * kSlice) : make_int2((int)s, 0);
    for (int j0 = 0; j0 < w; j0 += U) {
      float4 va[U];
#pragma unroll
      for (int u = 0; u < U; ++u) va[u] = __ldg(v + e[u].x);
      int2 en[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + U + u;
        en[u] = (j < c) ? __ldcs(p + (int64_t)j * kSlice) : make_int2((int)s, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float a = __int_as_float(e[u].y);
        ax = fmaf(a, fmaf(kap, vb.x, -va[u].x), ax);
        ay = fmaf(a, fmaf(kap, vb.y, -va[u].y), ay);
        az = fmaf(a, fmaf(kap, vb.z, -va[u].z), az);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = en[u];
    }
  }
  // with Jacobi every row is multiplied by its invD (1 on wall rows unless a row
  // scale is set: x 1.0f leaves them exact)
  const float sc = JACOBI ? op.invD[s] : 1.f;
  if (kd == KIND_FLUID) return make_float4((vb.x + ax) * sc, (vb.y + ay) * sc, (vb.z + az) * sc, 0.f);
  if (kd == KIND_SHEPARD) return make_float4((vb.x - ax) * sc, (vb.y - ay) * sc, (vb.z - az) * sc, 0.f);
  return make_float4(vb.x * sc, vb.y * sc, vb.z * sc, 0.f);
}

// the row-loop forms of the solver's apply: 0..3 = (U, PF) in {(8,0), (4,0),
// (8,1), (4,1)} above, 4 = the coefficient stream staged through shared memory
// by bulk copies, 5 = neighbour vectors staged per slice in shared memory
// (solver.cu); the batched solver uses forms 0..3
constexpr int kApplyVariants = 6;
constexpr int kApplyVariantsRegister = 4;
// form 5: each slice's neighbour union staged in shared memory (apply_union.cu);
// unions larger than this keep the global-gather path
constexpr int kUnionCap = 512;

}  // namespace sph
