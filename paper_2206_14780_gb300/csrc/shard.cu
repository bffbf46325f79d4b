// One system solved over several sub-domains ("ranks"), the domain decomposition
// of paper Sec. 7 and Sec. 7.1, with every rank's data in its own allocations
// and every cross-rank read going through an explicit halo exchange or a
// reduction of per-layer partials.  All ranks run on the calling GPU here (the
// emulated form); the data plane of a real multi-GPU run replaces two kernels:
// the halo gather (k_sh_exchange: a send/recv of the inner-edge rows) and the
// combine of the layer partials (an all-gather of at most layers x 6 doubles,
// summed in layer order on every rank).
//
// Partition.  The cells of the neighbour grid are grouped into layers along the
// longest axis (cell side >= 2h, so a neighbour is always in the same or an
// adjacent layer); each rank owns a contiguous run of layers, balanced by
// particle count.  Rows are numbered layer by layer (within a layer in the
// handle's cell-sorted order) and each layer is padded to whole 32-row slices,
// so no slice straddles two layers or two ranks.  A rank's local rows are its
// owned rows, then its halo: exactly the rows outside the rank that its own
// rows' operator entries reference (the "outer edge" particles of Sec. 7.1).
// Its local operator holds the global operator's rows unchanged (same entries,
// same order), with columns renumbered locally.
//
// Per BiCGSTAB iteration (the restructured listing of Sec. 4.2, paper-exact
// gamma' from a direct dot): p update (in place), halo exchange of p, A p with
// the delta dot, r* update (in place), halo exchange of r*, A r* with its dots,
// x/r update with gamma' and r.r.  The paper exchanges A p and A r* instead and
// updates the halo copies of p in place; exchanging p and r* moves the same
// amount of data.  The Jacobi diagonal, r0 and r0^ need no exchange: every
// rank computes its own rows and the halo rows are never read for them.
//
// Reductions.  Every dot kernel leaves one float32 warp sum per slice (as
// float64); each rank folds its layers' slices, one warp per layer in a fixed
// lane-strided order; the layer partials of all ranks are then summed in layer
// order.  Nothing in that chain depends on where the rank boundaries fall, so
// every scalar -- and hence every iterate -- is bit-identical for any number
// of ranks.  Each rank keeps its own copy of the solver scalars, updated from
// the same sums.
//
// Refinement: after each inner pass x64 += d on owned rows, the float32 hi/lo
// split of x64 is exchanged for the halo rows, and the float64-accurate true
// residual b - A x is recomputed on owned rows (double-float arithmetic on the
// hi + lo coefficients, as the single-domain solver's residual).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "apply.cuh"
#include "bicgstab_scalars.cuh"
#include "residual_row.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kMaxRanks = 64;

// what one rank holds on its device
struct Rank {
  int64_t n_owned = 0;      // owned rows incl. layer padding (a multiple of 32)
  int64_t n_halo = 0;       // halo rows
  int64_t n_local = 0;      // n_owned + n_halo rounded up to 32
  int64_t nslices = 0;      // owned slices
  int64_t slice0 = 0;       // first global slice of the rank
  int32_t layer0 = 0, layer1 = 0;
  DBuf<int64_t> off;        // [nslices + 1]
  DBuf<int32_t> cnt;        // [n_local]
  DBuf<int2> ih;            // local SELL-32 entries (local column, coefficient bits)
  DBuf<float> lo;           // float32 lo of the coefficients
  DBuf<uint8_t> kind;       // [n_local]
  DBuf<float> invD;         // [n_local]
  DBuf<double> D64;         // [n_local]
  DBuf<int32_t> caller;     // [n_owned]: caller index of an owned row, -1 for padding
  DBuf<int32_t> slices;     // [nslices] interior slices (no halo column) first, then edge slices
  int64_t n_interior = 0;   // interior slices
  DBuf<float4> r, rh, p, Ap, rs, As, d, x2;   // x2: [2 n_local]
  DBuf<double> x64, b64, r64;                 // [n_local][3]
  OpView view() const {
    return OpView{off.p, cnt.p, ih.p, kind.p, invD.p, nslices, n_local, nullptr, nullptr, nullptr, nullptr, 0};
  }
};

struct Vec4 {
  float4* r;
  float4* rh;
  float4* p;
  float4* Ap;
  float4* rs;
  float4* As;
  float4* d;
};

// ---- reductions ---------------------------------------------------------------

// float32 warp sum of v (xor butterfly: the same order for every slice)
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per rank: layer partials [layer][K] from the slice partials [global slice][K];
// block l (32 threads) folds layer layer0 + l: lane i takes slices i, i + 32, ...
template <int K>
__global__ void k_sh_layer_reduce(const double* __restrict__ slice_part, const int64_t* __restrict__ layer_slice,
                                  int32_t layer0, double* __restrict__ layer_part) {
  const int layer = layer0 + blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t s0 = layer_slice[layer], s1 = layer_slice[layer + 1];
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int64_t sl = s0 + lane; sl < s1; sl += 32) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += slice_part[sl * kMaxDots + k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum_d(acc[k]);
    if (lane == 0) layer_part[(int64_t)layer * kMaxDots + k] = v;
  }
}

enum : int { CMB_INIT = 0, CMB_DELTA, CMB_OMEGA, CMB_UPDATE, CMB_NORM };

// the layer partials of every rank summed in layer order, then each rank's own
// scalar copy updated (one warp; lanes 0..2 are the three components)
template <int K, int MODE>
__global__ void k_sh_combine(const double* __restrict__ layer_part, int nlayers, SolverScalars* S, int ranks,
                             double eps2, int maxit, double* __restrict__ out) {
  __shared__ double res[K > 0 ? K : 1];
  const int lane = threadIdx.x;
  if (lane < K) {
    double a = 0.0;
    for (int l = 0; l < nlayers; ++l) a += layer_part[(int64_t)l * kMaxDots + lane];
    res[lane] = a;
  }
  __syncwarp();
  if (MODE == CMB_NORM) {
    if (lane < K) out[lane] = res[lane];
    return;
  }
  for (int q = 0; q < ranks; ++q) {
    SolverScalars* Sq = S + q;
    if (MODE == CMB_INIT) {
      if (lane == 0) scal_init(Sq, res, eps2, maxit);
    } else if (Sq->done) {
      // a pass that has stopped runs no further scalar step (as the loop kernels)
    } else if (MODE == CMB_DELTA) {
      scal_after_delta_w(Sq, res);
    } else if (MODE == CMB_OMEGA) {
      scal_after_omega_w(Sq, res);
    } else {
      scal_after_update_w(Sq, res, res + 3);
    }
    __syncwarp();
  }
}

// ---- row kernels (owned rows only; one warp per slice where dots are formed) ----

// r = rh = float32(r64 / D), d = 0; per-slice r.r
__global__ void __launch_bounds__(kBlock) k_sh_pass_init(int64_t nslices, const double* __restrict__ r64,
                                                         const double* __restrict__ D64, Vec4 V,
                                                         double* __restrict__ slice_part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nw) {
    const int64_t s = sl * kSlice + lane;
    const double sc = 1.0 / D64[s];
    const float4 r = make_float4((float)(r64[3 * s] * sc), (float)(r64[3 * s + 1] * sc), (float)(r64[3 * s + 2] * sc),
                                 0.f);
    V.r[s] = r;
    V.rh[s] = r;
    V.d[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float a0 = warp_sum_f(r.x * r.x), a1 = warp_sum_f(r.y * r.y), a2 = warp_sum_f(r.z * r.z);
    if (lane == 0) {
      slice_part[sl * kMaxDots + 0] = a0;
      slice_part[sl * kMaxDots + 1] = a1;
      slice_part[sl * kMaxDots + 2] = a2;
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_sh_p_update(int64_t n, Vec4 V, const SolverScalars* __restrict__ S) {
  if (S->done) return;
  const float b0 = (float)S->beta[0], b1 = (float)S->beta[1], b2 = (float)S->beta[2];
  const float a0 = (float)S->alpha_p[0], a1 = (float)S->alpha_p[1], a2 = (float)S->alpha_p[2];
  const bool useP = (b0 != 0.f) || (b1 != 0.f) || (b2 != 0.f);
  const bool useA = (a0 != 0.f) || (a1 != 0.f) || (a2 != 0.f);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float4 p = V.r[s];
    if (useP) {
      const float4 q = V.p[s];
      p.x = fmaf(b0, q.x, p.x);
      p.y = fmaf(b1, q.y, p.y);
      p.z = fmaf(b2, q.z, p.z);
    }
    if (useA) {
      const float4 q = V.Ap[s];
      p.x = fmaf(-a0, q.x, p.x);
      p.y = fmaf(-a1, q.y, p.y);
      p.z = fmaf(-a2, q.z, p.z);
    }
    p.w = 0.f;
    V.p[s] = p;
  }
}

__global__ void __launch_bounds__(kBlock) k_sh_rstar(int64_t n, Vec4 V, const SolverScalars* __restrict__ S) {
  if (S->done) return;
  const float a0 = (float)S->alpha[0], a1 = (float)S->alpha[1], a2 = (float)S->alpha[2];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 r = V.r[s], ap = V.Ap[s];
    V.rs[s] = make_float4(fmaf(-a0, ap.x, r.x), fmaf(-a1, ap.y, r.y), fmaf(-a2, ap.z, r.z), 0.f);
  }
}

// halo rows of every rank: dst[i] = the owner's value (pointer tables per rank)
__global__ void k_sh_exchange(int64_t m, const int32_t* __restrict__ dst_rank, const int32_t* __restrict__ dst_row,
                              const int32_t* __restrict__ src_rank, const int32_t* __restrict__ src_row,
                              float4* const* __restrict__ ptr, int per_row) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float4* src = ptr[src_rank[i]] + (int64_t)per_row * src_row[i];
    float4* dst = ptr[dst_rank[i]] + (int64_t)per_row * dst_row[i];
    for (int k = 0; k < per_row; ++k) dst[k] = src[k];
  }
}

// y = D^-1 A v with the phase's dots per slice: PH 0: r0^.Ap (3); PH 1: r*.Ar*, Ar*.Ar* (6)
// over the slices slist[k0 .. k1) (slist null: slices k0 .. k1)
template <int PH>
__global__ void __launch_bounds__(kBlock) k_sh_apply(OpView op, const float4* __restrict__ v, float4* __restrict__ y,
                                                     const float4* __restrict__ rh, const SolverScalars* __restrict__ S,
                                                     double* __restrict__ slice_part,
                                                     const int32_t* __restrict__ slist, int64_t k0, int64_t k1) {
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = k0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); k < k1; k += nw) {
    const int64_t sl = slist ? slist[k] : k;
    const int64_t s = sl * kSlice + lane;
    float4 vb;
    const float4 o = apply_row<4, true, true>(op, v, sl, lane, vb);
    y[s] = o;
    if (PH == 0) {
      const float4 h = rh[s];
      const float a0 = warp_sum_f(h.x * o.x), a1 = warp_sum_f(h.y * o.y), a2 = warp_sum_f(h.z * o.z);
      if (lane == 0) {
        slice_part[sl * kMaxDots + 0] = a0;
        slice_part[sl * kMaxDots + 1] = a1;
        slice_part[sl * kMaxDots + 2] = a2;
      }
    } else {
      const float a0 = warp_sum_f(vb.x * o.x), a1 = warp_sum_f(vb.y * o.y), a2 = warp_sum_f(vb.z * o.z);
      const float a3 = warp_sum_f(o.x * o.x), a4 = warp_sum_f(o.y * o.y), a5 = warp_sum_f(o.z * o.z);
      if (lane == 0) {
        double* q = slice_part + sl * kMaxDots;
        q[0] = a0;
        q[1] = a1;
        q[2] = a2;
        q[3] = a3;
        q[4] = a4;
        q[5] = a5;
      }
    }
  }
}

// r = r* - omega Ar*; d += alpha p + omega r*; per-slice r0^.r and r.r
__global__ void __launch_bounds__(kBlock) k_sh_xr_update(int64_t nslices, Vec4 V, const SolverScalars* __restrict__ S,
                                                         double* __restrict__ slice_part) {
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float w0 = (float)S->omega[0], w1 = (float)S->omega[1], w2 = (float)S->omega[2];
  const float al0 = (float)S->alpha[0], al1 = (float)S->alpha[1], al2 = (float)S->alpha[2];
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nw) {
    const int64_t s = sl * kSlice + lane;
    const float4 rs = V.rs[s], as = V.As[s], h = V.rh[s], p = V.p[s];
    float4 d = V.d[s];
    const float4 r = make_float4(fmaf(-w0, as.x, rs.x), fmaf(-w1, as.y, rs.y), fmaf(-w2, as.z, rs.z), 0.f);
    d.x = fmaf(w0, rs.x, fmaf(al0, p.x, d.x));
    d.y = fmaf(w1, rs.y, fmaf(al1, p.y, d.y));
    d.z = fmaf(w2, rs.z, fmaf(al2, p.z, d.z));
    V.r[s] = r;
    V.d[s] = d;
    const float g0 = warp_sum_f(h.x * r.x), g1 = warp_sum_f(h.y * r.y), g2 = warp_sum_f(h.z * r.z);
    const float q0 = warp_sum_f(r.x * r.x), q1 = warp_sum_f(r.y * r.y), q2 = warp_sum_f(r.z * r.z);
    if (lane == 0) {
      double* q = slice_part + sl * kMaxDots;
      q[0] = g0;
      q[1] = g1;
      q[2] = g2;
      q[3] = q0;
      q[4] = q1;
      q[5] = q2;
    }
  }
}

// x64 += d, then the float32 hi / lo split of x64 (owned rows)
__global__ void k_sh_add_split(int64_t n, const float4* __restrict__ d, int add, double* __restrict__ x,
                               float4* __restrict__ x2) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    double x0 = x[3 * s], x1 = x[3 * s + 1], x2c = x[3 * s + 2];
    if (add) {
      const float4 v = d[s];
      x0 += (double)v.x;
      x1 += (double)v.y;
      x2c += (double)v.z;
      x[3 * s] = x0;
      x[3 * s + 1] = x1;
      x[3 * s + 2] = x2c;
    }
    const float h0 = (float)x0, h1 = (float)x1, h2 = (float)x2c;
    x2[2 * s] = make_float4(h0, h1, h2, 0.f);
    x2[2 * s + 1] = make_float4((float)(x0 - (double)h0), (float)(x1 - (double)h1), (float)(x2c - (double)h2), 0.f);
  }
}

// r64 = b - A x (owned rows; padding rows give 0); per-slice r64.r64 in float64
__global__ void __launch_bounds__(kBlock) k_sh_residual(OpView op, const float* __restrict__ op_lo,
                                                        const float4* __restrict__ x2, const double* __restrict__ x,
                                                        const double* __restrict__ b, const int32_t* __restrict__ caller,
                                                        double* __restrict__ r, double* __restrict__ slice_part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < op.nslices; sl += nw) {
    const int64_t s = sl * kSlice + lane;
    const uint8_t k = op.kind[s];
    const float kap = (k == KIND_FLUID) ? 1.f : 0.f;
    DFAcc a0, a1, a2;
    residual_row_df(op, op_lo, x2, sl, lane, kap, a0, a1, a2);
    const double sg = (k == KIND_FLUID) ? 1.0 : (k == KIND_SHEPARD ? -1.0 : 0.0);
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    if (caller[s] >= 0) {
      r0 = b[3 * s] - (x[3 * s] + sg * a0.value());
      r1 = b[3 * s + 1] - (x[3 * s + 1] + sg * a1.value());
      r2 = b[3 * s + 2] - (x[3 * s + 2] + sg * a2.value());
    }
    r[3 * s] = r0;
    r[3 * s + 1] = r1;
    r[3 * s + 2] = r2;
    const double q0 = warp_sum_d(r0 * r0), q1 = warp_sum_d(r1 * r1), q2 = warp_sum_d(r2 * r2);
    if (lane == 0) {
      slice_part[sl * kMaxDots + 0] = q0;
      slice_part[sl * kMaxDots + 1] = q1;
      slice_part[sl * kMaxDots + 2] = q2;
    }
  }
}

// b.b per slice (owned rows)
__global__ void k_sh_norm_b(int64_t nslices, const double* __restrict__ b, double* __restrict__ slice_part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nw) {
    const int64_t s = sl * kSlice + lane;
    const double q0 = warp_sum_d(b[3 * s] * b[3 * s]), q1 = warp_sum_d(b[3 * s + 1] * b[3 * s + 1]),
                 q2 = warp_sum_d(b[3 * s + 2] * b[3 * s + 2]);
    if (lane == 0) {
      slice_part[sl * kMaxDots + 0] = q0;
      slice_part[sl * kMaxDots + 1] = q1;
      slice_part[sl * kMaxDots + 2] = q2;
    }
  }
}

// caller-order [n][3] -> owned rows (padding rows 0), and back
__global__ void k_sh_gather(int64_t n, const int32_t* __restrict__ caller, const double* __restrict__ src,
                            double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = caller[s];
    dst[3 * s] = i >= 0 ? src[3 * (int64_t)i] : 0.0;
    dst[3 * s + 1] = i >= 0 ? src[3 * (int64_t)i + 1] : 0.0;
    dst[3 * s + 2] = i >= 0 ? src[3 * (int64_t)i + 2] : 0.0;
  }
}

__global__ void k_sh_scatter(int64_t n, const int32_t* __restrict__ caller, const double* __restrict__ src,
                             double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = caller[s];
    if (i >= 0) {
      dst[3 * (int64_t)i] = src[3 * s];
      dst[3 * (int64_t)i + 1] = src[3 * s + 1];
      dst[3 * (int64_t)i + 2] = src[3 * s + 2];
    }
  }
}

}  // namespace

// ---- partition (host only) -----------------------------------------------------

sph_status shard_plan(int64_t n, const int32_t* layer, int32_t nlayers, int32_t ranks, int64_t* virt,
                      int32_t* rank_first_layer, int64_t* layer_first_virt) {
  if (n < 1 || !layer || nlayers < 1 || ranks < 1 || ranks > kMaxRanks || !virt || !rank_first_layer ||
      !layer_first_virt) {
    set_error("sph_shard_plan: need n >= 1, nlayers >= 1, 1 <= ranks <= %d and non-null arrays", kMaxRanks);
    return SPH_ERR_INVALID;
  }
  if (ranks > nlayers) {
    set_error("sph_shard_plan: %d ranks need at least as many layers (%d)", ranks, nlayers);
    return SPH_ERR_INVALID;
  }
  std::vector<int64_t> count(nlayers, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (layer[i] < 0 || layer[i] >= nlayers) {
      set_error("sph_shard_plan: row %lld has layer %d outside 0..%d", (long long)i, layer[i], nlayers - 1);
      return SPH_ERR_INVALID;
    }
    ++count[layer[i]];
  }
  // layers padded to whole slices, numbered in order
  layer_first_virt[0] = 0;
  for (int l = 0; l < nlayers; ++l)
    layer_first_virt[l + 1] = layer_first_virt[l] + (count[l] + kSlice - 1) / kSlice * kSlice;
  // rows keep their order within a layer
  std::vector<int64_t> next(layer_first_virt, layer_first_virt + nlayers);
  for (int64_t i = 0; i < n; ++i) virt[i] = next[layer[i]]++;
  // rank q starts at the first layer whose preceding rows reach q / ranks of all
  // rows, each rank keeping at least one layer
  rank_first_layer[0] = 0;
  int l = 0;
  int64_t before = 0;
  for (int q = 1; q < ranks; ++q) {
    const double target = (double)n * q / ranks;
    while (l < nlayers - (ranks - q) && (double)(before + count[l]) <= target) before += count[l++];
    if (l < rank_first_layer[q - 1] + 1) {
      before += count[l];
      ++l;
    }
    rank_first_layer[q] = l;
  }
  rank_first_layer[ranks] = nlayers;
  return SPH_OK;
}

}  // namespace sph

// The opaque handle of the sharded solve.
struct sph_shard {
  int ranks = 0;
  int axis = 0;
  int nlayers = 0;
  int device = 0;
  int64_t n = 0;
  sph_neighbors* H = nullptr;
  uint64_t op_version = 0;
  std::vector<sph::Rank> rk;
  std::vector<int32_t> rank_first_layer;
  sph::DBuf<int64_t> layer_slice;        // [nlayers + 1] global slice offsets of the layers
  sph::DBuf<double> slice_part;          // [total slices][kMaxDots]  (each rank writes its own slices)
  sph::DBuf<double> layer_part;          // [nlayers][kMaxDots]       (the all-gathered layer partials)
  sph::DBuf<sph::SolverScalars> scal;    // [ranks] each rank's own copy
  sph::DBuf<double> outv;                // [4] norms read by the host
  // halo exchange list over all ranks
  int64_t n_exchange = 0;
  sph::DBuf<int32_t> ex_dst_rank, ex_dst_row, ex_src_rank, ex_src_row;
  sph::DBuf<float4*> ptr_tab;            // [8][ranks] per-vector pointer tables
  std::vector<int64_t> halo_rows;
  sph::SolverScalars* host_scal = nullptr;
  // striping: the halo exchange on its own stream while the interior slices compute
  bool striped = false;
  cudaStream_t xstream = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
};

namespace sph {

namespace {

enum { TAB_P = 0, TAB_RS = 1, TAB_X2 = 2 };

sph_status shard_release(sph_shard* Z) {
  for (auto& R : Z->rk) {
    R.off.release();
    R.cnt.release();
    R.ih.release();
    R.lo.release();
    R.kind.release();
    R.invD.release();
    R.D64.release();
    R.caller.release();
    R.slices.release();
    for (DBuf<float4>* v : {&R.r, &R.rh, &R.p, &R.Ap, &R.rs, &R.As, &R.d, &R.x2}) v->release();
    R.x64.release();
    R.b64.release();
    R.r64.release();
  }
  Z->layer_slice.release();
  Z->slice_part.release();
  Z->layer_part.release();
  Z->scal.release();
  Z->outv.release();
  Z->ex_dst_rank.release();
  Z->ex_dst_row.release();
  Z->ex_src_rank.release();
  Z->ex_src_row.release();
  Z->ptr_tab.release();
  if (Z->host_scal) cudaFreeHost(Z->host_scal);
  Z->host_scal = nullptr;
  if (Z->ev_ready) cudaEventDestroy(Z->ev_ready);
  if (Z->ev_done) cudaEventDestroy(Z->ev_done);
  if (Z->xstream) cudaStreamDestroy(Z->xstream);
  Z->ev_ready = Z->ev_done = nullptr;
  Z->xstream = nullptr;
  return SPH_OK;
}

template <class T>
sph_status upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t st) {
  SPH_TRY(d.alloc(h.size() ? h.size() : 1));
  if (!h.empty()) SPH_TRY_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return SPH_OK;
}

template <class T>
sph_status download(std::vector<T>& h, const DBuf<T>& d, size_t count, cudaStream_t st) {
  h.resize(count);
  if (count) SPH_TRY_CUDA(cudaMemcpyAsync(h.data(), d.p, count * sizeof(T), cudaMemcpyDeviceToHost, st));
  return SPH_OK;
}

sph_status shard_build(sph_shard* Z, cudaStream_t st) {
  sph_neighbors* H = Z->H;
  const int64_t n = H->n, np = H->n_pad;
  // longest axis of the box; its cell layers
  int axis = 0;
  for (int a = 1; a < 3; ++a)
    if (H->grid.L[a] > H->grid.L[axis]) axis = a;
  Z->axis = axis;
  Z->nlayers = H->grid.ncell[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? H->grid.ncell[0] : (int64_t)H->grid.ncell[0] * H->grid.ncell[1]);
  // the operator and particle bookkeeping, on the host
  std::vector<int32_t> key, perm, cnt;
  std::vector<int64_t> off;
  std::vector<int2> ih;
  std::vector<float> lo, invD;
  std::vector<uint8_t> kind;
  std::vector<double> D64;
  SPH_TRY(download(key, H->key_s, n, st));
  SPH_TRY(download(perm, H->perm, n, st));
  SPH_TRY(download(cnt, H->op_cnt, np, st));
  SPH_TRY(download(off, H->op_off, H->nslices + 1, st));
  SPH_TRY(download(kind, H->op_kind, np, st));
  SPH_TRY(download(invD, H->invD, np, st));
  SPH_TRY(download(D64, H->D64, np, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  SPH_TRY(download(ih, H->op_ih, off[H->nslices], st));
  SPH_TRY(download(lo, H->op_lo, off[H->nslices], st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> layer(n);
  for (int64_t s = 0; s < n; ++s) layer[s] = (int32_t)((key[s] / stride) % H->grid.ncell[axis]);
  const int R = Z->ranks;
  std::vector<int64_t> virt(n), layer_virt(Z->nlayers + 1);
  Z->rank_first_layer.assign(R + 1, 0);
  SPH_TRY(shard_plan(n, layer.data(), Z->nlayers, R, virt.data(), Z->rank_first_layer.data(), layer_virt.data()));
  const int64_t nvirt = layer_virt[Z->nlayers];
  std::vector<int64_t> sorted_of_virt(nvirt, -1);
  for (int64_t s = 0; s < n; ++s) sorted_of_virt[virt[s]] = s;
  std::vector<int64_t> layer_slice(Z->nlayers + 1);
  for (int l = 0; l <= Z->nlayers; ++l) layer_slice[l] = layer_virt[l] / kSlice;
  SPH_TRY(upload(Z->layer_slice, layer_slice, st));
  // owner of every virtual row
  std::vector<int32_t> owner(nvirt);
  for (int q = 0; q < R; ++q)
    for (int64_t v = layer_virt[Z->rank_first_layer[q]]; v < layer_virt[Z->rank_first_layer[q + 1]]; ++v) owner[v] = q;
  Z->rk.clear();
  Z->rk.resize(R);
  Z->halo_rows.assign(R, 0);
  std::vector<int32_t> exr_d, exi_d, exr_s, exi_s;
  for (int q = 0; q < R; ++q) {
    Rank& K = Z->rk[q];
    K.layer0 = Z->rank_first_layer[q];
    K.layer1 = Z->rank_first_layer[q + 1];
    const int64_t v0 = layer_virt[K.layer0], v1 = layer_virt[K.layer1];
    K.n_owned = v1 - v0;
    K.nslices = K.n_owned / kSlice;
    K.slice0 = v0 / kSlice;
    // halo: the non-owned columns of the owned rows, in virtual order
    std::vector<int64_t> halo;
    for (int64_t v = v0; v < v1; ++v) {
      const int64_t s = sorted_of_virt[v];
      if (s < 0) continue;
      const int64_t o = off[s / kSlice] + s % kSlice;
      for (int j = 0; j < cnt[s]; ++j) {
        const int64_t col = virt[ih[o + (int64_t)j * kSlice].x];
        if (col < v0 || col >= v1) halo.push_back(col);
      }
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    K.n_halo = (int64_t)halo.size();
    K.n_local = (K.n_owned + K.n_halo + kSlice - 1) / kSlice * kSlice;
    Z->halo_rows[q] = K.n_halo;
    auto local_of = [&](int64_t col) -> int32_t {
      if (col >= v0 && col < v1) return (int32_t)(col - v0);
      return (int32_t)(K.n_owned + (std::lower_bound(halo.begin(), halo.end(), col) - halo.begin()));
    };
    for (int64_t h = 0; h < K.n_halo; ++h) {
      const int64_t col = halo[h];
      exr_d.push_back(q);
      exi_d.push_back((int32_t)(K.n_owned + h));
      const int src = owner[col];
      exr_s.push_back(src);
      exi_s.push_back((int32_t)(col - layer_virt[Z->rank_first_layer[src]]));
    }
    // local SELL-32 of the owned rows: the global rows unchanged, columns renumbered
    std::vector<int64_t> loff(K.nslices + 1, 0);
    std::vector<int32_t> lcnt(K.n_local, 0), lcaller(K.n_owned, -1);
    std::vector<uint8_t> lkind(K.n_local, KIND_IDENTITY);
    std::vector<float> linvD(K.n_local, 1.f);
    std::vector<double> lD64(K.n_local, 1.0);
    for (int64_t i = 0; i < K.n_owned; ++i) {
      const int64_t s = sorted_of_virt[v0 + i];
      if (s < 0) continue;
      lcnt[i] = cnt[s];
      lkind[i] = kind[s];
      linvD[i] = invD[s];
      lD64[i] = D64[s];
      lcaller[i] = perm[s];
    }
    for (int64_t sl = 0; sl < K.nslices; ++sl) {
      int w = 0;
      for (int l = 0; l < kSlice; ++l) w = std::max(w, lcnt[sl * kSlice + l]);
      loff[sl + 1] = loff[sl] + (int64_t)w * kSlice;
    }
    std::vector<int2> lih(std::max<int64_t>(loff[K.nslices], 1), make_int2(0, 0));
    std::vector<float> llo(lih.size(), 0.f);
    for (int64_t i = 0; i < K.n_owned; ++i) {
      const int64_t s = sorted_of_virt[v0 + i];
      if (s < 0) continue;
      const int64_t o = off[s / kSlice] + s % kSlice;
      const int64_t lo0 = loff[i / kSlice] + i % kSlice;
      for (int j = 0; j < cnt[s]; ++j) {
        const int2 e = ih[o + (int64_t)j * kSlice];
        lih[lo0 + (int64_t)j * kSlice] = make_int2(local_of(virt[e.x]), e.y);
        llo[lo0 + (int64_t)j * kSlice] = lo[o + (int64_t)j * kSlice];
      }
    }
    SPH_TRY(upload(K.off, loff, st));
    SPH_TRY(upload(K.cnt, lcnt, st));
    SPH_TRY(upload(K.ih, lih, st));
    SPH_TRY(upload(K.lo, llo, st));
    SPH_TRY(upload(K.kind, lkind, st));
    SPH_TRY(upload(K.invD, linvD, st));
    SPH_TRY(upload(K.D64, lD64, st));
    SPH_TRY(upload(K.caller, lcaller, st));
    // slices whose rows reference no halo row can be applied before the exchange
    std::vector<int32_t> inner, edge;
    for (int64_t sl = 0; sl < K.nslices; ++sl) {
      bool halo_ref = false;
      for (int64_t e = loff[sl]; e < loff[sl + 1] && !halo_ref; ++e) halo_ref = lih[e].x >= K.n_owned;
      (halo_ref ? edge : inner).push_back((int32_t)sl);
    }
    K.n_interior = (int64_t)inner.size();
    inner.insert(inner.end(), edge.begin(), edge.end());
    if (inner.empty()) inner.push_back(0);
    SPH_TRY(upload(K.slices, inner, st));
    for (DBuf<float4>* v : {&K.r, &K.rh, &K.p, &K.Ap, &K.rs, &K.As, &K.d}) {
      SPH_TRY(v->alloc(K.n_local));
      SPH_TRY_CUDA(cudaMemsetAsync(v->p, 0, K.n_local * sizeof(float4), st));
    }
    SPH_TRY(K.x2.alloc(2 * K.n_local));
    SPH_TRY_CUDA(cudaMemsetAsync(K.x2.p, 0, 2 * K.n_local * sizeof(float4), st));
    SPH_TRY(K.x64.alloc(3 * K.n_local));
    SPH_TRY(K.b64.alloc(3 * K.n_local));
    SPH_TRY(K.r64.alloc(3 * K.n_local));
  }
  Z->n_exchange = (int64_t)exr_d.size();
  SPH_TRY(upload(Z->ex_dst_rank, exr_d, st));
  SPH_TRY(upload(Z->ex_dst_row, exi_d, st));
  SPH_TRY(upload(Z->ex_src_rank, exr_s, st));
  SPH_TRY(upload(Z->ex_src_row, exi_s, st));
  std::vector<float4*> tab(3 * R);
  for (int q = 0; q < R; ++q) {
    tab[TAB_P * R + q] = Z->rk[q].p.p;
    tab[TAB_RS * R + q] = Z->rk[q].rs.p;
    tab[TAB_X2 * R + q] = Z->rk[q].x2.p;
  }
  SPH_TRY(upload(Z->ptr_tab, tab, st));
  SPH_TRY(Z->slice_part.alloc((size_t)(nvirt / kSlice) * kMaxDots));
  SPH_TRY_CUDA(cudaMemsetAsync(Z->slice_part.p, 0, (size_t)(nvirt / kSlice) * kMaxDots * sizeof(double), st));
  SPH_TRY(Z->layer_part.alloc((size_t)Z->nlayers * kMaxDots));
  SPH_TRY(Z->scal.alloc(R));
  SPH_TRY_CUDA(cudaMemsetAsync(Z->scal.p, 0, R * sizeof(SolverScalars), st));
  SPH_TRY(Z->outv.alloc(4));
  if (!Z->host_scal) SPH_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&Z->host_scal), sizeof(SolverScalars)));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  Z->op_version = H->op_version;
  return SPH_OK;
}

int rows_grid(const sph_neighbors* H, int64_t rows) { return grid_for(H, rows); }

// every rank's layer reduce, then the combine
template <int K, int MODE>
sph_status reduce_all(sph_shard* Z, cudaStream_t st, double eps2 = 0.0, int maxit = 0) {
  for (const Rank& R : Z->rk) {
    const int nl = R.layer1 - R.layer0;
    SPH_LAUNCH(k_sh_layer_reduce<K>, nl, 32, 0, st)(Z->slice_part.p, Z->layer_slice.p, R.layer0, Z->layer_part.p);
  }
  auto combine = k_sh_combine<K, MODE>;
  SPH_LAUNCH(combine, 1, 32, 0, st)(Z->layer_part.p, Z->nlayers, Z->scal.p, Z->ranks, eps2, maxit, Z->outv.p);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

sph_status exchange(sph_shard* Z, int tab, int per_row, cudaStream_t st) {
  if (Z->n_exchange == 0) return SPH_OK;
  SPH_LAUNCH(k_sh_exchange, rows_grid(Z->H, Z->n_exchange), kBlock, 0, st)(
      Z->n_exchange, Z->ex_dst_rank.p, Z->ex_dst_row.p, Z->ex_src_rank.p, Z->ex_src_row.p,
      Z->ptr_tab.p + (size_t)tab * Z->ranks, per_row);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

Vec4 vecs(Rank& R) { return Vec4{R.r.p, R.rh.p, R.p.p, R.Ap.p, R.rs.p, R.As.p, R.d.p}; }

double* part_of(sph_shard* Z, const Rank& R) { return Z->slice_part.p + R.slice0 * kMaxDots; }

// the halo exchange of p (PH 0) or r* (PH 1) and every rank's apply of it with the
// phase's per-slice dots.  Striped (Sec. 7.1's overlap of transfers with computation):
// the exchange runs on its own stream while the interior slices, which reference
// no halo row, are applied; the edge slices follow once it is done.  Each slice's
// result and dots are the same either way, so the iterates do not change.
template <int PH>
sph_status apply_phase(sph_shard* Z, cudaStream_t st) {
  const int tab = PH == 0 ? TAB_P : TAB_RS;
  auto launch = [&](int q, const int32_t* slist, int64_t k0, int64_t k1) {
    Rank& R = Z->rk[q];
    SPH_LAUNCH(k_sh_apply<PH>, rows_grid(Z->H, R.n_owned), kBlock, 0, st)(
        R.view(), PH == 0 ? R.p.p : R.rs.p, PH == 0 ? R.Ap.p : R.As.p, R.rh.p, Z->scal.p + q, part_of(Z, R), slist,
        k0, k1);
  };
  if (!Z->striped || Z->n_exchange == 0) {
    SPH_TRY(exchange(Z, tab, 1, st));
    for (int q = 0; q < Z->ranks; ++q) launch(q, nullptr, 0, Z->rk[q].nslices);
    return SPH_OK;
  }
  SPH_TRY_CUDA(cudaEventRecord(Z->ev_ready, st));
  SPH_TRY_CUDA(cudaStreamWaitEvent(Z->xstream, Z->ev_ready, 0));
  SPH_TRY(exchange(Z, tab, 1, Z->xstream));
  SPH_TRY_CUDA(cudaEventRecord(Z->ev_done, Z->xstream));
  for (int q = 0; q < Z->ranks; ++q)
    if (Z->rk[q].n_interior > 0) launch(q, Z->rk[q].slices.p, 0, Z->rk[q].n_interior);
  SPH_TRY_CUDA(cudaStreamWaitEvent(st, Z->ev_done, 0));
  for (int q = 0; q < Z->ranks; ++q)
    if (Z->rk[q].n_interior < Z->rk[q].nslices) launch(q, Z->rk[q].slices.p, Z->rk[q].n_interior, Z->rk[q].nslices);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

// x64 (+ d when add), its hi/lo split, the split's halo exchange, r64 = b - A x and |r64|^2 per component
sph_status shard_residual(sph_shard* Z, bool add, cudaStream_t st, double rr[3]) {
  for (Rank& R : Z->rk)
    SPH_LAUNCH(k_sh_add_split, rows_grid(Z->H, R.n_owned), kBlock, 0, st)(R.n_owned, R.d.p, add ? 1 : 0, R.x64.p,
                                                                        R.x2.p);
  SPH_TRY(exchange(Z, TAB_X2, 2, st));
  for (Rank& R : Z->rk)
    SPH_LAUNCH(k_sh_residual, rows_grid(Z->H, R.n_owned), kBlock, 0, st)(R.view(), R.lo.p, R.x2.p, R.x64.p, R.b64.p,
                                                                       R.caller.p, R.r64.p, part_of(Z, R));
  SPH_TRY((reduce_all<3, CMB_NORM>(Z, st)));
  SPH_TRY_CUDA(cudaMemcpyAsync(rr, Z->outv.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

}  // namespace

sph_status shard_create(sph_neighbors* H, const sph_visc_params* P, int32_t ranks, sph_shard** out, cudaStream_t st) {
  if (!H || !P || !out || ranks < 1 || ranks > kMaxRanks) {
    set_error("sph_shard_create: need a handle, parameters, an output and 1 <= ranks <= %d", kMaxRanks);
    return SPH_ERR_INVALID;
  }
  if (H->row_scaled) {
    set_error("sph_shard_create: the sharded solve uses the Jacobi diagonal alone; clear the row scale first");
    return SPH_ERR_INVALID;
  }
  SPH_TRY(ensure_operator(H, P, st));
  sph_shard* Z = new sph_shard();
  Z->ranks = ranks;
  Z->H = H;
  Z->n = H->n;
  Z->device = H->device;
  sph_status s = shard_build(Z, st);
  if (s == SPH_OK && (cudaStreamCreateWithFlags(&Z->xstream, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&Z->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&Z->ev_done, cudaEventDisableTiming) != cudaSuccess)) {
    set_error("sph_shard_create: could not create the exchange stream and its events");
    s = SPH_ERR_CUDA;
  }
  if (s != SPH_OK) {
    shard_release(Z);
    delete Z;
    return s;
  }
  *out = Z;
  return SPH_OK;
}

sph_status shard_destroy(sph_shard* Z) {
  if (!Z) return SPH_OK;
  shard_release(Z);
  delete Z;
  return SPH_OK;
}

sph_status shard_set_striping(sph_shard* Z, int32_t on) {
  if (!Z || (on != 0 && on != 1)) {
    set_error("sph_shard_set_striping: null shard or a flag other than 0 / 1");
    return SPH_ERR_INVALID;
  }
  Z->striped = on != 0;
  return SPH_OK;
}

sph_status shard_info(const sph_shard* Z, int32_t* axis, int32_t* layers, int64_t* owned, int64_t* halo,
                      int64_t* exchanged) {
  if (!Z) {
    set_error("sph_shard_info: null shard");
    return SPH_ERR_INVALID;
  }
  if (axis) *axis = Z->axis;
  if (layers) *layers = Z->nlayers;
  for (int q = 0; q < Z->ranks; ++q) {
    if (owned) owned[q] = Z->rk[q].n_owned;
    if (halo) halo[q] = Z->halo_rows[q];
  }
  if (exchanged) *exchanged = Z->n_exchange;
  return SPH_OK;
}

sph_status shard_solve(sph_shard* Z, const sph_solve_opts* O, const double* b, double* x, sph_solve_report* Rp,
                       cudaStream_t st) {
  if (!Z || !O || !b || !x || !Rp) {
    set_error("sph_shard_solve: null argument");
    return SPH_ERR_INVALID;
  }
  if (O->precision != SPH_PREC_MIXED || O->method != SPH_SOLVER_BICGSTAB || !O->jacobi || O->merged_reductions) {
    set_error("sph_shard_solve: the sharded solve is the mixed-precision Jacobi-scaled BiCGSTAB with direct "
              "reductions (precision 0, method 0, jacobi 1, merged_reductions 0)");
    return SPH_ERR_INVALID;
  }
  if (Z->H->op_version != Z->op_version || !Z->H->op_valid) {
    set_error("sph_shard_solve: the handle's operator changed since sph_shard_create; create the shard again");
    return SPH_ERR_INVALID;
  }
  const double rtol = O->rtol > 0.0 ? O->rtol : 1e-6;
  const double eps_floor = O->eps_inner > 0.0 ? O->eps_inner : 2e-2;
  const int maxit = O->maxit > 0 ? O->maxit : 10000;
  const int max_ref = O->max_refine > 0 ? O->max_refine : 20;
  const int chunk = O->chunk > 0 ? O->chunk : 8;
  sph_neighbors* H = Z->H;
  for (Rank& R : Z->rk) {
    SPH_LAUNCH(k_sh_gather, rows_grid(H, R.n_owned), kBlock, 0, st)(R.n_owned, R.caller.p, b, R.b64.p);
    SPH_LAUNCH(k_sh_gather, rows_grid(H, R.n_owned), kBlock, 0, st)(R.n_owned, R.caller.p, x, R.x64.p);
    SPH_LAUNCH(k_sh_norm_b, rows_grid(H, R.n_owned), kBlock, 0, st)(R.nslices, R.b64.p, part_of(Z, R));
  }
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY((reduce_all<3, CMB_NORM>(Z, st)));
  double bb[3];
  SPH_TRY_CUDA(cudaMemcpyAsync(bb, Z->outv.p, sizeof(bb), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bb[0] + bb[1] + bb[2]);
  std::memset(Rp, 0, sizeof(*Rp));
  double rr[3];
  SPH_TRY(shard_residual(Z, false, st, rr));
  int total = 0, passes = 0;
  sph_status status = SPH_NOT_CONVERGED;
  SolverScalars* S0 = Z->scal.p;
  for (int ref = 0;; ++ref) {
    const double rnorm = std::sqrt(rr[0] + rr[1] + rr[2]);
    if (!std::isfinite(rnorm)) {
      set_error("sph_shard_solve: the true residual is not finite");
      status = SPH_ERR_NONFINITE;
      break;
    }
    if (rnorm <= rtol * bnorm) {
      status = SPH_OK;
      break;
    }
    if (ref >= max_ref || total >= maxit) break;
    const double eps = std::fmax(eps_floor, 0.25 * rtol * bnorm / rnorm);
    for (Rank& R : Z->rk)
      SPH_LAUNCH(k_sh_pass_init, rows_grid(H, R.n_owned), kBlock, 0, st)(R.nslices, R.r64.p, R.D64.p, vecs(R),
                                                                          part_of(Z, R));
    SPH_TRY((reduce_all<3, CMB_INIT>(Z, st, eps * eps, maxit - total)));
    for (;;) {
      for (int it = 0; it < chunk; ++it) {
        for (int q = 0; q < Z->ranks; ++q) {
          Rank& R = Z->rk[q];
          SPH_LAUNCH(k_sh_p_update, rows_grid(H, R.n_owned), kBlock, 0, st)(R.n_owned, vecs(R), Z->scal.p + q);
        }
        SPH_TRY(apply_phase<0>(Z, st));
        SPH_TRY((reduce_all<3, CMB_DELTA>(Z, st)));
        for (int q = 0; q < Z->ranks; ++q) {
          Rank& R = Z->rk[q];
          SPH_LAUNCH(k_sh_rstar, rows_grid(H, R.n_owned), kBlock, 0, st)(R.n_owned, vecs(R), Z->scal.p + q);
        }
        SPH_TRY(apply_phase<1>(Z, st));
        SPH_TRY((reduce_all<6, CMB_OMEGA>(Z, st)));
        for (int q = 0; q < Z->ranks; ++q) {
          Rank& R = Z->rk[q];
          SPH_LAUNCH(k_sh_xr_update, rows_grid(H, R.n_owned), kBlock, 0, st)(R.nslices, vecs(R), Z->scal.p + q,
                                                                             part_of(Z, R));
        }
        SPH_TRY((reduce_all<6, CMB_UPDATE>(Z, st)));
      }
      SPH_TRY_CUDA(cudaGetLastError());
      SPH_TRY_CUDA(cudaMemcpyAsync(Z->host_scal, S0, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
      SPH_TRY_CUDA(cudaStreamSynchronize(st));
      if (Z->host_scal->done) break;
    }
    const SolverScalars& hs = *Z->host_scal;
    total += hs.iter;
    passes++;
    for (int c = 0; c < 3; ++c) {
      Rp->state[c] = (int8_t)hs.state[c];
      Rp->stalled_any[c] |= (int8_t)hs.stalled_any[c];
    }
    SPH_TRY(shard_residual(Z, true, st, rr));
    if (hs.iter == 0) {
      const double rn = std::sqrt(rr[0] + rr[1] + rr[2]);
      status = rn <= rtol * bnorm ? SPH_OK : SPH_NOT_CONVERGED;
      break;
    }
  }
  for (Rank& R : Z->rk) SPH_LAUNCH(k_sh_scatter, rows_grid(H, R.n_owned), kBlock, 0, st)(R.n_owned, R.caller.p, R.x64.p, x);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  Rp->iters = total;
  Rp->refinements = passes;
  Rp->true_rel_res = bnorm > 0.0 ? std::sqrt(rr[0] + rr[1] + rr[2]) / bnorm : std::sqrt(rr[0] + rr[1] + rr[2]);
  for (int c = 0; c < 3; ++c) Rp->true_rel_res_c[c] = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : std::sqrt(rr[c]);
  Rp->status = status;
  if (status == SPH_NOT_CONVERGED)
    set_error("sph_shard_solve: true residual %.3e above rtol %.1e after %d iterations / %d passes", Rp->true_rel_res,
              rtol, total, passes);
  return status;
}

}  // namespace sph
