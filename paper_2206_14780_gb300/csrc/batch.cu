// Batched ensemble solve: S independent scenes (each with its own A(dt)) solved
// together, every scene by the restructured BiCGSTAB of paper Sec. 4.2 with its
// own scalars, states and stopping decision.
//
// Layout: the scenes' rows are concatenated (each scene padded to whole 32-row
// slices by its handle); work is split into tiles of up to 32 slices (1024 rows,
// one 256-thread block, 4 slices per warp) that never span two scenes.  Operators stay on their handles; a
// per-scene descriptor points at them.  Dot products are reduced per tile
// (float32 warps, float64 blocks) into a per-tile partial, and the last tile of
// a scene to arrive (ticket on a per-scene counter) sums that scene's partials
// in a fixed order and runs the scene's scalar update.
//
// One refinement pass is four launches: float64 residual per scene (decides on
// the device which scenes still exceed rtol), pass initialisation, one
// persistent cooperative kernel that runs all BiCGSTAB iterations of the active
// scenes with grid barriers between phases, and x += d.  The whole solve is one
// CUDA graph launch: the pass sits in the body of a conditional WHILE node whose
// last kernel decides on the device whether another pass follows (some scene
// still above rtol, passes left, no barrier timed out); where the driver cannot
// build that graph, the pass alone is captured and replayed by the host.  Converged scenes are skipped tile by
// tile, so the grid keeps working on the scenes that remain.  Every grid
// barrier spins a bounded number of times and reports SPH_ERR_TIMEOUT instead
// of hanging.
#include <cmath>
#include <cstring>
#include <vector>

#include "apply.cuh"
#include "bicgstab_scalars.cuh"
#include "dfloat.cuh"
#include "reduce.cuh"
#include "residual_row.cuh"
#include "sph_internal.cuh"

namespace sph {

// A tile is a run of consecutive SELL slices of one scene taken by one block
// (each warp takes every 8th or 4th slice of it).  Its length is autotuned
// among kTileCands on the first solve, after the row-loop form and block size;
// the default is the middle one.
constexpr int kTileCands[3] = {16, 32, 64};
constexpr int kTileDefault = 1;
constexpr float kTileMargin = 0.97f;

struct SceneDesc {
  OpView op;
  const float* op_lo;
  const double* D64;
  int64_t row_off;     // first row of the scene in the concatenated vectors
  int64_t n;           // particles of the scene
  int32_t tile_begin, tile_end;
  double bb;           // ||b||^2 of the scene (all components)
  int32_t maxit;
  int32_t pad;
};

struct BatchCtrl {
  int32_t active;        // scenes progressing in the current pass
  int32_t need;          // scenes above rtol at the last residual
  int32_t error;         // a grid barrier timed out
  int32_t passes;
  unsigned int bar_count;
  unsigned int bar_gen;
};

struct BatchVecs {
  float4 *r, *rh, *p, *Ap, *rs, *As, *d, *x2;   // x2: x split hi, lo interleaved [2 rows]
  double *x64, *b64, *r64;
};

struct BatchView {
  const SceneDesc* sc;
  const int32_t* tile_scene;
  const int32_t* tile_slice0;
  const int32_t* tile_nsl;
  int32_t ntiles;
  int32_t nscenes;
  BatchVecs V;
  SolverScalars* S;            // [nscenes]
  double* partials;            // [ntiles][kMaxDots]
  unsigned int* scene_cnt;     // [nscenes] ticket counters
  double* rr64;                // [nscenes][3] true residual squares
  int32_t* total_iters;        // [nscenes]
  int32_t* passes;             // [nscenes]
  int32_t* stalled_any;        // [nscenes][3]
  BatchCtrl* ctrl;
  double rtol;
  double eps_floor;
};

namespace {

constexpr long long kBarrierSpins = 20000000;   // ~1-2 s of __nanosleep(64) before giving up

// Grid-wide barrier for the co-resident (cooperative) grid, with a bounded wait.
__device__ __forceinline__ bool grid_sync(BatchCtrl* ctrl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &ctrl->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&ctrl->bar_count, 1u) == gridDim.x - 1) {
      ctrl->bar_count = 0u;
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > kBarrierSpins || *(volatile int32_t*)&ctrl->error) {
          atomicExch(&ctrl->error, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int32_t*)&ctrl->error == 0;
}

// ticket of one tile of `scene`; true in every thread of the scene's last tile
__device__ __forceinline__ bool arrive_scene(unsigned int* cnt, int ntiles_scene) {
  __shared__ unsigned int ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
  __syncthreads();
  return ticket == (unsigned int)(ntiles_scene - 1);
}

// sum of the partials of tiles [b, e) -> res[0..K) (shared), counter re-armed
template <int K, int NB = kBlock>
__device__ __forceinline__ void scene_sum(const double* partials, int b, int e, unsigned int* cnt, double* res) {
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int t = b + threadIdx.x; t < e; t += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + (size_t)t * kMaxDots + k);
  }
  __shared__ double sm[NB / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    constexpr int P = K <= 1 ? 1 : (K <= 2 ? 2 : (K <= 4 ? 4 : (K <= 8 ? 8 : (K <= 16 ? 16 : 32))));
    int idx;
    const double x = warp_sum_multi<K>(acc, idx);
    if ((lane & (32 / P - 1)) == 0 && idx < K) sm[warp][idx] = x;
  }
  __syncthreads();
  cross_warp_sum<K, NB / 32>(sm, res);
  if (threadIdx.x == 0) *cnt = 0u;
  __syncthreads();
}

// rows of tile t handled by this thread: local rows first, first + blockDim.x, ... < end
__device__ __forceinline__ void tile_rows(const BatchView& B, int t, int64_t& first, int64_t& end) {
  first = (int64_t)B.tile_slice0[t] * kSlice + threadIdx.x;
  end = ((int64_t)B.tile_slice0[t] + B.tile_nsl[t]) * kSlice;
}

// ---- residual per scene (double-float pair sums) + which scenes need a pass --

__global__ void __launch_bounds__(kBlock) kb_split(BatchView B, int64_t nrows) {
  if (threadIdx.x == 0 && blockIdx.x == 0) B.ctrl->need = 0;   // counted by kb_residual
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nrows; s += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = B.V.x64[3 * s], x1 = B.V.x64[3 * s + 1], x2 = B.V.x64[3 * s + 2];
    const float h0 = (float)x0, h1 = (float)x1, h2 = (float)x2;
    B.V.x2[2 * s] = make_float4(h0, h1, h2, 0.f);
    B.V.x2[2 * s + 1] = make_float4((float)(x0 - (double)h0), (float)(x1 - (double)h1), (float)(x2 - (double)h2), 0.f);
  }
}

__global__ void __launch_bounds__(kBlock) kb_residual(BatchView B) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {   // counted by kb_init
    B.ctrl->active = 0;
    B.ctrl->passes += 1;
  }
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const int sc = B.tile_scene[t];
    const SceneDesc& d = B.sc[sc];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc2[3] = {0.0, 0.0, 0.0};
    for (int w = warp; w < B.tile_nsl[t]; w += kBlock / 32) {
      const int64_t sl = B.tile_slice0[t] + w;
      const int64_t s = sl * kSlice + lane;
      const OpView& op = d.op;
      const float4* x2 = B.V.x2 + 2 * d.row_off;
      const uint8_t k = op.kind[s];
      const float kap = (k == KIND_FLUID) ? 1.f : 0.f;
      DFAcc a0, a1, a2;
      residual_row_df(op, d.op_lo, x2, sl, lane, kap, a0, a1, a2);
      const double sg = (k == KIND_FLUID) ? 1.0 : (k == KIND_SHEPARD ? -1.0 : 0.0);
      const int64_t g = d.row_off + s;
      double r[3] = {0.0, 0.0, 0.0};
      if (s < d.n) {
        r[0] = B.V.b64[3 * g] - (B.V.x64[3 * g] + sg * a0.value());
        r[1] = B.V.b64[3 * g + 1] - (B.V.x64[3 * g + 1] + sg * a1.value());
        r[2] = B.V.b64[3 * g + 2] - (B.V.x64[3 * g + 2] + sg * a2.value());
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        B.V.r64[3 * g + q] = r[q];
        acc2[q] += r[q] * r[q];
      }
    }
    block_partials_f64<3>(acc2, B.partials + (size_t)t * kMaxDots);
    if (arrive_scene(B.scene_cnt + sc, d.tile_end - d.tile_begin)) {
      __shared__ double res[3];
      scene_sum<3>(B.partials, d.tile_begin, d.tile_end, B.scene_cnt + sc, res);
      if (threadIdx.x == 0) {
        double* rr = B.rr64 + 3 * sc;
        rr[0] = res[0];
        rr[1] = res[1];
        rr[2] = res[2];
        const double rn = sqrt(res[0] + res[1] + res[2]);
        if (!(rn <= B.rtol * sqrt(d.bb))) atomicAdd(&B.ctrl->need, 1);
      }
    }
  }
}

// pass start: for a scene still above rtol, r = r0^ = D^-1 r64 (float32), d = 0,
// gamma = r.r and tau^2 from eps = max(eps_floor, rtol |b| / (4 |r64|)); a scene
// already at rtol is marked done (frozen) for this pass.
__global__ void __launch_bounds__(kBlock) kb_init(BatchView B) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const int sc = B.tile_scene[t];
    const SceneDesc& d = B.sc[sc];
    const double* rr = B.rr64 + 3 * sc;
    const double rn = sqrt(rr[0] + rr[1] + rr[2]);
    const bool need = !(rn <= B.rtol * sqrt(d.bb));
    double acc[3] = {0.0, 0.0, 0.0};
    int64_t s0, s1;
    tile_rows(B, t, s0, s1);
    for (int64_t s = s0; s < s1; s += kBlock) {
      const int64_t g = d.row_off + s;
      float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
      if (need) {
        const double sc_ = 1.0 / d.D64[s];
        r = make_float4((float)(B.V.r64[3 * g] * sc_), (float)(B.V.r64[3 * g + 1] * sc_),
                        (float)(B.V.r64[3 * g + 2] * sc_), 0.f);
      }
      B.V.r[g] = r;
      B.V.rh[g] = r;
      B.V.d[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      acc[0] += (double)r.x * r.x;
      acc[1] += (double)r.y * r.y;
      acc[2] += (double)r.z * r.z;
    }
    block_partials_f64<3>(acc, B.partials + (size_t)t * kMaxDots);
    if (arrive_scene(B.scene_cnt + sc, d.tile_end - d.tile_begin)) {
      __shared__ double res[3];
      scene_sum<3>(B.partials, d.tile_begin, d.tile_end, B.scene_cnt + sc, res);
      if (threadIdx.x == 0) {
        SolverScalars* S = B.S + sc;
        const double eps = need ? fmax(B.eps_floor, 0.25 * B.rtol * sqrt(d.bb) / fmax(rn, 1e-300)) : 1.0;
        const int left = d.maxit - B.total_iters[sc];
        scal_init(S, res, eps * eps, left > 0 ? left : 0);
        if (!need || left <= 0) {
          for (int c = 0; c < 3; ++c)
            if (S->state[c] == SPH_PROGRESSING) S->state[c] = SPH_CONVERGED;
          S->done = 1;
        }
        if (need) B.passes[sc] += 1;
        if (!S->done) atomicAdd(&B.ctrl->active, 1);
      }
    }
  }
}

// One BiCGSTAB pass for every active scene: loops over iterations until no
// scene progresses, with a grid barrier between the phases of an iteration.
template <int U, bool PF, int NB>
__global__ void __launch_bounds__(NB) kb_pass(BatchView B, int iter_cap) {
  for (int it = 0; it < iter_cap; ++it) {
    if (*(volatile int32_t*)&B.ctrl->active == 0) break;
    // phase 1: p = r + beta p - alpha' Ap
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const int sc = B.tile_scene[t];
      const SolverScalars* S = B.S + sc;
      if (S->done) continue;
      const SceneDesc& d = B.sc[sc];
      const float b0 = (float)S->beta[0], b1 = (float)S->beta[1], b2 = (float)S->beta[2];
      const float a0 = (float)S->alpha_p[0], a1 = (float)S->alpha_p[1], a2 = (float)S->alpha_p[2];
      const bool useP = b0 != 0.f || b1 != 0.f || b2 != 0.f, useA = a0 != 0.f || a1 != 0.f || a2 != 0.f;
      int64_t s0, s1;
      tile_rows(B, t, s0, s1);
      for (int64_t s = s0; s < s1; s += NB) {
        const int64_t g = d.row_off + s;
        float4 p = B.V.r[g];
        if (useP) {
          const float4 q = B.V.p[g];
          p.x = fmaf(b0, q.x, p.x);
          p.y = fmaf(b1, q.y, p.y);
          p.z = fmaf(b2, q.z, p.z);
        }
        if (useA) {
          const float4 q = B.V.Ap[g];
          p.x = fmaf(-a0, q.x, p.x);
          p.y = fmaf(-a1, q.y, p.y);
          p.z = fmaf(-a2, q.z, p.z);
        }
        p.w = 0.f;
        B.V.p[g] = p;
      }
    }
    if (!grid_sync(B.ctrl)) return;
    // phase 2: Ap = D^-1 A p; delta = r0^.Ap per scene
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const int sc = B.tile_scene[t];
      SolverScalars* S = B.S + sc;
      if (S->done) continue;
      const SceneDesc& d = B.sc[sc];
      float acc[3] = {0.f, 0.f, 0.f};
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int w = warp; w < B.tile_nsl[t]; w += NB / 32) {
        const int64_t sl = B.tile_slice0[t] + w;
        float4 vb;
        const float4 o = apply_row<U, PF, true>(d.op, B.V.p + d.row_off, sl, lane, vb);
        const int64_t g = d.row_off + sl * kSlice + lane;
        B.V.Ap[g] = o;
        const float4 h = B.V.rh[g];
        acc[0] = fmaf(h.x, o.x, acc[0]);
        acc[1] = fmaf(h.y, o.y, acc[1]);
        acc[2] = fmaf(h.z, o.z, acc[2]);
      }
      block_partials<3, NB>(acc, B.partials + (size_t)t * kMaxDots);
      if (arrive_scene(B.scene_cnt + sc, d.tile_end - d.tile_begin)) {
        __shared__ double res[3];
        scene_sum<3, NB>(B.partials, d.tile_begin, d.tile_end, B.scene_cnt + sc, res);
        if (threadIdx.x < 32) scal_after_delta_w(S, res);
      }
    }
    if (!grid_sync(B.ctrl)) return;
    // phase 3: r* = r - alpha Ap
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const int sc = B.tile_scene[t];
      const SolverScalars* S = B.S + sc;
      if (S->done) continue;
      const SceneDesc& d = B.sc[sc];
      const float a0 = (float)S->alpha[0], a1 = (float)S->alpha[1], a2 = (float)S->alpha[2];
      int64_t s0, s1;
      tile_rows(B, t, s0, s1);
      for (int64_t s = s0; s < s1; s += NB) {
        const int64_t g = d.row_off + s;
        const float4 r = B.V.r[g], ap = B.V.Ap[g];
        B.V.rs[g] = make_float4(fmaf(-a0, ap.x, r.x), fmaf(-a1, ap.y, r.y), fmaf(-a2, ap.z, r.z), 0.f);
      }
    }
    if (!grid_sync(B.ctrl)) return;
    // phase 4: Ar* and omega = (r*.Ar*) / (Ar*.Ar*) per scene
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const int sc = B.tile_scene[t];
      SolverScalars* S = B.S + sc;
      if (S->done) continue;
      const SceneDesc& d = B.sc[sc];
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int w = warp; w < B.tile_nsl[t]; w += NB / 32) {
        const int64_t sl = B.tile_slice0[t] + w;
        float4 vb;
        const float4 o = apply_row<U, PF, true>(d.op, B.V.rs + d.row_off, sl, lane, vb);
        const int64_t g = d.row_off + sl * kSlice + lane;
        B.V.As[g] = o;
        acc[0] = fmaf(vb.x, o.x, acc[0]);
        acc[1] = fmaf(vb.y, o.y, acc[1]);
        acc[2] = fmaf(vb.z, o.z, acc[2]);
        acc[3] = fmaf(o.x, o.x, acc[3]);
        acc[4] = fmaf(o.y, o.y, acc[4]);
        acc[5] = fmaf(o.z, o.z, acc[5]);
      }
      block_partials<6, NB>(acc, B.partials + (size_t)t * kMaxDots);
      if (arrive_scene(B.scene_cnt + sc, d.tile_end - d.tile_begin)) {
        __shared__ double res[6];
        scene_sum<6, NB>(B.partials, d.tile_begin, d.tile_end, B.scene_cnt + sc, res);
        if (threadIdx.x < 32) scal_after_omega_w(S, res);
      }
    }
    if (!grid_sync(B.ctrl)) return;
    // phase 5: r = r* - omega Ar*; d += alpha p + omega r*; gamma' = r0^.r, r.r; states
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
      const int sc = B.tile_scene[t];
      SolverScalars* S = B.S + sc;
      if (S->done) continue;
      const SceneDesc& d = B.sc[sc];
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float w0 = (float)S->omega[0], w1 = (float)S->omega[1], w2 = (float)S->omega[2];
      const float l0 = (float)S->alpha[0], l1 = (float)S->alpha[1], l2 = (float)S->alpha[2];
      int64_t s0, s1;
      tile_rows(B, t, s0, s1);
      for (int64_t s = s0; s < s1; s += NB) {
        const int64_t g = d.row_off + s;
        const float4 rs = B.V.rs[g], as = B.V.As[g], h = B.V.rh[g], p = B.V.p[g];
        float4 dd = B.V.d[g];
        const float4 r = make_float4(fmaf(-w0, as.x, rs.x), fmaf(-w1, as.y, rs.y), fmaf(-w2, as.z, rs.z), 0.f);
        dd.x = fmaf(w0, rs.x, fmaf(l0, p.x, dd.x));
        dd.y = fmaf(w1, rs.y, fmaf(l1, p.y, dd.y));
        dd.z = fmaf(w2, rs.z, fmaf(l2, p.z, dd.z));
        B.V.r[g] = r;
        B.V.d[g] = dd;
        acc[0] = fmaf(h.x, r.x, acc[0]);
        acc[1] = fmaf(h.y, r.y, acc[1]);
        acc[2] = fmaf(h.z, r.z, acc[2]);
        acc[3] = fmaf(r.x, r.x, acc[3]);
        acc[4] = fmaf(r.y, r.y, acc[4]);
        acc[5] = fmaf(r.z, r.z, acc[5]);
      }
      block_partials<6, NB>(acc, B.partials + (size_t)t * kMaxDots);
      if (arrive_scene(B.scene_cnt + sc, d.tile_end - d.tile_begin)) {
        __shared__ double res[6];
        scene_sum<6, NB>(B.partials, d.tile_begin, d.tile_end, B.scene_cnt + sc, res);
        if (threadIdx.x < 32) scal_after_update_w(S, res, res + 3);
        __syncwarp();
        if (threadIdx.x == 0) {
          B.total_iters[sc] += 1;
          for (int c = 0; c < 3; ++c)
            if (S->stalled_any[c]) B.stalled_any[3 * sc + c] = 1;
          if (S->done) atomicSub(&B.ctrl->active, 1);
        }
      }
    }
    if (!grid_sync(B.ctrl)) return;
  }
}

__global__ void __launch_bounds__(kBlock) kb_add(BatchView B, int64_t nrows) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nrows; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = B.V.d[s];
    B.V.x64[3 * s] += (double)v.x;
    B.V.x64[3 * s + 1] += (double)v.y;
    B.V.x64[3 * s + 2] += (double)v.z;
  }
}

// the whole solve as one graph: after each pass, keep looping while some scene was
// above rtol at the pass's residual, no barrier timed out and passes remain
__global__ void kb_loop_ctrl(const BatchCtrl* __restrict__ ctrl, cudaGraphConditionalHandle h, int max_passes) {
  const bool more = ctrl->error == 0 && ctrl->need > 0 && ctrl->passes < max_passes;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void kb_gather(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                          double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * s + k] = (s < n) ? src[3 * (int64_t)perm[s] + k] : 0.0;
  }
}

__global__ void kb_scatter(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                           double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * (int64_t)perm[s] + k] = src[3 * s + k];
  }
}

__global__ void kb_norm2(const double* __restrict__ b, int64_t n_pad, double* out) {
  // one block per scene (b points at the scene's rows); float64 squares per component
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] = fma(b[3 * i + k], b[3 * i + k], acc[k]);
  }
  __shared__ double sm[kBlock / 32][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sm[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// variants 0..7: row-loop form (v & 3: (U, PF) = (8,0), (4,0), (8,1), (4,1)) and
// block size (v >> 2: 256 or 128 threads, 8 or 4 warps per 32-slice tile)
constexpr int kPassVariants = 8;
using PassFn = void (*)(BatchView, int);
PassFn pass_kernel(int variant) {
  switch (variant) {
    case 1: return kb_pass<4, false, 256>;
    case 2: return kb_pass<8, true, 256>;
    case 3: return kb_pass<4, true, 256>;
    case 4: return kb_pass<8, false, 128>;
    case 5: return kb_pass<4, false, 128>;
    case 6: return kb_pass<8, true, 128>;
    case 7: return kb_pass<4, true, 128>;
    default: return kb_pass<8, false, 256>;
  }
}
int pass_block(int variant) { return (variant >> 2) == 1 ? 128 : 256; }

}  // namespace

}  // namespace sph

using namespace sph;

struct sph_batch {
  int nscenes = 0;
  std::vector<sph_neighbors*> handles;
  std::vector<sph_visc_params> params;
  std::vector<int64_t> row_off;
  std::vector<uint64_t> rs_version;   // each handle's row-scale version at creation
  int64_t nrows = 0;
  int32_t ntiles = 0;
  int device = 0, num_sms = 0;
  DBuf<SceneDesc> desc;
  DBuf<int32_t> tile_scene, tile_slice0, tile_nsl;
  DBuf<float4> vec;            // 9 float4 vectors back to back
  DBuf<double> dvec;           // x64, b64, r64
  DBuf<SolverScalars> S;
  DBuf<double> partials, rr64;
  DBuf<unsigned int> scene_cnt;
  DBuf<int32_t> iters, passes, stalled;
  DBuf<BatchCtrl> ctrl;
  BatchCtrl* host_ctrl = nullptr;
  int variant = -1;            // autotuned form (row loop, block size) of the persistent kernel
  int grid = 0;                // grid of the auxiliary kernels
  int grids[kPassVariants] = {};   // co-resident grid of each persistent-kernel variant
  int occ[kPassVariants] = {};     // resident blocks per SM of each variant
  float tune_ms[kPassVariants] = {};
  int tile = kTileDefault;     // index into kTileCands
  bool tile_fixed = false;     // set by sph_batch_set_tile: the tuner keeps it
  float tile_ms[3] = {};       // tuning time of the chosen variant at each tile length
  std::vector<SceneDesc> hdesc;   // host copy of the scene descriptors
  cudaGraphExec_t graph = nullptr;
  bool graph_ok = false;
  double graph_rtol = -1.0, graph_eps = -1.0;
  int graph_cap = 0;
  // every pass of a solve in one graph launch: the pass inside a conditional WHILE node
  cudaGraphExec_t solve_graph = nullptr;
  bool solve_graph_tried = false;
  int solve_graph_passes = 0;
};

namespace {

BatchView batch_view(sph_batch* Bt, double rtol, double eps) {
  BatchView B{};
  B.sc = Bt->desc.p;
  B.tile_scene = Bt->tile_scene.p;
  B.tile_slice0 = Bt->tile_slice0.p;
  B.tile_nsl = Bt->tile_nsl.p;
  B.ntiles = Bt->ntiles;
  B.nscenes = Bt->nscenes;
  float4* v = Bt->vec.p;
  const int64_t N = Bt->nrows;
  B.V = BatchVecs{v, v + N, v + 2 * N, v + 3 * N, v + 4 * N, v + 5 * N, v + 6 * N, v + 7 * N,
                  Bt->dvec.p, Bt->dvec.p + 3 * N, Bt->dvec.p + 6 * N};
  B.S = Bt->S.p;
  B.partials = Bt->partials.p;
  B.scene_cnt = Bt->scene_cnt.p;
  B.rr64 = Bt->rr64.p;
  B.total_iters = Bt->iters.p;
  B.passes = Bt->passes.p;
  B.stalled_any = Bt->stalled.p;
  B.ctrl = Bt->ctrl.p;
  B.rtol = rtol;
  B.eps_floor = eps;
  return B;
}

sph_status launch_pass(sph_batch* Bt, const BatchView& B, int cap, cudaStream_t st) {
  const PassFn kern = pass_kernel(Bt->variant < 0 ? 0 : Bt->variant);
  BatchView bv = B;
  int c = cap;
  void* args[] = {&bv, &c};
  cudaLaunchConfig_t cfg{};
  const int var = Bt->variant < 0 ? 0 : Bt->variant;
  cfg.gridDim = dim3(Bt->grids[var]);
  cfg.blockDim = dim3(pass_block(var));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  SPH_TRY_CUDA(cudaLaunchKernelExC(&cfg, (const void*)kern, args));
  return SPH_OK;
}

// the four launches of one refinement pass
sph_status enqueue_pass(sph_batch* Bt, const BatchView& B, int cap, cudaStream_t st) {
  const int g = Bt->grid;
  SPH_LAUNCH(kb_split, g, kBlock, 0, st)(B, Bt->nrows);
  SPH_LAUNCH(kb_residual, g, kBlock, 0, st)(B);
  SPH_LAUNCH(kb_init, g, kBlock, 0, st)(B);
  SPH_TRY(launch_pass(Bt, B, cap, st));
  SPH_LAUNCH(kb_add, g, kBlock, 0, st)(B, Bt->nrows);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

// Cuts every scene into tiles of kTileCands[ti] slices (the last one of a scene
// shorter), uploads the tile table and the descriptors' tile ranges, and sizes
// each variant's co-resident grid.  The device arrays hold the tiles of the
// shortest candidate.
sph_status build_tiles(sph_batch* Bt, int ti, cudaStream_t st) {
  const int64_t T = kTileCands[ti];
  std::vector<int32_t> ts, t0, tn;
  for (int s = 0; s < Bt->nscenes; ++s) {
    const sph_neighbors* H = Bt->handles[s];
    SceneDesc& d = Bt->hdesc[s];
    d.tile_begin = (int32_t)ts.size();
    for (int64_t sl = 0; sl < H->nslices; sl += T) {
      ts.push_back(s);
      t0.push_back((int32_t)sl);
      tn.push_back((int32_t)((H->nslices - sl) < T ? (H->nslices - sl) : T));
    }
    d.tile_end = (int32_t)ts.size();
  }
  if ((int64_t)ts.size() > (int64_t)Bt->tile_scene.n) {
    set_error("sph_batch: tile table larger than its allocation");
    return SPH_ERR_INVALID;
  }
  Bt->ntiles = (int32_t)ts.size();
  Bt->tile = ti;
  SPH_TRY_CUDA(cudaMemcpyAsync(Bt->tile_scene.p, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(Bt->tile_slice0.p, t0.data(), t0.size() * 4, cudaMemcpyHostToDevice, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(Bt->tile_nsl.p, tn.data(), tn.size() * 4, cudaMemcpyHostToDevice, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(Bt->desc.p, Bt->hdesc.data(), Bt->nscenes * sizeof(SceneDesc), cudaMemcpyHostToDevice,
                               st));
  // pageable sources: the copies above complete before the host vectors go
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  for (int v = 0; v < kPassVariants; ++v) {
    int g = Bt->num_sms * (Bt->occ[v] > 0 ? Bt->occ[v] : 1);
    if (g > Bt->ntiles) g = Bt->ntiles;
    Bt->grids[v] = g;
  }
  Bt->grid = Bt->grids[0];
  return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_batch_create(sph_neighbors* const* handles, const sph_visc_params* params, int32_t nscenes,
                            sph_batch** out, void* stream) {
  clear_error();
  if (!handles || !params || !out || nscenes < 1) {
    set_error("sph_batch_create: need nscenes >= 1 handles and parameter sets");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  sph_batch* Bt = new sph_batch();
  auto fail = [&](sph_status s) {
    sph_batch_destroy(Bt);
    *out = nullptr;
    return s;
  };
  Bt->nscenes = nscenes;
  Bt->hdesc.assign(nscenes, SceneDesc{});
  int64_t rows = 0, max_tiles = 0;
  for (int s = 0; s < nscenes; ++s) {
    sph_neighbors* H = handles[s];
    if (!H) {
      set_error("sph_batch_create: handle %d is null", s);
      return fail(SPH_ERR_INVALID);
    }
    sph_status e = ensure_operator(H, &params[s], st);
    if (e == SPH_OK) e = row_scale_refresh(H, st);
    if (e != SPH_OK) return fail(e);
    Bt->handles.push_back(H);
    Bt->params.push_back(params[s]);
    Bt->row_off.push_back(rows);
    Bt->rs_version.push_back(H->rs_version);
    SceneDesc& d = Bt->hdesc[s];
    d.op = op_view(H);
    d.op_lo = H->op_lo.p;
    d.D64 = H->D64.p;
    if (H->row_scaled) {  // the preconditioner's diagonal D / s
      d.op.invD = H->invD_sc.p;
      d.D64 = H->D64_sc.p;
    }
    d.row_off = rows;
    d.n = H->n;
    max_tiles += (H->nslices + kTileCands[0] - 1) / kTileCands[0];
    rows += H->n_pad;
  }
  Bt->nrows = rows;
  if (cudaGetDevice(&Bt->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&Bt->num_sms, cudaDevAttrMultiProcessorCount, Bt->device) != cudaSuccess) {
    set_error("sph_batch_create: no CUDA device");
    return fail(SPH_ERR_CUDA);
  }
#define BTRY(x)                      \
  do {                               \
    sph_status s_ = (x);             \
    if (s_ != SPH_OK) return fail(s_); \
  } while (0)
  BTRY(Bt->desc.alloc(nscenes));
  BTRY(Bt->tile_scene.alloc(max_tiles));
  BTRY(Bt->tile_slice0.alloc(max_tiles));
  BTRY(Bt->tile_nsl.alloc(max_tiles));
  BTRY(Bt->vec.alloc(9 * rows));
  BTRY(Bt->dvec.alloc(12 * rows));   // x64, b64, r64, saved x0
  BTRY(Bt->S.alloc(nscenes));
  BTRY(Bt->partials.alloc((size_t)max_tiles * kMaxDots));
  BTRY(Bt->rr64.alloc(3 * nscenes));
  BTRY(Bt->scene_cnt.alloc(nscenes));
  BTRY(Bt->iters.alloc(nscenes));
  BTRY(Bt->passes.alloc(nscenes));
  BTRY(Bt->stalled.alloc(3 * nscenes));
  BTRY(Bt->ctrl.alloc(1));
  if (cudaMallocHost(reinterpret_cast<void**>(&Bt->host_ctrl), sizeof(BatchCtrl)) != cudaSuccess) {
    set_error("sph_batch_create: pinned allocation failed");
    return fail(SPH_ERR_NOMEM);
  }
  if (cudaMemsetAsync(Bt->scene_cnt.p, 0, nscenes * sizeof(unsigned int), st) != cudaSuccess ||
      cudaMemsetAsync(Bt->ctrl.p, 0, sizeof(BatchCtrl), st) != cudaSuccess) {
    set_error("sph_batch_create: upload failed");
    return fail(SPH_ERR_CUDA);
  }
  // grid of each cooperative variant: every block resident at once
  for (int v = 0; v < kPassVariants; ++v) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, (const void*)pass_kernel(v), pass_block(v), 0);
    Bt->occ[v] = o;
  }
  BTRY(build_tiles(Bt, kTileDefault, st));
  *out = Bt;
  return SPH_OK;
#undef BTRY
}

sph_status sph_batch_destroy(sph_batch* Bt) {
  if (!Bt) return SPH_OK;
  if (Bt->graph) cudaGraphExecDestroy(Bt->graph);
  if (Bt->solve_graph) cudaGraphExecDestroy(Bt->solve_graph);
  Bt->desc.release();
  Bt->tile_scene.release();
  Bt->tile_slice0.release();
  Bt->tile_nsl.release();
  Bt->vec.release();
  Bt->dvec.release();
  Bt->S.release();
  Bt->partials.release();
  Bt->rr64.release();
  Bt->scene_cnt.release();
  Bt->iters.release();
  Bt->passes.release();
  Bt->stalled.release();
  Bt->ctrl.release();
  if (Bt->host_ctrl) cudaFreeHost(Bt->host_ctrl);
  delete Bt;
  return SPH_OK;
}

sph_status sph_batch_solve(sph_batch* Bt, const sph_solve_opts* O, const double* const* b, double* const* x,
                           sph_solve_report* reports, void* stream) {
  clear_error();
  if (!Bt || !O || !b || !x || !reports) {
    set_error("sph_batch_solve: null argument");
    return SPH_ERR_INVALID;
  }
  if (O->precision != SPH_PREC_MIXED) {
    set_error("sph_batch_solve: only SPH_PREC_MIXED is batched");
    return SPH_ERR_INVALID;
  }
  if (O->method != SPH_SOLVER_BICGSTAB || !O->jacobi) {
    set_error("sph_batch_solve: the batch runs the Jacobi-scaled BiCGSTAB (method 0, jacobi 1)");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double rtol = O->rtol > 0.0 ? O->rtol : 1e-6;
  const double eps = O->eps_inner > 0.0 ? O->eps_inner : 2e-2;
  const int maxit = O->maxit > 0 ? O->maxit : 10000;
  const int max_ref = O->max_refine > 0 ? O->max_refine : 30;
  const int S = Bt->nscenes;
  const int64_t N = Bt->nrows;
  for (int s = 0; s < S; ++s) {
    if (!b[s] || !x[s]) {
      set_error("sph_batch_solve: b/x of scene %d is null", s);
      return SPH_ERR_INVALID;
    }
    sph_neighbors* H = Bt->handles[s];
    // the operator may have been rebuilt since the batch was made
    if (!H->op_valid || H->op_mu_version != H->mu_version || H->rs_version != Bt->rs_version[s] ||
        (H->row_scaled && H->rs_op_version != H->op_version)) {
      set_error("sph_batch_solve: scene %d's handle changed after sph_batch_create", s);
      return SPH_ERR_INVALID;
    }
    const int64_t o = Bt->row_off[s];
    SPH_LAUNCH(kb_gather, grid_for(H, H->n_pad), kBlock, 0, st)(b[s], H->perm.p, H->n, H->n_pad,
                                                                  Bt->dvec.p + 3 * N + 3 * o);
    SPH_LAUNCH(kb_gather, grid_for(H, H->n_pad), kBlock, 0, st)(x[s], H->perm.p, H->n, H->n_pad, Bt->dvec.p + 3 * o);
    SPH_LAUNCH(kb_norm2, 1, kBlock, 0, st)(Bt->dvec.p + 3 * N + 3 * o, H->n_pad, Bt->rr64.p + 3 * s);
  }
  SPH_TRY_CUDA(cudaGetLastError());
  // per-scene ||b||^2 into the descriptors, counters and reports cleared
  std::vector<double> rr(3 * S);
  SPH_TRY_CUDA(cudaMemcpyAsync(rr.data(), Bt->rr64.p, 3 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  std::vector<double> bb(S), bbc(3 * S);
  for (int s = 0; s < S; ++s) {
    for (int c = 0; c < 3; ++c) bbc[3 * s + c] = rr[3 * s + c];
    bb[s] = rr[3 * s] + rr[3 * s + 1] + rr[3 * s + 2];
    Bt->hdesc[s].bb = bb[s];
    Bt->hdesc[s].maxit = maxit;
  }
  SPH_TRY_CUDA(cudaMemcpyAsync(Bt->desc.p, Bt->hdesc.data(), S * sizeof(SceneDesc), cudaMemcpyHostToDevice, st));
  // pageable source: complete before the host copy can change
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  SPH_TRY_CUDA(cudaMemsetAsync(Bt->iters.p, 0, S * sizeof(int32_t), st));
  SPH_TRY_CUDA(cudaMemsetAsync(Bt->passes.p, 0, S * sizeof(int32_t), st));
  SPH_TRY_CUDA(cudaMemsetAsync(Bt->stalled.p, 0, 3 * S * sizeof(int32_t), st));
  SPH_TRY_CUDA(cudaMemsetAsync(Bt->ctrl.p, 0, sizeof(BatchCtrl), st));
  BatchView B = batch_view(Bt, rtol, eps);
  const int cap = maxit;

  // autotune the persistent kernel once: first its row-loop form and block size
  // at the default tile length, then the tile length for that variant; each
  // candidate runs one pass of at most 16 iterations from the same start, timed
  // with events, and the fastest is kept
  if (Bt->variant < 0) {
    cudaEvent_t e0, e1;
    SPH_TRY_CUDA(cudaEventCreate(&e0));
    SPH_TRY_CUDA(cudaEventCreate(&e1));
    double* x0save = Bt->dvec.p + 9 * N;
    SPH_TRY_CUDA(cudaMemcpyAsync(x0save, Bt->dvec.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    auto time_pass = [&](float& ms) -> sph_status {
      SPH_TRY_CUDA(cudaMemcpyAsync(Bt->dvec.p, x0save, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
      SPH_TRY_CUDA(cudaMemsetAsync(Bt->iters.p, 0, S * sizeof(int32_t), st));
      SPH_TRY_CUDA(cudaMemsetAsync(Bt->ctrl.p, 0, sizeof(BatchCtrl), st));
      SPH_TRY_CUDA(cudaEventRecord(e0, st));
      SPH_TRY(enqueue_pass(Bt, B, 16, st));
      SPH_TRY_CUDA(cudaEventRecord(e1, st));
      SPH_TRY_CUDA(cudaEventSynchronize(e1));
      ms = 0.f;
      SPH_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      SPH_TRY_CUDA(cudaMemcpy(Bt->host_ctrl, Bt->ctrl.p, sizeof(BatchCtrl), cudaMemcpyDeviceToHost));
      if (Bt->host_ctrl->error) {
        set_error("sph_batch_solve: a grid barrier timed out (autotune)");
        return SPH_ERR_TIMEOUT;
      }
      return SPH_OK;
    };
    sph_status ts = SPH_OK;
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < kPassVariants && ts == SPH_OK; ++v) {
      Bt->variant = v;
      float ms = 0.f;
      ts = time_pass(ms);
      Bt->tune_ms[v] = ms;
      if (ms < best) {
        best = ms;
        bestv = v;
      }
    }
    Bt->variant = bestv;
    int bestt = Bt->tile;
    for (int ti = 0; ti < 3 && ts == SPH_OK && !Bt->tile_fixed; ++ti) {
      if (ti == kTileDefault) {
        Bt->tile_ms[ti] = best;
        continue;
      }
      ts = build_tiles(Bt, ti, st);
      if (ts != SPH_OK) break;
      B = batch_view(Bt, rtol, eps);
      float ms = 0.f;
      ts = time_pass(ms);
      Bt->tile_ms[ti] = ms;
      // the tuning pass has every scene active; a whole solve ends with a few
      // large scenes alone, where long tiles leave blocks idle: leave the
      // default only for a clear gain
      if (ms < kTileMargin * best) {
        best = ms;
        bestt = ti;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ts != SPH_OK) {
      Bt->variant = -1;
      return ts;
    }
    SPH_TRY(build_tiles(Bt, bestt, st));
    B = batch_view(Bt, rtol, eps);
    // restore x0 and the reports
    SPH_TRY_CUDA(cudaMemcpyAsync(Bt->dvec.p, x0save, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SPH_TRY_CUDA(cudaMemsetAsync(Bt->iters.p, 0, S * sizeof(int32_t), st));
    SPH_TRY_CUDA(cudaMemsetAsync(Bt->passes.p, 0, S * sizeof(int32_t), st));
    SPH_TRY_CUDA(cudaMemsetAsync(Bt->stalled.p, 0, 3 * S * sizeof(int32_t), st));
    SPH_TRY_CUDA(cudaMemsetAsync(Bt->ctrl.p, 0, sizeof(BatchCtrl), st));
  }

  // capture one refinement pass in a graph (rebuilt when rtol/eps/cap change), and the
  // whole solve as that pass inside a conditional WHILE node
  if (!Bt->graph || Bt->graph_rtol != rtol || Bt->graph_eps != eps || Bt->graph_cap != cap ||
      Bt->solve_graph_passes != max_ref + 2) {
    if (Bt->solve_graph) {
      cudaGraphExecDestroy(Bt->solve_graph);
      Bt->solve_graph = nullptr;
    }
    Bt->solve_graph_tried = false;
    Bt->solve_graph_passes = max_ref + 2;
    if (Bt->graph) {
      cudaGraphExecDestroy(Bt->graph);
      Bt->graph = nullptr;
    }
    Bt->graph_ok = false;
    cudaStream_t cs;
    SPH_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) ok = enqueue_pass(Bt, B, cap, cs) == SPH_OK;
    ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok && g;
    if (ok) ok = cudaGraphInstantiate(&Bt->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    Bt->graph_ok = ok;
    if (!ok) Bt->graph = nullptr;
    Bt->graph_rtol = rtol;
    Bt->graph_eps = eps;
    Bt->graph_cap = cap;
  }

  if (!Bt->solve_graph_tried) {
    Bt->solve_graph_tried = true;
    cudaStream_t cs;
    SPH_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h{};
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    if (ok) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
      if (ok) {
        ok = enqueue_pass(Bt, B, cap, cs) == SPH_OK;
        kb_loop_ctrl<<<1, 1, 0, cs>>>(Bt->ctrl.p, h, max_ref + 2);
        ok = cudaGetLastError() == cudaSuccess && ok;
        cudaGraph_t captured = nullptr;
        ok = cudaStreamEndCapture(cs, &captured) == cudaSuccess && ok;
      }
    }
    if (ok) ok = cudaGraphInstantiate(&Bt->solve_graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!ok) Bt->solve_graph = nullptr;
  }

  sph_status status = SPH_NOT_CONVERGED;
  if (Bt->solve_graph) {
    SPH_TRY_CUDA(cudaGraphLaunch(Bt->solve_graph, st));
    SPH_TRY_CUDA(cudaMemcpyAsync(Bt->host_ctrl, Bt->ctrl.p, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    note_launches(6 * Bt->host_ctrl->passes);   // per pass: the five pass kernels and the loop test
    if (Bt->host_ctrl->error) {
      set_error("sph_batch_solve: a grid barrier timed out");
      return SPH_ERR_TIMEOUT;
    }
    if (Bt->host_ctrl->need == 0) status = SPH_OK;
  }
  for (int ref = 0; ref <= max_ref + 1 && !Bt->solve_graph; ++ref) {
    if (Bt->graph_ok) {
      SPH_TRY_CUDA(cudaGraphLaunch(Bt->graph, st));
      note_launches(5);   // kb_split, kb_residual, kb_init, kb_pass, kb_add
    } else {
      SPH_TRY(enqueue_pass(Bt, B, cap, st));
    }
    SPH_TRY_CUDA(cudaMemcpyAsync(Bt->host_ctrl, Bt->ctrl.p, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    if (Bt->host_ctrl->error) {
      set_error("sph_batch_solve: a grid barrier timed out");
      return SPH_ERR_TIMEOUT;
    }
    if (Bt->host_ctrl->need == 0) {   // every scene was at rtol before this pass
      status = SPH_OK;
      break;
    }
  }
  // reports
  std::vector<int32_t> its(S), pas(S), stl(3 * S);
  std::vector<SolverScalars> hs(S);
  SPH_TRY_CUDA(cudaMemcpyAsync(rr.data(), Bt->rr64.p, 3 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(its.data(), Bt->iters.p, S * 4, cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(pas.data(), Bt->passes.p, S * 4, cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(stl.data(), Bt->stalled.p, 3 * S * 4, cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(hs.data(), Bt->S.p, S * sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
  for (int s = 0; s < S; ++s) {
    sph_neighbors* H = Bt->handles[s];
    SPH_LAUNCH(kb_scatter, grid_for(H, H->n), kBlock, 0, st)(Bt->dvec.p + 3 * Bt->row_off[s], H->perm.p, H->n, x[s]);
  }
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  for (int s = 0; s < S; ++s) {
    sph_solve_report& R = reports[s];
    std::memset(&R, 0, sizeof(R));
    const double rn = std::sqrt(rr[3 * s] + rr[3 * s + 1] + rr[3 * s + 2]);
    const double bn = std::sqrt(bb[s]);
    R.iters = its[s];
    R.refinements = pas[s];
    R.true_rel_res = bn > 0.0 ? rn / bn : rn;
    for (int c = 0; c < 3; ++c) {
      R.state[c] = (int8_t)hs[s].state[c];
      R.stalled_any[c] = (int8_t)stl[3 * s + c];
      R.true_rel_res_c[c] = bbc[3 * s + c] > 0.0 ? std::sqrt(rr[3 * s + c] / bbc[3 * s + c]) : std::sqrt(rr[3 * s + c]);
    }
    R.status = (R.true_rel_res <= rtol) ? SPH_OK : SPH_NOT_CONVERGED;
    if (R.status != SPH_OK) status = SPH_NOT_CONVERGED;
  }
  if (status == SPH_NOT_CONVERGED) set_error("sph_batch_solve: some scenes stayed above rtol");
  return status;
}

sph_status sph_batch_info(const sph_batch* Bt, int32_t* variant, int32_t* graph, float* tune_ms4, int32_t* grid) {
  clear_error();
  if (!Bt) {
    set_error("sph_batch_info: null batch");
    return SPH_ERR_INVALID;
  }
  if (variant) *variant = Bt->variant;
  if (graph) *graph = Bt->solve_graph ? 2 : (Bt->graph_ok ? 1 : 0);
  if (grid) *grid = Bt->grids[Bt->variant < 0 ? 0 : Bt->variant];
  if (tune_ms4)
    for (int v = 0; v < kPassVariants; ++v) tune_ms4[v] = Bt->tune_ms[v];
  return SPH_OK;
}

sph_status sph_batch_set_tile(sph_batch* Bt, int32_t tile_slices, void* stream) {
  clear_error();
  if (!Bt) {
    set_error("sph_batch_set_tile: null batch");
    return SPH_ERR_INVALID;
  }
  int ti = -1;
  for (int i = 0; i < 3; ++i)
    if (kTileCands[i] == tile_slices) ti = i;
  if (ti < 0) {
    set_error("sph_batch_set_tile: tile length %d is not one of %d, %d, %d", tile_slices, kTileCands[0],
              kTileCands[1], kTileCands[2]);
    return SPH_ERR_INVALID;
  }
  SPH_TRY(build_tiles(Bt, ti, reinterpret_cast<cudaStream_t>(stream)));
  Bt->tile_fixed = true;
  if (Bt->graph) {   // the captured pass holds the old tile count
    cudaGraphExecDestroy(Bt->graph);
    Bt->graph = nullptr;
    Bt->graph_ok = false;
  }
  if (Bt->solve_graph) {
    cudaGraphExecDestroy(Bt->solve_graph);
    Bt->solve_graph = nullptr;
  }
  Bt->solve_graph_tried = false;
  return SPH_OK;
}

sph_status sph_batch_tiles(const sph_batch* Bt, int32_t* tile_slices, int32_t* ntiles, int32_t* candidates,
                           float* tune_ms) {
  clear_error();
  if (!Bt) {
    set_error("sph_batch_tiles: null batch");
    return SPH_ERR_INVALID;
  }
  if (tile_slices) *tile_slices = kTileCands[Bt->tile];
  if (ntiles) *ntiles = Bt->ntiles;
  for (int i = 0; i < 3; ++i) {
    if (candidates) candidates[i] = kTileCands[i];
    if (tune_ms) tune_ms[i] = Bt->tile_ms[i];
  }
  return SPH_OK;
}

}  // extern "C"
