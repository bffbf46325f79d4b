// Restructured BiCGSTAB (paper Sec. 4.2) with the per-component stopping logic,
// run as float32 passes inside float64 iterative refinement.
//
// One inner pass solves (D^-1 A) d = D^-1 r64 for the three components at once.
// Iteration i (restructured listing of Sec. 4.2):
//   p     = r + beta p - alpha' A p           (a zero coefficient skips its vector)
//   delta = r0^ . A p ;  alpha = gamma / delta
//   r*    = r - alpha A p ;  d += alpha p   (applied in the x/r update kernel)
//   omega = (r* . A r*) / (A r* . A r*)
//   r     = r* - omega A r* ;  d += omega r*
//   gamma' = r0^ . r ;  alpha' = gamma' / delta ;  beta = alpha' / omega
// delta = 0 (or non-finite) sets alpha = alpha' = beta = 0 and marks the
// component stalled; the iteration still completes; the pass stops when no
// component is progressing (converged: r.r < tau^2; stalled) -- one exit point.
// A component that is no longer progressing is frozen (alpha = omega = 0).
//
// Kernels of one iteration (each grid-wide dot goes through the last-block
// reduction of reduce.cuh, so no extra launch and no host round trip):
//   paper-exact (merged_reductions = 0):
//     k_p_update, k_apply_dot<DELTA>, k_rstar, k_apply_dot<OMEGA>, k_xr_update(+gamma', r.r)
//   merged (= 1): gamma' and r.r from the omega reduction, and the p update of
//     the next iteration fused into the x/r update:
//     k_apply_dot<DELTA>, k_rstar, k_apply_dot<OMEGA_MERGED>, k_xrp_update
//
// The loop's kernels go out as programmatic dependent launches (launch_pdl):
// each one's launch is processed while its predecessor runs, and it waits at its
// first instruction for the predecessor's completion.
//
// Outer loop: r64 = b - A x in float64 (hi + lo coefficients), stop when
// ||r64|| / ||b|| <= rtol, else run a pass on D^-1 r64, add d to x (float64)
// and update r64 -= A d in double-float arithmetic; the residual that accepts
// the solution is recomputed from x.
#include <cmath>
#include <cstring>

#include "apply.cuh"
#include "bulk.cuh"
#include "bicgstab_scalars.cuh"
#include "reduce.cuh"
#include "sph_internal.cuh"

namespace sph {


namespace {

enum Phase : int { PH_DELTA = 0, PH_OMEGA = 1, PH_OMEGA_MERGED = 2, PH_CG = 3 };

struct Vecs {
  float4* r;
  float4* rh;
  float4* p;
  float4* Ap;
  float4* rs;
  float4* As;
  float4* d;
};

// ---- kernels ----------------------------------------------------------------

// r = rh = float32(r64 / D) (Jacobi) and d = 0; then gamma = tau^2 base = r.r
__global__ void __launch_bounds__(kBlock) k_pass_init(const double* __restrict__ r64, const double* __restrict__ D64,
                                                      int jacobi, int64_t n_pad, Vecs V, double eps2, int maxit,
                                                      SolverScalars* S, double* partials, unsigned int* counter) {
  double accd[3] = {0.0, 0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const double sc = jacobi ? 1.0 / D64[s] : 1.0;
    const float4 r = make_float4((float)(r64[3 * s] * sc), (float)(r64[3 * s + 1] * sc), (float)(r64[3 * s + 2] * sc),
                                 0.f);
    V.r[s] = r;
    V.rh[s] = r;
    V.d[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    accd[0] += (double)r.x * r.x;
    accd[1] += (double)r.y * r.y;
    accd[2] += (double)r.z * r.z;
  }
  block_partials_f64<3>(accd, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x == 0) scal_init(S, res, eps2, maxit);
  }
}

// p = r + beta p - alpha' Ap
__global__ void __launch_bounds__(kBlock) k_p_update(int64_t n_pad, Vecs V, const SolverScalars* __restrict__ S) {
  griddep_wait();
  if (S->done) return;
  const float b0 = (float)S->beta[0], b1 = (float)S->beta[1], b2 = (float)S->beta[2];
  const float a0 = (float)S->alpha_p[0], a1 = (float)S->alpha_p[1], a2 = (float)S->alpha_p[2];
  const bool useP = (b0 != 0.f) || (b1 != 0.f) || (b2 != 0.f);
  const bool useA = (a0 != 0.f) || (a1 != 0.f) || (a2 != 0.f);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
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

// y = D^-1 A v with the dots of the phase.
//   PH_DELTA:        v = p,  y = Ap; dots r0^.Ap                       (K = 3)
//   PH_OMEGA:        v = r*, y = Ar*; dots r*.Ar*, Ar*.Ar*             (K = 6)
//   PH_OMEGA_MERGED: + r0^.r*, r0^.Ar*, r*.r*                          (K = 15)
//   PH_CG:           y = A v without the Jacobi scaling (the rotated CG keeps
//                    the matrix symmetric and preconditions through z = D^-1 r);
//                    v = p, y = Ap; dots p.Ap                          (K = 3)
template <int PH>
struct PhaseDots {
  static constexpr int K = (PH == PH_DELTA || PH == PH_CG) ? 3 : (PH == PH_OMEGA ? 6 : 15);
};

template <int PH>
__device__ __forceinline__ void dots_row(float* acc, float4 o, float4 vb, const float4* __restrict__ rh, int64_t s) {
  if (PH == PH_DELTA) {
    const float4 h = rh[s];
    acc[0] = fmaf(h.x, o.x, acc[0]);
    acc[1] = fmaf(h.y, o.y, acc[1]);
    acc[2] = fmaf(h.z, o.z, acc[2]);
  } else if (PH == PH_CG) {
    acc[0] = fmaf(vb.x, o.x, acc[0]);
    acc[1] = fmaf(vb.y, o.y, acc[1]);
    acc[2] = fmaf(vb.z, o.z, acc[2]);
  } else {
    acc[0] = fmaf(vb.x, o.x, acc[0]);
    acc[1] = fmaf(vb.y, o.y, acc[1]);
    acc[2] = fmaf(vb.z, o.z, acc[2]);
    acc[3] = fmaf(o.x, o.x, acc[3]);
    acc[4] = fmaf(o.y, o.y, acc[4]);
    acc[5] = fmaf(o.z, o.z, acc[5]);
    if (PH == PH_OMEGA_MERGED) {
      const float4 h = rh[s];
      acc[6] = fmaf(h.x, vb.x, acc[6]);
      acc[7] = fmaf(h.y, vb.y, acc[7]);
      acc[8] = fmaf(h.z, vb.z, acc[8]);
      acc[9] = fmaf(h.x, o.x, acc[9]);
      acc[10] = fmaf(h.y, o.y, acc[10]);
      acc[11] = fmaf(h.z, o.z, acc[11]);
      acc[12] = fmaf(vb.x, vb.x, acc[12]);
      acc[13] = fmaf(vb.y, vb.y, acc[13]);
      acc[14] = fmaf(vb.z, vb.z, acc[14]);
    }
  }
}

// block partials, then the last block sums them and updates the scalars
template <int PH>
__device__ __forceinline__ void dots_finish(const float (&acc)[PhaseDots<PH>::K], SolverScalars* S,
                                            double* partials, unsigned int* counter) {
  constexpr int K = PhaseDots<PH>::K;
  block_partials<K>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[K];
    prefetch_scalars(S, sizeof(SolverScalars));
    final_sum<K>(partials, counter, res);
    if (threadIdx.x < 32) {
      if (PH == PH_DELTA) {
        scal_after_delta_w(S, res);
      } else if (PH == PH_CG) {
        scal_cg_alpha_w(S, res);
      } else {
        scal_after_omega_w(S, res);
        if (PH == PH_OMEGA_MERGED) {
          __syncwarp();
          double gn[3], rr[3];
          for (int c = 0; c < 3; ++c) {
            const double om = S->omega[c];
            gn[c] = res[6 + c] - om * res[9 + c];
            rr[c] = res[12 + c] - 2.0 * om * res[c] + om * om * res[3 + c];
          }
          scal_after_update_w(S, gn, rr);
        }
      }
    }
  }
}

template <int PH, int U, bool PF>
__global__ void __launch_bounds__(kBlock, 4) k_apply_dot(OpView op, const float4* __restrict__ v, float4* __restrict__ y,
                                                      const float4* __restrict__ rh, SolverScalars* S,
                                                      double* partials, unsigned int* counter) {
  constexpr int K = PhaseDots<PH>::K;
  griddep_wait();
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  // grid-stride: at any moment the grid works on one band of consecutive slices,
  // so the neighbour vectors they gather are shared in L2 across the SMs
  // (contiguous per-warp ranges, balanced by bytes, measured 9% slower)
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < op.nslices; sl += nwarps) {
    const int64_t s = sl * kSlice + lane;
    float4 vb;
    const float4 o = apply_row<U, PF, PH != PH_CG>(op, v, sl, lane, vb);
    y[s] = o;
    dots_row<PH>(acc, o, vb, rh, s);
  }
  dots_finish<PH>(acc, S, partials, counter);
}

// Row-loop form 4: the coefficient stream staged through shared memory.  Each
// warp owns kStageBuf buffers of kStageCh entries x 32 rows (2 KB) and an
// mbarrier per buffer; lane 0 fills them with bulk asynchronous copies
// (cp.async.bulk, bulk.cuh), running ahead over the warp's slices in order, so
// the stream's bytes in flight cost no registers and each warp keeps up to
// kStageBuf x 2 KB of it in flight.  The lanes read their entry of each staged
// row from shared memory (conflict-free: 32 consecutive int2) and gather the
// neighbour vectors kStageU at a time, as the register forms do.  Every issued
// copy is consumed before the warp leaves its loop.  A wait that does not
// complete within ~2 s of SM clock sets S->fault, stops the warp issuing,
// waits (bounded) for its copies still in flight and lets the kernel finish;
// the host then reports SPH_ERR_TIMEOUT.
constexpr int kStageCh = 8;
constexpr int kStageBuf = 2;
constexpr int kStageU = 4;
constexpr long long kStageWaitCycles = 4000000000ll;

template <int PH>
__global__ void __launch_bounds__(kBlock, 4) k_apply_dot_staged(OpView op, const float4* __restrict__ v,
                                                             float4* __restrict__ y, const float4* __restrict__ rh,
                                                             SolverScalars* S, double* partials,
                                                             unsigned int* counter) {
  constexpr int K = PhaseDots<PH>::K;
  constexpr int kWarps = kBlock / 32;
  __shared__ __align__(128) int2 sbuf[kWarps][kStageBuf][kStageCh * kSlice];
  __shared__ __align__(8) uint64_t sbar[kWarps][kStageBuf];
  griddep_wait();
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (lane == 0) {
    for (int b = 0; b < kStageBuf; ++b) mbar_init(&sbar[wid][b], 1);
    fence_mbarrier_init();
  }
  __syncwarp();

  // producer cursor: next chunk (slice psl, chunk pch of pnch) to copy
  int64_t psl = gw;
  int pch = 0;
  int pnch = psl < op.nslices ? (int)(((op.off[psl + 1] - op.off[psl]) / kSlice + kStageCh - 1) / kStageCh) : 0;
  uint32_t inflight = 0;   // bit b: buffer b has a copy not yet waited for
  bool stop = false;       // set on a fault: issue nothing more
  auto produce = [&](int b) {
    while (psl < op.nslices && pch >= pnch) {
      psl += nw;
      pch = 0;
      pnch = psl < op.nslices ? (int)(((op.off[psl + 1] - op.off[psl]) / kSlice + kStageCh - 1) / kStageCh) : 0;
    }
    if (stop || psl >= op.nslices) return;
    if (lane == 0) {
      const int w = (int)((op.off[psl + 1] - op.off[psl]) / kSlice);
      const int ne = min(kStageCh, w - pch * kStageCh);
      const uint32_t bytes = (uint32_t)ne * kSlice * (uint32_t)sizeof(int2);
      fence_proxy_async();
      mbar_expect_tx(&sbar[wid][b], bytes);
      bulk_g2s(&sbuf[wid][b][0], op.ih + op.off[psl] + (int64_t)pch * kStageCh * kSlice, bytes, &sbar[wid][b]);
    }
    inflight |= 1u << b;
    ++pch;
  };
  uint32_t par = 0;        // bit b: parity of the next phase to complete on buffer b
  for (int b = 0; b < kStageBuf; ++b) produce(b);

  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  int cb = 0;
  for (int64_t sl = gw; sl < op.nslices && !stop; sl += nw) {
    const int64_t s = sl * kSlice + lane;
    const int c = op.cnt[s];
    const uint8_t kd = op.kind[s];
    const float4 vb = v[s];
    const float kap = (kd == KIND_FLUID) ? 1.f : 0.f;
    const int w = (int)((op.off[sl + 1] - op.off[sl]) / kSlice);
    const int nch = (w + kStageCh - 1) / kStageCh;
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int ch = 0; ch < nch; ++ch) {
      const bool ok = mbar_wait(&sbar[wid][cb], (par >> cb) & 1u, kStageWaitCycles);
      if (__any_sync(0xffffffffu, !ok)) {
        stop = true;
        if (lane == 0) atomicExch(&S->fault, 1);
        break;
      }
      par ^= 1u << cb;
      inflight &= ~(1u << cb);
      const int2* __restrict__ eb = &sbuf[wid][cb][0];
#pragma unroll
      for (int j0 = 0; j0 < kStageCh; j0 += kStageU) {
        int2 e[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
          const int j = ch * kStageCh + j0 + u;
          e[u] = (j < c) ? eb[(j0 + u) * kSlice + lane] : make_int2((int)s, 0);
        }
        float4 va[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) va[u] = __ldg(v + e[u].x);
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
          const float a = __int_as_float(e[u].y);
          ax = fmaf(a, fmaf(kap, vb.x, -va[u].x), ax);
          ay = fmaf(a, fmaf(kap, vb.y, -va[u].y), ay);
          az = fmaf(a, fmaf(kap, vb.z, -va[u].z), az);
        }
      }
      __syncwarp();
      produce(cb);
      cb = cb + 1 == kStageBuf ? 0 : cb + 1;
    }
    if (stop) break;
    float4 o;
    const float sc = op.invD[s];
    if (kd == KIND_FLUID) {
      o = make_float4((vb.x + ax) * sc, (vb.y + ay) * sc, (vb.z + az) * sc, 0.f);
    } else if (kd == KIND_SHEPARD) {
      o = make_float4((vb.x - ax) * sc, (vb.y - ay) * sc, (vb.z - az) * sc, 0.f);
    } else {
      o = make_float4(vb.x * sc, vb.y * sc, vb.z * sc, 0.f);
    }
    y[s] = o;
    dots_row<PH>(acc, o, vb, rh, s);
  }
  // after a fault: wait (bounded) for the copies this warp still has in flight
  for (int b = 0; b < kStageBuf; ++b)
    if (inflight & (1u << b)) mbar_wait(&sbar[wid][b], (par >> b) & 1u, kStageWaitCycles);
  dots_finish<PH>(acc, S, partials, counter);
}

// Row-loop form 5: each slice's distinct neighbour vectors gathered once into
// shared memory (the unions of apply_union.cu, ~350 rows for ~2,400 entries on
// the lava boxes), then every entry of the slice reads its neighbour from there:
// about seven times fewer global gathers than the register forms.  The entry
// stream (position in the union, coefficient) is loaded kUnionU entries at a
// time with the next group in flight.  A slice marked -1 (union above
// kUnionCap) runs the register form.  Measured slower than the register forms on
// the lava boxes: its 8 KB of shared memory per warp allow 24 resident warps per
// SM instead of 32, and the stream, not the gathers, then sets the pace.
constexpr int kUnionU = 4;

size_t union_smem_bytes() { return (size_t)(kBlock / 32) * kUnionCap * sizeof(float4); }

template <int PH>
__global__ void __launch_bounds__(kBlock, 3) k_apply_dot_union(OpView op, const float4* __restrict__ v,
                                                            float4* __restrict__ y, const float4* __restrict__ rh,
                                                            SolverScalars* S, double* partials,
                                                            unsigned int* counter) {
  constexpr int K = PhaseDots<PH>::K;
  extern __shared__ __align__(16) float4 vsm[];   // [kBlock / 32][kUnionCap]
  griddep_wait();
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  float4* vs = vsm + (threadIdx.x >> 5) * kUnionCap;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < op.nslices; sl += nwarps) {
    const int64_t s = sl * kSlice + lane;
    const int nu = op.unum[sl];
    float4 o, vb;
    if (nu < 0) {
      o = apply_row<4, true, true>(op, v, sl, lane, vb);
    } else {
      const int64_t o0 = op.off[sl];
      const int32_t* __restrict__ U = op.uni + o0;
      for (int i0 = 0; i0 < nu; i0 += 8 * kSlice) {
        float4 t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * kSlice + lane;
          t[u] = i < nu ? __ldg(v + U[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * kSlice + lane;
          if (i < nu) vs[i] = t[u];
        }
      }
      __syncwarp();
      const int c = op.cnt[s];
      const uint8_t kd = op.kind[s];
      vb = v[s];
      const float kap = (kd == KIND_FLUID) ? 1.f : 0.f;
      const int w = (int)((op.off[sl + 1] - o0) / kSlice);
      const int2* __restrict__ p = op.loc + o0 + lane;
      float ax = 0.f, ay = 0.f, az = 0.f;
      int2 e[kUnionU];
#pragma unroll
      for (int u = 0; u < kUnionU; ++u) e[u] = (u < c) ? __ldcs(p + (int64_t)u * kSlice) : make_int2(0, 0);
      for (int j0 = 0; j0 < w; j0 += kUnionU) {
        int2 en[kUnionU];
#pragma unroll
        for (int u = 0; u < kUnionU; ++u) {
          const int j = j0 + kUnionU + u;
          en[u] = (j < c) ? __ldcs(p + (int64_t)j * kSlice) : make_int2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < kUnionU; ++u) {
          const float4 va = vs[e[u].x];
          const float a = __int_as_float(e[u].y);
          ax = fmaf(a, fmaf(kap, vb.x, -va.x), ax);
          ay = fmaf(a, fmaf(kap, vb.y, -va.y), ay);
          az = fmaf(a, fmaf(kap, vb.z, -va.z), az);
        }
#pragma unroll
        for (int u = 0; u < kUnionU; ++u) e[u] = en[u];
      }
      __syncwarp();
      const float sc = op.invD[s];
      if (kd == KIND_FLUID) {
        o = make_float4((vb.x + ax) * sc, (vb.y + ay) * sc, (vb.z + az) * sc, 0.f);
      } else if (kd == KIND_SHEPARD) {
        o = make_float4((vb.x - ax) * sc, (vb.y - ay) * sc, (vb.z - az) * sc, 0.f);
      } else {
        o = make_float4(vb.x * sc, vb.y * sc, vb.z * sc, 0.f);
      }
    }
    y[s] = o;
    dots_row<PH>(acc, o, vb, rh, s);
  }
  dots_finish<PH>(acc, S, partials, counter);
}

}  // namespace

// [phase][variant] with variants (U, PF) = (8,0), (4,0), (8,1), (4,1) as in apply.cuh,
// 4 = the stream staged through shared memory by bulk copies, 5 = per-slice
// neighbour unions in shared memory; the CG phase has the register forms only
// (its 4 and 5 are the (4,1) form)
ApplyDotFn apply_kernel(int phase, int variant) {
  static const ApplyDotFn table[4][kApplyVariants] = {
      {k_apply_dot<PH_DELTA, 8, false>, k_apply_dot<PH_DELTA, 4, false>, k_apply_dot<PH_DELTA, 8, true>,
       k_apply_dot<PH_DELTA, 4, true>, k_apply_dot_staged<PH_DELTA>, k_apply_dot_union<PH_DELTA>},
      {k_apply_dot<PH_OMEGA, 8, false>, k_apply_dot<PH_OMEGA, 4, false>, k_apply_dot<PH_OMEGA, 8, true>,
       k_apply_dot<PH_OMEGA, 4, true>, k_apply_dot_staged<PH_OMEGA>, k_apply_dot_union<PH_OMEGA>},
      {k_apply_dot<PH_OMEGA_MERGED, 8, false>, k_apply_dot<PH_OMEGA_MERGED, 4, false>,
       k_apply_dot<PH_OMEGA_MERGED, 8, true>, k_apply_dot<PH_OMEGA_MERGED, 4, true>,
       k_apply_dot_staged<PH_OMEGA_MERGED>, k_apply_dot_union<PH_OMEGA_MERGED>},
      {k_apply_dot<PH_CG, 8, false>, k_apply_dot<PH_CG, 4, false>, k_apply_dot<PH_CG, 8, true>,
       k_apply_dot<PH_CG, 4, true>, k_apply_dot<PH_CG, 4, true>, k_apply_dot<PH_CG, 4, true>}};
  return table[phase < 0 ? 0 : (phase > 3 ? 3 : phase)][variant < 0 || variant >= kApplyVariants ? 0 : variant];
}

size_t apply_smem(int variant) { return variant == 5 ? union_smem_bytes() : 0; }

// one-time opt-in of the forms that use more than 48 KB of dynamic shared memory
static sph_status apply_attrs() {
  static bool done = false;
  if (done) return SPH_OK;
  for (int ph = 0; ph < 3; ++ph) {
    SPH_TRY_CUDA(cudaFuncSetAttribute((const void*)apply_kernel(ph, 5), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)apply_smem(5)));
    // the register forms use no shared memory beyond their reductions: ask for
    // the largest L1, which holds the gathered neighbour vectors
    for (int v = 0; v < kApplyVariantsRegister; ++v)
      SPH_TRY_CUDA(cudaFuncSetAttribute((const void*)apply_kernel(ph, v),
                                        cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxL1));
  }
  for (int v = 0; v < kApplyVariantsRegister; ++v)
    SPH_TRY_CUDA(cudaFuncSetAttribute((const void*)apply_kernel(PH_CG, v), cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxL1));
  done = true;
  return SPH_OK;
}

// what a form needs before it can run on H (form 5: the per-slice unions)
sph_status apply_prepare(sph_neighbors* H, int variant, cudaStream_t st) {
  SPH_TRY(apply_attrs());
  if (variant == 5) SPH_TRY(ensure_union(H, st));
  return SPH_OK;
}

namespace {

// r* = r - alpha Ap (the matching d += alpha p is folded into the x/r update)
__global__ void __launch_bounds__(kBlock) k_rstar(int64_t n_pad, Vecs V, const SolverScalars* __restrict__ S) {
  griddep_wait();
  if (S->done) return;
  const float a0 = (float)S->alpha[0], a1 = (float)S->alpha[1], a2 = (float)S->alpha[2];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 r = V.r[s], ap = V.Ap[s];
    V.rs[s] = make_float4(fmaf(-a0, ap.x, r.x), fmaf(-a1, ap.y, r.y), fmaf(-a2, ap.z, r.z), 0.f);
  }
}

// r = r* - omega Ar* ; d += alpha p + omega r* ; dots r0^.r, r.r (paper-exact gamma')
__global__ void __launch_bounds__(kBlock) k_xr_update(int64_t n_pad, Vecs V, SolverScalars* S, double* partials,
                                                      unsigned int* counter) {
  griddep_wait();
  if (S->done) return;
  const float w0 = (float)S->omega[0], w1 = (float)S->omega[1], w2 = (float)S->omega[2];
  const float al0 = (float)S->alpha[0], al1 = (float)S->alpha[1], al2 = (float)S->alpha[2];
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 rs = V.rs[s], as = V.As[s], h = V.rh[s], p = V.p[s];
    float4 d = V.d[s];
    const float4 r = make_float4(fmaf(-w0, as.x, rs.x), fmaf(-w1, as.y, rs.y), fmaf(-w2, as.z, rs.z), 0.f);
    d.x = fmaf(w0, rs.x, fmaf(al0, p.x, d.x));
    d.y = fmaf(w1, rs.y, fmaf(al1, p.y, d.y));
    d.z = fmaf(w2, rs.z, fmaf(al2, p.z, d.z));
    V.r[s] = r;
    V.d[s] = d;
    acc[0] = fmaf(h.x, r.x, acc[0]);
    acc[1] = fmaf(h.y, r.y, acc[1]);
    acc[2] = fmaf(h.z, r.z, acc[2]);
    acc[3] = fmaf(r.x, r.x, acc[3]);
    acc[4] = fmaf(r.y, r.y, acc[4]);
    acc[5] = fmaf(r.z, r.z, acc[5]);
  }
  block_partials<6>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[6];
    prefetch_scalars(S, sizeof(SolverScalars));
    final_sum<6>(partials, counter, res);
    if (threadIdx.x < 32) scal_after_update_w(S, res, res + 3);
  }
}

// merged form: r = r* - omega Ar* ; d += alpha p + omega r* ; p = r + beta p - alpha' Ap.
// Runs for the iteration whose omega kernel set the stop flag too (the
// iteration completes); `pad` carries "skip" and is re-armed by the last block.
__global__ void __launch_bounds__(kBlock) k_xrp_update(int64_t n_pad, Vecs V, SolverScalars* S,
                                                       unsigned int* counter) {
  griddep_wait();
  if (S->pad) return;
  const float w0 = (float)S->omega[0], w1 = (float)S->omega[1], w2 = (float)S->omega[2];
  const float b0 = (float)S->beta[0], b1 = (float)S->beta[1], b2 = (float)S->beta[2];
  const float a0 = (float)S->alpha_p[0], a1 = (float)S->alpha_p[1], a2 = (float)S->alpha_p[2];
  const float al0 = (float)S->alpha[0], al1 = (float)S->alpha[1], al2 = (float)S->alpha[2];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 rs = V.rs[s], as = V.As[s], p = V.p[s], ap = V.Ap[s];
    float4 d = V.d[s];
    const float4 r = make_float4(fmaf(-w0, as.x, rs.x), fmaf(-w1, as.y, rs.y), fmaf(-w2, as.z, rs.z), 0.f);
    d.x = fmaf(w0, rs.x, fmaf(al0, p.x, d.x));
    d.y = fmaf(w1, rs.y, fmaf(al1, p.y, d.y));
    d.z = fmaf(w2, rs.z, fmaf(al2, p.z, d.z));
    V.r[s] = r;
    V.d[s] = d;
    V.p[s] = make_float4(fmaf(-a0, ap.x, fmaf(b0, p.x, r.x)), fmaf(-a1, ap.y, fmaf(b1, p.y, r.y)),
                         fmaf(-a2, ap.z, fmaf(b2, p.z, r.z)), 0.f);
  }
  if (arrive_last(counter)) {
    if (threadIdx.x == 0) {
      S->pad = S->done;
      *counter = 0u;
    }
  }
}

// ---- rotated CG (Sec. 4.1), Jacobi-preconditioned through z = D^-1 r (App. B) ----
// One pass solves A d = r64 (the matrix itself, kept symmetric); per iteration
//   k_cg_p:            p = z + beta p   (z = w r, w = 1/D or 1; beta = 0 reads no p)
//   k_apply_dot<PH_CG>: Ap = A p, p.Ap  -> alpha = gamma / p.Ap
//   k_cg_xr:           r -= alpha Ap, d += alpha p; r.z and r.r -> beta, states

// r = float32(r64), d = 0; gamma = r.z, r.r
__global__ void __launch_bounds__(kBlock) k_cg_init(const double* __restrict__ r64, const float* __restrict__ invD,
                                                    int jacobi, int64_t n_pad, Vecs V, double eps2, int maxit,
                                                    SolverScalars* S, double* partials, unsigned int* counter) {
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 r = make_float4((float)r64[3 * s], (float)r64[3 * s + 1], (float)r64[3 * s + 2], 0.f);
    const float w = jacobi ? invD[s] : 1.f;
    V.r[s] = r;
    V.d[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    acc[0] = fmaf(r.x, w * r.x, acc[0]);
    acc[1] = fmaf(r.y, w * r.y, acc[1]);
    acc[2] = fmaf(r.z, w * r.z, acc[2]);
    acc[3] = fmaf(r.x, r.x, acc[3]);
    acc[4] = fmaf(r.y, r.y, acc[4]);
    acc[5] = fmaf(r.z, r.z, acc[5]);
  }
  block_partials<6>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[6];
    final_sum<6>(partials, counter, res);
    if (threadIdx.x == 0) scal_cg_init(S, res, res + 3, eps2, maxit);
  }
}

// p = z + beta p
__global__ void __launch_bounds__(kBlock) k_cg_p(int64_t n_pad, Vecs V, const float* __restrict__ invD, int jacobi,
                                                 const SolverScalars* __restrict__ S) {
  griddep_wait();
  if (S->done) return;
  const float b0 = (float)S->beta[0], b1 = (float)S->beta[1], b2 = (float)S->beta[2];
  const bool useP = (b0 != 0.f) || (b1 != 0.f) || (b2 != 0.f);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 r = V.r[s];
    const float w = jacobi ? invD[s] : 1.f;
    float4 p = make_float4(w * r.x, w * r.y, w * r.z, 0.f);
    if (useP) {
      const float4 q = V.p[s];
      p.x = fmaf(b0, q.x, p.x);
      p.y = fmaf(b1, q.y, p.y);
      p.z = fmaf(b2, q.z, p.z);
    }
    V.p[s] = p;
  }
}

// r -= alpha Ap; d += alpha p; dots r.z, r.r
__global__ void __launch_bounds__(kBlock) k_cg_xr(int64_t n_pad, Vecs V, const float* __restrict__ invD, int jacobi,
                                                  SolverScalars* S, double* partials, unsigned int* counter) {
  griddep_wait();
  if (S->done) return;
  const float a0 = (float)S->alpha[0], a1 = (float)S->alpha[1], a2 = (float)S->alpha[2];
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 ap = V.Ap[s], p = V.p[s];
    float4 r = V.r[s], d = V.d[s];
    r.x = fmaf(-a0, ap.x, r.x);
    r.y = fmaf(-a1, ap.y, r.y);
    r.z = fmaf(-a2, ap.z, r.z);
    d.x = fmaf(a0, p.x, d.x);
    d.y = fmaf(a1, p.y, d.y);
    d.z = fmaf(a2, p.z, d.z);
    V.r[s] = r;
    V.d[s] = d;
    const float w = jacobi ? invD[s] : 1.f;
    acc[0] = fmaf(r.x, w * r.x, acc[0]);
    acc[1] = fmaf(r.y, w * r.y, acc[1]);
    acc[2] = fmaf(r.z, w * r.z, acc[2]);
    acc[3] = fmaf(r.x, r.x, acc[3]);
    acc[4] = fmaf(r.y, r.y, acc[4]);
    acc[5] = fmaf(r.z, r.z, acc[5]);
  }
  block_partials<6>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[6];
    prefetch_scalars(S, sizeof(SolverScalars));
    final_sum<6>(partials, counter, res);
    if (threadIdx.x < 32) scal_cg_update_w(S, res, res + 3);
  }
}

// identity rows (dynamic walls) take x = b before a CG solve: their exact value,
// which keeps the wall rows of every residual zero, so the iteration only ever
// sees the symmetric fluid block (the reduced system of Sec. 4)
__global__ void k_identity_rows_take_b(const uint8_t* __restrict__ kind, int64_t n_pad, const double* __restrict__ b,
                                       double* __restrict__ x) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (kind[s] == KIND_IDENTITY) {
      x[3 * s] = b[3 * s];
      x[3 * s + 1] = b[3 * s + 1];
      x[3 * s + 2] = b[3 * s + 2];
    }
  }
}

// x64 += d
__global__ void k_add_correction(int64_t n_pad, const float4* __restrict__ d, double* __restrict__ x) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = d[s];
    x[3 * s] += (double)v.x;
    x[3 * s + 1] += (double)v.y;
    x[3 * s + 2] += (double)v.z;
  }
}

__global__ void k_gather_d3(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                            double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      const int64_t i = perm[s];
      dst[3 * s] = src[3 * i];
      dst[3 * s + 1] = src[3 * i + 1];
      dst[3 * s + 2] = src[3 * i + 2];
    } else {
      dst[3 * s] = dst[3 * s + 1] = dst[3 * s + 2] = 0.0;
    }
  }
}

__global__ void k_scatter_d3(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                             double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[s];
    dst[3 * i] = src[3 * s];
    dst[3 * i + 1] = src[3 * s + 1];
    dst[3 * i + 2] = src[3 * s + 2];
  }
}

// squares per component of an [n_pad][3] float64 array, grid-reduced into out[3]
__global__ void __launch_bounds__(kBlock) k_norm2_d3(const double* __restrict__ a, int64_t n_pad, double* partials,
                                                     unsigned int* counter, double* out) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    acc[0] += a[3 * s] * a[3 * s];
    acc[1] += a[3 * s + 1] * a[3 * s + 1];
    acc[2] += a[3 * s + 2] * a[3 * s + 2];
  }
  block_partials_f64<3>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x < 3) out[threadIdx.x] = res[threadIdx.x];
  }
}

}  // namespace

// Counters: one per reduction site, so consecutive kernels never share one.
enum { CNT_INIT = 0, CNT_DELTA, CNT_OMEGA, CNT_XR, CNT_XRP, CNT_RES, CNT_NORM, CNT_TUNE, CNT_CG_A, CNT_CG_XR, CNT_COUNT };

sph_status ensure_workspace(sph_neighbors* H) {
  const int64_t np = H->n_pad;
  SPH_TRY(H->v_r.alloc(np));
  SPH_TRY(H->v_rh.alloc(np));
  SPH_TRY(H->v_p.alloc(np));
  SPH_TRY(H->v_Ap.alloc(np));
  SPH_TRY(H->v_rs.alloc(np));
  SPH_TRY(H->v_As.alloc(np));
  SPH_TRY(H->v_d.alloc(np));
  SPH_TRY(H->x64.alloc(3 * np));
  SPH_TRY(H->b64.alloc(3 * np));
  SPH_TRY(H->r64.alloc(3 * np));
  SPH_TRY(H->v_x2.alloc(2 * np));
  if (H->red_grid == 0) {
    int occ = 0;
    // the largest grid any apply variant runs with (partials are sized for it)
    int best = 1;
    for (int ph = 0; ph < 3; ++ph)
      for (int v = 0; v < kApplyVariants; ++v) {
        if (apply_attrs() != SPH_OK) return SPH_ERR_CUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)apply_kernel(ph, v), kBlock, apply_smem(v));
        best = occ > best ? occ : best;
      }
    H->red_grid = H->num_sms * best;
  }
  SPH_TRY(H->partials.alloc((size_t)H->red_grid * kMaxDots));
  if (!H->counters.p) {
    SPH_TRY(H->counters.alloc(CNT_COUNT));
    SPH_TRY_CUDA(cudaMemset(H->counters.p, 0, CNT_COUNT * sizeof(unsigned int)));
  }
  SPH_TRY(H->scal.alloc(1));
  if (!H->host_scal) SPH_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&H->host_scal), sizeof(SolverScalars)));
  if (!H->host_flags) SPH_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&H->host_flags), 64));
  return SPH_OK;
}

static int red_grid_for(const sph_neighbors* H, int64_t items) {
  int64_t want = (items + kBlock - 1) / kBlock;
  if (want > H->red_grid) want = H->red_grid;
  return want < 1 ? 1 : (int)want;
}

// r64 -= A d after x64 += d, and the new rr[3] (synchronises)
static sph_status residual_update(sph_neighbors* H, cudaStream_t st, const float4* d, double rr[3]) {
  const int grid = red_grid_for(H, H->n_pad);
  double* dev_out = reinterpret_cast<double*>(H->scal.p) + offsetof(SolverScalars, dots) / sizeof(double);
  launch_residual_update(H, grid, d, H->r64.p, H->partials.p, H->counters.p + CNT_RES, dev_out, st);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaMemcpyAsync(rr, dev_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

// r64 = b64 - A x64 and rr[3] into H->host_flags area (synchronises)
static sph_status true_residual(sph_neighbors* H, cudaStream_t st, double rr[3]) {
  const int grid = red_grid_for(H, H->n_pad);
  double* dev_out = reinterpret_cast<double*>(H->scal.p) + offsetof(SolverScalars, dots) / sizeof(double);
  launch_residual_f64(H, grid, H->x64.p, H->b64.p, H->r64.p, H->partials.p, H->counters.p + CNT_RES, dev_out, st);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaMemcpyAsync(rr, dev_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

// a kernel of the BiCGSTAB loop: a programmatic dependent launch unless the
// solve asked for plain stream order (every such kernel starts with griddep_wait)
template <typename... KArgs, typename... Args>
static cudaError_t loop_launch(bool pdl, void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t st,
                               Args... args) {
  if (pdl) return launch_pdl(kernel, grid, kBlock, smem, st, args...);
  SPH_LAUNCH(kernel, grid, kBlock, smem, st)(static_cast<KArgs>(args)...);
  return cudaGetLastError();
}

template <int PH>
static cudaError_t launch_apply_dot(sph_neighbors* H, bool pdl, int grid, const OpView& op, const float4* v,
                                    float4* y, const float4* rh, SolverScalars* S, unsigned int* counter,
                                    cudaStream_t st) {
  const bool forced = H->force_form >= 0;
  // the CG phase runs the register form the tuner chose for the delta phase (same dots)
  const int tp = PH == PH_CG ? PH_DELTA : PH;
  int var = forced ? H->force_form : H->apply_var[tp];
  int tg = forced ? H->force_grid : H->apply_grid[tp];
  if (PH == PH_CG && var >= kApplyVariantsRegister) {
    var = kApplyVariantsRegister - 1;
    tg = 0;
  }
  const int g = tg > 0 && tg < grid ? tg : grid;
  const ApplyDotFn kern = apply_kernel(PH, var);
  prof_begin(H, st, PH == PH_DELTA ? 0 : 1);
  const cudaError_t e = loop_launch(pdl, kern, g, apply_smem(var), st, op, v, y, rh, S, H->partials.p, counter);
  prof_end(H, st);
  return e;
}

sph_status solve_mixed(sph_neighbors* H, const sph_visc_params* P, const sph_solve_opts* O, const double* b,
                       double* x, sph_solve_report* R, cudaStream_t st) {
  SPH_TRY(ensure_operator(H, P, st));
  SPH_TRY(ensure_workspace(H));
  // balanced slice ranges for the grid of the float64 residual kernels
  SPH_TRY(ensure_wpart(H, red_grid_for(H, H->n_pad), st));
  SPH_TRY(autotune_apply(H, O->merged_reductions != 0, H->counters.p + CNT_TUNE, st));
  const int64_t np = H->n_pad;
  const int grid_rows = red_grid_for(H, np);
  const int grid_slices = red_grid_for(H, H->nslices * 32);
  // the chosen forms' prerequisites (the unions of form 5 follow the operator)
  SPH_TRY(apply_prepare(H, H->apply_var[PH_DELTA], st));
  SPH_TRY(apply_prepare(H, H->apply_var[O->merged_reductions ? PH_OMEGA_MERGED : PH_OMEGA], st));
  H->force_form = -1;
  if (O->launch_mode < 0 || O->launch_mode > 1) {
    set_error("sph_visc_solve: launch_mode %d is neither 0 nor 1", O->launch_mode);
    return SPH_ERR_INVALID;
  }
  if (O->apply_form < 0 || O->apply_form > kApplyVariants) {
    set_error("sph_visc_solve: apply_form %d outside 0..%d", O->apply_form, kApplyVariants);
    return SPH_ERR_INVALID;
  }
  const bool cg = O->method == SPH_SOLVER_CG;
  if (O->method != SPH_SOLVER_BICGSTAB && O->method != SPH_SOLVER_CG) {
    set_error("sph_visc_solve: unknown method %d", O->method);
    return SPH_ERR_INVALID;
  }
  if (cg && P->boundary != SPH_BC_DYNAMIC) {
    set_error("sph_visc_solve: the conjugate gradient needs a symmetric matrix, which the dummy boundary "
              "model does not give (Sec. 4): use SPH_BC_DYNAMIC or BiCGSTAB");
    return SPH_ERR_INVALID;
  }
  if (cg && O->apply_form > kApplyVariantsRegister) {
    set_error("sph_visc_solve: apply_form %d is a BiCGSTAB form; the conjugate gradient takes 0..%d", O->apply_form,
              kApplyVariantsRegister);
    return SPH_ERR_INVALID;
  }
  if (!cg && !O->jacobi) {
    set_error("sph_visc_solve: the mixed-precision BiCGSTAB always scales by the Jacobi diagonal (jacobi = 1)");
    return SPH_ERR_INVALID;
  }
  if (O->apply_form > 0) {
    SPH_TRY(apply_prepare(H, O->apply_form - 1, st));
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)apply_kernel(PH_DELTA, O->apply_form - 1), kBlock,
                                                  apply_smem(O->apply_form - 1));
    H->force_form = O->apply_form - 1;
    H->force_grid = H->num_sms * (occ > 0 ? occ : 1);
  }
  if (H->row_scaled && !O->jacobi) {
    set_error("sph_visc_solve: a row scale multiplies the Jacobi diagonal (jacobi = 1)");
    return SPH_ERR_INVALID;
  }
  SPH_TRY(row_scale_refresh(H, st));
  Vecs V{H->v_r.p, H->v_rh.p, H->v_p.p, H->v_Ap.p, H->v_rs.p, H->v_As.p, H->v_d.p};
  // the preconditioner's diagonal: D, or D / s with a row scale s
  OpView op = op_view(H);
  if (H->row_scaled) op.invD = H->invD_sc.p;
  const float* invD = op.invD;
  const double* D64 = H->row_scaled ? H->D64_sc.p : H->D64.p;
  SolverScalars* S = H->scal.p;
  unsigned int* C = H->counters.p;
  SPH_TRY_CUDA(cudaMemsetAsync(&S->fault, 0, sizeof(int32_t), st));

  SPH_LAUNCH(k_gather_d3, grid_for(H, np), kBlock, 0, st)(b, H->perm.p, H->n, np, H->b64.p);
  SPH_LAUNCH(k_gather_d3, grid_for(H, np), kBlock, 0, st)(x, H->perm.p, H->n, np, H->x64.p);
  if (cg) SPH_LAUNCH(k_identity_rows_take_b, grid_for(H, np), kBlock, 0, st)(H->op_kind.p, np, H->b64.p, H->x64.p);
  SPH_TRY_CUDA(cudaGetLastError());
  double* dev_dots = reinterpret_cast<double*>(S) + offsetof(SolverScalars, dots) / sizeof(double);
  SPH_LAUNCH(k_norm2_d3, grid_rows, kBlock, 0, st)(H->b64.p, np, H->partials.p, C + CNT_NORM, dev_dots);
  SPH_TRY_CUDA(cudaGetLastError());
  double bb[3];
  SPH_TRY_CUDA(cudaMemcpyAsync(bb, dev_dots, sizeof(bb), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bb[0] + bb[1] + bb[2]);

  const double rtol = O->rtol > 0.0 ? O->rtol : 1e-6;
  const double eps_floor = O->eps_inner > 0.0 ? O->eps_inner : 2e-2;
  const int maxit = O->maxit > 0 ? O->maxit : 10000;
  const int max_ref = O->max_refine > 0 ? O->max_refine : 20;
  const int chunk0 = O->chunk > 0 ? O->chunk : 8;
  const bool merged = O->merged_reductions != 0;
  const int jacobi = O->jacobi ? 1 : 0;
  const bool pdl = O->launch_mode == 0;

  std::memset(R, 0, sizeof(*R));
  int total_iters = 0, passes = 0;
  // Launch chunks: the host checks the device's stop flag after each chunk, and
  // iterations launched past a pass's convergence exit at once but still cost a
  // launch each.  Passes of one system take similar iteration counts, so the
  // first chunk of a pass runs to just short of the same pass of the last solve
  // with the same dt (or of the previous pass), then chunks of 4 follow; without
  // a prediction the chunks double from `chunk`.
  int prev_pass = 0;
  int new_len[sph_neighbors::kPassHist] = {};
  int slot = H->pass_dt[0] == P->dt ? 0 : (H->pass_dt[1] == P->dt ? 1 : -1);
  if (slot < 0) {   // a new time step: take the slot used longest ago, empty
    slot = H->pass_slot_next;
    H->pass_slot_next ^= 1;
    H->pass_dt[slot] = P->dt;
    for (int k = 0; k < sph_neighbors::kPassHist; ++k) H->pass_len[slot][k] = 0;
  } else {
    H->pass_slot_next = slot ^ 1;
  }
  const int* hist = H->pass_len[slot];
  double rr[3] = {0, 0, 0};
  sph_status status = SPH_NOT_CONVERGED;
  // r64 after a pass comes from the update r64 -= A d (rr_full = false); the
  // first residual, the one that accepts the solution and the one reported are
  // recomputed as b - A x64 from x (rr_full = true)
  bool rr_full = false, have_rr = false;
  for (int ref = 0;; ++ref) {
    if (!have_rr) {
      SPH_TRY(true_residual(H, st, rr));
      rr_full = true;
    }
    have_rr = false;
    if (!std::isfinite(rr[0]) || !std::isfinite(rr[1]) || !std::isfinite(rr[2])) {
      set_error("sph_visc_solve: the true residual is not finite");
      status = SPH_ERR_NONFINITE;
      break;
    }
    double rnorm = std::sqrt(rr[0] + rr[1] + rr[2]);
    if (rnorm <= rtol * bnorm && !rr_full) {
      SPH_TRY(true_residual(H, st, rr));
      rr_full = true;
      rnorm = std::sqrt(rr[0] + rr[1] + rr[2]);
      if (!std::isfinite(rnorm)) {
        set_error("sph_visc_solve: the true residual is not finite");
        status = SPH_ERR_NONFINITE;
        break;
      }
    }
    if (rnorm <= rtol * bnorm) {
      status = SPH_OK;
      break;
    }
    if (ref >= max_ref || total_iters >= maxit) break;
    // inner pass: ask it for what the outer loop still needs (with a 4x margin),
    // but never for more than eps_floor (float32 recursions stall below that)
    const double eps = std::fmax(eps_floor, 0.25 * rtol * bnorm / rnorm);
    if (cg) {
      SPH_LAUNCH(k_cg_init, grid_rows, kBlock, 0, st)(H->r64.p, invD, jacobi, np, V, eps * eps, maxit - total_iters, S,
                                                      H->partials.p, C + CNT_INIT);
    } else {
      SPH_LAUNCH(k_pass_init, grid_rows, kBlock, 0, st)(H->r64.p, D64, jacobi, np, V, eps * eps, maxit - total_iters,
                                                        S, H->partials.p, C + CNT_INIT);
    }
    SPH_TRY_CUDA(cudaGetLastError());
    if (merged && !cg) SPH_LAUNCH(k_p_update, grid_rows, kBlock, 0, st)(np, V, S);
    const int pred = (passes < sph_neighbors::kPassHist && hist[passes] > 0) ? hist[passes] : prev_pass;
    // a long pass: stop two short of the prediction (the last iterations then
    // come in chunks of 4); a short one (a few iterations, as in the small
    // systems of a time step): launch exactly the prediction, since a default
    // chunk of 8 would mostly launch iterations that exit at once
    int chunk = pred > chunk0 + 2 ? pred - 2 : (pred > 0 ? pred : chunk0);
    int iter_seen = 0;
    for (;;) {
      cudaError_t le = cudaSuccess;
      auto keep = [&le](cudaError_t e) {
        if (le == cudaSuccess) le = e;
      };
      for (int it = 0; it < chunk; ++it) {
        if (cg) {
          keep(loop_launch(pdl, k_cg_p, grid_rows, 0, st, np, V, invD, jacobi, S));
          keep(launch_apply_dot<PH_CG>(H, pdl, grid_slices, op, V.p, V.Ap, V.rh, S, C + CNT_CG_A, st));
          keep(loop_launch(pdl, k_cg_xr, grid_rows, 0, st, np, V, invD, jacobi, S, H->partials.p, C + CNT_CG_XR));
          continue;
        }
        if (!merged) keep(loop_launch(pdl, k_p_update, grid_rows, 0, st, np, V, S));
        keep(launch_apply_dot<PH_DELTA>(H, pdl, grid_slices, op, V.p, V.Ap, V.rh, S, C + CNT_DELTA, st));
        keep(loop_launch(pdl, k_rstar, grid_rows, 0, st, np, V, S));
        if (merged) {
          keep(launch_apply_dot<PH_OMEGA_MERGED>(H, pdl, grid_slices, op, V.rs, V.As, V.rh, S, C + CNT_OMEGA, st));
          keep(loop_launch(pdl, k_xrp_update, grid_rows, 0, st, np, V, S, C + CNT_XRP));
        } else {
          keep(launch_apply_dot<PH_OMEGA>(H, pdl, grid_slices, op, V.rs, V.As, V.rh, S, C + CNT_OMEGA, st));
          keep(loop_launch(pdl, k_xr_update, grid_rows, 0, st, np, V, S, H->partials.p, C + CNT_XR));
        }
      }
      SPH_TRY_CUDA(le);
      SPH_TRY_CUDA(cudaGetLastError());
      SPH_TRY_CUDA(cudaMemcpyAsync(H->host_scal, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
      SPH_TRY_CUDA(cudaStreamSynchronize(st));
      prof_flush(H, (cg ? 1 : 2) * (H->host_scal->iter - iter_seen));
      iter_seen = H->host_scal->iter;
      if (H->host_scal->fault) {
        set_error("sph_visc_solve: an operator apply gave up waiting for its staged coefficients");
        return SPH_ERR_TIMEOUT;
      }
      if (H->host_scal->done) break;
      chunk = pred > 0 ? (pred <= 2 ? 2 : 4) : (chunk < 64 ? chunk * 2 : chunk);
    }
    const SolverScalars& hs = *H->host_scal;
    total_iters += hs.iter;
    if (passes < sph_neighbors::kPassHist) new_len[passes] = hs.iter;
    prev_pass = hs.iter;
    passes++;
    for (int c = 0; c < 3; ++c) {
      R->state[c] = (int8_t)hs.state[c];
      R->stalled_any[c] |= (int8_t)hs.stalled_any[c];
    }
    SPH_LAUNCH(k_add_correction, grid_for(H, np), kBlock, 0, st)(np, V.d, H->x64.p);
    SPH_TRY_CUDA(cudaGetLastError());
    if (hs.iter == 0) {  // nothing progressed: a further pass would repeat it
      SPH_TRY(true_residual(H, st, rr));
      rr_full = true;
      const double rnorm2 = std::sqrt(rr[0] + rr[1] + rr[2]);
      status = rnorm2 <= rtol * bnorm ? SPH_OK : SPH_NOT_CONVERGED;
      break;
    }
    SPH_TRY(residual_update(H, st, V.d, rr));
    have_rr = true;
    rr_full = false;
  }
  if (!rr_full && status != SPH_ERR_NONFINITE) SPH_TRY(true_residual(H, st, rr));
  for (int k = 0; k < sph_neighbors::kPassHist; ++k) H->pass_len[slot][k] = new_len[k];
  SPH_LAUNCH(k_scatter_d3, grid_for(H, H->n), kBlock, 0, st)(H->x64.p, H->perm.p, H->n, x);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  R->iters = total_iters;
  R->refinements = passes;
  R->true_rel_res = bnorm > 0.0 ? std::sqrt(rr[0] + rr[1] + rr[2]) / bnorm : std::sqrt(rr[0] + rr[1] + rr[2]);
  for (int c = 0; c < 3; ++c)
    R->true_rel_res_c[c] = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : std::sqrt(rr[c]);
  R->status = status;
  if (status == SPH_NOT_CONVERGED)
    set_error("sph_visc_solve: true residual %.3e above rtol %.1e after %d iterations / %d passes",
              R->true_rel_res, rtol, total_iters, passes);
  return status;
}

sph_status visc_residual(sph_neighbors* H, const sph_visc_params* P, const double* x, const double* b, double* r,
                         cudaStream_t st) {
  if (!H || !x || !b || !r) {
    set_error("sph_visc_residual: null argument");
    return SPH_ERR_INVALID;
  }
  SPH_TRY(ensure_operator(H, P, st));
  SPH_TRY(ensure_workspace(H));
  const int64_t np = H->n_pad;
  SPH_LAUNCH(k_gather_d3, grid_for(H, np), kBlock, 0, st)(b, H->perm.p, H->n, np, H->b64.p);
  SPH_LAUNCH(k_gather_d3, grid_for(H, np), kBlock, 0, st)(x, H->perm.p, H->n, np, H->x64.p);
  SPH_TRY_CUDA(cudaGetLastError());
  double rr[3];
  SPH_TRY(true_residual(H, st, rr));
  SPH_LAUNCH(k_scatter_d3, grid_for(H, H->n), kBlock, 0, st)(H->r64.p, H->perm.p, H->n, r);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
