// All-float64 solve (SPH_PREC_FP64): the restructured BiCGSTAB of paper Sec. 4.2
// with float64 vectors, float64 coefficients (a = hi + lo) and float64 dots.
// It iterates on x itself (no correction vector); the outer loop only checks
// the float64 true residual, so one pass usually suffices.  It exists for the
// precision study against the mixed solve: on this GPU float64 arithmetic runs
// at a small fraction of the float32 rate, so it is the slow reference mode.
#include <cmath>
#include <cstring>

#include "apply.cuh"
#include "bicgstab_scalars.cuh"
#include "reduce.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

enum Phase64 : int { P64_DELTA = 0, P64_OMEGA = 1, P64_OMEGA_MERGED = 2 };

struct Vecs64 {
  double* r;
  double* rh;
  double* p;
  double* Ap;
  double* rs;
  double* As;
  double* x;
};

template <int U>
__device__ __forceinline__ void apply_row64(const OpView& op, const float* __restrict__ op_lo,
                                            const double* __restrict__ D64, const double* __restrict__ v, int64_t sl,
                                            int lane, double out[3], double vb[3]) {
  const int64_t s = sl * kSlice + lane;
  const int c = op.cnt[s];
  const uint8_t kd = op.kind[s];
  vb[0] = v[3 * s];
  vb[1] = v[3 * s + 1];
  vb[2] = v[3 * s + 2];
  const double kap = (kd == KIND_FLUID) ? 1.0 : 0.0;
  const int64_t o0 = op.off[sl];
  const int w = (int)((op.off[sl + 1] - o0) / kSlice);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int j0 = 0; j0 < w; j0 += U) {
    int2 e[U];
    float lo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = j0 + u < c;
      const int64_t idx = o0 + lane + (int64_t)(j0 + u) * kSlice;
      e[u] = in ? __ldcs(op.ih + idx) : make_int2((int)s, 0);
      lo[u] = in ? __ldcs(op_lo + idx) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double a = (double)__int_as_float(e[u].y) + (double)lo[u];
      const int64_t t = e[u].x;
      a0 = fma(a, fma(kap, vb[0], -v[3 * t]), a0);
      a1 = fma(a, fma(kap, vb[1], -v[3 * t + 1]), a1);
      a2 = fma(a, fma(kap, vb[2], -v[3 * t + 2]), a2);
    }
  }
  if (kd == KIND_FLUID) {
    const double sc = 1.0 / D64[s];
    out[0] = (vb[0] + a0) * sc;
    out[1] = (vb[1] + a1) * sc;
    out[2] = (vb[2] + a2) * sc;
  } else if (kd == KIND_SHEPARD) {
    out[0] = vb[0] - a0;
    out[1] = vb[1] - a1;
    out[2] = vb[2] - a2;
  } else {
    out[0] = vb[0];
    out[1] = vb[1];
    out[2] = vb[2];
  }
}

__global__ void __launch_bounds__(kBlock) k64_pass_init(const double* __restrict__ r64, const double* __restrict__ D64,
                                                        int64_t n_pad, Vecs64 V, double eps2, int maxit,
                                                        SolverScalars* S, double* partials, unsigned int* counter) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const double sc = 1.0 / D64[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double r = r64[3 * s + k] * sc;
      V.r[3 * s + k] = r;
      V.rh[3 * s + k] = r;
      acc[k] += r * r;
    }
  }
  block_partials_f64<3>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x == 0) scal_init(S, res, eps2, maxit);
  }
}

__global__ void __launch_bounds__(kBlock) k64_p_update(int64_t n_pad, Vecs64 V, const SolverScalars* __restrict__ S) {
  if (S->done) return;
  const double be[3] = {S->beta[0], S->beta[1], S->beta[2]};
  const double ap[3] = {S->alpha_p[0], S->alpha_p[1], S->alpha_p[2]};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double p = V.r[3 * s + k];
      if (be[k] != 0.0) p = fma(be[k], V.p[3 * s + k], p);
      if (ap[k] != 0.0) p = fma(-ap[k], V.Ap[3 * s + k], p);
      V.p[3 * s + k] = p;
    }
  }
}

template <int PH>
__global__ void __launch_bounds__(kBlock) k64_apply_dot(OpView op, const float* __restrict__ op_lo,
                                                        const double* __restrict__ D64, const double* __restrict__ v,
                                                        double* __restrict__ y, const double* __restrict__ rh,
                                                        SolverScalars* S, double* partials, unsigned int* counter) {
  constexpr int K = PH == P64_DELTA ? 3 : (PH == P64_OMEGA ? 6 : 15);
  if (S->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < op.nslices; sl += nwarps) {
    const int64_t s = sl * kSlice + lane;
    double o[3], vb[3];
    apply_row64<4>(op, op_lo, D64, v, sl, lane, o, vb);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      y[3 * s + k] = o[k];
      const double h = rh[3 * s + k];
      if (PH == P64_DELTA) {
        acc[k] = fma(h, o[k], acc[k]);
      } else {
        acc[k] = fma(vb[k], o[k], acc[k]);
        acc[3 + k] = fma(o[k], o[k], acc[3 + k]);
        if (PH == P64_OMEGA_MERGED) {
          acc[6 + k] = fma(h, vb[k], acc[6 + k]);
          acc[9 + k] = fma(h, o[k], acc[9 + k]);
          acc[12 + k] = fma(vb[k], vb[k], acc[12 + k]);
        }
      }
    }
  }
  block_partials_f64<K>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[K];
    final_sum<K>(partials, counter, res);
    if (threadIdx.x == 0) {
      if (PH == P64_DELTA) {
        scal_after_delta(S, res);
      } else {
        scal_after_omega(S, res);
        if (PH == P64_OMEGA_MERGED) {
          double gn[3], rr[3];
          for (int c = 0; c < 3; ++c) {
            const double om = S->omega[c];
            gn[c] = res[6 + c] - om * res[9 + c];
            rr[c] = res[12 + c] - 2.0 * om * res[c] + om * om * res[3 + c];
          }
          scal_after_update(S, gn, rr);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kBlock) k64_rstar(int64_t n_pad, Vecs64 V, const SolverScalars* __restrict__ S) {
  if (S->done) return;
  const double al[3] = {S->alpha[0], S->alpha[1], S->alpha[2]};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) V.rs[3 * s + k] = fma(-al[k], V.Ap[3 * s + k], V.r[3 * s + k]);
  }
}

// r = r* - omega Ar*; x += alpha p + omega r*; (paper-exact) dots r0^.r and r.r
template <bool MERGED>
__global__ void __launch_bounds__(kBlock) k64_xr_update(int64_t n_pad, Vecs64 V, SolverScalars* S, double* partials,
                                                        unsigned int* counter) {
  if (MERGED ? S->pad : S->done) return;
  const double om[3] = {S->omega[0], S->omega[1], S->omega[2]};
  const double al[3] = {S->alpha[0], S->alpha[1], S->alpha[2]};
  const double be[3] = {S->beta[0], S->beta[1], S->beta[2]};
  const double ap[3] = {S->alpha_p[0], S->alpha_p[1], S->alpha_p[2]};
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t i = 3 * s + k;
      const double rs = V.rs[i], p = V.p[i];
      const double r = fma(-om[k], V.As[i], rs);
      V.x[i] = fma(om[k], rs, fma(al[k], p, V.x[i]));
      V.r[i] = r;
      if (MERGED) {
        V.p[i] = fma(-ap[k], V.Ap[i], fma(be[k], p, r));
      } else {
        acc[k] = fma(V.rh[i], r, acc[k]);
        acc[3 + k] = fma(r, r, acc[3 + k]);
      }
    }
  }
  if (MERGED) {
    if (arrive_last(counter)) {
      if (threadIdx.x == 0) {
        S->pad = S->done;
        *counter = 0u;
      }
    }
    return;
  }
  block_partials_f64<6>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[6];
    final_sum<6>(partials, counter, res);
    if (threadIdx.x == 0) scal_after_update(S, res, res + 3);
  }
}

__global__ void k64_gather(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                           double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * s + k] = (s < n) ? src[3 * (int64_t)perm[s] + k] : 0.0;
  }
}

__global__ void k64_scatter(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                            double* __restrict__ dst) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * (int64_t)perm[s] + k] = src[3 * s + k];
  }
}

__global__ void __launch_bounds__(kBlock) k64_norm2(const double* __restrict__ a, int64_t n_pad, double* partials,
                                                    unsigned int* counter, double* out) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] = fma(a[3 * s + k], a[3 * s + k], acc[k]);
  }
  block_partials_f64<3>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x < 3) out[threadIdx.x] = res[threadIdx.x];
  }
}

}  // namespace

enum { C64_INIT = 0, C64_DELTA, C64_OMEGA, C64_XR, C64_RES, C64_NORM, C64_COUNT };

sph_status solve_fp64(sph_neighbors* H, const sph_visc_params* P, const sph_solve_opts* O, const double* b, double* x,
                      sph_solve_report* R, cudaStream_t st) {
  SPH_TRY(ensure_operator(H, P, st));
  SPH_TRY(ensure_workspace(H));
  const int64_t np = H->n_pad;
  for (int k = 0; k < 6; ++k) SPH_TRY(H->w64[k].alloc(3 * np));
  if (!H->counters64.p) {
    SPH_TRY(H->counters64.alloc(C64_COUNT));
    SPH_TRY_CUDA(cudaMemset(H->counters64.p, 0, C64_COUNT * sizeof(unsigned int)));
  }
  Vecs64 V{H->w64[0].p, H->w64[1].p, H->w64[2].p, H->w64[3].p, H->w64[4].p, H->w64[5].p, H->x64.p};
  const OpView op = op_view(H);
  SolverScalars* S = H->scal.p;
  unsigned int* C = H->counters64.p;
  auto rgrid = [&](int64_t items) {
    int64_t want = (items + kBlock - 1) / kBlock;
    if (want > H->red_grid) want = H->red_grid;
    return want < 1 ? 1 : (int)want;
  };
  const int grid_rows = rgrid(np), grid_slices = rgrid(H->nslices * 32);
  SPH_LAUNCH(k64_gather, grid_for(H, np), kBlock, 0, st)(b, H->perm.p, H->n, np, H->b64.p);
  SPH_LAUNCH(k64_gather, grid_for(H, np), kBlock, 0, st)(x, H->perm.p, H->n, np, H->x64.p);
  SPH_TRY_CUDA(cudaGetLastError());
  double* dev_dots = reinterpret_cast<double*>(S) + offsetof(SolverScalars, dots) / sizeof(double);
  SPH_LAUNCH(k64_norm2, grid_rows, kBlock, 0, st)(H->b64.p, np, H->partials.p, C + C64_NORM, dev_dots);
  double bb[3];
  SPH_TRY_CUDA(cudaMemcpyAsync(bb, dev_dots, sizeof(bb), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bb[0] + bb[1] + bb[2]);
  const double rtol = O->rtol > 0.0 ? O->rtol : 1e-6;
  const double eps_floor = O->eps_inner > 0.0 ? std::fmin(O->eps_inner, 1e-10) : 1e-12;
  const int maxit = O->maxit > 0 ? O->maxit : 10000;
  const int max_ref = O->max_refine > 0 ? O->max_refine : 20;
  const int chunk0 = O->chunk > 0 ? O->chunk : 8;
  const bool merged = O->merged_reductions != 0;

  std::memset(R, 0, sizeof(*R));
  int total_iters = 0, passes = 0;
  double rr[3] = {0, 0, 0};
  sph_status status = SPH_NOT_CONVERGED;
  for (int ref = 0;; ++ref) {
    launch_residual_f64(H, grid_slices, H->x64.p, H->b64.p, H->r64.p, H->partials.p, C + C64_RES, dev_dots, st);
    SPH_TRY_CUDA(cudaGetLastError());
    SPH_TRY_CUDA(cudaMemcpyAsync(rr, dev_dots, sizeof(rr), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    if (!std::isfinite(rr[0]) || !std::isfinite(rr[1]) || !std::isfinite(rr[2])) {
      set_error("sph_visc_solve: the true residual is not finite");
      status = SPH_ERR_NONFINITE;
      break;
    }
    const double rnorm = std::sqrt(rr[0] + rr[1] + rr[2]);
    if (rnorm <= rtol * bnorm) {
      status = SPH_OK;
      break;
    }
    if (ref >= max_ref || total_iters >= maxit) break;
    const double eps = std::fmax(eps_floor, 0.25 * rtol * bnorm / rnorm);
    SPH_LAUNCH(k64_pass_init, grid_rows, kBlock, 0, st)(H->r64.p, H->D64.p, np, V, eps * eps, maxit - total_iters, S,
                                                        H->partials.p, C + C64_INIT);
    if (merged) SPH_LAUNCH(k64_p_update, grid_rows, kBlock, 0, st)(np, V, S);
    int chunk = chunk0;
    for (;;) {
      for (int it = 0; it < chunk; ++it) {
        if (!merged) SPH_LAUNCH(k64_p_update, grid_rows, kBlock, 0, st)(np, V, S);
        SPH_LAUNCH(k64_apply_dot<P64_DELTA>, grid_slices, kBlock, 0, st)(op, H->op_lo.p, H->D64.p, V.p, V.Ap, V.rh,
                                                                         S, H->partials.p, C + C64_DELTA);
        SPH_LAUNCH(k64_rstar, grid_rows, kBlock, 0, st)(np, V, S);
        if (merged) {
          SPH_LAUNCH(k64_apply_dot<P64_OMEGA_MERGED>, grid_slices, kBlock, 0, st)(
              op, H->op_lo.p, H->D64.p, V.rs, V.As, V.rh, S, H->partials.p, C + C64_OMEGA);
          SPH_LAUNCH(k64_xr_update<true>, grid_rows, kBlock, 0, st)(np, V, S, H->partials.p, C + C64_XR);
        } else {
          SPH_LAUNCH(k64_apply_dot<P64_OMEGA>, grid_slices, kBlock, 0, st)(op, H->op_lo.p, H->D64.p, V.rs, V.As,
                                                                           V.rh, S, H->partials.p, C + C64_OMEGA);
          SPH_LAUNCH(k64_xr_update<false>, grid_rows, kBlock, 0, st)(np, V, S, H->partials.p, C + C64_XR);
        }
      }
      SPH_TRY_CUDA(cudaGetLastError());
      SPH_TRY_CUDA(cudaMemcpyAsync(H->host_scal, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
      SPH_TRY_CUDA(cudaStreamSynchronize(st));
      if (H->host_scal->done) break;
      chunk = chunk < 64 ? chunk * 2 : chunk;
    }
    const SolverScalars& hs = *H->host_scal;
    total_iters += hs.iter;
    passes++;
    for (int c = 0; c < 3; ++c) {
      R->state[c] = (int8_t)hs.state[c];
      R->stalled_any[c] |= (int8_t)hs.stalled_any[c];
    }
    if (hs.iter == 0) break;
  }
  SPH_LAUNCH(k64_scatter, grid_for(H, H->n), kBlock, 0, st)(H->x64.p, H->perm.p, H->n, x);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  R->iters = total_iters;
  R->refinements = passes;
  R->true_rel_res = bnorm > 0.0 ? std::sqrt(rr[0] + rr[1] + rr[2]) / bnorm : std::sqrt(rr[0] + rr[1] + rr[2]);
  for (int c = 0; c < 3; ++c) R->true_rel_res_c[c] = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : std::sqrt(rr[c]);
  R->status = status;
  if (status == SPH_NOT_CONVERGED)
    set_error("sph_visc_solve (fp64): true residual %.3e above rtol %.1e after %d iterations", R->true_rel_res, rtol,
              total_iters);
  return status;
}

}  // namespace sph
