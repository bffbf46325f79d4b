// Per-row preconditioner scale on top of the Jacobi diagonal.
//
// The solves precondition A x = b from the left by D^-1 (App. B); a row scale s
// turns that into S D^-1 with S = diag(s), s > 0: the inner iteration then works
// on (S D^-1 A) d = S D^-1 r, whose solution is the same d, while the stopping
// test stays on the float64 true residual of A x = b.  This is the diagonal
// preconditioner-scale alternative to the learned warm start: a scale per
// particle (the three velocity components share the operator, so a diagonal
// block is one number) held fixed during a solve.
//
// Also here: the squared norms of the rows of D^-1 A, 1 + sum_j (a_j / D)^2 over
// a fluid row's coefficients (1 + sum_j S_j^2 over a dummy-wall row's Shepard
// weights, 1 for an identity row); the closed-form scale, factor x norm2^-power on
// the dummy-wall rows only; and the learned scale, the warm-start network's
// architecture evaluated on the same 16 features, whose first output is the log of
// a wall row's scale.
#include <cuda_bf16.h>

#include <cmath>

#include "apply.cuh"
#include "sph_internal.cuh"

namespace sph {
namespace {

// learned scales are exp(y) with y clamped to this range
constexpr float kLogScaleMin = -8.f, kLogScaleMax = 2.f;

// squared norm of sorted row s of D^-1 A from the stored float32 coefficients
__device__ __forceinline__ float row_norm2(const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                                           const int2* __restrict__ ih, const float* __restrict__ invD, int64_t s) {
  const int2* p = ih + off[s / kSlice] + s % kSlice;
  const int c = cnt[s];
  float acc = 0.f;
  for (int j = 0; j < c; ++j) {
    const float a = __int_as_float(p[(int64_t)j * kSlice].y);
    acc = fmaf(a, a, acc);
  }
  const float w = invD[s];
  return fmaf(w * w, acc, 1.f);
}

// out[perm[s]] = squared norm of row s of D^-1 A (mode 0), or the wall scale:
// 1 on fluid and identity rows, factor norm2^-power on Shepard rows (mode 1)
__global__ void k_row_norms(const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                            const int2* __restrict__ ih, const uint8_t* __restrict__ kind,
                            const float* __restrict__ invD, const int32_t* __restrict__ perm, int64_t n, int mode,
                            float factor, float power, float* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float v;
    if (mode == 0) {
      v = row_norm2(off, cnt, ih, invD, s);
    } else {
      v = kind[s] == KIND_SHEPARD ? (power != 0.f ? factor * powf(row_norm2(off, cnt, ih, invD, s), -power) : factor)
                                  : 1.f;
    }
    out[perm[s]] = v;
  }
}

// training targets of the learned scale: (log of the closed-form wall scale, 0, 0, 0)
// and the mask of the wall rows (caller order)
__global__ void k_scale_targets(const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                                const int2* __restrict__ ih, const uint8_t* __restrict__ kind,
                                const float* __restrict__ invD, const uint8_t* __restrict__ type,
                                const int32_t* __restrict__ perm, int64_t n, float log_factor, float power,
                                float4* __restrict__ tgt, uint8_t* __restrict__ mask) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const float t = kind[s] == KIND_SHEPARD
                        ? log_factor - (power != 0.f ? power * logf(row_norm2(off, cnt, ih, invD, s)) : 0.f)
                        : 0.f;
    const int64_t i = perm[s];
    tgt[i] = make_float4(t, 0.f, 0.f, 0.f);
    mask[i] = type[s] == SPH_FLUID ? 0 : 1;
  }
}

// the learned scale from the network's outputs y (caller order): exp of the
// clamped first output on wall rows, 1 on fluid rows
__global__ void k_scale_from_net(const float4* __restrict__ y, const uint8_t* __restrict__ type,
                                 const int32_t* __restrict__ perm, int64_t n, float* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[s];
    out[i] = type[s] == SPH_FLUID ? 1.f : expf(fminf(fmaxf(y[i].x, kLogScaleMin), kLogScaleMax));
  }
}

// flag[0] = 1 when some s[i] is not a positive finite number
__global__ void k_rs_check(const float* __restrict__ sc, int64_t n, int32_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = sc[i];
    if (!(v > 0.f) || !isfinite(v)) atomicExch(flag, 1);
  }
}

// scaled diagonals of the sorted rows; padding rows keep theirs
__global__ void k_rs_apply(const float* __restrict__ rs, const int32_t* __restrict__ perm,
                           const float* __restrict__ invD, const double* __restrict__ D64, int64_t n, int64_t n_pad,
                           float* __restrict__ invD_sc, double* __restrict__ D64_sc) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const float sc = s < n ? rs[perm[s]] : 1.f;
    invD_sc[s] = invD[s] * sc;
    D64_sc[s] = D64[s] / (double)sc;
  }
}

sph_status row_norms_impl(sph_neighbors* H, const sph_visc_params* P, int mode, double factor, double power,
                          float* out, cudaStream_t st) {
  SPH_TRY(ensure_operator(H, P, st));
  SPH_LAUNCH(k_row_norms, grid_for(H, H->n), kBlock, 0, st)(H->op_off.p, H->op_cnt.p, H->op_ih.p, H->op_kind.p,
                                                             H->invD.p, H->perm.p, H->n, mode, (float)factor,
                                                             (float)power, out);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace

sph_status features_impl(sph_neighbors* H, const sph_visc_params* P, const float* vel, __nv_bfloat16* feats,
                         cudaStream_t st, bool walls_only);
sph_status mlp_forward_launch(const sph_mlp* M, const __nv_bfloat16* feats, int64_t m, float4* out, int num_sms,
                              cudaStream_t st);

sph_status row_scale_refresh(sph_neighbors* H, cudaStream_t st) {
  if (!H->row_scaled || H->rs_op_version == H->op_version) return SPH_OK;
  SPH_TRY(H->invD_sc.alloc(H->n_pad));
  SPH_TRY(H->D64_sc.alloc(H->n_pad));
  SPH_LAUNCH(k_rs_apply, grid_for(H, H->n_pad), kBlock, 0, st)(H->rs_caller.p, H->perm.p, H->invD.p, H->D64.p, H->n,
                                                                H->n_pad, H->invD_sc.p, H->D64_sc.p);
  SPH_TRY_CUDA(cudaGetLastError());
  H->rs_op_version = H->op_version;
  return SPH_OK;
}

}  // namespace sph

using namespace sph;

extern "C" {

sph_status sph_row_norms(sph_neighbors* h, const sph_visc_params* params, float* norm2, void* stream) {
  clear_error();
  if (!h || !params || !norm2) {
    set_error("sph_row_norms: null argument");
    return SPH_ERR_INVALID;
  }
  return row_norms_impl(h, params, 0, 1.0, 0.0, norm2, reinterpret_cast<cudaStream_t>(stream));
}

static bool scale_args_ok(const char* fn, double factor, double power) {
  if (!std::isfinite(power) || power < 0.0 || power > 64.0 || !std::isfinite(factor) || !(factor >= 1e-6) ||
      factor > 1e6) {
    set_error("%s: factor %g outside [1e-6, 1e6] or power %g outside [0, 64]", fn, factor, power);
    return false;
  }
  return true;
}

sph_status sph_wall_row_scale(sph_neighbors* h, const sph_visc_params* params, double factor, double power,
                              float* scale, void* stream) {
  clear_error();
  if (!h || !params || !scale) {
    set_error("sph_wall_row_scale: null argument");
    return SPH_ERR_INVALID;
  }
  if (!scale_args_ok("sph_wall_row_scale", factor, power)) return SPH_ERR_INVALID;
  return row_norms_impl(h, params, 1, factor, power, scale, reinterpret_cast<cudaStream_t>(stream));
}

sph_status sph_set_row_scale(sph_neighbors* h, const float* scale, void* stream) {
  clear_error();
  if (!h) {
    set_error("sph_set_row_scale: null handle");
    return SPH_ERR_INVALID;
  }
  ++h->rs_version;
  if (!scale) {
    h->row_scaled = false;
    return SPH_OK;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(h->rs_caller.alloc(h->n));
  SPH_TRY_CUDA(cudaMemsetAsync(h->flags.p, 0, sizeof(int32_t), st));
  SPH_LAUNCH(k_rs_check, grid_for(h, h->n), kBlock, 0, st)(scale, h->n, h->flags.p);
  SPH_TRY_CUDA(cudaGetLastError());
  int32_t f = 0;
  SPH_TRY_CUDA(cudaMemcpyAsync(&f, h->flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  if (f) {
    h->row_scaled = false;
    set_error("sph_set_row_scale: a scale is not a positive finite number");
    return SPH_ERR_NONFINITE;
  }
  SPH_TRY_CUDA(cudaMemcpyAsync(h->rs_caller.p, scale, (size_t)h->n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  h->row_scaled = true;
  h->rs_op_version = ~0ull;
  return SPH_OK;
}

sph_status sph_mlp_scale_targets(sph_neighbors* h, const sph_visc_params* params, double factor, double power,
                                 float* targets, uint8_t* mask, void* stream) {
  clear_error();
  if (!h || !params || !targets || !mask) {
    set_error("sph_mlp_scale_targets: null argument");
    return SPH_ERR_INVALID;
  }
  if (!scale_args_ok("sph_mlp_scale_targets", factor, power)) return SPH_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(ensure_operator(h, params, st));
  SPH_LAUNCH(k_scale_targets, grid_for(h, h->n), kBlock, 0, st)(h->op_off.p, h->op_cnt.p, h->op_ih.p, h->op_kind.p,
                                                                 h->invD.p, h->type_s.p, h->perm.p, h->n,
                                                                 (float)std::log(factor), (float)power,
                                                                 reinterpret_cast<float4*>(targets), mask);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

sph_status sph_mlp_row_scale(sph_neighbors* h, const sph_visc_params* params, const sph_mlp* mlp, const float* vel,
                             float* scale, void* stream) {
  clear_error();
  if (!h || !params || !mlp || !vel) {
    set_error("sph_mlp_row_scale: null argument");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(h->feat_out.alloc(h->n * 8));      // bf16 features [n][16]
  SPH_TRY(h->feat_delta.alloc(h->n));        // float4 network outputs
  __nv_bfloat16* f = reinterpret_cast<__nv_bfloat16*>(h->feat_out.p);
  SPH_TRY(features_impl(h, params, vel, f, st, true));   // only the wall rows' scales are used
  SPH_TRY(mlp_forward_launch(mlp, f, h->n, h->feat_delta.p, h->num_sms, st));
  // without an output array the scale goes straight into the handle: exp of a clamped
  // value (NaN clamps to the lower bound) is positive and finite, so unlike
  // sph_set_row_scale nothing needs checking and nothing synchronises
  float* out = scale;
  if (!out) {
    SPH_TRY(h->rs_caller.alloc(h->n));
    out = h->rs_caller.p;
  }
  SPH_LAUNCH(k_scale_from_net, grid_for(h, h->n), kBlock, 0, st)(h->feat_delta.p, h->type_s.p, h->perm.p, h->n, out);
  SPH_TRY_CUDA(cudaGetLastError());
  if (!scale) {
    ++h->rs_version;
    h->row_scaled = true;
    h->rs_op_version = ~0ull;
  }
  return SPH_OK;
}

}  // extern "C"
