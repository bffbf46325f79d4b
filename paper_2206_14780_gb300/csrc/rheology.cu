// Shear-rate-dependent viscosity (paper Sec. 2.1 Eq. papa and Sec. 2.4), lagged:
// computed from the previous step's velocities so the viscous system stays
// linear (Sec. 3.3).
//
//   grad u_b = sum_a V_a |F_ab| r_ab (x) u_ab       V_a = m_a / rho_a
//   gdot = (grad u + grad u^T) / 2,  D = sqrt(2 gdot:gdot)
//   mu_b = tau0 Ybar(D) + mu0
//   Ybar(D) = m T(m D)           for m D < 0.5   (T: 8-term Horner series)
//           = (1 - e^{-m D}) / D  otherwise
// One thread per fluid row, float32 sums over the neighbour list; wall
// neighbours contribute their prescribed wall velocity.
#include <cmath>

#include "sph_internal.cuh"

namespace sph {

namespace {

__global__ void k_set_mu(const float* __restrict__ mu, const int32_t* __restrict__ perm, int64_t n,
                         float* __restrict__ mu_s, int32_t* __restrict__ flags) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const float m = mu[perm[s]];
    if (!(isfinite(m) && m > 0.f)) atomicOr(&flags[0], 1);
    mu_s[s] = m;
  }
}

// T(x) = 1 - x/2 (1 - x/3 (... (1 - x/7 (1 - x/8)) ...)), the MacLaurin series of
// (1 - e^-x)/x truncated after 8 terms (Sec. 2.4)
__device__ __forceinline__ float series_T(float x) {
  float t = 1.f;
  t = fmaf(-x * (1.f / 8.f), t, 1.f);
  t = fmaf(-x * (1.f / 7.f), t, 1.f);
  t = fmaf(-x * (1.f / 6.f), t, 1.f);
  t = fmaf(-x * (1.f / 5.f), t, 1.f);
  t = fmaf(-x * (1.f / 4.f), t, 1.f);
  t = fmaf(-x * (1.f / 3.f), t, 1.f);
  t = fmaf(-x * (1.f / 2.f), t, 1.f);
  return t;
}

struct MuGeom {
  float L[3], invL[3];
  int periodic[3];
  float inv_h;
  float absf_scale;  // |f| constant / h^5: 105/(128 pi) (Wendland) or 2 / w_G (Gaussian)
  int gauss;         // 1: truncated Gaussian, |f| ~ e^{-q^2}; 0: Wendland, |f| ~ (2 - q)^3
};

__global__ void __launch_bounds__(kBlock) k_mu_pass(const float4* __restrict__ pos_s, const float* __restrict__ rho_s,
                                                    const uint8_t* __restrict__ type_s,
                                                    const int32_t* __restrict__ cnt,
                                                    const int64_t* __restrict__ slice_off,
                                                    const int32_t* __restrict__ nbr,
                                                    const int32_t* __restrict__ perm, const float4* __restrict__ vel,
                                                    const float4* __restrict__ wall_vel, int64_t n, MuGeom g,
                                                    float tau0, float mu0, float mreg, float* __restrict__ mu_out,
                                                    float* __restrict__ mu_s) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ib = perm[s];
    if (type_s[s] != SPH_FLUID) {
      mu_out[ib] = mu0;
      if (mu_s) mu_s[s] = mu0;
      continue;
    }
    const float4 pb = pos_s[s];
    const float4 ub = vel[ib];
    float G[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      const float4 pa = pos_s[t];
      const int32_t ia = perm[t];
      const float4 ua = (type_s[t] == SPH_FLUID) ? vel[ia] : wall_vel[ia];
      float d[3] = {pa.x - pb.x, pa.y - pb.y, pa.z - pb.z};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax)
        if (g.periodic[ax]) d[ax] -= g.L[ax] * rintf(d[ax] * g.invL[ax]);
      const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const float q = r * g.inv_h;
      const float tq = fmaxf(2.f - q, 0.f);
      const float kq = g.gauss ? expf(-q * q) : tq * tq * tq;
      const float w = (pa.w / rho_s[t]) * g.absf_scale * kq;
      const float du[3] = {ua.x - ub.x, ua.y - ub.y, ua.z - ub.z};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int k = 0; k < 3; ++k) G[i][k] = fmaf(w * d[i], du[k], G[i][k]);
      }
    }
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float e = 0.5f * (G[i][k] + G[k][i]);
        ss = fmaf(e, e, ss);
      }
    }
    const float D = sqrtf(2.f * ss);
    const float x = mreg * D;
    const float Y = (x < 0.5f) ? mreg * series_T(x) : -expm1f(-x) / D;
    const float mu = fmaf(tau0, Y, mu0);
    mu_out[ib] = mu;
    if (mu_s) mu_s[s] = mu;
  }
}

}  // namespace

sph_status set_viscosity_impl(sph_neighbors* H, const float* mu, cudaStream_t st) {
  SPH_TRY_CUDA(cudaMemsetAsync(H->flags.p, 0, sizeof(int32_t), st));
  SPH_LAUNCH(k_set_mu, grid_for(H, H->n), kBlock, 0, st)(mu, H->perm.p, H->n, H->mu_s.p, H->flags.p);
  SPH_TRY_CUDA(cudaGetLastError());
  int32_t f = 0;
  SPH_TRY_CUDA(cudaMemcpyAsync(&f, H->flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  H->mu_version++;
  if (f) {
    set_error("sph_set_viscosity: non-finite or non-positive viscosity");
    return SPH_ERR_NONFINITE;
  }
  return SPH_OK;
}

sph_status mu_papanastasiou(sph_neighbors* H, const float* vel, const float* wall_vel, double tau0, double mu0,
                            double m, float* mu_out, int set_handle, cudaStream_t st) {
  MuGeom g{};
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = (float)H->grid.L[ax];
    g.invL[ax] = (float)(1.0 / H->grid.L[ax]);
    g.periodic[ax] = H->grid.periodic[ax];
  }
  const double h = (double)H->h;
  g.inv_h = (float)(1.0 / h);
  g.gauss = H->kernel == SPH_KERNEL_GAUSSIAN ? 1 : 0;
  g.absf_scale = (float)((g.gauss ? 2.0 / gauss_norm() : 105.0 / (128.0 * M_PI)) / (h * h * h * h * h));
  SPH_LAUNCH(k_mu_pass, grid_for(H, H->n), kBlock, 0, st)(
      H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p, H->slice_off.p, H->nbr.p, H->perm.p,
      reinterpret_cast<const float4*>(vel), reinterpret_cast<const float4*>(wall_vel), H->n, g, (float)tau0,
      (float)mu0, (float)m, mu_out, set_handle ? H->mu_s.p : nullptr);
  SPH_TRY_CUDA(cudaGetLastError());
  if (set_handle) H->mu_version++;
  return SPH_OK;
}

}  // namespace sph
