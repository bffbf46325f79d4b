// Per-particle features of the learned warm start and the warm-start x0.
//
// Sixteen features per particle (bf16, caller order), velocities scaled by
// U = RMS of |v^n| over the fluid:
//   0-2   v / U
//   3-5   e1 / U,  e1 = D^-1 (v - A v)         explicit viscous increment
//                                               dt L v, Jacobi-scaled (fluid rows)
//   6-8   e2 / U,  e2 = D^-1 (e1 - A e1)       the next (second Neumann) term
//   9     log10(mu) / 5
//   10    log10(D) / 4, D = 1 + dt sum c        local stiffness
//   11    distance to the nearest wall neighbour / (2h), 1 without one
//   12    Shepard sum over fluid neighbours and self of W V
//   13    neighbour count / 80
//   14    |v_b| / (|v_b| + RMS of |v_a| over the neighbours)
//   15    1 for wall particles
// Wall rows get zeros in 3-8 (their operator rows are not the viscous term).
#include <cuda_bf16.h>

#include <cmath>

#include "reduce.cuh"
#include "sph_internal.cuh"

struct sph_mlp;

namespace sph {

sph_status mlp_forward_launch(const sph_mlp* M, const __nv_bfloat16* feats, int64_t m, float4* out, int num_sms,
                              cudaStream_t st);
int mlp_mode(const sph_mlp* M);

namespace {

__global__ void k_feat_gather(const float4* __restrict__ v, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                              float4* __restrict__ vs) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      const float4 t = v[perm[s]];
      vs[s] = make_float4(t.x, t.y, t.z, 0.f);
    } else {
      vs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// e = D^-1 (v - y) on fluid rows, 0 elsewhere
__global__ void k_feat_incr(const float4* __restrict__ v, const float4* __restrict__ y, const float* __restrict__ invD,
                            const uint8_t* __restrict__ type, int64_t n, int64_t n_pad, float4* __restrict__ e) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n && type[s] == SPH_FLUID) {
      const float4 a = v[s], b = y[s];
      const float d = invD[s];
      e[s] = make_float4((a.x - b.x) * d, (a.y - b.y) * d, (a.z - b.z) * d, 0.f);
    } else {
      e[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// sum over fluid rows of |v|^2 and their count -> out[0], out[1]
__global__ void __launch_bounds__(kBlock) k_feat_scale(const float4* __restrict__ v, const uint8_t* __restrict__ type,
                                                       int64_t n, double* partials, unsigned int* counter,
                                                       double* out) {
  double acc[2] = {0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (type[s] == SPH_FLUID) {
      const float4 a = v[s];
      acc[0] += (double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z;
      acc[1] += 1.0;
    }
  }
  block_partials_f64<2>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[2];
    final_sum<2>(partials, counter, res);
    if (threadIdx.x < 2) out[threadIdx.x] = res[threadIdx.x];
  }
}

// d_i <- d_i - (S d)_i on fluid rows (caller order in and out, thread per sorted
// row): the Shepard average over fluid neighbours and the particle itself
__global__ void __launch_bounds__(kBlock) k_highpass(const float4* __restrict__ pos, const float* __restrict__ rho,
                                                     const uint8_t* __restrict__ type,
                                                     const int32_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ slice_off,
                                                     const int32_t* __restrict__ nbr, const int32_t* __restrict__ perm,
                                                     int64_t n, float L0, float L1, float L2, float iL0, float iL1,
                                                     float iL2, int p0, int p1, int p2, float inv_h,
                                                     const float4* __restrict__ d, float4* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[s];
    const float4 di = d[i];
    if (type[s] != SPH_FLUID) {
      out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float4 pb = pos[s];
    float wsum = pb.w / rho[s];   // W(0) = 1 in the units of the weights below
    float sx = wsum * di.x, sy = wsum * di.y, sz = wsum * di.z;
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      if (type[t] != SPH_FLUID) continue;
      const float4 pa = pos[t];
      float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
      if (p0) dx -= L0 * rintf(dx * iL0);
      if (p1) dy -= L1 * rintf(dy * iL1);
      if (p2) dz -= L2 * rintf(dz * iL2);
      const float q = sqrtf(dx * dx + dy * dy + dz * dz) * inv_h;
      const float tw = fmaxf(1.f - 0.5f * q, 0.f);
      const float tw2 = tw * tw;
      const float w = tw2 * tw2 * fmaf(2.f, q, 1.f) * (pa.w / rho[t]);   // Wendland, constant factor dropped
      const float4 da = d[perm[t]];
      sx = fmaf(w, da.x, sx);
      sy = fmaf(w, da.y, sy);
      sz = fmaf(w, da.z, sz);
      wsum += w;
    }
    const float iw = 1.f / wsum;
    out[i] = make_float4(di.x - sx * iw, di.y - sy * iw, di.z - sz * iw, 0.f);
  }
}

// Shepard denominators N_s = sum over {s} and its fluid neighbours of W V (sorted,
// fluid rows; 1 on walls), in the weights of k_highpass
__global__ void __launch_bounds__(kBlock) k_shep_den(const float4* __restrict__ pos, const float* __restrict__ rho,
                                                     const uint8_t* __restrict__ type,
                                                     const int32_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ slice_off,
                                                     const int32_t* __restrict__ nbr, int64_t n, float L0, float L1,
                                                     float L2, float iL0, float iL1, float iL2, int p0, int p1, int p2,
                                                     float inv_h, float* __restrict__ den) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (type[s] != SPH_FLUID) {
      den[s] = 1.f;
      continue;
    }
    const float4 pb = pos[s];
    float wsum = pb.w / rho[s];
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      if (type[t] != SPH_FLUID) continue;
      const float4 pa = pos[t];
      float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
      if (p0) dx -= L0 * rintf(dx * iL0);
      if (p1) dy -= L1 * rintf(dy * iL1);
      if (p2) dz -= L2 * rintf(dz * iL2);
      const float q = sqrtf(dx * dx + dy * dy + dz * dz) * inv_h;
      const float tw = fmaxf(1.f - 0.5f * q, 0.f);
      const float tw2 = tw * tw;
      wsum += tw2 * tw2 * fmaf(2.f, q, 1.f) * (pa.w / rho[t]);
    }
    den[s] = wsum;
  }
}

// out_b = q_b - (S^T q)_b on fluid rows (sorted), (S^T q)_b = V_b sum over a in {b}
// and the fluid neighbours of b of W_ab q_a / N_a; 0 on walls
__global__ void __launch_bounds__(kBlock) k_highpass_T(const float4* __restrict__ pos, const float* __restrict__ rho,
                                                       const uint8_t* __restrict__ type,
                                                       const int32_t* __restrict__ cnt,
                                                       const int64_t* __restrict__ slice_off,
                                                       const int32_t* __restrict__ nbr, int64_t n, float L0, float L1,
                                                       float L2, float iL0, float iL1, float iL2, int p0, int p1,
                                                       int p2, float inv_h, const float* __restrict__ den,
                                                       const float4* __restrict__ q, float4* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (type[s] != SPH_FLUID) {
      out[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float4 pb = pos[s];
    const float4 qb = q[s];
    const float ib = 1.f / den[s];
    float sx = qb.x * ib, sy = qb.y * ib, sz = qb.z * ib;   // the a = b term, W(0) = 1
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      if (type[t] != SPH_FLUID) continue;
      const float4 pa = pos[t];
      float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
      if (p0) dx -= L0 * rintf(dx * iL0);
      if (p1) dy -= L1 * rintf(dy * iL1);
      if (p2) dz -= L2 * rintf(dz * iL2);
      const float qq = sqrtf(dx * dx + dy * dy + dz * dz) * inv_h;
      const float tw = fmaxf(1.f - 0.5f * qq, 0.f);
      const float tw2 = tw * tw;
      const float w = tw2 * tw2 * fmaf(2.f, qq, 1.f) / den[t];
      const float4 qa = q[t];
      sx = fmaf(w, qa.x, sx);
      sy = fmaf(w, qa.y, sy);
      sz = fmaf(w, qa.z, sz);
    }
    const float Vb = pb.w / rho[s];
    out[s] = make_float4(qb.x - Vb * sx, qb.y - Vb * sy, qb.z - Vb * sz, 0.f);
  }
}

struct FeatGeom {
  float L[3], invL[3];
  int periodic[3];
  float inv_h, inv_2h, w_scale;  // Wendland: w_scale = 21/(16 pi) / h^3
  int gauss;                     // truncated Gaussian: W = w_scale (e^{-q^2} - g_tail), w_scale = 1/(w_G h^3)
  float g_tail;
};

// W(r) of the handle's kernel for q = r / h inside the support
__device__ __forceinline__ float feat_w(const FeatGeom& g, float q) {
  if (g.gauss) return g.w_scale * (__expf(-q * q) - g.g_tail);
  const float tq = fmaxf(1.f - 0.5f * q, 0.f);
  const float t2 = tq * tq;
  return g.w_scale * t2 * t2 * (2.f * q + 1.f);
}

__global__ void __launch_bounds__(kBlock) k_features(const float4* __restrict__ pos, const float* __restrict__ rho,
                                                     const float* __restrict__ mu, const uint8_t* __restrict__ type,
                                                     const double* __restrict__ D64,
                                                     const int32_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ slice_off,
                                                     const int32_t* __restrict__ nbr, const int32_t* __restrict__ perm,
                                                     const float4* __restrict__ v, const float4* __restrict__ e1,
                                                     const float4* __restrict__ e2, int64_t n, FeatGeom g,
                                                     const double* __restrict__ scale, int walls_only,
                                                     __nv_bfloat16* __restrict__ feats) {
  const float U = (float)sqrt(scale[0] / fmax(scale[1], 1.0));
  const float iU = U > 0.f ? 1.f / U : 0.f;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (walls_only && type[s] == SPH_FLUID) {   // zeros: the caller reads the wall rows only
      uint4* out = reinterpret_cast<uint4*>(feats + (int64_t)perm[s] * 16);
      out[0] = make_uint4(0u, 0u, 0u, 0u);
      out[1] = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    const float4 pb = pos[s];
    const float4 vb = v[s];
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    float dmin = 1.f, shep = feat_w(g, 0.f) * (pb.w / rho[s]), v2 = 0.f;
    double dsum = 0.0;   // D over the fluid neighbours (feature 10 of a wall row)
    int nfl = 0;
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      const float4 pa = pos[t];
      float d[3] = {pa.x - pb.x, pa.y - pb.y, pa.z - pb.z};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax)
        if (g.periodic[ax]) d[ax] -= g.L[ax] * rintf(d[ax] * g.invL[ax]);
      const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (type[t] == SPH_FLUID) {
        shep += feat_w(g, r * g.inv_h) * (pa.w / rho[t]);
        dsum += D64[t];
        ++nfl;
      } else {
        dmin = fminf(dmin, r * g.inv_2h);
      }
      const float4 va = v[t];
      v2 += va.x * va.x + va.y * va.y + va.z * va.z;
    }
    const bool fluid = type[s] == SPH_FLUID;
    const float vn = sqrtf(vb.x * vb.x + vb.y * vb.y + vb.z * vb.z);
    const float rms = c > 0 ? sqrtf(v2 / (float)c) : 0.f;
    float f[16];
    f[0] = vb.x * iU;
    f[1] = vb.y * iU;
    f[2] = vb.z * iU;
    const float4 a = e1[s], b = e2[s];
    f[3] = fluid ? a.x * iU : 0.f;
    f[4] = fluid ? a.y * iU : 0.f;
    f[5] = fluid ? a.z * iU : 0.f;
    f[6] = fluid ? b.x * iU : 0.f;
    f[7] = fluid ? b.y * iU : 0.f;
    f[8] = fluid ? b.z * iU : 0.f;
    f[9] = log10f(mu[s]) * 0.2f;
    // log10 D / 4; on a wall row (D = 1) the mean D of its fluid neighbours, the
    // stiffness its row couples to
    f[10] = (float)(log10(fluid ? D64[s] : (nfl > 0 ? dsum / nfl : 1.0)) * 0.25);
    f[11] = dmin;
    f[12] = shep;
    f[13] = (float)c * (1.f / 80.f);
    f[14] = (vn + rms) > 0.f ? vn / (vn + rms) : 0.f;
    f[15] = fluid ? 0.f : 1.f;
    __nv_bfloat16* out = feats + (int64_t)perm[s] * 16;
#pragma unroll
    for (int k = 0; k < 16; k += 2)
      *reinterpret_cast<__nv_bfloat162*>(out + k) = __floats2bfloat162_rn(f[k], f[k + 1]);
  }
}

// x0 = v + U delta on fluid rows (v alone when delta is null), b on walls (caller order)
__global__ void k_warm_x0(const float4* __restrict__ vel, const float4* __restrict__ delta,
                          const uint8_t* __restrict__ ptype, const double* __restrict__ b, int64_t n,
                          const double* __restrict__ scale, double* __restrict__ x0) {
  const double U = delta ? sqrt(scale[0] / fmax(scale[1], 1.0)) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (ptype[i] == SPH_FLUID) {
      const float4 v = vel[i], d = delta ? delta[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      x0[3 * i] = (double)v.x + U * (double)d.x;
      x0[3 * i + 1] = (double)v.y + U * (double)d.y;
      x0[3 * i + 2] = (double)v.z + U * (double)d.z;
    } else {
      x0[3 * i] = b[3 * i];
      x0[3 * i + 1] = b[3 * i + 1];
      x0[3 * i + 2] = b[3 * i + 2];
    }
  }
}

// training targets (x* - v) / U and the fluid mask (caller order)
__global__ void k_targets(const float4* __restrict__ vel, const double* __restrict__ xs,
                          const uint8_t* __restrict__ ptype, int64_t n, const double* __restrict__ scale,
                          float4* __restrict__ tgt, uint8_t* __restrict__ mask) {
  const double U = sqrt(scale[0] / fmax(scale[1], 1.0));
  const double iU = U > 0.0 ? 1.0 / U : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = vel[i];
    const bool fl = ptype[i] == SPH_FLUID;
    tgt[i] = fl ? make_float4((float)((xs[3 * i] - v.x) * iU), (float)((xs[3 * i + 1] - v.y) * iU),
                              (float)((xs[3 * i + 2] - v.z) * iU), 0.f)
                : make_float4(0.f, 0.f, 0.f, 0.f);
    mask[i] = fl ? 1 : 0;
  }
}

// x0 (caller, double) -> sorted float4; wall rows zeroed when fluid_only
__global__ void k_x0_sorted(const double* __restrict__ x0, const int32_t* __restrict__ perm,
                            const uint8_t* __restrict__ type, int fluid_only, int64_t n, int64_t n_pad,
                            float4* __restrict__ xs) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n && (!fluid_only || type[s] == SPH_FLUID)) {
      const int64_t i = perm[s];
      xs[s] = make_float4((float)x0[3 * i], (float)x0[3 * i + 1], (float)x0[3 * i + 2], 0.f);
    } else {
      xs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// dummy-wall closure (Eq. dummyvel): x0_wall = b_wall - (A x~)_wall, where x~ is
// x0 with its wall rows zeroed, so A x~ on a wall row is the Shepard average of
// the fluid x0 (dynamic walls: identity rows, x0_wall = b)
__global__ void k_wall_close(const float4* __restrict__ Ax, const double* __restrict__ b,
                             const int32_t* __restrict__ perm, const uint8_t* __restrict__ type, int64_t n,
                             double* __restrict__ x0) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (type[s] != SPH_FLUID) {
      const int64_t i = perm[s];
      const float4 a = Ax[s];
      x0[3 * i] = b[3 * i] - (double)a.x;
      x0[3 * i + 1] = b[3 * i + 1] - (double)a.y;
      x0[3 * i + 2] = b[3 * i + 2] - (double)a.z;
    }
  }
}

// r = b - A x0 on fluid rows (sorted), weight w = 1/D (jacobi) or 1: z = w^2 r and
// out[0] = sum w^2 |r|^2, out[1] = sum |b|^2 over the fluid rows
__global__ void __launch_bounds__(kBlock) k_resid_z(const float4* __restrict__ Ax, const double* __restrict__ b,
                                                    const int32_t* __restrict__ perm,
                                                    const uint8_t* __restrict__ type, const float* __restrict__ invD,
                                                    int jacobi, int64_t n, int64_t n_pad, float4* __restrict__ z,
                                                    double* partials, unsigned int* counter, double* out) {
  double acc[2] = {0.0, 0.0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < n && type[s] == SPH_FLUID) {
      const int64_t i = perm[s];
      const float d = jacobi ? invD[s] : 1.f;
      const float4 a = Ax[s];
      const float rx = (float)b[3 * i] - a.x, ry = (float)b[3 * i + 1] - a.y, rz = (float)b[3 * i + 2] - a.z;
      acc[0] += (double)(rx * d) * (rx * d) + (double)(ry * d) * (ry * d) + (double)(rz * d) * (rz * d);
      acc[1] += b[3 * i] * b[3 * i] + b[3 * i + 1] * b[3 * i + 1] + b[3 * i + 2] * b[3 * i + 2];
      o = make_float4(rx * d * d, ry * d * d, rz * d * d, 0.f);
    }
    z[s] = o;
  }
  block_partials_f64<2>(acc, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[2];
    final_sum<2>(partials, counter, res);
    if (threadIdx.x < 2) out[threadIdx.x] = res[threadIdx.x];
  }
}

// pseudo-targets t = y + g (A z) on fluid rows (caller order), mask = fluid, with
// g = 1 / U for the plain loss and g = count U / sum w^2 |r|^2 for the log loss
__global__ void k_resid_targets(const float4* __restrict__ y, const float4* __restrict__ Az,
                                const int32_t* __restrict__ perm, const uint8_t* __restrict__ type, int64_t n,
                                const double* __restrict__ scale, const double* __restrict__ sums, int log_loss,
                                float4* __restrict__ tgt, uint8_t* __restrict__ mask) {
  const double U = sqrt(scale[0] / fmax(scale[1], 1.0));
  double g = 0.0;
  if (log_loss)
    g = sums[0] > 0.0 ? scale[1] * U / sums[0] : 0.0;
  else
    g = U > 0.0 ? 1.0 / U : 0.0;
  const float gf = (float)g;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[s];
    const bool fl = type[s] == SPH_FLUID;
    const float4 a = y[i], q = Az[s];
    tgt[i] = fl ? make_float4(a.x + q.x * gf, a.y + q.y * gf, a.z + q.z * gf, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    mask[i] = fl ? 1 : 0;
  }
}

}  // namespace

// features of the particle set on handle H for velocities vel (caller order);
// leaves the scale sums (|v|^2, count) in H->feat_scale (device).  walls_only:
// the wall rows' features alone (fluid rows zero); a wall row's Neumann
// increments are zero by definition, so the two operator applies are skipped
sph_status features_impl(sph_neighbors* H, const sph_visc_params* P, const float* vel, __nv_bfloat16* feats,
                         cudaStream_t st, bool walls_only) {
  SPH_TRY(ensure_operator(H, P, st));
  SPH_TRY(ensure_workspace(H));
  SPH_TRY(H->feat_tmp.alloc(4 * H->n_pad));
  SPH_TRY(H->feat_scale.alloc(2));
  const int64_t np = H->n_pad;
  float4* vs = H->feat_tmp.p;
  float4* y = vs + np;
  float4* e1 = vs + 2 * np;
  float4* e2 = vs + 3 * np;
  const int grid = grid_for(H, np);
  SPH_LAUNCH(k_feat_gather, grid, kBlock, 0, st)(reinterpret_cast<const float4*>(vel), H->perm.p, H->n, np, vs);
  if (!walls_only) {
    launch_apply_f32(H, vs, y, false, st);
    SPH_LAUNCH(k_feat_incr, grid, kBlock, 0, st)(vs, y, H->invD.p, H->type_s.p, H->n, np, e1);
    launch_apply_f32(H, e1, y, false, st);
    SPH_LAUNCH(k_feat_incr, grid, kBlock, 0, st)(e1, y, H->invD.p, H->type_s.p, H->n, np, e2);
  }
  int rg = grid < H->red_grid ? grid : H->red_grid;
  SPH_LAUNCH(k_feat_scale, rg, kBlock, 0, st)(vs, H->type_s.p, H->n, H->partials.p, H->counters.p + 7,
                                              H->feat_scale.p);
  FeatGeom g{};
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = (float)H->grid.L[ax];
    g.invL[ax] = (float)(1.0 / H->grid.L[ax]);
    g.periodic[ax] = H->grid.periodic[ax];
  }
  const double h = (double)H->h;
  g.inv_h = (float)(1.0 / h);
  g.inv_2h = (float)(0.5 / h);
  g.gauss = H->kernel == SPH_KERNEL_GAUSSIAN ? 1 : 0;
  g.w_scale = (float)(g.gauss ? 1.0 / (gauss_norm() * h * h * h) : 21.0 / (16.0 * M_PI) / (h * h * h));
  g.g_tail = (float)std::exp(-kGaussK * kGaussK);
  SPH_LAUNCH(k_features, grid_for(H, H->n), kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->mu_s.p, H->type_s.p, H->D64.p,
                                                           H->cnt.p, H->slice_off.p, H->nbr.p, H->perm.p, vs, e1, e2,
                                                           H->n, g, H->feat_scale.p, walls_only ? 1 : 0, feats);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

// x0 (caller order, device double [n][3]) gets its dummy-wall rows from Eq.
// dummyvel given its fluid rows; uses feat_tmp slots 0 and 1
static void wall_closure(sph_neighbors* H, double* x0, const double* b, cudaStream_t st) {
  const int64_t np = H->n_pad;
  float4* xs = H->feat_tmp.p;
  float4* ax = xs + np;
  SPH_LAUNCH(k_x0_sorted, grid_for(H, np), kBlock, 0, st)(x0, H->perm.p, H->type_s.p, 1, H->n, np, xs);
  launch_apply_f32(H, xs, ax, false, st);
  SPH_LAUNCH(k_wall_close, grid_for(H, H->n), kBlock, 0, st)(ax, b, H->perm.p, H->type_s.p, H->n, x0);
}

// out = delta - S delta (SPH_MLP_HIGHPASS), caller order, out != delta
static void highpass(sph_neighbors* H, const float4* delta, float4* out, cudaStream_t st) {
  float L[3], iL[3];
  for (int k = 0; k < 3; ++k) {
    L[k] = (float)H->grid.L[k];
    iL[k] = (float)(1.0 / H->grid.L[k]);
  }
  SPH_LAUNCH(k_highpass, grid_for(H, H->n), kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p, H->slice_off.p,
                                                           H->nbr.p, H->perm.p, H->n, L[0], L[1], L[2], iL[0], iL[1],
                                                           iL[2], H->grid.periodic[0], H->grid.periodic[1],
                                                           H->grid.periodic[2], (float)(1.0 / (double)H->h), delta,
                                                           out);
}

// out = q - S^T q (sorted, fluid rows) with the Shepard denominators in den
static void highpass_T(sph_neighbors* H, const float4* q, float* den, float4* out, cudaStream_t st) {
  float L[3], iL[3];
  for (int k = 0; k < 3; ++k) {
    L[k] = (float)H->grid.L[k];
    iL[k] = (float)(1.0 / H->grid.L[k]);
  }
  const float ih = (float)(1.0 / (double)H->h);
  const int* pr = H->grid.periodic;
  SPH_LAUNCH(k_shep_den, grid_for(H, H->n), kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p,
                                                           H->slice_off.p, H->nbr.p, H->n, L[0], L[1], L[2], iL[0],
                                                           iL[1], iL[2], pr[0], pr[1], pr[2], ih, den);
  SPH_LAUNCH(k_highpass_T, grid_for(H, H->n), kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p,
                                                             H->slice_off.p, H->nbr.p, H->n, L[0], L[1], L[2], iL[0],
                                                             iL[1], iL[2], pr[0], pr[1], pr[2], ih, den, q, out);
}

}  // namespace sph

using namespace sph;

extern "C" {

sph_status sph_mlp_features(sph_neighbors* h, const sph_visc_params* params, const float* vel, uint16_t* feats,
                            double* scale_out, void* stream) {
  clear_error();
  if (!h || !params || !vel || !feats) {
    set_error("sph_mlp_features: null argument");
    return SPH_ERR_INVALID;
  }

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(features_impl(h, params, vel, reinterpret_cast<__nv_bfloat16*>(feats), st, false));
  if (scale_out) {
    double sc[2];
    SPH_TRY_CUDA(cudaMemcpyAsync(sc, h->feat_scale.p, sizeof(sc), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    *scale_out = std::sqrt(sc[0] / (sc[1] > 1.0 ? sc[1] : 1.0));
  }
  return SPH_OK;
}

sph_status sph_mlp_targets(sph_neighbors* h, const float* vel, const double* x_star, const uint8_t* ptype,
                           float* targets, uint8_t* mask, void* stream) {
  clear_error();
  if (!h || !vel || !x_star || !ptype || !targets || !mask || !h->feat_scale.p) {
    set_error("sph_mlp_targets: null argument (call sph_mlp_features first)");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_LAUNCH(k_targets, grid_for(h, h->n), kBlock, 0, st)(reinterpret_cast<const float4*>(vel), x_star, ptype, h->n,
                                                          h->feat_scale.p, reinterpret_cast<float4*>(targets), mask);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // extern "C"

namespace sph {
// x0 = v^n on fluid rows with the dummy-wall closure (sph_warm_start without a network)
sph_status warm_start_plain(sph_neighbors* h, const sph_visc_params* params, const float* vel, const uint8_t* ptype,
                            const double* b, double* x0, cudaStream_t st) {
  SPH_TRY(ensure_operator(h, params, st));
  SPH_TRY(ensure_workspace(h));
  SPH_TRY(h->feat_tmp.alloc(4 * h->n_pad));
  SPH_LAUNCH(k_warm_x0, grid_for(h, h->n), kBlock, 0, st)(reinterpret_cast<const float4*>(vel), nullptr, ptype, b,
                                                          h->n, h->feat_scale.p, x0);
  wall_closure(h, x0, b, st);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}
}  // namespace sph

extern "C" {

sph_status sph_warm_start(sph_neighbors* h, const sph_visc_params* params, const sph_mlp* mlp, const float* vel,
                          const uint8_t* ptype, const double* b, double* x0, void* stream) {
  clear_error();
  if (!h || !params || !vel || !ptype || !b || !x0) {
    set_error("sph_warm_start: null argument");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float4* delta = nullptr;
  if (mlp && h->kernel != SPH_KERNEL_WENDLAND) {
    set_error("sph_warm_start: the warm-start network takes Wendland-kernel scenes (pass no network)");
    return SPH_ERR_INVALID;
  }
  if (mlp) {
    SPH_TRY(h->feat_out.alloc(h->n * 8));      // bf16 features [n][16]
    SPH_TRY(h->feat_delta.alloc(h->n));        // float4 network outputs
    __nv_bfloat16* f = reinterpret_cast<__nv_bfloat16*>(h->feat_out.p);
    SPH_TRY(features_impl(h, params, vel, f, st, false));
    SPH_TRY(mlp_forward_launch(mlp, f, h->n, h->feat_delta.p, h->num_sms, st));
    delta = h->feat_delta.p;
    if (mlp_mode(mlp) & SPH_MLP_HIGHPASS) {
      SPH_TRY(h->feat_hp.alloc(h->n));
      highpass(h, h->feat_delta.p, h->feat_hp.p, st);
      delta = h->feat_hp.p;
    }
  } else {
    SPH_TRY(ensure_operator(h, params, st));
    SPH_TRY(ensure_workspace(h));
    SPH_TRY(h->feat_tmp.alloc(4 * h->n_pad));
  }
  SPH_LAUNCH(k_warm_x0, grid_for(h, h->n), kBlock, 0, st)(reinterpret_cast<const float4*>(vel), delta, ptype, b, h->n,
                                                          h->feat_scale.p, x0);
  wall_closure(h, x0, b, st);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

/* Residual-loss training targets (the declaration states the loss and the
   identity behind them).  Buffers: x64 holds x0 in caller order, feat_tmp slots
   0-3 the sorted x0, A x0, z and A z, r64[0..1] the two sums. */
sph_status sph_mlp_residual_targets(sph_neighbors* h, const sph_visc_params* params, const sph_mlp* mlp,
                                    const float* vel, const uint8_t* ptype, const double* b, int flags,
                                    uint16_t* feats, float* targets, uint8_t* mask, double* loss_host,
                                    void* stream) {
  clear_error();
  if (!h || !params || !mlp || !vel || !ptype || !b || !feats || !targets || !mask) {
    set_error("sph_mlp_residual_targets: null argument");
    return SPH_ERR_INVALID;
  }
  if (flags & ~(SPH_RLOSS_JACOBI | SPH_RLOSS_LOG)) {
    set_error("sph_mlp_residual_targets: unknown flags %d", flags);
    return SPH_ERR_INVALID;
  }
  if (h->kernel != SPH_KERNEL_WENDLAND) {
    set_error("sph_mlp_residual_targets: the warm-start network takes Wendland-kernel scenes");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  __nv_bfloat16* f = reinterpret_cast<__nv_bfloat16*>(feats);
  SPH_TRY(features_impl(h, params, vel, f, st, false));
  SPH_TRY(h->feat_delta.alloc(h->n));
  SPH_TRY(h->x64.alloc(3 * h->n_pad));
  SPH_TRY(h->r64.alloc(3 * h->n_pad));
  SPH_TRY(mlp_forward_launch(mlp, f, h->n, h->feat_delta.p, h->num_sms, st));
  const bool hp = (mlp_mode(mlp) & SPH_MLP_HIGHPASS) != 0;
  const float4* dx0 = h->feat_delta.p;
  if (hp) {
    SPH_TRY(h->feat_hp.alloc(h->n));
    SPH_TRY(h->feat_den.alloc(h->n_pad));
    highpass(h, h->feat_delta.p, h->feat_hp.p, st);
    dx0 = h->feat_hp.p;
  }
  double* x0 = h->x64.p;
  SPH_LAUNCH(k_warm_x0, grid_for(h, h->n), kBlock, 0, st)(reinterpret_cast<const float4*>(vel), dx0, ptype, b, h->n,
                                                          h->feat_scale.p, x0);
  wall_closure(h, x0, b, st);
  const int64_t np = h->n_pad;
  float4* xs = h->feat_tmp.p;
  float4* ax = xs + np;
  float4* z = xs + 2 * np;
  float4* az = xs + 3 * np;
  SPH_LAUNCH(k_x0_sorted, grid_for(h, np), kBlock, 0, st)(x0, h->perm.p, h->type_s.p, 0, h->n, np, xs);
  launch_apply_f32(h, xs, ax, false, st);
  const int rg = grid_for(h, np) < h->red_grid ? grid_for(h, np) : h->red_grid;
  double* sums = h->r64.p;
  SPH_LAUNCH(k_resid_z, rg, kBlock, 0, st)(ax, b, h->perm.p, h->type_s.p, h->invD.p, (flags & SPH_RLOSS_JACOBI) ? 1 : 0,
                                           h->n, np, z, h->partials.p, h->counters.p + 7, sums);
  launch_apply_f32(h, z, az, false, st);
  const float4* grad = az;
  if (hp) {                           // P^T = I - S^T in front of A z (slot 0 is free again)
    highpass_T(h, az, h->feat_den.p, xs, st);
    grad = xs;
  }
  SPH_LAUNCH(k_resid_targets, grid_for(h, h->n), kBlock, 0, st)(h->feat_delta.p, grad, h->perm.p, h->type_s.p, h->n,
                                                                h->feat_scale.p, sums, (flags & SPH_RLOSS_LOG) ? 1 : 0,
                                                                reinterpret_cast<float4*>(targets), mask);
  SPH_TRY_CUDA(cudaGetLastError());
  if (loss_host) {
    double v[4];
    SPH_TRY_CUDA(cudaMemcpyAsync(v, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaMemcpyAsync(v + 2, h->feat_scale.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    if (flags & SPH_RLOSS_LOG) {
      *loss_host = (v[0] > 0.0 && v[1] > 0.0) ? std::log(v[0] / v[1]) : 0.0;
    } else {
      const double U2 = v[2] / (v[3] > 1.0 ? v[3] : 1.0);
      *loss_host = (U2 > 0.0 && v[3] > 0.0) ? v[0] / (U2 * v[3]) : 0.0;
    }
  }
  return SPH_OK;
}

}  // extern "C"
