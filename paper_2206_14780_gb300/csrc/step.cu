// One semi-implicit predictor/corrector time step (paper Sec. 3.3) around the
// viscous solve: the equation of state, the dummy-wall pressure, the inviscid
// acceleration and continuity produce the right-hand sides of the two viscous
// systems A^n(dt/2) V = B and A^{n+1/2}(dt) V = B, and the particles move:
//
//   abar^n, drho^n at (r^n, u^n, rho^n, mu^n)
//   solve A^n(dt/2) V = u^n + dt/2 abar^n          -> u^{n+1/2}
//   r^{n+1/2} = r^n + dt/2 u^n,  rho^{n+1/2} = rho^n + dt/2 drho^n
//   mu^{n+1/2} = mu(r^{n+1/2}, u^{n+1/2})           (Papanastasiou, if set)
//   abar, drho at the half state
//   solve A^{n+1/2}(dt) V = u^n + dt abar^{n+1/2}   -> u^{n+1}
//   r^{n+1} = r^n + dt/2 (u^n + u^{n+1}),  rho^{n+1} = rho^n + dt drho^{n+1/2}
//
// with (Eq. cole-pressure) P = c0^2 rho0 / zeta ((rho / rho0)^zeta - 1),
// (Eq. dummyP, walls at constant velocity) P_w = (sum_F P_a W + g . sum_F rho_a
// (r_w - r_a) W) / sum_F W and rho_w = EOS^-1(P_w), and, with
// grad_b W_ab = |F_ab| (r_a - r_b) (the signs under which pressure repels and
// compression raises the density),
//   abar_b    = g - sum_a m_a (P_a / rho_a^2 + P_b / rho_b^2) |F_ab| (r_a - r_b)
//   drho_b/dt = sum_a m_a (u_b - u_a) . (r_a - r_b) |F_ab|
// (fluid rows; the density rate also on dynamic walls, whose density evolves;
// dummy walls take theirs from the closure).  Walls move with their prescribed
// velocity.  Position and density updates are evaluated in float64 with one
// rounding per operation (no contraction) and stored as float32, so the half
// step's positions -- and hence its neighbour lists -- are reproducible.
#include <cmath>
#include <cstring>

#include "sph_internal.cuh"

namespace sph {

// the step's device buffers, owned by the handle (caller order unless noted)
struct StepStage {
  DBuf<float4> r_n, u_n, acc, u_k;
  DBuf<float> rho_n, drho, P_s;   // P_s: sorted order
  DBuf<double> b, x, x_prev, sums;
  void release() {
    u_k.release();
    x_prev.release();
    sums.release();
    r_n.release();
    u_n.release();
    acc.release();
    rho_n.release();
    drho.release();
    P_s.release();
    b.release();
    x.release();
  }
};

void release_step_stage(sph_neighbors* H) {
  if (H && H->step) {
    H->step->release();
    delete H->step;
    H->step = nullptr;
  }
}

namespace {

struct StepGeom {
  float L[3], invL[3];
  int periodic[3];
  float inv_h;
  float absf_scale;   // |f| constant / h^5 (105/(128 pi) Wendland, 2 / w_G Gaussian)
  float w_scale;      // w constant / h^3 (21/(16 pi) Wendland, 1 / w_G Gaussian)
  int gauss;
  float gauss_tail;   // e^{-9}
  double lo[3], hi[3];
};

__device__ __forceinline__ void min_image(float* d, const StepGeom& g) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax)
    if (g.periodic[ax]) d[ax] -= g.L[ax] * rintf(d[ax] * g.invL[ax]);
}

// |F| (r) and W (r) of the chosen kernel, from q = r / h
__device__ __forceinline__ float kernel_absf(float q, const StepGeom& g) {
  if (g.gauss) return g.absf_scale * expf(-q * q);
  const float t = fmaxf(2.f - q, 0.f);
  return g.absf_scale * t * t * t;
}
__device__ __forceinline__ float kernel_w(float q, const StepGeom& g) {
  if (g.gauss) return g.w_scale * (expf(-q * q) - g.gauss_tail);
  const float t = fmaxf(1.f - 0.5f * q, 0.f);
  const float t2 = t * t;
  return g.w_scale * t2 * t2 * fmaf(2.f, q, 1.f);
}

__device__ __forceinline__ double eos_d(double rho, double rho0, double c0, double zeta) {
  return c0 * c0 * rho0 / zeta * (pow(rho / rho0, zeta) - 1.0);
}

// P = EOS(rho) on every sorted row (dummy walls are overwritten by the closure)
__global__ void k_step_eos(const float* __restrict__ rho_s, int64_t n, double rho0, double c0, double zeta,
                           float* __restrict__ P_s) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    P_s[s] = (float)eos_d((double)rho_s[s], rho0, c0, zeta);
}

// dummy walls (Eq. dummyP): pressure from the fluid neighbours, density by the
// inverse EOS, written to the handle's sorted copy and to the caller's array
__global__ void k_step_dummy(const float4* __restrict__ pos_s, float* __restrict__ rho_s,
                             const uint8_t* __restrict__ type_s, const int32_t* __restrict__ cnt,
                             const int64_t* __restrict__ slice_off, const int32_t* __restrict__ nbr,
                             const int32_t* __restrict__ perm, int64_t n, StepGeom g, double gx, double gy, double gz,
                             double rho0, double c0, double zeta, float* __restrict__ P_s, float* __restrict__ rho_c) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (type_s[s] == SPH_FLUID) continue;
    const float4 pb = pos_s[s];
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    double S = 0.0, num = 0.0;
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      if (type_s[t] != SPH_FLUID) continue;
      const float4 pa = pos_s[t];
      float d[3] = {pb.x - pa.x, pb.y - pa.y, pb.z - pa.z};   // r_w - r_a
      min_image(d, g);
      const float q = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * g.inv_h;
      const double w = (double)kernel_w(q, g);
      const double gr = gx * d[0] + gy * d[1] + gz * d[2];
      S += w;
      num += w * ((double)P_s[t] + gr * (double)rho_s[t]);
    }
    const double P = S > 0.0 ? num / S : 0.0;
    const double r = rho0 * pow(P * zeta / (c0 * c0 * rho0) + 1.0, 1.0 / zeta);
    P_s[s] = (float)P;
    rho_s[s] = (float)r;
    rho_c[perm[s]] = (float)r;
  }
}

// abar (fluid rows) and drho/dt (fluid and dynamic walls), caller order
__global__ void __launch_bounds__(kBlock) k_step_forces(const float4* __restrict__ pos_s, const float* __restrict__ rho_s,
                                                        const uint8_t* __restrict__ type_s,
                                                        const int32_t* __restrict__ cnt,
                                                        const int64_t* __restrict__ slice_off,
                                                        const int32_t* __restrict__ nbr,
                                                        const int32_t* __restrict__ perm, const float4* __restrict__ vel,
                                                        const float* __restrict__ P_s, int64_t n, StepGeom g, double gx,
                                                        double gy, double gz, int dummy, float4* __restrict__ acc,
                                                        float* __restrict__ drho) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ib = perm[s];
    const bool fluid = type_s[s] == SPH_FLUID;
    if (!fluid && dummy) {
      acc[ib] = make_float4(0.f, 0.f, 0.f, 0.f);
      drho[ib] = 0.f;
      continue;
    }
    const float4 pb = pos_s[s];
    const float4 ub = vel[ib];
    const float rb = rho_s[s];
    const float Pb = P_s[s] / (rb * rb);
    double ax = 0.0, ay = 0.0, az = 0.0, dr = 0.0;
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    for (int j = 0; j < c; ++j) {
      const int32_t t = nbr[base + (int64_t)j * kSlice];
      const float4 pa = pos_s[t];
      float d[3] = {pa.x - pb.x, pa.y - pb.y, pa.z - pb.z};   // r_a - r_b
      min_image(d, g);
      const float q = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * g.inv_h;
      const float mF = pa.w * kernel_absf(q, g);
      const float ra = rho_s[t];
      const float cp = mF * (P_s[t] / (ra * ra) + Pb);
      ax -= (double)(cp * d[0]);
      ay -= (double)(cp * d[1]);
      az -= (double)(cp * d[2]);
      const float4 ua = vel[perm[t]];
      dr += (double)(mF * ((ub.x - ua.x) * d[0] + (ub.y - ua.y) * d[1] + (ub.z - ua.z) * d[2]));
    }
    acc[ib] = fluid ? make_float4((float)(ax + gx), (float)(ay + gy), (float)(az + gz), 0.f)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    drho[ib] = (float)dr;
  }
}

// b = u^n + hdt abar on fluid rows; 2 u_w (dummy) or u_w (dynamic) on walls
__global__ void k_step_rhs(const float4* __restrict__ u_n, const float4* __restrict__ acc,
                           const uint8_t* __restrict__ type, int64_t n, double hdt, int dummy, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 u = u_n[i];
    if (type[i] == SPH_FLUID) {
      const float4 a = acc[i];
      b[3 * i] = __dadd_rn((double)u.x, __dmul_rn(hdt, (double)a.x));
      b[3 * i + 1] = __dadd_rn((double)u.y, __dmul_rn(hdt, (double)a.y));
      b[3 * i + 2] = __dadd_rn((double)u.z, __dmul_rn(hdt, (double)a.z));
    } else {
      const double f = dummy ? 2.0 : 1.0;
      b[3 * i] = f * (double)u.x;
      b[3 * i + 1] = f * (double)u.y;
      b[3 * i + 2] = f * (double)u.z;
    }
  }
}

__device__ __forceinline__ float advance(double base, double v, double scale, int ax, const StepGeom& g) {
  double p = __dadd_rn(base, __dmul_rn(v, scale));
  if (g.periodic[ax]) {
    const double L = g.hi[ax] - g.lo[ax];
    if (p >= g.hi[ax]) p = p - L;
    if (p < g.lo[ax]) p = p + L;
  }
  return (float)p;
}

// corrector = 0: r = r^n + hdt u^n (walls u_w), rho = rho^n + hdt drho, u = x (fluid)
// corrector = 1: r = r^n + hdt (u^n + x) (walls 2 u_w), rho = rho^n + dt drho, u = x (fluid)
__global__ void k_step_move(const float4* __restrict__ r_n, const float4* __restrict__ u_n,
                            const float* __restrict__ rho_n, const float* __restrict__ drho,
                            const double* __restrict__ x, const uint8_t* __restrict__ type, int64_t n, double hdt,
                            double rdt, int corrector, StepGeom g, float4* __restrict__ pos, float4* __restrict__ vel,
                            float* __restrict__ rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 r = r_n[i], u = u_n[i];
    const bool fluid = type[i] == SPH_FLUID;
    double v[3] = {(double)u.x, (double)u.y, (double)u.z};
    if (corrector) {
      for (int k = 0; k < 3; ++k) v[k] = fluid ? __dadd_rn(v[k], x[3 * i + k]) : 2.0 * v[k];
    }
    float4 p = r;
    p.x = advance((double)r.x, v[0], hdt, 0, g);
    p.y = advance((double)r.y, v[1], hdt, 1, g);
    p.z = advance((double)r.z, v[2], hdt, 2, g);
    pos[i] = p;
    rho[i] = (float)__dadd_rn((double)rho_n[i], __dmul_rn((double)drho[i], rdt));
    if (fluid) vel[i] = make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f);
  }
}

// u_k = x on fluid rows (the prescribed wall velocity on wall rows), for the mu pass
__global__ void k_step_uk(const double* __restrict__ x, const float4* __restrict__ u_n, const uint8_t* __restrict__ type,
                          int64_t n, float4* __restrict__ u_k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u_k[i] = type[i] == SPH_FLUID ? make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f) : u_n[i];
}

// sums[0] += |x - x_prev|^2, sums[1] += |x|^2 over fluid rows
__global__ void k_step_change(const double* __restrict__ x, const double* __restrict__ xp,
                              const uint8_t* __restrict__ type, int64_t n, double* __restrict__ sums) {
  double a = 0.0, c = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (type[i] != SPH_FLUID) continue;
    for (int k = 0; k < 3; ++k) {
      const double d = x[3 * i + k] - xp[3 * i + k];
      a += d * d;
      c += x[3 * i + k] * x[3 * i + k];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums, a);
    atomicAdd(sums + 1, c);
  }
}

StepGeom step_geom(const sph_neighbors* H, const sph_state* S) {
  StepGeom g{};
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = (float)H->grid.L[ax];
    g.invL[ax] = (float)(1.0 / H->grid.L[ax]);
    g.periodic[ax] = H->grid.periodic[ax];
    g.lo[ax] = S->lo[ax];
    g.hi[ax] = S->hi[ax];
  }
  const double h = (double)H->h;
  g.inv_h = (float)(1.0 / h);
  g.gauss = H->kernel == SPH_KERNEL_GAUSSIAN ? 1 : 0;
  const double wg = gauss_norm();
  g.absf_scale = (float)((g.gauss ? 2.0 / wg : 105.0 / (128.0 * M_PI)) / (h * h * h * h * h));
  g.w_scale = (float)((g.gauss ? 1.0 / wg : 21.0 / (16.0 * M_PI)) / (h * h * h));
  g.gauss_tail = (float)std::exp(-kGaussK * kGaussK);
  return g;
}

sph_scene scene_of(const sph_state* S) {
  sph_scene sc{};
  sc.n = S->n;
  sc.pos = S->pos;
  sc.rho = S->rho;
  sc.mu = S->mu;
  sc.ptype = S->ptype;
  for (int ax = 0; ax < 3; ++ax) {
    sc.lo[ax] = S->lo[ax];
    sc.hi[ax] = S->hi[ax];
    sc.periodic[ax] = S->periodic[ax];
  }
  sc.h = S->h;
  sc.kernel = S->kernel;
  return sc;
}

// neighbours at the state's positions, mu (with a rheology), pressures with the
// dummy-wall closure, abar and drho
sph_status evaluate(sph_state* S, const sph_step_params* Pp, sph_neighbors** handle, cudaStream_t st) {
  const sph_scene sc = scene_of(S);
  SPH_TRY(build_neighbors(&sc, Pp->max_neighbors > 0 ? Pp->max_neighbors : 128, handle, st));
  sph_neighbors* H = *handle;
  if (!H->step) H->step = new StepStage();
  StepStage& T = *H->step;
  SPH_TRY(T.acc.alloc(H->n));
  SPH_TRY(T.drho.alloc(H->n));
  SPH_TRY(T.P_s.alloc(H->n_pad));
  if (Pp->rheology == 1)
    SPH_TRY(mu_papanastasiou(H, S->vel, S->vel, Pp->tau0, Pp->mu0, Pp->m, S->mu, 1, st));
  const StepGeom g = step_geom(H, S);
  const int grid = grid_for(H, H->n);
  SPH_LAUNCH(k_step_eos, grid, kBlock, 0, st)(H->rho_s.p, H->n, Pp->rho0, Pp->c0, Pp->zeta, T.P_s.p);
  const int dummy = Pp->boundary == SPH_BC_DUMMY ? 1 : 0;
  if (dummy) {
    SPH_LAUNCH(k_step_dummy, grid, kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p, H->slice_off.p,
                                                   H->nbr.p, H->perm.p, H->n, g, Pp->g[0], Pp->g[1], Pp->g[2],
                                                   Pp->rho0, Pp->c0, Pp->zeta, T.P_s.p, S->rho);
    H->mu_version++;   // the walls' densities enter A(dt): set it up again
  }
  SPH_LAUNCH(k_step_forces, grid, kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->type_s.p, H->cnt.p, H->slice_off.p,
                                                  H->nbr.p, H->perm.p, reinterpret_cast<const float4*>(S->vel),
                                                  T.P_s.p, H->n, g, Pp->g[0], Pp->g[1], Pp->g[2], dummy, T.acc.p,
                                                  T.drho.p);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace

sph_status time_step(sph_state* S, const sph_step_params* Pp, const sph_solve_opts* O, sph_neighbors** handle,
                     sph_step_report* R, cudaStream_t st) {
  if (!S || !Pp || !O || !handle || !R || !S->pos || !S->vel || !S->rho || !S->mu || !S->ptype || S->n < 1) {
    set_error("sph_step: null argument or empty state");
    return SPH_ERR_INVALID;
  }
  if (!(Pp->dt > 0.0) || !(Pp->rho0 > 0.0) || !(Pp->c0 > 0.0) || !(Pp->zeta > 0.0) ||
      (Pp->rheology != 0 && Pp->rheology != 1) || (Pp->rheology == 1 && !(Pp->mu0 > 0.0 && Pp->m > 0.0 && Pp->tau0 >= 0.0))) {
    set_error("sph_step: need dt, rho0, c0, zeta > 0 and rheology 0 or 1 (with tau0 >= 0, mu0 > 0, m > 0)");
    return SPH_ERR_INVALID;
  }
  std::memset(R, 0, sizeof(*R));
  const int64_t n = S->n;
  const double dt = Pp->dt, hdt = 0.5 * Pp->dt;
  const int dummy = Pp->boundary == SPH_BC_DUMMY ? 1 : 0;
  // predictor: the state at n
  SPH_TRY(evaluate(S, Pp, handle, st));
  sph_neighbors* H = *handle;
  StepStage& T = *H->step;
  SPH_TRY(T.r_n.alloc(n));
  SPH_TRY(T.u_n.alloc(n));
  SPH_TRY(T.rho_n.alloc(n));
  SPH_TRY(T.b.alloc(3 * n));
  SPH_TRY(T.x.alloc(3 * n));
  SPH_TRY_CUDA(cudaMemcpyAsync(T.r_n.p, S->pos, n * sizeof(float4), cudaMemcpyDeviceToDevice, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(T.u_n.p, S->vel, n * sizeof(float4), cudaMemcpyDeviceToDevice, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(T.rho_n.p, S->rho, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  const StepGeom g0 = step_geom(H, S);
  const int grid = grid_for(H, n);
  const sph_visc_params half{hdt, Pp->boundary, Pp->mean};
  const sph_visc_params full{dt, Pp->boundary, Pp->mean};
  SPH_LAUNCH(k_step_rhs, grid, kBlock, 0, st)(T.u_n.p, T.acc.p, S->ptype, n, hdt, dummy, T.b.p);
  SPH_TRY(warm_start_plain(H, &half, S->vel, S->ptype, T.b.p, T.x.p, st));
  sph_status s1 = solve_mixed(H, &half, O, T.b.p, T.x.p, &R->half, st);
  if (s1 != SPH_OK && s1 != SPH_NOT_CONVERGED) return s1;
  SPH_LAUNCH(k_step_move, grid, kBlock, 0, st)(T.r_n.p, T.u_n.p, T.rho_n.p, T.drho.p, T.x.p, S->ptype, n, hdt, hdt, 0,
                                               g0, reinterpret_cast<float4*>(S->pos), reinterpret_cast<float4*>(S->vel),
                                               S->rho);
  SPH_TRY_CUDA(cudaGetLastError());
  // corrector: the state at n + 1/2
  SPH_TRY(evaluate(S, Pp, handle, st));
  H = *handle;
  StepStage& T2 = *H->step;
  SPH_LAUNCH(k_step_rhs, grid, kBlock, 0, st)(T2.u_n.p, T2.acc.p, S->ptype, n, dt, dummy, T2.b.p);
  SPH_TRY(warm_start_plain(H, &full, S->vel, S->ptype, T2.b.p, T2.x.p, st));
  sph_status s2 = solve_mixed(H, &full, O, T2.b.p, T2.x.p, &R->full, st);
  if (s2 != SPH_OK && s2 != SPH_NOT_CONVERGED) return s2;
  // the non-linear form: mu from the new velocities at r^{n+1/2}, solve again
  if (Pp->rheology == 1 && Pp->picard > 0) {
    const double tol = Pp->picard_tol > 0.0 ? Pp->picard_tol : 1e-6;
    SPH_TRY(T2.u_k.alloc(n));
    SPH_TRY(T2.x_prev.alloc(3 * n));
    SPH_TRY(T2.sums.alloc(2));
    for (int k = 0; k < Pp->picard; ++k) {
      SPH_LAUNCH(k_step_uk, grid, kBlock, 0, st)(T2.x.p, T2.u_n.p, S->ptype, n, T2.u_k.p);
      SPH_TRY(mu_papanastasiou(H, reinterpret_cast<const float*>(T2.u_k.p), reinterpret_cast<const float*>(T2.u_k.p),
                               Pp->tau0, Pp->mu0, Pp->m, S->mu, 1, st));
      SPH_TRY_CUDA(cudaMemcpyAsync(T2.x_prev.p, T2.x.p, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      s2 = solve_mixed(H, &full, O, T2.b.p, T2.x.p, &R->full, st);
      if (s2 != SPH_OK && s2 != SPH_NOT_CONVERGED) return s2;
      SPH_TRY_CUDA(cudaMemsetAsync(T2.sums.p, 0, 2 * sizeof(double), st));
      SPH_LAUNCH(k_step_change, grid, kBlock, 0, st)(T2.x.p, T2.x_prev.p, S->ptype, n, T2.sums.p);
      double sums[2];
      SPH_TRY_CUDA(cudaMemcpyAsync(sums, T2.sums.p, sizeof(sums), cudaMemcpyDeviceToHost, st));
      SPH_TRY_CUDA(cudaStreamSynchronize(st));
      R->picard_passes = k + 1;
      R->picard_change = sums[1] > 0.0 ? std::sqrt(sums[0] / sums[1]) : std::sqrt(sums[0]);
      if (R->picard_change <= tol) break;
    }
  }
  SPH_LAUNCH(k_step_move, grid, kBlock, 0, st)(T2.r_n.p, T2.u_n.p, T2.rho_n.p, T2.drho.p, T2.x.p, S->ptype, n, hdt, dt,
                                               1, g0, reinterpret_cast<float4*>(S->pos),
                                               reinterpret_cast<float4*>(S->vel), S->rho);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return (s1 == SPH_OK && s2 == SPH_OK) ? SPH_OK : SPH_NOT_CONVERGED;
}

}  // namespace sph
