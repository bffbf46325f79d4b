// Scalar side of the restructured BiCGSTAB (paper Sec. 4.2) and of the rotated
// CG (Sec. 4.1, at the end of this file): run by thread 0 of
// the last block after each grid reduction, shared by the float32 and float64
// solves.  States per component follow the "Stopping criterion" paragraph:
// converged (r.r < tau^2), stalled (delta = 0, or a coefficient that zeroes out)
// or progressing; a component that is not progressing is frozen (alpha = omega
// = 0) and the pass stops when none progresses.
#pragma once

#include "sph_internal.cuh"

namespace sph {

constexpr double kFltMin = 1.17549435082228750797e-38;  // 2^-126: the tau^2 floor (Sec. 4.1)

// Each scalar step is written per component c; the plain forms run the three
// components on one thread (batched solver), the _w forms on lanes 0..2 of the
// calling warp (every lane of the warp calls them), so the float64 divisions of
// the three components run side by side in the last block's tail.

__device__ inline void scal_delta_c(SolverScalars* S, const double* dots, int c) {
  if (S->state[c] != SPH_PROGRESSING) {
    S->alpha[c] = 0.0;
    S->stall_now[c] = 0;
    return;
  }
  const double d = dots[c];
  S->delta[c] = d;
  double a = 0.0;
  int stall = 0;
  if (d == 0.0 || !isfinite(d)) {
    stall = 1;
  } else {
    a = S->gamma[c] / d;
    if (!isfinite(a)) {
      a = 0.0;
      stall = 1;
    }
  }
  S->alpha[c] = a;
  S->stall_now[c] = stall;
}

__device__ inline void scal_omega_c(SolverScalars* S, const double* dots, int c) {
  if (S->state[c] != SPH_PROGRESSING) {
    S->omega[c] = 0.0;
    return;
  }
  const double sA = dots[c], AA = dots[3 + c];
  double om = (AA > 0.0 && isfinite(AA)) ? sA / AA : 0.0;
  if (!isfinite(om)) om = 0.0;
  S->omega[c] = om;
}

// gamma' and r.r of component c known: alpha', beta and its state (returned)
__device__ inline int scal_update_c(SolverScalars* S, const double* gam_new, const double* rr, int c) {
  if (S->state[c] != SPH_PROGRESSING) {
    S->alpha_p[c] = 0.0;
    S->beta[c] = 0.0;
    return S->state[c];
  }
  const double om = S->omega[c];
  const bool ok = !S->stall_now[c] && om != 0.0;
  double ap = ok ? gam_new[c] / S->delta[c] : 0.0;
  double be = ok ? ap / om : 0.0;
  if (!isfinite(ap) || !isfinite(be)) {
    ap = 0.0;
    be = 0.0;
  }
  if (!isfinite(gam_new[c]) || !isfinite(rr[c])) S->nonfinite = 1;
  S->alpha_p[c] = ap;
  S->beta[c] = be;
  S->gamma[c] = gam_new[c];
  S->rr[c] = rr[c];
  int st;
  if (rr[c] < S->tau2[c]) st = SPH_CONVERGED;
  else if (S->stall_now[c] || om == 0.0 || !isfinite(rr[c])) st = SPH_STALLED;
  else st = SPH_PROGRESSING;
  if (st == SPH_STALLED) S->stalled_any[c] = 1;
  S->state[c] = st;
  return st;
}

__device__ inline void scal_after_delta(SolverScalars* S, const double* dots) {
  for (int c = 0; c < 3; ++c) scal_delta_c(S, dots, c);
}

__device__ inline void scal_after_omega(SolverScalars* S, const double* dots) {
  for (int c = 0; c < 3; ++c) scal_omega_c(S, dots, c);
}

// gamma' and r.r known: alpha', beta, states, iteration count, stop flag.
__device__ inline void scal_after_update(SolverScalars* S, const double* gam_new, const double* rr) {
  int progressing = 0;
  for (int c = 0; c < 3; ++c) progressing += scal_update_c(S, gam_new, rr, c) == SPH_PROGRESSING;
  S->iter += 1;
  S->done = (progressing == 0 || S->iter >= S->maxit) ? 1 : 0;
}

__device__ inline void scal_after_delta_w(SolverScalars* S, const double* dots) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) scal_delta_c(S, dots, lane);
}

__device__ inline void scal_after_omega_w(SolverScalars* S, const double* dots) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) scal_omega_c(S, dots, lane);
}

__device__ inline void scal_after_update_w(SolverScalars* S, const double* gam_new, const double* rr) {
  const int lane = threadIdx.x & 31;
  const int st = lane < 3 ? scal_update_c(S, gam_new, rr, lane) : SPH_CONVERGED;
  const unsigned prog = __ballot_sync(0xffffffffu, st == SPH_PROGRESSING);
  if (lane == 0) {
    S->iter += 1;
    S->done = (prog == 0u || S->iter >= S->maxit) ? 1 : 0;
  }
}

// pass initialisation from gamma0 = r0.r0 (= b.b of the inner system)
__device__ inline void scal_init(SolverScalars* S, const double* g, double eps2, int maxit) {
  int progressing = 0;
  for (int c = 0; c < 3; ++c) {
    S->gamma[c] = g[c];
    S->rr[c] = g[c];
    S->tau2[c] = fmax(eps2 * g[c], kFltMin);
    S->alpha[c] = S->alpha_p[c] = S->beta[c] = S->omega[c] = S->delta[c] = 0.0;
    S->stall_now[c] = 0;
    S->stalled_any[c] = 0;
    const int st = (g[c] == 0.0 || g[c] < S->tau2[c]) ? SPH_CONVERGED : SPH_PROGRESSING;
    S->state[c] = st;
    progressing += (st == SPH_PROGRESSING);
  }
  S->iter = 0;
  S->maxit = maxit;
  S->nonfinite = 0;
  S->done = progressing == 0 ? 1 : 0;
  S->pad = S->done;
}

// ---- rotated conjugate gradient (Sec. 4.1, second listing) ---------------------
// Per iteration: p = z + beta p (z = D^-1 r with Jacobi, App. B; z = r without);
// alpha = gamma / (p.Ap) with gamma = r.z; r -= alpha Ap; x += alpha p;
// gamma' = r.z'; beta = gamma' / gamma; converged when r.r < tau^2.  "Stopping
// criterion" of Sec. 4.1: alpha = 0 in finite precision while r is not small is a
// stall (a p.Ap that is zero or not finite, or an alpha that is not finite, gives
// alpha = 0); the iteration completes and the pass exits at its single end point.

__device__ inline void scal_cg_alpha_c(SolverScalars* S, const double* dots, int c) {
  if (S->state[c] != SPH_PROGRESSING) {
    S->alpha[c] = 0.0;
    S->stall_now[c] = 0;
    return;
  }
  const double d = dots[c];
  S->delta[c] = d;
  double a = (d != 0.0 && isfinite(d)) ? S->gamma[c] / d : 0.0;
  if (!isfinite(a)) a = 0.0;
  S->alpha[c] = a;
  S->stall_now[c] = a == 0.0 ? 1 : 0;
}

__device__ inline int scal_cg_update_c(SolverScalars* S, const double* gam_new, const double* rr, int c) {
  if (S->state[c] != SPH_PROGRESSING) {
    S->beta[c] = 0.0;
    return S->state[c];
  }
  double be = S->stall_now[c] ? 0.0 : gam_new[c] / S->gamma[c];
  if (!isfinite(be)) be = 0.0;
  if (!isfinite(gam_new[c]) || !isfinite(rr[c])) S->nonfinite = 1;
  S->beta[c] = be;
  S->gamma[c] = gam_new[c];
  S->rr[c] = rr[c];
  int st;
  if (rr[c] < S->tau2[c]) st = SPH_CONVERGED;
  else if (S->stall_now[c] || !isfinite(rr[c])) st = SPH_STALLED;
  else st = SPH_PROGRESSING;
  if (st == SPH_STALLED) S->stalled_any[c] = 1;
  S->state[c] = st;
  return st;
}

__device__ inline void scal_cg_alpha_w(SolverScalars* S, const double* dots) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) scal_cg_alpha_c(S, dots, lane);
}

__device__ inline void scal_cg_update_w(SolverScalars* S, const double* gam_new, const double* rr) {
  const int lane = threadIdx.x & 31;
  const int st = lane < 3 ? scal_cg_update_c(S, gam_new, rr, lane) : SPH_CONVERGED;
  const unsigned prog = __ballot_sync(0xffffffffu, st == SPH_PROGRESSING);
  if (lane == 0) {
    S->iter += 1;
    S->done = (prog == 0u || S->iter >= S->maxit) ? 1 : 0;
  }
}

// CG pass initialisation: gamma = r0.z0, tau^2 base = r0.r0
__device__ inline void scal_cg_init(SolverScalars* S, const double* gz, const double* rr, double eps2, int maxit) {
  int progressing = 0;
  for (int c = 0; c < 3; ++c) {
    S->gamma[c] = gz[c];
    S->rr[c] = rr[c];
    S->tau2[c] = fmax(eps2 * rr[c], kFltMin);
    S->alpha[c] = S->alpha_p[c] = S->beta[c] = S->omega[c] = S->delta[c] = 0.0;
    S->stall_now[c] = 0;
    S->stalled_any[c] = 0;
    const int st = (rr[c] == 0.0 || rr[c] < S->tau2[c]) ? SPH_CONVERGED : SPH_PROGRESSING;
    S->state[c] = st;
    progressing += (st == SPH_PROGRESSING);
  }
  S->iter = 0;
  S->maxit = maxit;
  S->nonfinite = 0;
  S->done = progressing == 0 ? 1 : 0;
  S->pad = S->done;
}

}  // namespace sph
