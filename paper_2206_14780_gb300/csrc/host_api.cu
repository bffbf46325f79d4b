// sph_visc_solve_host: one viscous solve from host buffers (include/sphvisc.h).
//
// The scene, b and v^n (or x) go to device staging owned by the handle with one
// cudaMemcpyAsync each, then the calls a device-side user would make run on the
// staged copies: sph_build_neighbors, sph_warm_start (no network), sph_visc_solve;
// the solution comes back with one more copy.  The staging is allocated on the
// first call and grows with n; sph_neighbors_destroy frees it.
#include <cstring>

#include "sph_internal.cuh"

using namespace sph;

extern "C" sph_status sph_visc_solve_host(const sph_scene* scene, int32_t max_neighbors,
                                          const sph_visc_params* params, const sph_solve_opts* opts,
                                          const float* vel, const double* b, double* x, sph_neighbors** handle,
                                          sph_solve_report* report, void* stream) {
  clear_error();
  if (!scene || !params || !opts || !b || !x || !handle || !report || !scene->pos || !scene->rho || !scene->mu ||
      !scene->ptype || scene->n < 1) {
    set_error("sph_visc_solve_host: null argument or n < 1");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = scene->n;
  // staging: the handle's if it has one, else a new one handed to the handle below
  HostStage* stage = (*handle && (*handle)->stage) ? (*handle)->stage : new HostStage();
  auto fail = [&](sph_status s) {
    if (!(*handle && (*handle)->stage == stage)) {
      stage->release();
      delete stage;
    }
    return s;
  };
#define TRYH(expr)                         \
  do {                                     \
    sph_status s__ = (expr);               \
    if (s__ != SPH_OK) return fail(s__);   \
  } while (0)
#define TRYH_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e__ = (call);                                                            \
    if (e__ != cudaSuccess) {                                                            \
      set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__));    \
      return fail(SPH_ERR_CUDA);                                                         \
    }                                                                                    \
  } while (0)
  TRYH(stage->pos.alloc(n));
  TRYH(stage->rho.alloc(n));
  TRYH(stage->mu.alloc(n));
  TRYH(stage->type.alloc(n));
  TRYH(stage->b.alloc(3 * n));
  TRYH(stage->x.alloc(3 * n));
  if (vel) TRYH(stage->vel.alloc(n));
  TRYH_CUDA(cudaMemcpyAsync(stage->pos.p, scene->pos, n * sizeof(float4), cudaMemcpyHostToDevice, st));
  TRYH_CUDA(cudaMemcpyAsync(stage->rho.p, scene->rho, n * sizeof(float), cudaMemcpyHostToDevice, st));
  TRYH_CUDA(cudaMemcpyAsync(stage->mu.p, scene->mu, n * sizeof(float), cudaMemcpyHostToDevice, st));
  TRYH_CUDA(cudaMemcpyAsync(stage->type.p, scene->ptype, n, cudaMemcpyHostToDevice, st));
  TRYH_CUDA(cudaMemcpyAsync(stage->b.p, b, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  if (vel)
    TRYH_CUDA(cudaMemcpyAsync(stage->vel.p, vel, n * sizeof(float4), cudaMemcpyHostToDevice, st));
  else
    TRYH_CUDA(cudaMemcpyAsync(stage->x.p, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  sph_scene dev = *scene;
  dev.pos = reinterpret_cast<const float*>(stage->pos.p);
  dev.rho = stage->rho.p;
  dev.mu = stage->mu.p;
  dev.ptype = stage->type.p;
  TRYH(sph_build_neighbors(&dev, max_neighbors, handle, stream));
  (*handle)->stage = stage;   // from here the handle owns the staging
#undef TRYH
#undef TRYH_CUDA
  if (vel)
    SPH_TRY(sph_warm_start(*handle, params, nullptr, reinterpret_cast<const float*>(stage->vel.p), stage->type.p,
                           stage->b.p, stage->x.p, stream));
  const sph_status s = sph_visc_solve(*handle, params, opts, stage->b.p, stage->x.p, report, stream);
  if (s != SPH_OK && s != SPH_NOT_CONVERGED) return s;
  SPH_TRY_CUDA(cudaMemcpyAsync(x, stage->x.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return s;
}
