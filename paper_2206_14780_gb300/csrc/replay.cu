// sph_bicgstab_replay: the solver's scalar steps on caller-given dot products.
//
// The restructured BiCGSTAB (paper Sec. 4.2) decides its per-component states in
// three places, each after a grid reduction: alpha from delta, omega from
// r*.Ar* and Ar*.Ar*, then alpha', beta and the state from gamma' and r.r.  The
// solver's kernels run these steps (bicgstab_scalars.cuh) on one warp of the
// last block; this entry point runs the same device functions, in the same
// order and on one warp, on dots chosen by the caller, so that every branch of
// the "Stopping criterion" safeguards can be driven on the GPU without a
// matrix that produces those dots.
#include <cstring>

#include "bicgstab_scalars.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kReplayIn = 15;    // delta[3], r*.Ar*[3], Ar*.Ar*[3], gamma'[3], r.r[3]
constexpr int kReplayOut = 20;   // alpha, omega, alpha', beta, state, stalled_any [3 each], iter, done
constexpr int kReplayMaxSteps = 100000;

__device__ void replay_record(const SolverScalars* S, double* o) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) {
    o[lane] = S->alpha[lane];
    o[3 + lane] = S->omega[lane];
    o[6 + lane] = S->alpha_p[lane];
    o[9 + lane] = S->beta[lane];
    o[12 + lane] = (double)S->state[lane];
    o[15 + lane] = (double)S->stalled_any[lane];
  }
  if (lane == 0) {
    o[18] = (double)S->iter;
    o[19] = (double)S->done;
  }
}

// one warp; the scalars live in shared memory like the last block's view of them
__global__ void k_replay(const double* __restrict__ gamma0, double eps2, int maxit, int nsteps,
                         const double* __restrict__ dots, double* __restrict__ out) {
  __shared__ SolverScalars S;
  if (threadIdx.x == 0) {
    memset(&S, 0, sizeof(S));
    scal_init(&S, gamma0, eps2, maxit);
  }
  __syncwarp();
  replay_record(&S, out);
  __syncwarp();
  for (int i = 0; i < nsteps; ++i) {
    const double* d = dots + (size_t)i * kReplayIn;
    // the solver's loop kernels return at once when the pass is done, so no
    // scalar step runs after the stop flag is set
    if (!S.done) {
      scal_after_delta_w(&S, d);
      __syncwarp();
      scal_after_omega_w(&S, d + 3);
      __syncwarp();
      scal_after_update_w(&S, d + 9, d + 12);
      __syncwarp();
    }
    replay_record(&S, out + (size_t)(i + 1) * kReplayOut);
    __syncwarp();
  }
}

}  // namespace

sph_status bicgstab_replay(const double* gamma0, double eps, int32_t maxit, int32_t nsteps, const double* dots,
                           double* out, cudaStream_t st) {
  if (!gamma0 || !out || (nsteps > 0 && !dots)) {
    set_error("sph_bicgstab_replay: null argument");
    return SPH_ERR_INVALID;
  }
  if (nsteps < 0 || nsteps > kReplayMaxSteps || maxit < 1 || !(eps >= 0.0)) {
    set_error("sph_bicgstab_replay: need 0 <= nsteps <= %d, maxit >= 1, eps >= 0", kReplayMaxSteps);
    return SPH_ERR_INVALID;
  }
  const size_t in_bytes = (size_t)nsteps * kReplayIn * sizeof(double);
  const size_t out_bytes = (size_t)(nsteps + 1) * kReplayOut * sizeof(double);
  DBuf<double> d_in, d_out, d_g;
  sph_status status = SPH_OK;
  do {
    if ((status = d_in.alloc((size_t)nsteps * kReplayIn)) != SPH_OK) break;
    if ((status = d_out.alloc((size_t)(nsteps + 1) * kReplayOut)) != SPH_OK) break;
    if ((status = d_g.alloc(3)) != SPH_OK) break;
    cudaError_t e = cudaMemcpyAsync(d_g.p, gamma0, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nsteps > 0) e = cudaMemcpyAsync(d_in.p, dots, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_error("sph_bicgstab_replay: copy in: %s", cudaGetErrorString(e));
      status = SPH_ERR_CUDA;
      break;
    }
    SPH_LAUNCH(k_replay, 1, 32, 0, st)(d_g.p, eps * eps, maxit, nsteps, d_in.p, d_out.p);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out.p, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("sph_bicgstab_replay: %s", cudaGetErrorString(e));
      status = SPH_ERR_CUDA;
    }
  } while (false);
  d_in.release();
  d_out.release();
  d_g.release();
  return status;
}

}  // namespace sph
