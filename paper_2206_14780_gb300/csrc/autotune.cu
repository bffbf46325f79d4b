// Autotuner of the operator apply: for each apply phase of the BiCGSTAB
// iteration (A p with the delta dot; A r* with the omega dots) it times the six
// row-loop forms -- the register forms of apply.cuh, (U, PF) = (8, plain),
// (4, plain), (8, prefetch), (4, prefetch), the form with the coefficient
// stream staged in shared memory by bulk copies, and the form with each slice's
// neighbour vectors staged in shared memory (solver.cu), each at its own
// full-occupancy grid -- on the handle's operator, and keeps the fastest.  The compiler schedules the unrolled gathers differently
// in each kernel (the dot accumulators change the register budget), so the best
// form differs per phase and is found by measurement, once per handle (again if
// the particle count changes by more than half).
#include <cmath>

#include "apply.cuh"
#include "sph_internal.cuh"

namespace sph {

sph_status autotune_apply(sph_neighbors* H, bool merged, unsigned int* counter, cudaStream_t st) {
  if (H->tuned && H->tuned_n_pad > 0 && std::fabs((double)H->n_pad / (double)H->tuned_n_pad - 1.0) < 0.5)
    return SPH_OK;
  SPH_TRY(H->scal_tune.alloc(1));
  const int64_t np = H->n_pad;
  SPH_TRY_CUDA(cudaMemsetAsync(H->v_p.p, 0, np * sizeof(float4), st));
  SPH_TRY_CUDA(cudaMemsetAsync(H->v_rh.p, 0, np * sizeof(float4), st));
  SPH_TRY_CUDA(cudaMemsetAsync(H->scal_tune.p, 0, sizeof(SolverScalars), st));
  SPH_TRY(apply_prepare(H, 5, st));        // the unions form 5 reads
  cudaEvent_t e0, e1;
  SPH_TRY_CUDA(cudaEventCreate(&e0));
  SPH_TRY_CUDA(cudaEventCreate(&e1));
  const OpView op = op_view(H);
  int64_t want = (H->nslices * 32 + kBlock - 1) / kBlock;
  sph_status status = SPH_OK;
  const int phases[2] = {0, merged ? 2 : 1};
  for (int pi = 0; pi < 2 && status == SPH_OK; ++pi) {
    const int ph = phases[pi];
    float best = 1e30f;
    for (int var = 0; var < kApplyVariants; ++var) {
      const ApplyDotFn kern = apply_kernel(ph, var);
      int occ = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)kern, kBlock, apply_smem(var));
      int64_t g = (int64_t)H->num_sms * (occ > 0 ? occ : 1);
      if (g > want) g = want;
      if (g > H->red_grid) g = H->red_grid;
      if (g < 1) g = 1;
      // The full resident grid leaves a ragged last round of slices (warps take
      // 7 or 8 of them on the 1.16M box); the register forms are also timed with
      // the smallest grid that needs the same number of rounds, where every warp
      // takes a full last round.
      int64_t grids[2] = {g, 0};
      if (var < kApplyVariantsRegister) {
        const int64_t wpb = kBlock / 32, rounds = (H->nslices + g * wpb - 1) / (g * wpb);
        const int64_t gb = (H->nslices + rounds * wpb - 1) / (rounds * wpb);
        if (gb >= 1 && gb < g) grids[1] = gb;
      }
      float ms_var = 1e30f;
      for (int gi = 0; gi < 2 && grids[gi] > 0; ++gi) {
        const int gg = (int)grids[gi];
        for (int k = 0; k < 2; ++k)
          SPH_LAUNCH(kern, gg, kBlock, apply_smem(var), st)(op, H->v_p.p, H->v_As.p, H->v_rh.p, H->scal_tune.p,
                                                            H->partials.p, counter);
        cudaEventRecord(e0, st);
        const int reps = 5;
        for (int k = 0; k < reps; ++k)
          SPH_LAUNCH(kern, gg, kBlock, apply_smem(var), st)(op, H->v_p.p, H->v_As.p, H->v_rh.p, H->scal_tune.p,
                                                            H->partials.p, counter);
        cudaEventRecord(e1, st);
        cudaError_t err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) {
          set_error("apply autotuner: %s", cudaGetErrorString(err));
          status = SPH_ERR_CUDA;
          break;
        }
        ms /= reps;
        ms_var = ms < ms_var ? ms : ms_var;
        if (ms < best) {
          best = ms;
          H->apply_var[ph] = var;
          H->apply_grid[ph] = gg;
        }
      }
      if (status != SPH_OK) break;
      H->tune_us[ph][var] = 1e3f * ms_var;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != SPH_OK) return status;
  int32_t fault = 0;
  SPH_TRY_CUDA(cudaMemcpyAsync(&fault, &H->scal_tune.p->fault, sizeof(fault), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  if (fault) {
    set_error("apply autotuner: a staged apply gave up waiting for its coefficients");
    return SPH_ERR_TIMEOUT;
  }
  H->tuned = true;
  H->tuned_n_pad = H->n_pad;
  return SPH_OK;
}

}  // namespace sph
