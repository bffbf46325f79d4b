// extern "C" entry points of include/sphvisc.h: argument checks, dispatch and
// the thread-local error message.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "apply.cuh"
#include "sph_internal.cuh"

namespace sph {

static thread_local char g_err[512] = {0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = 0; }

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void prof_begin(sph_neighbors* H, cudaStream_t st, int phase) {
  const int idx = H->prof_seq++;
  H->prof_armed = false;
  if (!H->prof_on || H->prof_used + 2 > 256 || (idx >> 1) % kProfStride != 0) return;
  H->prof_phase[H->prof_used / 2] = phase;
  H->prof_idx[H->prof_used / 2] = idx;
  cudaEventRecord(H->prof_ev[H->prof_used], st);
  H->prof_armed = true;
}
void prof_end(sph_neighbors* H, cudaStream_t st) {
  if (!H->prof_armed) return;
  cudaEventRecord(H->prof_ev[H->prof_used + 1], st);
  H->prof_used += 2;
  H->prof_armed = false;
}
void standalone_begin(sph_neighbors* H, cudaStream_t st) {
  if (H->prof_on && H->sa_ev[0]) cudaEventRecord(H->sa_ev[0], st);
}
sph_status standalone_end(sph_neighbors* H, cudaStream_t st, int form) {
  if (!H->prof_on || !H->sa_ev[0]) return SPH_OK;
  SPH_TRY_CUDA(cudaEventRecord(H->sa_ev[1], st));
  SPH_TRY_CUDA(cudaEventSynchronize(H->sa_ev[1]));
  float ms = 0.f;
  SPH_TRY_CUDA(cudaEventElapsedTime(&ms, H->sa_ev[0], H->sa_ev[1]));
  H->sa_ms[form] += ms;
  H->sa_n[form] += 1;
  return SPH_OK;
}
void prof_flush(sph_neighbors* H, int valid_launches) {
  if (!H->prof_on) return;
  const int pairs = H->prof_used / 2;
  for (int k = 0; k < pairs; ++k) {
    if (H->prof_idx[k] >= valid_launches) continue;   // launched after convergence: exits at once
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, H->prof_ev[2 * k], H->prof_ev[2 * k + 1]) == cudaSuccess) {
      H->prof_ms += ms;
      H->prof_n += 1;
      const int ph = H->prof_phase[k] ? 1 : 0;
      H->prof_ms_ph[ph] += ms;
      H->prof_n_ph[ph] += 1;
    }
  }
  H->prof_used = 0;
  H->prof_seq = 0;
}

sph_status set_viscosity_impl(sph_neighbors* H, const float* mu, cudaStream_t st);
sph_status mu_papanastasiou(sph_neighbors* H, const float* vel, const float* wall_vel, double tau0, double mu0,
                            double m, float* mu_out, int set_handle, cudaStream_t st);

}  // namespace sph

using namespace sph;

static inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char* sph_last_error(void) { return g_err; }

const char* sph_version(void) { return "sphvisc 0.1 (sm_103a)"; }

sph_status sph_build_neighbors(const sph_scene* scene, int32_t max_neighbors, sph_neighbors** handle,
                               void* stream) {
  clear_error();
  return build_neighbors(scene, max_neighbors, handle, as_stream(stream));
}

sph_status sph_neighbors_info(const sph_neighbors* h, int64_t* n, int64_t* nnz, int32_t* max_count) {
  clear_error();
  if (!h) {
    set_error("sph_neighbors_info: null handle");
    return SPH_ERR_INVALID;
  }
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (max_count) *max_count = h->max_cnt;
  return SPH_OK;
}

sph_status sph_neighbors_export(const sph_neighbors* h, int64_t* offsets, int32_t* idx, void* stream) {
  clear_error();
  return export_neighbors(h, offsets, idx, as_stream(stream));
}

sph_status sph_set_viscosity(sph_neighbors* h, const float* mu, void* stream) {
  clear_error();
  if (!h || !mu) {
    set_error("sph_set_viscosity: null argument");
    return SPH_ERR_INVALID;
  }
  return set_viscosity_impl(h, mu, as_stream(stream));
}

sph_status sph_neighbors_destroy(sph_neighbors* h) {
  clear_error();
  if (!h) return SPH_OK;
  h->pos_s.release();
  h->rho_s.release();
  h->mu_s.release();
  h->type_s.release();
  h->perm.release();
  h->iperm.release();
  h->key_s.release();
  h->cell_start.release();
  h->cell_rank.release();
  h->cnt.release();
  h->slice_off.release();
  h->nbr.release();
  h->op_cnt.release();
  h->op_off.release();
  h->op_ih.release();
  h->op_lo.release();
  h->op_kind.release();
  h->invD.release();
  h->D64.release();
  h->aux_df.release();
  h->feat_tmp.release();
  h->feat_scale.release();
  h->feat_out.release();
  h->feat_delta.release();
  h->feat_hp.release();
  h->feat_den.release();
  h->v_x2.release();
  h->tmp_i32a.release();
  h->tmp_i32b.release();
  h->tmp_i64.release();
  h->flags.release();
  h->v_r.release();
  h->v_rh.release();
  h->v_p.release();
  h->v_Ap.release();
  h->v_rs.release();
  h->v_As.release();
  h->v_d.release();
  h->v_tmp.release();
  h->x64.release();
  h->b64.release();
  h->r64.release();
  h->partials.release();
  h->counters.release();
  h->counters64.release();
  h->scal.release();
  h->scal_tune.release();
  for (auto& w : h->w64) w.release();
  h->op_loc.release();
  h->uni.release();
  h->unum.release();
  h->wpart.release();
  if (h->stage) {
    h->stage->release();
    delete h->stage;
  }
  release_step_stage(h);
  h->otf_g.release();
  h->otf_im.release();
  h->otf_rb.release();
  h->rs_caller.release();
  h->invD_sc.release();
  h->D64_sc.release();
  for (auto& e : h->prof_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->sa_ev)
    if (e) cudaEventDestroy(e);
  if (h->host_scal) cudaFreeHost(h->host_scal);
  if (h->host_flags) cudaFreeHost(h->host_flags);
  delete h;
  return SPH_OK;
}

sph_status sph_visc_setup(sph_neighbors* h, const sph_visc_params* params, void* stream) {
  clear_error();
  if (!h) {
    set_error("sph_visc_setup: null handle");
    return SPH_ERR_INVALID;
  }
  return ensure_operator(h, params, as_stream(stream));
}

sph_status sph_visc_apply(sph_neighbors* h, const sph_visc_params* params, const float* v, float* y,
                          void* stream) {
  clear_error();
  if (v == y && v) {
    set_error("sph_visc_apply: v and y must not overlap");
    return SPH_ERR_INVALID;
  }
  return visc_apply(h, params, v, y, as_stream(stream));
}

sph_status sph_visc_apply_otf(sph_neighbors* h, const sph_visc_params* params, const float* v, float* y,
                              void* stream) {
  clear_error();
  if (v == y && v) {
    set_error("sph_visc_apply_otf: v and y must not overlap");
    return SPH_ERR_INVALID;
  }
  return visc_apply_otf(h, params, v, y, as_stream(stream));
}

sph_status sph_visc_apply_noalloc(sph_neighbors* h, const sph_visc_params* params, const float* v, float* y,
                                  void* stream) {
  clear_error();
  return visc_apply_noalloc(h, params, v, y, as_stream(stream));
}

sph_status sph_visc_residual(sph_neighbors* h, const sph_visc_params* params, const double* x, const double* b,
                             double* r, void* stream) {
  clear_error();
  return visc_residual(h, params, x, b, r, as_stream(stream));
}

sph_status sph_visc_solve(sph_neighbors* h, const sph_visc_params* params, const sph_solve_opts* opts,
                          const double* b, double* x, sph_solve_report* report, void* stream) {
  clear_error();
  if (!h || !params || !opts || !b || !x || !report) {
    set_error("sph_visc_solve: null argument");
    return SPH_ERR_INVALID;
  }
  if (opts->rtol < 0.0 || opts->eps_inner < 0.0 || opts->eps_inner >= 1.0 || opts->maxit < 0 ||
      opts->max_refine < 0 || opts->chunk < 0) {
    set_error("sph_visc_solve: invalid options (rtol >= 0, 0 <= eps_inner < 1, maxit/max_refine/chunk >= 0)");
    return SPH_ERR_INVALID;
  }
  if (opts->apply_form < 0 || opts->apply_form > kApplyVariants || opts->launch_mode < 0 || opts->launch_mode > 1) {
    set_error("sph_visc_solve: apply_form %d outside 0..%d or launch_mode %d neither 0 nor 1", opts->apply_form,
              kApplyVariants, opts->launch_mode);
    return SPH_ERR_INVALID;
  }
  if (opts->precision == SPH_PREC_FP64 && (opts->method != SPH_SOLVER_BICGSTAB || !opts->jacobi)) {
    set_error("sph_visc_solve: the float64 solve is the Jacobi-scaled BiCGSTAB (method 0, jacobi 1)");
    return SPH_ERR_INVALID;
  }
  if (opts->precision == SPH_PREC_FP64 && h->row_scaled) {
    set_error("sph_visc_solve: a row scale applies to the mixed-precision solves; clear it for the float64 solve");
    return SPH_ERR_INVALID;
  }
  if (opts->precision == SPH_PREC_MIXED) return solve_mixed(h, params, opts, b, x, report, as_stream(stream));
  if (opts->precision == SPH_PREC_FP64) return solve_fp64(h, params, opts, b, x, report, as_stream(stream));
  set_error("sph_visc_solve: unknown precision %d", opts->precision);
  return SPH_ERR_INVALID;
}

sph_status sph_mu_papanastasiou(sph_neighbors* h, const float* vel, const float* wall_vel, double tau0, double mu0,
                                double m, float* mu_out, int32_t set_handle, void* stream) {
  clear_error();
  if (!h || !vel || !wall_vel || !mu_out) {
    set_error("sph_mu_papanastasiou: null argument");
    return SPH_ERR_INVALID;
  }
  if (!(tau0 >= 0.0) || !(mu0 > 0.0) || !(m > 0.0)) {
    set_error("sph_mu_papanastasiou: need tau0 >= 0, mu0 > 0, m > 0");
    return SPH_ERR_INVALID;
  }
  return mu_papanastasiou(h, vel, wall_vel, tau0, mu0, m, mu_out, set_handle, as_stream(stream));
}

sph_status sph_step(sph_state* state, const sph_step_params* params, const sph_solve_opts* opts,
                    sph_neighbors** handle, sph_step_report* report, void* stream) {
  clear_error();
  return time_step(state, params, opts, handle, report, as_stream(stream));
}

sph_status sph_shard_plan(int64_t n, const int32_t* layer, int32_t nlayers, int32_t ranks, int64_t* virt,
                          int32_t* rank_first_layer, int64_t* layer_first_virt) {
  clear_error();
  return shard_plan(n, layer, nlayers, ranks, virt, rank_first_layer, layer_first_virt);
}

sph_status sph_shard_create(sph_neighbors* h, const sph_visc_params* params, int32_t ranks, sph_shard** shard,
                            void* stream) {
  clear_error();
  return shard_create(h, params, ranks, shard, as_stream(stream));
}

sph_status sph_shard_info(const sph_shard* shard, int32_t* axis, int32_t* layers, int64_t* owned, int64_t* halo,
                          int64_t* exchanged) {
  clear_error();
  return shard_info(shard, axis, layers, owned, halo, exchanged);
}

sph_status sph_shard_set_striping(sph_shard* shard, int32_t on) {
  clear_error();
  return shard_set_striping(shard, on);
}

sph_status sph_shard_solve(sph_shard* shard, const sph_solve_opts* opts, const double* b, double* x,
                           sph_solve_report* report, void* stream) {
  clear_error();
  return shard_solve(shard, opts, b, x, report, as_stream(stream));
}

sph_status sph_shard_destroy(sph_shard* shard) {
  clear_error();
  return shard_destroy(shard);
}

sph_status sph_bicgstab_replay(const double* gamma0, double eps, int32_t maxit, int32_t nsteps, const double* dots,
                               double* out, void* stream) {
  clear_error();
  return bicgstab_replay(gamma0, eps, maxit, nsteps, dots, out, as_stream(stream));
}

sph_status sph_profile_enable(sph_neighbors* h, int32_t on) {
  clear_error();
  if (!h) {
    set_error("sph_profile_enable: null handle");
    return SPH_ERR_INVALID;
  }
  if (on) {
    for (auto& e : h->prof_ev)
      if (!e) SPH_TRY_CUDA(cudaEventCreate(&e));
    for (auto& e : h->sa_ev)
      if (!e) SPH_TRY_CUDA(cudaEventCreate(&e));
  }
  h->prof_on = on != 0;
  h->prof_used = 0;
  h->prof_seq = 0;
  h->prof_armed = false;
  return SPH_OK;
}

sph_status sph_profile_read(sph_neighbors* h, sph_profile_counters* out, int32_t reset) {
  clear_error();
  if (!out) {
    set_error("sph_profile_read: null output");
    return SPH_ERR_INVALID;
  }
  std::memset(out, 0, sizeof(*out));
  out->launches = g_launches.load();
  if (h) {
    out->apply_launches = h->prof_n;
    out->apply_ms = h->prof_ms;
    out->op_nnz = h->op_nnz;
    out->apply_bytes = 8 * h->op_nnz + (16 + 16 + 16 + 9) * h->n;
    for (int k = 0; k < 2; ++k) {
      out->phase_launches[k] = h->prof_n_ph[k];
      out->phase_ms[k] = h->prof_ms_ph[k];
    }
    out->apply_variant[0] = h->apply_var[0];
    out->apply_variant[1] = h->apply_var[1] > h->apply_var[2] ? h->apply_var[1] : h->apply_var[2];
    for (int ph = 0; ph < 3; ++ph)
      for (int v = 0; v < kApplyVariants; ++v) out->tune_us[ph][v] = h->tune_us[ph][v];
    for (int f = 0; f < 2; ++f) {
      out->standalone_launches[f] = h->sa_n[f];
      out->standalone_ms[f] = h->sa_ms[f];
    }
    out->otf_bytes = 4 * h->nnz + (16 + 16 + 16 + 4 + 4 + 4 + 1) * h->n;
    out->apply_grid[0] = h->apply_grid[0];
    out->apply_grid[1] = h->apply_grid[1] > 0 ? h->apply_grid[1] : h->apply_grid[2];
    if (reset) {
      h->prof_n = 0;
      h->prof_ms = 0.0;
      h->prof_n_ph[0] = h->prof_n_ph[1] = 0;
      h->prof_ms_ph[0] = h->prof_ms_ph[1] = 0.0;
      h->sa_n[0] = h->sa_n[1] = 0;
      h->sa_ms[0] = h->sa_ms[1] = 0.0;
    }
  }
  return SPH_OK;
}

}  // extern "C"
