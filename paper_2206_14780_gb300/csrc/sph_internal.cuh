// Internal declarations of the sphvisc library (not part of the C ABI).
//
// Data layout in HBM (all in the cell-sorted particle order "s"):
//   pos_s   float4[n_pad]   x, y, z, m
//   rho_s, mu_s float[n_pad]; type_s uint8[n_pad]
//   perm    int32[n]        sorted -> caller index;  iperm: caller -> sorted
//   neighbour lists: sliced ELL with slices of 32 rows (SELL-32): row s of
//   slice k = s / 32 keeps its j-th entry at slice_off[k] + 32 j + (s % 32),
//   so a warp reading entry j of its 32 rows touches 128 consecutive bytes.
//   The lists have a fixed capacity (slice_off[k] = 32 k max_neighbors: built
//   in one pass); the operator keeps its own SELL-32 with each slice as wide as
//   its longest row (only the entries with a coefficient).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>

#include "sphvisc.h"

namespace sph {

constexpr int kSlice = 32;        // rows per SELL slice (one warp)
constexpr int kBlock = 256;       // threads per block of the row kernels
constexpr int kMaxDots = 15;      // float64 partial sums one reduction may carry

// truncated Gaussian kernel (Sec. 5.2): radius k = 3 and its normalisation
// w_G = pi^{3/2} erf(k) - (2 pi / 3) e^{-k^2} k (3 + 2 k^2)
constexpr double kGaussK = 3.0;
inline double gauss_norm() {
  const double k = kGaussK, pi = 3.14159265358979323846;
  return std::pow(pi, 1.5) * std::erf(k) - 2.0 * pi / 3.0 * std::exp(-k * k) * k * (3.0 + 2.0 * k * k);
}

void set_error(const char* fmt, ...);
void clear_error();
void note_launch();        // counts kernel launches (sph_profile_read)
void note_launches(int k); // graph replays: the kernels each replay runs

// every kernel launch of the library goes through this macro so it is counted
#define SPH_LAUNCH(kernel, ...) ::sph::note_launch(), kernel<<<__VA_ARGS__>>>

// Programmatic dependent launch of a kernel of the BiCGSTAB loop: the launch is
// processed while its predecessor on the stream is still running, and the
// kernel's first statement, griddep_wait(), holds its threads until that
// predecessor has completed and its memory is visible (so the data order is
// the stream's).  No kernel triggers its dependants early, so a dependant is
// scheduled once every block of its predecessor has exited: an early trigger
// (griddepcontrol.launch_dependents at kernel start) let the dependant's
// waiting blocks take SM slots during the predecessor's tail and measured
// 0.8 ms per solve slower on the 1.16M box.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
  note_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// first statement of every kernel launch_pdl may launch (a no-op otherwise)
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define SPH_TRY_CUDA(call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::sph::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return (e_ == cudaErrorMemoryAllocation) ? SPH_ERR_NOMEM : SPH_ERR_CUDA;             \
    }                                                                                    \
  } while (0)

#define SPH_TRY(expr)                         \
  do {                                        \
    sph_status s_ = (expr);                   \
    if (s_ != SPH_OK) return s_;              \
  } while (0)

// A device allocation owned by the handle.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  sph_status alloc(size_t count) {
    if (count <= n && p) return SPH_OK;
    release();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
      return SPH_ERR_NOMEM;
    }
    n = count;
    return SPH_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Scalars of one inner BiCGSTAB pass, float64, in device memory.
struct SolverScalars {
  double gamma[3];     // r0^ . r
  double delta[3];     // r0^ . A p
  double alpha[3];     // gamma / delta
  double alpha_p[3];   // alpha' = gamma_{i+1} / delta_i
  double beta[3];      // alpha' / omega
  double omega[3];     // (r*.Ar*) / (Ar*.Ar*)
  double rr[3];        // r . r after the update
  double tau2[3];      // max(eps^2 b.b, FLT_MIN)
  double dots[kMaxDots];  // last raw reduction result (debug / outer norms)
  int32_t state[3];    // SPH_CONVERGED / SPH_STALLED / SPH_PROGRESSING
  int32_t stall_now[3];
  int32_t stalled_any[3];
  int32_t iter;        // iterations of this pass
  int32_t maxit;       // cap for this pass
  int32_t done;        // 1: no component progressing or cap reached
  int32_t nonfinite;   // a scalar went NaN/Inf
  int32_t pad;
  int32_t fault;       // an apply kernel gave up a bounded wait (SPH_ERR_TIMEOUT)
  int32_t pad2;
};

struct Grid {
  int ncell[3];
  double cell[3];     // cell side per axis (>= 2h)
  double lo[3];
  double L[3];        // hi - lo
  int periodic[3];
  int64_t ncells;
};

}  // namespace sph

namespace sph {
struct StepStage;   // step.cu: the time step's buffers (owned by the handle)
// device staging of sph_visc_solve_host (owned by the handle)
struct HostStage {
  DBuf<float4> pos, vel;
  DBuf<float> rho, mu;
  DBuf<uint8_t> type;
  DBuf<double> b, x;
  void release() {
    pos.release();
    vel.release();
    rho.release();
    mu.release();
    type.release();
    b.release();
    x.release();
  }
};
}  // namespace sph

// The opaque handle of the C ABI.
struct sph_neighbors {
  int64_t n = 0;
  int64_t n_pad = 0;        // n rounded up to a whole number of slices
  int64_t nslices = 0;
  sph::Grid grid{};
  float h = 0.f;
  int kernel = SPH_KERNEL_WENDLAND;   // smoothing kernel (support radius 2h or 3h)
  int device = 0;
  int num_sms = 0;

  // cell-sorted particle copy
  sph::DBuf<float4> pos_s;
  sph::DBuf<float> rho_s, mu_s;
  sph::DBuf<uint8_t> type_s;
  sph::DBuf<int32_t> perm, iperm, key_s;
  sph::DBuf<int32_t> cell_start;   // [ncells + 1], indexed by Morton rank of the cell
  sph::DBuf<int32_t> cell_rank;    // [ncells] row-major cell -> rank along a Morton curve
  int rank_dims[3] = {0, 0, 0};

  // neighbour SELL-32
  sph::DBuf<int32_t> cnt;          // [n_pad]
  sph::DBuf<int64_t> slice_off;    // [nslices + 1]
  sph::DBuf<int32_t> nbr;          // [nnz_pad = n_pad max_neighbors] neighbour rows
  int64_t nnz = 0, nnz_pad = 0;
  int32_t max_cnt = 0;

  // operator (coefficients of A(dt)) SELL-32
  bool op_valid = false;
  sph_visc_params op_params{};
  uint64_t mu_version = 0, op_mu_version = ~0ull;
  sph::DBuf<int32_t> op_cnt;       // [n_pad]
  sph::DBuf<int64_t> op_off;       // [nslices + 1]
  sph::DBuf<int2> op_ih;           // [op_nnz_pad] (row, bits of float32 hi)
  sph::DBuf<float> op_lo;          // a = hi + lo reproduces the float64 coefficient
  sph::DBuf<uint8_t> op_kind;      // 0 fluid (difference form), 1 Shepard wall, 2 identity
  sph::DBuf<float> invD;           // float32 1/D (Jacobi), 1 for wall rows
  sph::DBuf<double> D64;           // float64 D
  sph::DBuf<float4> aux_df;        // per particle (m / rho, 1 / mu) as double-float pairs
  int64_t op_nnz_pad = 0;
  uint64_t op_version = 0;         // bumped whenever the operator is rebuilt
  sph::DBuf<int32_t> wpart;        // balanced per-warp slice ranges (OpView::wpart)
  sph::HostStage* stage = nullptr; // sph_visc_solve_host's device copies of its host buffers
  sph::StepStage* step = nullptr;  // sph_step's buffers
  int64_t wpart_nw = 0;
  uint64_t wpart_version = ~0ull;  // op_version they were cut for

  // shared-memory apply form (apply_union.cu): per-slice neighbour unions
  bool union_valid = false;
  uint64_t union_op_version = 0;
  sph::DBuf<int2> op_loc;          // [op_nnz_pad] (position in the slice's union, coefficient bits)
  sph::DBuf<int32_t> uni;          // [op_nnz_pad] the slice's distinct neighbour rows, at its offset
  sph::DBuf<int32_t> unum;         // [nslices] union size, -1 above kUnionCap

  // on-the-fly apply (apply_otf.cu): packed geometry for the operator of op_version
  bool otf_valid = false;
  uint64_t otf_op_version = 0;
  sph::DBuf<float4> otf_g;         // (x, y, z, +-V), V = m / rho, negative for walls
  sph::DBuf<float> otf_im, otf_rb; // 1/mu (or mu), R_b = 2 dt 105/(128 pi) / (h^5 rho_b)

  // scratch used by builds and solves
  sph::DBuf<int32_t> tmp_i32a, tmp_i32b;
  sph::DBuf<int64_t> tmp_i64;
  sph::DBuf<int32_t> flags;        // device error flags [8]

  // solver workspace
  sph::DBuf<float4> v_r, v_rh, v_p, v_Ap, v_rs, v_As, v_d, v_tmp;
  sph::DBuf<double> x64, b64, r64;   // [n_pad][3]
  sph::DBuf<float4> v_x2;            // x64 split into float32 hi, lo interleaved [2 n_pad] (residual)
  sph::DBuf<double> partials;        // [grid][kMaxDots]
  sph::DBuf<unsigned int> counters;  // last-block counters
  sph::DBuf<unsigned int> counters64;  // last-block counters of the float64 solve
  sph::DBuf<sph::SolverScalars> scal;
  int32_t* host_flags = nullptr;     // pinned [4]
  sph::SolverScalars* host_scal = nullptr;  // pinned
  int red_grid = 0;                  // blocks of the reducing kernels
  // apply autotuner (autotune.cu): chosen row-loop form and grid per phase
  int apply_var[3] = {0, 0, 0};
  int apply_grid[3] = {0, 0, 0};
  float tune_us[3][6] = {};
  bool tuned = false;
  int64_t tuned_n_pad = 0;
  int force_form = -1;               // sph_solve_opts.apply_form - 1 for the current solve
  // iterations of each inner pass of the last mixed solve with each of two time
  // steps (sizes the launch chunks; a time step alternates the predictor's dt/2
  // and the corrector's dt on one handle)
  static constexpr int kPassHist = 16;
  int pass_len[2][kPassHist] = {};
  double pass_dt[2] = {-1.0, -1.0};
  int pass_slot_next = 0;
  int force_grid = 0;
  sph::DBuf<sph::SolverScalars> scal_tune;

  // instrumentation (sph_profile_*)
  bool prof_on = false;
  cudaEvent_t prof_ev[256] = {};
  int prof_used = 0;
  double prof_ms = 0.0;
  int64_t prof_n = 0;
  int prof_phase[128] = {};
  int prof_idx[128] = {};      // launch index within the chunk of each recorded pair
  int prof_seq = 0;            // apply launches since the last flush
  bool prof_armed = false;     // the current launch has its begin event recorded
  double prof_ms_ph[2] = {0.0, 0.0};
  int64_t prof_n_ph[2] = {0, 0};
  int64_t op_nnz = 0;
  // stand-alone applies (sph_visc_apply, sph_visc_apply_otf): [0] stored, [1] on the fly
  cudaEvent_t sa_ev[2] = {};
  double sa_ms[2] = {0.0, 0.0};
  int64_t sa_n[2] = {0, 0};

  // learned warm start (features.cu)
  sph::DBuf<float4> feat_tmp;        // sorted v, A v, e1, e2
  sph::DBuf<double> feat_scale;      // sum |v|^2 and count over the fluid
  sph::DBuf<uint32_t> feat_out;      // bf16 features [n][16]
  sph::DBuf<float4> feat_delta;      // network output [n]
  sph::DBuf<float4> feat_hp;         // high-passed network output [n] (caller order)
  sph::DBuf<float> feat_den;         // Shepard denominators [n_pad] (sorted)

  // float64 solve vectors r, r0^, p, Ap, r*, Ar* ([n_pad][3] each)
  sph::DBuf<double> w64[7];

  // per-row preconditioner scale (row_scale.cu): s (caller order) multiplies the
  // Jacobi diagonal's inverse of every row in the mixed-precision solves
  bool row_scaled = false;
  sph::DBuf<float> rs_caller;        // [n] s, caller order
  sph::DBuf<float> invD_sc;          // [n_pad] s / D (sorted)
  sph::DBuf<double> D64_sc;          // [n_pad] D / s (sorted)
  uint64_t rs_op_version = ~0ull;    // op_version the scaled diagonals were made for
  uint64_t rs_version = 0;           // bumped by every sph_set_row_scale
};

namespace sph {

// neighbors.cu
sph_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t m, cudaStream_t st);
sph_status slice_offsets(const int32_t* cnt, int64_t nslices, int64_t* off, int32_t* width_tmp,
                         cudaStream_t st);

sph_status build_slices(sph_neighbors* H, const int32_t* cnt, int64_t* off, int64_t* total_pad, int64_t* total,
                        int32_t* maxc, cudaStream_t st);
sph_status build_neighbors(const sph_scene* sc, int32_t maxnb, sph_neighbors** out, cudaStream_t st);
sph_status export_neighbors(const sph_neighbors* H, int64_t* offsets, int32_t* idx, cudaStream_t st);

// operator.cu
void launch_residual_f64(const sph_neighbors* H, int grid, const double* x, const double* b, double* r,
                         double* partials, unsigned int* counter, double* res_out, cudaStream_t st);
// r -= A d (sorted [n_pad][3] float64 r, float32 d), same reduction outputs
void launch_residual_update(const sph_neighbors* H, int grid, const float4* d, double* r, double* partials,
                            unsigned int* counter, double* res_out, cudaStream_t st);
// per-warp slice ranges balanced by streamed bytes for a grid of `grid` blocks of
// kBlock threads (rebuilt when the operator or the warp count changes)
sph_status ensure_wpart(sph_neighbors* H, int grid, cudaStream_t st);
sph_status visc_apply(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y, cudaStream_t st);
sph_status visc_apply_noalloc(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y,
                              cudaStream_t st);
sph_status ensure_operator(sph_neighbors* H, const sph_visc_params* P, cudaStream_t st);
void launch_apply_f32(const sph_neighbors* H, const float4* v, float4* y, bool jacobi, cudaStream_t st);
// apply_otf.cu: y = A v with the coefficients recomputed per pair
void launch_apply_otf(const sph_neighbors* H, const float4* v, float4* y, bool jacobi, cudaStream_t st);
// apply_union.cu: per-slice unions for apply form 5 (built once per operator)
sph_status ensure_union(sph_neighbors* H, cudaStream_t st);
// dynamic shared memory of an apply form (bytes) and its one-time attribute set-up
size_t apply_smem(int variant);
sph_status apply_prepare(sph_neighbors* H, int variant, cudaStream_t st);
sph_status visc_apply_otf(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y, cudaStream_t st);
// CUDA-event timing of one stand-alone apply launch when profiling is on (synchronises)
void standalone_begin(sph_neighbors* H, cudaStream_t st);
sph_status standalone_end(sph_neighbors* H, cudaStream_t st, int form);
struct OpView;
OpView op_view(const sph_neighbors* H);

// row_scale.cu: the scaled diagonals for the operator of H->op_version (no-op
// without a row scale)
sph_status row_scale_refresh(sph_neighbors* H, cudaStream_t st);
using ApplyDotFn = void (*)(OpView, const float4*, float4*, const float4*, SolverScalars*, double*, unsigned int*);
ApplyDotFn apply_kernel(int phase, int variant);
sph_status autotune_apply(sph_neighbors* H, bool merged, unsigned int* counter, cudaStream_t st);

// solver.cu
sph_status solve_mixed(sph_neighbors* H, const sph_visc_params* P, const sph_solve_opts* O,
                       const double* b, double* x, sph_solve_report* R, cudaStream_t st);
sph_status visc_residual(sph_neighbors* H, const sph_visc_params* P, const double* x, const double* b, double* r,
                         cudaStream_t st);
sph_status ensure_workspace(sph_neighbors* H);
sph_status solve_fp64(sph_neighbors* H, const sph_visc_params* P, const sph_solve_opts* O,
                      const double* b, double* x, sph_solve_report* R, cudaStream_t st);

int grid_for(const sph_neighbors* H, int64_t work_items, int block = kBlock);

// shard.cu: one system over several sub-domains (sph_shard_*)
sph_status shard_plan(int64_t n, const int32_t* layer, int32_t nlayers, int32_t ranks, int64_t* virt,
                      int32_t* rank_first_layer, int64_t* layer_first_virt);
sph_status shard_create(sph_neighbors* H, const sph_visc_params* P, int32_t ranks, sph_shard** out, cudaStream_t st);
sph_status shard_destroy(sph_shard* Z);
sph_status shard_set_striping(sph_shard* Z, int32_t on);
sph_status shard_info(const sph_shard* Z, int32_t* axis, int32_t* layers, int64_t* owned, int64_t* halo,
                      int64_t* exchanged);
sph_status shard_solve(sph_shard* Z, const sph_solve_opts* O, const double* b, double* x, sph_solve_report* R,
                       cudaStream_t st);

// step.cu: the semi-implicit predictor/corrector step (sph_step)
sph_status time_step(sph_state* S, const sph_step_params* P, const sph_solve_opts* O, sph_neighbors** handle,
                     sph_step_report* R, cudaStream_t st);
void release_step_stage(sph_neighbors* H);
// features.cu: x0 = v^n with the dummy-wall closure
sph_status warm_start_plain(sph_neighbors* h, const sph_visc_params* params, const float* vel, const uint8_t* ptype,
                            const double* b, double* x0, cudaStream_t st);
sph_status mu_papanastasiou(sph_neighbors* H, const float* vel, const float* wall_vel, double tau0, double mu0,
                            double m, float* mu_out, int set_handle, cudaStream_t st);

// replay.cu: the solver's scalar steps on caller-given dots (sph_bicgstab_replay)
sph_status bicgstab_replay(const double* gamma0, double eps, int32_t maxit, int32_t nsteps, const double* dots,
                           double* out, cudaStream_t st);

// event pair around the two apply launches of every kProfStride-th iteration
// when profiling is on (sampling keeps the event records from slowing the
// loop they time); prof_flush folds the recorded pairs of launches that did
// work into prof_ms (call only after a stream synchronisation)
constexpr int kProfStride = 8;
void prof_begin(sph_neighbors* H, cudaStream_t st, int phase = 0);
void prof_end(sph_neighbors* H, cudaStream_t st);
void prof_flush(sph_neighbors* H, int valid_launches);

}  // namespace sph
