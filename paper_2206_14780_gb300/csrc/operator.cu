// The viscous matrix A(dt) (paper Sec. 3.2), its float32 apply and its float64
// true residual.
//
// Row kinds (stored per row):
//   0 fluid    (A v)_b = v_b + sum_a a_ba (v_b - v_a),  a_ba = dt c_ab,
//              c_ab = 2 mubar_ab m_a |F_ab| / (rho_a rho_b)      (Eqs. kab, diag, offdiag)
//   1 Shepard  (A v)_b = v_b + sum_{a fluid} a_ba v_a,  a_ba = W_ba / S_b
//              (dummy wall, Eq. implicit-system-dummy-full)
//   2 identity (A v)_b = v_b  (dynamic wall; dummy wall with S_b = 0)
// The fluid rows use the difference form: its float32 rounding stays relative
// to the result even when dt sum c is in the thousands.
//
// Coefficients are evaluated once per (dt, boundary, mean, mu) in double-float
// arithmetic (dfloat.cuh; float64 only for per-row constants) and kept as a
// float32 pair a = hi + lo: the float32 apply reads hi only, the float64-accurate
// residual reads hi + lo (relative error a few 2^-45).
#include <cmath>

#include "apply.cuh"
#include "dfloat.cuh"
#include "reduce.cuh"
#include "residual_row.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

struct OpGeom {
  double L[3];
  double invL[3];
  int periodic[3];
  double h;
  double inv_h;
};

// per particle: V = m / rho and 1 / mu, evaluated in float64 once per particle
// and kept as double-float pairs (V hi, V lo, 1/mu hi, 1/mu lo)
__global__ void k_op_aux(const float4* __restrict__ pos, const float* __restrict__ rho, const float* __restrict__ mu,
                         int64_t n_pad, float4* __restrict__ aux) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const dfl V = df_from_double((double)pos[s].w / (double)rho[s]);
    const dfl im = df_from_double(1.0 / (double)mu[s]);
    aux[s] = make_float4(V.hi, V.lo, im.hi, im.lo);
  }
}

// Geometry of the double-float set-up: periods as (hi, lo), 1/h as (hi, lo)
struct OpGeomDF {
  dfl L[3];
  float invL[3];
  int periodic[3];
  dfl inv_h;
};

// |r_a - r_b| in double-float: the coordinate differences of the float32
// positions exactly (TwoSum), the minimum image by a whole period, the squared
// norm with exact products, one Newton step on the root
__device__ __forceinline__ dfl pair_r_df(float4 pa, float4 pb, const OpGeomDF& g) {
  dfl d[3] = {df_exact_sum(pa.x, -pb.x), df_exact_sum(pa.y, -pb.y), df_exact_sum(pa.z, -pb.z)};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (g.periodic[ax]) {
      const float k = rintf(d[ax].hi * g.invL[ax]);
      if (k != 0.f) d[ax] = df_add(d[ax], dfl{-k * g.L[ax].hi, -k * g.L[ax].lo});
    }
  }
  const dfl r2 = df_add(df_add(df_mul(d[0], d[0]), df_mul(d[1], d[1])), df_mul(d[2], d[2]));
  return df_sqrt(r2);
}

// Wendland psi_{3,1} without its constant factor (it cancels in W / S):
// (1 - q/2)^4 (2q + 1), zero for q >= 2
__device__ __forceinline__ dfl wendland_w_df(dfl q) {
  dfl t = df_add(dfl{1.f, 0.f}, dfl{-0.5f * q.hi, -0.5f * q.lo});
  if (t.hi <= 0.f) return dfl{0.f, 0.f};
  const dfl t2 = df_mul(t, t);
  return df_mul(df_mul(t2, t2), df_add(dfl{1.f, 0.f}, dfl{2.f * q.hi, 2.f * q.lo}));
}

// truncated Gaussian (Sec. 5.2, radius 3h): e^{-q^2} from the double-float q,
// the exponential in float64 once per pair (the set-up runs once per A(dt))
__device__ __forceinline__ dfl gauss_e_df(dfl q) { return df_from_double(exp(-df_to_double(df_mul(q, q)))); }

// the fluid coefficient's kernel factor: (2 - q)^3 (Wendland) or e^{-q^2} (Gaussian),
// each without the constant of |f| (it is in R_b)
__device__ __forceinline__ dfl fluid_kernel_df(dfl q, int gauss) {
  if (gauss) return gauss_e_df(q);
  dfl tq = df_add(dfl{2.f, 0.f}, df_neg(q));
  if (tq.hi <= 0.f) tq = dfl{0.f, 0.f};
  return df_mul(df_mul(tq, tq), tq);
}

// the Shepard weight w(q) without its constant: Wendland, or e^{-q^2} - e^{-9}
__device__ __forceinline__ dfl shepard_w_df(dfl q, int gauss, double gauss_tail) {
  if (gauss) return df_from_double(exp(-df_to_double(df_mul(q, q))) - gauss_tail);
  return wendland_w_df(q);
}

__global__ void k_op_count(const uint8_t* __restrict__ type, const int32_t* __restrict__ cnt,
                           const int64_t* __restrict__ slice_off, const int32_t* __restrict__ nbr, int64_t n,
                           int64_t n_pad, int boundary, int32_t* __restrict__ op_cnt, uint8_t* __restrict__ kind) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s >= n) {
      op_cnt[s] = 0;
      kind[s] = KIND_IDENTITY;
      continue;
    }
    const int c = cnt[s];
    if (type[s] == SPH_FLUID) {
      op_cnt[s] = c;
      kind[s] = KIND_FLUID;
      continue;
    }
    if (boundary != SPH_BC_DUMMY) {
      op_cnt[s] = 0;
      kind[s] = KIND_IDENTITY;
      continue;
    }
    // every neighbour lies strictly inside 2h, so each fluid neighbour has
    // W > 0 and the Shepard sum is positive exactly when there is one (a sum
    // that still rounds to zero is handled by k_op_fill as an identity row)
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    int nf = 0;
    for (int j = 0; j < c; ++j) nf += type[nbr[base + (int64_t)j * kSlice]] == SPH_FLUID ? 1 : 0;
    op_cnt[s] = nf;
    kind[s] = nf > 0 ? KIND_SHEPARD : KIND_IDENTITY;
  }
}

// Coefficients of A(dt) (Eq. kab with |F|, Eqs. diag, offdiag and dummyvel) in
// double-float arithmetic (relative error a few 2^-45), stored as the float32
// pair (hi, lo) that the float32 apply and the double-float residual read;
// float64 is used once per row (R_b, D) only, and for the Gaussian's exponential.
//   fluid row b:  a_ba = dt c_ab = R_b V_a mubar k(q), D_b = 1 + sum a, with
//                 Wendland  k = (2 - q)^3,  R_b = 2 dt (105 / (128 pi)) / (h^5 rho_b)
//                 Gaussian  k = e^{-q^2},   R_b = 2 dt (2 / w_G) / (h^5 rho_b)
//   dummy wall:   a_ba = W_ba / S_b over fluid neighbours
__global__ void k_op_fill(const float4* __restrict__ pos, const float* __restrict__ rho, const float* __restrict__ mu,
                          const uint8_t* __restrict__ type, const float4* __restrict__ aux,
                          const int32_t* __restrict__ cnt, const int64_t* __restrict__ slice_off,
                          const int32_t* __restrict__ nbr, const uint8_t* __restrict__ kind,
                          const int64_t* __restrict__ op_off, int64_t n, int64_t n_pad, OpGeom g64, double dt, int mean,
                          int gauss, double kf, double gauss_tail, int2* __restrict__ op_ih, float* __restrict__ op_lo,
                          float* __restrict__ invD, double* __restrict__ D64) {
  OpGeomDF g;
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = df_from_double(g64.L[ax]);
    g.invL[ax] = (float)g64.invL[ax];
    g.periodic[ax] = g64.periodic[ax];
  }
  g.inv_h = df_from_double(g64.inv_h);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s >= n || kind[s] == KIND_IDENTITY) {
      invD[s] = 1.f;
      D64[s] = 1.0;
      continue;
    }
    const float4 pb = pos[s];
    const int c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    const int64_t obase = op_off[s / kSlice] + (s % kSlice);
    int o = 0;
    if (kind[s] == KIND_FLUID) {
      const float mu_b = mu[s];
      const float4 ab = aux[s];
      const dfl imu_b{ab.z, ab.w};
      const dfl Rb = df_from_double(kf / (double)rho[s]);
      dfl sum{0.f, 0.f};
      for (int j = 0; j < c; ++j) {
        const int32_t t = nbr[base + (int64_t)j * kSlice];
        const float4 pa = pos[t];
        const float4 at = aux[t];
        const dfl q = df_mul(pair_r_df(pa, pb, g), g.inv_h);
        const dfl tq3 = fluid_kernel_df(q, gauss);
        dfl mub{mu_b, 0.f};
        if (type[t] == SPH_FLUID) {
          if (mean == SPH_MEAN_ARITHMETIC) {
            const dfl m2 = df_exact_sum(mu[t], mu_b);
            mub = dfl{0.5f * m2.hi, 0.5f * m2.lo};
          } else {
            const dfl h = df_rcp(df_add(dfl{at.z, at.w}, imu_b));
            mub = dfl{2.f * h.hi, 2.f * h.lo};
          }
        }
        const dfl a = df_mul(df_mul(Rb, dfl{at.x, at.y}), df_mul(mub, tq3));
        const int64_t e = obase + (int64_t)o * kSlice;
        op_ih[e] = make_int2(t, __float_as_int(a.hi));
        op_lo[e] = a.lo;
        sum = df_add(sum, a);
        ++o;
      }
      const double D = 1.0 + df_to_double(sum);
      D64[s] = D;
      invD[s] = __double2float_rn(1.0 / D);
    } else {  // Shepard wall row: W_ba / S_b over fluid neighbours
      dfl S{0.f, 0.f};
      for (int j = 0; j < c; ++j) {
        const int32_t t = nbr[base + (int64_t)j * kSlice];
        if (type[t] != SPH_FLUID) continue;
        S = df_add(S, shepard_w_df(df_mul(pair_r_df(pos[t], pb, g), g.inv_h), gauss, gauss_tail));
      }
      // S rounds to zero only if every fluid neighbour sits at q = 2 to within
      // rounding: zero coefficients then make the row an identity row (as an
      // empty Shepard sum does)
      const dfl invS = S.hi > 0.f ? df_rcp(S) : dfl{0.f, 0.f};
      for (int j = 0; j < c; ++j) {
        const int32_t t = nbr[base + (int64_t)j * kSlice];
        if (type[t] != SPH_FLUID) continue;
        const dfl a = df_mul(shepard_w_df(df_mul(pair_r_df(pos[t], pb, g), g.inv_h), gauss, gauss_tail), invS);
        const int64_t e = obase + (int64_t)o * kSlice;
        op_ih[e] = make_int2(t, __float_as_int(a.hi));
        op_lo[e] = a.lo;
        ++o;
      }
      invD[s] = 1.f;
      D64[s] = 1.0;
    }
  }
}

// y = A v (or D^-1 A v) in float32, one warp per 32-row slice, one row per lane.
template <bool JACOBI>
__global__ void __launch_bounds__(kBlock) k_apply_f32(OpView op, const float4* __restrict__ v, float4* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < op.nslices; sl += nwarps) {
    float4 vb;
    y[sl * kSlice + lane] = apply_row<8, false, JACOBI>(op, v, sl, lane, vb);
  }
}

__global__ void k_gather_f4(const float* __restrict__ v_caller, const int32_t* __restrict__ perm, int64_t n,
                            int64_t n_pad, float4* __restrict__ v_s) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      const float4 t = reinterpret_cast<const float4*>(v_caller)[perm[s]];
      v_s[s] = make_float4(t.x, t.y, t.z, 0.f);
    } else {
      v_s[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

__global__ void k_scatter_f4(const float4* __restrict__ y_s, const int32_t* __restrict__ perm, int64_t n,
                             float* __restrict__ y_caller) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<float4*>(y_caller)[perm[s]] = y_s[s];
}

// x64 -> float32 hi + lo (x = hi + lo to ~2^-48 relative)
__global__ void k_split_x(const double* __restrict__ x, int64_t n_pad, float4* __restrict__ x2) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = x[3 * s], x1 = x[3 * s + 1], x2c = x[3 * s + 2];
    const float h0 = (float)x0, h1 = (float)x1, h2 = (float)x2c;
    x2[2 * s] = make_float4(h0, h1, h2, 0.f);
    x2[2 * s + 1] = make_float4((float)(x0 - (double)h0), (float)(x1 - (double)h1), (float)(x2c - (double)h2), 0.f);
  }
}

// float64-accurate residual r = b - A x on sorted [n_pad][3] arrays, float32
// arithmetic per pair and float64 per row; partial sums of r_c^2 (K = 3) go
// through the grid reduction into res_out[0..3) when partials is given.
__global__ void __launch_bounds__(kBlock, 4) k_residual_df(OpView op, const float* __restrict__ op_lo,
                                                        const float4* __restrict__ x2,
                                                        const double* __restrict__ x, const double* __restrict__ b,
                                                        double* __restrict__ r, int64_t n, double* __restrict__ partials,
                                                        unsigned int* counter, double* __restrict__ res_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc2[3] = {0.0, 0.0, 0.0};
  const SliceRange R = warp_slices(op, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nwarps);
  for (int64_t sl = R.first; sl < R.end; sl += R.step) {
    const int64_t s = sl * kSlice + lane;
    const uint8_t k = op.kind[s];
    const float kap = (k == KIND_FLUID) ? 1.f : 0.f;
    DFAcc a0, a1, a2;
    residual_row_df(op, op_lo, x2, sl, lane, kap, a0, a1, a2);
    const double sg = (k == KIND_FLUID) ? 1.0 : (k == KIND_SHEPARD ? -1.0 : 0.0);
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    if (s < n) {
      r0 = b[3 * s] - (x[3 * s] + sg * a0.value());
      r1 = b[3 * s + 1] - (x[3 * s + 1] + sg * a1.value());
      r2 = b[3 * s + 2] - (x[3 * s + 2] + sg * a2.value());
    }
    r[3 * s] = r0;
    r[3 * s + 1] = r1;
    r[3 * s + 2] = r2;
    acc2[0] += r0 * r0;
    acc2[1] += r1 * r1;
    acc2[2] += r2 * r2;
  }
  if (partials == nullptr) return;
  block_partials_f64<3>(acc2, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x < 3) res_out[threadIdx.x] = res[threadIdx.x];
  }
}

// r64 -= A d for the float32 correction d of a refinement pass (x64 += d runs
// beside it), so r64 stays b - A x64 without re-reading x in two halves: A d is
// formed in double-float arithmetic on a = hi + lo, its error a few 2^-46 of the
// sum of |a_ba (d_b - d_a)|, far below the residual levels the solve resolves.
// Partial sums of the new r_c^2 go through the grid reduction into res_out.
__global__ void __launch_bounds__(kBlock, 4) k_residual_update_df(OpView op, const float* __restrict__ op_lo,
                                                               const float4* __restrict__ d, double* __restrict__ r,
                                                               int64_t n, double* __restrict__ partials,
                                                               unsigned int* counter, double* __restrict__ res_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc2[3] = {0.0, 0.0, 0.0};
  const SliceRange R = warp_slices(op, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nwarps);
  for (int64_t sl = R.first; sl < R.end; sl += R.step) {
    const int64_t s = sl * kSlice + lane;
    const uint8_t k = op.kind[s];
    const float kap = (k == KIND_FLUID) ? 1.f : 0.f;
    DFAcc a0, a1, a2;
    float4 db;
    residual_row_f32x(op, op_lo, d, sl, lane, kap, db, a0, a1, a2);
    const double sg = (k == KIND_FLUID) ? 1.0 : (k == KIND_SHEPARD ? -1.0 : 0.0);
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    if (s < n) {
      r0 = r[3 * s] - ((double)db.x + sg * a0.value());
      r1 = r[3 * s + 1] - ((double)db.y + sg * a1.value());
      r2 = r[3 * s + 2] - ((double)db.z + sg * a2.value());
    }
    r[3 * s] = r0;
    r[3 * s + 1] = r1;
    r[3 * s + 2] = r2;
    acc2[0] += r0 * r0;
    acc2[1] += r1 * r1;
    acc2[2] += r2 * r2;
  }
  block_partials_f64<3>(acc2, partials + (size_t)blockIdx.x * kMaxDots);
  if (arrive_last(counter)) {
    __shared__ double res[3];
    final_sum<3>(partials, counter, res);
    if (threadIdx.x < 3) res_out[threadIdx.x] = res[threadIdx.x];
  }
}

// Cut the slices into nw contiguous ranges of about equal streamed bytes: slice
// k costs 8 B per stored entry slot (its padded width x 32) plus 57 B per row
// (the row data of the apply), and warp w starts at the first slice whose
// prefix cost reaches w / nw of the total.
__global__ void k_wpart(const int64_t* __restrict__ off, int64_t nslices, int64_t nw, int32_t* __restrict__ wpart) {
  const double row_cost = 57.0 * kSlice;
  const double total = 8.0 * (double)off[nslices] + row_cost * (double)nslices;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w <= nw; w += (int64_t)gridDim.x * blockDim.x) {
    if (w == nw) {
      wpart[w] = (int32_t)nslices;
      continue;
    }
    const double target = total * (double)w / (double)nw;
    int64_t lo = 0, hi = nslices;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (8.0 * (double)off[mid] + row_cost * (double)mid < target) lo = mid + 1;
      else hi = mid;
    }
    wpart[w] = (int32_t)lo;
  }
}

}  // namespace

sph_status ensure_wpart(sph_neighbors* H, int grid, cudaStream_t st) {
  const int64_t nw = (int64_t)grid * (kBlock / 32);
  if (H->wpart_nw == nw && H->wpart_version == H->op_version) return SPH_OK;
  SPH_TRY(H->wpart.alloc(nw + 1));
  SPH_LAUNCH(k_wpart, grid_for(H, nw + 1), kBlock, 0, st)(H->op_off.p, H->nslices, nw, H->wpart.p);
  SPH_TRY_CUDA(cudaGetLastError());
  H->wpart_nw = nw;
  H->wpart_version = H->op_version;
  return SPH_OK;
}

sph_status ensure_operator(sph_neighbors* H, const sph_visc_params* P, cudaStream_t st) {
  if (!P || !(P->dt > 0.0) || !std::isfinite(P->dt) || (P->boundary != SPH_BC_DUMMY && P->boundary != SPH_BC_DYNAMIC) ||
      (P->mean != SPH_MEAN_HARMONIC && P->mean != SPH_MEAN_ARITHMETIC)) {
    set_error("viscous parameters: dt must be positive and finite, boundary/mean one of the enums");
    return SPH_ERR_INVALID;
  }
  if (H->op_valid && H->op_params.dt == P->dt && H->op_params.boundary == P->boundary &&
      H->op_params.mean == P->mean && H->op_mu_version == H->mu_version)
    return SPH_OK;
  OpGeom g{};
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = H->grid.L[ax];
    g.invL[ax] = 1.0 / H->grid.L[ax];
    g.periodic[ax] = H->grid.periodic[ax];
  }
  g.h = (double)H->h;
  g.inv_h = 1.0 / g.h;
  SPH_TRY(H->op_cnt.alloc(H->n_pad));
  SPH_TRY(H->op_kind.alloc(H->n_pad));
  SPH_TRY(H->op_off.alloc(H->nslices + 1));
  SPH_TRY(H->invD.alloc(H->n_pad));
  SPH_TRY(H->D64.alloc(H->n_pad));
  const int grid = grid_for(H, H->n_pad);
  SPH_LAUNCH(k_op_count, grid, kBlock, 0, st)(H->type_s.p, H->cnt.p, H->slice_off.p, H->nbr.p, H->n, H->n_pad,
                                              P->boundary, H->op_cnt.p, H->op_kind.p);
  SPH_TRY_CUDA(cudaGetLastError());
  int64_t total_pad = 0, total = 0;
  int32_t maxc = 0;
  SPH_TRY(build_slices(H, H->op_cnt.p, H->op_off.p, &total_pad, &total, &maxc, st));
  SPH_TRY(H->op_ih.alloc(total_pad > 0 ? total_pad : 1));
  SPH_TRY(H->op_lo.alloc(total_pad > 0 ? total_pad : 1));
  H->op_nnz_pad = total_pad;
  H->op_nnz = total;
  SPH_TRY(H->aux_df.alloc(H->n_pad));
  SPH_LAUNCH(k_op_aux, grid, kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->mu_s.p, H->n_pad, H->aux_df.p);
  const int gauss = H->kernel == SPH_KERNEL_GAUSSIAN ? 1 : 0;
  const double inv_h5 = g.inv_h * g.inv_h * g.inv_h * g.inv_h * g.inv_h;
  const double kf = 2.0 * P->dt * (gauss ? 2.0 / gauss_norm() : 105.0 / (128.0 * M_PI)) * inv_h5;
  SPH_LAUNCH(k_op_fill, grid, kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->mu_s.p, H->type_s.p, H->aux_df.p, H->cnt.p,
                                             H->slice_off.p, H->nbr.p, H->op_kind.p, H->op_off.p, H->n, H->n_pad, g,
                                             P->dt, P->mean, gauss, kf, std::exp(-kGaussK * kGaussK), H->op_ih.p,
                                             H->op_lo.p, H->invD.p, H->D64.p);
  SPH_TRY_CUDA(cudaGetLastError());
  H->op_valid = true;
  H->op_params = *P;
  H->op_mu_version = H->mu_version;
  ++H->op_version;
  return SPH_OK;
}

void launch_residual_f64(const sph_neighbors* H, int grid, const double* x, const double* b, double* r,
                         double* partials, unsigned int* counter, double* res_out, cudaStream_t st) {
  SPH_LAUNCH(k_split_x, grid_for(H, H->n_pad), kBlock, 0, st)(x, H->n_pad, H->v_x2.p);
  SPH_LAUNCH(k_residual_df, grid, kBlock, 0, st)(op_view(H), H->op_lo.p, H->v_x2.p, x, b, r, H->n,
                                                 partials, counter, res_out);
}

void launch_residual_update(const sph_neighbors* H, int grid, const float4* d, double* r, double* partials,
                            unsigned int* counter, double* res_out, cudaStream_t st) {
  SPH_LAUNCH(k_residual_update_df, grid, kBlock, 0, st)(op_view(H), H->op_lo.p, d, r, H->n, partials, counter,
                                                        res_out);
}

OpView op_view(const sph_neighbors* H) {
  const bool u = H->union_valid && H->union_op_version == H->op_version;
  const bool wp = H->wpart_version == H->op_version && H->wpart_nw > 0;
  return OpView{H->op_off.p, H->op_cnt.p, H->op_ih.p, H->op_kind.p, H->invD.p, H->nslices, H->n_pad,
                u ? H->op_loc.p : nullptr, u ? H->uni.p : nullptr, u ? H->unum.p : nullptr,
                wp ? H->wpart.p : nullptr, wp ? H->wpart_nw : 0};
}

void launch_apply_f32(const sph_neighbors* H, const float4* v, float4* y, bool jacobi, cudaStream_t st) {
  const int grid = grid_for(H, H->nslices * 32);
  const OpView op = op_view(H);
  auto kern = jacobi ? k_apply_f32<true> : k_apply_f32<false>;
  SPH_LAUNCH(kern, grid, kBlock, 0, st)(op, v, y);
}

sph_status visc_apply(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y, cudaStream_t st) {
  if (!H || !v || !y) {
    set_error("sph_visc_apply: null argument");
    return SPH_ERR_INVALID;
  }
  SPH_TRY(ensure_operator(H, P, st));
  SPH_TRY(H->v_tmp.alloc(2 * H->n_pad));
  float4* vs = H->v_tmp.p;
  float4* ys = H->v_tmp.p + H->n_pad;
  const int grid = grid_for(H, H->n_pad);
  SPH_LAUNCH(k_gather_f4, grid, kBlock, 0, st)(v, H->perm.p, H->n, H->n_pad, vs);
  SPH_TRY_CUDA(cudaGetLastError());
  standalone_begin(H, st);
  launch_apply_f32(H, vs, ys, false, st);
  SPH_TRY(standalone_end(H, st, 0));
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_scatter_f4, grid, kBlock, 0, st)(ys, H->perm.p, H->n, y);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
