// The operator apply with the coefficients recomputed on the fly (the form of
// the paper's own GPU code, App. A and App. B), next to the stored-coefficient
// form of apply.cuh, so the two can be measured against each other.
//
// Per pair it reads the neighbour index (4 B, the neighbour list's SELL-32
// layout) instead of the stored (index, coefficient) pair (8 B), and gathers the
// neighbour's packed geometry (x, y, z, +-V with V = m / rho, negative for wall
// particles) and 1/mu (mu for the arithmetic mean) besides its velocity.  It then
// forms, in float32,
//   fluid row b:  a = dt c_ab = R_b V_a mubar (2 - q)^3, R_b = 2 dt (105 / (128 pi)) / (h^5 rho_b)
//                 (Eq. kab with Sec. 5.2's F taken as |F|, the reading used throughout)
//                 y_b = v_b + sum a (v_b - v_a)   [ / (1 + sum a) with Jacobi ]
//   dummy wall:   y_b = v_b + sum_fluid W_ab v_a / sum_fluid W_ab   (Eq. dummyvel)
//   identity:     y_b = v_b
// Row kinds come from the stored operator's count pass (op_kind), so a dummy
// wall row with an empty Shepard sum is an identity row here too.
#include <cmath>

#include "apply.cuh"
#include "sph_internal.cuh"

namespace sph {

struct OtfView {
  const int64_t* off;   // neighbour-list slice offsets [nslices + 1]
  const int32_t* cnt;   // neighbour count per sorted row
  const int32_t* nbr;   // neighbour rows (SELL-32)
  const float4* g;      // (x, y, z, +-V)
  const float* im;      // 1/mu (harmonic mean) or mu (arithmetic mean)
  const float* rb;      // R_b per row
  const uint8_t* kind;  // KIND_FLUID / KIND_SHEPARD / KIND_IDENTITY
  int64_t nslices;
  float L[3], invL[3];
  int periodic[3];
  float inv_h;
};

namespace {

constexpr int kOtfU = 4;  // neighbours in flight per thread

template <bool JACOBI, bool HARMONIC>
__device__ __forceinline__ float4 apply_row_otf(const OtfView& o, const float4* __restrict__ v, int64_t sl,
                                                int lane) {
  const int64_t s = sl * kSlice + lane;
  const uint8_t kd = o.kind[s];
  const float4 vb = v[s];
  const int c = o.cnt[s];
  // longest list of the slice (the list layout may be wider than that); taken
  // before any lane leaves, every lane of the warp is here
  const int w = __reduce_max_sync(0xffffffffu, kd == KIND_IDENTITY ? 0 : c);
  if (kd == KIND_IDENTITY) return make_float4(vb.x, vb.y, vb.z, 0.f);
  const bool fluid = kd == KIND_FLUID;
  const float4 gb = o.g[s];
  const float imb = o.im[s];
  const float Rb = o.rb[s];
  const float mub_wall = HARMONIC ? 1.f / imb : imb;   // fluid-wall pairs: the row's own mu
  const int64_t o0 = o.off[sl];
  const int32_t* __restrict__ p = o.nbr + o0 + lane;
  float ax = 0.f, ay = 0.f, az = 0.f, sa = 0.f;
  for (int j0 = 0; j0 < w; j0 += kOtfU) {
    int32_t t[kOtfU];
#pragma unroll
    for (int u = 0; u < kOtfU; ++u) t[u] = (j0 + u < c) ? __ldcs(p + (int64_t)(j0 + u) * kSlice) : -1;
    float4 ga[kOtfU], va[kOtfU];
    float ia[kOtfU];
#pragma unroll
    for (int u = 0; u < kOtfU; ++u) {
      const int32_t tt = t[u] >= 0 ? t[u] : (int32_t)s;
      ga[u] = __ldg(o.g + tt);
      va[u] = __ldg(v + tt);
      ia[u] = __ldg(o.im + tt);
    }
#pragma unroll
    for (int u = 0; u < kOtfU; ++u) {
      float d[3] = {ga[u].x - gb.x, ga[u].y - gb.y, ga[u].z - gb.z};
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (o.periodic[k]) d[k] = fmaf(-o.L[k], rintf(d[k] * o.invL[k]), d[k]);
      const float q = sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]))) * o.inv_h;
      const bool valid = t[u] >= 0;
      const bool nfluid = ga[u].w > 0.f;
      if (fluid) {
        const float tq = fmaxf(2.f - q, 0.f);
        const float mub = nfluid ? (HARMONIC ? __fdividef(2.f, ia[u] + imb) : 0.5f * (ia[u] + imb)) : mub_wall;
        const float a = valid ? Rb * fabsf(ga[u].w) * mub * (tq * tq * tq) : 0.f;
        ax = fmaf(a, vb.x - va[u].x, ax);
        ay = fmaf(a, vb.y - va[u].y, ay);
        az = fmaf(a, vb.z - va[u].z, az);
        sa += a;
      } else {
        // Wendland psi_{3,1} up to its constant factor, which cancels in W / S
        const float tw = fmaxf(1.f - 0.5f * q, 0.f);
        const float tw2 = tw * tw;
        const float W = (valid && nfluid) ? tw2 * tw2 * fmaf(2.f, q, 1.f) : 0.f;
        ax = fmaf(W, va[u].x, ax);
        ay = fmaf(W, va[u].y, ay);
        az = fmaf(W, va[u].z, az);
        sa += W;
      }
    }
  }
  if (fluid) {
    const float sc = JACOBI ? 1.f / (1.f + sa) : 1.f;
    return make_float4((vb.x + ax) * sc, (vb.y + ay) * sc, (vb.z + az) * sc, 0.f);
  }
  // KIND_SHEPARD rows have a positive float64 Shepard sum; in float32 a lone
  // neighbour at q just below 2 can still round to W = 0
  const float iS = sa > 0.f ? 1.f / sa : 0.f;
  return make_float4(fmaf(ax, iS, vb.x), fmaf(ay, iS, vb.y), fmaf(az, iS, vb.z), 0.f);
}

template <bool JACOBI, bool HARMONIC>
__global__ void __launch_bounds__(kBlock) k_apply_otf(OtfView o, const float4* __restrict__ v,
                                                      float4* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < o.nslices; sl += nwarps)
    y[sl * kSlice + lane] = apply_row_otf<JACOBI, HARMONIC>(o, v, sl, lane);
}

__global__ void k_otf_pack(const float4* __restrict__ pos, const float* __restrict__ rho,
                           const float* __restrict__ mu, const uint8_t* __restrict__ type, int64_t n, int64_t n_pad,
                           int harmonic, double kf, float4* __restrict__ g, float* __restrict__ im,
                           float* __restrict__ rb) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      const float4 p = pos[s];
      const float V = p.w / rho[s];
      g[s] = make_float4(p.x, p.y, p.z, type[s] == SPH_FLUID ? V : -V);
      im[s] = harmonic ? 1.f / mu[s] : mu[s];
      rb[s] = (float)(kf / (double)rho[s]);
    } else {
      g[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      im[s] = 1.f;
      rb[s] = 0.f;
    }
  }
}

__global__ void k_gather_f4_otf(const float* __restrict__ v_caller, const int32_t* __restrict__ perm, int64_t n,
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

__global__ void k_scatter_f4_otf(const float4* __restrict__ y_s, const int32_t* __restrict__ perm, int64_t n,
                                 float* __restrict__ y_caller) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<float4*>(y_caller)[perm[s]] = y_s[s];
}

}  // namespace

// Packed geometry of the on-the-fly form for the operator parameters P (rebuilt
// with the stored operator: same dt, boundary, mean and viscosities).
static sph_status ensure_otf(sph_neighbors* H, const sph_visc_params* P, cudaStream_t st) {
  SPH_TRY(ensure_operator(H, P, st));
  if (H->otf_valid && H->otf_op_version == H->op_version) return SPH_OK;
  SPH_TRY(H->otf_g.alloc(H->n_pad));
  SPH_TRY(H->otf_im.alloc(H->n_pad));
  SPH_TRY(H->otf_rb.alloc(H->n_pad));
  const double h = (double)H->h;
  const double kf = 2.0 * P->dt * (105.0 / (128.0 * M_PI)) / (h * h * h * h * h);
  SPH_LAUNCH(k_otf_pack, grid_for(H, H->n_pad), kBlock, 0, st)(H->pos_s.p, H->rho_s.p, H->mu_s.p, H->type_s.p, H->n,
                                                               H->n_pad, P->mean == SPH_MEAN_HARMONIC ? 1 : 0, kf,
                                                               H->otf_g.p, H->otf_im.p, H->otf_rb.p);
  SPH_TRY_CUDA(cudaGetLastError());
  H->otf_valid = true;
  H->otf_op_version = H->op_version;
  return SPH_OK;
}

static OtfView otf_view(const sph_neighbors* H) {
  OtfView o{};
  o.off = H->slice_off.p;
  o.cnt = H->cnt.p;
  o.nbr = H->nbr.p;
  o.g = H->otf_g.p;
  o.im = H->otf_im.p;
  o.rb = H->otf_rb.p;
  o.kind = H->op_kind.p;
  o.nslices = H->nslices;
  for (int k = 0; k < 3; ++k) {
    o.L[k] = (float)H->grid.L[k];
    o.invL[k] = (float)(1.0 / H->grid.L[k]);
    o.periodic[k] = H->grid.periodic[k];
  }
  o.inv_h = (float)(1.0 / (double)H->h);
  return o;
}

void launch_apply_otf(const sph_neighbors* H, const float4* v, float4* y, bool jacobi, cudaStream_t st) {
  const int grid = grid_for(H, H->nslices * 32);
  const OtfView o = otf_view(H);
  const bool harm = H->op_params.mean == SPH_MEAN_HARMONIC;
  auto kern = jacobi ? (harm ? k_apply_otf<true, true> : k_apply_otf<true, false>)
                     : (harm ? k_apply_otf<false, true> : k_apply_otf<false, false>);
  SPH_LAUNCH(kern, grid, kBlock, 0, st)(o, v, y);
}

sph_status visc_apply_otf(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y, cudaStream_t st) {
  if (!H || !v || !y) {
    set_error("sph_visc_apply_otf: null argument");
    return SPH_ERR_INVALID;
  }
  if (H->kernel != SPH_KERNEL_WENDLAND) {
    set_error("sph_visc_apply_otf: the on-the-fly coefficients are written for the Wendland kernel");
    return SPH_ERR_INVALID;
  }
  SPH_TRY(ensure_otf(H, P, st));
  SPH_TRY(H->v_tmp.alloc(2 * H->n_pad));
  float4* vs = H->v_tmp.p;
  float4* ys = H->v_tmp.p + H->n_pad;
  const int grid = grid_for(H, H->n_pad);
  SPH_LAUNCH(k_gather_f4_otf, grid, kBlock, 0, st)(v, H->perm.p, H->n, H->n_pad, vs);
  standalone_begin(H, st);
  launch_apply_otf(H, vs, ys, false, st);
  SPH_TRY(standalone_end(H, st, 1));
  SPH_LAUNCH(k_scatter_f4_otf, grid, kBlock, 0, st)(ys, H->perm.p, H->n, y);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
