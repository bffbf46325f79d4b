// Cell binning, counting sort and neighbour lists (paper Sec. 5.2: a Wendland
// particle at h = 1.3 dp has about 80 neighbours; App. A: the relative position
// is one difference so r_ab = -r_ba bit for bit).
//
// Steps (one launch each):
//   keys      cell of every particle: floor((x - lo) / cell) per axis in float64,
//             wrapped on periodic axes, clamped on open ones; per-cell counts.
//             Cells are ordered along a Morton (Z-order) curve: segment r of the
//             sorted order holds the cell of rank r, so 32-row slices and the
//             slices a block works on are compact in space and their neighbour
//             gathers share cache lines (the apply is bound by those gathers)
//   scan      exclusive prefix sum of the counts -> cell_start
//   scatter   particles into their cell's segment (atomics: any order)
//   order     each segment sorted by caller index (makes the layout deterministic)
//   gather    sorted copies of pos / rho / mu / type, perm and iperm
//   count     neighbours per particle over the 27 surrounding cells
//   slices    SELL-32 slice widths and offsets
//   fill      the lists, in the same deterministic order as count
//
// The predicate is decided exactly as the float64 definition: a float32 test
// decides every pair outside a band around (R h)^2 (R h: the kernel support radius) whose half-width bounds the
// float32 rounding of r^2; pairs inside the band are recomputed in float64 with
// the same operations, in the same order and without contraction.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sph_internal.cuh"

namespace sph {

namespace {

enum : int32_t { FLAG_NONFINITE = 1, FLAG_CAPACITY = 2, FLAG_CELLFULL = 4 };

__global__ void k_cell_keys(const float4* __restrict__ pos, int64_t n, Grid g, const int32_t* __restrict__ rank,
                            int32_t* __restrict__ key, int32_t* __restrict__ cell_count, int32_t* __restrict__ flags,
                            unsigned int* __restrict__ max_abs_bits) {
  float local_max = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float4 p = pos[i];
    float c3[3] = {p.x, p.y, p.z};
    bool finite = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w);
    if (!finite) atomicOr(&flags[0], FLAG_NONFINITE);
    int c[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      double u = finite ? ((double)c3[ax] - g.lo[ax]) / g.cell[ax] : 0.0;
      u = fmin(fmax(u, -1.0e9), 1.0e9);
      long long k = (long long)floor(u);
      int nc = g.ncell[ax];
      if (g.periodic[ax]) {
        k %= nc;
        if (k < 0) k += nc;
      } else {
        k = k < 0 ? 0 : (k >= nc ? nc - 1 : k);
      }
      c[ax] = (int)k;
      if (finite) local_max = fmaxf(local_max, fabsf(c3[ax]));
    }
    int32_t kk = c[0] + g.ncell[0] * (c[1] + g.ncell[1] * c[2]);
    key[i] = kk;
    atomicAdd(&cell_count[rank[kk]], 1);
  }
  // warp max then one atomic per warp (non-negative floats order like their bits)
  for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_abs_bits, __float_as_uint(local_max));
}

// Single-block exclusive scan of m int32 values, each multiplied by `mul`;
// out has m + 1 entries (out[m] = total).  Also reports the largest input.
template <class TOut>
__global__ void k_scan(const int32_t* __restrict__ in, TOut* __restrict__ out, int64_t m, int64_t mul,
                       int32_t* __restrict__ max_out) {
  __shared__ long long s[1024];
  __shared__ int smax[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (m + 1023) / 1024;
  const int64_t b = (int64_t)t * chunk;
  const int64_t e = b + chunk < m ? b + chunk : m;
  long long sum = 0;
  int mx = 0;
  for (int64_t i = b; i < e; ++i) {
    int v = in[i];
    sum += (long long)v * mul;
    mx = v > mx ? v : mx;
  }
  s[t] = sum;
  smax[t] = mx;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long v = t >= off ? s[t - off] : 0;
    int w = t >= off ? smax[t - off] : 0;
    __syncthreads();
    s[t] += v;
    smax[t] = smax[t] > w ? smax[t] : w;
    __syncthreads();
  }
  long long run = s[t] - sum;
  for (int64_t i = b; i < e; ++i) {
    out[i] = (TOut)run;
    run += (long long)in[i] * mul;
  }
  if (t == 1023) {
    out[m] = (TOut)s[1023];
    if (max_out) *max_out = smax[1023];
  }
}

__global__ void k_cell_scatter(const int32_t* __restrict__ key, const int32_t* __restrict__ rank, int64_t n,
                               const int32_t* __restrict__ cell_start, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = rank[key[i]];
    int32_t slot = cell_start[k] + atomicAdd(&cursor[k], 1);
    out[slot] = (int32_t)i;
  }
}

// Orders each cell's segment by caller index (insertion sort, one thread per
// cell; segments hold ~20 particles at the densities of SPH).
__global__ void k_cell_order(const int32_t* __restrict__ cell_start, int64_t ncells, int32_t* __restrict__ ids) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
    int32_t b = cell_start[c], e = cell_start[c + 1];
    for (int32_t i = b + 1; i < e; ++i) {
      int32_t v = ids[i];
      int32_t j = i - 1;
      while (j >= b && ids[j] > v) {
        ids[j + 1] = ids[j];
        --j;
      }
      ids[j + 1] = v;
    }
  }
}

__global__ void k_gather_sorted(const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                                const float4* __restrict__ pos, const float* __restrict__ rho,
                                const float* __restrict__ mu, const uint8_t* __restrict__ ptype,
                                const int32_t* __restrict__ key, int32_t* __restrict__ iperm,
                                float4* __restrict__ pos_s, float* __restrict__ rho_s, float* __restrict__ mu_s,
                                uint8_t* __restrict__ type_s, int32_t* __restrict__ key_s,
                                int32_t* __restrict__ flags) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      int32_t i = perm[s];
      iperm[i] = (int32_t)s;
      pos_s[s] = pos[i];
      float r = rho[i], m = mu[i];
      if (!(isfinite(r) && r > 0.f && isfinite(m) && m > 0.f)) atomicOr(&flags[0], FLAG_NONFINITE);
      rho_s[s] = r;
      mu_s[s] = m;
      uint8_t t = ptype[i];
      type_s[s] = t > 1 ? 1 : t;
      key_s[s] = key[i];
    } else {
      pos_s[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      rho_s[s] = 1.f;
      mu_s[s] = 1.f;
      type_s[s] = 1;
      key_s[s] = 0;
    }
  }
}

// float64 form of the neighbour predicate, operation for operation.
__device__ __forceinline__ bool pair_inside_f64(float4 pt, float4 ps, const Grid& g, double R2) {
  double d[3] = {__dsub_rn((double)pt.x, (double)ps.x), __dsub_rn((double)pt.y, (double)ps.y),
                 __dsub_rn((double)pt.z, (double)ps.z)};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (g.periodic[ax]) {
      double L = g.L[ax];
      double k = rint(__ddiv_rn(d[ax], L));
      d[ax] = __dsub_rn(d[ax], __dmul_rn(L, k));
    }
  }
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < R2;
}

struct Band {
  float lo2, hi2;   // float32 r^2 below lo2: inside; at or above hi2: outside
  double R2;        // (R h)^2 in float64, R h the support radius
  float L[3], invL[3];
};

// One pass over the 27 cells around each particle: the count and the list at
// once.  Lists live in a fixed-capacity SELL-32 layout (every slice maxnb
// entries wide, entry j of row s at (s / 32) 32 maxnb + 32 j + s % 32), so no
// counting pass has to size them first; a row with more than maxnb neighbours
// raises FLAG_CAPACITY and keeps its first maxnb.
__global__ void __launch_bounds__(kBlock) k_neighbors(const float4* __restrict__ pos_s, const int32_t* __restrict__ key_s,
                                                      const int32_t* __restrict__ rank,
                                                      const int32_t* __restrict__ cell_start, int64_t n, int64_t n_pad,
                                                      Grid g, Band band, int32_t maxnb, int32_t* __restrict__ cnt,
                                                      int32_t* __restrict__ nbr, int32_t* __restrict__ flags) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s >= n) {
      cnt[s] = 0;
      continue;
    }
    const float4 ps = pos_s[s];
    const int32_t key = key_s[s];
    const int nx = g.ncell[0], ny = g.ncell[1], nz = g.ncell[2];
    const int cx = key % nx, cy = (key / nx) % ny, cz = key / (nx * ny);
    int32_t count = 0;
    const int64_t base = (s / kSlice) * (int64_t)kSlice * maxnb + (s % kSlice);
    for (int dz = -1; dz <= 1; ++dz) {
      int z = cz + dz;
      if (g.periodic[2]) z = (z + nz) % nz;
      else if (z < 0 || z >= nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int y = cy + dy;
        if (g.periodic[1]) y = (y + ny) % ny;
        else if (y < 0 || y >= ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          int x = cx + dx;
          if (g.periodic[0]) x = (x + nx) % nx;
          else if (x < 0 || x >= nx) continue;
          const int32_t cell = rank[x + nx * (y + ny * z)];
          const int32_t tb = cell_start[cell], te = cell_start[cell + 1];
          for (int32_t t = tb; t < te; ++t) {
            if (t == s) continue;
            const float4 pt = pos_s[t];
            float d0 = pt.x - ps.x, d1 = pt.y - ps.y, d2 = pt.z - ps.z;
            if (g.periodic[0]) d0 -= band.L[0] * rintf(d0 * band.invL[0]);
            if (g.periodic[1]) d1 -= band.L[1] * rintf(d1 * band.invL[1]);
            if (g.periodic[2]) d2 -= band.L[2] * rintf(d2 * band.invL[2]);
            const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
            bool in;
            if (r2 < band.lo2) in = true;
            else if (r2 >= band.hi2) in = false;
            else in = pair_inside_f64(pt, ps, g, band.R2);
            if (in) {
              if (count < maxnb) nbr[base + (int64_t)count * kSlice] = t;
              ++count;
            }
          }
        }
      }
    }
    if (count > maxnb) {
      atomicOr(&flags[0], FLAG_CAPACITY);
      count = maxnb;
    }
    cnt[s] = count;
  }
}

// slice offsets of the fixed-capacity list layout
__global__ void k_fixed_offsets(int64_t nslices, int64_t width, int64_t* __restrict__ off) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nslices; k += (int64_t)gridDim.x * blockDim.x)
    off[k] = k * kSlice * width;
}

// slice widths (max count over the 32 rows), total entries and the largest row
__global__ void k_slice_width(const int32_t* __restrict__ cnt, int64_t nslices, int32_t* __restrict__ width,
                              unsigned long long* __restrict__ total, int32_t* __restrict__ maxc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < nslices; k += nwarps) {
    int c = cnt[k * kSlice + lane];
    int m = c;
    unsigned long long sum = (unsigned long long)c;
    for (int o = 16; o > 0; o >>= 1) {
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
      width[k] = m;
      atomicAdd(total, sum);
      atomicMax(maxc, m);
    }
  }
}

// caller-order CSR export: row lengths, then entries mapped through perm and sorted
__global__ void k_export_counts(const int32_t* __restrict__ iperm, const int32_t* __restrict__ cnt, int64_t n,
                                int32_t* __restrict__ rowlen) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rowlen[i] = cnt[iperm[i]];
}

__global__ void k_export_fill(const int32_t* __restrict__ iperm, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ cnt, const int64_t* __restrict__ slice_off,
                              const int32_t* __restrict__ nbr, int64_t n, const int64_t* __restrict__ offsets,
                              int32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = iperm[i];
    const int32_t c = cnt[s];
    const int64_t base = slice_off[s / kSlice] + (s % kSlice);
    int32_t* row = idx + offsets[i];
    for (int32_t j = 0; j < c; ++j) {
      int32_t v = perm[nbr[base + (int64_t)j * kSlice]];
      int32_t k = j - 1;
      while (k >= 0 && row[k] > v) {
        row[k + 1] = row[k];
        --k;
      }
      row[k + 1] = v;
    }
  }
}

}  // namespace

// rank[row-major cell] = position of the cell along the Morton curve that
// interleaves the bits of its (x, y, z) cell coordinates (ties impossible); grids
// of more than 2^24 cells keep the row-major order (the host table and its sort
// would cost more than the locality gains)
static void morton_ranks(const int nc[3], std::vector<int32_t>& rank) {
  auto spread = [](uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
  };
  const int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
  rank.assign((size_t)ncells, 0);
  if (ncells > ((int64_t)1 << 24)) {
    for (int64_t c = 0; c < ncells; ++c) rank[(size_t)c] = (int32_t)c;
    return;
  }
  std::vector<std::pair<uint64_t, int32_t>> code((size_t)ncells);
  for (int z = 0; z < nc[2]; ++z)
    for (int y = 0; y < nc[1]; ++y)
      for (int x = 0; x < nc[0]; ++x) {
        const int64_t c = x + (int64_t)nc[0] * (y + (int64_t)nc[1] * z);
        code[(size_t)c] = {spread((uint64_t)x) | (spread((uint64_t)y) << 1) | (spread((uint64_t)z) << 2), (int32_t)c};
      }
  std::sort(code.begin(), code.end());
  for (int64_t r = 0; r < ncells; ++r) rank[(size_t)code[(size_t)r].second] = (int32_t)r;
}

int grid_for(const sph_neighbors* H, int64_t work_items, int block) {
  int64_t want = (work_items + block - 1) / block;
  int64_t cap = (int64_t)(H->num_sms > 0 ? H->num_sms : 148) * 16;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

sph_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t m, cudaStream_t st) {
  SPH_LAUNCH(k_scan<int64_t>, 1, 1024, 0, st)(in, out, m, 1, nullptr);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

sph_status slice_offsets(const int32_t* cnt, int64_t nslices, int64_t* off, int32_t* width_tmp, cudaStream_t st) {
  (void)cnt;
  SPH_LAUNCH(k_scan<int64_t>, 1, 1024, 0, st)(width_tmp, off, nslices, kSlice, nullptr);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

// Builds slice widths + offsets for a per-row count array; returns the padded
// entry total, the true entry total and the largest row (synchronises).
sph_status build_slices(sph_neighbors* H, const int32_t* cnt, int64_t* off, int64_t* total_pad,
                        int64_t* total, int32_t* maxc, cudaStream_t st) {
  SPH_TRY(H->tmp_i32b.alloc(H->nslices + 1));
  SPH_TRY(H->tmp_i64.alloc(4));
  SPH_TRY_CUDA(cudaMemsetAsync(H->tmp_i64.p, 0, 4 * sizeof(int64_t), st));
  int grid = grid_for(H, H->nslices * 32);
  SPH_LAUNCH(k_slice_width, grid, kBlock, 0, st)(cnt, H->nslices, H->tmp_i32b.p,
                                         reinterpret_cast<unsigned long long*>(H->tmp_i64.p),
                                         reinterpret_cast<int32_t*>(H->tmp_i64.p + 1));
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_scan<int64_t>, 1, 1024, 0, st)(H->tmp_i32b.p, off, H->nslices, kSlice, nullptr);
  SPH_TRY_CUDA(cudaGetLastError());
  int64_t host[2];
  SPH_TRY_CUDA(cudaMemcpyAsync(host, H->tmp_i64.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaMemcpyAsync(total_pad, off + H->nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  *total = host[0];
  *maxc = (int32_t)(host[1] & 0xffffffff);
  return SPH_OK;
}

sph_status build_neighbors(const sph_scene* sc, int32_t maxnb, sph_neighbors** out, cudaStream_t st) {
  if (!sc || !out) {
    set_error("sph_build_neighbors: null scene or handle pointer");
    return SPH_ERR_INVALID;
  }
  if (sc->n < 1 || sc->n > (int64_t)INT32_MAX - 64 || !sc->pos || !sc->rho || !sc->mu || !sc->ptype) {
    set_error("sph_build_neighbors: n must be in [1, 2^31-64] and every array non-null");
    return SPH_ERR_INVALID;
  }
  if (!(sc->h > 0.f) || !std::isfinite(sc->h)) {
    set_error("sph_build_neighbors: h must be positive and finite");
    return SPH_ERR_INVALID;
  }
  if (maxnb < 1 || maxnb > 1024) {
    set_error("sph_build_neighbors: max_neighbors must be in [1, 1024]");
    return SPH_ERR_INVALID;
  }
  if (sc->kernel != SPH_KERNEL_WENDLAND && sc->kernel != SPH_KERNEL_GAUSSIAN) {
    set_error("sph_build_neighbors: unknown kernel %d", sc->kernel);
    return SPH_ERR_INVALID;
  }
  Grid g{};
  // the support radius: 2h (Wendland) or 3h (truncated Gaussian)
  const double rsup = (sc->kernel == SPH_KERNEL_GAUSSIAN ? 3.0 : 2.0) * (double)sc->h;
  int64_t ncells = 1;
  for (int ax = 0; ax < 3; ++ax) {
    double L = sc->hi[ax] - sc->lo[ax];
    if (!(L > 0.0) || !std::isfinite(L)) {
      set_error("sph_build_neighbors: hi[%d] must exceed lo[%d]", ax, ax);
      return SPH_ERR_INVALID;
    }
    // cells strictly larger than the support radius (with a relative margin for rounding)
    double nc = std::floor(L / (rsup * (1.0 + 1e-6)));
    if (nc < 1.0) nc = 1.0;
    if (nc > 1.0e6) nc = 1.0e6;
    g.periodic[ax] = sc->periodic[ax] ? 1 : 0;
    if (g.periodic[ax] && nc < 3.0) {
      set_error("sph_build_neighbors: periodic axis %d is shorter than three cells of the support radius "
                "(L = %g, radius = %g)", ax, L, rsup);
      return SPH_ERR_INVALID;
    }
    g.ncell[ax] = (int)nc;
    g.cell[ax] = L / nc;
    g.lo[ax] = sc->lo[ax];
    g.L[ax] = L;
    ncells *= (int64_t)nc;
  }
  if (ncells > (int64_t)1 << 30) {
    set_error("sph_build_neighbors: %lld cells exceed the 2^30 limit (box too large for h)", (long long)ncells);
    return SPH_ERR_INVALID;
  }
  g.ncells = ncells;

  bool fresh = (*out == nullptr);
  sph_neighbors* H = fresh ? new sph_neighbors() : *out;
  auto fail = [&](sph_status s) {
    if (fresh) {
      sph_neighbors_destroy(H);
      *out = nullptr;
    }
    return s;
  };
#define TRYF(expr)                      \
  do {                                  \
    sph_status s__ = (expr);            \
    if (s__ != SPH_OK) return fail(s__); \
  } while (0)
#define TRYF_CUDA(call)                                                                         \
  do {                                                                                          \
    cudaError_t e__ = (call);                                                                   \
    if (e__ != cudaSuccess) {                                                                   \
      set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__));           \
      return fail(SPH_ERR_CUDA);                                                                \
    }                                                                                           \
  } while (0)

  TRYF_CUDA(cudaGetDevice(&H->device));
  TRYF_CUDA(cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, H->device));
  const int64_t n = sc->n;
  if (H->row_scaled && H->n != n) {   // a caller-order row scale no longer fits
    H->row_scaled = false;
    ++H->rs_version;
  }
  H->n = n;
  H->n_pad = (n + kSlice - 1) / kSlice * kSlice;
  H->nslices = H->n_pad / kSlice;
  H->grid = g;
  H->h = sc->h;
  H->kernel = sc->kernel;
  H->op_valid = false;
  H->mu_version++;

  TRYF(H->pos_s.alloc(H->n_pad));
  TRYF(H->rho_s.alloc(H->n_pad));
  TRYF(H->mu_s.alloc(H->n_pad));
  TRYF(H->type_s.alloc(H->n_pad));
  TRYF(H->perm.alloc(n));
  TRYF(H->iperm.alloc(n));
  TRYF(H->key_s.alloc(H->n_pad));
  TRYF(H->cell_start.alloc(ncells + 1));
  TRYF(H->cnt.alloc(H->n_pad));
  TRYF(H->slice_off.alloc(H->nslices + 1));
  TRYF(H->tmp_i32a.alloc(n > ncells ? n : ncells));           // keys, then cursors
  TRYF(H->tmp_i64.alloc(ncells + 1 > 4 ? ncells + 1 : 4));
  TRYF(H->flags.alloc(8));
  TRYF(H->tmp_i32b.alloc(ncells));
  TRYF_CUDA(cudaMemsetAsync(H->flags.p, 0, 8 * sizeof(int32_t), st));
  TRYF_CUDA(cudaMemsetAsync(H->tmp_i32b.p, 0, ncells * sizeof(int32_t), st));

  const float4* pos = reinterpret_cast<const float4*>(sc->pos);
  int32_t* key = H->tmp_i32a.p;
  int grid_n = grid_for(H, n);
  if (H->rank_dims[0] != g.ncell[0] || H->rank_dims[1] != g.ncell[1] || H->rank_dims[2] != g.ncell[2]) {
    TRYF(H->cell_rank.alloc(ncells));
    std::vector<int32_t> rank;
    morton_ranks(g.ncell, rank);
    TRYF_CUDA(cudaMemcpy(H->cell_rank.p, rank.data(), ncells * sizeof(int32_t), cudaMemcpyHostToDevice));
    for (int ax = 0; ax < 3; ++ax) H->rank_dims[ax] = g.ncell[ax];
  }
  SPH_LAUNCH(k_cell_keys, grid_n, kBlock, 0, st)(pos, n, g, H->cell_rank.p, key, H->tmp_i32b.p, H->flags.p,
                                         reinterpret_cast<unsigned int*>(H->flags.p + 1));
  TRYF_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_scan<int32_t>, 1, 1024, 0, st)(H->tmp_i32b.p, H->cell_start.p, ncells, 1, H->flags.p + 2);
  TRYF_CUDA(cudaGetLastError());
  int32_t hflags[8];
  TRYF_CUDA(cudaMemcpyAsync(hflags, H->flags.p, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRYF_CUDA(cudaStreamSynchronize(st));
  if (hflags[0] & FLAG_NONFINITE) {
    set_error("sph_build_neighbors: non-finite particle position or mass");
    return fail(SPH_ERR_NONFINITE);
  }
  const int32_t max_cell = hflags[2];
  if ((int64_t)max_cell > 64LL * (maxnb + 1)) {
    set_error("sph_build_neighbors: a cell holds %d particles, more than any %d-neighbour particle set allows",
              max_cell, maxnb);
    return fail(SPH_ERR_CAPACITY);
  }
  float max_abs;
  std::memcpy(&max_abs, &hflags[1], sizeof(float));

  // scatter into segments (cursor counts reuse tmp_i32b), order, gather
  TRYF_CUDA(cudaMemsetAsync(H->tmp_i32b.p, 0, ncells * sizeof(int32_t), st));
  SPH_LAUNCH(k_cell_scatter, grid_n, kBlock, 0, st)(key, H->cell_rank.p, n, H->cell_start.p, H->tmp_i32b.p,
                                                    H->perm.p);
  TRYF_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_cell_order, grid_for(H, ncells), kBlock, 0, st)(H->cell_start.p, ncells, H->perm.p);
  TRYF_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_gather_sorted, grid_for(H, H->n_pad), kBlock, 0, st)(
      H->perm.p, n, H->n_pad, pos, sc->rho, sc->mu, sc->ptype, key, H->iperm.p, H->pos_s.p, H->rho_s.p, H->mu_s.p,
      H->type_s.p, H->key_s.p, H->flags.p);
  TRYF_CUDA(cudaGetLastError());

  // band of the float32 filter: coordinate differences carry at most a few
  // float32 roundings of the largest coordinate or period E; r^2 then errs by
  // at most 2 sqrt(3) (R h) E + 3 E^2 plus its own three roundings
  double big = (double)max_abs;
  for (int ax = 0; ax < 3; ++ax) {
    big = std::fmax(big, std::fabs(sc->lo[ax]));
    big = std::fmax(big, std::fabs(sc->hi[ax]));
    big = std::fmax(big, g.L[ax]);
  }
  const double E = 4.0 * big * std::ldexp(1.0, -23);
  Band band{};
  band.R2 = rsup * rsup;
  const double B = 4.0 * rsup * E + 3.0 * E * E + 1e-6 * band.R2;
  band.lo2 = (float)std::fmax(0.0, (band.R2 - B) * (1.0 - 1e-7));
  band.hi2 = (float)((band.R2 + B) * (1.0 + 1e-7));
  for (int ax = 0; ax < 3; ++ax) {
    band.L[ax] = (float)g.L[ax];
    band.invL[ax] = (float)(1.0 / g.L[ax]);
  }

  int grid_p = grid_for(H, H->n_pad);
  TRYF(H->nbr.alloc(H->n_pad * (int64_t)maxnb));
  SPH_LAUNCH(k_neighbors, grid_p, kBlock, 0, st)(H->pos_s.p, H->key_s.p, H->cell_rank.p, H->cell_start.p, n, H->n_pad, g,
                                                 band, maxnb, H->cnt.p, H->nbr.p, H->flags.p);
  TRYF_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_fixed_offsets, grid_for(H, H->nslices + 1), kBlock, 0, st)(H->nslices, maxnb, H->slice_off.p);
  TRYF_CUDA(cudaGetLastError());
  // entry total and the longest row (k_slice_width's widths land in scratch)
  TRYF(H->tmp_i32b.alloc(H->nslices + 1 > ncells ? H->nslices + 1 : ncells));
  TRYF_CUDA(cudaMemsetAsync(H->tmp_i64.p, 0, 2 * sizeof(int64_t), st));
  SPH_LAUNCH(k_slice_width, grid_for(H, H->nslices * 32), kBlock, 0, st)(
      H->cnt.p, H->nslices, H->tmp_i32b.p, reinterpret_cast<unsigned long long*>(H->tmp_i64.p),
      reinterpret_cast<int32_t*>(H->tmp_i64.p + 1));
  TRYF_CUDA(cudaGetLastError());
  int64_t tot[2];
  TRYF_CUDA(cudaMemcpyAsync(hflags, H->flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRYF_CUDA(cudaMemcpyAsync(tot, H->tmp_i64.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TRYF_CUDA(cudaStreamSynchronize(st));
  if (hflags[0] & FLAG_NONFINITE) {
    set_error("sph_build_neighbors: non-finite or non-positive density / viscosity");
    return fail(SPH_ERR_NONFINITE);
  }
  if (hflags[0] & FLAG_CAPACITY) {
    set_error("sph_build_neighbors: a particle has more than max_neighbors = %d neighbours", maxnb);
    return fail(SPH_ERR_CAPACITY);
  }
  const int64_t total = tot[0], total_pad = H->n_pad * (int64_t)maxnb;
  const int32_t maxc = (int32_t)(tot[1] & 0xffffffff);
  H->nnz = total;
  H->nnz_pad = total_pad;
  H->max_cnt = maxc;
  *out = H;
  return SPH_OK;
#undef TRYF
#undef TRYF_CUDA
}

sph_status export_neighbors(const sph_neighbors* H, int64_t* offsets, int32_t* idx, cudaStream_t st) {
  if (!H || !offsets || (!idx && H->nnz > 0)) {
    set_error("sph_neighbors_export: null argument");
    return SPH_ERR_INVALID;
  }
  sph_neighbors* M = const_cast<sph_neighbors*>(H);
  SPH_TRY(M->tmp_i32a.alloc(H->n));
  int grid = grid_for(H, H->n);
  SPH_LAUNCH(k_export_counts, grid, kBlock, 0, st)(H->iperm.p, H->cnt.p, H->n, M->tmp_i32a.p);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_scan<int64_t>, 1, 1024, 0, st)(M->tmp_i32a.p, offsets, H->n, 1, nullptr);
  SPH_TRY_CUDA(cudaGetLastError());
  if (H->nnz > 0) {
    SPH_LAUNCH(k_export_fill, grid, kBlock, 0, st)(H->iperm.p, H->perm.p, H->cnt.p, H->slice_off.p, H->nbr.p, H->n, offsets,
                                           idx);
    SPH_TRY_CUDA(cudaGetLastError());
  }
  SPH_TRY_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

}  // namespace sph
