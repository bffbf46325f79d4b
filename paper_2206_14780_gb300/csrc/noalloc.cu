// sph_visc_apply_noalloc: y = A(dt) v without any device allocation.
//
// The cell-sorted copies of v and y live in a file-scope device array instead
// of handle workspace.  In host code the array's name is only a host-side
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int64_t kMaxRows = SPH_NOALLOC_MAX_ROWS;
constexpr int kMaxDevices = 64;

// [0, kMaxRows): sorted v; [kMaxRows, 2 kMaxRows): sorted y.  8 MiB.
__device__ __align__(256) float4 g_noalloc_scratch[2 * kMaxRows];

// The address is looked up once per device and kept: it stays valid for the
// life of the device's primary context.  cudaDeviceReset destroys that context
// (and the array's storage with it), so a process that resets a device must not
// call sph_visc_apply_noalloc on it afterwards.
std::mutex g_mutex;
float4* g_scratch_ptr[kMaxDevices] = {};

sph_status scratch_for_current_device(float4** out) {
  int dev = 0;
  SPH_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sph_visc_apply_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
    return SPH_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("sph_visc_apply_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return SPH_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<float4*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SPH_OK;
}

__global__ void k_na_gather(const float4* __restrict__ v, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                            float4* __restrict__ vs) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      const float4 t = v[perm[s]];
      vs[s] = make_float4(t.x, t.y, t.z, 0.f);
    } else {
      vs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

__global__ void k_na_scatter(const float4* __restrict__ ys, const int32_t* __restrict__ perm, int64_t n,
                             float4* __restrict__ y) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    y[perm[s]] = ys[s];
}

}  // namespace

sph_status visc_apply_noalloc(sph_neighbors* H, const sph_visc_params* P, const float* v, float* y,
                              cudaStream_t st) {
  if (!H || !P || !v || !y) {
    set_error("sph_visc_apply_noalloc: null argument");
    return SPH_ERR_INVALID;
  }
  {
    // [v, v + 16 n) and [y, y + 16 n) must be disjoint
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(v), b0 = reinterpret_cast<uintptr_t>(y);
    const uintptr_t len = (uintptr_t)H->n * sizeof(float4);
    if (a0 < b0 + len && b0 < a0 + len) {
      set_error("sph_visc_apply_noalloc: v and y must not overlap");
      return SPH_ERR_INVALID;
    }
  }
  if (!H->op_valid || H->op_params.dt != P->dt || H->op_params.boundary != P->boundary ||
      H->op_params.mean != P->mean || H->op_mu_version != H->mu_version) {
    set_error("sph_visc_apply_noalloc: the coefficients for these parameters are not set up on the handle "
              "(call sph_visc_setup first; it may allocate)");
    return SPH_ERR_INVALID;
  }
  if (H->n_pad > kMaxRows) {
    set_error("sph_visc_apply_noalloc: %lld rows exceed SPH_NOALLOC_MAX_ROWS = %lld", (long long)H->n_pad,
              (long long)kMaxRows);
    return SPH_ERR_INVALID;
  }
  float4* scr = nullptr;
  SPH_TRY(scratch_for_current_device(&scr));
  float4* vs = scr;
  float4* ys = scr + kMaxRows;
  const int grid = grid_for(H, H->n_pad);
  SPH_LAUNCH(k_na_gather, grid, kBlock, 0, st)(reinterpret_cast<const float4*>(v), H->perm.p, H->n, H->n_pad, vs);
  SPH_TRY_CUDA(cudaGetLastError());
  launch_apply_f32(H, vs, ys, false, st);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_LAUNCH(k_na_scatter, grid, kBlock, 0, st)(ys, H->perm.p, H->n, reinterpret_cast<float4*>(y));
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
