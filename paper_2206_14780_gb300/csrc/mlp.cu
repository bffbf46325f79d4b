// Learned warm start: per-particle features, a 16-64-64-64-3 MLP on BF16 tensor
// cores (FP32 accumulation), its training kernels, and the warm-start x0.
//
// The paper names a better initial guess as future work (Sec. 8); the network
// predicts delta = (x* - v^n) / U from local features and the solve starts
// from x0 = v^n + U delta on fluid rows, the dummy-wall rows of x0 following
// from the fluid ones by Eq. dummyvel (features.cu).
//
// Inference (sph_mlp_forward, sph_warm_start) runs on the tcgen05 tensor cores
// (mlp_tc.cu), and so does training (sph_mlp_grad, sph_mlp_train_step): the loss
// and per-block partial gradients come from the tcgen05 kernel of mlp_train_tc.cu,
// summed here in block order, followed by an Adam step on float32 master weights
// and a repack of the bf16 weights.
//
// Parameter vector (float32, 9,603 entries, row-major [out][in]):
//   W1 64x16 @0, b1 @1024, W2 64x64 @1088, b2 @5184, W3 64x64 @5248, b3 @9344,
//   W4 3x64 @9408, b4 @9600.
#include <cuda_bf16.h>

#include <cmath>
#include <cstddef>
#include <cstring>

#include "sph_internal.cuh"

namespace sph {

constexpr int kNP = 9603;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248, OFF_B3 = 9344,
              OFF_W4 = 9408, OFF_B4 = 9600;
// bf16 weight pack (row-major [out][in]; W4 padded to 8 rows) and float32 biases
struct MlpPack {
  __nv_bfloat16 W1[64 * 16];
  __nv_bfloat16 W2[64 * 64];
  __nv_bfloat16 W3[64 * 64];
  __nv_bfloat16 W4[8 * 64];
  float b1[64], b2[64], b3[64], b4[8];
};

}  // namespace sph

struct sph_mlp {
  sph::DBuf<float> theta, m, v, grad, partial, loss;
  sph::DBuf<sph::MlpPack> pack;
  sph::DBuf<int> fault;          // set when a tensor-core kernel gave up a wait
  int64_t step = 0;
  int mode = 0;                  // SPH_MLP_HIGHPASS: x0 correction is y - S y
  int partial_blocks = 0;
};

namespace sph {
namespace {

__global__ void k_mlp_pack(const float* __restrict__ th, MlpPack* __restrict__ P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 64 * 64; i += gridDim.x * blockDim.x) {
    P->W2[i] = __float2bfloat16_rn(th[OFF_W2 + i]);
    P->W3[i] = __float2bfloat16_rn(th[OFF_W3 + i]);
    if (i < 64 * 16) P->W1[i] = __float2bfloat16_rn(th[OFF_W1 + i]);
    if (i < 8 * 64) {
      const int o4 = i / 64, k4 = i % 64;
      P->W4[i] = __float2bfloat16_rn((o4 < 3) ? th[OFF_W4 + o4 * 64 + k4] : 0.f);
    }
    if (i < 64) {
      P->b1[i] = th[OFF_B1 + i];
      P->b2[i] = th[OFF_B2 + i];
      P->b3[i] = th[OFF_B3 + i];
    }
    if (i < 8) P->b4[i] = (i < 3) ? th[OFF_B4 + i] : 0.f;
  }
}

// grad[i] = sum over the partial gradients of the nblocks training CTAs; loss = sum of
// their losses * inv_cnt.  One block per 32 parameters: warp g sums the partials
// g, g + 8, g + 16, ... in order, then the eight warp sums are added in warp order,
// so the result does not depend on the run.
constexpr int kReduceWarps = 8;
__global__ void __launch_bounds__(kReduceWarps * 32)
    k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ loss_part, int nblocks, float inv_cnt,
                 float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float part[kReduceWarps][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < kNP)
    for (int b = g; b < nblocks; b += kReduceWarps) s += partial[(size_t)b * kNP + i];
  part[g][lane] = s;
  __syncthreads();
  if (g == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kReduceWarps; ++w) t += part[w][lane];
    if (i < kNP) grad[i] = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 32) {
    float t = 0.f;
    for (int b = 0; b < nblocks; ++b) t += loss_part[b];
    *loss = t * inv_cnt;
  }
}

// Adam (Kingma & Ba): float32 master weights and moments, bias-corrected step
__global__ void k_mlp_adam(float* __restrict__ th, float* __restrict__ mom, float* __restrict__ vel,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * mom[i] + (1.f - b1) * gi;
    const float vi = b2 * vel[i] + (1.f - b2) * gi * gi;
    mom[i] = mi;
    vel[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

const void* mlp_pack_ptr(const sph_mlp* M) { return M->pack.p; }
int mlp_mode(const sph_mlp* M) { return M ? M->mode : 0; }

void mlp_pack_layout(size_t* off_w1, size_t* off_w2, size_t* off_w3, size_t* off_w4, size_t* off_b) {
  *off_w1 = offsetof(MlpPack, W1);
  *off_w2 = offsetof(MlpPack, W2);
  *off_w3 = offsetof(MlpPack, W3);
  *off_w4 = offsetof(MlpPack, W4);
  *off_b = offsetof(MlpPack, b1);
}

sph_status mlp_grad_tc(const sph_mlp* M, const __nv_bfloat16* feats, const float4* tgt, const uint8_t* mask,
                       int64_t m, float inv_cnt, float* partial, float* loss_part, int* err, int blocks,
                       cudaStream_t st);
int64_t mlp_grad_blocks(int64_t m, int num_sms);

sph_status mlp_forward_tc(const sph_mlp* M, const __nv_bfloat16* feats, int64_t m, float4* out, int* err,
                          int num_sms, cudaStream_t st);

// the inference forward: tcgen05 kernel of mlp_tc.cu
sph_status mlp_forward_launch(const sph_mlp* M, const __nv_bfloat16* feats, int64_t m, float4* out, int num_sms,
                              cudaStream_t st) {
  if (m <= 0) return SPH_OK;
  return mlp_forward_tc(M, feats, m, out, M->fault.p, num_sms, st);
}

static sph_status check_fault(const sph_mlp* M) {
  int f = 0;
  SPH_TRY_CUDA(cudaMemcpy(&f, M->fault.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (f) {
    set_error("warm-start network: a tensor-core kernel gave up waiting for its MMAs");
    return SPH_ERR_TIMEOUT;
  }
  return SPH_OK;
}

}  // namespace sph

using namespace sph;

extern "C" {

sph_status sph_mlp_create(const float* params, sph_mlp** out) {
  clear_error();
  if (!out) {
    set_error("sph_mlp_create: null output");
    return SPH_ERR_INVALID;
  }
  sph_mlp* M = new sph_mlp();
  auto fail = [&](sph_status s) {
    sph_mlp_destroy(M);
    *out = nullptr;
    return s;
  };
  if (M->theta.alloc(kNP) || M->m.alloc(kNP) || M->v.alloc(kNP) || M->grad.alloc(kNP) || M->loss.alloc(1) ||
      M->pack.alloc(1) || M->fault.alloc(1))
    return fail(SPH_ERR_NOMEM);
  if (cudaMemset(M->m.p, 0, kNP * 4) != cudaSuccess || cudaMemset(M->v.p, 0, kNP * 4) != cudaSuccess ||
      cudaMemset(M->theta.p, 0, kNP * 4) != cudaSuccess || cudaMemset(M->fault.p, 0, sizeof(int)) != cudaSuccess) {
    set_error("sph_mlp_create: memset failed");
    return fail(SPH_ERR_CUDA);
  }
  if (params) {
    sph_status s = sph_mlp_set_params(M, params);
    if (s != SPH_OK) return fail(s);
  } else {
    SPH_LAUNCH(k_mlp_pack, 16, 256, 0, 0)(M->theta.p, M->pack.p);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("sph_mlp_create: pack failed");
    return fail(SPH_ERR_CUDA);
  }
  *out = M;
  return SPH_OK;
}

sph_status sph_mlp_set_params(sph_mlp* M, const float* params) {
  clear_error();
  if (!M || !params) {
    set_error("sph_mlp_set_params: null argument");
    return SPH_ERR_INVALID;
  }
  for (int i = 0; i < kNP; ++i)
    if (!std::isfinite(params[i])) {
      set_error("sph_mlp_set_params: parameter %d is not finite", i);
      return SPH_ERR_NONFINITE;
    }
  SPH_TRY_CUDA(cudaMemcpy(M->theta.p, params, kNP * 4, cudaMemcpyHostToDevice));
  SPH_TRY_CUDA(cudaMemset(M->m.p, 0, kNP * 4));
  SPH_TRY_CUDA(cudaMemset(M->v.p, 0, kNP * 4));
  M->step = 0;
  SPH_LAUNCH(k_mlp_pack, 16, 256, 0, 0)(M->theta.p, M->pack.p);
  SPH_TRY_CUDA(cudaGetLastError());
  SPH_TRY_CUDA(cudaDeviceSynchronize());
  return SPH_OK;
}

sph_status sph_mlp_get_params(const sph_mlp* M, float* params) {
  clear_error();
  if (!M || !params) {
    set_error("sph_mlp_get_params: null argument");
    return SPH_ERR_INVALID;
  }
  SPH_TRY_CUDA(cudaMemcpy(params, M->theta.p, kNP * 4, cudaMemcpyDeviceToHost));
  return check_fault(M);
}

sph_status sph_mlp_set_mode(sph_mlp* M, int32_t mode) {
  clear_error();
  if (!M || (mode & ~SPH_MLP_HIGHPASS)) {
    set_error("sph_mlp_set_mode: null network or unknown mode bits %d", mode);
    return SPH_ERR_INVALID;
  }
  M->mode = mode;
  return SPH_OK;
}

sph_status sph_mlp_destroy(sph_mlp* M) {
  if (!M) return SPH_OK;
  M->theta.release();
  M->m.release();
  M->v.release();
  M->grad.release();
  M->partial.release();
  M->loss.release();
  M->pack.release();
  M->fault.release();
  delete M;
  return SPH_OK;
}

sph_status sph_mlp_forward(const sph_mlp* M, const uint16_t* feats, int64_t m, float* out, void* stream) {
  clear_error();
  if (!M || !feats || !out || m < 0) {
    set_error("sph_mlp_forward: null argument or negative count");
    return SPH_ERR_INVALID;
  }
  if (m == 0) return SPH_OK;
  int dev = 0, sms = 0;
  SPH_TRY_CUDA(cudaGetDevice(&dev));
  SPH_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPH_TRY(mlp_forward_launch(M, reinterpret_cast<const __nv_bfloat16*>(feats), m, reinterpret_cast<float4*>(out), sms,
                             reinterpret_cast<cudaStream_t>(stream)));
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

static sph_status mlp_grad_impl(sph_mlp* M, const uint16_t* feats, const float* targets, const uint8_t* mask,
                                int64_t m, float inv_cnt, cudaStream_t st) {
  int dev = 0, sms = 0;
  SPH_TRY_CUDA(cudaGetDevice(&dev));
  SPH_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = mlp_grad_blocks(m, sms);
  if (M->partial_blocks < blocks) {
    SPH_TRY(M->partial.alloc((size_t)blocks * kNP + blocks));
    M->partial_blocks = (int)blocks;
  }
  float* loss_part = M->partial.p + (size_t)blocks * kNP;
  SPH_TRY(mlp_grad_tc(M, reinterpret_cast<const __nv_bfloat16*>(feats), reinterpret_cast<const float4*>(targets),
                      mask, m, inv_cnt, M->partial.p, loss_part, M->fault.p, (int)blocks, st));
  SPH_LAUNCH(k_mlp_reduce, (kNP + 31) / 32, kReduceWarps * 32, 0, st)(M->partial.p, loss_part, (int)blocks, inv_cnt,
                                                                      M->grad.p, M->loss.p);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

sph_status sph_mlp_grad(sph_mlp* M, const uint16_t* feats, const float* targets, const uint8_t* mask, int64_t m,
                        int64_t count, float* grad_out, float* loss_out, void* stream) {
  clear_error();
  if (!M || !feats || !targets || m < 1 || count < 1) {
    set_error("sph_mlp_grad: null argument, empty batch or count < 1");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(mlp_grad_impl(M, feats, targets, mask, m, 1.f / (float)count, st));
  if (grad_out) SPH_TRY_CUDA(cudaMemcpyAsync(grad_out, M->grad.p, kNP * 4, cudaMemcpyDeviceToDevice, st));
  if (loss_out) SPH_TRY_CUDA(cudaMemcpyAsync(loss_out, M->loss.p, 4, cudaMemcpyDeviceToDevice, st));
  return SPH_OK;
}

sph_status sph_mlp_train_step(sph_mlp* M, const uint16_t* feats, const float* targets, const uint8_t* mask,
                              int64_t m, int64_t count, float lr, float* loss_host, void* stream) {
  clear_error();
  if (!M || !feats || !targets || m < 1 || count < 1 || !(lr > 0.f)) {
    set_error("sph_mlp_train_step: bad argument");
    return SPH_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SPH_TRY(mlp_grad_impl(M, feats, targets, mask, m, 1.f / (float)count, st));
  M->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
  SPH_LAUNCH(k_mlp_adam, (kNP + 255) / 256, 256, 0, st)(M->theta.p, M->m.p, M->v.p, M->grad.p, lr, b1, b2, eps, c1,
                                                        c2);
  SPH_LAUNCH(k_mlp_pack, 16, 256, 0, st)(M->theta.p, M->pack.p);
  SPH_TRY_CUDA(cudaGetLastError());
  if (loss_host) {
    SPH_TRY_CUDA(cudaMemcpyAsync(loss_host, M->loss.p, 4, cudaMemcpyDeviceToHost, st));
    SPH_TRY_CUDA(cudaStreamSynchronize(st));
    SPH_TRY(check_fault(M));
  }
  return SPH_OK;
}

}  // extern "C"
