// Learned warm start: per-particle features, a 16-64-64-64-3 MLP on BF16 tensor
// cores (FP32 accumulation), its training kernels, and the warm-start x0.
//
// The paper names a better initial guess as future work (Sec. 8); the network
// predicts delta = (x* - v^n) / U from local features and the solve starts
// from x0 = v^n + U delta on fluid rows, the dummy-wall rows of x0 following
// from the fluid ones by Eq. dummyvel (features.cu).
//
// Inference (sph_mlp_forward, sph_warm_start) runs on the tcgen05 tensor cores
// (mlp_tc.cu).  Training (sph_mlp_grad, sph_mlp_train_step) runs forward and
// backward per warp with mma.sync.m16n8k16 (bf16 x bf16 -> f32), keeping every
// activation and data gradient in registers.  One warp owns 16 particles.  The
// accumulator fragment of two adjacent 8-column tiles is, lane for lane, the A
// fragment of the next 16-wide K chunk, so hidden activations stay in registers
// between layers (bias, SiLU and the bf16 rounding are applied in place).  The backward pass reuses the same trick for the data gradients
// (delta W with W^T kept in shared memory); the weight gradients
// dW = delta^T a are products over the warp's 16 rows with operands read from
// per-warp shared-memory tiles.
//
// Parameter vector (float32, 9,603 entries, row-major [out][in]):
//   W1 64x16 @0, b1 @1024, W2 64x64 @1088, b2 @5184, W3 64x64 @5248, b3 @9344,
//   W4 3x64 @9408, b4 @9600.
#include <cuda_bf16.h>

#include <cmath>
#include <cstddef>
#include <cstring>

#include "reduce.cuh"
#include "sph_internal.cuh"

namespace sph {

constexpr int kNP = 9603;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248, OFF_B3 = 9344,
              OFF_W4 = 9408, OFF_B4 = 9600;
constexpr int kFeat = 16;

// bf16 weight packs (row-major [out][in] and transposed [in][out]), padded W4
struct MlpPack {
  __nv_bfloat16 W1[64 * 16], W1T[16 * 64];
  __nv_bfloat16 W2[64 * 64], W2T[64 * 64];
  __nv_bfloat16 W3[64 * 64], W3T[64 * 64];
  __nv_bfloat16 W4[8 * 64], W4T[64 * 8];
  float b1[64], b2[64], b3[64], b4[8];
};

}  // namespace sph

struct sph_mlp {
  sph::DBuf<float> theta, m, v, grad, partial, loss;
  sph::DBuf<sph::MlpPack> pack;
  sph::DBuf<int> fault;          // set when a tensor-core forward gave up a wait
  int64_t step = 0;
  int mode = 0;                  // SPH_MLP_HIGHPASS: x0 correction is y - S y
  int partial_blocks = 0;
};

namespace sph {
namespace {

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack_bf(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A(16x16, row) * B(16x8, col) + D, bf16 in, f32 accumulate
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__global__ void k_mlp_pack(const float* __restrict__ th, MlpPack* __restrict__ P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 64 * 64; i += gridDim.x * blockDim.x) {
    const int o = i / 64, k = i % 64;
    P->W2[i] = __float2bfloat16_rn(th[OFF_W2 + i]);
    P->W2T[k * 64 + o] = __float2bfloat16_rn(th[OFF_W2 + i]);
    P->W3[i] = __float2bfloat16_rn(th[OFF_W3 + i]);
    P->W3T[k * 64 + o] = __float2bfloat16_rn(th[OFF_W3 + i]);
    if (i < 64 * 16) {
      const int o1 = i / 16, k1 = i % 16;
      P->W1[i] = __float2bfloat16_rn(th[OFF_W1 + i]);
      P->W1T[k1 * 64 + o1] = __float2bfloat16_rn(th[OFF_W1 + i]);
    }
    if (i < 8 * 64) {
      const int o4 = i / 64, k4 = i % 64;
      const float w = (o4 < 3) ? th[OFF_W4 + o4 * 64 + k4] : 0.f;
      P->W4[i] = __float2bfloat16_rn(w);
      P->W4T[k4 * 8 + o4] = __float2bfloat16_rn(w);
    }
    if (i < 64) {
      P->b1[i] = th[OFF_B1 + i];
      P->b2[i] = th[OFF_B2 + i];
      P->b3[i] = th[OFF_B3 + i];
    }
    if (i < 8) P->b4[i] = (i < 3) ? th[OFF_B4 + i] : 0.f;
  }
}

// cooperative copy of the weight pack into shared memory
__device__ __forceinline__ void load_pack(const MlpPack* __restrict__ g, MlpPack* s) {
  const int4* src = reinterpret_cast<const int4*>(g);
  int4* dst = reinterpret_cast<int4*>(s);
  for (int i = threadIdx.x; i < (int)(sizeof(MlpPack) / 16); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// hidden layer: c[8][4] (16 x 64 outputs) from A fragments over K = 16 * KC
template <int KC>
__device__ __forceinline__ void layer(float c[8][4], const uint32_t a[KC][4], const __nv_bfloat16* W, int ldw,
                                      const float* bias, int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
    c[j][0] = b0;
    c[j][1] = b1;
    c[j][2] = b0;
    c[j][3] = b1;
#pragma unroll
    for (int m = 0; m < KC; ++m) {
      uint32_t b[2];
      b[0] = ld32(W + (8 * j + g) * ldw + 16 * m + 2 * t);
      b[1] = ld32(W + (8 * j + g) * ldw + 16 * m + 2 * t + 8);
      mma16816(c[j], a[m], b);
    }
  }
}

// SiLU in place and repack as the A fragments of the next layer (4 K chunks)
__device__ __forceinline__ void act_to_a(float c[8][4], uint32_t a[4][4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m][0] = pack2(silu(c[2 * m][0]), silu(c[2 * m][1]));
    a[m][1] = pack2(silu(c[2 * m][2]), silu(c[2 * m][3]));
    a[m][2] = pack2(silu(c[2 * m + 1][0]), silu(c[2 * m + 1][1]));
    a[m][3] = pack2(silu(c[2 * m + 1][2]), silu(c[2 * m + 1][3]));
  }
}

__device__ __forceinline__ void load_a0(const __nv_bfloat16* __restrict__ f, int64_t m, int64_t r0, int g, int t,
                                        uint32_t a[4]) {
  const int64_t ra = r0 + g, rb = r0 + g + 8;
  a[0] = ra < m ? ld32(f + ra * kFeat + 2 * t) : 0u;
  a[1] = rb < m ? ld32(f + rb * kFeat + 2 * t) : 0u;
  a[2] = ra < m ? ld32(f + ra * kFeat + 2 * t + 8) : 0u;
  a[3] = rb < m ? ld32(f + rb * kFeat + 2 * t + 8) : 0u;
}


// per-warp shared scratch of the training kernel
struct WarpTile {
  float z[3][16][64];            // pre-activations of the hidden layers
  __nv_bfloat16 a[4][16][64];    // layer inputs: a0 (16 wide) .. a3
  __nv_bfloat16 d[16][64];       // current backpropagated delta (bf16)
};
constexpr int kTrainWarps = 4;

// store a c[8][4] fragment (16 x 64) into a row-major [16][64] tile
__device__ __forceinline__ void store_c_f32(float (*dst)[64], const float c[8][4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    dst[g][8 * j + 2 * t] = c[j][0];
    dst[g][8 * j + 2 * t + 1] = c[j][1];
    dst[g + 8][8 * j + 2 * t] = c[j][2];
    dst[g + 8][8 * j + 2 * t + 1] = c[j][3];
  }
}
__device__ __forceinline__ void store_a_bf16(__nv_bfloat16 (*dst)[64], const uint32_t a[4][4], int g, int t) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    *reinterpret_cast<uint32_t*>(&dst[g][16 * m + 2 * t]) = a[m][0];
    *reinterpret_cast<uint32_t*>(&dst[g + 8][16 * m + 2 * t]) = a[m][1];
    *reinterpret_cast<uint32_t*>(&dst[g][16 * m + 2 * t + 8]) = a[m][2];
    *reinterpret_cast<uint32_t*>(&dst[g + 8][16 * m + 2 * t + 8]) = a[m][3];
  }
}

// dW[o][i] += sum_r d[r][o] * act[r][i] over the warp's 16 rows; o < NO (m tiles of 16),
// i < NI (n tiles of 8); accumulated into the block's shared gradient gW[o * ldg + i]
template <int MT, int NT>
__device__ __forceinline__ void weight_grad(const __nv_bfloat16 (*d)[64], const __nv_bfloat16 (*act)[64],
                                            float* gW, int ldg, int o_lim, int g, int t) {
#pragma unroll
  for (int mi = 0; mi < MT; ++mi) {
    uint32_t a[4];
    const int o0 = 16 * mi + g, o1 = o0 + 8;
    a[0] = pack_bf(d[2 * t][o0], d[2 * t + 1][o0]);
    a[1] = pack_bf(d[2 * t][o1], d[2 * t + 1][o1]);
    a[2] = pack_bf(d[2 * t + 8][o0], d[2 * t + 9][o0]);
    a[3] = pack_bf(d[2 * t + 8][o1], d[2 * t + 9][o1]);
#pragma unroll
    for (int ni = 0; ni < NT; ++ni) {
      uint32_t b[2];
      const int i0 = 8 * ni + g;
      b[0] = pack_bf(act[2 * t][i0], act[2 * t + 1][i0]);
      b[1] = pack_bf(act[2 * t + 8][i0], act[2 * t + 9][i0]);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(c, a, b);
      const int ia = 8 * ni + 2 * t;
      if (o0 < o_lim) {
        atomicAdd(&gW[o0 * ldg + ia], c[0]);
        atomicAdd(&gW[o0 * ldg + ia + 1], c[1]);
      }
      if (o1 < o_lim) {
        atomicAdd(&gW[o1 * ldg + ia], c[2]);
        atomicAdd(&gW[o1 * ldg + ia + 1], c[3]);
      }
    }
  }
}

// data gradient: da (16 x 64) = delta (16 x 16*KC) * W (16*KC x 64), with W^T [64][ldw]
template <int KC>
__device__ __forceinline__ void data_grad(float c[8][4], const uint32_t dA[KC][4], const __nv_bfloat16* WT, int ldw,
                                          int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
    for (int m = 0; m < KC; ++m) {
      uint32_t b[2];
      b[0] = ld32(WT + (8 * j + g) * ldw + 16 * m + 2 * t);
      b[1] = (16 * m + 2 * t + 8 < ldw) ? ld32(WT + (8 * j + g) * ldw + 16 * m + 2 * t + 8) : 0u;
      mma16816(c[j], dA[m], b);
    }
  }
}

// delta = da * SiLU'(z): bias gradients (float32 sums), bf16 tile for dW, A fragments for the next data gradient
__device__ __forceinline__ void delta_hidden(float c[8][4], const float (*z)[64], float* gb, __nv_bfloat16 (*dt)[64],
                                             uint32_t dA[4][4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i0 = 8 * j + 2 * t;
    c[j][0] *= dsilu(z[g][i0]);
    c[j][1] *= dsilu(z[g][i0 + 1]);
    c[j][2] *= dsilu(z[g + 8][i0]);
    c[j][3] *= dsilu(z[g + 8][i0 + 1]);
    atomicAdd(&gb[i0], c[j][0] + c[j][2]);
    atomicAdd(&gb[i0 + 1], c[j][1] + c[j][3]);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    dA[m][0] = pack2(c[2 * m][0], c[2 * m][1]);
    dA[m][1] = pack2(c[2 * m][2], c[2 * m][3]);
    dA[m][2] = pack2(c[2 * m + 1][0], c[2 * m + 1][1]);
    dA[m][3] = pack2(c[2 * m + 1][2], c[2 * m + 1][3]);
  }
  store_a_bf16(dt, dA, g, t);
}

// loss and gradient over m rows: block partial gradients [grid][kNP] and losses
__global__ void __launch_bounds__(kTrainWarps * 32) k_mlp_grad(const MlpPack* __restrict__ Pg,
                                                                const __nv_bfloat16* __restrict__ feats,
                                                                const float4* __restrict__ tgt,
                                                                const uint8_t* __restrict__ mask, int64_t m,
                                                                float inv_cnt, float* __restrict__ partial,
                                                                float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem[];
  MlpPack& P = *reinterpret_cast<MlpPack*>(smem);
  float* G = reinterpret_cast<float*>(smem + sizeof(MlpPack));                       // [kNP]
  WarpTile* tiles = reinterpret_cast<WarpTile*>(smem + sizeof(MlpPack) + ((kNP * 4 + 15) / 16) * 16);
  __shared__ float sloss;
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) G[i] = 0.f;
  if (threadIdx.x == 0) sloss = 0.f;
  load_pack(Pg, &P);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, wid = threadIdx.x >> 5;
  WarpTile& T = tiles[wid];
  const int64_t warps = (int64_t)gridDim.x * kTrainWarps;
  float lsum = 0.f;
  for (int64_t w = (int64_t)blockIdx.x * kTrainWarps + wid; w * 16 < m; w += warps) {
    const int64_t r0 = w * 16;
    // ---- forward, keeping z and the layer inputs
    uint32_t a0[1][4];
    load_a0(feats, m, r0, g, t, a0[0]);
    *reinterpret_cast<uint32_t*>(&T.a[0][g][2 * t]) = a0[0][0];
    *reinterpret_cast<uint32_t*>(&T.a[0][g + 8][2 * t]) = a0[0][1];
    *reinterpret_cast<uint32_t*>(&T.a[0][g][2 * t + 8]) = a0[0][2];
    *reinterpret_cast<uint32_t*>(&T.a[0][g + 8][2 * t + 8]) = a0[0][3];
    float c[8][4];
    uint32_t a[4][4];
    layer<1>(c, a0, P.W1, 16, P.b1, g, t);
    store_c_f32(T.z[0], c, g, t);
    act_to_a(c, a);
    store_a_bf16(T.a[1], a, g, t);
    layer<4>(c, a, P.W2, 64, P.b2, g, t);
    store_c_f32(T.z[1], c, g, t);
    act_to_a(c, a);
    store_a_bf16(T.a[2], a, g, t);
    layer<4>(c, a, P.W3, 64, P.b3, g, t);
    store_c_f32(T.z[2], c, g, t);
    act_to_a(c, a);
    store_a_bf16(T.a[3], a, g, t);
    float y[4] = {P.b4[2 * t], P.b4[2 * t + 1], P.b4[2 * t], P.b4[2 * t + 1]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t b[2];
      b[0] = ld32(P.W4 + g * 64 + 16 * k + 2 * t);
      b[1] = ld32(P.W4 + g * 64 + 16 * k + 2 * t + 8);
      mma16816(y, a[k], b);
    }
    // ---- output delta d4 = 2 (y - t) / count on masked rows, columns < 3
    float d4[4];
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    const bool va = ra < m && (!mask || mask[ra]), vb = rb < m && (!mask || mask[rb]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = 2 * t + (q & 1);
      const bool valid = col < 3 && ((q < 2) ? va : vb);
      const int64_t row = (q < 2) ? ra : rb;
      const float target = valid ? reinterpret_cast<const float*>(tgt)[row * 4 + col] : 0.f;
      const float diff = valid ? (y[q] - target) : 0.f;
      lsum += diff * diff;
      d4[q] = 2.f * diff * inv_cnt;
    }
    if (2 * t < 3) {
      atomicAdd(&G[OFF_B4 + 2 * t], d4[0] + d4[2]);
      if (2 * t + 1 < 3) atomicAdd(&G[OFF_B4 + 2 * t + 1], d4[1] + d4[3]);
    }
    // d4 as a bf16 16 x 8 tile (columns 8.. of the scratch stay zero)
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 64; j += 8) {
      if (j == 0) {
        T.d[g][2 * t] = __float2bfloat16_rn(d4[0]);
        T.d[g][2 * t + 1] = __float2bfloat16_rn(d4[1]);
        T.d[g + 8][2 * t] = __float2bfloat16_rn(d4[2]);
        T.d[g + 8][2 * t + 1] = __float2bfloat16_rn(d4[3]);
      } else {
        T.d[g][j + 2 * t] = __float2bfloat16_rn(0.f);
        T.d[g][j + 2 * t + 1] = __float2bfloat16_rn(0.f);
        T.d[g + 8][j + 2 * t] = __float2bfloat16_rn(0.f);
        T.d[g + 8][j + 2 * t + 1] = __float2bfloat16_rn(0.f);
      }
    }
    __syncwarp();
    // dW4[o][i] = sum_r d4[r][o] a3[r][i]   (o < 3)
    weight_grad<1, 8>(T.d, T.a[3], G + OFF_W4, 64, 3, g, t);
    // da3 = d4 (16 x 16, columns >= 8 zero) * W4 (16 x 64) with W4T [64][8]
    uint32_t dA4[1][4];
    dA4[0][0] = pack2(d4[0], d4[1]);
    dA4[0][1] = pack2(d4[2], d4[3]);
    dA4[0][2] = 0u;
    dA4[0][3] = 0u;
    data_grad<1>(c, dA4, P.W4T, 8, g, t);
    uint32_t dA[4][4];
    __syncwarp();
    delta_hidden(c, T.z[2], G + OFF_B3, T.d, dA, g, t);
    __syncwarp();
    weight_grad<4, 8>(T.d, T.a[2], G + OFF_W3, 64, 64, g, t);
    data_grad<4>(c, dA, P.W3T, 64, g, t);
    __syncwarp();
    delta_hidden(c, T.z[1], G + OFF_B2, T.d, dA, g, t);
    __syncwarp();
    weight_grad<4, 8>(T.d, T.a[1], G + OFF_W2, 64, 64, g, t);
    data_grad<4>(c, dA, P.W2T, 64, g, t);
    __syncwarp();
    delta_hidden(c, T.z[0], G + OFF_B1, T.d, dA, g, t);
    __syncwarp();
    weight_grad<4, 2>(T.d, T.a[0], G + OFF_W1, 16, 64, g, t);
    __syncwarp();
  }
  atomicAdd(&sloss, lsum);
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * kNP;
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) out[i] = G[i];
  if (threadIdx.x == 0) loss_part[blockIdx.x] = sloss;
}

// grad[i] = sum over blocks (fixed order); loss = sum of block losses * inv_cnt
__global__ void k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ loss_part, int nblocks,
                             float inv_cnt, float* __restrict__ grad, float* __restrict__ loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * kNP + i];
    grad[i] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += loss_part[b];
    *loss = s * inv_cnt;
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

int mlp_train_smem() {
  return (int)(sizeof(MlpPack) + ((kNP * 4 + 15) / 16) * 16 + kTrainWarps * sizeof(WarpTile));
}

const void* mlp_pack_ptr(const sph_mlp* M) { return M->pack.p; }
int mlp_mode(const sph_mlp* M) { return M ? M->mode : 0; }

void mlp_pack_layout(size_t* off_w1, size_t* off_w2, size_t* off_w3, size_t* off_w4, size_t* off_b) {
  *off_w1 = offsetof(MlpPack, W1);
  *off_w2 = offsetof(MlpPack, W2);
  *off_w3 = offsetof(MlpPack, W3);
  *off_w4 = offsetof(MlpPack, W4);
  *off_b = offsetof(MlpPack, b1);
}

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
    set_error("warm-start network: a tensor-core forward gave up waiting for its MMAs");
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
  const int smem = mlp_train_smem();
  static bool attr_set = false;
  if (!attr_set) {
    SPH_TRY_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr_set = true;
  }
  int64_t blocks = (m + 16 * kTrainWarps - 1) / (16 * kTrainWarps);
  if (blocks > sms) blocks = sms;
  if (blocks < 1) blocks = 1;
  if (M->partial_blocks < blocks) {
    SPH_TRY(M->partial.alloc((size_t)blocks * kNP + blocks));
    M->partial_blocks = (int)blocks;
  }
  float* loss_part = M->partial.p + (size_t)blocks * kNP;
  SPH_LAUNCH(k_mlp_grad, (int)blocks, kTrainWarps * 32, smem, st)(
      M->pack.p, reinterpret_cast<const __nv_bfloat16*>(feats), reinterpret_cast<const float4*>(targets), mask, m,
      inv_cnt, M->partial.p, loss_part);
  SPH_LAUNCH(k_mlp_reduce, (kNP + 255) / 256, 256, 0, st)(M->partial.p, loss_part, (int)blocks, inv_cnt, M->grad.p,
                                                          M->loss.p);
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
