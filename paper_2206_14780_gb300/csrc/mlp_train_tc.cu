// Warm-start network training on the 5th-generation tensor cores (tcgen05): the
// mean-squared-error loss and its gradient with respect to all 9,603 parameters.
//
// Two CTAs of 8 warps per SM walk 128-row tiles (persistent over the tiles), so
// one CTA's epilogues overlap the other's MMAs.  Each row is one particle; warps w
// and w + 4 share the tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31 (one row
// per thread) and split every 64-column layer into two halves.  Every product of a
// tile is one tcgen05.mma chain issued by one thread:
//
//   forward      Z_l  = A_{l-1} W_l^T               K-major tiles, as in inference
//   data grad    DA   = Delta_{l+1} W_{l+1}         B = the W_{l+1} tile read MN-major
//   weight grad  dW_l += Delta_l^T A_{l-1}          both operands MN-major: the
//                                                   row-by-row tiles read with the
//                                                   tile's 128 rows as the K index
//
// Tensor memory (256 columns per CTA): Z (64) holds the forward's pre-activations in
// turn and, in the backward pass, Z_3 (kept) and Z_2, Z_1 (recomputed by the same
// MMAs, so SiLU' sees the forward's float32 values); DA (64) the output Y and then
// the data gradients; the weight gradients accumulate over all of the CTA's tiles
// and are written once, as the CTA's partial gradient, at the end.  dW_3 and dW_2
// share one 128-row accumulator: the hidden-delta tile keeps two 64-column halves
// per 8-row group, and Delta_3 is written to the first half with the second zeroed,
// Delta_2 to the second with the first zeroed, so the M = 128 MMA over both halves
// adds Delta_3^T A_2 to rows 0..63 and Delta_2^T A_1 to rows 64..127.  dW_1 and
// dW_4^T have 16 columns each; their rows 64..127 read bytes beyond the operand
// (padded tile memory) and are never read back.  Bias gradients are column sums of
// the float32 deltas (a transposing warp reduction, kept per lane).
//
// Rounding points follow the float64 reference: inputs, weights, hidden activations
// and backpropagated deltas enter products as bf16; accumulation, biases, SiLU' and
// the bias sums are float32.  Each partial gradient is deterministic (fixed tile
// order per CTA), and the partials are summed in block order by the caller.
//
// Waits on the MMA mbarrier are bounded; on a timeout the kernel sets *err, frees
// its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "sph_internal.cuh"
#include "tcgen05.cuh"

namespace sph {

struct MlpPack;
const void* mlp_pack_ptr(const sph_mlp* M);
void mlp_pack_layout(size_t* off_w1, size_t* off_w2, size_t* off_w3, size_t* off_w4, size_t* off_b);

namespace {

constexpr int kNP = 9603;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248, OFF_B3 = 9344,
              OFF_W4 = 9408, OFF_B4 = 9600;
constexpr int kRows = 128;
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;
constexpr long long kMmaWaitCycles = 4000000000ll;

// tensor-memory columns
constexpr uint32_t TZ = 0, TDA = 64, TW23 = 128, TW1 = 192, TW4 = 208;

// shared-memory map (bytes from the dynamic base)
constexpr int SM_W1 = 0;                  // 64 x 16  [out][in], SBO 256
constexpr int SM_W2 = SM_W1 + 2048;       // 64 x 64, SBO 1024
constexpr int SM_W3 = SM_W2 + 8192;
constexpr int SM_W4 = SM_W3 + 8192;       // 16 x 64 (rows 3..15 zero)
constexpr int SM_X = SM_W4 + 2048;        // 128 x 16 features, SBO 256
constexpr int SM_A1 = SM_X + 4096;        // 128 x 64 activations, SBO 1024
constexpr int SM_A2 = SM_A1 + 16384;
constexpr int SM_A3 = SM_A2 + 16384;      // + 1 KB read by the M = 128 dW_4^T MMA
constexpr int SM_D4 = SM_A3 + 16384 + 1024;   // 128 x 16 output deltas, SBO 256
constexpr int SM_DL = SM_D4 + 4096;       // 128 x (64 + 64) hidden deltas in two halves, SBO 2048
constexpr int SM_B = SM_DL + 32768;       // biases: 64 + 64 + 64 + 8 float
constexpr int SM_BAR = SM_B + 800;        // mbarrier (8 B) + tensor-memory address (4 B)
constexpr int SM_END = SM_BAR + 16;
constexpr int SM_RED = SM_A1;             // after the last tile: 8 warps x 32 x 3 bias partials, 8 x 4, 8
constexpr int kSmemDyn = SM_END;
static_assert(kSmemDyn <= 111 * 1024, "two CTAs per SM need at most 111 KB each");
static_assert((8 * 32 * 3 + 8 * 4 + 8) * 4 <= 16384, "reduction scratch exceeds its alias");
static_assert(SM_X % 1024 == 0 && SM_A1 % 1024 == 0 && SM_A3 % 1024 == 0 && SM_DL % 1024 == 0, "tile alignment");

// SiLU and its derivative with the fast reciprocal (relative error ~1e-7, far below
// the bf16 rounding that follows)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// v[0..31] per lane -> the returned value of lane l is the sum of v[l] over the warp
__device__ __forceinline__ float transpose_sum32(float v[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < s; ++j) {
      const float send = up ? v[j] : v[j + s];
      const float keep = up ? v[j + s] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  return v;
}

// 32 values -> bf16 -> four 16-byte chunks of row `row`, columns c0 .. c0 + 31, of a
// row-by-row tile whose 8-row groups are sbo bytes apart
__device__ __forceinline__ void store_row32(char* tile, int row, int c0, const float v[32], int sbo = 1024) {
#pragma unroll
  for (int g = 0; g < 4; ++g)
    *reinterpret_cast<uint4*>(tile + tc::cm_off(row, c0 + 8 * g, sbo)) =
        make_uint4(pack2(v[8 * g], v[8 * g + 1]), pack2(v[8 * g + 2], v[8 * g + 3]), pack2(v[8 * g + 4], v[8 * g + 5]),
                   pack2(v[8 * g + 6], v[8 * g + 7]));
}

__global__ void __launch_bounds__(kThreads, 2)
    k_mlp_grad_tc(const char* __restrict__ pack, int64_t off_w1, int64_t off_w2, int64_t off_w3, int64_t off_w4,
                  int64_t off_b, const __nv_bfloat16* __restrict__ feats, const float4* __restrict__ tgt,
                  const uint8_t* __restrict__ mask, int64_t m, float inv_cnt, float* __restrict__ partial,
                  float* __restrict__ loss_part, int* err) {
  extern __shared__ __align__(1024) char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane, half = warp >> 2, c0 = 32 * half;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM_BAR + 8);
  float* bias = reinterpret_cast<float*>(smem + SM_B);

  // weights into row-by-row tiles (16-byte chunks of 8 bf16 along the inner index)
  for (int i = tid; i < 64 * 2; i += kThreads) {            // W1 [64][16]
    const int n = i >> 1, c = i & 1;
    *reinterpret_cast<uint4*>(smem + SM_W1 + tc::cm_off(n, 8 * c, 256)) =
        *reinterpret_cast<const uint4*>(pack + off_w1 + (size_t)(n * 16 + 8 * c) * 2);
  }
  for (int i = tid; i < 64 * 8; i += kThreads) {            // W2, W3 [64][64]
    const int n = i >> 3, c = i & 7;
    const int o = tc::cm_off(n, 8 * c, 1024);
    const size_t src = (size_t)(n * 64 + 8 * c) * 2;
    *reinterpret_cast<uint4*>(smem + SM_W2 + o) = *reinterpret_cast<const uint4*>(pack + off_w2 + src);
    *reinterpret_cast<uint4*>(smem + SM_W3 + o) = *reinterpret_cast<const uint4*>(pack + off_w3 + src);
  }
  for (int i = tid; i < 16 * 8; i += kThreads) {            // W4 [16][64], rows >= 3 zero
    const int n = i >> 3, c = i & 7;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (n < 3) w = *reinterpret_cast<const uint4*>(pack + off_w4 + (size_t)(n * 64 + 8 * c) * 2);
    *reinterpret_cast<uint4*>(smem + SM_W4 + tc::cm_off(n, 8 * c, 1024)) = w;
  }
  for (int i = tid; i < 200; i += kThreads) bias[i] = *reinterpret_cast<const float*>(pack + off_b + (size_t)i * 4);
  // the padding behind A3 (read into dW_4^T rows that are never read back) and the
  // hidden-delta tile (its second halves must be zero before the first Delta_3)
  for (int i = tid; i < 64; i += kThreads)
    reinterpret_cast<uint4*>(smem + SM_A3 + 16384)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < 32768 / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem + SM_DL)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbarrier_init();
  }
  if (warp == 0) tc::alloc(tslot, kTmemCols);
  fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);

  const uint32_t aX = smem_addr(smem + SM_X), aA1 = smem_addr(smem + SM_A1), aA2 = smem_addr(smem + SM_A2),
                 aA3 = smem_addr(smem + SM_A3), aD4 = smem_addr(smem + SM_D4), aDL = smem_addr(smem + SM_DL);
  const uint32_t aW1 = smem_addr(smem + SM_W1), aW2 = smem_addr(smem + SM_W2), aW3 = smem_addr(smem + SM_W3),
                 aW4 = smem_addr(smem + SM_W4);
  constexpr uint32_t id64 = tc::idesc_bf16(128, 64), id16 = tc::idesc_bf16(128, 16);
  constexpr uint32_t idB64 = tc::idesc_bf16(128, 64, false, true);                  // B read MN-major
  constexpr uint32_t idT64 = tc::idesc_bf16(128, 64, true, true), idT16 = tc::idesc_bf16(128, 16, true, true);

  float lsum = 0.f, bs1 = 0.f, bs2 = 0.f, bs3 = 0.f, bs4[3] = {0.f, 0.f, 0.f};
  uint32_t phase = 0;
  bool failed = false, first = true;

  // Z = A W^T over K = 64 (four K = 16 steps) for a hidden tile A and weight tile W
  auto mma_forward64 = [&](uint32_t d, uint32_t a, uint32_t w, uint32_t idesc) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      tc::mma(tbase + d, tc::desc_k(a + 256 * k, 1024), tc::desc_k(w + 256 * k, 1024), idesc, k > 0 ? 1u : 0u);
  };
  // DA = Delta W over K = 64 output features: Delta = the half of the delta tile at
  // dl (K-major, SBO 2048), W = a 64 x 64 weight tile read MN-major
  auto mma_data_grad = [&](uint32_t dl, uint32_t w) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      tc::mma(tbase + TDA, tc::desc_k(dl + 256 * k, 2048), tc::desc_mn(w + 2048 * k, 1024), idB64, k > 0 ? 1u : 0u);
  };

  // one tcgen05 stage: operands written by every thread -> one thread issues and
  // commits -> every thread waits for the MMAs (bounded)
  auto stage = [&](int which) -> bool {
    fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t acc0 = first ? 0u : 1u;
      switch (which) {
        case 0:   // Z = X W1^T
          tc::mma(tbase + TZ, tc::desc_k(aX, 256), tc::desc_k(aW1, 256), id64, 0u);
          break;
        case 1:   // Z = A1 W2^T
          mma_forward64(TZ, aA1, aW2, id64);
          break;
        case 2:   // Z = A2 W3^T (kept as Z_3 for the backward pass)
          mma_forward64(TZ, aA2, aW3, id64);
          break;
        case 3:   // Y = A3 W4^T (in the DA columns)
          mma_forward64(TDA, aA3, aW4, id16);
          break;
        case 4:   // dW4^T += A3^T D4 ; DA = D4 W4
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            tc::mma(tbase + TW4, tc::desc_mn(aA3 + 2048 * kk, 1024), tc::desc_mn(aD4 + 512 * kk, 256), idT16,
                    (kk > 0) ? 1u : acc0);
          tc::mma(tbase + TDA, tc::desc_k(aD4, 256), tc::desc_mn(aW4, 1024), idB64, 0u);
          break;
        case 5:   // [dW3 | dW2] += [Delta_3 | 0]^T A2 ; DA = Delta_3 W3 ; Z = A1 W2^T (Z_2 again)
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            tc::mma(tbase + TW23, tc::desc_mn(aDL + 4096 * kk, 2048), tc::desc_mn(aA2 + 2048 * kk, 1024), idT64,
                    (kk > 0) ? 1u : acc0);
          mma_data_grad(aDL, aW3);
          mma_forward64(TZ, aA1, aW2, id64);
          break;
        case 6:   // [dW3 | dW2] += [0 | Delta_2]^T A1 ; DA = Delta_2 W2 ; Z = X W1^T (Z_1 again)
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            tc::mma(tbase + TW23, tc::desc_mn(aDL + 4096 * kk, 2048), tc::desc_mn(aA1 + 2048 * kk, 1024), idT64,
                    1u);
          mma_data_grad(aDL + 1024, aW2);
          tc::mma(tbase + TZ, tc::desc_k(aX, 256), tc::desc_k(aW1, 256), id64, 0u);
          break;
        default:  // dW1 += Delta_1^T X (rows 64..127: the stale second half, never read back)
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            tc::mma(tbase + TW1, tc::desc_mn(aDL + 4096 * kk, 2048), tc::desc_mn(aX + 512 * kk, 256), idT16,
                    (kk > 0) ? 1u : acc0);
          break;
      }
      tc::commit(bar);
    }
    const bool ok = mbar_wait(bar, phase, kMmaWaitCycles);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      return false;
    }
    tc::fence_after();
    return true;
  };

  // hidden layer l (0-based) forward epilogue: A = bf16(SiLU(Z + b)), this thread's half row
  auto epi_hidden = [&](int l, char* A) {
    float v[32];
    tc::ld32(tlane + TZ + c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = silu(v[j] + bias[64 * l + c0 + j]);
    store_row32(A, row, c0, v);
  };
  // backward epilogue of layer l: Delta = DA * SiLU'(Z + b) -> half `dh` of the delta
  // tile (bf16), the other half zeroed when `zero_other`; returns the float32 column
  // sum over the warp's rows (lane j: column c0 + j)
  auto epi_back = [&](int l, int dh, bool zero_other) -> float {
    uint32_t rd[32], rz[32];
    tc::ld32_nowait(tlane + TDA + c0, rd);
    tc::ld32_nowait(tlane + TZ + c0, rz);
    tc::wait_ld();
    float d[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = __uint_as_float(rd[j]) * dsilu(__uint_as_float(rz[j]) + bias[64 * l + c0 + j]);
    char* DL = smem + SM_DL;
    store_row32(DL + 1024 * dh, row, c0, d, 2048);
    if (zero_other) {
#pragma unroll
      for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4*>(DL + 1024 * (1 - dh) + tc::cm_off(row, c0 + 8 * g, 2048)) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    return transpose_sum32(d, lane);
  };

  const int64_t ntiles = (m + kRows - 1) / kRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t p = tile * kRows + row;
    if (half == 0) {
      uint4 f0 = make_uint4(0u, 0u, 0u, 0u), f1 = f0;
      if (p < m) {
        const uint4* src = reinterpret_cast<const uint4*>(feats + p * 16);
        f0 = src[0];
        f1 = src[1];
      }
      *reinterpret_cast<uint4*>(smem + SM_X + tc::cm_off(row, 0, 256)) = f0;
      *reinterpret_cast<uint4*>(smem + SM_X + tc::cm_off(row, 8, 256)) = f1;
    }
    if (!stage(0)) { failed = true; break; }
    epi_hidden(0, smem + SM_A1);
    if (!stage(1)) { failed = true; break; }
    epi_hidden(1, smem + SM_A2);
    if (!stage(2)) { failed = true; break; }
    epi_hidden(2, smem + SM_A3);
    if (!stage(3)) { failed = true; break; }
    if (half == 0) {  // output: loss, d4 = 2 (y - t) / count on masked rows, bf16 D4 row
      float y[4];
      tc::ld4(tlane + TDA, y);
      const bool valid = p < m && (!mask || mask[p]);
      float d4[3];
      const float4 t = valid ? tgt[p] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float tv[3] = {t.x, t.y, t.z};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float diff = valid ? (y[c] + bias[192 + c] - tv[c]) : 0.f;
        lsum += diff * diff;
        d4[c] = 2.f * diff * inv_cnt;
        bs4[c] += warp_sum(d4[c]);
      }
      *reinterpret_cast<uint4*>(smem + SM_D4 + tc::cm_off(row, 0, 256)) =
          make_uint4(pack2(d4[0], d4[1]), pack2(d4[2], 0.f), 0u, 0u);
      *reinterpret_cast<uint4*>(smem + SM_D4 + tc::cm_off(row, 8, 256)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (!stage(4)) { failed = true; break; }
    bs3 += epi_back(2, 0, true);
    if (!stage(5)) { failed = true; break; }
    bs2 += epi_back(1, 1, true);
    if (!stage(6)) { failed = true; break; }
    bs1 += epi_back(0, 0, false);
    if (!stage(7)) { failed = true; break; }
    first = false;
  }

  if (!failed) {
    float* out = partial + (size_t)blockIdx.x * kNP;
    // weight gradients: dW1 and dW4^T rows in lanes 0..63 (warps 0, 1), dW3 rows o in
    // lanes 0..63 and dW2 rows o in lanes 64..127 of the shared accumulator
    if ((warp & 3) < 2 && half == 0) {
      float v[16];
      tc::ld16(tlane + TW1, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) out[OFF_W1 + row * 16 + i] = first ? 0.f : v[i];
      float w4[4];
      tc::ld4(tlane + TW4, w4);
#pragma unroll
      for (int o = 0; o < 3; ++o) out[OFF_W4 + o * 64 + row] = first ? 0.f : w4[o];
    }
    {
      float v[32];
      tc::ld32(tlane + TW23 + c0, v);
      const int o = row & 63;
      float* dst = out + (row < 64 ? OFF_W3 : OFF_W2) + o * 64 + c0;
#pragma unroll
      for (int i = 0; i < 32; ++i) dst[i] = first ? 0.f : v[i];
    }
    // bias gradients: lane l of warp w holds column 32 (w / 4) + l summed over its rows
    float* red = reinterpret_cast<float*>(smem + SM_RED);
    red[(0 * 8 + warp) * 32 + lane] = bs1;
    red[(1 * 8 + warp) * 32 + lane] = bs2;
    red[(2 * 8 + warp) * 32 + lane] = bs3;
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) red[8 * 32 * 3 + warp * 4 + c] = bs4[c];
    }
    const float ls = warp_sum(lsum);
    if (lane == 0) red[8 * 32 * 3 + 8 * 4 + warp] = ls;
    __syncthreads();
    if (tid < 192) {
      const int l = tid / 64, col = tid % 64, h = col / 32;
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < 4; ++w) s += red[(l * 8 + 4 * h + w) * 32 + (col & 31)];
      const int off = l == 0 ? OFF_B1 : (l == 1 ? OFF_B2 : OFF_B3);
      out[off + col] = s;
    } else if (tid < 195) {
      const int c = tid - 192;
      float s = 0.f;
      for (int w = 0; w < 4; ++w) s += red[8 * 32 * 3 + w * 4 + c];
      out[OFF_B4 + c] = s;
    } else if (tid == 195) {
      float s = 0.f;
      for (int w = 0; w < 8; ++w) s += red[8 * 32 * 3 + 8 * 4 + w];
      loss_part[blockIdx.x] = s;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::dealloc(tbase, kTmemCols);
  }
}

}  // namespace

// per-block partial gradients [blocks][9603] and losses [blocks] of the network M
// over m rows, on tensor cores; blocks <= number of 128-row tiles; *err (device) is
// set when a wait on the tensor cores gave up
sph_status mlp_grad_tc(const sph_mlp* M, const __nv_bfloat16* feats, const float4* tgt, const uint8_t* mask,
                       int64_t m, float inv_cnt, float* partial, float* loss_part, int* err, int blocks,
                       cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    SPH_TRY_CUDA(cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn));
    attr_set = true;
  }
  size_t ow1, ow2, ow3, ow4, ob;
  mlp_pack_layout(&ow1, &ow2, &ow3, &ow4, &ob);
  SPH_LAUNCH(k_mlp_grad_tc, blocks, kThreads, kSmemDyn, st)(
      reinterpret_cast<const char*>(mlp_pack_ptr(M)), (int64_t)ow1, (int64_t)ow2, (int64_t)ow3, (int64_t)ow4,
      (int64_t)ob, feats, tgt, mask, m, inv_cnt, partial, loss_part, err);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

// grid of the training kernel: one CTA per 128-row tile, at most two per SM
int64_t mlp_grad_blocks(int64_t m, int num_sms) {
  int64_t blocks = (m + kRows - 1) / kRows;
  if (blocks > 2 * (int64_t)num_sms) blocks = 2 * (int64_t)num_sms;
  return blocks < 1 ? 1 : blocks;
}

}  // namespace sph
