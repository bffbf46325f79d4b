// Warm-start network forward on the 5th-generation tensor cores (tcgen05).
//
// A group of 4 warps runs 128 particles per tile through the 16-64-64-64-3 MLP:
// every layer is one tcgen05.mma chain D[128 x N] = A[128 x K] B[K x N] with
// A (the tile's features or hidden activations) and B (a weight matrix) in
// shared memory as bf16 and D (float32) in tensor memory; one elected thread of
// the group issues the MMAs and commits them to the group's mbarrier.  Between
// layers each warp reads its 32 rows of D back with tcgen05.ld, adds the bias,
// applies SiLU, rounds to bf16 and writes the next layer's A operand.  The
// rounding points are those of the float64 reference (inputs, weights and hidden
// activations in bf16; float32 accumulation; biases in float32).
//
// One CTA per SM holds the weights once and kGroups = 8 such groups, each with
// its own tile, operand buffers, mbarrier, named barrier and 64 tensor-memory
// columns (all 512 of the SM), so eight tiles are in flight per SM and one
// group's epilogue overlaps the others' MMAs and transcendentals.  (Four-warp
// CTAs with a weight copy each were capped at five per SM by shared memory.)
//
// Shared-memory operands use the no-swizzle K-major "core matrix" layout of the
// tcgen05 matrix descriptors: 8 rows x 16 bytes (8 bf16) per 128-byte core
// matrix; core matrices adjacent along K are LBO = 128 bytes apart and 8-row
// groups SBO bytes apart (SBO = 16 * K bytes).  An MMA consumes K = 16, i.e. two
// core matrices along K, so the k-th chunk's descriptor starts 256 k bytes in.
//
// Waits on a group's mbarrier are bounded; on a timeout the group sets *err and
// stops, and the CTA frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "sph_internal.cuh"
#include "tcgen05.cuh"

namespace sph {

struct MlpPack;
const void* mlp_pack_ptr(const sph_mlp* M);
void mlp_pack_layout(size_t* off_w1, size_t* off_w2, size_t* off_w3, size_t* off_w4, size_t* off_b);

namespace {

constexpr int kTile = 128;
constexpr int kGroups = 8;                  // tiles in flight per CTA (one CTA per SM)
constexpr int kThreads = kTile * kGroups;   // 1024
constexpr int kTmemCols = 64 * kGroups;     // 512: the whole tensor memory of the SM
constexpr long long kMmaWaitCycles = 4000000000ll;

// shared-memory map (bytes from the dynamic base, 1024-aligned pieces)
constexpr int SM_W1 = 0;                 // 64 x 16   bf16, SBO 256
constexpr int SM_W2 = SM_W1 + 2048;      // 64 x 64   bf16, SBO 1024
constexpr int SM_W3 = SM_W2 + 8192;      // 64 x 64
constexpr int SM_W4 = SM_W3 + 8192;      // 16 x 64 (rows 3..15 zero)
constexpr int SM_B = SM_W4 + 2048;       // biases: 64 + 64 + 64 + 4 float
constexpr int SM_BAR = SM_B + 1024;      // kGroups mbarriers (8 B each) + tensor-memory address (4 B)
constexpr int SM_G0 = SM_BAR + 1024;     // per group: X (128 x 16 bf16, SBO 256) then H (128 x 64, SBO 1024)
constexpr int SM_GSTRIDE = 4096 + 16384;
constexpr int kSmemDyn = SM_G0 + kGroups * SM_GSTRIDE;
static_assert(kSmemDyn <= 227 * 1024, "shared-memory map exceeds the per-CTA limit");
static_assert(196 * 4 <= SM_BAR - SM_B && 8 * kGroups + 4 <= SM_G0 - SM_BAR, "shared-memory map overlaps");

// barrier among the 128 threads of group g (named barrier 1 + g)
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kTile) : "memory");
}
// the same, returning whether any of the group's threads passed v = true
__device__ __forceinline__ bool group_sync_or(int g, bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.s32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, %3, pi;\n\t"
      "selp.s32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(v ? 1 : 0), "r"(1 + g), "r"(kTile)
      : "memory");
  return r != 0;
}

// z sigmoid(z) = h (1 + tanh h), h = z / 2, with the hardware tanh of the PTX
// instruction tanh.approx.f32: one transcendental per activation instead of an
// exponential and a reciprocal, which halves the epilogue's load on the
// transcendental pipe.  Its absolute error (about 5e-4 in tanh, so 2.5e-4 |z| in
// SiLU) stays below the bf16 rounding of the activation that follows for the
// activations that carry the layer's output.
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu_tc(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_hw(h), h);
}

// D (columns 0..63 of this thread's row) + bias -> SiLU -> bf16 -> H (A operand)
__device__ __forceinline__ void epilogue_hidden(uint32_t tbase, int warp, int row, const float* bias, char* H) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float v[32];
    tc::ld32(tbase + ((uint32_t)(32 * warp) << 16) + 32 * half, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 32 * half + 8 * g + 2 * q;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(silu_tc(v[8 * g + 2 * q] + bias[c]),
                                                        silu_tc(v[8 * g + 2 * q + 1] + bias[c + 1]));
        w[q] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      *reinterpret_cast<uint4*>(H + tc::cm_off(row, 32 * half + 8 * g, 1024)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward_tc(const char* __restrict__ pack, int64_t off_w1,
                                                                int64_t off_w2, int64_t off_w3, int64_t off_w4,
                                                                int64_t off_b, const __nv_bfloat16* __restrict__ feats,
                                                                int64_t m, float4* __restrict__ out, int* err) {
  extern __shared__ __align__(1024) char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = warp >> 2, gtid = tid & (kTile - 1), gw = warp & 3;   // group, thread and warp in it
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SM_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM_BAR + 8 * kGroups);
  float* bias = reinterpret_cast<float*>(smem + SM_B);

  // weights into the core-matrix layout (16-byte chunks of 8 bf16 along K), once per CTA
  for (int i = tid; i < 64 * 2; i += kThreads) {            // W1: 64 rows x 2 chunks
    const int n = i >> 1, c = i & 1;
    *reinterpret_cast<uint4*>(smem + SM_W1 + tc::cm_off(n, 8 * c, 256)) =
        *reinterpret_cast<const uint4*>(pack + off_w1 + (size_t)(n * 16 + 8 * c) * 2);
  }
  for (int i = tid; i < 64 * 8; i += kThreads) {            // W2, W3: 64 rows x 8 chunks
    const int n = i >> 3, c = i & 7;
    *reinterpret_cast<uint4*>(smem + SM_W2 + tc::cm_off(n, 8 * c, 1024)) =
        *reinterpret_cast<const uint4*>(pack + off_w2 + (size_t)(n * 64 + 8 * c) * 2);
    *reinterpret_cast<uint4*>(smem + SM_W3 + tc::cm_off(n, 8 * c, 1024)) =
        *reinterpret_cast<const uint4*>(pack + off_w3 + (size_t)(n * 64 + 8 * c) * 2);
  }
  for (int i = tid; i < 16 * 8; i += kThreads) {            // W4: 16 rows (3 used) x 8 chunks
    const int n = i >> 3, c = i & 7;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (n < 3) w = *reinterpret_cast<const uint4*>(pack + off_w4 + (size_t)(n * 64 + 8 * c) * 2);
    *reinterpret_cast<uint4*>(smem + SM_W4 + tc::cm_off(n, 8 * c, 1024)) = w;
  }
  for (int i = tid; i < 196; i += kThreads) bias[i] = *reinterpret_cast<const float*>(pack + off_b + (size_t)i * 4);
  if (tid < kGroups) {
    mbar_init(bars + tid, 1);
    fence_mbarrier_init();
  }
  if (warp == 0) tc::alloc(tslot, kTmemCols);
  fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tcol = *tslot + 64u * g;   // this group's 64 columns
  uint64_t* bar = bars + g;
  char* X = smem + SM_G0 + g * SM_GSTRIDE;
  char* H = X + 4096;

  const uint32_t aX = smem_addr(X), aH = smem_addr(H);
  const uint32_t aW1 = smem_addr(smem + SM_W1), aW2 = smem_addr(smem + SM_W2), aW3 = smem_addr(smem + SM_W3),
                 aW4 = smem_addr(smem + SM_W4);
  constexpr uint32_t id64 = tc::idesc_bf16(128, 64), id16 = tc::idesc_bf16(128, 16);
  uint32_t phase = 0;
  const int64_t ntiles = (m + kTile - 1) / kTile;
  for (int64_t tile = (int64_t)blockIdx.x * kGroups + g; tile < ntiles; tile += (int64_t)gridDim.x * kGroups) {
    const int64_t p = tile * kTile + gtid;
    // features of this thread's particle -> X (two 16-byte chunks)
    uint4 f0 = make_uint4(0u, 0u, 0u, 0u), f1 = f0;
    if (p < m) {
      const uint4* src = reinterpret_cast<const uint4*>(feats + p * 16);
      f0 = src[0];
      f1 = src[1];
    }
    *reinterpret_cast<uint4*>(X + tc::cm_off(gtid, 0, 256)) = f0;
    *reinterpret_cast<uint4*>(X + tc::cm_off(gtid, 8, 256)) = f1;
    bool failed = false;
    for (int layer = 0; layer < 4; ++layer) {
      fence_proxy_async();     // this thread's operand writes -> the tensor cores
      tc::fence_before();
      group_sync(g);
      if (gtid == 0) {
        tc::fence_after();
        if (layer == 0) {
          tc::mma(tcol, tc::desc_k(aX, 256), tc::desc_k(aW1, 256), id64, 0u);
        } else {
          const uint32_t aW = layer == 1 ? aW2 : (layer == 2 ? aW3 : aW4);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma(tcol, tc::desc_k(aH + 256 * k, 1024), tc::desc_k(aW + 256 * k, 1024),
                    layer == 3 ? id16 : id64, k > 0 ? 1u : 0u);
        }
        tc::commit(bar);
      }
      const bool ok = mbar_wait(bar, phase, kMmaWaitCycles);
      phase ^= 1u;
      if (group_sync_or(g, !ok)) {
        failed = true;
        if (gtid == 0) atomicExch(err, 1);
        break;
      }
      tc::fence_after();
      if (layer < 3) {
        epilogue_hidden(tcol, gw, gtid, bias + 64 * layer, H);
      } else {
        float v[4];
        tc::ld4(tcol + ((uint32_t)(32 * gw) << 16), v);
        if (p < m) out[p] = make_float4(v[0] + bias[192], v[1] + bias[193], v[2] + bias[194], 0.f);
      }
    }
    if (failed) break;
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::dealloc(*tslot, kTmemCols);
  }
}

}  // namespace

// out[m][4] = (delta, 0) for the network M on tensor cores; *err (device) is
// set when a wait on the tensor cores gave up
sph_status mlp_forward_tc(const sph_mlp* M, const __nv_bfloat16* feats, int64_t m, float4* out, int* err,
                          int num_sms, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    SPH_TRY_CUDA(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn));
    attr_set = true;
  }
  size_t ow1, ow2, ow3, ow4, ob;
  mlp_pack_layout(&ow1, &ow2, &ow3, &ow4, &ob);
  int64_t blocks = ((m + kTile - 1) / kTile + kGroups - 1) / kGroups;
  if (blocks > num_sms) blocks = num_sms;   // one CTA per SM: it takes all of the SM's tensor memory
  if (blocks < 1) blocks = 1;
  SPH_LAUNCH(k_mlp_forward_tc, (int)blocks, kThreads, kSmemDyn, st)(reinterpret_cast<const char*>(mlp_pack_ptr(M)),
                                                                 (int64_t)ow1, (int64_t)ow2, (int64_t)ow3,
                                                                 (int64_t)ow4, (int64_t)ob, feats, m, out, err);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
