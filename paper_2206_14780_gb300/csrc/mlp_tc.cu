// Warm-start network forward on the 5th-generation tensor cores (tcgen05).
//
// One CTA of 4 warps runs 128 particles per tile through the 16-64-64-64-3 MLP:
// every layer is one tcgen05.mma chain D[128 x N] = A[128 x K] B[K x N] with
// A (the tile's features or hidden activations) and B (a weight matrix) in
// shared memory as bf16 and D (float32) in tensor memory; one elected thread
// issues the MMAs and commits them to an mbarrier.  Between layers each warp
// reads its 32 rows of D back with tcgen05.ld, adds the bias, applies SiLU,
// rounds to bf16 and writes the next layer's A operand.  The rounding points
// are those of the float64 reference (inputs, weights and hidden activations in
// bf16; float32 accumulation; biases in float32).
//
// Shared-memory operands use the no-swizzle K-major "core matrix" layout of the
// tcgen05 matrix descriptors: 8 rows x 16 bytes (8 bf16) per 128-byte core
// matrix; core matrices adjacent along K are LBO = 128 bytes apart and 8-row
// groups SBO bytes apart (SBO = 16 * K bytes).  An MMA consumes K = 16, i.e. two
// core matrices along K, so the k-th chunk's descriptor starts 256 k bytes in.
//
// Tensor memory: 64 columns per CTA (D of every layer in columns 0-63; layer 4
// uses 0-15 after layer 3's epilogue has read them).  The dynamic shared-memory
// request (44 KB) keeps at most five CTAs on an SM, so their 320 columns never
// exceed the SM's 512 and tcgen05.alloc never waits.  Waits on the MMA mbarrier are bounded; on a timeout the kernel
// sets *err, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "bulk.cuh"
#include "sph_internal.cuh"

namespace sph {

struct MlpPack;
const void* mlp_pack_ptr(const sph_mlp* M);
void mlp_pack_layout(size_t* off_w1, size_t* off_w2, size_t* off_w3, size_t* off_w4, size_t* off_b);

namespace {

constexpr int kTile = 128;
constexpr int kTmemCols = 64;
constexpr int kSmemDyn = 44 * 1024;
constexpr long long kMmaWaitCycles = 4000000000ll;

// shared-memory map (bytes from the dynamic base, 1024-aligned pieces)
constexpr int SM_W1 = 0;                 // 64 x 16   bf16, SBO 256
constexpr int SM_W2 = SM_W1 + 2048;      // 64 x 64   bf16, SBO 1024
constexpr int SM_W3 = SM_W2 + 8192;      // 64 x 64
constexpr int SM_W4 = SM_W3 + 8192;      // 16 x 64 (rows 3..15 zero)
constexpr int SM_X = SM_W4 + 2048;       // 128 x 16  bf16, SBO 256
constexpr int SM_H = SM_X + 4096;        // 128 x 64  bf16, SBO 1024
constexpr int SM_B = SM_H + 16384;       // biases: 64 + 64 + 64 + 4 float
constexpr int SM_BAR = SM_B + 784;       // mbarrier (8 B) + tensor-memory address (4 B)
constexpr int SM_END = SM_BAR + 16;
static_assert(SM_END <= kSmemDyn, "shared-memory map exceeds the request");

// byte offset of element (row, k) in a core-matrix K-major operand
__device__ __forceinline__ int cm_off(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((128u >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D float32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive float32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float v[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
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
    tc_ld32(tbase + ((uint32_t)(32 * warp) << 16) + 32 * half, v);
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
      *reinterpret_cast<uint4*>(H + cm_off(row, 32 * half + 8 * g, 1024)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void __launch_bounds__(kTile) k_mlp_forward_tc(const char* __restrict__ pack, int64_t off_w1,
                                                          int64_t off_w2, int64_t off_w3, int64_t off_w4,
                                                          int64_t off_b, const __nv_bfloat16* __restrict__ feats,
                                                          int64_t m, float4* __restrict__ out, int* err) {
  extern __shared__ __align__(1024) char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM_BAR + 8);
  float* bias = reinterpret_cast<float*>(smem + SM_B);

  // weights into the core-matrix layout (16-byte chunks of 8 bf16 along K)
  for (int i = tid; i < 64 * 2; i += kTile) {               // W1: 64 rows x 2 chunks
    const int n = i >> 1, c = i & 1;
    *reinterpret_cast<uint4*>(smem + SM_W1 + cm_off(n, 8 * c, 256)) =
        *reinterpret_cast<const uint4*>(pack + off_w1 + (size_t)(n * 16 + 8 * c) * 2);
  }
  for (int i = tid; i < 64 * 8; i += kTile) {               // W2, W3: 64 rows x 8 chunks
    const int n = i >> 3, c = i & 7;
    *reinterpret_cast<uint4*>(smem + SM_W2 + cm_off(n, 8 * c, 1024)) =
        *reinterpret_cast<const uint4*>(pack + off_w2 + (size_t)(n * 64 + 8 * c) * 2);
    *reinterpret_cast<uint4*>(smem + SM_W3 + cm_off(n, 8 * c, 1024)) =
        *reinterpret_cast<const uint4*>(pack + off_w3 + (size_t)(n * 64 + 8 * c) * 2);
  }
  for (int i = tid; i < 16 * 8; i += kTile) {               // W4: 16 rows (3 used) x 8 chunks
    const int n = i >> 3, c = i & 7;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (n < 3) w = *reinterpret_cast<const uint4*>(pack + off_w4 + (size_t)(n * 64 + 8 * c) * 2);
    *reinterpret_cast<uint4*>(smem + SM_W4 + cm_off(n, 8 * c, 1024)) = w;
  }
  for (int i = tid; i < 196; i += kTile)
    bias[i] = *reinterpret_cast<const float*>(pack + off_b + (size_t)i * 4);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbarrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  const uint32_t aX = smem_addr(smem + SM_X), aH = smem_addr(smem + SM_H);
  const uint32_t aW1 = smem_addr(smem + SM_W1), aW2 = smem_addr(smem + SM_W2), aW3 = smem_addr(smem + SM_W3),
                 aW4 = smem_addr(smem + SM_W4);
  constexpr uint32_t id64 = idesc_bf16(128, 64), id16 = idesc_bf16(128, 16);
  uint32_t phase = 0;
  bool failed = false;
  const int64_t ntiles = (m + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t p = tile * kTile + tid;
    // features of this thread's particle -> X (two 16-byte chunks)
    uint4 f0 = make_uint4(0u, 0u, 0u, 0u), f1 = f0;
    if (p < m) {
      const uint4* src = reinterpret_cast<const uint4*>(feats + p * 16);
      f0 = src[0];
      f1 = src[1];
    }
    *reinterpret_cast<uint4*>(smem + SM_X + cm_off(tid, 0, 256)) = f0;
    *reinterpret_cast<uint4*>(smem + SM_X + cm_off(tid, 8, 256)) = f1;
    for (int layer = 0; layer < 4 && !failed; ++layer) {
      fence_proxy_async();     // this thread's operand writes -> the tensor cores
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        if (layer == 0) {
          tc_mma(tbase, smem_desc(aX, 256), smem_desc(aW1, 256), id64, 0u);
        } else {
          const uint32_t aW = layer == 1 ? aW2 : (layer == 2 ? aW3 : aW4);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc_mma(tbase, smem_desc(aH + 256 * k, 1024), smem_desc(aW + 256 * k, 1024),
                   layer == 3 ? id16 : id64, k > 0 ? 1u : 0u);
        }
        tc_commit(bar);
      }
      const bool ok = mbar_wait(bar, phase, kMmaWaitCycles);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      if (layer < 3) {
        epilogue_hidden(tbase, warp, tid, bias + 64 * layer, smem + SM_H);
      } else {
        float v[4];
        tc_ld4(tbase + ((uint32_t)(32 * warp) << 16), v);
        if (p < m) out[p] = make_float4(v[0] + bias[192], v[1] + bias[193], v[2] + bias[194], 0.f);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
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
  int64_t blocks = (m + kTile - 1) / kTile;
  const int64_t cap = (int64_t)num_sms * 5;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  SPH_LAUNCH(k_mlp_forward_tc, (int)blocks, kTile, kSmemDyn, st)(reinterpret_cast<const char*>(mlp_pack_ptr(M)),
                                                                 (int64_t)ow1, (int64_t)ow2, (int64_t)ow3,
                                                                 (int64_t)ow4, (int64_t)ob, feats, m, out, err);
  SPH_TRY_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // namespace sph
