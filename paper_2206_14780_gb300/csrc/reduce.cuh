// Grid-wide float64 reductions without an extra launch.
//
// Every thread carries K float32 partial sums of its rows.  A warp folds them
// with shuffles in float32 (32 terms), the block folds its warps in float64 (a
// shuffle tree) and writes one float64 partial per value; the last block to
// arrive (a ticket on a global counter after a memory fence) folds all block
// partials in a fixed order, so the result is deterministic, and runs the
// scalar update.  Float64 runs at a small fraction of the float32 rate on this
// part, so the number of dependent float64 additions in that serial tail is
// kept small.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// out[k] = sum over the W warps of sm[w][k] (k < K), as a shuffle tree inside
// groups of W consecutive lanes: log2(W) dependent float64 additions instead of
// W - 1.  Every thread of the block calls it (the first warps do the work).
template <int K, int W>
__device__ __forceinline__ void cross_warp_sum(const double (*sm)[K > 0 ? K : 1], double* __restrict__ out) {
  constexpr int N = K * W;
  constexpr int NT = (N + 31) / 32 * 32;
  static_assert(32 % W == 0, "W must divide the warp");
  const int t = threadIdx.x;
  if (t < NT) {
    double x = t < N ? sm[t % W][t / W] : 0.0;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (t < N && t % W == 0) out[t / W] = x;
  }
}

template <int K, int NB = kBlock>
__device__ __forceinline__ void block_partials(const float (&v)[K], double* __restrict__ out) {
  __shared__ double sm[NB / 32][K > 0 ? K : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[warp][k] = (double)x;
  }
  __syncthreads();
  cross_warp_sum<K, NB / 32>(sm, out);
}

template <int K>
__device__ __forceinline__ void block_partials_f64(const double (&v)[K], double* __restrict__ out) {
  __shared__ double sm[kBlock / 32][K > 0 ? K : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[warp][k] = x;
  }
  __syncthreads();
  cross_warp_sum<K, kBlock / 32>(sm, out);
}

// True in every thread of the last block to finish (after its partial is stored).
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ unsigned int ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  return ticket == gridDim.x - 1;
}

// Sum of all block partials (called by every thread of the last block); the
// result is left in res[0..K) in shared memory; the counter is re-armed.
template <int K>
__device__ __forceinline__ void final_sum(const double* partials, unsigned int* counter, double* res) {
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + (size_t)b * kMaxDots + k);
  }
  __shared__ double sm[kBlock / 32][K > 0 ? K : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[warp][k] = x;
  }
  __syncthreads();
  cross_warp_sum<K, kBlock / 32>(sm, res);
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
}

}  // namespace sph
