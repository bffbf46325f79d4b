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

// Sums of K float64 values over the 32 lanes of a warp at once, by a transposing
// butterfly: with P the power of two >= K, each of the first log2(P) levels
// hands half of a lane's remaining values to its partner and adds the other
// half, so a lane ends with one value (the sum over the lanes that differ in
// those bits); the remaining levels are plain shuffle additions.  That is
// P - 1 + 5 - log2(P) float64 additions per lane instead of 5 K.  Returns the
// lane's total and sets `index` to the value it holds; only lanes whose low
// 5 - log2(P) bits are zero hold a finished total (index < K: a real value).
template <int K>
__device__ __forceinline__ double warp_sum_multi(const double (&in)[K], int& index) {
  constexpr int P = K <= 1 ? 1 : (K <= 2 ? 2 : (K <= 4 ? 4 : (K <= 8 ? 8 : (K <= 16 ? 16 : 32))));
  constexpr int LP = P == 1 ? 0 : (P == 2 ? 1 : (P == 4 ? 2 : (P == 8 ? 3 : (P == 16 ? 4 : 5))));
  const int lane = threadIdx.x & 31;
  double v[P];
#pragma unroll
  for (int i = 0; i < P; ++i) v[i] = i < K ? in[i] : 0.0;
  int idx = 0;
#pragma unroll
  for (int L = 0; L < LP; ++L) {
    const int o = 16 >> L, c = P >> (L + 1);
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < c; ++i) {
      const double send = hi ? v[i] : v[i + c];
      const double keep = hi ? v[i + c] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (hi) idx += c;
  }
#pragma unroll
  for (int o = 16 >> LP; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  index = idx;
  return v[0];
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
  {
    constexpr int P = K <= 1 ? 1 : (K <= 2 ? 2 : (K <= 4 ? 4 : (K <= 8 ? 8 : (K <= 16 ? 16 : 32))));
    int idx;
    const double x = warp_sum_multi<K>(v, idx);
    if ((lane & (32 / P - 1)) == 0 && idx < K) sm[warp][idx] = x;
  }
  __syncthreads();
  cross_warp_sum<K, kBlock / 32>(sm, out);
}

// Pulls the solver scalars (written by earlier kernels, read by the scalar
// update at the end of the last block's tail) into L1 while the final sum runs,
// so the update's dependent loads do not each wait for L2.
__device__ __forceinline__ void prefetch_scalars(const void* S, size_t bytes) {
  const int i = threadIdx.x;
  if ((size_t)i * 128 < bytes)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(S) + 128 * i));
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
  // The first kRounds rounds of partials (all of them up to kRounds x the block
  // size) are loaded before any is added, so their L2 latencies overlap; a
  // round past the grid adds an exact zero, so the sums are those of the plain
  // loop, in the same order.
  constexpr int kRounds = 3;
  {
    double q[kRounds][K];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int b = threadIdx.x + r * blockDim.x;
#pragma unroll
      for (int k = 0; k < K; ++k) q[r][k] = b < (int)gridDim.x ? __ldcg(partials + (size_t)b * kMaxDots + k) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += q[r][k];
    }
  }
  for (int b = threadIdx.x + kRounds * blockDim.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + (size_t)b * kMaxDots + k);
  }
  __shared__ double sm[kBlock / 32][K > 0 ? K : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    constexpr int P = K <= 1 ? 1 : (K <= 2 ? 2 : (K <= 4 ? 4 : (K <= 8 ? 8 : (K <= 16 ? 16 : 32))));
    int idx;
    const double x = warp_sum_multi<K>(acc, idx);
    if ((lane & (32 / P - 1)) == 0 && idx < K) sm[warp][idx] = x;
  }
  __syncthreads();
  cross_warp_sum<K, kBlock / 32>(sm, res);
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
}

}  // namespace sph
