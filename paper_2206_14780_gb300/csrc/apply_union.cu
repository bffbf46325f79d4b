// Per-slice neighbour unions for the shared-memory apply form.
//
// The 32 rows of a SELL slice are consecutive along the Morton cell order, so
// they share most of their neighbours: on the lava boxes a slice's ~2,400
// stored entries reference ~350 distinct rows.  For every slice this set-up
// lists those distinct rows once (sorted, in `uni`, at the slice's own offset
// of the operator storage) and rewrites each entry as (position in that list,
// coefficient) in `op_loc`, so the apply can gather each neighbour vector into
// shared memory once per slice and read it from there for every entry.  A
// slice whose union exceeds kUnionCap is marked -1 in `unum` and keeps the
// global-gather path.
//
// One block per slice (grid-stride): the slice's valid entries are loaded into
// shared memory, sorted by a bitonic network, deduplicated with a block scan,
// and every entry's column is found in the sorted union by binary search.
#include <climits>

#include "apply.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kUB = 256;           // threads per set-up block
constexpr int kUMax = 4096;        // entries per slice: 32 rows x at most 128 neighbours

__global__ void __launch_bounds__(kUB) k_union_build(OpView op, int64_t nslices, int32_t* __restrict__ uni,
                                                     int32_t* __restrict__ unum, int2* __restrict__ op_loc) {
  __shared__ int32_t key[kUMax];
  __shared__ int32_t uk[kUMax];
  __shared__ int32_t wsum[kUB / 32];
  __shared__ int32_t total;
  const int tid = threadIdx.x;
  for (int64_t sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
    const int64_t o0 = op.off[sl];
    const int E = (int)(op.off[sl + 1] - o0);          // 32 x slice width
    if (E > kUMax) {                                   // wider than any list allows: global path
      if (tid == 0) unum[sl] = -1;
      continue;
    }
    int P = 32;
    while (P < E) P <<= 1;
    for (int i = tid; i < P; i += kUB) {
      int32_t k = INT_MAX;
      if (i < E) {
        const int r = i & 31, j = i >> 5;
        if (j < op.cnt[sl * kSlice + r]) k = op.ih[o0 + i].x;
      }
      key[i] = k;
    }
    __syncthreads();
    // bitonic sort of key[0..P)
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = tid; i < P; i += kUB) {
          const int pj = i ^ stride;
          if (pj > i) {
            const bool up = (i & size) == 0;
            const int32_t a = key[i], b = key[pj];
            if ((a > b) == up) {
              key[i] = b;
              key[pj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    // distinct valid keys: count per thread over a contiguous chunk, block scan, write
    const int per = P / kUB > 0 ? P / kUB : 1;
    const int b0 = tid * per;
    int cnt = 0;
    for (int i = b0; i < b0 + per && i < P; ++i) {
      const int32_t k = key[i];
      if (k != INT_MAX && (i == 0 || key[i - 1] != k)) ++cnt;
    }
    // exclusive scan of cnt over the block
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < kUB / 32; ++w) {
        const int t = wsum[w];
        wsum[w] = acc;
        acc += t;
      }
      total = acc;
    }
    __syncthreads();
    int pos = wsum[warp] + incl - cnt;
    for (int i = b0; i < b0 + per && i < P; ++i) {
      const int32_t k = key[i];
      if (k != INT_MAX && (i == 0 || key[i - 1] != k)) {
        uk[pos] = k;
        uni[o0 + pos] = k;
        ++pos;
      }
    }
    __syncthreads();
    const int nu = total;
    if (tid == 0) unum[sl] = nu <= kUnionCap ? nu : -1;
    // entries -> (position in the union, coefficient)
    for (int i = tid; i < E; i += kUB) {
      const int r = i & 31, j = i >> 5;
      int2 out = make_int2(0, 0);
      if (j < op.cnt[sl * kSlice + r]) {
        const int2 e = op.ih[o0 + i];
        int lo = 0, hi = nu;                 // first position with uk[pos] >= e.x
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (uk[mid] < e.x) lo = mid + 1;
          else hi = mid;
        }
        out = make_int2(lo, e.y);
      }
      op_loc[o0 + i] = out;
    }
    __syncthreads();
  }
}

}  // namespace

sph_status ensure_union(sph_neighbors* H, cudaStream_t st) {
  if (H->union_valid && H->union_op_version == H->op_version) return SPH_OK;
  const int64_t nnz = H->op_nnz_pad > 0 ? H->op_nnz_pad : 1;
  SPH_TRY(H->op_loc.alloc(nnz));
  SPH_TRY(H->uni.alloc(nnz));
  SPH_TRY(H->unum.alloc(H->nslices > 0 ? H->nslices : 1));
  if (H->nslices > 0) {
    int grid = H->num_sms * 8;
    if (grid > H->nslices) grid = (int)H->nslices;
    SPH_LAUNCH(k_union_build, grid, kUB, 0, st)(op_view(H), H->nslices, H->uni.p, H->unum.p, H->op_loc.p);
    SPH_TRY_CUDA(cudaGetLastError());
  }
  H->union_valid = true;
  H->union_op_version = H->op_version;
  return SPH_OK;
}

}  // namespace sph
