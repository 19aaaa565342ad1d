// Batch launches of the ray caster (many views, one persistent launch) and
// the longest-first tile schedule built from the costs a previous launch
// recorded.
#include "ro_render_kernel.cuh"

namespace ro {
namespace {

// Log-scale bucket of a tile cost: exact below 8, then 8 buckets per octave
// (monotone in the cost, 240 buckets for 32-bit costs).
__device__ __forceinline__ int cost_bucket(uint32_t c) {
  if (c < 8u) return (int)c;
  const int e = 31 - __clz((int)c);
  return (e - 2) * 8 + (int)((c >> (e - 3)) & 7u);
}

constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 256;

// One block: histogram of the buckets, offsets from the most expensive
// bucket down, then every tile placed at its bucket's next position.  A
// tile's cost is the sum over its parts (the bands of rows warps refill
// with).  The order within a bucket is whatever the shared-memory counters
// give: any order renders the same images, only the launch's tail changes.
__global__ void __launch_bounds__(kOrderThreads) cost_order_kernel(const uint32_t* __restrict__ cost, uint32_t n,
                                                                  uint32_t* __restrict__ order) {
  __shared__ uint32_t s_hist[kOrderBuckets];
  __shared__ uint32_t s_off[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_hist[b] = 0;
  __syncthreads();
  auto tile_cost = [&](uint32_t t) {
    uint32_t c = 0;
    for (int p = 0; p < kTileParts; ++p) c += __ldg(cost + (size_t)t * kTileParts + p);
    return c;
  };
  for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) atomicAdd(&s_hist[cost_bucket(tile_cost(t))], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {
      s_off[b] = run;
      run += s_hist[b];
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
    const uint32_t pos = atomicAdd(&s_off[cost_bucket(tile_cost(t))], 1u);
    order[pos] = t;
  }
}

}  // namespace

cudaError_t launch_render_batch(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  if (a.g.sf != 0) return launch_render_batch_lp(a, debug, s, blocks_out);
  return launch_any<true, 0>(a, debug, s, blocks_out);
}

cudaError_t launch_cost_order(const uint32_t* cost, uint32_t n_tiles, uint32_t* order, cudaStream_t s) {
  cost_order_kernel<<<1, kOrderThreads, 0, s>>>(cost, n_tiles, order);
  return cudaGetLastError();
}

}  // namespace ro
