// Request and usage compaction (Sec. 4: the per-frame request list with a
// global limit keeps the device-to-host copy small; Sec. 5.3: usage stamps
// drive LRU eviction).
//
// Three passes over a byte-flag array, no atomics: (1) one count per 4096-flag
// tile, (2) one block turns the tile counts into exclusive offsets, (3) every
// tile re-reads its flags, ranks them with a warp shuffle scan plus a block
// scan of the warp totals, writes the IDs that fall below the capacity in
// ascending flag order, and clears the flags.
#include "ro_internal.h"

namespace ro {
namespace {

__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t v) {
  // 1 in the low bit of every non-zero byte
  const uint32_t t = (v | (v >> 1) | (v >> 2) | (v >> 3) | (v >> 4) | (v >> 5) | (v >> 6) | (v >> 7)) & 0x01010101u;
  return t;
}

__device__ __forceinline__ uint32_t count16(const uint4& v) {
  return __popc(nonzero_bytes(v.x)) + __popc(nonzero_bytes(v.y)) + __popc(nonzero_bytes(v.z)) +
         __popc(nonzero_bytes(v.w));
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  uint32_t tot = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kCompactThreads / 32; ++w) tot += s_warp[w];
  return tot;
}

__global__ void __launch_bounds__(kCompactThreads) count_kernel(const __grid_constant__ CompactArgs a) {
  __shared__ uint32_t s_warp[kCompactThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kCompactPerThread;
  uint32_t c = 0;
  if (base < a.n) c = count16(*reinterpret_cast<const uint4*>(a.flags + base));
  const uint32_t tot = block_sum(c, s_warp);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = tot;
}

// Exclusive scan of the tile counts by a single block; writes the total.
__global__ void __launch_bounds__(1024) scan_kernel(const __grid_constant__ CompactArgs a) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < a.n_tiles; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < a.n_tiles ? a.block_counts[i] : 0;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t wv = lane < (int)(blockDim.x / 32) ? s_warp[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wv, o);
        if (lane >= o) wv += y;
      }
      s_warp[lane] = wv;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t warp_off = warp > 0 ? s_warp[warp - 1] : 0;
    const uint32_t carry = s_carry;
    if (i < a.n_tiles) a.block_counts[i] = carry + warp_off + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + warp_off + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.total = s_carry;
}

__device__ __forceinline__ uint32_t brick_id_of(const Geometry& g, uint64_t f) {
  // page table p with pt_off[p] <= f < pt_off[p + 1]
  int lo = 0, hi = g.m * g.k;  // invariant: pt_off[lo] <= f < pt_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (g.pt_off[mid] <= f) lo = mid;
    else hi = mid;
  }
  const uint32_t local = (uint32_t)(f - g.pt_off[lo]);
  const int l = lo % g.k;
  const uint32_t nx = (uint32_t)g.nb[l][0], ny = (uint32_t)g.nb[l][1];
  const uint32_t bx = local % nx, by = (local / nx) % ny, bz = local / (nx * ny);
  return ((uint32_t)lo << 24) | (bz << 16) | (by << 8) | bx;
}

__global__ void __launch_bounds__(kCompactThreads) write_kernel(const __grid_constant__ CompactArgs a) {
  __shared__ uint32_t s_warp[kCompactThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kCompactPerThread;
  uint4 v = make_uint4(0, 0, 0, 0);
  if (base < a.n) v = *reinterpret_cast<const uint4*>(a.flags + base);
  const uint32_t c = count16(v);
  // exclusive rank of this thread's flags within the tile
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t warp_off = 0;
  for (int w = 0; w < warp; ++w) warp_off += s_warp[w];
  uint32_t pos = a.block_counts[blockIdx.x] + warp_off + x - c;
  if (c) {
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
    for (int q = 0; q < 16; ++q) {
      if ((words[q >> 2] >> (8 * (q & 3))) & 0xFFu) {
        if (pos < a.cap) {
          const uint64_t f = base + q;
          a.out[pos] = a.id_mode == 0 ? brick_id_of(a.g, f) : (uint32_t)f;
        }
        ++pos;
      }
    }
    *reinterpret_cast<uint4*>(a.flags + base) = make_uint4(0, 0, 0, 0);
  }
}

// last_used[slot] = frame for every used slot; clears the usage flags.
__global__ void usage_kernel(const __grid_constant__ UsageArgs a) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    if (a.used[i]) {
      a.last_used[i] = a.frame;
      a.used[i] = 0;
    }
  }
}

}  // namespace

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s) {
  if (a.n_tiles == 0) return cudaSuccess;
  count_kernel<<<a.n_tiles, kCompactThreads, 0, s>>>(a);
  scan_kernel<<<1, 1024, 0, s>>>(a);
  write_kernel<<<a.n_tiles, kCompactThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_usage(const UsageArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  uint32_t blocks = (a.n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  usage_kernel<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ro
