// Residency-octree and page-table updates (Sec. 5.3) and the brick-cache
// slot scatter.
//
// Leaf masks are recomputed from the page table: a leaf (extent a power of
// two <= B) lies inside exactly one brick of every level, so bit l of a leaf
// is "the owner brick of level l is resident".  Inner nodes are recomputed as
// the bitwise OR of their children's masks and the hull of their ranges when
// all children are valid, else the range given for the node, else INVALID,
// depth by depth from the leaves up; then, from the root down, every INVALID
// word takes the depth of its nearest valid ancestor (Sec. 5.2).  Every write
// recomputes a word from the final page table / children / parent, so
// concurrent writers of the same word store the same value: no atomics.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ro_internal.h"

namespace ro {
namespace {

__global__ void fill_words_kernel(uint32_t* __restrict__ w, uint64_t n, uint32_t value) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    w[i] = value;
}

// Every n-th word starting at `first` (one channel's column of the octree).
__global__ void fill_strided_kernel(uint32_t* __restrict__ w, uint64_t count, uint32_t stride, uint32_t value) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
    w[i * stride] = value;
}

// Copy each staged brick into its slot (16-byte vectors; slot_pitch is a
// multiple of 256) and write the page-table entries of inserted (slot + 1)
// and evicted (0) bricks.
// A raw value in the cache's sample format: round(v * 2^-S) to
// binary16 (sf 1) or bfloat16 (sf 2), S = 8 or 16 bits, nearest even; the
// scaling by a power of two is exact in binary32.
__device__ __forceinline__ uint16_t to_format(uint32_t v, int sf, int bpv) {
  const float x = (float)v * (bpv == 1 ? 0.00390625f : 1.52587890625e-05f);
  if (sf == 1) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__global__ void __launch_bounds__(256) scatter_kernel(const __grid_constant__ ScatterArgs a) {
  const uint32_t b = blockIdx.x;
  if (b < a.n_ins) {
    const uint32_t slot = a.ins_slot[b];
    if (slot >= a.cache_slots) { if (threadIdx.x == 0) *a.err = kErrSlot; return; }
    const uint8_t* srow = a.staging + (size_t)b * a.slot_pitch;
    uint8_t* drow = a.cache + (size_t)slot * a.slot_pitch;
    if (a.sf == 0) {
      const uint4* src = reinterpret_cast<const uint4*>(srow);
      uint4* dst = reinterpret_cast<uint4*>(drow);
      for (uint32_t i = threadIdx.x; i < a.slot_pitch / 16; i += blockDim.x) dst[i] = src[i];
    } else {
      // eight voxels per step: raw u16 (16 bytes) or u8 (8 bytes) in, 16 bytes out
      uint16_t* dst = reinterpret_cast<uint16_t*>(drow);
      const uint32_t n8 = a.n_el / 8;
      for (uint32_t i = threadIdx.x; i < n8; i += blockDim.x) {
        uint32_t v[8];
        if (a.bpv == 2) {
          const uint4 r = reinterpret_cast<const uint4*>(srow)[i];
          const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) { v[2 * q] = w[q] & 0xFFFFu; v[2 * q + 1] = w[q] >> 16; }
        } else {
          const uint2 r = reinterpret_cast<const uint2*>(srow)[i];
#pragma unroll
          for (int q = 0; q < 4; ++q) { v[q] = (r.x >> (8 * q)) & 0xFFu; v[4 + q] = (r.y >> (8 * q)) & 0xFFu; }
        }
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          o[q] = (uint32_t)to_format(v[2 * q], a.sf, a.bpv) | ((uint32_t)to_format(v[2 * q + 1], a.sf, a.bpv) << 16);
        reinterpret_cast<uint4*>(dst)[i] = make_uint4(o[0], o[1], o[2], o[3]);
      }
      for (uint32_t i = n8 * 8 + threadIdx.x; i < a.n_el; i += blockDim.x) {
        const uint32_t v = a.bpv == 2 ? reinterpret_cast<const uint16_t*>(srow)[i] : srow[i];
        dst[i] = to_format(v, a.sf, a.bpv);
      }
    }
    if (threadIdx.x == 0) {
      const uint32_t pi = a.ins_index[b];
      if (pi >= a.n_bricks) *a.err = kErrPageIndex;
      else a.pt[pi] = slot + 1;
      a.last_used[slot] = a.frame;   // a fresh brick counts as used now (LRU)
    }
  } else {
    const uint32_t e = b - a.n_ins;
    if (e < a.n_ev && threadIdx.x == 0) {
      const uint32_t pi = a.ev_index[e];
      if (pi >= a.n_bricks) *a.err = kErrPageIndex;
      else a.pt[pi] = 0;
    }
  }
}

__device__ __forceinline__ uint32_t quant(uint32_t v, int bpv) { return bpv == 1 ? (v > 255 ? 255 : v) : (v >> 8); }

// Leaf metadata writes: keep the mask, replace min8/max8 (Sec. 7 layout).
__global__ void write_meta_kernel(const __grid_constant__ UpdateArgs a) {
  const Geometry& g = a.g;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_meta; i += gridDim.x * blockDim.x) {
    const MetaItem it = a.meta[i];
    const uint64_t nl = (uint64_t)g.nleaf[0] * g.nleaf[1] * g.nleaf[2];
    if (it.leaf >= nl || it.channel >= (uint32_t)g.m) { *a.err = kErrUpdate; continue; }
    uint32_t* p = a.octree + (g.node_off[g.D] + it.leaf) * g.mp + it.channel;
    uint32_t mn8, mx8;
    if (it.vmin > it.vmax) { mn8 = 255; mx8 = kUnknownDepth; }   // the pointer pass fills the depth in
    else { mn8 = quant(it.vmin, g.bpv); mx8 = quant(it.vmax, g.bpv); }
    *p = (*p & 0xFFFFu) | (mn8 << 16) | (mx8 << 24);
  }
}

// One block per item: recompute the channel's mask of every leaf in the box.
__global__ void __launch_bounds__(256) leaf_masks_kernel(const __grid_constant__ UpdateArgs a) {
  const Geometry& g = a.g;
  const UpdateItem it = a.items[blockIdx.x];
  const uint32_t nx = it.hi[0] - it.lo[0], ny = it.hi[1] - it.lo[1], nz = it.hi[2] - it.lo[2];
  const uint64_t total = (uint64_t)nx * ny * nz;
  const int c = (int)it.channel;
  for (uint64_t q = threadIdx.x; q < total; q += blockDim.x) {
    const uint32_t lx = it.lo[0] + (uint32_t)(q % nx), ly = it.lo[1] + (uint32_t)((q / nx) % ny),
                   lz = it.lo[2] + (uint32_t)(q / ((uint64_t)nx * ny));
    if (lx >= (uint32_t)g.nleaf[0] || ly >= (uint32_t)g.nleaf[1] || lz >= (uint32_t)g.nleaf[2]) continue;
    uint32_t mask = 0;
    for (int l = 0; l < g.k; ++l) {
      // leaf origin in level-0 voxels, divided by the level-l brick extent
      const uint32_t bx = (lx << g.leaf_log2[0]) >> (g.blog2 + g.lsh[l][0]),
                     by = (ly << g.leaf_log2[1]) >> (g.blog2 + g.lsh[l][1]),
                     bz = (lz << g.leaf_log2[2]) >> (g.blog2 + g.lsh[l][2]);
      const uint64_t pi = g.pt_off[c * g.k + l] + ((uint64_t)bz * g.nb[l][1] + by) * g.nb[l][0] + bx;
      if (a.pt[pi] != 0) mask |= 1u << l;
    }
    uint32_t* p = a.octree + (g.node_off[g.D] + ((uint64_t)lz * g.nleaf[1] + ly) * g.nleaf[0] + lx) * g.mp + c;
    *p = (*p & 0xFFFF0000u) | mask;
  }
}

// One block per item: recompute every depth-d node above the item's leaf box
// from its (up to 8) children at depth d + 1.
__global__ void __launch_bounds__(256) reduce_depth_kernel(const __grid_constant__ UpdateArgs a) {
  const Geometry& g = a.g;
  const int d = a.depth;
  const int sh = g.D - d;
  const UpdateItem it = a.items[blockIdx.x];
  uint32_t lo[3], hi[3];
  for (int q = 0; q < 3; ++q) {
    lo[q] = it.lo[q] >> sh;
    hi[q] = ((it.hi[q] - 1) >> sh) + 1;
    if (hi[q] > (uint32_t)g.nn[d][q]) hi[q] = (uint32_t)g.nn[d][q];
  }
  const uint32_t nx = hi[0] - lo[0], ny = hi[1] - lo[1], nz = hi[2] - lo[2];
  const uint64_t total = (uint64_t)nx * ny * nz;
  const int c = (int)it.channel;
  for (uint64_t q = threadIdx.x; q < total; q += blockDim.x) {
    const uint32_t jx = lo[0] + (uint32_t)(q % nx), jy = lo[1] + (uint32_t)((q / nx) % ny),
                   jz = lo[2] + (uint32_t)(q / ((uint64_t)nx * ny));
    uint32_t mask = 0, mn = 255, mx = 0;
    bool invalid = false;
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          const uint32_t kx = 2 * jx + cx, ky = 2 * jy + cy, kz = 2 * jz + cz;
          if (kx >= (uint32_t)g.nn[d + 1][0] || ky >= (uint32_t)g.nn[d + 1][1] || kz >= (uint32_t)g.nn[d + 1][2]) continue;
          const uint32_t w =
              a.octree[(g.node_off[d + 1] + ((uint64_t)kz * g.nn[d + 1][1] + ky) * g.nn[d + 1][0] + kx) * g.mp + c];
          mask |= w & 0xFFFFu;
          const uint32_t wmn = (w >> 16) & 0xFFu, wmx = w >> 24;
          if (wmn > wmx) invalid = true;
          mn = wmn < mn ? wmn : mn;
          mx = wmx > mx ? wmx : mx;
        }
    const uint64_t n = g.node_off[d] + ((uint64_t)jz * g.nn[d][1] + jy) * g.nn[d][0] + jx;
    if (invalid) {
      const uint32_t gv = a.given[n * g.mp + c];
      if (gv & kGivenBit) { mn = gv & 0xFFu; mx = (gv >> 8) & 0xFFu; }
      else { mn = 255; mx = kUnknownDepth; }
    }
    a.octree[n * g.mp + c] = mask | (mn << 16) | (mx << 24);
  }
}

// Ranges given for inner nodes (meta[].leaf holds the node index).
__global__ void write_given_kernel(const __grid_constant__ UpdateArgs a) {
  const Geometry& g = a.g;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_meta; i += gridDim.x * blockDim.x) {
    const MetaItem it = a.meta[i];
    if (it.leaf >= g.node_off[g.D] || it.channel >= (uint32_t)g.m) { *a.err = kErrUpdate; continue; }
    a.given[(uint64_t)it.leaf * g.mp + it.channel] =
        it.vmin > it.vmax ? 0u : kGivenBit | (quant(it.vmax, g.bpv) << 8) | quant(it.vmin, g.bpv);
  }
}

// One block per item: every depth-d node (d >= 1) over the item's leaf box
// that is INVALID for the item's channel points to its parent if the parent
// is valid, else to where the parent points.
__global__ void __launch_bounds__(256) pointer_depth_kernel(const __grid_constant__ UpdateArgs a) {
  const Geometry& g = a.g;
  const int d = a.depth;
  const int sh = g.D - d;
  const UpdateItem it = a.items[blockIdx.x];
  uint32_t lo[3], hi[3];
  for (int q = 0; q < 3; ++q) {
    lo[q] = it.lo[q] >> sh;
    hi[q] = ((it.hi[q] - 1) >> sh) + 1;
    if (hi[q] > (uint32_t)g.nn[d][q]) hi[q] = (uint32_t)g.nn[d][q];
  }
  const uint32_t nx = hi[0] - lo[0], ny = hi[1] - lo[1], nz = hi[2] - lo[2];
  const uint64_t total = (uint64_t)nx * ny * nz;
  const int c = (int)it.channel;
  for (uint64_t q = threadIdx.x; q < total; q += blockDim.x) {
    const uint32_t jx = lo[0] + (uint32_t)(q % nx), jy = lo[1] + (uint32_t)((q / nx) % ny),
                   jz = lo[2] + (uint32_t)(q / ((uint64_t)nx * ny));
    uint32_t* p = a.octree + (g.node_off[d] + ((uint64_t)jz * g.nn[d][1] + jy) * g.nn[d][0] + jx) * g.mp + c;
    const uint32_t w = *p;
    if (((w >> 16) & 0xFFu) <= (w >> 24)) continue;   // valid
    const uint32_t pw =
        a.octree[(g.node_off[d - 1] + ((uint64_t)(jz >> 1) * g.nn[d - 1][1] + (jy >> 1)) * g.nn[d - 1][0] + (jx >> 1)) *
                     g.mp + c];
    const uint32_t ptr = ((pw >> 16) & 0xFFu) <= (pw >> 24) ? (uint32_t)(d - 1) : (pw >> 24);
    *p = (w & 0x00FFFFFFu) | (ptr << 24);
  }
}

}  // namespace

cudaError_t launch_fill_words(uint32_t* words, uint64_t n, uint32_t value, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  fill_words_kernel<<<(unsigned)blocks, 256, 0, s>>>(words, n, value);
  return cudaGetLastError();
}

cudaError_t launch_fill_strided(uint32_t* first, uint64_t count, uint32_t stride, uint32_t value, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  fill_strided_kernel<<<(unsigned)blocks, 256, 0, s>>>(first, count, stride, value);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s) {
  if (a.n_ins + a.n_ev == 0) return cudaSuccess;
  scatter_kernel<<<a.n_ins + a.n_ev, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_write_meta(const UpdateArgs& a, cudaStream_t s) {
  if (a.n_meta == 0) return cudaSuccess;
  uint32_t blocks = (a.n_meta + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  write_meta_kernel<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_leaf_masks(const UpdateArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  leaf_masks_kernel<<<a.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_write_given(const UpdateArgs& a, cudaStream_t s) {
  if (a.n_meta == 0) return cudaSuccess;
  uint32_t blocks = (a.n_meta + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  write_given_kernel<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pointer_depth(const UpdateArgs& a, cudaStream_t s) {
  if (a.n_items == 0 || a.depth < 1) return cudaSuccess;
  pointer_depth_kernel<<<a.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_depth(const UpdateArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  reduce_depth_kernel<<<a.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ro
