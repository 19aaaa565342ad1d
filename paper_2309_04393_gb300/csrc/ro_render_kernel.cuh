// Mixed-resolution multi-volume ray caster through the residency octree
// (Sec. 6.1, Algorithm 1 and the multi-channel walk; Sec. 6.2; Sec. 7): the
// kernel template shared by the single-view and the batch launches.
//
// Persistent blocks, one per SM; each warp renders tiles of 32 pixels.  The
// channels' transfer-function LUTs and bucket-occupancy prefix sums live in
// shared memory; node words, page-table entries and brick-cache voxels are
// read through the read-only path.  Requests and usage are emitted with plain
// byte stores of 1 (idempotent: no atomics).  Every decision is taken in
// binary32 with the operation order of the design contract (built with
// --fmad=false: every fused multiply-add below is an explicit fmaf).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ro_internal.h"

namespace ro {
namespace {

enum : int { kEmpty = 0, kHomog = 1, kUnmapped = 2, kBrick = 3, kInvalid = 4 };

// bit budgets of the packed warp shuffles below
static_assert(kMaxC <= 16, "a channel set fits 16 bits");
static_assert(kMaxDepth < 31, "depth 31 marks an out-of-range node");
static_assert(kMaxViews <= (1 << 13), "a view index fits 13 bits");

// 2^23 + v for an integer 0 <= v < 2^23, exactly: v in the significand of 2^23
__device__ __forceinline__ float biased(uint32_t v) { return __uint_as_float(0x4B000000u | v); }

// floor(x * 2^e) for 0 <= x * 2^e < 2^23 (the product is exact): the sum
// x * 2^e + 2^23 rounded down is 2^23 + floor(x * 2^e), whose low bits are it
__device__ __forceinline__ int floor_scaled(float x, float p2) {
  return __float_as_int(__fmaf_rd(x, p2, 8388608.0f)) - 0x4B000000;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ uint32_t fnv_word(uint32_t h, uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    h ^= (w >> (8 * b)) & 0xFFu;
    h *= 16777619u;
  }
  return h;
}

// Per-channel state at one node (Algorithm 1 order: empty, homogeneous,
// partially mapped at a usable level).
template <int BPV>
__device__ __forceinline__ int classify(uint32_t w, const uint16_t* pre, int ld, int k) {
  const uint32_t mn = (w >> 16) & 0xFFu, mx = w >> 24;
  if (mn > mx) return kInvalid;
  if (pre[mx + 1] == pre[mn]) return kEmpty;
  if (BPV == 1 && mn == mx) return kHomog;
  const uint32_t usable = (w & 0xFFFFu) & (~0u << ld) & ((1u << k) - 1u);
  return usable ? kBrick : kUnmapped;
}

__device__ __forceinline__ bool terminal(int s) { return s == kEmpty || s == kHomog || s == kUnmapped; }

// CPL consecutive node words (one vector load; CPL = 4, 2 or 1).
template <int CPL>
__device__ __forceinline__ void load_cpl(const uint32_t* p, uint32_t (&w)[CPL]) {
  if constexpr (CPL == 4) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (CPL == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = v.x; w[1] = v.y;
  } else {
    w[0] = __ldg(p);
  }
}

struct Ray {
  float o[3], d[3];
  float t0, t1;
  bool hit;
};

// Pixel-centre ray (pixel i at i + 0.5), voxel-space origin/direction and
// slab interval.
__device__ Ray make_ray(const Geometry& g, const ViewArgs& V, int px, int py) {
  Ray r;
  float o[3], d[3];
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  if (V.persp) {
    const float u = __fdiv_rn(fx, (float)V.W), w = __fdiv_rn(fy, (float)V.H);
    const float sa = (2.0f * u - 1.0f) * V.tan_x;
    const float sb = (1.0f - 2.0f * w) * V.tan_y;
    float dd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] = fmaf(sb, V.up[k], fmaf(sa, V.right[k], V.fwd[k]));
    const float n2 = fmaf(dd[2], dd[2], fmaf(dd[1], dd[1], dd[0] * dd[0]));
    const float len = __fsqrt_rn(n2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = V.eye[k];
      d[k] = __fdiv_rn(dd[k], len);
    }
  } else {
    const float sa = (fx - 0.5f * (float)V.W) * V.pixel;
    const float sb = (0.5f * (float)V.H - fy) * V.pixel;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = fmaf(sb, V.up[k], fmaf(sa, V.right[k], V.eye[k]));
      d[k] = V.fwd[k];
    }
  }
  float tmin = -INFINITY, tmax = INFINITY;
  r.hit = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.o[k] = __fdiv_rn(o[k], g.spacing[k]);
    r.d[k] = __fdiv_rn(d[k], g.spacing[k]);
    if (r.d[k] != 0.0f) {
      const float ta = __fdiv_rn(0.0f - r.o[k], r.d[k]);
      const float tb = __fdiv_rn((float)g.dims0[k] - r.o[k], r.d[k]);
      tmin = fmaxf(tmin, fminf(ta, tb));
      tmax = fminf(tmax, fmaxf(ta, tb));
    } else if (r.o[k] < 0.0f || r.o[k] >= (float)g.dims0[k]) {
      r.hit = false;
    }
  }
  r.t0 = fmaxf(tmin, 0.0f);
  r.t1 = tmax;
  if (!(r.t0 < r.t1)) r.hit = false;
  return r;
}

__device__ __forceinline__ void position(const Geometry& g, const Ray& r, float t, float (&x)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = fminf(fmaxf(fmaf(t, r.d[k], r.o[k]), 0.0f), g.dimm[k]);
}

__device__ __forceinline__ void node_coords(const Geometry& g, int d, const float (&x)[3], int (&j)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) j[k] = floor_scaled(x[k], pow2f(-(g.leaf_log2[k] + g.D - d)));
}

// Trilinear sample of a level-l apron slot, in two parts: the
// in-slot offset of the lower corner and the lerp weights depend only on the
// position and the level (every channel's bricks share one grid), so they
// are computed once per level and sample; the fetch reads one channel's
// corners from its owner's slot and lerps along x, then y, then z.
struct TriCoords {
  int idx;        // element offset of the lower corner inside the apron slot
  float f[3];     // lerp weights (binary32)
  uint32_t h[3];  // the weights in a 16-bit sample format: (f0, f0), (f1, f1), f2
};

// Two 16-bit values packed into one 32-bit register, low half first.
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x5410); }

__device__ __forceinline__ __half __low2half_any(__half2 v) { return __low2half(v); }
__device__ __forceinline__ __half __high2half_any(__half2 v) { return __high2half(v); }
__device__ __forceinline__ __nv_bfloat16 __low2half_any(__nv_bfloat162 v) { return __low2bfloat16(v); }
__device__ __forceinline__ __nv_bfloat16 __high2half_any(__nv_bfloat162 v) { return __high2bfloat16(v); }

template <int SF> struct Fmt;
template <> struct Fmt<1> {
  using T = __half;
  using T2 = __half2;
  static __device__ __forceinline__ uint32_t dup(float f) {
    const __half2 v = __float2half2_rn(f);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  static __device__ __forceinline__ T2 v2(uint32_t u) { return *reinterpret_cast<const T2*>(&u); }
  static __device__ __forceinline__ uint32_t u2(T2 h) { return *reinterpret_cast<const uint32_t*>(&h); }
  static __device__ __forceinline__ float to_float(T h) { return __half2float(h); }
};
template <> struct Fmt<2> {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ uint32_t dup(float f) {
    const __nv_bfloat162 v = __float2bfloat162_rn(f);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  static __device__ __forceinline__ T2 v2(uint32_t u) { return *reinterpret_cast<const T2*>(&u); }
  static __device__ __forceinline__ uint32_t u2(T2 h) { return *reinterpret_cast<const uint32_t*>(&h); }
  static __device__ __forceinline__ float to_float(T h) { return __bfloat162float(h); }
};

// Per-level tables read with a per-lane level index, kept in shared memory:
// level dims - 1 (clamp bounds) and the per-axis log2 voxel extents.
struct LevelTabs {
  float ldimf[kMaxL][3];
  int lsh[kMaxL][3];
  int lstep[kMaxL];
};

template <int EC, int SF>
__device__ __forceinline__ void tri_coords(const Geometry& g, const LevelTabs& lt, int l, const float (&x)[3],
                                           TriCoords& tc) {
  const int E = EC ? EC : (int)g.edge;  // apron-slot edge, a compile-time constant for 32^3 bricks
  int li[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int sh = lt.lsh[l][k];        // level-l voxels are 2^sh level-0 voxels long along axis k
    const float xl = x[k] * pow2f(-sh);
    float u = xl - 0.5f;
    u = fminf(fmaxf(u, 0.0f), lt.ldimf[l][k]);
    const float tu = __fadd_rd(u, 8388608.0f);      // 2^23 + floor(u), u >= 0
    const int i0 = __float_as_int(tu) - 0x4B000000;
    tc.f[k] = u - (tu - 8388608.0f);
    const int b = floor_scaled(x[k], pow2f(-(g.blog2 + sh)));
    li[k] = i0 - (b * g.B - 1);
  }
  tc.idx = (li[2] * E + li[1]) * E + li[0];
  if constexpr (SF != 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) tc.h[k] = Fmt<SF>::dup(tc.f[k]);
  }
}

// The eight corners of a trilinear footprint as raw integers (u8 / u16
// values, or the 16-bit patterns of the binary16 / bfloat16 formats), loaded
// apart from their use so that several channels' corners are in flight at
// once.  base + idx must address a voxel whose 2x2x2 block lies in its slot.
template <int BPV, int EC, int SF>
__device__ __forceinline__ void tri_load(const Geometry& g, const uint8_t* base, int idx, uint32_t (&r)[8]) {
  const int E = EC ? EC : (int)g.edge;
  if constexpr (BPV == 1 && SF == 0) {
    const uint8_t* p = base + idx;
    r[0] = __ldg(p); r[1] = __ldg(p + 1); r[2] = __ldg(p + E); r[3] = __ldg(p + E + 1);
    r[4] = __ldg(p + E * E); r[5] = __ldg(p + E * E + 1); r[6] = __ldg(p + E * E + E); r[7] = __ldg(p + E * E + E + 1);
  } else {
    const uint16_t* p = reinterpret_cast<const uint16_t*>(base) + idx;
    r[0] = __ldg(p); r[1] = __ldg(p + 1); r[2] = __ldg(p + E); r[3] = __ldg(p + E + 1);
    r[4] = __ldg(p + E * E); r[5] = __ldg(p + E * E + 1); r[6] = __ldg(p + E * E + E); r[7] = __ldg(p + E * E + E + 1);
  }
}

// b - a per component with one rounding each (as a binary32 subtraction:
// fma(a, -1, b) rounds the exact difference once).
__device__ __forceinline__ float2 sub2(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.0f, -1.0f), b); }

// Lerps along x, then y, then z (each fma(f, b - a, a)) of loaded corners;
// the binary32 path runs the x lerps and the y lerps two at a time in packed
// binary32 operations, each component rounded as its scalar operation.
template <int BPV, int SF>
__device__ __forceinline__ float tri_lerp(const uint32_t (&r)[8], const TriCoords& tc) {
  if constexpr (SF != 0) {
    // the slot holds the format's values; x lerps on the pairs (v0, v2) /
    // (v1, v3) and (v4, v6) / (v5, v7), the y lerp on (c00, c01) / (c10,
    // c11), the z lerp alone: each d = b - a, then fma(f, d, a), one
    // rounding per operation as in the format's arithmetic
    using F = Fmt<SF>;
    const typename F::T2 A = F::v2(pack2(r[0], r[2])), B = F::v2(pack2(r[1], r[3]));
    const typename F::T2 A2 = F::v2(pack2(r[4], r[6])), B2 = F::v2(pack2(r[5], r[7]));
    const typename F::T2 f0 = F::v2(tc.h[0]), f1 = F::v2(tc.h[1]);
    const typename F::T2 cx0 = __hfma2(f0, __hsub2(B, A), A);      // (c00, c10)
    const typename F::T2 cx1 = __hfma2(f0, __hsub2(B2, A2), A2);   // (c01, c11)
    const uint32_t u0 = F::u2(cx0), u1 = F::u2(cx1);
    const typename F::T2 lo = F::v2(pack2(u0, u1)), hi = F::v2(pack2(u0 >> 16, u1 >> 16));
    const typename F::T2 cy = __hfma2(f1, __hsub2(hi, lo), lo);    // (c0, c1)
    const typename F::T c0 = __low2half_any(cy), c1 = __high2half_any(cy);
    const typename F::T f2 = __low2half_any(F::v2(tc.h[2]));
    const typename F::T c = __hfma(f2, __hsub(c1, c0), c0);
    return F::to_float(c) * (BPV == 1 ? 256.0f : 65536.0f);
  } else {
    // the corners as binary32 values (exact): the lower corners a = A - 2^23
    // from their biased forms A = 2^23 + a, and the differences b - a = B - A
    // (exact: both sides are integers below 2^16)
    const float2 f0 = make_float2(tc.f[0], tc.f[0]), f1 = make_float2(tc.f[1], tc.f[1]);
    const float2 A0 = make_float2(biased(r[0]), biased(r[2])), B0 = make_float2(biased(r[1]), biased(r[3]));
    const float2 A1 = make_float2(biased(r[4]), biased(r[6])), B1 = make_float2(biased(r[5]), biased(r[7]));
    const float2 m23 = make_float2(-8388608.0f, -8388608.0f);
    const float2 a0 = __fadd2_rn(A0, m23), a1 = __fadd2_rn(A1, m23);
    const float2 cx0 = __ffma2_rn(f0, sub2(B0, A0), a0);   // (c00, c10)
    const float2 cx1 = __ffma2_rn(f0, sub2(B1, A1), a1);   // (c01, c11)
    const float2 ya = make_float2(cx0.x, cx1.x), yb = make_float2(cx0.y, cx1.y);
    const float2 cy = __ffma2_rn(f1, sub2(yb, ya), ya);    // (c0, c1)
    return fmaf(tc.f[2], cy.y - cy.x, cy.x);
  }
}

// TF lookup (linear between the 256 LUT entries) at the unclamped TF
// coordinate xq = (v - lo) * scale, and opacity correction for a step of 2^s
// (s squarings of 1 - alpha, Sec. 6.1): returns the corrected opacity's
// complement q and the colour (r, g) and b.  The four component lerps run as
// two packed binary32 operations, each component rounded as a scalar fma.
__device__ __forceinline__ void shade(const float4* __restrict__ lut, float xq, int s, float& q, float2& rg,
                                      float& b) {
  xq = fminf(fmaxf(xq, 0.0f), 255.0f);
  // j = min(floor(xq), 254) as 2^23 + j: the sum rounded down is exact
  const float tj = fminf(__fadd_rd(xq, 8388608.0f), 8388862.0f);
  const int j = __float_as_int(tj) - 0x4B000000;
  const float fr = xq - (tj - 8388608.0f);
  const float4 L0 = lut[j], L1 = lut[j + 1];
  const float2 ff = make_float2(fr, fr);
  const float2 lrg = make_float2(L0.x, L0.y), lba = make_float2(L0.z, L0.w);
  rg = __ffma2_rn(ff, sub2(make_float2(L1.x, L1.y), lrg), lrg);
  const float2 ba = __ffma2_rn(ff, sub2(make_float2(L1.z, L1.w), lba), lba);
  b = ba.x;
  const float al = fminf(fmaxf(ba.y, 0.0f), 1.0f);
  q = 1.0f - al;
  for (int e = 0; e < s; ++e) q = q * q;
}

// Per-ray cache of the last classification: the final node, the desired
// levels it was made for (their lod value: the desired levels and the
// traversal depth are functions of it) and whether every channel may be
// skipped there.  A sample that lands in the same node with the same desired
// levels gets the same decisions (the walk, the states, the selected slots
// and levels), provided the node lies inside one brick of every level a
// channel may use; requests and usage flags are then already set (the stores
// are idempotent).
struct NodeCache {
  // d (bits 0-4, 31 = none) | lod (5-8) | all_skip (9) | one_brick (10) |
  // finest level read (11-15, 31 = none) | channels read from a brick (16-20) |
  // step exponent of the finest level read, else of the finest desired (21-25)
  uint32_t meta;
  int jn[3];             // node coordinates at depth d
  uint32_t act;          // channels with a value at this node (brick or node value)
  __device__ __forceinline__ int d() const { return (meta & 31u) == 31u ? -1 : (int)(meta & 31u); }
  __device__ __forceinline__ int lod() const { return (int)((meta >> 5) & 15u); }
  __device__ __forceinline__ bool all_skip() const { return (meta >> 9) & 1u; }
  __device__ __forceinline__ bool one_brick() const { return (meta >> 10) & 1u; }
  __device__ __forceinline__ uint32_t n_brick() const { return (meta >> 16) & 31u; }
  __device__ __forceinline__ int step() const { return (int)((meta >> 21) & 31u); }
  __device__ __forceinline__ void clear() { meta = 31u; }
  __device__ __forceinline__ void set(int d, int lod, bool all_skip, bool one_brick, int s_sel, uint32_t n_brick,
                                      int step) {
    meta = (uint32_t)d | ((uint32_t)lod << 5) | ((uint32_t)all_skip << 9) | ((uint32_t)one_brick << 10) |
           ((uint32_t)(s_sel == 99 ? 31 : s_sel) << 11) | (n_brick << 16) | ((uint32_t)step << 21);
  }
};

// Per-lane selection word (one per channel, in shared memory): bits 31..27
// the level read (0..15) or kSelHomog, bits 26..0 the slot or the node value.
constexpr uint32_t kSelNone = 0xFFFFFFFFu;
constexpr uint32_t kSelHomog = 30u;
constexpr uint32_t kSelMask = (1u << 27) - 1u;

// Per-thread counters of the current ray (its counts stay below 2^28): the
// evaluated samples and brick reads are the ray's own n_eval and n_bs; at
// every refill the unit adds them to its 64-bit row in shared memory.
struct Counters {
  uint32_t homog;   // rays hit and skips go straight to the warp's shared row
};

template <int BPV, bool DBG>
__device__ __forceinline__ void write_pixel(const ViewArgs& V, uint32_t pix, float4 col,
                                            uint32_t h, uint32_t n_eval, int i, uint32_t n_bs) {
  const size_t p = (size_t)(pix >> 16) * V.W + (pix & 0xFFFFu);
  V.image[p] = make_float4(fminf(col.x, 1.0f), fminf(col.y, 1.0f), fminf(col.z, 1.0f), 1.0f - col.w);
  if constexpr (DBG) {
    if (V.dbg_hash) V.dbg_hash[p] = h;
    if (V.dbg_n_eval) V.dbg_n_eval[p] = n_eval;
    if (V.dbg_i_end) V.dbg_i_end[p] = (uint32_t)i;
    if (V.dbg_n_bs) V.dbg_n_bs[p] = n_bs;
  }
}

// Persistent launch.  Each warp takes the next tile of 32 pixels (8 x 4 by
// default) from a counter once all its lanes are free, so the 32 rays of a
// warp stay neighbours and their footprints share cache lines.  A batch
// launch renders many views: the counter runs over the tiles of all views
// (optionally through a schedule `order`), and each warp copies the view of
// its current tile into shared memory.
// One loop iteration = one lattice step of every active lane, in three
// phases: (1) per lane, the sample position and desired levels, and whether
// the cached node still applies; (2) for the lanes that need a new node, the
// warp walks the octree cooperatively, one lane per channel, 32 / MP rays at
// a time, and writes each ray's states and brick selections; (3) per lane,
// the skip or the evaluated sample.
template <bool BATCH>
__device__ __forceinline__ const ViewArgs& view_of(const RenderArgs& a, const ViewArgs* sv) {
  if constexpr (BATCH) return *sv;
  else return a.v;
}

template <int MP, int BPV, int EC, bool DBG, bool BATCH, int SF>
__global__ void __launch_bounds__(render_threads(BATCH), 1) render_kernel(const __grid_constant__ RenderArgs a) {
  extern __shared__ float4 smem[];
  float4* s_lut = smem;
  uint16_t* s_pre = reinterpret_cast<uint16_t*>(s_lut + MP * 256);
  uint32_t* s_sel = reinterpret_cast<uint32_t*>(smem) + MP * 256 * 4 + ((MP * 257 * 2 + 15) & ~15) / 4;
  const Geometry& g = a.g;
  const int m = g.m, k = g.k;
  for (int q = threadIdx.x; q < m * 256; q += blockDim.x) s_lut[q] = a.lut[q];
  for (int q = threadIdx.x; q < m * 257; q += blockDim.x) s_pre[q] = a.prefix[q];
  // per-channel tables read with a per-lane channel index live in shared
  // memory (a constant-bank read with divergent indices is replayed per index)
  __shared__ float2 s_tf[kMaxC];
  __shared__ uint32_t s_pto[kMaxC * kMaxL + 1];
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    if constexpr (BATCH) s_tf[q] = a.tf_dev[q];
    else s_tf[q] = make_float2(a.tf_lo[q], a.tf_scale[q]);
  }
  for (int q = threadIdx.x; q <= m * k; q += blockDim.x) s_pto[q] = g.pt_off[q];
  // per-depth node tables and per-level brick counts (indexed per lane)
  __shared__ unsigned long long s_noff[kMaxDepth + 2];
  __shared__ int s_nn[kMaxDepth + 1][3];
  __shared__ int s_nb[kMaxL][3];
  __shared__ LevelTabs s_lt;
  for (int q = threadIdx.x; q < 3 * kMaxL; q += blockDim.x) {
    s_lt.ldimf[q / 3][q % 3] = g.ldimf[q / 3][q % 3];
    s_lt.lsh[q / 3][q % 3] = g.lsh[q / 3][q % 3];
  }
  for (int q = threadIdx.x; q < kMaxL; q += blockDim.x) s_lt.lstep[q] = g.lstep[q];
  for (int q = threadIdx.x; q <= g.D + 1; q += blockDim.x) s_noff[q] = g.node_off[q];
  for (int q = threadIdx.x; q < 3 * (g.D + 1); q += blockDim.x) s_nn[q / 3][q % 3] = g.nn[q / 3][q % 3];
  for (int q = threadIdx.x; q < 3 * k; q += blockDim.x) s_nb[q / 3][q % 3] = g.nb[q / 3][q % 3];
  // the octree's top depths (those whose words fit kTopWords) in shared memory
  constexpr int kThreads = render_threads(BATCH);
  uint32_t* s_top = s_sel + MP * kThreads;
  // per warp: the last kWalkCache walk results (see phase 1), none yet
  uint32_t* s_wc = s_top + kTopWords + (threadIdx.x >> 5) * (kWalkCache * kWalkEntry);
  if ((threadIdx.x & 31) < kWalkCache) s_wc[(threadIdx.x & 31) * kWalkEntry] = 0u;
  // per thread: its current ray (origin, t0; direction, t1) and its colour
  // and transmittance (C0, C1, C2, T), kept in shared memory rather than
  // registers
  float4* s_ray = reinterpret_cast<float4*>(s_top + kTopWords + (kThreads / 32) * kWalkCache * kWalkEntry) +
                  2 * threadIdx.x;
  float4* s_col = reinterpret_cast<float4*>(s_top + kTopWords + (kThreads / 32) * kWalkCache * kWalkEntry) +
                  2 * kThreads + threadIdx.x;
  auto ray_get = [&]() {
    const float4 u = s_ray[0], v = s_ray[1];
    Ray q;
    q.o[0] = u.x; q.o[1] = u.y; q.o[2] = u.z; q.t0 = u.w;
    q.d[0] = v.x; q.d[1] = v.y; q.d[2] = v.z; q.t1 = v.w;
    q.hit = true;
    return q;
  };
  int top_d = -1;
  while (top_d < g.D && g.node_off[top_d + 2] * MP <= (uint64_t)kTopWords) ++top_d;
  const uint32_t n_top = top_d >= 0 ? (uint32_t)(g.node_off[top_d + 1] * MP) : 0u;
  for (uint32_t q = threadIdx.x; q < n_top; q += blockDim.x) s_top[q] = __ldg(a.octree + q);
  constexpr int kUnits = 32 / kRefillLanes;       // refill units per warp
  __shared__ unsigned long long s_red[kThreads / 32 * kUnits][kStats];
  for (int q = threadIdx.x; q < kThreads / 32 * kUnits * kStats; q += blockDim.x) (&s_red[0][0])[q] = 0;
  // batch: first tile of every view (view v owns [s_base[v], s_base[v + 1]))
  // and the current view of each warp
  __shared__ uint32_t s_base[BATCH ? kMaxViews + 1 : 1];
  __shared__ ViewArgs s_view[BATCH ? kThreads / 32 * kUnits : 1];
  if constexpr (BATCH) {
    for (int q = threadIdx.x; q < a.n_views; q += blockDim.x) s_base[q] = a.views[q].tile_base;
    if (threadIdx.x == 0) s_base[a.n_views] = (uint32_t)(a.n_rays >> 5);
  }
  __syncthreads();
  // channels whose TF has a transparent first knot (bit c)
  uint32_t knot0_clear = 0;
  for (int c = 0; c < m; ++c) knot0_clear |= (s_lut[c * 256].w <= 0.0f ? 1u : 0u) << c;

  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int stride = blockDim.x;
  uint32_t* my_sel = s_sel + threadIdx.x;
  // a warp refills in units of kRefillLanes lanes: each unit takes the next
  // kRefillLanes rays of a tile (a band of whole tile rows) once all its
  // lanes are free, so that its rays stay neighbours
  const int unit = lane / kRefillLanes, ulane = lane % kRefillLanes;
  const unsigned umask = (kRefillLanes == 32 ? FULL : ((1u << kRefillLanes) - 1u)) << (unit * kRefillLanes);
  const int row = warp * kUnits + unit;            // this unit's statistics row / view copy
  const ViewArgs& V = view_of<BATCH>(a, &s_view[BATCH ? row : 0]);
  const int twl = a.tile_wlog2, tw = 1 << twl;
  constexpr int G = 32 / MP;                       // rays walked per cooperative pass
  const int grp = lane / MP, ch = lane % MP;
  const unsigned gmask = (MP == 32 ? FULL : ((1u << MP) - 1u)) << (grp * MP);
  const unsigned lt_mask = (1u << lane) - 1u;

  Counters cnt = {0};
  uint32_t h = 0, n_eval = 0, n_bs = 0;
  // adds the unit's counters to its row and clears them (all lanes of the
  // unit call it; each lane has had one ray since the last refill)
  auto flush = [&]() {
    const uint32_t vals[3] = {n_eval, n_bs, cnt.homog};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      unsigned long long v = vals[q];
#pragma unroll
      for (int o = kRefillLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(umask, v, o);
      if (ulane == 0) s_red[row][q + 1] += v;
    }
    cnt = {0};
    n_eval = n_bs = 0;
  };
  uint32_t pix = 0;    // py << 16 | px
  int i = 0, lod = 0;
  NodeCache nc;
  nc.clear();
  nc.jn[0] = nc.jn[1] = nc.jn[2] = 0;
  nc.act = 0;
  uint32_t wc_next = 0;   // next walk-cache entry to fill (warp-uniform)
  bool active = false, done = false;
  uint32_t cur_tile = 0xFFFFFFFFu, iters = 0;  // current tile part (tile * kUnits + part) and its loop iterations
  uint32_t vid = 0;                            // the view of the current rays (batch)

  for (;;) {
    // ------------------------------------------------------------- refill
    const unsigned busy = __ballot_sync(FULL, active);
    const bool unit_free = (busy & umask) == 0 && !done;
    if (__any_sync(FULL, unit_free)) {
      if (unit_free) {
        flush();
        if (a.tile_cost && ulane == 0 && cur_tile != 0xFFFFFFFFu) a.tile_cost[cur_tile] = iters;
        iters = 0;
        unsigned long long base = 0;
        if (ulane == 0) base = atomicAdd(a.work, (unsigned long long)kRefillLanes);
        base = __shfl_sync(umask, base, unit * kRefillLanes);
        if (base >= a.n_rays) {
          done = true;
          cur_tile = 0xFFFFFFFFu;
        } else {
          const uint32_t pos = (uint32_t)(base >> 5), part = (uint32_t)(base & 31u) / kRefillLanes;
          const uint32_t w = part * kRefillLanes + (uint32_t)ulane;   // ray of the tile
          const uint32_t tile = a.order ? __ldg(a.order + pos) : pos;
          cur_tile = tile * kUnits + part;
          if constexpr (BATCH) {
            // the view owning `tile`: last v with s_base[v] <= tile
            int lo = 0, hi = a.n_views - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (s_base[mid] <= tile) lo = mid;
              else hi = mid - 1;
            }
            vid = (uint32_t)lo;
            const uint4* srcv = reinterpret_cast<const uint4*>(a.views + lo);
            uint4* dstv = reinterpret_cast<uint4*>(&s_view[row]);
            for (int q = ulane; q < (int)(sizeof(ViewArgs) / 16); q += kRefillLanes) dstv[q] = __ldg(srcv + q);
            __syncwarp(umask);
          }
          const uint32_t t = tile - V.tile_base;
          const int px = (int)((t % V.tiles_x) * (uint32_t)tw + (w & (uint32_t)(tw - 1)));
          const int py = (int)((t / V.tiles_x) * (uint32_t)(32 >> twl) + (w >> twl));
          pix = ((uint32_t)py << 16) | (uint32_t)px;
          bool hit_now = false;
          if (px < V.W && py < V.H) {
            const Ray r = make_ray(g, V, px, py);
            s_ray[0] = make_float4(r.o[0], r.o[1], r.o[2], r.t0);
            s_ray[1] = make_float4(r.d[0], r.d[1], r.d[2], r.t1);
            i = 0;
            lod = 0;
            *s_col = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            h = 2166136261u;
            n_eval = n_bs = 0;
            nc.clear();
            if (r.hit) {
              active = true;
              hit_now = true;
            } else {
              write_pixel<BPV, DBG>(V, pix, *s_col, h, n_eval, i, n_bs);
            }
          }
          const unsigned hits = __ballot_sync(umask, hit_now);
          if (ulane == 0) s_red[row][0] += __popc(hits);
        }
      }
      __syncwarp();
    }
    if (__all_sync(FULL, done)) break;
    ++iters;

    // ------------------------------------- phase 1: sample, levels, node?
    float x[3] = {0.0f, 0.0f, 0.0f};
    int L[3] = {0, 0, 0};
    uint64_t ldp = 0;
    int lminu = 15, st = 0, dstart = 0;
    bool need = false, same_node = false;
    if (active) {
      const Ray r = ray_get();
      const float t = fmaf((float)i, V.dt, r.t0);
      if (i >= kMaxSamples || !(t < r.t1)) {
        write_pixel<BPV, DBG>(V, pix, *s_col, h, n_eval, i, n_bs);
        active = false;
      } else {
        position(g, r, t, x);
        // lod = #{l in 1..k-1 : t >= lod_t[l]} (Sec. 6.2); t never decreases along
        // a ray and the thresholds are non-decreasing, so the count only grows
        while (lod < k - 1 && t >= V.lod_t[lod + 1]) ++lod;
#pragma unroll
        for (int q = 0; q < 3; ++q) L[q] = floor_scaled(x[q], pow2f(-g.leaf_log2[q]));
        const int ncd = nc.d();
        const bool same_levels = ncd >= 0 && lod == nc.lod();
        if (same_levels) {
          const int sh = g.D - ncd;
          same_node = (L[0] >> sh) == nc.jn[0] && (L[1] >> sh) == nc.jn[1] && (L[2] >> sh) == nc.jn[2];
        }
        need = !(same_node && nc.one_brick());
        // a new node: the desired levels, their finest and its traversal depth
        if (need) {
          ldp = V.ldp_tab[lod];
          lminu = V.lminu_tab[lod];
          st = V.sdepth[lminu];
        }
        // a walk another ray of this tile made for the same node and desired
        // levels gives the same final node, states and selections (the node
        // lies inside one brick of every usable level): take it instead
        if (need) {
#pragma unroll 1
          for (int q = 1; q <= kWalkCache; ++q) {
            const int e = (int)((wc_next + kWalkCache - q) % kWalkCache);   // most recent first
            const uint4 hd = *reinterpret_cast<const uint4*>(s_wc + e * kWalkEntry);
            if (!(hd.x & 1u) || (int)((hd.x >> 6) & 15u) != lod || (hd.x >> 21) != vid) continue;
            const int ed = (int)((hd.x >> 1) & 31u), esh = g.D - ed;
            if ((uint32_t)(L[0] >> esh) != hd.y || (uint32_t)(L[1] >> esh) != hd.z || (uint32_t)(L[2] >> esh) != hd.w)
              continue;
            const uint32_t eact = s_wc[e * kWalkEntry + 4];
            for (uint32_t mm2 = eact; mm2; mm2 &= mm2 - 1u) {
              const int c = __ffs(mm2) - 1;
              my_sel[c * stride] = s_wc[e * kWalkEntry + 5 + c];
            }
            const int ef = (int)((hd.x >> 11) & 31u);
            nc.set(ed, lod, ((hd.x >> 10) & 1u) != 0, true, ef == 31 ? 99 : ef, (hd.x >> 16) & 31u,
                   s_lt.lstep[ef == 31 ? lminu : ef]);
            nc.jn[0] = (int)hd.y; nc.jn[1] = (int)hd.z; nc.jn[2] = (int)hd.w;
            nc.act = eact;
            need = false;
            same_node = true;
            break;
          }
        }
        // the walk (Sec. 6.1) resumes below the deepest ancestor shared with the
        // previous sample: those depths were found not all terminal
        if (need) {
          const int d0 = V.start_depth < st ? V.start_depth : st;
          dstart = d0;
          if (same_node) {
            dstart = ncd;
          } else if (same_levels) {
            // deepest shared ancestor: along each axis the node coordinates at
            // depth ncd agree above their highest differing bit
            const int sh = g.D - ncd;
            const uint32_t dx = (uint32_t)((L[0] >> sh) ^ nc.jn[0]) | (uint32_t)((L[1] >> sh) ^ nc.jn[1]) |
                                (uint32_t)((L[2] >> sh) ^ nc.jn[2]);
            int dca = dx ? ncd - (32 - __clz((int)dx)) : ncd;
            dca = dca < 0 ? 0 : dca;
            dstart = dca + 1 > d0 ? dca + 1 : d0;
          }
        }
      }
    }

    // ------------------------------ phase 2: cooperative walk + selection
    unsigned pending = __ballot_sync(FULL, need);
    while (pending) {
      // the q-th lane of `pending` (in lane order) is walked by group q
      unsigned rest = pending;
#pragma unroll
      for (int q = 0; q < G; ++q) rest &= rest - 1u;
      const unsigned taken = pending & ~rest;
      pending = rest;
      unsigned pm = taken;
      for (int q = 0; q < grp && pm; ++q) pm &= pm - 1u;
      const int src = pm ? __ffs(pm) - 1 : lane;
      const bool gact = pm != 0;
      const float sx0 = __shfl_sync(FULL, x[0], src), sx1 = __shfl_sync(FULL, x[1], src),
                  sx2 = __shfl_sync(FULL, x[2], src);
      const int sL0 = __shfl_sync(FULL, L[0], src), sL1 = __shfl_sync(FULL, L[1], src),
                sL2 = __shfl_sync(FULL, L[2], src);
      const uint32_t ldp_lo = __shfl_sync(FULL, (uint32_t)ldp, src),
                     ldp_hi = __shfl_sync(FULL, (uint32_t)(ldp >> 32), src);
      const uint64_t sldp = ((uint64_t)ldp_hi << 32) | ldp_lo;
      // traversal depth, start depth, finest desired level, lod, same node, view
      const uint32_t pk = __shfl_sync(FULL, (uint32_t)st | ((uint32_t)dstart << 5) | ((uint32_t)lminu << 10) |
                                                ((uint32_t)lod << 14) | ((uint32_t)same_node << 18) | (vid << 19), src);
      const int sst = (int)(pk & 31u), sds = (int)((pk >> 5) & 31u), slm = (int)((pk >> 10) & 15u),
                slod = (int)((pk >> 14) & 15u);
      const bool ssame = ((pk >> 18) & 1u) != 0;
      const uint32_t svid = BATCH ? pk >> 19 : 0u;
      const bool cact = gact && ch < m;
      const int ld = cact ? (int)((sldp >> (4 * ch)) & 15) : 0;
      const uint16_t* pre = s_pre + ch * 257;

      // the walk (Sec. 6.1), kWalkWin depths at a time: every node word of
      // the window is loaded before any is classified.  A channel's terminal
      // states are inherited by the node's children, so the group's final
      // depth is the first at which all its channels are terminal, or the
      // traversal depth, or the start depth when the cached node still holds.
      int dfin = -1;                 // final depth of this lane's group
      bool bad = false;
      uint32_t w = 0;                // this lane's channel word at the final depth
      uint32_t rw = 0;               // the same, an INVALID word read through its pointer
      int sc = kEmpty;
      for (int d0 = sds;; d0 += kWalkWin) {
        uint32_t wv[kWalkWin];
        unsigned tm = 0, stop = 0, badm = 0;
#pragma unroll
        for (int q = 0; q < kWalkWin; ++q) {
          const int dd = d0 + q;
          wv[q] = 0u;
          if (gact && dfin < 0 && dd <= sst) {
            const int sh = g.D - dd;
            const uint64_t node = s_noff[dd] + ((uint64_t)(sL2 >> sh) * s_nn[dd][1] + (sL1 >> sh)) * s_nn[dd][0] + (sL0 >> sh);
            if (node >= s_noff[dd + 1]) badm |= 1u << q;
            else if (cact) wv[q] = dd <= top_d ? s_top[node * MP + ch] : __ldg(a.octree + node * MP + ch);
          }
        }
        // an INVALID word whose channel has a valid ancestor is read with the
        // ancestor's range and its own mask (Sec. 5.2: the pointer to the node
        // of the next lower subdivision level with valid information)
        uint32_t rv[kWalkWin];
#pragma unroll
        for (int q = 0; q < kWalkWin; ++q) {
          const uint32_t wq = wv[q], pd = wq >> 24;
          rv[q] = wq;
          if (cact && ((wq >> 16) & 0xFFu) > pd && (int)pd < d0 + q) {
            const int sh = g.D - (int)pd;
            const uint64_t an = s_noff[pd] + ((uint64_t)(sL2 >> sh) * s_nn[pd][1] + (sL1 >> sh)) * s_nn[pd][0] + (sL0 >> sh);
            const uint32_t aw = (int)pd <= top_d ? s_top[an * MP + ch] : __ldg(a.octree + an * MP + ch);
            rv[q] = (wq & 0xFFFFu) | (aw & 0xFFFF0000u);
          }
        }
#pragma unroll
        for (int q = 0; q < kWalkWin; ++q) {
          const int dd = d0 + q;
          if (!cact || terminal(classify<BPV>(rv[q], pre, ld, k))) tm |= 1u << q;
          if (dd >= sst || dd >= g.D || (ssame && dd == sds)) stop |= 1u << q;
        }
        stop |= badm;
        if constexpr (MP > 1) {
          // over the group's lanes: all terminal (AND), any stop (OR)
          unsigned tg = 0, sg = 0;
#pragma unroll
          for (int q = 0; q < kWalkWin; ++q) {
            const unsigned bt = __ballot_sync(FULL, (tm >> q) & 1u) & gmask;
            const unsigned bs = __ballot_sync(FULL, (stop >> q) & 1u) & gmask;
            tg |= (bt == gmask ? 1u : 0u) << q;
            sg |= (bs != 0u ? 1u : 0u) << q;
          }
          tm = tg;
          stop = sg;
        }
        const unsigned fin = (tm | stop) & ((1u << kWalkWin) - 1u);
        if (gact && dfin < 0 && fin) {
          const int q = __ffs(fin) - 1;
          dfin = d0 + q;
          bad = (badm & ((2u << q) - 1u)) != 0;
#pragma unroll
          for (int qq = 0; qq < kWalkWin; ++qq)
            if (qq == q) { w = wv[qq]; rw = rv[qq]; }
          if (cact) sc = classify<BPV>(rw, pre, ld, k);
        }
        if (__all_sync(FULL, !gact || dfin >= 0)) break;
      }
      const int d = dfin < 0 ? 0 : dfin;
      const int fsh = g.D - d;
      const int jn0 = sL0 >> fsh, jn1 = sL1 >> fsh, jn2 = sL2 >> fsh;
      const uint64_t node = s_noff[d] + ((uint64_t)jn2 * s_nn[d][1] + jn1) * s_nn[d][0] + jn0;
      const bool gbad = (__ballot_sync(FULL, bad) & gmask) != 0;
      // page-table index of this lane's channel at level l (owner brick of the sample)
      auto pt_index = [&](int l) -> uint64_t {
        const int bx = floor_scaled(sx0, pow2f(-(g.blog2 + s_lt.lsh[l][0]))),
                  by = floor_scaled(sx1, pow2f(-(g.blog2 + s_lt.lsh[l][1]))),
                  bz = floor_scaled(sx2, pow2f(-(g.blog2 + s_lt.lsh[l][2])));
        return s_pto[ch * k + l] + ((uint64_t)bz * s_nb[l][1] + by) * s_nb[l][0] + bx;
      };

      // requests of channels with nothing usable here; node requests of
      // channels whose own metadata is missing here (reportNodeRequest),
      // unless the ancestor's range shows the node empty or homogeneous
      if (cact && !gbad) {
        const bool no_use = ((w & 0xFFFFu) & (~0u << ld) & ((1u << k) - 1u)) == 0;
        if (sc == kUnmapped || (sc == kInvalid && no_use)) {
          const uint64_t pi = pt_index(ld);
          if (pi >= g.n_bricks) *a.err = kErrPageIndex;
          else a.req[pi] = 1;
        }
        const bool missing = ((w >> 16) & 0xFFu) > (w >> 24);
        if (missing && sc != kEmpty && sc != kHomog) a.node_req[node * m + ch] = 1;
      }
      const unsigned nonskip = __ballot_sync(FULL, cact && sc != kEmpty && sc != kUnmapped);
      const bool all_skip = (nonskip & gmask) == 0;

      // brick selection (Algorithm 1): the desired level, else request it and
      // take the next coarser resident level.  The page-table entries of the
      // first two levels the node is partially mapped in are fetched together.
      uint32_t sel = kSelNone;
      int found = 99;
      if (cact && !gbad && !all_skip && sc != kEmpty && sc != kUnmapped) {
        if (sc == kHomog) {
          sel = (kSelHomog << 27) | ((rw >> 16) & 0xFFu);
        } else {
          uint32_t cand = (w & 0xFFFFu) & (~0u << ld) & ((1u << k) - 1u);
          if (cand) {
            const int l1 = __ffs(cand) - 1;
            cand &= cand - 1u;
            const int l2 = cand ? __ffs(cand) - 1 : l1;
            if (cand) cand &= cand - 1u;
            const uint64_t p1 = pt_index(l1), p2 = pt_index(l2);
            if (p1 >= g.n_bricks || p2 >= g.n_bricks) {
              *a.err = kErrPageIndex;
            } else {
              const uint32_t e1 = __ldg(a.pt + p1), e2 = l2 != l1 ? __ldg(a.pt + p2) : 0u;
              if (l1 != ld || e1 == 0) {             // the desired brick is absent
                const uint64_t pd = l1 == ld ? p1 : pt_index(ld);
                if (pd >= g.n_bricks) *a.err = kErrPageIndex;
                else a.req[pd] = 1;
              }
              uint32_t e = e1 ? e1 : e2;
              int lf = e1 ? l1 : l2;
              while (e == 0 && cand) {               // further coarser levels, one at a time
                lf = __ffs(cand) - 1;
                cand &= cand - 1u;
                const uint64_t pl = pt_index(lf);
                if (pl >= g.n_bricks) { *a.err = kErrPageIndex; break; }
                e = __ldg(a.pt + pl);
              }
              if (e != 0) {
                if (e - 1 >= g.cache_slots) {
                  *a.err = kErrSlot;
                } else {
                  sel = ((uint32_t)lf << 27) | (e - 1);
                  a.used[e - 1] = 1;
                  found = lf;
                }
              }
            }
          }
        }
      }
      if (cact) s_sel[ch * stride + warp * 32 + src] = sel;
      const unsigned chmask = MP == 32 ? FULL : ((1u << MP) - 1u);
      const uint32_t act = (__ballot_sync(FULL, sel != kSelNone) >> (grp * MP)) & chmask;
      const uint32_t nbrk = __popc((__ballot_sync(FULL, sel != kSelNone && (sel >> 27) != kSelHomog) >> (grp * MP)) & chmask);
#pragma unroll
      for (int o = 1; o < MP; o <<= 1) {
        const int other = __shfl_xor_sync(FULL, found, o);
        found = other < found ? other : found;
      }
      // remember the walk for the tile's other rays when its node lies
      // inside one brick of every usable level
      {
        const int esh = g.D - d;
        const bool keep = gact && !gbad && g.leaf_log2[0] + esh <= g.blog2 + s_lt.lsh[slm][0] &&
                          g.leaf_log2[1] + esh <= g.blog2 + s_lt.lsh[slm][1] &&
                          g.leaf_log2[2] + esh <= g.blog2 + s_lt.lsh[slm][2];
        const unsigned heads = __ballot_sync(FULL, keep && ch == 0);
        // at most kWalkCache groups of a pass store, each in its own entry
        const uint32_t rank = __popc(heads & ((1u << (grp * MP)) - 1u));
        if (keep && rank < (uint32_t)kWalkCache) {
          const uint32_t e = (wc_next + rank) % kWalkCache;
          uint32_t* ent = s_wc + e * kWalkEntry;
          if (cact) ent[5 + ch] = sel;
          if (ch == 0) {
            ent[1] = (uint32_t)jn0; ent[2] = (uint32_t)jn1; ent[3] = (uint32_t)jn2;
            ent[4] = act;
            ent[0] = 1u | ((uint32_t)d << 1) | ((uint32_t)slod << 6) | ((uint32_t)all_skip << 10) |
                     ((uint32_t)(found == 99 ? 31 : found) << 11) | (nbrk << 16) | (svid << 21);
          }
        }
        wc_next = (wc_next + min(__popc(heads), kWalkCache)) % kWalkCache;
        __syncwarp();
      }
      // hand the walk's result to the lanes it was for
      const bool mine = (taken >> lane) & 1u;
      const int from = mine ? __popc(taken & lt_mask) * MP : lane;
      const int oj0 = __shfl_sync(FULL, jn0, from), oj1 = __shfl_sync(FULL, jn1, from),
                oj2 = __shfl_sync(FULL, jn2, from);
      // depth (31: a node index out of range), all-skip, finest level read,
      // brick channels, channel set
      const uint32_t ow = __shfl_sync(FULL, (uint32_t)(gbad ? 31 : d) | ((uint32_t)all_skip << 5) |
                                                ((uint32_t)(found == 99 ? 31 : found) << 6) | (nbrk << 11) |
                                                (act << 16), from);
      const int od = (int)(ow & 31u);
      const bool obad = od == 31;
      const bool oskip = ((ow >> 5) & 1u) != 0;
      const int osel = ((ow >> 6) & 31u) == 31u ? 99 : (int)((ow >> 6) & 31u);
      const uint32_t onb = (ow >> 11) & 31u, oact = ow >> 16;
      (void)slm;
      if (mine) {
        if (obad) {
          *a.err = kErrNodeIndex;
          write_pixel<BPV, DBG>(V, pix, *s_col, h, n_eval, i, n_bs);
          active = false;
        } else {
          const int esh = g.D - od;
          const bool ob = g.leaf_log2[0] + esh <= g.blog2 + s_lt.lsh[lminu][0] &&
                          g.leaf_log2[1] + esh <= g.blog2 + s_lt.lsh[lminu][1] &&
                          g.leaf_log2[2] + esh <= g.blog2 + s_lt.lsh[lminu][2];
          nc.set(od, lod, oskip, ob, osel, onb, s_lt.lstep[osel == 99 ? lminu : osel]);
          nc.jn[0] = oj0; nc.jn[1] = oj1; nc.jn[2] = oj2;
          nc.act = oact;
        }
      }
    }
    __syncwarp();

    // ----------------------------------------- phase 3: skip or evaluate
    if (!active) continue;
    if (nc.all_skip() && V.skip) {
      // first lattice index whose sample lies outside the node (Algorithm 1):
      // estimate from the node box's exit distance, then correct with the
      // same position arithmetic
      const int d = nc.d();
      const Ray r = ray_get();
      float tb = r.t1;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int sh = g.leaf_log2[q] + g.D - d;
        const float lo = (float)(nc.jn[q] << sh), hi = (float)((nc.jn[q] + 1) << sh);
        if (r.d[q] > 0.0f) tb = fminf(tb, __fdiv_rn(hi - r.o[q], r.d[q]));
        else if (r.d[q] < 0.0f) tb = fminf(tb, __fdiv_rn(lo - r.o[q], r.d[q]));
      }
      float fj = ceilf(__fdiv_rn(tb - r.t0, V.dt));
      fj = fminf(fmaxf(fj, (float)(i + 1)), (float)kMaxSamples);
      int j = (int)fj;
      auto inside = [&](int jj) -> bool {
        const float tj = fmaf((float)jj, V.dt, r.t0);
        if (!(tj < r.t1)) return false;
        float xj[3];
        int jc[3];
        position(g, r, tj, xj);
        node_coords(g, d, xj, jc);
        return jc[0] == nc.jn[0] && jc[1] == nc.jn[1] && jc[2] == nc.jn[2];
      };
      while (j < kMaxSamples && inside(j)) ++j;
      while (j > i + 1 && !inside(j - 1)) --j;
      if constexpr (DBG) {
        h = fnv_word(h, (uint32_t)i);
        h = fnv_word(h, 0xFFFFFFFFu);
        h = fnv_word(h, (uint32_t)d);
        h = fnv_word(h, (uint32_t)j);
      }
      atomicAdd(&s_red[warp][4], 1ull);
      atomicAdd(&s_red[warp][5], (unsigned long long)(j - i));
      i = j;
      continue;
    }

    // shade, composite front to back, stop early once transmittance is low
    // step exponent of the finest level read (or desired): the opacity
    // correction and the next lattice index use 2^s
    const int s = nc.step();
    float2 col01 = make_float2(0.0f, 0.0f);
    float col2 = 0.0f, trans = 1.0f;
    const uint32_t nbk = nc.n_brick();
    cnt.homog += __popc(nc.act) - nbk;
    n_bs += nbk;
    // per channel: TF, opacity correction, additive colour (channel order)
    auto add = [&](int c, float val) {
      const float2 tf = s_tf[c];
      const float xq = (val - tf.x) * tf.y;
      // a value at or below the window start maps to knot 0; with a
      // transparent knot 0 the channel adds exactly nothing (a' = 0, q = 1)
      if (!(xq > 0.0f) && ((knot0_clear >> c) & 1u)) return;
      float q, cb;
      float2 rg;
      shade(s_lut + c * 256, xq, s, q, rg, cb);
      const float ap = 1.0f - q;
      col01 = __ffma2_rn(make_float2(ap, ap), rg, col01);
      col2 = fmaf(ap, cb, col2);
      trans = trans * q;
    };
    auto hash_sel = [&](int c, uint32_t sel) {
      if constexpr (DBG) {
        const uint32_t lb = sel >> 27;
        h = fnv_word(h, (uint32_t)i);
        h = fnv_word(h, (uint32_t)c);
        if (lb == kSelHomog) {
          h = fnv_word(h, 0xFFu);
          h = fnv_word(h, 0xFFFFFFFFu);
        } else {
          const uint32_t bx = (uint32_t)(x[0] * pow2f(-(g.blog2 + s_lt.lsh[lb][0]))),
                         by = (uint32_t)(x[1] * pow2f(-(g.blog2 + s_lt.lsh[lb][1]))),
                         bz = (uint32_t)(x[2] * pow2f(-(g.blog2 + s_lt.lsh[lb][2])));
          h = fnv_word(h, lb);
          h = fnv_word(h, ((uint32_t)(c * k + (int)lb) << 24) | (bz << 16) | (by << 8) | bx);
        }
      }
    };
    // two channels per step: both channels' corners are loaded before
    // either is interpolated (a homogeneous channel loads a dummy footprint
    // at the start of slot 0 and takes the node's value)
    int tl = -1;
    TriCoords tc, tcb;
    uint32_t mm = nc.act;
    while (mm) {
      const int ca = __ffs(mm) - 1;
      mm &= mm - 1u;
      const bool two = mm != 0;
      const int cb = two ? __ffs(mm) - 1 : ca;
      if (two) mm &= mm - 1u;
      const uint32_t sa = my_sel[ca * stride], sb = two ? my_sel[cb * stride] : sa;
      const uint32_t la = sa >> 27, lb = sb >> 27;
      const bool ha = BPV == 1 && la == kSelHomog, hb = BPV == 1 && lb == kSelHomog;
      if (!ha && (int)la != tl) {  // channels at one level share the corner offset and weights
        tl = (int)la;
        tri_coords<EC, SF>(g, s_lt, tl, x, tc);
      }
      if (!hb && lb != la) tri_coords<EC, SF>(g, s_lt, (int)lb, x, tcb);
      else tcb = tc;
      uint32_t ra[8], rb[8];
      tri_load<BPV, EC, SF>(g, a.cache + (ha ? 0 : (size_t)(sa & kSelMask) * g.slot_pitch), ha ? 0 : tc.idx, ra);
      tri_load<BPV, EC, SF>(g, a.cache + (hb ? 0 : (size_t)(sb & kSelMask) * g.slot_pitch), hb ? 0 : tcb.idx, rb);
      const float va = ha ? (float)(sa & kSelMask) : tri_lerp<BPV, SF>(ra, tc);
      hash_sel(ca, sa);
      add(ca, va);
      if (two) {
        const float vb = hb ? (float)(sb & kSelMask) : tri_lerp<BPV, SF>(rb, tcb);
        hash_sel(cb, sb);
        add(cb, vb);
      }
    }
    float4 cc = *s_col;                     // (C0, C1, C2, T)
    cc.x = fmaf(cc.w, col01.x, cc.x);
    cc.y = fmaf(cc.w, col01.y, cc.y);
    cc.z = fmaf(cc.w, col2, cc.z);
    cc.w = cc.w * trans;
    *s_col = cc;
    ++n_eval;
    if (cc.w < V.ert) {
      write_pixel<BPV, DBG>(V, pix, cc, h, n_eval, i, n_bs);
      active = false;
      continue;
    }
    i += 1 << s;
  }

  // per-block counters, reduced without atomics
  flush();
  __syncthreads();
  if (threadIdx.x < kStats) {
    unsigned long long v = 0;
    for (int q = 0; q < kThreads / 32 * kUnits; ++q) v += s_red[q][threadIdx.x];
    a.block_stats[(size_t)blockIdx.x * kStats + threadIdx.x] = v;
  }
}

template <int MP, int BPV, int EC, bool DBG, bool BATCH, int SF>
cudaError_t launch_one(const RenderArgs& a, cudaStream_t s, int* blocks_out) {
  const size_t smem = render_smem_bytes(MP, BATCH);
  auto kern = render_kernel<MP, BPV, EC, DBG, BATCH, SF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  constexpr int kThreads = render_threads(BATCH);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t need = (a.n_rays + kThreads - 1) / kThreads;
  int blocks = sms * per_sm;
  if ((uint64_t)blocks > need) blocks = (int)need;
  kern<<<blocks, kThreads, smem, s>>>(a);
  *blocks_out = blocks;
  return cudaGetLastError();
}

template <int MP, int BPV, int EC, bool BATCH, int SF>
cudaError_t launch_ec(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  return debug ? launch_one<MP, BPV, EC, true, BATCH, SF>(a, s, blocks_out) : launch_one<MP, BPV, EC, false, BATCH, SF>(a, s, blocks_out);
}

template <int MP, int BPV, bool BATCH, int SF>
cudaError_t launch_mp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  return a.g.edge == 34 ? launch_ec<MP, BPV, 34, BATCH, SF>(a, debug, s, blocks_out) : launch_ec<MP, BPV, 0, BATCH, SF>(a, debug, s, blocks_out);
}

template <int MP, bool BATCH, int SF>
cudaError_t launch_bpv(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  return a.g.bpv == 1 ? launch_mp<MP, 1, BATCH, SF>(a, debug, s, blocks_out) : launch_mp<MP, 2, BATCH, SF>(a, debug, s, blocks_out);
}

template <bool BATCH, int SF>
cudaError_t launch_any(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  switch (a.g.mp) {
    case 1: return launch_bpv<1, BATCH, SF>(a, debug, s, blocks_out);
    case 2: return launch_bpv<2, BATCH, SF>(a, debug, s, blocks_out);
    case 4: return launch_bpv<4, BATCH, SF>(a, debug, s, blocks_out);
    case 8: return launch_bpv<8, BATCH, SF>(a, debug, s, blocks_out);
    case 16: return launch_bpv<16, BATCH, SF>(a, debug, s, blocks_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace ro
