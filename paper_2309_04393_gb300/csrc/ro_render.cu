// Mixed-resolution multi-volume ray caster through the residency octree
// (Sec. 6.1, Algorithm 1 and the multi-channel walk; Sec. 6.2; Sec. 7).
//
// One thread per pixel, 16 x 16 pixels per block (8 x 4 per warp).  The
// channels' transfer-function LUTs and bucket-occupancy prefix sums live in
// shared memory; node words, page-table entries and brick-cache voxels are
// read through the read-only path.  Requests and usage are emitted with plain
// byte stores of 1 (idempotent: no atomics).  Every decision is taken in
// binary32 with the operation order of the design contract (built with
// --fmad=false: every fused multiply-add below is an explicit fmaf).
#include "ro_internal.h"

namespace ro {
namespace {

enum : int { kEmpty = 0, kHomog = 1, kUnmapped = 2, kBrick = 3, kInvalid = 4 };

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

template <int MP>
__device__ __forceinline__ void load_words(const uint32_t* __restrict__ oct, uint64_t node, int m, uint32_t (&w)[MP]) {
  const uint32_t* p = oct + node * MP;
  if constexpr (MP >= 4) {
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + q);
      w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
  } else if constexpr (MP == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = v.x; w[1] = v.y;
  } else {
    w[0] = __ldg(p);
  }
  (void)m;
}

struct Ray {
  float o[3], d[3];
  float t0, t1;
  bool hit;
};

// Pixel-centre ray, voxel-space origin/direction and slab interval (R17).
__device__ Ray make_ray(const RenderArgs& a, int px, int py) {
  Ray r;
  float o[3], d[3];
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  if (a.persp) {
    const float u = __fdiv_rn(fx, (float)a.W), w = __fdiv_rn(fy, (float)a.H);
    const float sa = (2.0f * u - 1.0f) * a.tan_x;
    const float sb = (1.0f - 2.0f * w) * a.tan_y;
    float dd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] = fmaf(sb, a.up[k], fmaf(sa, a.right[k], a.fwd[k]));
    const float n2 = fmaf(dd[2], dd[2], fmaf(dd[1], dd[1], dd[0] * dd[0]));
    const float len = __fsqrt_rn(n2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = a.eye[k];
      d[k] = __fdiv_rn(dd[k], len);
    }
  } else {
    const float sa = (fx - 0.5f * (float)a.W) * a.pixel;
    const float sb = (0.5f * (float)a.H - fy) * a.pixel;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = fmaf(sb, a.up[k], fmaf(sa, a.right[k], a.eye[k]));
      d[k] = a.fwd[k];
    }
  }
  float tmin = -INFINITY, tmax = INFINITY;
  r.hit = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.o[k] = __fdiv_rn(o[k], a.g.spacing[k]);
    r.d[k] = __fdiv_rn(d[k], a.g.spacing[k]);
    if (r.d[k] != 0.0f) {
      const float ta = __fdiv_rn(0.0f - r.o[k], r.d[k]);
      const float tb = __fdiv_rn((float)a.g.dims0[k] - r.o[k], r.d[k]);
      tmin = fmaxf(tmin, fminf(ta, tb));
      tmax = fminf(tmax, fmaxf(ta, tb));
    } else if (r.o[k] < 0.0f || r.o[k] >= (float)a.g.dims0[k]) {
      r.hit = false;
    }
  }
  r.t0 = fmaxf(tmin, 0.0f);
  r.t1 = tmax;
  if (!(r.t0 < r.t1)) r.hit = false;
  return r;
}

__device__ __forceinline__ void position(const RenderArgs& a, const Ray& r, float t, float (&x)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = fminf(fmaxf(fmaf(t, r.d[k], r.o[k]), 0.0f), a.g.dimm[k]);
}

__device__ __forceinline__ void node_coords(const Geometry& g, int d, const float (&x)[3], int (&j)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) j[k] = (int)(x[k] * pow2f(-(g.leaf_log2[k] + g.D - d)));
}

// Trilinear sample of a level-l apron slot (R15): corners are read from the
// owner's slot, lerps along x, then y, then z.
template <int BPV>
__device__ __forceinline__ float trilinear(const RenderArgs& a, uint32_t slot, int l, const float (&x)[3]) {
  const Geometry& g = a.g;
  const int E = (int)g.edge;
  int li[3];
  float f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float xl = x[k] * pow2f(-l);
    float u = xl - 0.5f;
    u = fminf(fmaxf(u, 0.0f), (float)(g.ldims[l][k] - 1));
    const int i0 = (int)u;
    f[k] = u - (float)i0;
    const int b = (int)(x[k] * pow2f(-(g.blog2 + l)));
    li[k] = i0 - (b * g.B - 1);
  }
  const size_t base = (size_t)slot * g.slot_pitch;
  const int idx = (li[2] * E + li[1]) * E + li[0];
  float v[8];
  if constexpr (BPV == 1) {
    const uint8_t* p = a.cache + base + idx;
    v[0] = (float)__ldg(p);
    v[1] = (float)__ldg(p + 1);
    v[2] = (float)__ldg(p + E);
    v[3] = (float)__ldg(p + E + 1);
    v[4] = (float)__ldg(p + E * E);
    v[5] = (float)__ldg(p + E * E + 1);
    v[6] = (float)__ldg(p + E * E + E);
    v[7] = (float)__ldg(p + E * E + E + 1);
  } else {
    const uint16_t* p = reinterpret_cast<const uint16_t*>(a.cache + base) + idx;
    v[0] = (float)__ldg(p);
    v[1] = (float)__ldg(p + 1);
    v[2] = (float)__ldg(p + E);
    v[3] = (float)__ldg(p + E + 1);
    v[4] = (float)__ldg(p + E * E);
    v[5] = (float)__ldg(p + E * E + 1);
    v[6] = (float)__ldg(p + E * E + E);
    v[7] = (float)__ldg(p + E * E + E + 1);
  }
  const float c00 = fmaf(f[0], v[1] - v[0], v[0]);
  const float c10 = fmaf(f[0], v[3] - v[2], v[2]);
  const float c01 = fmaf(f[0], v[5] - v[4], v[4]);
  const float c11 = fmaf(f[0], v[7] - v[6], v[6]);
  const float c0 = fmaf(f[1], c10 - c00, c00);
  const float c1 = fmaf(f[1], c11 - c01, c01);
  return fmaf(f[2], c1 - c0, c0);
}

// TF lookup (R16) and opacity correction for a step of 2^s (R12): returns
// the corrected opacity's complement q and the colour.
__device__ __forceinline__ void shade(const RenderArgs& a, const float4* __restrict__ lut, int c, float val, int s,
                                      float& q, float& r, float& gg, float& b) {
  const float t = val - a.tf_lo[c];
  float xq = t * a.tf_scale[c];
  xq = fminf(fmaxf(xq, 0.0f), 255.0f);
  int j = (int)xq;
  j = j > 254 ? 254 : j;
  const float fr = xq - (float)j;
  const float4 L0 = lut[j], L1 = lut[j + 1];
  r = fmaf(fr, L1.x - L0.x, L0.x);
  gg = fmaf(fr, L1.y - L0.y, L0.y);
  b = fmaf(fr, L1.z - L0.z, L0.z);
  float al = fmaf(fr, L1.w - L0.w, L0.w);
  al = fminf(fmaxf(al, 0.0f), 1.0f);
  q = 1.0f - al;
  for (int e = 0; e < s; ++e) q = q * q;
}

// Per-ray cache of the last classification: the final node, the desired
// levels it was made for and each channel's state.  A sample that lands in
// the same node with the same desired levels gets the same decisions (the
// walk, the states, the selected slots and levels), provided the node lies
// inside one brick of every level a channel may use; requests and usage flags
// are then already set (the stores are idempotent).
struct NodeCache {
  int d;                 // final depth, -1 = empty
  int jn[3];             // node coordinates at depth d
  uint64_t ldp;          // desired levels (4 bits per channel)
  int st;                // traversal depth
  bool all_skip, one_brick;
  int s_sel;             // finest level read from a brick, 99 = none
};

// Per-lane selection word (one per channel, in shared memory): bits 31..27
// the level read (0..15) or kSelHomog, bits 26..0 the slot or the node value.
constexpr uint32_t kSelNone = 0xFFFFFFFFu;
constexpr uint32_t kSelHomog = 30u;
constexpr uint32_t kSelMask = (1u << 27) - 1u;

struct RayState {
  Ray r;
  int px, py, i;
  float C0, C1, C2, T;
  uint32_t h, n_eval, n_bs;
  NodeCache nc;
};

struct Counters {
  unsigned long long hit, eval, bs, homog, skip, skipped;
};

// One lattice step of one ray (one evaluated sample, or one skip).  Returns
// true once the ray is finished (left the volume, terminated early, or hit a
// guard).
template <int MP, int BPV, bool DBG>
__device__ __forceinline__ bool ray_step(const RenderArgs& a, const float4* __restrict__ s_lut,
                                         const uint16_t* __restrict__ s_pre, uint32_t* my_sel, int stride,
                                         RayState& R, Counters& cnt) {
  const Geometry& g = a.g;
  const int m = g.m, k = g.k;
  if (R.i >= kMaxSamples) return true;
  const float t = fmaf((float)R.i, a.dt, R.r.t0);
  if (!(t < R.r.t1)) return true;
  float x[3];
  position(a, R.r, t, x);

  // desired level per channel (R7), packed 4 bits per channel
  int lod = 0;
  for (int l = 1; l < k; ++l) lod += (t >= a.lod_t[l]);
  uint64_t ldp = 0;
  int lminu = 15;
#pragma unroll 1
  for (int c = 0; c < m; ++c) {
    int l = lod < a.lmin[c] ? a.lmin[c] : lod;
    l = l > a.lmax[c] ? a.lmax[c] : l;
    ldp |= (uint64_t)l << (4 * c);
    lminu = l < lminu ? l : lminu;
  }
  const int st = a.sdepth[lminu];
  int L[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) L[q] = (int)(x[q] * pow2f(-g.leaf_log2[q]));
  NodeCache& nc = R.nc;
  const bool same_levels = nc.d >= 0 && ldp == nc.ldp && st == nc.st;
  bool same_node = false;
  if (same_levels) {
    const int sh = g.D - nc.d;
    same_node = (L[0] >> sh) == nc.jn[0] && (L[1] >> sh) == nc.jn[1] && (L[2] >> sh) == nc.jn[2];
  }

  if (!(same_node && nc.one_brick)) {
    // walk (R9); depths whose nodes the previous sample shared and found not
    // all terminal are not visited again
    const int d0 = a.start_depth < st ? a.start_depth : st;
    int d = d0;
    if (same_node) {
      d = nc.d;
    } else if (same_levels) {
      int dca = 0;
      for (int q = nc.d; q >= 0; --q) {
        const int sh = g.D - q, up = nc.d - q;
        if ((L[0] >> sh) == (nc.jn[0] >> up) && (L[1] >> sh) == (nc.jn[1] >> up) && (L[2] >> sh) == (nc.jn[2] >> up)) {
          dca = q;
          break;
        }
      }
      d = dca + 1 > d0 ? dca + 1 : d0;
    }
    int jn[3];
    uint64_t node, states;
    for (;;) {
      const int sh = g.D - d;
      jn[0] = L[0] >> sh; jn[1] = L[1] >> sh; jn[2] = L[2] >> sh;
      node = g.node_off[d] + ((uint64_t)jn[2] * g.nn[d][1] + jn[1]) * g.nn[d][0] + jn[0];
      if (node >= g.node_off[d + 1]) { *a.err = kErrNodeIndex; return true; }
      const uint32_t* wp = a.octree + node * MP;
      bool all = true;
      states = 0;
#pragma unroll 1
      for (int c = 0; c < m; ++c) {
        const int sc = classify<BPV>(__ldg(wp + c), s_pre + c * 257, (int)((ldp >> (4 * c)) & 15), k);
        states |= (uint64_t)sc << (4 * c);
        all = all && terminal(sc);
      }
      if (all || d == st || same_node) break;
      ++d;
    }

    // requests of channels with nothing usable here, node requests of INVALID
    // channels, then brick selection (R11): desired level, else request it
    // and take the next coarser resident level
    const uint32_t* wp = a.octree + node * MP;
    bool all_skip = true;
    int s_sel = 99;
#pragma unroll 1
    for (int c = 0; c < m; ++c) {
      const uint32_t w = __ldg(wp + c);
      const int ld = (int)((ldp >> (4 * c)) & 15);
      const int sc = (int)((states >> (4 * c)) & 15);
      if (sc != kEmpty && sc != kUnmapped) all_skip = false;
      const bool no_use = ((w & 0xFFFFu) & (~0u << ld) & ((1u << k) - 1u)) == 0;
      if (sc == kUnmapped || (sc == kInvalid && no_use)) {
        const int bsh = g.blog2 + ld;
        const int bx = (int)(x[0] * pow2f(-bsh)), by = (int)(x[1] * pow2f(-bsh)), bz = (int)(x[2] * pow2f(-bsh));
        const uint64_t pi = g.pt_off[c * k + ld] + ((uint64_t)bz * g.nb[ld][1] + by) * g.nb[ld][0] + bx;
        if (pi >= g.n_bricks) { *a.err = kErrPageIndex; return true; }
        a.req[pi] = 1;
      }
      if (sc == kInvalid) a.node_req[node * m + c] = 1;
    }
#pragma unroll 1
    for (int c = 0; c < m; ++c) {
      uint32_t sel = kSelNone;
      const int sc = (int)((states >> (4 * c)) & 15);
      if (!all_skip && sc != kEmpty && sc != kUnmapped) {
        const uint32_t w = __ldg(wp + c);
        if (sc == kHomog) {
          sel = (kSelHomog << 27) | ((w >> 16) & 0xFFu);
        } else {
          const int ld = (int)((ldp >> (4 * c)) & 15);
          if (((w & 0xFFFFu) & (~0u << ld) & ((1u << k) - 1u)) != 0) {
            for (int l = ld; l < k; ++l) {
              const int bsh = g.blog2 + l;
              const int bx = (int)(x[0] * pow2f(-bsh)), by = (int)(x[1] * pow2f(-bsh)), bz = (int)(x[2] * pow2f(-bsh));
              const uint64_t pi = g.pt_off[c * k + l] + ((uint64_t)bz * g.nb[l][1] + by) * g.nb[l][0] + bx;
              if (pi >= g.n_bricks) { *a.err = kErrPageIndex; return true; }
              uint32_t e = 0;
              if ((w >> l) & 1u) e = __ldg(a.pt + pi);
              if (e != 0) {
                if (e - 1 >= g.cache_slots) { *a.err = kErrSlot; return true; }
                sel = ((uint32_t)l << 27) | (e - 1);
                a.used[e - 1] = 1;
                s_sel = l < s_sel ? l : s_sel;
                break;
              }
              if (l == ld) a.req[pi] = 1;
            }
          }
        }
      }
      my_sel[c * stride] = sel;
    }
    nc.d = d;
    nc.jn[0] = jn[0]; nc.jn[1] = jn[1]; nc.jn[2] = jn[2];
    nc.ldp = ldp;
    nc.st = st;
    nc.all_skip = all_skip;
    nc.s_sel = s_sel;
    const int esh = g.D - d;
    nc.one_brick = g.leaf_log2[0] + esh <= g.blog2 + lminu && g.leaf_log2[1] + esh <= g.blog2 + lminu &&
                   g.leaf_log2[2] + esh <= g.blog2 + lminu;
  }

  if (nc.all_skip && a.skip) {
    // first lattice index whose sample lies outside the node (R10): estimate
    // from the node box's exit distance, then correct with the same position
    // arithmetic
    const int d = nc.d;
    float tb = R.r.t1;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int sh = g.leaf_log2[q] + g.D - d;
      const float lo = (float)(nc.jn[q] << sh), hi = (float)((nc.jn[q] + 1) << sh);
      if (R.r.d[q] > 0.0f) tb = fminf(tb, __fdiv_rn(hi - R.r.o[q], R.r.d[q]));
      else if (R.r.d[q] < 0.0f) tb = fminf(tb, __fdiv_rn(lo - R.r.o[q], R.r.d[q]));
    }
    float fj = ceilf(__fdiv_rn(tb - R.r.t0, a.dt));
    fj = fminf(fmaxf(fj, (float)(R.i + 1)), (float)kMaxSamples);
    int j = (int)fj;
    auto inside = [&](int jj) -> bool {
      const float tj = fmaf((float)jj, a.dt, R.r.t0);
      if (!(tj < R.r.t1)) return false;
      float xj[3];
      int jc[3];
      position(a, R.r, tj, xj);
      node_coords(g, d, xj, jc);
      return jc[0] == nc.jn[0] && jc[1] == nc.jn[1] && jc[2] == nc.jn[2];
    };
    while (j < kMaxSamples && inside(j)) ++j;
    while (j > R.i + 1 && !inside(j - 1)) --j;
    if constexpr (DBG) {
      R.h = fnv_word(R.h, (uint32_t)R.i);
      R.h = fnv_word(R.h, 0xFFFFFFFFu);
      R.h = fnv_word(R.h, (uint32_t)d);
      R.h = fnv_word(R.h, (uint32_t)j);
    }
    ++cnt.skip;
    cnt.skipped += (unsigned long long)(j - R.i);
    R.i = j;
    return false;
  }

  // shade and composite (R12-R14)
  const int s = nc.s_sel == 99 ? lminu : nc.s_sel;
  float col0 = 0.0f, col1 = 0.0f, col2 = 0.0f, trans = 1.0f;
#pragma unroll 1
  for (int c = 0; c < m; ++c) {
    const uint32_t sel = my_sel[c * stride];
    if (sel == kSelNone) continue;
    const uint32_t lb = sel >> 27;
    float val;
    if (lb == kSelHomog) {
      val = (float)(sel & kSelMask);
      ++cnt.homog;
      if constexpr (DBG) {
        R.h = fnv_word(R.h, (uint32_t)R.i); R.h = fnv_word(R.h, (uint32_t)c);
        R.h = fnv_word(R.h, 0xFFu); R.h = fnv_word(R.h, 0xFFFFFFFFu);
      }
    } else {
      val = trilinear<BPV>(a, sel & kSelMask, (int)lb, x);
      ++cnt.bs;
      ++R.n_bs;
      if constexpr (DBG) {
        const int bsh = g.blog2 + (int)lb;
        const uint32_t bx = (uint32_t)(x[0] * pow2f(-bsh)), by = (uint32_t)(x[1] * pow2f(-bsh)),
                       bz = (uint32_t)(x[2] * pow2f(-bsh));
        R.h = fnv_word(R.h, (uint32_t)R.i); R.h = fnv_word(R.h, (uint32_t)c); R.h = fnv_word(R.h, lb);
        R.h = fnv_word(R.h, ((uint32_t)(c * k + (int)lb) << 24) | (bz << 16) | (by << 8) | bx);
      }
    }
    float q, cr, cg, cb;
    shade(a, s_lut + c * 256, c, val, s, q, cr, cg, cb);
    const float ap = 1.0f - q;
    col0 = fmaf(ap, cr, col0);
    col1 = fmaf(ap, cg, col1);
    col2 = fmaf(ap, cb, col2);
    trans = trans * q;
  }
  R.C0 = fmaf(R.T, col0, R.C0);
  R.C1 = fmaf(R.T, col1, R.C1);
  R.C2 = fmaf(R.T, col2, R.C2);
  R.T = R.T * trans;
  ++R.n_eval;
  ++cnt.eval;
  if (R.T < a.ert) return true;
  R.i += 1 << s;
  return false;
}

template <int BPV, bool DBG>
__device__ __forceinline__ void finish_ray(const RenderArgs& a, const RayState& R) {
  const size_t p = (size_t)R.py * a.W + R.px;
  a.image[p] = make_float4(fminf(R.C0, 1.0f), fminf(R.C1, 1.0f), fminf(R.C2, 1.0f), 1.0f - R.T);
  if constexpr (DBG) {
    if (a.dbg_hash) a.dbg_hash[p] = R.h;
    if (a.dbg_n_eval) a.dbg_n_eval[p] = R.n_eval;
    if (a.dbg_i_end) a.dbg_i_end[p] = (uint32_t)R.i;
    if (a.dbg_n_bs) a.dbg_n_bs[p] = R.n_bs;
  }
}

// Persistent launch: every lane takes the next ray from a shared counter (in
// 8 x 4 pixel tiles, warp-aggregated) whenever its previous ray is finished,
// so lanes stay busy however long individual rays run.
template <int MP, int BPV, bool DBG>
__global__ void __launch_bounds__(kRenderThreads, 2) render_kernel(const __grid_constant__ RenderArgs a) {
  extern __shared__ float4 smem[];
  float4* s_lut = smem;
  uint16_t* s_pre = reinterpret_cast<uint16_t*>(s_lut + MP * 256);
  uint32_t* s_sel = reinterpret_cast<uint32_t*>(smem) + MP * 256 * 4 + ((MP * 257 * 2 + 15) & ~15) / 4;
  const int m = a.g.m;
  for (int i = threadIdx.x; i < m * 256; i += blockDim.x) s_lut[i] = a.lut[i];
  for (int i = threadIdx.x; i < m * 257; i += blockDim.x) s_pre[i] = a.prefix[i];
  __syncthreads();

  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* my_sel = s_sel + threadIdx.x;
  const int stride = blockDim.x;
  Counters cnt = {0, 0, 0, 0, 0, 0};
  RayState R;
  bool active = false, done = false;
  for (;;) {
    const unsigned need = __ballot_sync(FULL, !active && !done);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(a.work, (unsigned long long)__popc(need));
      base = __shfl_sync(FULL, base, leader);
      if (!active && !done) {
        const unsigned long long ray = base + __popc(need & ((1u << lane) - 1u));
        if (ray >= a.n_rays) {
          done = true;
        } else {
          const uint32_t tile = (uint32_t)(ray >> 5), w = (uint32_t)(ray & 31);
          R.px = (int)((tile % a.tiles_x) * 8 + (w & 7));
          R.py = (int)((tile / a.tiles_x) * 4 + (w >> 3));
          if (R.px < a.W && R.py < a.H) {
            R.r = make_ray(a, R.px, R.py);
            R.i = 0;
            R.C0 = R.C1 = R.C2 = 0.0f;
            R.T = 1.0f;
            R.h = 2166136261u;
            R.n_eval = R.n_bs = 0;
            R.nc.d = -1;
            if (R.r.hit) {
              active = true;
              ++cnt.hit;
            } else {
              finish_ray<BPV, DBG>(a, R);
            }
          }
        }
      }
    }
    if (__all_sync(FULL, done)) break;
    if (active && ray_step<MP, BPV, DBG>(a, s_lut, s_pre, my_sel, stride, R, cnt)) {
      finish_ray<BPV, DBG>(a, R);
      active = false;
    }
  }

  // per-block counters, reduced without atomics
  __shared__ unsigned long long s_red[kRenderThreads / 32][kStats];
  unsigned long long vals[kStats] = {cnt.hit, cnt.eval, cnt.bs, cnt.homog, cnt.skip, cnt.skipped, 0, 0};
#pragma unroll
  for (int q = 0; q < kStats; ++q) {
    unsigned long long v = vals[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (lane == 0) s_red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < kStats) {
    unsigned long long v = 0;
    for (int q = 0; q < kRenderThreads / 32; ++q) v += s_red[q][threadIdx.x];
    a.block_stats[(size_t)blockIdx.x * kStats + threadIdx.x] = v;
  }
}

// Bucket-occupancy prefix sums per channel (R5): one block per channel.
__global__ void __launch_bounds__(256) prefix_kernel(const __grid_constant__ PrefixArgs a) {
  __shared__ uint16_t s_occ[256];
  __shared__ uint16_t s_scan[257];
  const int c = blockIdx.x, q = threadIdx.x;
  const float4* L = a.lut + c * 256;
  float vlo, vhi;
  if (a.bpv == 1) { vlo = (float)q; vhi = (float)q; }
  else { vlo = (float)(q * 256); vhi = (float)(q * 256 + 255); }
  auto coord = [&](float v) {
    const float t = v - a.tf_lo[c];
    const float xq = t * a.tf_scale[c];
    return fminf(fmaxf(xq, 0.0f), 255.0f);
  };
  const float xa = coord(vlo), xb = coord(vhi);
  const float x0 = fminf(xa, xb), x1 = fmaxf(xa, xb);
  const int j0 = (int)floorf(x0);
  int j1 = (int)ceilf(x1);
  j1 = j1 > 255 ? 255 : j1;
  int occ = 0;
  for (int j = j0; j <= j1; ++j) occ |= L[j].w > 0.0f;
  s_occ[q] = (uint16_t)occ;
  __syncthreads();
  if (q == 0) {
    uint16_t run = 0;
    s_scan[0] = 0;
    for (int b = 0; b < 256; ++b) { run = (uint16_t)(run + s_occ[b]); s_scan[b + 1] = run; }
  }
  __syncthreads();
  a.prefix[c * 257 + q] = s_scan[q];
  if (q == 0) a.prefix[c * 257 + 256] = s_scan[256];
}

template <int MP, int BPV, bool DBG>
cudaError_t launch_one(const RenderArgs& a, cudaStream_t s, int* blocks_out) {
  const size_t smem = render_smem_bytes(MP);
  auto kern = render_kernel<MP, BPV, DBG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRenderThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t need = (a.n_rays + kRenderThreads - 1) / kRenderThreads;
  int blocks = sms * per_sm;
  if ((uint64_t)blocks > need) blocks = (int)need;
  kern<<<blocks, kRenderThreads, smem, s>>>(a);
  *blocks_out = blocks;
  return cudaGetLastError();
}

template <int MP, int BPV>
cudaError_t launch_mp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  return debug ? launch_one<MP, BPV, true>(a, s, blocks_out) : launch_one<MP, BPV, false>(a, s, blocks_out);
}

template <int MP>
cudaError_t launch_bpv(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  return a.g.bpv == 1 ? launch_mp<MP, 1>(a, debug, s, blocks_out) : launch_mp<MP, 2>(a, debug, s, blocks_out);
}

}  // namespace

size_t render_smem_bytes(int mp) {
  return (size_t)mp * 256 * sizeof(float4) + (((size_t)mp * 257 * 2 + 15) & ~(size_t)15) +
         (size_t)mp * kRenderThreads * sizeof(uint32_t);
}

cudaError_t launch_render(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  switch (a.g.mp) {
    case 1: return launch_bpv<1>(a, debug, s, blocks_out);
    case 2: return launch_bpv<2>(a, debug, s, blocks_out);
    case 4: return launch_bpv<4>(a, debug, s, blocks_out);
    case 8: return launch_bpv<8>(a, debug, s, blocks_out);
    case 16: return launch_bpv<16>(a, debug, s, blocks_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prefix(const PrefixArgs& a, cudaStream_t s) {
  prefix_kernel<<<a.m, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ro
