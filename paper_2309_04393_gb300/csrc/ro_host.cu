// Host side of the C ABI (include/ro.h): descriptor validation, device-arena
// layout, the LRU slot policy (Sec. 5.3), update item lists, frame constants,
// and the bounded waits on the context's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "ro.h"
#include "ro_internal.h"
#include "ro_mc.h"

using ro::Geometry;

namespace {

constexpr uint64_t kAlign = 256;
constexpr uint32_t kMaxItems = 65536;           // update items per chunk
constexpr uint32_t kMaxStatBlocks = 65536;      // render blocks whose counters are kept
constexpr uint32_t kItemLeaves = 4096;          // leaves per update item (boxes are split)

uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

bool is_pow2(uint32_t v) { return v && !(v & (v - 1)); }

int ilog2(uint32_t v) {
  int r = 0;
  while ((1u << r) < v) ++r;
  return r;
}

constexpr int kParts = 12;

struct Layout {
  uint64_t off[kParts];
  ro_buffer_sizes sz;
  uint64_t req_pad, node_req_pad, used_pad;
  uint64_t sc_counts, sc_totals, sc_items, sc_meta, sc_ins_index, sc_ins_slot, sc_ev_index, sc_stats, sc_err, sc_work;
  uint64_t fr_lut, fr_prefix, li_req, li_node;
  uint64_t oc_given;                             // octree part: ranges given for inner nodes after the words
  uint64_t ba_views, ba_tf, ba_order, ba_cost;   // batch region: view table, TF ranges, schedule, tile costs
  uint32_t max_tiles;
};

std::string g_create_error = "ok";

ro_status make_geometry(const ro_desc* d, Geometry* g, std::string* why) {
  auto fail = [&](const char* m) {
    *why = m;
    return RO_ERR_INVALID_ARG;
  };
  if (!d) return fail("null descriptor");
  std::memset(g, 0, sizeof(*g));
  for (int a = 0; a < 3; ++a) {
    if (d->dims[a] < 1 || d->dims[a] > (1u << 24)) return fail("dims must be in [1, 2^24]");
    if (!(d->spacing[a] > 0.0f) || !std::isfinite(d->spacing[a])) return fail("spacing must be positive and finite");
  }
  if (d->channels < 1 || d->channels > RO_MAX_CHANNELS) return fail("channels must be in [1, 16]");
  if (d->value_bits != 8 && d->value_bits != 16) return fail("value_bits must be 8 or 16");
  if (d->brick != 8 && d->brick != 16 && d->brick != 32 && d->brick != 64) return fail("brick must be 8, 16, 32 or 64");
  if (d->levels < 1 || d->levels > RO_MAX_LEVELS) return fail("levels must be in [1, 16]");
  if (d->channels * d->levels > 256) return fail("channels * levels must be <= 256 (8-bit page-table id)");
  for (int a = 0; a < 3; ++a)
    if (!is_pow2(d->leaf_extent[a]) || d->leaf_extent[a] > d->brick) return fail("leaf_extent must be powers of two <= brick");
  if (d->cache_slots < 1 || d->cache_slots > (1u << 27)) return fail("cache_slots must be in [1, 2^27]");
  if (d->max_requests < 1 || d->max_upload < 1 || d->max_meta < 1) return fail("max_requests/max_upload/max_meta must be >= 1");
  g->m = (int)d->channels;
  g->mp = 1;
  while (g->mp < g->m) g->mp <<= 1;
  g->k = (int)d->levels;
  g->B = (int)d->brick;
  g->blog2 = ilog2(d->brick);
  g->bpv = d->value_bits / 8;
  if (d->sample_format > 2) return fail("sample_format must be 0, 1 or 2");
  g->sf = (int)d->sample_format;
  g->cbpv = g->sf ? 2 : g->bpv;
  g->edge = d->brick + 2;
  g->cache_slots = d->cache_slots;
  for (int a = 0; a < 3; ++a) {
    g->dims0[a] = (int)d->dims[a];
    g->spacing[a] = d->spacing[a];
    g->dimm[a] = std::nextafter((float)d->dims[a], 0.0f);
    g->leaf_log2[a] = ilog2(d->leaf_extent[a]);
  }
  for (int l = 0; l < RO_MAX_LEVELS; ++l)
    if (d->keep_axes[l] > 7 || (l >= g->k - 1 && d->keep_axes[l] != 0))
      return fail("keep_axes: three axis bits per level transition, zero beyond the last level");
  // level geometry per axis: an axis not kept is halved (rounding up)
  for (int l = 0; l < ro::kMaxL; ++l) {
    double s0 = INFINITY, sl = INFINITY;
    for (int a = 0; a < 3; ++a) {
      int sh = 0;
      for (int q = 0; q < l; ++q) sh += (d->keep_axes[q] >> a) & 1 ? 0 : 1;
      g->lsh[l][a] = sh;
      s0 = std::min(s0, (double)d->spacing[a]);
      sl = std::min(sl, (double)d->spacing[a] * std::ldexp(1.0, sh));
    }
    // step exponent: largest s with 2^s min(spacing) <= the smallest extent of a level-l voxel
    int s = 0;
    while (std::ldexp(s0, s + 1) <= sl) ++s;
    g->lstep[l] = s;
  }
  for (int l = 0; l < g->k; ++l)
    for (int a = 0; a < 3; ++a) {
      int v = g->dims0[a];
      for (int q = 0; q < l; ++q)
        if (!((d->keep_axes[q] >> a) & 1)) v = (v + 1) / 2;
      g->ldims[l][a] = v;
      g->ldimf[l][a] = (float)(v - 1);
      g->nb[l][a] = (v + g->B - 1) / g->B;
      if (g->nb[l][a] > 256) return fail("more than 256 bricks per axis (8-bit brick offsets)");
    }
  uint64_t off = 0;
  for (int c = 0; c < g->m; ++c)
    for (int l = 0; l < g->k; ++l) {
      g->pt_off[c * g->k + l] = (uint32_t)off;
      off += (uint64_t)g->nb[l][0] * g->nb[l][1] * g->nb[l][2];
      if (off >= 0xFFFFFFFFull) return fail("too many bricks");
    }
  g->pt_off[g->m * g->k] = (uint32_t)off;
  g->n_bricks = off;
  int D = 0;
  for (int a = 0; a < 3; ++a) {
    const int nl = (g->dims0[a] + (int)d->leaf_extent[a] - 1) / (int)d->leaf_extent[a];
    g->nleaf[a] = nl;
    D = std::max(D, ilog2((uint32_t)nl));
  }
  if (D > ro::kMaxDepth) return fail("octree too deep");
  g->D = D;
  uint64_t noff = 0;
  for (int dd = 0; dd <= D; ++dd) {
    g->node_off[dd] = noff;
    uint64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const uint64_t e = (uint64_t)d->leaf_extent[a] << (D - dd);
      g->nn[dd][a] = (int)((g->dims0[a] + e - 1) / e);
      cnt *= (uint64_t)g->nn[dd][a];
    }
    noff += cnt;
  }
  g->node_off[D + 1] = noff;
  g->n_nodes = noff;
  const uint64_t slot_bytes = (uint64_t)g->edge * g->edge * g->edge * g->cbpv;
  g->slot_pitch = (uint32_t)align_up(slot_bytes, kAlign);
  return RO_OK;
}

void make_layout(const ro_desc* d, const Geometry& g, Layout* L) {
  std::memset(L, 0, sizeof(*L));
  ro_buffer_sizes& s = L->sz;
  s.slot_pitch = g.slot_pitch;
  s.n_bricks = g.n_bricks;
  s.n_nodes = g.n_nodes;
  s.depth = (uint32_t)g.D;
  s.channel_stride = (uint32_t)g.mp;
  L->req_pad = align_up(g.n_bricks, ro::kCompactTile);
  L->node_req_pad = align_up(g.n_nodes * (uint64_t)g.m, ro::kCompactTile);
  L->used_pad = align_up(d->cache_slots, ro::kCompactTile);
  s.cache = (uint64_t)d->cache_slots * g.slot_pitch;
  s.page_table = align_up(g.n_bricks * 4, kAlign);
  L->oc_given = align_up(g.n_nodes * (uint64_t)g.mp * 4, kAlign);
  s.octree = L->oc_given + align_up(g.node_off[g.D] * (uint64_t)g.mp * 4, kAlign);
  s.req_flags = L->req_pad;
  s.node_req_flags = L->node_req_pad;
  s.used_flags = L->used_pad;
  s.last_used = align_up((uint64_t)d->cache_slots * 4, kAlign);
  s.staging = (uint64_t)d->max_upload * g.slot_pitch;
  L->fr_lut = 0;
  L->fr_prefix = (uint64_t)ro::kMaxC * 256 * 16;
  s.frame = align_up(L->fr_prefix + (uint64_t)ro::kMaxC * 257 * 2, kAlign);
  L->li_req = 0;
  L->li_node = align_up((uint64_t)d->max_requests * 4, kAlign);
  s.lists = L->li_node + align_up((uint64_t)d->max_requests * 4, kAlign);
  L->max_tiles = (uint32_t)(std::max(L->req_pad, L->node_req_pad) / ro::kCompactTile);
  uint64_t o = 0;
  L->sc_counts = o; o = align_up(o + (uint64_t)L->max_tiles * 4, kAlign);
  L->sc_totals = o; o = align_up(o + 64, kAlign);
  L->sc_items = o; o = align_up(o + (uint64_t)kMaxItems * sizeof(ro::UpdateItem), kAlign);
  L->sc_meta = o; o = align_up(o + (uint64_t)d->max_meta * sizeof(ro::MetaItem), kAlign);
  L->sc_ins_index = o; o = align_up(o + (uint64_t)d->max_upload * 4, kAlign);
  L->sc_ins_slot = o; o = align_up(o + (uint64_t)d->max_upload * 4, kAlign);
  L->sc_ev_index = o; o = align_up(o + (uint64_t)d->max_upload * 4, kAlign);
  L->sc_stats = o; o = align_up(o + (uint64_t)kMaxStatBlocks * ro::kStats * 8, kAlign);
  L->sc_err = o; o = align_up(o + 64, kAlign);
  L->sc_work = o; o = align_up(o + 64, kAlign);
  s.scratch = o;
  L->ba_views = 0;
  L->ba_tf = (uint64_t)ro::kMaxViews * sizeof(ro::ViewArgs);
  L->ba_order = align_up(L->ba_tf + (uint64_t)ro::kMaxC * 8, kAlign);
  L->ba_cost = align_up(L->ba_order + (uint64_t)d->max_batch_tiles * 4, kAlign);
  s.batch = d->max_batch_tiles ? align_up(L->ba_cost + (uint64_t)d->max_batch_tiles * ro::kTileParts * 4, kAlign) : 0;
  const uint64_t parts[kParts] = {s.cache, s.page_table, s.octree, s.req_flags, s.node_req_flags, s.used_flags,
                                  s.last_used, s.staging, s.frame, s.lists, s.scratch, s.batch};
  uint64_t tot = 0;
  for (int i = 0; i < kParts; ++i) {
    L->off[i] = tot;
    tot = align_up(tot + parts[i], kAlign);
  }
  s.total = tot;
}

}  // namespace

struct ro_ctx {
  ro_desc desc;
  Geometry g;
  Layout L;
  uint8_t* arena = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  uint8_t *cache, *req, *node_req, *used, *staging, *scratch;
  uint32_t *pt, *octree, *given, *last_used, *req_out, *node_out, *err;
  float4* lut;
  uint16_t* prefix;
  std::vector<uint32_t> slot_of_brick;   // page-table index -> slot or RO_NONE
  std::vector<uint32_t> brick_of_slot;   // slot -> page-table index or RO_NONE
  std::vector<uint32_t> free_slots;      // descending, pop_back gives the lowest
  std::vector<uint32_t> pending;         // page-table indices changed since the last update
  std::vector<uint32_t> stamps;          // host copy of last_used (LRU), refreshed by ro_read_requests
  cudaEvent_t ev_copy = nullptr;         // an async upload's copy into the staging area has landed
  cudaEvent_t ev_scatter = nullptr;      // the last scatter has read the staging area
  bool copy_pending = false;
  std::vector<float4> host_lut;
  // batches: device view table / TF ranges / schedule / tile costs in the
  // arena; pinned upload area [views | TF ranges | LUTs]; the captured graph
  ro::ViewArgs* b_views = nullptr;
  float2* b_tf = nullptr;
  uint32_t *b_order = nullptr, *b_cost = nullptr;
  uint8_t* b_pinned = nullptr;
  cudaEvent_t b_uploaded = nullptr;   // recorded by the graph once its uploads are done
  cudaStream_t b_capture = nullptr;   // private stream the graph is captured on
  cudaGraph_t b_graph = nullptr;
  cudaGraphExec_t b_exec = nullptr;
  std::vector<uint32_t> b_key;        // layout the graph was captured for
  uint32_t b_blocks = 0;
  uint32_t frame = 0;
  uint32_t timeout_ms = 30000;
  uint32_t last_blocks = 0;
  ro_status latched = RO_OK;
  std::string err_msg = "ok";
};

namespace {

ro_status set_err(ro_ctx* c, ro_status s, const std::string& m) {
  c->err_msg = m;
  if (s == RO_ERR_CUDA || s == RO_ERR_INTERNAL) c->latched = s;
  return s;
}

ro_status cuda_check(ro_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return RO_OK;
  return set_err(c, RO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RO_TRY(expr)                 \
  do {                               \
    ro_status _s = (expr);           \
    if (_s != RO_OK) return _s;      \
  } while (0)

// Waits for an event against the context's deadline.
ro_status wait_event(ro_ctx* c, cudaEvent_t ev, const char* where) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return RO_OK;
    if (e != cudaErrorNotReady) return cuda_check(c, e, where);
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > (long long)c->timeout_ms) return set_err(c, RO_ERR_TIMEOUT, std::string(where) + ": stream wait timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

ro_status wait_stream(ro_ctx* c, const char* where) {
  RO_TRY(cuda_check(c, cudaEventRecord(c->ev, c->stream), where));
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(c->ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_check(c, e, where);
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > (long long)c->timeout_ms) return set_err(c, RO_ERR_TIMEOUT, std::string(where) + ": stream wait timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  uint32_t e = 0;
  RO_TRY(cuda_check(c, cudaMemcpy(&e, c->err, 4, cudaMemcpyDeviceToHost), where));
  if (e != 0) return set_err(c, RO_ERR_INTERNAL, std::string(where) + ": device index guard fired (code " + std::to_string(e) + ")");
  return RO_OK;
}

bool decode_id(const ro_ctx* c, uint32_t id, int* ch, int* l, uint32_t* pi) {
  const Geometry& g = c->g;
  const uint32_t p = id >> 24;
  if (p >= (uint32_t)(g.m * g.k)) return false;
  const int lv = (int)(p % (uint32_t)g.k);
  const uint32_t bz = (id >> 16) & 0xFF, by = (id >> 8) & 0xFF, bx = id & 0xFF;
  if (bx >= (uint32_t)g.nb[lv][0] || by >= (uint32_t)g.nb[lv][1] || bz >= (uint32_t)g.nb[lv][2]) return false;
  *ch = (int)(p / (uint32_t)g.k);
  *l = lv;
  *pi = g.pt_off[p] + (bz * (uint32_t)g.nb[lv][1] + by) * (uint32_t)g.nb[lv][0] + bx;
  return true;
}

// page-table index -> (channel, level, brick coords)
void index_to_brick(const Geometry& g, uint32_t pi, int* ch, int* l, uint32_t b[3]) {
  int p = 0;
  while (p + 1 < g.m * g.k && g.pt_off[p + 1] <= pi) ++p;
  *ch = p / g.k;
  *l = p % g.k;
  const uint32_t local = pi - g.pt_off[p];
  const uint32_t nx = (uint32_t)g.nb[*l][0], ny = (uint32_t)g.nb[*l][1];
  b[0] = local % nx;
  b[1] = (local / nx) % ny;
  b[2] = local / (nx * ny);
}

// Leaf boxes of one channel, split into items of at most kItemLeaves leaves.
void push_box(std::vector<ro::UpdateItem>& items, uint32_t ch, const uint32_t lo[3], const uint32_t hi[3]) {
  const uint32_t nx = hi[0] - lo[0], ny = hi[1] - lo[1];
  uint32_t sx = nx, sy = ny, sz;
  if (sx > kItemLeaves) sx = kItemLeaves;
  if ((uint64_t)sx * sy > kItemLeaves) sy = std::max(1u, kItemLeaves / sx);
  sz = std::max(1u, kItemLeaves / (sx * sy));
  for (uint32_t z = lo[2]; z < hi[2]; z += sz)
    for (uint32_t y = lo[1]; y < hi[1]; y += sy)
      for (uint32_t x = lo[0]; x < hi[0]; x += sx) {
        ro::UpdateItem it{};
        it.lo[0] = x; it.lo[1] = y; it.lo[2] = z;
        it.hi[0] = std::min(x + sx, hi[0]); it.hi[1] = std::min(y + sy, hi[1]); it.hi[2] = std::min(z + sz, hi[2]);
        it.channel = ch;
        items.push_back(it);
      }
}

}  // namespace

extern "C" {

ro_status ro_query_sizes(const ro_desc* desc, ro_buffer_sizes* out) {
  if (!out) return RO_ERR_INVALID_ARG;
  Geometry g;
  std::string why;
  ro_status s = make_geometry(desc, &g, &why);
  if (s != RO_OK) {
    g_create_error = why;
    return s;
  }
  Layout L;
  make_layout(desc, g, &L);
  *out = L.sz;
  return RO_OK;
}

ro_status ro_create(const ro_desc* desc, void* arena_device, uint64_t arena_bytes, void* stream, ro_ctx** out) {
  if (!out) return RO_ERR_INVALID_ARG;
  *out = nullptr;
  ro_ctx* c = new (std::nothrow) ro_ctx();
  if (!c) return RO_ERR_CAPACITY;
  std::string why;
  ro_status s = make_geometry(desc, &c->g, &why);
  if (s != RO_OK) {
    g_create_error = why;
    delete c;
    return s;
  }
  c->desc = *desc;
  make_layout(desc, c->g, &c->L);
  if (!arena_device || (reinterpret_cast<uintptr_t>(arena_device) % kAlign) != 0) {
    g_create_error = "arena must be a 256-byte aligned device pointer";
    delete c;
    return RO_ERR_INVALID_ARG;
  }
  if (arena_bytes < c->L.sz.total) {
    g_create_error = "arena smaller than ro_query_sizes().total";
    delete c;
    return RO_ERR_CAPACITY;
  }
  c->arena = static_cast<uint8_t*>(arena_device);
  c->stream = static_cast<cudaStream_t>(stream);
  const uint64_t* o = c->L.off;
  c->cache = c->arena + o[0];
  c->pt = reinterpret_cast<uint32_t*>(c->arena + o[1]);
  c->octree = reinterpret_cast<uint32_t*>(c->arena + o[2]);
  c->given = reinterpret_cast<uint32_t*>(c->arena + o[2] + c->L.oc_given);
  c->req = c->arena + o[3];
  c->node_req = c->arena + o[4];
  c->used = c->arena + o[5];
  c->last_used = reinterpret_cast<uint32_t*>(c->arena + o[6]);
  c->staging = c->arena + o[7];
  c->lut = reinterpret_cast<float4*>(c->arena + o[8] + c->L.fr_lut);
  c->prefix = reinterpret_cast<uint16_t*>(c->arena + o[8] + c->L.fr_prefix);
  c->req_out = reinterpret_cast<uint32_t*>(c->arena + o[9] + c->L.li_req);
  c->node_out = reinterpret_cast<uint32_t*>(c->arena + o[9] + c->L.li_node);
  c->scratch = c->arena + o[10];
  c->err = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_err);
  if (desc->max_batch_tiles) {
    uint8_t* b = c->arena + o[11];
    c->b_views = reinterpret_cast<ro::ViewArgs*>(b + c->L.ba_views);
    c->b_tf = reinterpret_cast<float2*>(b + c->L.ba_tf);
    c->b_order = reinterpret_cast<uint32_t*>(b + c->L.ba_order);
    c->b_cost = reinterpret_cast<uint32_t*>(b + c->L.ba_cost);
  }
  c->slot_of_brick.assign(c->g.n_bricks, RO_NONE);
  c->brick_of_slot.assign(desc->cache_slots, RO_NONE);
  c->free_slots.resize(desc->cache_slots);
  for (uint32_t i = 0; i < desc->cache_slots; ++i) c->free_slots[i] = desc->cache_slots - 1 - i;
  c->host_lut.resize((size_t)ro::kMaxC * 256);
  c->stamps.assign(desc->cache_slots, 0u);
  cudaError_t e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_scatter, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaEventCreate: ") + cudaGetErrorString(e);
    delete c;
    return RO_ERR_CUDA;
  }
  const ro_buffer_sizes& z = c->L.sz;
  cudaStream_t st = c->stream;
  e = cudaMemsetAsync(c->pt, 0, z.page_table, st);
  // every node INVALID without a valid ancestor, empty mask; no range given
  if (e == cudaSuccess) e = ro::launch_fill_words(c->octree, c->g.n_nodes * (uint64_t)c->g.mp, ro::kInvalidUnknown, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->given, 0, z.octree - c->L.oc_given, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->req, 0, z.req_flags, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->node_req, 0, z.node_req_flags, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->used, 0, z.used_flags, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->last_used, 0, z.last_used, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->scratch, 0, z.scratch, st);
  if (e == cudaSuccess && z.batch) e = cudaMemsetAsync(c->arena + o[11], 0, z.batch, st);
  if (e != cudaSuccess) {
    g_create_error = std::string("initialisation: ") + cudaGetErrorString(e);
    cudaEventDestroy(c->ev);
    delete c;
    return RO_ERR_CUDA;
  }
  *out = c;
  return RO_OK;
}

ro_status ro_destroy(ro_ctx* c) {
  if (!c) return RO_ERR_INVALID_ARG;
  ro_status s = RO_OK;
  if (c->latched == RO_OK) s = wait_stream(c, "ro_destroy");
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->ev_copy) cudaEventDestroy(c->ev_copy);
  if (c->ev_scatter) cudaEventDestroy(c->ev_scatter);
  if (c->b_exec) cudaGraphExecDestroy(c->b_exec);
  if (c->b_graph) cudaGraphDestroy(c->b_graph);
  if (c->b_uploaded) cudaEventDestroy(c->b_uploaded);
  if (c->b_capture) cudaStreamDestroy(c->b_capture);
  if (c->b_pinned) cudaFreeHost(c->b_pinned);
  delete c;
  return s == RO_ERR_INTERNAL ? RO_OK : s;
}

ro_status ro_set_timeout(ro_ctx* c, uint32_t ms) {
  if (!c || ms == 0) return RO_ERR_INVALID_ARG;
  c->timeout_ms = ms;
  return RO_OK;
}

const char* ro_last_error(const ro_ctx* c) { return c ? c->err_msg.c_str() : g_create_error.c_str(); }

uint32_t ro_brick_index(const ro_ctx* c, uint32_t id) {
  if (!c) return RO_NONE;
  int ch, l;
  uint32_t pi;
  return decode_id(c, id, &ch, &l, &pi) ? pi : RO_NONE;
}

extern "C++" {
namespace {

// Validation of brick IDs shared by the two ways of making bricks resident.
ro_status check_ids(ro_ctx* c, uint32_t n, const uint32_t* ids, std::vector<uint32_t>& pis, const char* where) {
  pis.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    int ch, l;
    if (!decode_id(c, ids[i], &ch, &l, &pis[i]))
      return set_err(c, RO_ERR_INVALID_ARG, std::string(where) + ": brick id outside the hierarchy");
  }
  std::vector<uint32_t> s(pis);
  std::sort(s.begin(), s.end());
  if (std::adjacent_find(s.begin(), s.end()) != s.end())
    return set_err(c, RO_ERR_INVALID_ARG, std::string(where) + ": duplicate brick id");
  return RO_OK;
}

// Slot choice (keep resident bricks' slots, then free slots, then LRU),
// then `fill` enqueues the n bricks' voxels into the staging rows and the
// scatter kernel writes slots and page-table entries.
template <class Fill>
ro_status place_bricks(ro_ctx* c, uint32_t n, const std::vector<uint32_t>& pis, Fill fill, uint32_t* out_slots,
                       uint32_t* out_evicted, const std::vector<uint32_t>* keep_slots = nullptr, bool async = false) {
  // slot choice: keep resident bricks' slots, then free slots, then LRU
  std::vector<uint32_t> slots(n, RO_NONE), evicted(n, RO_NONE);
  std::vector<uint8_t> taken;  // slots assigned in this call
  uint32_t need = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (c->slot_of_brick[pis[i]] != RO_NONE) slots[i] = c->slot_of_brick[pis[i]];
    else ++need;
  }
  const uint32_t from_free = std::min<uint32_t>(need, (uint32_t)c->free_slots.size());
  std::vector<uint32_t> lru;
  if (need > from_free) {
    // usage stamps as of the last ro_read_requests, fresh bricks stamped at
    // their upload: no wait for the stream (a render may still be running)
    const std::vector<uint32_t>& stamps = c->stamps;
    std::vector<uint8_t> keep(c->desc.cache_slots, 0);
    for (uint32_t i = 0; i < n; ++i)
      if (slots[i] != RO_NONE) keep[slots[i]] = 1;
    if (keep_slots)
      for (uint32_t sl : *keep_slots) keep[sl] = 1;
    std::vector<uint32_t> cand;
    cand.reserve(c->desc.cache_slots);
    for (uint32_t sl = 0; sl < c->desc.cache_slots; ++sl)
      if (c->brick_of_slot[sl] != RO_NONE && !keep[sl]) cand.push_back(sl);
    const uint32_t want = need - from_free;
    if (cand.size() < want) return set_err(c, RO_ERR_CAPACITY, "ro_upload_bricks: not enough evictable slots");
    std::partial_sort(cand.begin(), cand.begin() + want, cand.end(), [&](uint32_t a, uint32_t b) {
      return stamps[a] != stamps[b] ? stamps[a] < stamps[b] : a < b;
    });
    lru.assign(cand.begin(), cand.begin() + want);
  }
  uint32_t used_free = 0, used_lru = 0;
  std::vector<uint32_t> ev_index;
  for (uint32_t i = 0; i < n; ++i) {
    if (slots[i] != RO_NONE) continue;
    uint32_t sl;
    if (used_free < from_free) {
      sl = c->free_slots.back();
      c->free_slots.pop_back();
      ++used_free;
    } else {
      sl = lru[used_lru++];
      const uint32_t old = c->brick_of_slot[sl];
      c->slot_of_brick[old] = RO_NONE;
      ev_index.push_back(old);
      c->pending.push_back(old);
      int ch, l;
      uint32_t b[3];
      index_to_brick(c->g, old, &ch, &l, b);
      evicted[i] = ((uint32_t)(ch * c->g.k + l) << 24) | (b[2] << 16) | (b[1] << 8) | b[0];
    }
    slots[i] = sl;
    c->brick_of_slot[sl] = pis[i];
    c->slot_of_brick[pis[i]] = sl;
    c->pending.push_back(pis[i]);
    c->stamps[sl] = c->frame;
  }
  cudaStream_t st = c->stream;
  RO_TRY(fill(st));
  uint32_t* d_ins_index = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_ins_index);
  uint32_t* d_ins_slot = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_ins_slot);
  uint32_t* d_ev_index = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_ev_index);
  RO_TRY(cuda_check(c, cudaMemcpyAsync(d_ins_index, pis.data(), 4ull * n, cudaMemcpyHostToDevice, st), "ro_upload_bricks"));
  RO_TRY(cuda_check(c, cudaMemcpyAsync(d_ins_slot, slots.data(), 4ull * n, cudaMemcpyHostToDevice, st), "ro_upload_bricks"));
  if (!ev_index.empty())
    RO_TRY(cuda_check(c, cudaMemcpyAsync(d_ev_index, ev_index.data(), 4ull * ev_index.size(), cudaMemcpyHostToDevice, st),
                      "ro_upload_bricks"));
  ro::ScatterArgs a{};
  a.staging = c->staging;
  a.cache = c->cache;
  a.pt = c->pt;
  a.ins_index = d_ins_index;
  a.ins_slot = d_ins_slot;
  a.n_ins = n;
  a.ev_index = d_ev_index;
  a.n_ev = (uint32_t)ev_index.size();
  a.slot_pitch = c->g.slot_pitch;
  a.cache_slots = c->desc.cache_slots;
  a.n_bricks = c->g.n_bricks;
  a.err = c->err;
  a.sf = c->g.sf;
  a.bpv = c->g.bpv;
  a.n_el = c->g.edge * c->g.edge * c->g.edge;
  a.last_used = c->last_used;
  a.frame = c->frame;
  RO_TRY(cuda_check(c, ro::launch_scatter(a, st), "ro_upload_bricks: scatter"));
  RO_TRY(cuda_check(c, cudaEventRecord(c->ev_scatter, st), "ro_upload_bricks: event"));
  // the caller's host buffers may be reused once the copies have landed
  // (an asynchronous upload leaves that wait to ro_upload_wait)
  if (!async) RO_TRY(wait_stream(c, "ro_upload_bricks"));
  if (out_slots) std::memcpy(out_slots, slots.data(), 4ull * n);
  if (out_evicted) std::memcpy(out_evicted, evicted.data(), 4ull * n);
  return RO_OK;
}

}  // namespace
}  // extern "C++"

ro_status ro_upload_bricks(ro_ctx* c, uint32_t n, const uint32_t* ids, const void* voxels, uint32_t* out_slots,
                           uint32_t* out_evicted) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (n == 0) return RO_OK;
  if (!ids || !voxels) return set_err(c, RO_ERR_INVALID_ARG, "ro_upload_bricks: null pointer");
  if (n > c->desc.max_upload || n > c->desc.cache_slots)
    return set_err(c, RO_ERR_CAPACITY, "ro_upload_bricks: n exceeds max_upload or cache_slots");
  std::vector<uint32_t> pis;
  RO_TRY(check_ids(c, n, ids, pis, "ro_upload_bricks"));
  RO_TRY(ro_upload_wait(c));   // a previous asynchronous copy must not race this one
  auto fill = [&](cudaStream_t st) {
    const uint64_t bytes = (uint64_t)c->g.edge * c->g.edge * c->g.edge * c->g.bpv;
    return cuda_check(c, cudaMemcpy2DAsync(c->staging, c->g.slot_pitch, voxels, bytes, bytes, n, cudaMemcpyHostToDevice, st),
                      "ro_upload_bricks: voxels");
  };
  return place_bricks(c, n, pis, fill, out_slots, out_evicted);
}

ro_status ro_upload_bricks_async(ro_ctx* c, uint32_t n, const uint32_t* ids, const void* voxels, uint32_t* out_slots,
                                 uint32_t* out_evicted, void* copy_stream) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (n == 0) return RO_OK;
  if (!ids || !voxels) return set_err(c, RO_ERR_INVALID_ARG, "ro_upload_bricks_async: null pointer");
  if (n > c->desc.max_upload || n > c->desc.cache_slots)
    return set_err(c, RO_ERR_CAPACITY, "ro_upload_bricks_async: n exceeds max_upload or cache_slots");
  std::vector<uint32_t> pis;
  RO_TRY(check_ids(c, n, ids, pis, "ro_upload_bricks_async"));
  RO_TRY(ro_upload_wait(c));   // the previous call's host buffer and copy are done with
  const cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
  auto fill = [&](cudaStream_t st) {
    const uint64_t bytes = (uint64_t)c->g.edge * c->g.edge * c->g.edge * c->g.bpv;
    // the staging area is free once the previous scatter has read it
    RO_TRY(cuda_check(c, cudaStreamWaitEvent(cs, c->ev_scatter, 0), "ro_upload_bricks_async: wait scatter"));
    RO_TRY(cuda_check(c, cudaMemcpy2DAsync(c->staging, c->g.slot_pitch, voxels, bytes, bytes, n, cudaMemcpyHostToDevice, cs),
                      "ro_upload_bricks_async: voxels"));
    RO_TRY(cuda_check(c, cudaEventRecord(c->ev_copy, cs), "ro_upload_bricks_async: event"));
    c->copy_pending = true;
    return cuda_check(c, cudaStreamWaitEvent(st, c->ev_copy, 0), "ro_upload_bricks_async: wait copy");
  };
  return place_bricks(c, n, pis, fill, out_slots, out_evicted, nullptr, true);
}

ro_status ro_upload_wait(ro_ctx* c) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (!c->copy_pending) return RO_OK;
  RO_TRY(wait_event(c, c->ev_copy, "ro_upload_wait"));
  c->copy_pending = false;
  return RO_OK;
}

ro_status ro_compensate_bricks(ro_ctx* c, ro_mc* mc, uint32_t n, const uint32_t* ids, uint32_t* out_slots) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (n == 0) return RO_OK;
  const char* where = "ro_compensate_bricks";
  if (!mc || !ids) return set_err(c, RO_ERR_INVALID_ARG, "ro_compensate_bricks: null pointer");
  if (c->g.edge != RO_MC_EDGE || c->g.bpv != 2 || c->g.sf != 0 || c->g.k < 2 || c->desc.keep_axes[0] != 0)
    return set_err(c, RO_ERR_INVALID_ARG,
                   "ro_compensate_bricks: needs 32^3 u16 bricks, raw samples, >= 2 levels, level 1 halving every axis");
  if (n > c->desc.max_upload || n > c->desc.cache_slots || n > ro::mc_max_batch(mc) ||
      2ull * n * sizeof(uint32_t) > (uint64_t)kMaxItems * sizeof(ro::UpdateItem))
    return set_err(c, RO_ERR_CAPACITY, "ro_compensate_bricks: n exceeds max_upload, cache_slots or the batch");
  std::vector<uint32_t> pis;
  RO_TRY(check_ids(c, n, ids, pis, where));
  std::vector<uint32_t> parent_slot(n), octant(n);
  for (uint32_t i = 0; i < n; ++i) {
    int ch, l;
    uint32_t b[3];
    index_to_brick(c->g, pis[i], &ch, &l, b);
    if (l != 0) return set_err(c, RO_ERR_INVALID_ARG, "ro_compensate_bricks: not a level-0 brick");
    if (c->slot_of_brick[pis[i]] != RO_NONE) return set_err(c, RO_ERR_INVALID_ARG, "ro_compensate_bricks: brick resident");
    const uint32_t pid = ((uint32_t)(ch * c->g.k + 1) << 24) | ((b[2] >> 1) << 16) | ((b[1] >> 1) << 8) | (b[0] >> 1);
    int pc, pl;
    uint32_t ppi;
    if (!decode_id(c, pid, &pc, &pl, &ppi) || c->slot_of_brick[ppi] == RO_NONE)
      return set_err(c, RO_ERR_INVALID_ARG, "ro_compensate_bricks: level-1 parent not resident");
    parent_slot[i] = c->slot_of_brick[ppi];
    octant[i] = (b[0] & 1u) | ((b[1] & 1u) << 1) | ((b[2] & 1u) << 2);
  }
  // parents' slots and octants in the update-item scratch (free during uploads)
  uint32_t* d_parent = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_items);
  uint32_t* d_oct = d_parent + n;
  auto fill = [&](cudaStream_t st) {
    RO_TRY(cuda_check(c, cudaMemcpyAsync(d_parent, parent_slot.data(), 4ull * n, cudaMemcpyHostToDevice, st), where));
    RO_TRY(cuda_check(c, cudaMemcpyAsync(d_oct, octant.data(), 4ull * n, cudaMemcpyHostToDevice, st), where));
    return cuda_check(c, ro::mc_synthesize(mc, n, c->cache, c->g.slot_pitch, d_parent, d_oct, c->staging, c->g.slot_pitch, st),
                      "ro_compensate_bricks: network");
  };
  return place_bricks(c, n, pis, fill, out_slots, nullptr, &parent_slot);  // parents are read, never evicted
}

}  // extern "C"

namespace {

// Last entry wins for a repeated (channel, index); input already in strictly
// increasing (channel, index) order needs no sort.
std::vector<ro::MetaItem> dedup_meta(const std::vector<ro::MetaItem>& in, uint64_t n_index) {
  auto key = [&](const ro::MetaItem& m) { return (uint64_t)m.channel * n_index + m.leaf; };
  bool sorted = true;
  for (size_t i = 1; i < in.size() && sorted; ++i) sorted = key(in[i - 1]) < key(in[i]);
  if (sorted) return in;
  std::vector<uint32_t> order(in.size());
  for (uint32_t i = 0; i < in.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key(in[a]) < key(in[b]); });
  std::vector<ro::MetaItem> out;
  out.reserve(in.size());
  for (size_t q = 0; q < order.size(); ++q)
    if (q + 1 == order.size() || key(in[order[q + 1]]) != key(in[order[q]])) out.push_back(in[order[q]]);
  return out;
}

// The update of Sec. 5.3 for leaf ranges `lm` (.leaf = leaf index), ranges
// given for inner nodes `im` (.leaf = node index) and the bricks changed
// since the last update: range writes, leaf masks, bottom-up recomputation
// of the changed boxes' ancestors, then the INVALID pointers from the root
// down over the same boxes.
ro_status run_update(ro_ctx* c, const std::vector<ro::MetaItem>& lm_in, const std::vector<ro::MetaItem>& im_in) {
  const Geometry& g = c->g;
  const uint64_t n_leaves = (uint64_t)g.nleaf[0] * g.nleaf[1] * g.nleaf[2];
  const std::vector<ro::MetaItem> mi = dedup_meta(lm_in, n_leaves);
  const std::vector<ro::MetaItem> gi = dedup_meta(im_in, g.node_off[g.D]);
  // items: leaf boxes of changed bricks (masks recomputed), then metadata leaves
  std::vector<ro::UpdateItem> brick_items, meta_items;
  std::sort(c->pending.begin(), c->pending.end());
  c->pending.erase(std::unique(c->pending.begin(), c->pending.end()), c->pending.end());
  for (uint32_t pi : c->pending) {
    int ch, l;
    uint32_t b[3], lo[3], hi[3];
    index_to_brick(g, pi, &ch, &l, b);
    for (int a = 0; a < 3; ++a) {
      const uint64_t v0 = (uint64_t)b[a] << (g.blog2 + g.lsh[l][a]);
      uint64_t v1 = (uint64_t)(b[a] + 1) << (g.blog2 + g.lsh[l][a]);
      if (v1 > (uint64_t)g.dims0[a]) v1 = (uint64_t)g.dims0[a];
      lo[a] = (uint32_t)(v0 >> g.leaf_log2[a]);
      hi[a] = (uint32_t)((v1 + (1ull << g.leaf_log2[a]) - 1) >> g.leaf_log2[a]);
    }
    push_box(brick_items, (uint32_t)ch, lo, hi);
  }
  // a channel with many changed leaves gets one whole-volume box instead of
  // one item per leaf
  std::vector<uint64_t> per_channel(g.m, 0);
  for (const ro::MetaItem& m : mi) ++per_channel[m.channel];
  for (int ch = 0; ch < g.m; ++ch)
    if (per_channel[ch] > n_leaves / 8) {
      const uint32_t lo[3] = {0, 0, 0};
      const uint32_t hi[3] = {(uint32_t)g.nleaf[0], (uint32_t)g.nleaf[1], (uint32_t)g.nleaf[2]};
      push_box(meta_items, (uint32_t)ch, lo, hi);
    }
  for (const ro::MetaItem& m : mi) {
    if (per_channel[m.channel] > n_leaves / 8) continue;
    uint32_t lo[3], hi[3];
    lo[0] = m.leaf % g.nleaf[0];
    lo[1] = (m.leaf / g.nleaf[0]) % g.nleaf[1];
    lo[2] = (uint32_t)(m.leaf / ((uint64_t)g.nleaf[0] * g.nleaf[1]));
    for (int a = 0; a < 3; ++a) hi[a] = lo[a] + 1;
    push_box(meta_items, m.channel, lo, hi);
  }
  // an inner node's range: the leaf box of its whole subtree (its ancestors
  // are recomputed, and its INVALID descendants may now point to it)
  for (const ro::MetaItem& m : gi) {
    int d = 0;
    while (g.node_off[d + 1] <= m.leaf) ++d;
    const uint64_t j = m.leaf - g.node_off[d];
    const uint32_t jn[3] = {(uint32_t)(j % g.nn[d][0]), (uint32_t)((j / g.nn[d][0]) % g.nn[d][1]),
                            (uint32_t)(j / ((uint64_t)g.nn[d][0] * g.nn[d][1]))};
    uint32_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = jn[a] << (g.D - d);
      hi[a] = std::min<uint32_t>((jn[a] + 1) << (g.D - d), (uint32_t)g.nleaf[a]);
    }
    push_box(meta_items, m.channel, lo, hi);
  }
  cudaStream_t st = c->stream;
  ro::UpdateArgs a{};
  a.g = g;
  a.pt = c->pt;
  a.octree = c->octree;
  a.given = c->given;
  a.err = c->err;
  ro::UpdateItem* d_items = reinterpret_cast<ro::UpdateItem*>(c->scratch + c->L.sc_items);
  ro::MetaItem* d_meta = reinterpret_cast<ro::MetaItem*>(c->scratch + c->L.sc_meta);
  // range writes in chunks of max_meta: leaves into the node words, inner
  // nodes into the given ranges
  for (int kind = 0; kind < 2; ++kind) {
    const std::vector<ro::MetaItem>& v = kind == 0 ? mi : gi;
    for (size_t q = 0; q < v.size(); q += c->desc.max_meta) {
      const uint32_t nm = (uint32_t)std::min<size_t>(c->desc.max_meta, v.size() - q);
      RO_TRY(cuda_check(c, cudaMemcpyAsync(d_meta, v.data() + q, nm * sizeof(ro::MetaItem), cudaMemcpyHostToDevice, st),
                        "ro_update_residency_octree: meta"));
      a.meta = d_meta;
      a.n_meta = nm;
      RO_TRY(cuda_check(c, kind == 0 ? ro::launch_write_meta(a, st) : ro::launch_write_given(a, st),
                        "ro_update_residency_octree: write_meta"));
      // the copy source is pageable host memory: the next chunk may reuse d_meta
      // only after this launch; stream order guarantees it
    }
  }
  a.n_meta = 0;
  // leaf masks + bottom-up passes + pointer passes, chunk by chunk
  std::vector<ro::UpdateItem> all(brick_items);
  const size_t n_brick_items = brick_items.size();
  all.insert(all.end(), meta_items.begin(), meta_items.end());
  for (size_t q = 0; q < all.size(); q += kMaxItems) {
    const uint32_t ni = (uint32_t)std::min<size_t>(kMaxItems, all.size() - q);
    RO_TRY(cuda_check(c, cudaMemcpyAsync(d_items, all.data() + q, ni * sizeof(ro::UpdateItem), cudaMemcpyHostToDevice, st),
                      "ro_update_residency_octree: items"));
    a.items = d_items;
    a.n_items = q < n_brick_items ? (uint32_t)std::min<size_t>(ni, n_brick_items - q) : 0;
    RO_TRY(cuda_check(c, ro::launch_leaf_masks(a, st), "ro_update_residency_octree: leaf masks"));
    a.n_items = ni;
    for (int d = g.D - 1; d >= 0; --d) {
      a.depth = d;
      RO_TRY(cuda_check(c, ro::launch_reduce_depth(a, st), "ro_update_residency_octree: reduce"));
    }
    // d_items is rewritten by the next chunk's copy, which stream order puts
    // after these launches
  }
  // pointers of INVALID words, after every chunk's ranges are final
  for (size_t q = 0; q < all.size(); q += kMaxItems) {
    const uint32_t ni = (uint32_t)std::min<size_t>(kMaxItems, all.size() - q);
    RO_TRY(cuda_check(c, cudaMemcpyAsync(d_items, all.data() + q, ni * sizeof(ro::UpdateItem), cudaMemcpyHostToDevice, st),
                      "ro_update_residency_octree: items"));
    a.items = d_items;
    a.n_items = ni;
    for (int d = 1; d <= g.D; ++d) {
      a.depth = d;
      RO_TRY(cuda_check(c, ro::launch_pointer_depth(a, st), "ro_update_residency_octree: pointers"));
    }
  }
  c->pending.clear();
  return RO_OK;
}

}  // namespace

extern "C" {

ro_status ro_update_residency_octree(ro_ctx* c, uint32_t n_meta, const ro_leaf_meta* meta) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (n_meta && !meta) return set_err(c, RO_ERR_INVALID_ARG, "ro_update_residency_octree: null meta");
  const Geometry& g = c->g;
  const uint64_t n_leaves = (uint64_t)g.nleaf[0] * g.nleaf[1] * g.nleaf[2];
  std::vector<ro::MetaItem> lm;
  lm.reserve(n_meta);
  for (uint32_t i = 0; i < n_meta; ++i) {
    if (meta[i].leaf >= n_leaves || meta[i].channel >= (uint32_t)g.m)
      return set_err(c, RO_ERR_INVALID_ARG, "ro_update_residency_octree: leaf or channel out of range");
    lm.push_back({meta[i].leaf, meta[i].channel, meta[i].vmin, meta[i].vmax});
  }
  return run_update(c, lm, {});
}

ro_status ro_update_node_metadata(ro_ctx* c, uint32_t n_meta, const ro_node_meta* meta) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (n_meta && !meta) return set_err(c, RO_ERR_INVALID_ARG, "ro_update_node_metadata: null meta");
  const Geometry& g = c->g;
  std::vector<ro::MetaItem> lm, im;
  for (uint32_t i = 0; i < n_meta; ++i) {
    if (meta[i].node >= g.n_nodes || meta[i].channel >= (uint32_t)g.m)
      return set_err(c, RO_ERR_INVALID_ARG, "ro_update_node_metadata: node or channel out of range");
    if (meta[i].node >= g.node_off[g.D])
      lm.push_back({(uint32_t)(meta[i].node - g.node_off[g.D]), meta[i].channel, meta[i].vmin, meta[i].vmax});
    else
      im.push_back({meta[i].node, meta[i].channel, meta[i].vmin, meta[i].vmax});
  }
  return run_update(c, lm, im);
}

namespace {

// Checks of one view's parameters shared by ro_render and ro_render_batch.
ro_status check_view(ro_ctx* c, const ro_camera* cam, const ro_render_params* p, const float* image, uint32_t W,
                     uint32_t H, const char* where) {
  const std::string w(where);
  if (!cam || !p || !image) return set_err(c, RO_ERR_INVALID_ARG, w + ": null pointer");
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return set_err(c, RO_ERR_INVALID_ARG, w + ": W and H must be in [1, 16384]");
  const Geometry& g = c->g;
  if (!(p->dt > 0.0f) || !std::isfinite(p->dt)) return set_err(c, RO_ERR_INVALID_ARG, w + ": dt must be positive");
  if (p->start_depth > (uint32_t)g.D) return set_err(c, RO_ERR_INVALID_ARG, w + ": start_depth beyond the octree depth");
  for (int l = 2; l < g.k; ++l)
    if (!(p->lod_t[l] >= p->lod_t[l - 1])) return set_err(c, RO_ERR_INVALID_ARG, w + ": lod_t must be non-decreasing");
  for (int ch = 0; ch < g.m; ++ch)
    if (p->lmin[ch] > p->lmax[ch] || p->lmax[ch] >= (uint32_t)g.k)
      return set_err(c, RO_ERR_INVALID_ARG, w + ": need lmin <= lmax < levels");
  return RO_OK;
}

ro_status check_tfs(ro_ctx* c, const ro_tf* tfs, const char* where) {
  if (!tfs) return set_err(c, RO_ERR_INVALID_ARG, std::string(where) + ": null pointer");
  for (int ch = 0; ch < c->g.m; ++ch)
    if (!tfs[ch].lut) return set_err(c, RO_ERR_INVALID_ARG, std::string(where) + ": null LUT");
  return RO_OK;
}

bool has_debug(const ro_render_params* p) {
  return p->debug_hash || p->debug_n_eval || p->debug_i_end || p->debug_n_bs;
}

// The per-view part of a launch: camera, per-level tables (Sec. 6.2,
// Algorithm 1) and outputs.  Tiles are 2^twl x 2^(5 - twl) pixels.
void fill_view(const ro_ctx* c, const ro_camera* cam, const ro_render_params* p, float* image, uint32_t W, uint32_t H,
               int twl, uint32_t tile_base, ro::ViewArgs* v) {
  const Geometry& g = c->g;
  std::memset(v, 0, sizeof(*v));
  for (int q = 0; q < 3; ++q) {
    v->eye[q] = cam->eye[q];
    v->fwd[q] = cam->forward[q];
    v->right[q] = cam->right[q];
    v->up[q] = cam->up[q];
  }
  v->persp = cam->perspective ? 1 : 0;
  v->tan_x = cam->tan_x;
  v->tan_y = cam->tan_y;
  v->pixel = cam->pixel;
  v->W = (int)W;
  v->H = (int)H;
  v->dt = p->dt;
  v->ert = p->ert;
  v->start_depth = (int)p->start_depth;
  v->skip = p->skip ? 1 : 0;
  v->tiles_x = (W + (1u << twl) - 1) >> twl;
  v->tile_base = tile_base;
  for (int l = 0; l < ro::kMaxL; ++l) v->lod_t[l] = p->lod_t[l];
  // traversal depth per level (Algorithm 1): deepest depth whose nodes are at least
  // one step long along every axis, physically
  for (int l = 0; l < ro::kMaxL; ++l) {
    const double step = (double)p->dt * std::ldexp(1.0, g.lstep[l]);
    int best = 0;
    for (int d = 0; d <= g.D; ++d) {
      double mn = INFINITY;
      for (int q = 0; q < 3; ++q) mn = std::min(mn, std::ldexp(1.0, g.leaf_log2[q] + g.D - d) * (double)g.spacing[q]);
      if (mn >= step) best = d;
    }
    v->sdepth[l] = best;
  }
  // desired levels of every channel for each value of lod (Sec. 6.2): the clamp
  // of lod to the channel's [lmin, lmax]
  for (int lod = 0; lod < ro::kMaxL; ++lod) {
    uint64_t ldp = 0;
    int lminu = 15;
    for (int ch = 0; ch < g.m; ++ch) {
      int l = lod < (int)p->lmin[ch] ? (int)p->lmin[ch] : lod;
      l = l > (int)p->lmax[ch] ? (int)p->lmax[ch] : l;
      ldp |= (uint64_t)l << (4 * ch);
      lminu = l < lminu ? l : lminu;
    }
    v->ldp_tab[lod] = ldp;
    v->lminu_tab[lod] = lminu;
  }
  v->image = reinterpret_cast<float4*>(image);
  v->dbg_hash = p->debug_hash;
  v->dbg_n_eval = p->debug_n_eval;
  v->dbg_i_end = p->debug_i_end;
  v->dbg_n_bs = p->debug_n_bs;
}

// The context-wide part of a launch.
void fill_common(ro_ctx* c, const ro_tf* tfs, ro::RenderArgs* a) {
  const Geometry& g = c->g;
  a->g = g;
  for (int ch = 0; ch < ro::kMaxC; ++ch) {
    a->tf_lo[ch] = ch < g.m ? tfs[ch].lo : 0.0f;
    a->tf_scale[ch] = ch < g.m ? tfs[ch].scale : 0.0f;
  }
  a->cache = c->cache;
  a->pt = c->pt;
  a->octree = c->octree;
  a->req = c->req;
  a->node_req = c->node_req;
  a->used = c->used;
  a->lut = c->lut;
  a->prefix = c->prefix;
  a->block_stats = reinterpret_cast<unsigned long long*>(c->scratch + c->L.sc_stats);
  a->err = c->err;
  a->work = reinterpret_cast<unsigned long long*>(c->scratch + c->L.sc_work);
}


}  // namespace

ro_status ro_render(ro_ctx* c, const ro_camera* cam, const ro_tf* tfs, const ro_render_params* p, float* image,
                    uint32_t W, uint32_t H) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  RO_TRY(check_view(c, cam, p, image, W, H, "ro_render"));
  RO_TRY(check_tfs(c, tfs, "ro_render"));
  if (p->order == 1 && c->desc.max_batch_tiles >= (uint64_t)((W + 7) / 8) * ((H + 3) / 4)) {
    // longest tiles first: the one-view batch path records and uses per-tile costs
    ro_view v{};
    v.camera = *cam;
    v.params = *p;
    v.image = image;
    v.W = W;
    v.H = H;
    const ro_schedule sc{8, 1};
    return ro_render_batch(c, 1, &v, tfs, &sc);
  }
  const uint64_t blocks = (uint64_t)((W + 15) / 16) * ((H + 15) / 16);
  if (blocks > kMaxStatBlocks) return set_err(c, RO_ERR_CAPACITY, "ro_render: image larger than 65536 blocks of 16x16");
  const Geometry& g = c->g;
  ro::RenderArgs a{};
  fill_common(c, tfs, &a);
  fill_view(c, cam, p, image, W, H, 3, 0, &a.v);
  a.tile_wlog2 = 3;
  a.n_rays = (uint64_t)a.v.tiles_x * ((H + 3) / 4) * 32;
  for (int ch = 0; ch < g.m; ++ch)
    std::memcpy(&c->host_lut[(size_t)ch * 256], tfs[ch].lut, 256 * sizeof(float4));
  cudaStream_t st = c->stream;
  RO_TRY(cuda_check(c, cudaMemcpyAsync(c->lut, c->host_lut.data(), (size_t)g.m * 256 * sizeof(float4), cudaMemcpyHostToDevice, st),
                    "ro_render: LUT upload"));
  ro::PrefixArgs pa{};
  pa.m = g.m;
  pa.bpv = g.bpv;
  for (int ch = 0; ch < ro::kMaxC; ++ch) {
    pa.tf_lo[ch] = a.tf_lo[ch];
    pa.tf_scale[ch] = a.tf_scale[ch];
  }
  pa.lut = c->lut;
  pa.prefix = c->prefix;
  RO_TRY(cuda_check(c, ro::launch_prefix(pa, st), "ro_render: prefix"));
  RO_TRY(cuda_check(c, cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), st), "ro_render: work counter"));
  int launched = 0;
  RO_TRY(cuda_check(c, ro::launch_render(a, has_debug(p), st, &launched), "ro_render: render"));
  c->last_blocks = (uint32_t)launched;
  ++c->frame;
  return RO_OK;
}

ro_status ro_render_batch(ro_ctx* c, uint32_t n_views, const ro_view* views, const ro_tf* tfs,
                          const ro_schedule* schedule) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  const char* where = "ro_render_batch";
  if (!views || n_views < 1 || n_views > (uint32_t)ro::kMaxViews)
    return set_err(c, RO_ERR_INVALID_ARG, "ro_render_batch: need 1 <= n_views <= RO_MAX_VIEWS and a view array");
  RO_TRY(check_tfs(c, tfs, where));
  const ro_schedule sched = schedule ? *schedule : ro_schedule{8, 0};
  if (!is_pow2(sched.tile_w) || sched.tile_w > 32 || sched.order > 1)
    return set_err(c, RO_ERR_INVALID_ARG, "ro_render_batch: tile_w must be 1, 2, 4, 8, 16 or 32 and order 0 or 1");
  if (!c->desc.max_batch_tiles) return set_err(c, RO_ERR_CAPACITY, "ro_render_batch: context created with max_batch_tiles = 0");
  const int twl = ilog2(sched.tile_w), thl = 5 - twl;
  bool debug = false;
  uint64_t tiles = 0;
  std::vector<uint32_t> key = {n_views, (uint32_t)twl, sched.order};
  for (uint32_t v = 0; v < n_views; ++v) {
    const ro_view& w = views[v];
    RO_TRY(check_view(c, &w.camera, &w.params, w.image, w.W, w.H, where));
    debug = debug || has_debug(&w.params);
    tiles += (uint64_t)((w.W + (1u << twl) - 1) >> twl) * ((w.H + (1u << thl) - 1) >> thl);
    key.push_back(w.W);
    key.push_back(w.H);
  }
  key.push_back(debug ? 1u : 0u);
  if (tiles > c->desc.max_batch_tiles) return set_err(c, RO_ERR_CAPACITY, "ro_render_batch: more tiles than max_batch_tiles");
  const Geometry& g = c->g;
  const size_t views_bytes = (size_t)ro::kMaxViews * sizeof(ro::ViewArgs);
  const size_t up_bytes = (size_t)c->L.ba_tf + (size_t)ro::kMaxC * 8;  // view table and TF ranges, one copy
  const size_t lut_bytes = (size_t)ro::kMaxC * 256 * sizeof(float4);
  if (!c->b_pinned) {
    RO_TRY(cuda_check(c, cudaMallocHost(reinterpret_cast<void**>(&c->b_pinned), up_bytes + lut_bytes), "ro_render_batch: pinned upload area"));
    std::memset(c->b_pinned, 0, up_bytes + lut_bytes);
    RO_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->b_uploaded, cudaEventDisableTiming), "ro_render_batch: event"));
    RO_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->b_capture, cudaStreamNonBlocking), "ro_render_batch: capture stream"));
  }
  // the previous batch must have read the upload area before it is refilled
  RO_TRY(wait_event(c, c->b_uploaded, "ro_render_batch: previous uploads"));
  ro::ViewArgs* hv = reinterpret_cast<ro::ViewArgs*>(c->b_pinned);
  uint32_t base = 0;
  for (uint32_t v = 0; v < n_views; ++v) {
    const ro_view& w = views[v];
    fill_view(c, &w.camera, &w.params, w.image, w.W, w.H, twl, base, &hv[v]);
    base += hv[v].tiles_x * ((w.H + (1u << thl) - 1) >> thl);
  }
  float2* htf = reinterpret_cast<float2*>(c->b_pinned + c->L.ba_tf);
  for (int ch = 0; ch < ro::kMaxC; ++ch)
    htf[ch] = ch < g.m ? make_float2(tfs[ch].lo, tfs[ch].scale) : make_float2(0.0f, 0.0f);
  float4* hlut = reinterpret_cast<float4*>(c->b_pinned + up_bytes);
  for (int ch = 0; ch < g.m; ++ch) std::memcpy(hlut + (size_t)ch * 256, tfs[ch].lut, 256 * sizeof(float4));
  (void)views_bytes;

  if (!c->b_exec || key != c->b_key) {
    if (c->b_exec) cudaGraphExecDestroy(c->b_exec);
    if (c->b_graph) cudaGraphDestroy(c->b_graph);
    c->b_exec = nullptr;
    c->b_graph = nullptr;
    c->b_key.clear();
    ro::RenderArgs a{};
    fill_common(c, tfs, &a);
    a.tile_wlog2 = twl;
    a.n_rays = tiles * 32;
    a.views = c->b_views;
    a.n_views = (int)n_views;
    a.order = sched.order == 1 ? c->b_order : nullptr;
    a.tile_cost = c->b_cost;
    a.tf_dev = c->b_tf;
    ro::PrefixArgs pa{};
    pa.m = g.m;
    pa.bpv = g.bpv;
    pa.tf_dev = c->b_tf;
    pa.lut = c->lut;
    pa.prefix = c->prefix;
    cudaStream_t cs = c->b_capture;
    RO_TRY(cuda_check(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "ro_render_batch: begin capture"));
    cudaError_t e = cudaMemcpyAsync(c->b_views, c->b_pinned, up_bytes, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->lut, hlut, (size_t)g.m * 256 * sizeof(float4), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->b_uploaded, cs, cudaEventRecordExternal);  // a node of the graph
    if (e == cudaSuccess) e = ro::launch_prefix(pa, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), cs);
    if (e == cudaSuccess && sched.order == 1) e = ro::launch_cost_order(c->b_cost, (uint32_t)tiles, c->b_order, cs);
    int launched = 0;
    if (e == cudaSuccess) e = ro::launch_render_batch(a, debug, cs, &launched);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->b_exec, graph, 0);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      c->b_exec = nullptr;
      return cuda_check(c, e, "ro_render_batch: capture");
    }
    c->b_graph = graph;
    c->b_key = key;
    c->b_blocks = (uint32_t)launched;
  }
  RO_TRY(cuda_check(c, cudaGraphLaunch(c->b_exec, c->stream), "ro_render_batch: graph launch"));
  c->last_blocks = c->b_blocks;
  ++c->frame;
  return RO_OK;
}

ro_status ro_autotune_batch(ro_ctx* c, uint32_t n_views, const ro_view* views, const ro_tf* tfs, ro_schedule* best,
                            float* best_ms) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if (!best) return set_err(c, RO_ERR_INVALID_ARG, "ro_autotune_batch: null result");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  RO_TRY(cuda_check(c, cudaEventCreate(&t0), "ro_autotune_batch: event"));
  if (cudaEventCreate(&t1) != cudaSuccess) {
    cudaEventDestroy(t0);
    return cuda_check(c, cudaErrorMemoryAllocation, "ro_autotune_batch: event");
  }
  ro_status s = RO_OK;
  float best_t = INFINITY;
  ro_schedule win{8, 0};
  const uint32_t widths[4] = {8, 4, 16, 32};
  for (uint32_t wi = 0; wi < 4 && s == RO_OK; ++wi) {
    for (uint32_t order = 0; order < 2 && s == RO_OK; ++order) {
      const ro_schedule sc{widths[wi], order};
      s = ro_render_batch(c, n_views, views, tfs, &sc);  // warm-up; records this tiling's costs
      for (int rep = 0; rep < 2 && s == RO_OK; ++rep) {
        s = cuda_check(c, cudaEventRecord(t0, c->stream), "ro_autotune_batch: event");
        if (s == RO_OK) s = ro_render_batch(c, n_views, views, tfs, &sc);
        if (s == RO_OK) s = cuda_check(c, cudaEventRecord(t1, c->stream), "ro_autotune_batch: event");
        if (s == RO_OK) s = wait_event(c, t1, "ro_autotune_batch");
        float ms = 0.0f;
        if (s == RO_OK) s = cuda_check(c, cudaEventElapsedTime(&ms, t0, t1), "ro_autotune_batch: timing");
        if (s == RO_OK && ms < best_t) {
          best_t = ms;
          win = sc;
        }
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (s != RO_OK) return s;
  RO_TRY(wait_stream(c, "ro_autotune_batch"));
  *best = win;
  if (best_ms) *best_ms = best_t;
  return RO_OK;
}

ro_status ro_replace_channel(ro_ctx* c, uint32_t ch) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  const Geometry& g = c->g;
  if (ch >= (uint32_t)g.m) return set_err(c, RO_ERR_INVALID_ARG, "ro_replace_channel: channel out of range");
  const uint64_t first = g.pt_off[ch * g.k], last = g.pt_off[(ch + 1) * g.k];
  // the channel's resident bricks give their slots back
  for (uint64_t pi = first; pi < last; ++pi) {
    const uint32_t sl = c->slot_of_brick[pi];
    if (sl == RO_NONE) continue;
    c->slot_of_brick[pi] = RO_NONE;
    c->brick_of_slot[sl] = RO_NONE;
    c->free_slots.push_back(sl);
  }
  std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<uint32_t>());
  c->pending.erase(std::remove_if(c->pending.begin(), c->pending.end(),
                                  [&](uint32_t pi) { return pi >= first && pi < last; }),
                   c->pending.end());
  cudaStream_t st = c->stream;
  RO_TRY(cuda_check(c, cudaMemsetAsync(c->pt + first, 0, (last - first) * 4, st), "ro_replace_channel: page tables"));
  RO_TRY(cuda_check(c, cudaMemsetAsync(c->req + first, 0, last - first, st), "ro_replace_channel: requests"));
  RO_TRY(cuda_check(c, ro::launch_fill_strided(c->octree + ch, g.n_nodes, (uint32_t)g.mp, ro::kInvalidUnknown, st),
                    "ro_replace_channel: octree"));
  RO_TRY(cuda_check(c, ro::launch_fill_strided(c->given + ch, g.node_off[g.D], (uint32_t)g.mp, 0u, st),
                    "ro_replace_channel: given ranges"));
  return RO_OK;
}

ro_status ro_read_requests(ro_ctx* c, uint32_t* ids, uint32_t cap, uint32_t* n, uint32_t* overflow, uint32_t* node_ids,
                           uint32_t node_cap, uint32_t* n_node) {
  if (!c) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  if ((cap && !ids) || (node_cap && !node_ids)) return set_err(c, RO_ERR_INVALID_ARG, "ro_read_requests: null list");
  const Geometry& g = c->g;
  cudaStream_t st = c->stream;
  uint32_t* counts = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_counts);
  uint32_t* totals = reinterpret_cast<uint32_t*>(c->scratch + c->L.sc_totals);
  ro::CompactArgs a{};
  a.g = g;
  a.block_counts = counts;
  a.flags = c->req;
  a.n = c->L.req_pad;
  a.n_tiles = (uint32_t)(c->L.req_pad / ro::kCompactTile);
  a.out = c->req_out;
  a.cap = c->desc.max_requests;
  a.total = totals;
  a.id_mode = 0;
  RO_TRY(cuda_check(c, ro::launch_compact(a, st), "ro_read_requests: compact"));
  a.flags = c->node_req;
  a.n = c->L.node_req_pad;
  a.n_tiles = (uint32_t)(c->L.node_req_pad / ro::kCompactTile);
  a.out = c->node_out;
  a.total = totals + 1;
  a.id_mode = 1;
  RO_TRY(cuda_check(c, ro::launch_compact(a, st), "ro_read_requests: compact nodes"));
  ro::UsageArgs u{};
  u.used = c->used;
  u.last_used = c->last_used;
  u.n = c->desc.cache_slots;
  u.frame = c->frame;
  RO_TRY(cuda_check(c, ro::launch_usage(u, st), "ro_read_requests: usage"));
  // wait (with the deadline) before any copy into pageable host memory: such
  // a copy would itself block until the stream reaches it
  RO_TRY(wait_stream(c, "ro_read_requests"));
  // the usage stamps the next uploads choose victims by (only needed once
  // the cache is full)
  if (c->free_slots.empty())
    RO_TRY(cuda_check(c, cudaMemcpyAsync(c->stamps.data(), c->last_used, 4ull * c->desc.cache_slots,
                                         cudaMemcpyDeviceToHost, st), "ro_read_requests: stamps"));
  uint32_t tot[2] = {0, 0};
  RO_TRY(cuda_check(c, cudaMemcpyAsync(tot, totals, 8, cudaMemcpyDeviceToHost, st), "ro_read_requests: totals"));
  const uint32_t nr = std::min({tot[0], cap, c->desc.max_requests});
  const uint32_t nn = std::min({tot[1], node_cap, c->desc.max_requests});
  if (nr) RO_TRY(cuda_check(c, cudaMemcpyAsync(ids, c->req_out, 4ull * nr, cudaMemcpyDeviceToHost, st), "ro_read_requests: ids"));
  if (nn)
    RO_TRY(cuda_check(c, cudaMemcpyAsync(node_ids, c->node_out, 4ull * nn, cudaMemcpyDeviceToHost, st), "ro_read_requests: nodes"));
  if (nr || nn) RO_TRY(wait_stream(c, "ro_read_requests"));
  if (n) *n = nr;
  if (overflow) *overflow = tot[0] - nr;
  if (n_node) *n_node = nn;
  return RO_OK;
}

ro_status ro_get_stats(ro_ctx* c, uint64_t out[8]) {
  if (!c || !out) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  RO_TRY(wait_stream(c, "ro_get_stats"));
  std::vector<unsigned long long> v((size_t)c->last_blocks * ro::kStats);
  if (!v.empty())
    RO_TRY(cuda_check(c, cudaMemcpyAsync(v.data(), c->scratch + c->L.sc_stats, v.size() * 8, cudaMemcpyDeviceToHost, c->stream),
                      "ro_get_stats"));
  for (int q = 0; q < 8; ++q) out[q] = 0;
  for (size_t b = 0; b < c->last_blocks; ++b)
    for (int q = 0; q < ro::kStats; ++q) out[q] += v[b * ro::kStats + q];
  return RO_OK;
}

ro_status ro_debug_read(ro_ctx* c, uint32_t what, void* host, uint64_t bytes) {
  if (!c || !host) return RO_ERR_INVALID_ARG;
  if (c->latched != RO_OK) return c->latched;
  const void* src = nullptr;
  uint64_t size = 0;
  switch (what) {
    case 0: src = c->octree; size = c->g.n_nodes * (uint64_t)c->g.mp * 4; break;
    case 1: src = c->pt; size = c->g.n_bricks * 4; break;
    case 2: src = c->last_used; size = 4ull * c->desc.cache_slots; break;
    case 3: src = c->req; size = c->g.n_bricks; break;
    case 4: src = c->used; size = c->desc.cache_slots; break;
    case 5: src = c->cache; size = (uint64_t)c->desc.cache_slots * c->g.slot_pitch; break;
    default: return set_err(c, RO_ERR_INVALID_ARG, "ro_debug_read: unknown array");
  }
  if (bytes != size) return set_err(c, RO_ERR_INVALID_ARG, "ro_debug_read: size mismatch");
  RO_TRY(wait_stream(c, "ro_debug_read"));
  RO_TRY(cuda_check(c, cudaMemcpyAsync(host, src, size, cudaMemcpyDeviceToHost, c->stream), "ro_debug_read"));
  return wait_stream(c, "ro_debug_read");
}

}  // extern "C"
