// Internal declarations shared by the library's translation units (host
// runtime and kernels).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct ro_mc;

namespace ro {

constexpr int kMaxC = 16;       // channels per context (RO_MAX_CHANNELS)
constexpr int kMaxL = 16;       // levels per context (RO_MAX_LEVELS)
constexpr int kMaxDepth = 24;   // octree depth bound (2^24 leaves per axis)
constexpr int kMaxSamples = 1 << 24;  // lattice indices stay exact in binary32
// threads of a persistent render block (one per SM; rays are taken in 8 x 4
// pixel tiles): 1024 for a single-view launch (64 registers a thread), 896
// for a batch launch, whose per-warp view copies and view index need more
// registers (72)
__host__ __device__ constexpr int render_threads(bool batch) { return batch ? 896 : 1024; }
constexpr int kStats = 8;             // per-block counters of the render kernel
constexpr int kWalkWin = 2;           // octree depths whose node words the walk loads at once
constexpr int kTopWords = 1024;       // node words of the octree's top depths kept in shared memory (4 KB)
constexpr int kWalkCache = 8;         // walk results a warp remembers (for the same view)
constexpr int kRefillLanes = 32;      // lanes that take new rays together (32: the whole tile)
constexpr int kTileParts = 32 / kRefillLanes;   // such bands per 32-pixel tile
constexpr int kWalkEntry = 24;        // words per remembered walk (header 5 + 16 selections, padded)

// Geometry derived once from the descriptor; copied by value into kernels.
struct Geometry {
  int dims0[3];
  float spacing[3];
  float dimm[3];              // largest binary32 value below dims0 (position clamp)
  int m, mp, k, B, blog2, bpv;
  int sf;                     // sample format: 0 raw / binary32 lerps, 1 binary16, 2 bfloat16
  int cbpv;                   // bytes per voxel in the cache (2 when sf != 0)
  int leaf_log2[3];
  int D;                      // octree depth (leaves at depth D)
  int ldims[kMaxL][3];        // level dims
  float ldimf[kMaxL][3];      // level dims - 1, as floats (trilinear clamp bound)
  int lsh[kMaxL][3];          // log2 of a level-l voxel's extent per axis, in level-0 voxels
  int lstep[kMaxL];           // step exponent after a sample read at level l
  int nb[kMaxL][3];           // bricks per axis per level
  uint32_t pt_off[kMaxC * kMaxL + 1];  // page-table offset of table c*k + l; [m*k] = n_bricks
  uint64_t node_off[kMaxDepth + 2];    // first node of each depth; [D+1] = n_nodes
  int nn[kMaxDepth + 1][3];   // nodes per axis per depth
  int nleaf[3];               // leaves per axis (= nn[D])
  uint64_t n_nodes, n_bricks;
  uint32_t cache_slots;
  uint32_t slot_pitch;        // bytes per cache slot
  uint32_t edge;              // B + 2 (apron slot edge)
};

// One view of a render launch: camera, image and per-view parameters.  A
// single-view launch carries it in its __grid_constant__ parameter; a batch
// keeps one per view in device memory and each warp copies the view of its
// current tile into shared memory.  Size a multiple of 16 bytes.
struct __align__(16) ViewArgs {
  float eye[3], fwd[3], right[3], up[3];
  int persp;
  float tan_x, tan_y, pixel;
  int W, H;
  float dt;
  float ert;
  int start_depth, skip;
  uint32_t tiles_x;                 // tiles per image row
  uint32_t tile_base;               // first tile of this view in the launch's tile space
  float lod_t[kMaxL];
  int sdepth[kMaxL];
  int lminu_tab[kMaxL];             // finest desired level per lod value
  uint64_t ldp_tab[kMaxL];          // desired levels of all channels (4 bits each) per lod value
  float4* image;
  uint32_t *dbg_hash, *dbg_n_eval, *dbg_i_end, *dbg_n_bs;
  uint64_t pad;
};
static_assert(sizeof(ViewArgs) % 16 == 0, "ViewArgs is copied in 16-byte pieces");

constexpr int kMaxViews = 256;      // views per batch (RO_MAX_VIEWS)

// Everything one render launch needs; passed as a __grid_constant__ parameter.
struct RenderArgs {
  Geometry g;
  ViewArgs v;                       // the view of a single-view launch
  float tf_lo[kMaxC], tf_scale[kMaxC];
  const uint8_t* cache;
  const uint32_t* pt;
  const uint32_t* octree;
  uint8_t* req;
  uint8_t* node_req;
  uint8_t* used;
  const float4* lut;          // m * 256 knots
  const uint16_t* prefix;     // m * 257 bucket-occupancy prefix sums
  unsigned long long* block_stats;  // kStats per block
  uint32_t* err;
  unsigned long long* work;         // ray counter of the persistent launch (zeroed before it)
  uint64_t n_rays;                  // tiles * 32
  int tile_wlog2;                   // tile width log2 (tile = 2^w x 2^(5-w) pixels)
  // batch launches
  const ViewArgs* views;            // n_views views, tile_base ascending
  int n_views;
  const uint32_t* order;            // schedule position -> tile, or null for the identity
  uint32_t* tile_cost;              // per tile part (tile * kTileParts + part): loop iterations (null = not recorded)
  const float2* tf_dev;             // batch: (lo, scale) per channel in device memory
};

struct PrefixArgs {
  int m, bpv;
  float tf_lo[kMaxC], tf_scale[kMaxC];
  const float2* tf_dev;       // if set, (lo, scale) per channel are read from here instead
  const float4* lut;
  uint16_t* prefix;
};

// One residency-octree update item: a box of leaves [lo, hi) of one channel
// whose words must be recomputed (leaf masks from the page table, then every
// ancestor by gathering its children).
struct UpdateItem {
  uint32_t lo[3], hi[3];
  uint32_t channel;
  uint32_t pad;
};

struct MetaItem {
  uint32_t leaf, channel, vmin, vmax;
};

// INVALID node words: min8 = 255, max8 = the depth of the nearest valid
// ancestor or kUnknownDepth.  Ranges given for inner nodes are kept apart as
// kGivenBit | max8 << 8 | min8 (0 = none given).
constexpr uint32_t kUnknownDepth = 254u;
constexpr uint32_t kInvalidUnknown = 0xFFu << 16 | kUnknownDepth << 24;
constexpr uint32_t kGivenBit = 1u << 16;

struct UpdateArgs {
  Geometry g;
  const uint32_t* pt;
  uint32_t* octree;
  uint32_t* given;           // ranges given for inner nodes, node * mp + channel
  const UpdateItem* items;
  uint32_t n_items;
  const MetaItem* meta;
  uint32_t n_meta;
  int depth;                 // depth being recomputed (reduce pass)
  uint32_t* err;
};

struct ScatterArgs {
  const uint8_t* staging;    // n bricks at slot_pitch
  uint8_t* cache;
  uint32_t* pt;
  const uint32_t* ins_index; // page-table index per inserted brick
  const uint32_t* ins_slot;
  uint32_t n_ins;
  const uint32_t* ev_index;  // page-table index per evicted brick
  uint32_t n_ev;
  uint32_t slot_pitch;
  uint32_t cache_slots;
  uint64_t n_bricks;
  uint32_t* err;
  int sf, bpv;               // sample format; raw bytes per voxel in the staging area
  uint32_t n_el;             // voxels per brick ((B+2)^3)
  uint32_t* last_used;       // usage stamps: an inserted brick's slot gets `frame`
  uint32_t frame;
};

struct CompactArgs {
  uint8_t* flags;            // n flags, cleared by the write pass
  uint64_t n;
  uint32_t* block_counts;    // scratch: one count per tile, then exclusive offsets
  uint32_t n_tiles;
  uint32_t* out;             // ids, capacity cap
  uint32_t cap;
  uint32_t* total;           // flags set
  int id_mode;               // 0: brick ids via page-table offsets, 1: the flag index itself
  Geometry g;
};

constexpr int kCompactThreads = 256;
constexpr int kCompactPerThread = 16;                         // one uint4 of flags
constexpr int kCompactTile = kCompactThreads * kCompactPerThread;

struct UsageArgs {
  uint8_t* used;
  uint32_t* last_used;
  uint32_t n;
  uint32_t frame;
};

// Error codes a kernel may store into the context's error word.
enum : uint32_t { kErrNone = 0, kErrNodeIndex = 1, kErrPageIndex = 2, kErrSlot = 3, kErrUpdate = 4 };

// Launchers (each returns the launch status).
cudaError_t launch_prefix(const PrefixArgs& a, cudaStream_t s);
cudaError_t launch_render(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out);
cudaError_t launch_render_batch(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out);
// the same launches for the binary16 / bfloat16 sample formats (g.sf != 0)
cudaError_t launch_render_lp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out);
cudaError_t launch_render_batch_lp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out);
// Tile order by descending recorded cost (counting sort over log-scale
// buckets; ties in any order).
cudaError_t launch_cost_order(const uint32_t* cost, uint32_t n_tiles, uint32_t* order, cudaStream_t s);
cudaError_t launch_fill_words(uint32_t* words, uint64_t n, uint32_t value, cudaStream_t s);
cudaError_t launch_fill_strided(uint32_t* first, uint64_t count, uint32_t stride, uint32_t value, cudaStream_t s);
cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s);
cudaError_t launch_write_meta(const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_leaf_masks(const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_reduce_depth(const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_write_given(const UpdateArgs& a, cudaStream_t s);   // inner-node ranges (meta[].leaf = node)
cudaError_t launch_pointer_depth(const UpdateArgs& a, cudaStream_t s); // INVALID pointers at a.depth >= 1
cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);
cudaError_t launch_usage(const UsageArgs& a, cudaStream_t s);

size_t render_smem_bytes(int mp, bool batch);

// Compensator entry points used by ro_compensate_bricks: the batch limit,
// and the synthesis of n level-0 apron slots (u16 raw values at out_pitch)
// from the level-1 parents' cache slots and the children's octants.
uint32_t mc_max_batch(const ::ro_mc* mc);
cudaError_t mc_synthesize(::ro_mc* mc, uint32_t n, const uint8_t* cache, uint32_t pitch, const uint32_t* parent_slots,
                          const uint32_t* octants, uint8_t* out, uint32_t out_pitch, cudaStream_t s);

}  // namespace ro
