/*
 * ro.h — C ABI of the residency-octree ray caster (GB300, sm_103a).
 *
 * The library implements the per-frame path of the Residency Octree method
 * (Herzberger et al., arXiv 2309.04393): a multi-channel multi-resolution
 * page-table hierarchy over one brick cache (Sec. 5.1), a residency octree
 * whose nodes hold per-channel partial-residency bitmasks and min/max
 * metadata (Sec. 5.2, Sec. 7), its incremental update (Sec. 5.3), and the
 * mixed-resolution multi-volume ray caster with empty-space skipping,
 * coarser-level substitution and ray-guided request emission (Sec. 6.1,
 * Algorithm 1; Sec. 6.2).
 *
 * Conventions for every call:
 *  - Every call returns an ro_status and never aborts.  A CUDA error is
 *    latched in the context: later calls return RO_ERR_CUDA until the
 *    context is destroyed.  ro_last_error() gives a one-line message.
 *  - Device memory is owned by the caller.  ro_query_sizes() says how many
 *    bytes one device arena needs; the caller allocates it (e.g. a torch
 *    uint8 tensor) and passes its pointer to ro_create().  The library never
 *    calls cudaMalloc.  Host buffers passed in are owned by the caller.
 *  - All device work is enqueued on the stream given to ro_create().  Calls
 *    that return host data (ro_read_requests, ro_upload_bricks when it must
 *    evict, ro_get_stats, ro_debug_read) wait for that stream by polling an
 *    event against a deadline (ro_set_timeout, default 30 s) and return
 *    RO_ERR_TIMEOUT when it passes.
 *  - Arrays are C order with x fastest ([z][y][x]).  Sizes are in voxels
 *    unless stated.  Positions are physical: the volume occupies
 *    [0, dims[a] * spacing[a]) on each axis.
 *  - Not thread-safe: one host thread per context.
 */
#ifndef RO_H
#define RO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RO_MAX_CHANNELS 16
#define RO_MAX_LEVELS 16
#define RO_MAX_VIEWS 256
#define RO_NONE 0xFFFFFFFFu

typedef enum {
  RO_OK = 0,
  RO_ERR_INVALID_ARG = 1, /* a size, pointer or id outside what the call accepts */
  RO_ERR_CUDA = 2,        /* a CUDA runtime error (latched) */
  RO_ERR_CAPACITY = 3,    /* arena too small, or more items than the descriptor allows */
  RO_ERR_TIMEOUT = 4,     /* the stream did not reach the call's event before the deadline */
  RO_ERR_INTERNAL = 5     /* a device-side index guard fired (latched) */
} ro_status;

/* Volume, cache and octree parameters, fixed at creation (Sec. 5.1: brick
 * size, cache size and channel count; Sec. 5.2: octree depth via the leaf
 * extent; Sec. 7: m, k chosen at initialisation).
 *  dims          level-0 voxels per axis, each >= 1
 *  spacing       physical size of a level-0 voxel per axis, > 0
 *  channels      m, 1..16
 *  value_bits    8 (u8) or 16 (u16) per voxel
 *  brick         B, brick edge in voxels: 8, 16, 32 or 64
 *  levels        k, 1..16, with m*k <= 256 (the 8-bit page-table id)
 *  leaf_extent   octree leaf extent in level-0 voxels per axis: a power of
 *                two <= B (so a leaf lies inside one brick of every level)
 *  cache_slots   brick cache capacity in bricks, >= 1
 *  max_requests  request-list limit per frame (Sec. 4), >= 1
 *  max_upload    bricks per ro_upload_bricks call, >= 1
 *  max_meta      leaf metadata entries per ro_update_residency_octree chunk
 *  max_batch_tiles  pixel tiles (32 pixels each) one ro_render_batch call may
 *                cover, summed over its views; 0 = no batches
 *  sample_format 0: the cache holds the raw values and trilinear lerps run in
 *                binary32; 1: binary16, 2: bfloat16 - the cache holds
 *                round(v * 2^-bits) in the format (2 bytes per voxel, also
 *                for 8-bit data), the lerps run in the format with one
 *                rounding per step and the result times 2^bits continues in
 *                binary32 (TF, opacity correction and compositing stay
 *                binary32)
 *  keep_axes     downsampling between levels (Sec. 8: anisotropic volumes
 *                and downsampling ratios, e.g. in two dimensions only): bit a
 *                of keep_axes[l] set = axis a (x, y, z) keeps its resolution
 *                from level l to level l + 1; clear = halved (ceil(d / 2)).
 *                All zero (the default) halves every axis at every level.
 *                Bits above 2 and entries l >= levels - 1 must be zero.
 *                The sampling step after a sample read at level l grows by
 *                2^s, s the largest exponent with 2^s * min(spacing) <= the
 *                smallest physical extent of a level-l voxel (s = l when
 *                every axis is halved).
 * Bricks per axis at every level must be <= 256 (the 8-bit offsets of the
 * brick ID, Sec. 7). */
typedef struct {
  uint32_t dims[3];
  float spacing[3];
  uint32_t channels;
  uint32_t value_bits;
  uint32_t brick;
  uint32_t levels;
  uint32_t leaf_extent[3];
  uint32_t cache_slots;
  uint32_t max_requests;
  uint32_t max_upload;
  uint32_t max_meta;
  uint32_t max_batch_tiles;
  uint32_t sample_format;
  uint32_t keep_axes[16];
} ro_desc;

/* Byte sizes of the parts of the device arena (all 256-byte aligned inside
 * it, in this order) and their sum. */
typedef struct {
  uint64_t cache;        /* cache_slots * slot_pitch voxels bytes */
  uint64_t page_table;   /* one u32 per brick of the virtual hierarchy: slot + 1, 0 = absent */
  uint64_t octree;       /* n_nodes * channel_stride u32 node words */
  uint64_t req_flags;    /* one byte per brick */
  uint64_t node_req_flags;/* one byte per (node, channel) */
  uint64_t used_flags;   /* one byte per slot */
  uint64_t last_used;    /* one u32 frame stamp per slot */
  uint64_t staging;      /* max_upload bricks, host-to-device landing area */
  uint64_t frame;        /* per-frame constants: LUTs, bucket prefix sums */
  uint64_t lists;        /* request / node-request output lists + counts */
  uint64_t scratch;      /* compaction partial counts, update item lists, stats */
  uint64_t total;
  uint64_t slot_pitch;   /* bytes per cache slot ((B+2)^3 voxels of 1 or 2 bytes, padded) */
  uint64_t n_bricks;     /* bricks of the virtual hierarchy, all channels and levels */
  uint64_t n_nodes;      /* octree nodes, all depths */
  uint32_t depth;        /* octree depth D (leaves at depth D) */
  uint32_t channel_stride;/* u32 words per node: channels rounded up to a power of two */
  uint64_t batch;        /* batch view table, tile schedule and tile costs (last in the arena) */
} ro_buffer_sizes;

typedef struct ro_ctx ro_ctx;

/* Fills *out for desc.  Returns RO_ERR_INVALID_ARG for a descriptor that
 * breaks any rule above. */
ro_status ro_query_sizes(const ro_desc* desc, ro_buffer_sizes* out);

/* Creates a context over the caller's device arena (arena_bytes >=
 * sizes.total, 256-byte aligned) on the CUDA stream `stream` (a
 * cudaStream_t; NULL = legacy default stream) of the current device.
 * Enqueues the initialisation: empty page tables, every node INVALID with an
 * empty mask for every channel (Sec. 5.2), cleared flags.  The arena must
 * stay allocated until ro_destroy. */
ro_status ro_create(const ro_desc* desc, void* arena_device, uint64_t arena_bytes, void* stream, ro_ctx** out);

/* Waits for the context's stream and frees the host-side context.  The
 * arena is the caller's to free afterwards. */
ro_status ro_destroy(ro_ctx* ctx);

/* Makes n bricks resident (Sec. 5.3, "Updating residency information" and
 * "LRU cache eviction").
 *  brick_ids  n IDs in the 32-bit format of Sec. 7: page-table id c*k + l in
 *             bits 31:24, then z, y, x brick offsets (8 bits each); no
 *             duplicates within one call.
 *  voxels     host pointer to n bricks of (B+2)^3 voxels each (u8 or u16 per
 *             value_bits), x fastest, holding level-l voxels b*B-1 .. (b+1)*B
 *             per axis clamped to the level (a one-voxel border).  Copied
 *             before the call returns; pinned memory makes the copy faster.
 *  out_slots  n slots chosen (host), may be NULL.
 *  out_evicted n IDs evicted to make room, RO_NONE where a free slot was
 *             used (host), may be NULL.
 * A brick already resident keeps its slot and gets its data rewritten.
 * Free slots are used first, in ascending order; then the least recently
 * used slots (stamped by ro_read_requests), never one chosen earlier in the
 * same call.  The page table is updated on the device; the octree masks
 * change at the next ro_update_residency_octree.  n <= max_upload and
 * n <= cache_slots, else RO_ERR_CAPACITY. */
ro_status ro_upload_bricks(ro_ctx* ctx, uint32_t n, const uint32_t* brick_ids, const void* voxels,
                           uint32_t* out_slots, uint32_t* out_evicted);

/* ro_upload_bricks with the host-to-device copy on copy_stream (a
 * cudaStream_t), so that it can run while a render enqueued earlier on the
 * context's stream is still running (Sec. 4: requested bricks stream in
 * while the renderer goes on).  voxels must be page-locked host memory
 * (cudaHostAlloc or registered) and stay unchanged until ro_upload_wait, or
 * the next upload call, returns.  The copy waits for the previous upload's
 * scatter (the staging area); the scatter into the cache and the page table
 * runs on the context's stream after the copy and after everything enqueued
 * there before this call, so a render never sees a slot change under it.
 * Slots are chosen as by ro_upload_bricks, from the usage stamps of the last
 * ro_read_requests; out_slots / out_evicted are filled before returning.
 * The call itself does not wait for the GPU. */
ro_status ro_upload_bricks_async(ro_ctx* ctx, uint32_t n, const uint32_t* brick_ids, const void* voxels,
                                 uint32_t* out_slots, uint32_t* out_evicted, void* copy_stream);

/* Waits (with the context's deadline) until the last asynchronous upload's
 * copy has landed; its host buffer may then be reused.  RO_OK at once when
 * none is pending. */
ro_status ro_upload_wait(ro_ctx* ctx);

/* Leaf metadata entry: raw value range of channel `channel` over leaf
 * `leaf` (x fastest over ceil(dims / leaf_extent) leaves per axis).  The
 * range must cover every level-0 voxel whose trilinear support reaches the
 * leaf.  vmin > vmax marks the leaf's channel INVALID again. */
typedef struct {
  uint32_t leaf;
  uint32_t channel;
  uint32_t vmin;
  uint32_t vmax;
} ro_leaf_meta;

/* Brings the residency octree up to date (Sec. 5.3): writes the n_meta leaf
 * ranges (quantised to the 8-bit node format of Sec. 7: u16 values >> 8),
 * recomputes the partial-residency masks of every leaf that overlaps a brick
 * uploaded or evicted since the previous call, and recomputes every
 * ancestor of a changed leaf as the bitwise OR of its children's masks and
 * the hull of their ranges when all children are valid, else the range
 * given for the node itself (ro_update_node_metadata), else INVALID.  An
 * INVALID word (Sec. 5.2) keeps its mask and holds min8 = 255 and max8 =
 * the depth of the node's nearest valid ancestor, or RO_UNKNOWN_DEPTH when
 * no ancestor is valid; the renderer reads such a word with that
 * ancestor's range.  No atomics.  meta is a host pointer (NULL if
 * n_meta = 0). */
ro_status ro_update_residency_octree(ro_ctx* ctx, uint32_t n_meta, const ro_leaf_meta* meta);

#define RO_UNKNOWN_DEPTH 254u

/* Metadata for a volume region of any size (Sec. 5.3: metadata arriving
 * for a region, e.g. in answer to a node request): the raw value range of
 * channel `channel` over node `node`, numbered as node requests number nodes
 * (depth-major from the root, then z, y, x; leaves last).  For a leaf it is
 * the leaf range of ro_leaf_meta.  For an inner node it is used while not all
 * of its children are valid (then their hull is tighter); it must cover
 * every level-0 voxel whose trilinear support reaches the node.
 * vmin > vmax withdraws a given range. */
typedef struct {
  uint32_t node;
  uint32_t channel;
  uint32_t vmin;
  uint32_t vmax;
} ro_node_meta;

/* Writes n_meta node ranges, then brings the octree up to date as
 * ro_update_residency_octree does (pending brick changes included); the
 * INVALID words below a node that gained a range point to it.  meta is a
 * host pointer (NULL if n_meta = 0); RO_ERR_INVALID_ARG for a node or
 * channel out of range. */
ro_status ro_update_node_metadata(ro_ctx* ctx, uint32_t n_meta, const ro_node_meta* meta);

/* Camera (physical units).  ortho (perspective = 0): pixel (i, j) starts at
 * eye + a*right + b*up, a = (i + 0.5 - W/2)*pixel, b = (H/2 - j - 0.5)*pixel,
 * and travels along forward.  perspective: rays start at eye along
 * normalize(forward + a*right + b*up), a = (2(i + 0.5)/W - 1)*tan_x,
 * b = (1 - 2(j + 0.5)/H)*tan_y.  forward/right/up are unit vectors. */
typedef struct {
  float eye[3];
  float forward[3];
  float right[3];
  float up[3];
  uint32_t perspective;
  float tan_x, tan_y;
  float pixel;
} ro_camera;

/* Transfer function of one channel: a raw value v maps to the LUT
 * coordinate clamp((v - lo) * scale, 0, 255) and to the RGBA interpolated
 * linearly between the 256 knots of lut (host pointer, 256*4 floats). */
typedef struct {
  float lo;
  float scale;
  const float* lut;
} ro_tf;

/* Per-frame rendering parameters.
 *  dt          lattice spacing along the ray, physical units, > 0
 *  lod_t       desired-level thresholds: lod(t) = #{l in 1..k-1 : t >= lod_t[l]}
 *              (t = physical distance from the ray origin); index 0 unused;
 *              lod_t[1..k-1] must be non-decreasing (+inf allowed)
 *  lmin, lmax  per-channel level range, 0 <= lmin <= lmax < k (Sec. 6.2)
 *  start_depth octree depth at which traversal starts (Sec. 7), <= depth
 *  skip        1 = empty-space skipping on
 *  ert         early ray termination once transmittance < ert; 0 = off
 *  debug_*     optional device pointers (W*H u32 each) for the per-pixel
 *              selection hash, evaluated samples, final lattice index and
 *              brick samples; NULL to skip.
 *  order       ro_render only: 0 = pixel tiles row by row; 1 = longest tiles
 *              first, by the per-tile costs the previous frame of the same
 *              size recorded (the frame then runs as a one-view batch, see
 *              ro_render_batch; needs max_batch_tiles >= its tiles, else
 *              rows are used).  Changes the speed only. */
typedef struct {
  float dt;
  float lod_t[RO_MAX_LEVELS];
  uint32_t lmin[RO_MAX_CHANNELS];
  uint32_t lmax[RO_MAX_CHANNELS];
  uint32_t start_depth;
  uint32_t skip;
  float ert;
  uint32_t* debug_hash;
  uint32_t* debug_n_eval;
  uint32_t* debug_i_end;
  uint32_t* debug_n_bs;
  uint32_t order;
} ro_render_params;

/* Renders one frame (Sec. 6): one thread per pixel marches its ray through
 * the residency octree, skips empty nodes, picks each channel's brick
 * (substituting coarser resident levels on a miss), samples it trilinearly,
 * applies the channel's TF with opacity correction for the adaptive step,
 * composites additively front to back with early termination, and flags
 * requested bricks, requested nodes and used slots with plain stores.
 *  tfs       host array of m transfer functions
 *  image     device pointer, W*H RGBA float32 (16 bytes per pixel), row j
 *            at image + 4*W*j; written for every pixel
 * 1 <= W, H <= 16384.  Enqueued on the stream; returns without waiting. */
ro_status ro_render(ro_ctx* ctx, const ro_camera* camera, const ro_tf* tfs, const ro_render_params* params,
                    float* image, uint32_t W, uint32_t H);

/* One view of a batch: its camera, parameters (as for ro_render, debug
 * pointers included) and image (device pointer, W*H RGBA float32). */
typedef struct {
  ro_camera camera;
  ro_render_params params;
  float* image;
  uint32_t W, H;
} ro_view;

/* How a batch's pixels are handed to the warps.
 *  tile_w  tile width in pixels: 1, 2, 4, 8, 16 or 32; a tile is tile_w x
 *          (32 / tile_w) pixels and one warp renders it
 *  order   0: views in order, tiles row by row within a view;
 *          1: tiles by descending cost recorded when the previous batch with
 *          the same tiling ran (longest first, which shortens the tail of the
 *          launch); tiles of equal cost in any order.
 * The schedule changes the speed only: every schedule renders the same
 * images, requests and counters. */
typedef struct {
  uint32_t tile_w;
  uint32_t order;
} ro_schedule;

/* Renders n_views views in one persistent launch (the per-pixel rays of
 * Sec. 6 are independent, so the views share one pool of warps and one
 * tail).  Each view is rendered exactly as ro_render would render it, with
 * the same transfer functions tfs (host array of m); requests, node
 * requests and usage flags of all views accumulate for ro_read_requests, and
 * ro_get_stats sums over the views.  The launch sequence (uploads of the view
 * table and the LUTs, prefix sums, schedule, ray casting) is captured once as
 * a CUDA graph per batch layout (view sizes, schedule, debug on/off) and
 * replayed while the layout stays the same; cameras, parameters, images and
 * TFs may change between calls.  The host waits (against the deadline) until
 * the previous batch's uploads have been read before refilling them.
 *  schedule  NULL = {8, 0}
 * 1 <= n_views <= RO_MAX_VIEWS; the views' tiles (ceil(W / tile_w) *
 * ceil(H / (32 / tile_w)) each) must not exceed max_batch_tiles in total
 * (RO_ERR_CAPACITY).  Enqueued on the stream; returns without waiting. */
ro_status ro_render_batch(ro_ctx* ctx, uint32_t n_views, const ro_view* views, const ro_tf* tfs,
                          const ro_schedule* schedule);

/* Picks the fastest schedule for this batch: every tile width of 4, 8, 16
 * and 32 pixels with both orders is rendered (once to warm up and record
 * costs, then timed twice with CUDA events; the faster run counts).  best
 * receives the winner and best_ms its time (may be NULL).  The renders are
 * real renders of the batch: they set its requests and usage flags.  Waits
 * for the stream. */
ro_status ro_autotune_batch(ro_ctx* ctx, uint32_t n_views, const ro_view* views, const ro_tf* tfs,
                            ro_schedule* best, float* best_ms);

/* Frees channel slot ch for another data-set channel (Sec. 5.1: the mapping
 * of data-set channels to the m channels of the structure changes at run
 * time; Sec. 5.2: the nodes' information for the new channel is INVALID
 * until it arrives).  The slot's bricks leave the cache (their slots become
 * free, their page-table entries 0), every octree node's word for ch becomes
 * INVALID with an empty mask, and the slot's pending brick requests are
 * dropped.  The caller keeps the mapping: from now on IDs and node requests
 * of ch refer to the new data-set channel, whose leaf metadata and bricks
 * arrive through ro_update_residency_octree and ro_upload_bricks as the
 * renderer requests them.  Enqueued on the stream. */
ro_status ro_replace_channel(ro_ctx* ctx, uint32_t ch);

/* Compacts the flags of the frames rendered since the previous call
 * (Sec. 4: a global request limit keeps the copy small): brick requests as
 * sorted IDs, node requests as node*m + channel, usage as
 * last_used[slot] = frame counter; clears every flag.  Waits for the stream.
 *  ids       host, capacity cap; receives min(total, cap, max_requests) IDs
 *            in ascending order
 *  n         number written; overflow = total - n
 *  node_ids  host, capacity node_cap (may be NULL with node_cap = 0) */
ro_status ro_read_requests(ro_ctx* ctx, uint32_t* ids, uint32_t cap, uint32_t* n, uint32_t* overflow,
                           uint32_t* node_ids, uint32_t node_cap, uint32_t* n_node);

/* Per-frame counters of the last ro_render, summed over its blocks:
 * [0] pixels whose ray hit the volume, [1] evaluated lattice samples,
 * [2] channel samples read from bricks, [3] samples rendered from
 * homogeneous nodes, [4] skips, [5] lattice samples skipped over.
 * Waits for the stream. */
ro_status ro_get_stats(ro_ctx* ctx, uint64_t out[8]);

/* Copies one internal array to the host (waits for the stream):
 * what = 0 octree words (n_nodes * channel_stride u32), 1 page table
 * (n_bricks u32), 2 last_used (cache_slots u32), 3 request flags (n_bricks
 * bytes), 4 used flags (cache_slots bytes), 5 the brick cache
 * (cache_slots * slot_pitch bytes).  bytes must equal the array's
 * size. */
ro_status ro_debug_read(ro_ctx* ctx, uint32_t what, void* host, uint64_t bytes);

/* Linear index of a brick ID in the page table (c*k + l table, then z, y,
 * x), or RO_NONE for an ID outside the hierarchy. */
uint32_t ro_brick_index(const ro_ctx* ctx, uint32_t brick_id);

/* Deadline for the waits above, in milliseconds (default 30000). */
ro_status ro_set_timeout(ro_ctx* ctx, uint32_t ms);

/* Message of the last error of this context (static storage while the
 * context lives); "ok" if none.  A NULL ctx gives the last ro_create error. */
const char* ro_last_error(const ro_ctx* ctx);

/* Flag compaction that allocates no memory.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory, such as a
 * plugin whose host application owns all GPU memory and gives it no
 * allocator, or a frame loop in which a device allocation would stall or
 * synchronise the GPU.  It runs the same compaction as the request readback
 * of ro_read_requests, without a context:
 *  flags    device pointer, n_flags bytes, 16-byte aligned; non-zero = set.
 *           Every flag is cleared.
 *  n_flags  a multiple of 16, at most 2^28 (268,435,456); larger sizes
 *           return RO_ERR_CAPACITY, other sizes RO_ERR_INVALID_ARG.
 *  ids      device pointer, cap u32: the indices of the set flags in
 *           ascending order, the first min(total, cap) of them (may be NULL
 *           when cap = 0).
 *  total    device pointer to one u32: the number of set flags.
 *  stream   cudaStream_t the work is enqueued on (NULL = legacy default
 *           stream); the call returns without waiting.
 * flags, ids, total and stream must belong to the calling thread's current
 * device: the scratch used is that device's copy.
 * Its per-tile counts live in one 256 KiB array in device memory, part of the
 * library itself, which every GPU that loads the library holds until the
 * process exits; it never calls cudaMalloc, cudaFree or any allocating
 * routine.  The first call on a device looks up that array's device address
 * (with the device current), so make the first call on each device before
 * any stream capture.  Every call overwrites the counts it uses before
 * reading them, and all calls share the one array: calls whose work overlaps
 * on the GPU (other streams, other threads) race and give wrong lists, so
 * order them on one stream or with events.  Returns RO_ERR_CUDA if the
 * lookup or the launch fails. */
ro_status ro_compact_flags_noalloc(uint8_t* flags, uint64_t n_flags, uint32_t* ids, uint32_t cap,
                                   uint32_t* total, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RO_H */
