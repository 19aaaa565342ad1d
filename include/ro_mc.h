/*
 * ro_mc.h — C ABI of the learned miss compensator (GB300, sm_103a).
 *
 * The paper renders a missing brick from the next coarser resident level
 * (Sec. 6.1, getAlternativeBrick; Sec. 6.2).  The compensator predicts the
 * missing level-0 brick from its resident level-1 parent instead:
 *  upsample  the level-0 apron grid (34^3 for 32^3 bricks) sampled
 *            trilinearly from the parent's apron slot at the renderer's
 *            voxel-centre coordinates (level-1 coordinate (X + 0.5) / 2 -
 *            0.5 for level-0 voxel X), values scaled by 2^-16;
 *  network   y = x0 + f(x0), f = four 3x3x3 convolutions with zero padding
 *            (1 -> 32 -> 32 -> 32 -> 1 channels, bias, ReLU after the first
 *            three), weights used in bfloat16, sums in binary32;
 *  training  mean squared error against the true level-0 slot, Adam.
 * Parameters are RO_MC_PARAMS floats: for each layer the weights W[tap][ci][co]
 * (tap = (dz * 3 + dy) * 3 + dx) followed by the biases [co].
 *
 * Conventions as in ro.h: every call returns an ro_status; device memory is
 * the caller's (one arena of ro_mc_query_bytes bytes); work is enqueued on
 * the stream given at creation (a training step runs its weight gradients
 * on an internal second stream that forks from and joins back into that
 * stream within the call); grids are device arrays, x fastest.
 * Gradients are summed with atomic adds, so their last bits depend on the
 * order blocks finish.
 */
#ifndef RO_MC_H
#define RO_MC_H

#include <stdint.h>

#include "ro.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RO_MC_EDGE 34
#define RO_MC_VOXELS (RO_MC_EDGE * RO_MC_EDGE * RO_MC_EDGE)
#define RO_MC_PARAMS 57121

typedef struct ro_mc ro_mc;

/* max_batch: grids per call (>= 1). */
typedef struct {
  uint32_t max_batch;
} ro_mc_desc;

/* Bytes of the device arena for desc (parameters, bfloat16 copies, Adam
 * moments, activations and gradients of max_batch grids). */
ro_status ro_mc_query_bytes(const ro_mc_desc* desc, uint64_t* bytes);

/* Creates a compensator over the caller's arena (256-byte aligned, at
 * least ro_mc_query_bytes bytes) on `stream` (a cudaStream_t), with one
 * internal stream and five events of its own (freed by ro_mc_destroy).
 * Parameters start at zero: set them with ro_mc_set_params. */
ro_status ro_mc_create(const ro_mc_desc* desc, void* arena_device, uint64_t arena_bytes, void* stream, ro_mc** out);

/* Waits for the stream and frees the host-side state. */
ro_status ro_mc_destroy(ro_mc* mc);

/* Copies RO_MC_PARAMS floats from the host, refreshes the bfloat16 copies
 * and zeroes the Adam moments and step count. */
ro_status ro_mc_set_params(ro_mc* mc, const float* host_params);

/* Copies the RO_MC_PARAMS binary32 parameters to the host (waits).
 * Returns RO_ERR_INTERNAL, with the parameters copied, once a tensor-core
 * convolution of this context gave up waiting for its matrix instructions
 * (half a second; its output grid is then incomplete).  The flag is latched
 * for the life of the context. */
ro_status ro_mc_get_params(ro_mc* mc, float* host_params);

/* n <= max_batch level-1 apron slots (device, n * RO_MC_VOXELS u16 raw
 * values) and the child octant of each (device, n u32: bit 0 x, bit 1 y,
 * bit 2 z) -> x0 (device, n * RO_MC_VOXELS floats, scaled by 2^-16). */
ro_status ro_mc_upsample(ro_mc* mc, uint32_t n, const uint16_t* l1_slots, const uint32_t* octants, float* x0);

/* y = x0 + f(x0) for n grids (device pointers, n * RO_MC_VOXELS floats). */
ro_status ro_mc_forward(ro_mc* mc, uint32_t n, const float* x0, float* y);

/* Loss (device, one float: the mean squared error over n grids) and its
 * gradients (device, RO_MC_PARAMS floats) for targets t (device, scaled). */
ro_status ro_mc_gradients(ro_mc* mc, uint32_t n, const float* x0, const float* target, float* grads, float* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * gradients of n grids; loss as above (device, may be NULL). */
ro_status ro_mc_train_step(ro_mc* mc, uint32_t n, const float* x0, const float* target, float lr, float* loss);

/* One Adam step (as ro_mc_train_step) on caller-given gradients (device,
 * RO_MC_PARAMS floats, the layout of the parameters), e.g. gradients of
 * several batches or of several data-parallel ranks summed and scaled by
 * the caller.  Advances the step count that the bias corrections use. */
ro_status ro_mc_apply_gradients(ro_mc* mc, const float* grads, float lr);

/* Copies the Adam moment estimates (RO_MC_PARAMS floats each: the moving
 * averages of the gradient and of its square, before bias correction) to
 * the host and returns the number of Adam steps taken since the last
 * ro_mc_set_params (step may be NULL).  Waits for the stream. */
ro_status ro_mc_get_moments(ro_mc* mc, float* host_m, float* host_v, uint32_t* step);

/* Makes n missing level-0 bricks resident with predicted data (the
 * substitution of Sec. 6.1 refined by the compensator): for each ID the
 * level-1 parent must be resident; its cache slot is upsampled to the
 * child's apron grid, the network's output y is converted to raw values
 * (round(y * 65536), clamped to [0, 65535]) and placed like ro_upload_bricks
 * places a brick (free slot, else least recently used; a parent of this call
 * is never evicted).  The renderer then samples the predicted brick and no
 * longer requests it; ro_upload_bricks of the same ID later replaces the
 * prediction with the real data.  Needs 32^3 u16 bricks, sample_format 0 and
 * at least 2 levels; n <= max_upload, n <= cache_slots and n <= the
 * compensator's max_batch (RO_ERR_CAPACITY).  IDs must be level 0, not
 * resident, without duplicates (RO_ERR_INVALID_ARG).  out_slots (host, may
 * be NULL) receives the slots.  Waits for the stream.  Should a tensor-core
 * wait of the network give up (the latched flag ro_mc_get_params reports),
 * the predictions placed by that call are incomplete. */
ro_status ro_compensate_bricks(ro_ctx* ctx, ro_mc* mc, uint32_t n, const uint32_t* level0_ids, uint32_t* out_slots);

#ifdef __cplusplus
}
#endif

#endif /* RO_MC_H */
