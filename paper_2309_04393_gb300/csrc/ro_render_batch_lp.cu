// Batch launches of the ray caster for the binary16 and bfloat16 sample
// formats.
#include "ro_render_kernel.cuh"

namespace ro {

cudaError_t launch_render_batch_lp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  if (a.g.sf == 1) return launch_any<true, 1>(a, debug, s, blocks_out);
  if (a.g.sf == 2) return launch_any<true, 2>(a, debug, s, blocks_out);
  return cudaErrorInvalidValue;
}

}  // namespace ro
