// Single-view launches of the ray caster for the binary16 and bfloat16
// sample formats; a translation unit of its own so that the
// instantiations compile in parallel with the others.
#include "ro_render_kernel.cuh"

namespace ro {

cudaError_t launch_render_lp(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  if (a.g.sf == 1) return launch_any<false, 1>(a, debug, s, blocks_out);
  if (a.g.sf == 2) return launch_any<false, 2>(a, debug, s, blocks_out);
  return cudaErrorInvalidValue;
}

}  // namespace ro
