// Single-view launches of the ray caster and the bucket-occupancy prefix
// sums of the transfer functions.
#include "ro_render_kernel.cuh"

namespace ro {
namespace {

// Bucket-occupancy prefix sums per channel (a bucket is occupied when the
// TF gives some value in it a non-zero opacity): one block per channel.
__global__ void __launch_bounds__(256) prefix_kernel(const __grid_constant__ PrefixArgs a) {
  __shared__ uint16_t s_occ[256];
  __shared__ uint16_t s_scan[257];
  const int c = blockIdx.x, q = threadIdx.x;
  const float4* L = a.lut + c * 256;
  float vlo, vhi;
  if (a.bpv == 1) { vlo = (float)q; vhi = (float)q; }
  else { vlo = (float)(q * 256); vhi = (float)(q * 256 + 255); }
  const float lo = a.tf_dev ? a.tf_dev[c].x : a.tf_lo[c], scale = a.tf_dev ? a.tf_dev[c].y : a.tf_scale[c];
  auto coord = [&](float v) {
    const float t = v - lo;
    const float xq = t * scale;
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

}  // namespace

size_t render_smem_bytes(int mp, bool batch) {
  const size_t threads = (size_t)render_threads(batch);
  return (size_t)mp * 256 * sizeof(float4) + (((size_t)mp * 257 * 2 + 15) & ~(size_t)15) +
         (size_t)mp * threads * sizeof(uint32_t) + (size_t)kTopWords * sizeof(uint32_t) +
         (threads / 32) * kWalkCache * kWalkEntry * sizeof(uint32_t) + 3 * threads * sizeof(float4);
}

cudaError_t launch_render(const RenderArgs& a, bool debug, cudaStream_t s, int* blocks_out) {
  if (a.g.sf != 0) return launch_render_lp(a, debug, s, blocks_out);
  return launch_any<false, 0>(a, debug, s, blocks_out);
}

cudaError_t launch_prefix(const PrefixArgs& a, cudaStream_t s) {
  prefix_kernel<<<a.m, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ro
