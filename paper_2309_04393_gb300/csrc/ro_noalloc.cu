// Flag compaction that allocates nothing (ro_compact_flags_noalloc).
//
// Some callers cannot allocate device memory at all: plugins whose host
// application owns every byte of GPU memory and hands them no allocator, and
// frame loops where a device allocation would stall or synchronise the GPU.
// For them this entry point runs the same three-pass compaction as the
// request readback, but keeps its per-tile counts in the file-scope device
// array below instead of in a context's arena.  The caller still passes the
// flag array, the output list and the output count.
#include <mutex>

#include "ro.h"
#include "ro_internal.h"

namespace {

// Per-tile counts of one call: one u32 per 4096 flags, so up to
// kStaticTiles * 4096 = 2^28 flags per call.  256 KiB, held by every GPU that
// loads the library until the process exits.
constexpr uint32_t kStaticTiles = 65536;
static __device__ __align__(256) uint32_t g_compact_scratch[kStaticTiles];

// Device address of g_compact_scratch for each device ordinal, looked up once
// per device with that device current (the host-side name of a __device__
// array is only a stand-in, never a device address).
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

}  // namespace

extern "C" ro_status ro_compact_flags_noalloc(uint8_t* flags, uint64_t n_flags, uint32_t* ids, uint32_t cap,
                                              uint32_t* total, void* stream) {
  if (!flags || !total || (cap && !ids)) return RO_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(flags) % 16) != 0 || (n_flags % 16) != 0) return RO_ERR_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t tiles = (n_flags + ro::kCompactTile - 1) / ro::kCompactTile;
  if (tiles > kStaticTiles) return RO_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RO_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_compact_scratch) != cudaSuccess || !p) return RO_ERR_CUDA;
      g_scratch_dev[dev] = p;
    }
    scratch = g_scratch_dev[dev];
  }
  if (tiles == 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st) == cudaSuccess ? RO_OK : RO_ERR_CUDA;
  ro::CompactArgs a{};
  a.flags = flags;
  a.n = n_flags;
  a.block_counts = static_cast<uint32_t*>(scratch);
  a.n_tiles = (uint32_t)tiles;
  a.out = ids;
  a.cap = cap;
  a.total = total;
  a.id_mode = 1;
  return ro::launch_compact(a, st) == cudaSuccess ? RO_OK : RO_ERR_CUDA;
}
