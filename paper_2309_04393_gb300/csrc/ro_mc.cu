// Learned miss compensator (include/ro_mc.h): upsample of a level-1 apron
// slot to the level-0 apron grid, a residual 3D CNN (four 3x3x3 'same'
// convolutions, 1 -> 32 -> 32 -> 32 -> 1), its gradients and Adam.
//
// Activations are channels-last binary32 grids of 34^3 voxels.  The weights
// take part as bfloat16 values (the parameters are rounded once per update
// into an effective binary32 copy); every sum is binary32.  Every product
// runs on the tensor cores with its operands rounded to bfloat16: the
// convolutions (each layer's forward pass, the last three layers' input
// gradients) on tcgen05, marching an 8 x 16 column along z with the three z
// taps of an input slice in one instruction; the weight gradients on
// mma.sync over 8 x 8 x 4 voxel tiles with their one-voxel halo (zero
// outside the grid).  The single-channel side of the first and last layers
// is padded with zeros.  An input-gradient pass is the forward kernel on the
// spatially flipped, channel-transposed weights.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "ro_internal.h"
#include "ro_mc.h"

namespace {

constexpr int EG = RO_MC_EDGE;        // grid edge
constexpr int NV = RO_MC_VOXELS;      // voxels per grid
constexpr int HID = 32;               // hidden channels
constexpr int TX = 8, TY = 8, TZ = 4; // voxel tile of one weight-gradient block
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int kTilesX = (EG + TX - 1) / TX, kTilesY = (EG + TY - 1) / TY, kTilesZ = (EG + TZ - 1) / TZ;

// layer shapes and offsets of W and b in the parameter vector
constexpr int kCin[4] = {1, HID, HID, HID};
constexpr int kCout[4] = {HID, HID, HID, 1};
constexpr int kWOff[4] = {0, 896, 28576, 56256};        // W of layer i
constexpr int kBOff[4] = {864, 28544, 56224, 57120};    // b of layer i (after W)
static_assert(kBOff[3] + 1 == RO_MC_PARAMS, "parameter layout");

// convolution epilogues: ReLU(sum + bias); the residual y = x0 + sum + bias
// (one output channel); the gradient passed where the layer's activation is
// positive
enum : int { kEpiRelu = 1, kEpiResidual = 2, kEpiMask = 3 };

// ------------------------------------------------------------- upsample
// Level-0 voxel X (relative to the child's apron origin) sits at level-1
// coordinate u = (X - 1 + 32 o + 0.5) / 2 - 0.5 relative to the parent's
// first interior voxel; slot index = floor(u) + 1; weights 0.25 / 0.75.
__global__ void upsample_kernel(const uint8_t* __restrict__ base, size_t pitch, const uint32_t* __restrict__ slot_of,
                                const uint32_t* __restrict__ octants, float* __restrict__ x0) {
  const int n = blockIdx.x;
  const uint16_t* s = reinterpret_cast<const uint16_t*>(base + (slot_of ? (size_t)slot_of[n] : (size_t)n) * pitch);
  const uint32_t o = octants[n];
  const int oc[3] = {(int)(o & 1u), (int)((o >> 1) & 1u), (int)((o >> 2) & 1u)};
  for (int v = blockIdx.y * blockDim.x + threadIdx.x; v < NV; v += gridDim.y * blockDim.x) {
    const int X[3] = {v % EG, (v / EG) % EG, v / (EG * EG)};
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int q = X[a] - 1 + 32 * oc[a];            // level-0 voxel relative to the parent's x2 origin
      // u = (q + 0.5) / 2 - 0.5 = q / 2 - 0.25: even q -> (q/2 - 1) + 0.75, odd q -> (q - 1)/2 + 0.25
      const int fl = (q >= 0 ? q : q - 1) / 2;        // floor(q / 2)
      if (q & 1) { i0[a] = fl; f[a] = 0.25f; }
      else { i0[a] = fl - 1; f[a] = 0.75f; }
    }
    float acc = 0.0f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float w = (dz ? f[2] : 1.0f - f[2]) * (dy ? f[1] : 1.0f - f[1]) * (dx ? f[0] : 1.0f - f[0]);
          const int idx = ((i0[2] + 1 + dz) * EG + (i0[1] + 1 + dy)) * EG + (i0[0] + 1 + dx);
          acc = fmaf(w, (float)s[idx], acc);
        }
    x0[(size_t)n * NV + v] = acc * 1.52587890625e-05f;  // 2^-16
  }
}

// blocks per grid of the voxel-wise kernels (upsample, to_raw): a batch of
// 32 grids gives 256 blocks
constexpr int kGridBlocks = 8;

// y (scaled) -> raw u16 values, nearest, clamped to [0, 65535], at out_pitch
__global__ void to_raw_kernel(const float* __restrict__ y, uint8_t* __restrict__ out, size_t out_pitch) {
  const int n = blockIdx.x;
  uint16_t* o = reinterpret_cast<uint16_t*>(out + (size_t)n * out_pitch);
  for (int v = blockIdx.y * blockDim.x + threadIdx.x; v < NV; v += gridDim.y * blockDim.x) {
    const float r = rintf(y[(size_t)n * NV + v] * 65536.0f);
    o[v] = (uint16_t)fminf(fmaxf(r, 0.0f), 65535.0f);
  }
}

// ----------------------------------------- warp-level tensor-core helpers
// Shared-memory rows of 32 bfloat16 channels padded to 80 bytes (the eight
// rows of an ldmatrix fall in different banks), ldmatrix and the mma.sync
// m16n8k16 bfloat16 product with binary32 accumulators, used by the
// weight-gradient kernel.
constexpr int kRowB = 80;                                  // bytes per shared row (32 bf16 + 8 pad)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------ fifth-generation tensor cores (tcgen05)
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint64_t kWaitNs = 500000000ull;           // half a second

// gives up after kWaitLimit polls or kWaitNs nanoseconds, whichever comes first
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    if (ok) return true;
    if ((it & 1023u) == 1023u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > kWaitNs) break;
    }
  }
  return false;
}


// The 32 -> 32 convolution on tcgen05.mma, with the three z taps folded
// into N.  The output slices of all columns (grid, 128-voxel run of the
// x-y plane, z) form one list, and a persistent block takes an equal
// contiguous share of it (two blocks per SM), so that no wave of blocks
// runs part-empty; within a column it marches along z: the weights stay in
// shared memory for the block's whole share, the input sits in a ring of
// four z slices (rounded to bfloat16), and while the matrix instructions
// of input slices s and s + 1 run, the block reads out output slice s - 2
// and stores input slice s + 3 of the halo.  A share that crosses into the
// next column starts a new march there (two more halo slices).  An input slice s contributes to output slices s + 1, s and s - 1 through the
// taps dz = 0, 1, 2 with the same input rows, so for each of the nine (dy,
// dx) taps one tcgen05.mma of M = 128 voxels, N = 96 (the three dz taps'
// 32 output channels side by side) and K = 16 reads the input tile once
// and adds into three accumulators: 18 instructions per input slice instead
// of 54 with N = 32, and a third of the operand reads from shared memory.
// The accumulators are a ring of eight 32-column blocks of tensor memory:
// output slice zo (relative to the block's first) lives in block
// (-zo - 1) mod 8, so slices zo, zo - 1, zo - 2 are consecutive columns; at
// the ring's end the instruction is split in two.  The first product
// of an output slice (input slice zo, tap (0, 0, 0), first K step)
// overwrites its block, so a block needs no zeroing after its slice has
// been read out.  The x-y plane is
// flattened with its one-voxel halo, 36 voxels a row (voxel (x, y) at
// f = (y + 1) 36 + x + 1), and a block's 128 accumulator rows are a run of
// 128 consecutive f (ten runs cover the 34 x 34 outputs; rows that fall on
// the halo columns or past the last output are computed and not stored).
// The input run the taps reach, 128 + 2 x 37 voxels, is stored once per
// slice as rows of 8 channels (16 bytes) in planes of one channel octet:
// core matrices are 8 consecutive rows (128 bytes apart), and the tap
// (dy, dx) moves the operand's start by (36 dy + dx) rows.
constexpr int kTzThreads = 256;
constexpr int kTzPadW = EG + 2;                              // 36: a halo row of the flattened plane
constexpr int kTzMTiles = (EG * kTzPadW - 2 + 127) / 128;    // 128-row runs covering the outputs: 10
constexpr int kTzRows = 128 + 2 * (kTzPadW + 1);             // input rows a run's taps reach: 202
constexpr int kTzMinShare = 4;                               // output slices a block takes at least
constexpr int kTzBlocksPerSm = 2;                            // resident blocks of the convolution per SM
constexpr int kTzPlane = kTzRows * 16;                       // one channel octet of a slice: 3,232 B (LBO)
constexpr int kTzRing = 4;                                   // input slices in shared memory

// Shapes of a z-folded convolution with CIN (1 or 32) input and COUT (1 or
// 32) output channels.  One input channel is padded to K = 16: its slice is
// one plane with the value in the first of each row's 8 channels, and the
// second 8-channel chunk is a plane of zeros.  One output channel is padded
// to 16 accumulator columns per z tap (N = 48).
template <int CIN, int COUT>
struct TzShape {
  static constexpr int KS = CIN == 1 ? 1 : 2;                // K steps of 16 input channels
  static constexpr int PLANES = CIN == 1 ? 2 : 4;            // 8-channel planes of an input slice
  static constexpr int SLICE = PLANES * kTzPlane;            // 5,760 or 11,520 B
  static constexpr int COUTP = COUT == 1 ? 16 : 32;          // accumulator columns of an output slice
  static constexpr int NB = 3 * COUTP;                       // B rows of a (dy, dx) tap: the three dz taps
  static constexpr int BKS = NB / 8 * 256;                   // B of one (dy, dx) tap and K step
  static constexpr int BTAP = KS * BKS;
  static constexpr int BBYTES = 9 * BTAP;
  static constexpr int COLS = 8 * COUTP;                     // tensor-memory columns: 8 blocks
  // shared memory; at least 76 KB when a block holds 256 columns of tensor
  // memory, so that no third block (which could not allocate) is resident
  static constexpr size_t SMEM_USED = (size_t)BBYTES + (size_t)kTzRing * SLICE;
  static constexpr size_t SMEM = COLS == 256 && SMEM_USED < 76 * 1024 ? 76 * 1024 : SMEM_USED;
};

__device__ __forceinline__ uint64_t umma_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // start >> 4; leading byte offset (next K chunk); stride byte offset (next
  // 8-row group); descriptor version 1; no swizzle
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t tz_idesc(int n) {
  // D binary32, A and B bfloat16, both K-major, N, M = 128
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D = A B (acc == 0) or D += A B
__device__ __forceinline__ void tz_mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc = 1u) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(d_tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// this thread's pieces of input slice gz, flattened rows f0 .. f0 + 201
// (zeros outside the grid): 8 channels (32 bytes) each for 32 channels, one
// value for one channel
// (INBF: the input is stored as bfloat16 values, 16 bytes per 8 channels,
// kept as they are); the slice is shared by NT threads, tid < NT
template <int CIN>
__host__ __device__ constexpr int tz_items() { return kTzRows * (CIN == 1 ? 1 : 4); }   // pieces of an input slice
template <int CIN, int NT>
__host__ __device__ constexpr int tz_per() { return (tz_items<CIN>() + NT - 1) / NT; }
template <int CIN, bool INBF, int NT>
__device__ __forceinline__ void tz_fetch(const void* __restrict__ src_v, int f0, int gz, int tid,
                                         float4 (&v)[tz_per<CIN, NT>()][2]) {
  using S = TzShape<CIN, 32>;
#pragma unroll
  for (int j = 0; j < tz_per<CIN, NT>(); ++j) {
    const int w = tid + j * NT;
    v[j][0] = v[j][1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int q = CIN == 1 ? 0 : w % 4, l = CIN == 1 ? w : w / 4;
    const int f = f0 + l;
    const int gx = f % kTzPadW - 1, gy = f / kTzPadW - 1;
    if (w < tz_items<CIN>() && gx >= 0 && gx < EG && gy >= 0 && gy < EG && gz >= 0 && gz < EG) {
      const size_t vox = (size_t)(gz * EG + gy) * EG + gx;
      if constexpr (CIN == 1) {
        v[j][0].x = __ldg(static_cast<const float*>(src_v) + vox);
      } else if constexpr (INBF) {
        v[j][0] = __ldg(reinterpret_cast<const float4*>(static_cast<const __nv_bfloat16*>(src_v) + vox * HID + 8 * q));
      } else {
        const float4* p4 = reinterpret_cast<const float4*>(static_cast<const float*>(src_v) + vox * HID + 8 * q);
        v[j][0] = __ldg(p4);
        v[j][1] = __ldg(p4 + 1);
      }
    }
  }
}

// ... rounded to bfloat16, into the octet planes of a ring slot (one
// channel: the value and seven zeros in plane 0)
template <int CIN, bool INBF, int NT>
__device__ __forceinline__ void tz_store(uint8_t* slot, int tid, const float4 (&v)[tz_per<CIN, NT>()][2]) {
  using S = TzShape<CIN, 32>;
#pragma unroll
  for (int j = 0; j < tz_per<CIN, NT>(); ++j) {
    const int w = tid + j * NT;
    if (w >= tz_items<CIN>()) continue;
    const int q = CIN == 1 ? 0 : w % 4, l = CIN == 1 ? w : w / 4;
    if constexpr (INBF) {
      *reinterpret_cast<float4*>(slot + q * kTzPlane + l * 16) = v[j][0];
    } else {
      __nv_bfloat162 h[4] = {__floats2bfloat162_rn(v[j][0].x, v[j][0].y), __floats2bfloat162_rn(v[j][0].z, v[j][0].w),
                             __floats2bfloat162_rn(v[j][1].x, v[j][1].y), __floats2bfloat162_rn(v[j][1].z, v[j][1].w)};
      *reinterpret_cast<uint4*>(slot + q * kTzPlane + l * 16) = *reinterpret_cast<const uint4*>(h);
    }
  }
}

// the 32-channel bfloat16 input slice gz, flattened rows f0 .. f0 + 201,
// copied into the octet planes of a ring slot without passing through
// registers (16-byte cp.async; pieces outside the grid are filled with
// zeros: source size 0), committed as one group
__device__ __forceinline__ void tz_copy_async(uint8_t* slot, const void* __restrict__ src_v, int f0, int gz, int tid) {
  const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(src_v);
  for (int w = tid; w < tz_items<HID>(); w += kTzThreads) {
    const int q = w % 4, l = w / 4;
    const int f = f0 + l;
    const int gx = f % kTzPadW - 1, gy = f / kTzPadW - 1;
    const bool in = gx >= 0 && gx < EG && gy >= 0 && gy < EG && gz >= 0 && gz < EG;
    const __nv_bfloat16* g = in ? src + ((size_t)(gz * EG + gy) * EG + gx) * HID + 8 * q : src;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_u32(slot + q * kTzPlane + l * 16)), "l"(g), "r"(in ? 16 : 0) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ int tz_block(int zo) { return ((-zo - 1) % 8 + 8) % 8; }

// in: binary32, or bfloat16 when INBF (the hidden activations and
// gradients); out: bfloat16 (the hidden activations, ReLU epilogue, and
// the hidden gradients, mask epilogue), or binary32 (the output y); aux:
// the activations (bfloat16) whose sign masks the gradient, or x0
// (binary32); db (mask epilogue): the bias gradient, += the sum over
// voxels of the binary32 gradient before it is rounded
template <int EPI, int CIN, int COUT, bool INBF>
__global__ void __launch_bounds__(kTzThreads, kTzBlocksPerSm) conv_tz_kernel(const void* __restrict__ in,
                                                               const __nv_bfloat16* __restrict__ wb,
                                                               const float* __restrict__ bias, void* __restrict__ out,
                                                               const void* __restrict__ aux, uint32_t n_grids,
                                                               float* __restrict__ db, uint32_t* __restrict__ err) {
  using S = TzShape<CIN, COUT>;
  constexpr int CP = S::COUTP;
  extern __shared__ __align__(128) uint8_t smz[];
  uint8_t* s_b = smz;                                        // 9 (dy, dx) taps x S::BTAP
  uint8_t* s_a = smz + S::BBYTES;                            // kTzRing input slices x S::SLICE
  __shared__ __align__(8) uint64_t s_mbar[4];        // input slice j commits to s_mbar[j % 4]
  __shared__ uint32_t s_tmem, s_fail;
  __shared__ float s_bias[HID];
  const int tid = threadIdx.x, warp = tid >> 5;
  // this block's share of the output slices (column-major: z fastest)
  const uint32_t total = n_grids * (uint32_t)(kTzMTiles * EG);
  const uint32_t w_begin = (uint32_t)((uint64_t)blockIdx.x * total / gridDim.x);
  const uint32_t w_end = (uint32_t)((uint64_t)(blockIdx.x + 1) * total / gridDim.x);
  // weights wb[tap][co][ci] (CP rows of 32 channels, 64 bytes, per tap): tap
  // (dz, dy, dx) goes to the B of (dy, dx), rows dz * CP + co, in the
  // canonical K-major layout; with one input channel only its first K step
  for (int q = tid; q < 27 * CP * 4; q += kTzThreads) {
    const int t = q / (CP * 4), co = (q / 4) % CP, ch = q % 4;
    if (ch >= 2 * S::KS) continue;
    const int nrow = (t / 9) * CP + co, c = t % 9;
    *reinterpret_cast<uint4*>(s_b + c * S::BTAP + (ch >> 1) * S::BKS + (nrow >> 3) * 256 + (ch & 1) * 128 +
                              (nrow & 7) * 16) = __ldg(reinterpret_cast<const uint4*>(wb) + q);
  }
  if (tid < COUT) s_bias[tid] = EPI == kEpiMask ? 0.0f : bias[tid];
  if constexpr (CIN == 1) {                                  // the zero chunk of every slot
    for (int q = tid; q < kTzRing * kTzPlane / 16; q += kTzThreads) {
      const int slot = q / (kTzPlane / 16), r = q % (kTzPlane / 16);
      *reinterpret_cast<uint4*>(s_a + slot * S::SLICE + kTzPlane + 16 * r) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_mbar[q])));
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_tmem)), "n"(S::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t a0 = smem_u32(s_a), b0 = smem_u32(s_b);
  constexpr int kAux = EPI == kEpiMask ? COUT / 8 : 1;       // 8 bfloat16 mask values, or x0
  static_assert(EPI != kEpiMask || COUT == HID, "the mask epilogue writes 32-channel gradients");
  float bacc[EPI == kEpiMask ? COUT : 1];                    // this row's gradient sums (bias gradient)
#pragma unroll
  for (int c = 0; c < (EPI == kEpiMask ? COUT : 1); ++c) bacc[c] = 0.0f;
  constexpr int kLd = kTzThreads;                          // threads staging an input slice
  const int issuer = 128;                                    // the thread issuing the matrix instructions
  int jb = 0;        // input slices issued by the earlier marches: the barriers' phases run on
  int issued = 0;    // input slices issued in all
  // the matrix instructions of input slice j of the current march (one
  // thread), committed to s_mbar[(jb + j) % 4]
  auto issue = [&](int j) {
    const int bb = tz_block(j);                              // block of output slice j (tap dz = 0)
    const uint32_t a_s = a0 + (uint32_t)((j % kTzRing) * S::SLICE);
    for (int c = 0; c < 9; ++c) {
      const int dy = c / 3, dx = c % 3;
#pragma unroll
      for (int ks = 0; ks < S::KS; ++ks) {
        const uint64_t da = umma_desc_kmajor(a_s + (uint32_t)(2 * ks * kTzPlane + (dy * kTzPadW + dx) * 16),
                                             kTzPlane, 128);
        const uint32_t bt = b0 + (uint32_t)(c * S::BTAP + ks * S::BKS);
        if (c == 0 && ks == 0) {
          // output slice j's first product overwrites its block (whatever
          // it held: the slice read out eight slices before, or nothing);
          // the dz = 1, 2 columns add to output slices j - 1 and j - 2
          const uint64_t db1 = umma_desc_kmajor(bt + (CP / 8) * 256, 128, 256);
          tz_mma(tmem + (uint32_t)(CP * bb), da, umma_desc_kmajor(bt, 128, 256), tz_idesc(CP), 0u);
          if (bb == 6) {                                     // blocks 7 | 0
            tz_mma(tmem + (uint32_t)(7 * CP), da, db1, tz_idesc(CP));
            tz_mma(tmem, da, umma_desc_kmajor(bt + (2 * CP / 8) * 256, 128, 256), tz_idesc(CP));
          } else {                                           // blocks bb + 1, bb + 2 (mod 8), adjacent
            tz_mma(tmem + (uint32_t)(CP * ((bb + 1) & 7)), da, db1, tz_idesc(2 * CP));
          }
        } else if (bb <= 5) {
          tz_mma(tmem + (uint32_t)(CP * bb), da, umma_desc_kmajor(bt, 128, 256), tz_idesc(3 * CP));
        } else if (bb == 6) {                                // blocks 6, 7 | 0
          tz_mma(tmem + (uint32_t)(6 * CP), da, umma_desc_kmajor(bt, 128, 256), tz_idesc(2 * CP));
          tz_mma(tmem, da, umma_desc_kmajor(bt + (2 * CP / 8) * 256, 128, 256), tz_idesc(CP));
        } else {                                             // block 7 | 0, 1
          tz_mma(tmem + (uint32_t)(7 * CP), da, umma_desc_kmajor(bt, 128, 256), tz_idesc(CP));
          tz_mma(tmem, da, umma_desc_kmajor(bt + (CP / 8) * 256, 128, 256), tz_idesc(2 * CP));
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&s_mbar[(jb + j) & 3])) : "memory");
  };
  for (uint32_t w = w_begin; w < w_end;) {
    // a march: output slices z0 .. z0 + nz - 1 of column col (grid n, run f0)
    const uint32_t col = w / EG;
    const int z0 = (int)(w % EG);
    const int nz = (int)min((uint32_t)(EG - z0), w_end - w);
    w += (uint32_t)nz;
    const int n = (int)(col / kTzMTiles);
    const int f0 = (int)(col % kTzMTiles) * 128;             // first input row; outputs from f0 + 37
    const void* src = static_cast<const uint8_t*>(in) + (size_t)n * NV * CIN * (INBF ? 2 : 4);
    // input slices 0, 1 and 2 (z0 - 1 .. z0 + 1) into ring slots 0-2; slice 3
    // into registers, stored in the first step (every instruction of the
    // previous march has completed: its last slice was awaited)
    // (bfloat16 input: slices 0-2 copied asynchronously, and slice i + 3
    // in step i, each its own group of copies)
    float4 pre[INBF ? 1 : tz_per<CIN, kLd>()][2];
    if constexpr (INBF) {
      for (int li = 0; li < 3; ++li) tz_copy_async(s_a + li * S::SLICE, src, f0, z0 - 1 + li, tid);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else {
      for (int li = 0; li < 3; ++li) {
        tz_fetch<CIN, INBF, kLd>(src, f0, z0 - 1 + li, tid, pre);
        tz_store<CIN, INBF, kLd>(s_a + li * S::SLICE, tid, pre);
      }
      tz_fetch<CIN, INBF, kLd>(src, f0, z0 + 2, tid, pre);
    }
    // this thread's accumulator row (warps 0-3): voxel (ex, ey) of each slice
    // (halo columns and rows past the plane are not stored); am holds its mask
    // row (input-gradient pass) or residual value, fetched a step ahead
    const int fr = f0 + kTzPadW + 1 + tid;
    const int ex = fr % kTzPadW - 1, ey = fr / kTzPadW - 1;
    const bool erow = warp < 4 && ex >= 0 && ex < EG && ey < EG;
    uint4 am[kAux];
#pragma unroll
    for (int c8 = 0; c8 < kAux; ++c8) am[c8] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // input slice i + 1 is issued in step i, while slice i - 1 is awaited:
    // at most three slices in flight, on three different barriers
    if (tid == issuer) issue(0);
    issued = jb + 1;
    for (int i = 0; i <= nz + 2; ++i) {
      if (i + 1 <= nz + 1 && tid == issuer) issue(i + 1);
      if (i + 1 <= nz + 1) issued = jb + i + 2;
      // input slice i + 3 into the slot input slice i - 1 leaves (every
      // instruction that read it has completed), before the readout so that
      // its copies are in flight meanwhile; fetch slice i + 4
      auto stage = [&]() {
        if constexpr (INBF) {
          // slice i + 3 copied into that slot (a group, empty past the
          // march's end)
          if (i + 3 <= nz + 1) tz_copy_async(s_a + ((i + 3) % kTzRing) * S::SLICE, src, f0, z0 - 1 + i + 3, tid);
          else asm volatile("cp.async.commit_group;" ::: "memory");
        } else {
          if (i + 3 <= nz + 1) tz_store<CIN, INBF, kLd>(s_a + ((i + 3) % kTzRing) * S::SLICE, tid, pre);
          if (i + 4 <= nz + 1) tz_fetch<CIN, INBF, kLd>(src, f0, z0 - 1 + i + 4, tid, pre);
        }
      };
      if (i == 0) stage();
      if (i >= 1) {
        // input slice i - 1 done: output slice i - 3 is complete; read it out
        // (warps 0-3: one accumulator row each)
        const int ip = i - 1, zo = i - 3, ipg = jb + ip;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&s_mbar[ipg & 3]), (uint32_t)((ipg >> 2) & 1)));
        if (!ok) {
          atomicExch(err, 1u);
          s_fail = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        stage();
        if (ok && warp < 4) {
          const uint32_t taddr = tmem + lane_base + (uint32_t)(CP * tz_block(zo));
          if (zo >= 0) {
            uint32_t r[CP];
            if constexpr (CP == 32)
              asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                           "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                           : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                             "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                             "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                             "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                             "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                           : "r"(taddr));
            else
              asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                           : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                             "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                             "=r"(r[14]), "=r"(r[15])
                           : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (erow) {
              const size_t v = (size_t)n * NV + (size_t)((z0 + zo) * EG + ey) * EG + ex;
              if constexpr (COUT == 1) {                       // y = x0 + f(x0): column 0, bias, residual
                static_cast<float*>(out)[v] = __uint_as_float(r[0]) + s_bias[0] + __uint_as_float(am[0].x);
              } else if constexpr (EPI == kEpiRelu) {          // the activation, stored as bfloat16
                uint4* o8 = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + v * HID);
#pragma unroll
                for (int c8 = 0; c8 < HID / 8; ++c8) {
                  uint32_t h[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const float lo = fmaxf(__uint_as_float(r[8 * c8 + 2 * e]) + s_bias[8 * c8 + 2 * e], 0.0f);
                    const float hi = fmaxf(__uint_as_float(r[8 * c8 + 2 * e + 1]) + s_bias[8 * c8 + 2 * e + 1], 0.0f);
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
                    h[e] = *reinterpret_cast<const uint32_t*>(&b2);
                  }
                  o8[c8] = make_uint4(h[0], h[1], h[2], h[3]);
                }
              } else {                                         // gradient where the activation is positive:
                // summed in binary32 for the bias gradient, stored as bfloat16
                uint4* o8 = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + v * HID);
#pragma unroll
                for (int c8 = 0; c8 < HID / 8; ++c8) {
                  uint32_t h[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const uint32_t mw = (&am[c8].x)[e];      // mask values of channels 8 c8 + 2 e, + 1
                    const int c = 8 * c8 + 2 * e;
                    const float lo = __uint_as_float(mw << 16) > 0.0f ? __uint_as_float(r[c]) : 0.0f;
                    const float hi = __uint_as_float(mw & 0xFFFF0000u) > 0.0f ? __uint_as_float(r[c + 1]) : 0.0f;
                    bacc[c] += lo;
                    bacc[c + 1] += hi;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
                    h[e] = *reinterpret_cast<const uint32_t*>(&b2);
                  }
                  o8[c8] = make_uint4(h[0], h[1], h[2], h[3]);
                }
              }
            }
          }
        }
      }
      // slice i + 2, needed by the next step's instructions, has arrived
      // once at most one group of copies is pending
      if constexpr (INBF) asm volatile("cp.async.wait_group 1;" ::: "memory");
      if constexpr (EPI != kEpiRelu) {                         // mask rows / residual of output slice i - 2
        const int zm = i - 2;
        if (erow && zm >= 0 && zm < nz) {
          const size_t v = (size_t)n * NV + (size_t)((z0 + zm) * EG + ey) * EG + ex;
          if constexpr (EPI == kEpiMask) {
            const uint4* a8 = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(aux) + v * COUT);
#pragma unroll
            for (int c8 = 0; c8 < kAux; ++c8) am[c8] = __ldg(a8 + c8);
          } else {
            am[0].x = __float_as_uint(__ldg(static_cast<const float*>(aux) + v));
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (s_fail) break;
    }
    if constexpr (INBF) asm volatile("cp.async.wait_group 0;" ::: "memory");
    jb += nz + 2;
    if (s_fail) break;
  }
  if (s_fail && issued > 0) {
    // a wait gave up: a last bounded wait for the newest commit before freeing
    const int ip = issued - 1;
    mbar_wait(smem_u32(&s_mbar[ip & 3]), (uint32_t)((ip >> 2) & 1));
  }
  if constexpr (EPI == kEpiMask) {
    // the bias gradient: the readout rows' sums through shared memory (the
    // ring, no longer read), then one add per channel and block
    __syncthreads();
    float* s_red = reinterpret_cast<float*>(s_a);            // COUT x 128 floats
    if (warp < 4) {
#pragma unroll
      for (int c = 0; c < COUT; ++c) s_red[c * 128 + tid] = bacc[c];
    }
    __syncthreads();
    if (tid < COUT && db != nullptr && !s_fail) {
      float t = 0.0f;
      for (int q = 0; q < 128; ++q) t += s_red[tid * 128 + q];
      atomicAdd(db + tid, t);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(S::COLS));
  }
}

static_assert(2 * TzShape<32, 32>::SMEM + 2 * 1024 <= 228 * 1024, "two blocks of the z-folded convolution per SM");
static_assert(3 * TzShape<1, 32>::SMEM > 227 * 1024 && 3 * TzShape<32, 32>::SMEM > 227 * 1024,
              "at most two blocks of 256 tensor-memory columns per SM");

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// Weight gradients of a 32 -> 32 layer on the tensor cores: for every tap
// dW[t] (32 x 32) = sum over voxels of in[v + off(t)]^T g[v], i.e. a GEMM
// with M = input channels, N = output channels, K = voxels.  Block
// (tile position, s) loops over grids s, s + kWgradSplitTc, ...; the input
// tile (halo) and the gradient tile enter shared memory as bfloat16 rows,
// and ldmatrix.trans turns the voxel rows into the K dimension of both
// operands.  Warp w of 16 accumulates taps w and w + 16 and adds its sums
// once (atomically) at the end.  The block keeps three buffers and copies
// the tiles of its next two grids with cp.async while the products of this
// grid run: a bfloat16 input (INBF: the hidden activations) straight into its
// rows, a binary32 input (the one-channel grid) and the binary32 gradient
// tile into staging areas that are rounded into the rows at the start of
// their step.  The bias gradient db[co] = sum over voxels of g[v][co] is
// summed in binary32 from the staging area.  With one input channel the
// taps take the M dimension instead: dW[t][co] = sum over voxels of
// x[v + off(t)] g[v][co], M = 27 taps (32 rows), N = 32 channels, K =
// voxels; warp w takes voxels 16 w .. 16 w + 15 of the tile, builds its A
// fragments from the bfloat16 halo values, and the warps' sums are added
// through shared memory at the end.  With one output channel the taps
// take the N dimension: dW[t][ci] = sum over halo voxels u of x[u][ci]
// g[u - off(t)] (zero where u - off(t) leaves the tile), M = 32 channels,
// N = 27 taps (32 columns), K = the 600 halo voxels; warp w takes chunks
// w, w + 16, w + 32 of 16 halo voxels and builds its B fragments from the
// bfloat16 gradient values of the tile.
constexpr int kWgradSplitTc = 2;
constexpr int kWgWarps = 16, kWgThreads = 32 * kWgWarps;   // two taps a warp
constexpr int kWgBufs = 3;                                  // tile buffers: two grids in flight
template <int CIN, int COUT, bool INBF>
__global__ void __launch_bounds__(kWgThreads, 1) wgrad_mma_kernel(const void* __restrict__ in,
                                                                const void* __restrict__ g, int n_grids,
                                                                float* __restrict__ dW, float* __restrict__ db) {
  // a single channel takes channel 0 of rows that are zero elsewhere: one
  // 16-channel m tile (input) or one 8-channel n tile (gradient)
  constexpr int MT = CIN == 1 ? 1 : 2, NT = COUT == 1 ? 1 : 4;
  extern __shared__ __align__(16) uint8_t smb[];
  const int tile = blockIdx.x;
  const int x0t = (tile % kTilesX) * TX, y0t = ((tile / kTilesX) % kTilesY) * TY, z0t = (tile / (kTilesX * kTilesY)) * TZ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g4 = lane >> 2, t4 = lane & 3;
  const int mi = lane >> 3, mr = lane & 7;
  constexpr int kTapsPerWarp = (27 + kWgWarps - 1) / kWgWarps;
  float acc[kTapsPerWarp][MT][NT][4];
  constexpr bool TAPS_N = CIN == HID && COUT == 1;           // one output channel: the taps as N
  float accn[TAPS_N ? 2 : 1][4][4];                          // [mt][tap n tile][fragment]
#pragma unroll
  for (int mt = 0; mt < (TAPS_N ? 2 : 1); ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) accn[mt][nt][q] = 0.0f;
#pragma unroll
  for (int j = 0; j < kTapsPerWarp; ++j)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][mt][nt][q] = 0.0f;
  // kWgBufs buffers of rows, each with binary32 staging areas for the
  // one-channel gradient tile and the one-channel input
  static_assert(INBF ? CIN == HID : CIN == 1, "the input is the bfloat16 activations or the one-channel grid");
  constexpr int kXB = HZ * HY * HX * kRowB, kGB = TZ * TY * TX * kRowB;
  // the 32-channel gradient is bfloat16 (copied into its rows as it is,
  // its bias gradient summed where it was made); the one-channel gradient
  // is binary32 (staged, rounded, summed here)
  constexpr bool GBF = COUT == HID;
  constexpr int kSF = GBF ? 0 : TZ * TY * TX, kSH = CIN == 1 ? HZ * HY * HX : 0;   // staging floats a buffer
  float* s_f = reinterpret_cast<float*>(smb + kWgBufs * (kXB + kGB));  // [buffer] TZ * TY * TX voxels (one channel)
  float* s_h = s_f + kWgBufs * kSF;                                    // [buffer] HZ * HY * HX voxels (one channel)
  if constexpr (CIN == 1 || COUT == 1) {                    // bytes no copy writes are zero (finite)
    for (int q = threadIdx.x; q < kWgBufs * (kXB + kGB) / 16; q += kWgThreads)
      reinterpret_cast<uint4*>(smb)[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
  }
  float4 bsum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  auto store1 = [](uint8_t* row, float v) { *reinterpret_cast<__nv_bfloat16*>(row) = __float2bfloat16_rn(v); };
  // the products of one grid's tiles: warp w, taps w and w + 16; with a
  // single channel on either side the two taps share the B fragments of
  // each group of 16 voxels (for the 32 -> 32 layers a warp runs its taps
  // one after the other: measured faster there)
  auto compute = [&](uint32_t xb, uint32_t gb) {
    auto tap_pos = [](int t) { return ((t / 9) * HY + (t / 3) % 3) * HX + t % 3; };
    auto load_b = [&](int kc, uint32_t (&b)[4][2]) {
      // B (voxels x output channels): voxel row r + 8 (i & 1), channels 8 (i >> 1) + 16 nj
      const int pb = 16 * kc + mr + 8 * (mi & 1);
#pragma unroll
      for (int nj = 0; nj < (NT + 1) / 2; ++nj)
        ldsm_x4_t(gb + pb * kRowB + 16 * (mi >> 1) + 32 * nj, b[2 * nj][0], b[2 * nj][1], b[2 * nj + 1][0],
                  b[2 * nj + 1][1]);
    };
    auto tap_kc = [&](int j, int t, int kc, const uint32_t (&b)[4][2]) {
      // A (input channels x voxels): voxel row r + 8 (i >> 1), channels 8 (i & 1) (+16 per m tile)
      const int pa = 16 * kc + mr + 8 * (mi >> 1);
      const int pos = ((pa / (TX * TY)) * HY + (pa / TX) % TY) * HX + pa % TX + tap_pos(t);
      uint32_t a[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        ldsm_x4_t(xb + pos * kRowB + 16 * (mi & 1) + 32 * mt, a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
          mma_bf16(acc[j][mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
    };
    if constexpr (CIN == HID && COUT == HID) {
#pragma unroll
      for (int j = 0; j < kTapsPerWarp; ++j) {
        const int t = warp + kWgWarps * j;
        if (t >= 27) break;
        for (int kc = 0; kc < (TZ * TY * TX) / 16; ++kc) {
          uint32_t b[4][2];
          load_b(kc, b);
          tap_kc(j, t, kc, b);
        }
      }
    } else {
      for (int kc = 0; kc < (TZ * TY * TX) / 16; ++kc) {
        uint32_t b[4][2];
        load_b(kc, b);
#pragma unroll
        for (int j = 0; j < kTapsPerWarp; ++j) {
          const int t = warp + kWgWarps * j;
          if (t < 27) tap_kc(j, t, kc, b);                   // warp-uniform
        }
      }
    }
  };
  // one input channel: the taps as M (see above); acc[mt][0][nt] holds
  // taps 16 mt + g4 (+ 8) and channels 8 nt + 2 t4 (+ 1) of this warp's
  // 16 voxels
  auto compute_taps = [&](const uint16_t* xh, uint32_t gb) {
    static_assert(CIN != 1 || (kWgWarps * 16 == TZ * TY * TX && MT == 1 && kTapsPerWarp == 2), "a 16-voxel chunk per warp");
    const int kc = warp;
    uint32_t b[4][2];
    {
      const int pb = 16 * kc + mr + 8 * (mi & 1);
#pragma unroll
      for (int nj = 0; nj < (NT + 1) / 2; ++nj)
        ldsm_x4_t(gb + pb * kRowB + 16 * (mi >> 1) + 32 * nj, b[2 * nj][0], b[2 * nj][1], b[2 * nj + 1][0],
                  b[2 * nj + 1][1]);
    }
    // halo index of tile voxels 16 kc + 2 t4 + {0, 1, 8, 9} (tap (0, 0, 0) at offset 0)
    int hp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pv = 16 * kc + 2 * t4 + (q & 1) + 8 * (q >> 1);
      hp[q] = ((pv / (TX * TY)) * HY + (pv / TX) % TY) * HX + pv % TX;
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t a[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {                          // rows (taps) 16 mt + g4 and + 8
        const int t = 16 * mt + g4 + 8 * h;
        const int toff = ((t / 9) * HY + (t / 3) % 3) * HX + t % 3;
        uint32_t lo = 0u, hi = 0u;
        if (t < 27) {
          lo = (uint32_t)xh[hp[0] + toff] | ((uint32_t)xh[hp[1] + toff] << 16);
          hi = (uint32_t)xh[hp[2] + toff] | ((uint32_t)xh[hp[3] + toff] << 16);
        }
        a[h] = lo;                                           // k 2 t4, 2 t4 + 1
        a[2 + h] = hi;                                       // k 2 t4 + 8, 2 t4 + 9
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][0][nt], a[0], a[1], a[2], a[3], b[nt][0], b[nt][1]);
    }
  };
  // one output channel: the taps as N (see above); accn[mt][nt] holds
  // channels 16 mt + g4 (+ 8) and taps 8 nt + 2 t4 (+ 1)
  auto compute_taps_n = [&](uint32_t xb, const uint16_t* gv) {
    constexpr int kChunks = (HZ * HY * HX + 15) / 16;        // 38; rows past the halo meet zero B values
    for (int kc = warp; kc < kChunks; kc += kWgWarps) {
      uint32_t a[2][4];
      const int pa = 16 * kc + mr + 8 * (mi >> 1);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        ldsm_x4_t(xb + pa * kRowB + 16 * (mi & 1) + 32 * mt, a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
      // halo coordinates of u = 16 kc + 2 t4 + {0, 1, 8, 9}
      int hx[4], hy[4], hz[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = 16 * kc + 2 * t4 + (q & 1) + 8 * (q >> 1);
        hx[q] = u % HX;
        hy[q] = (u / HX) % HY;
        hz[q] = u / (HX * HY);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int t = 8 * nt + g4;                           // this lane's tap (B column)
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        uint32_t bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int vx = hx[q] - dx, vy = hy[q] - dy, vz = hz[q] - dz;
          const bool in = t < 27 && vx >= 0 && vx < TX && vy >= 0 && vy < TY && vz >= 0 && vz < TZ;
          bv[q] = in ? (uint32_t)gv[(vz * TY + vy) * TX + vx] : 0u;
        }
        const uint32_t b0 = bv[0] | (bv[1] << 16), b1 = bv[2] | (bv[3] << 16);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(accn[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
      }
    }
  };
  // grid n's tiles into buffer buf with cp.async, one group: the bfloat16
  // input straight into its rows, the binary32 input and gradient into
  // their staging areas (zero-filled outside the grid: source size 0)
  auto copy = [&](int n, int buf) {
    uint8_t* sx = smb + buf * (kXB + kGB);
    if constexpr (INBF) {
      const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(in) + (size_t)n * NV * HID;
      for (int q = threadIdx.x; q < HZ * HY * HX * (HID / 8); q += kWgThreads) {
        const int c8 = q % (HID / 8), p = q / (HID / 8);
        const int hx = p % HX, hy = (p / HX) % HY, hz = p / (HX * HY);
        const int gx = x0t + hx - 1, gy = y0t + hy - 1, gz = z0t + hz - 1;
        const bool ok = gx >= 0 && gx < EG && gy >= 0 && gy < EG && gz >= 0 && gz < EG;
        const __nv_bfloat16* sp = ok ? src + ((size_t)(gz * EG + gy) * EG + gx) * HID + 8 * c8 : src;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                     :: "r"(smem_u32(sx + p * kRowB + 16 * c8)), "l"(sp), "r"(ok ? 16 : 0) : "memory");
      }
    } else {
      const float* src = static_cast<const float*>(in) + (size_t)n * NV;
      for (int p = threadIdx.x; p < HZ * HY * HX; p += kWgThreads) {
        const int hx = p % HX, hy = (p / HX) % HY, hz = p / (HX * HY);
        const int gx = x0t + hx - 1, gy = y0t + hy - 1, gz = z0t + hz - 1;
        const bool ok = gx >= 0 && gx < EG && gy >= 0 && gy < EG && gz >= 0 && gz < EG;
        const float* sp = ok ? src + (size_t)(gz * EG + gy) * EG + gx : src;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                     :: "r"(smem_u32(s_h + buf * kSH + p)), "l"(sp), "r"(ok ? 4 : 0) : "memory");
      }
    }
    for (int q = threadIdx.x; q < TZ * TY * TX * (GBF ? HID / 8 : 1); q += kWgThreads) {
      const int c8 = GBF ? q % (HID / 8) : 0, p = GBF ? q / (HID / 8) : q;
      const int gx = x0t + p % TX, gy = y0t + (p / TX) % TY, gz = z0t + p / (TX * TY);
      const bool ok = gx < EG && gy < EG && gz < EG;        // voxels outside the grid add nothing
      const size_t vox = (size_t)(gz * EG + gy) * EG + gx;
      if constexpr (GBF) {
        const __nv_bfloat16* gs = static_cast<const __nv_bfloat16*>(g) + (size_t)n * NV * HID;
        const __nv_bfloat16* sp = ok ? gs + vox * HID + 8 * c8 : gs;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                     :: "r"(smem_u32(sx + kXB + p * kRowB + 16 * c8)), "l"(sp), "r"(ok ? 16 : 0) : "memory");
      } else {
        const float* gs = static_cast<const float*>(g) + (size_t)n * NV;
        const float* sp = ok ? gs + vox : gs;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                     :: "r"(smem_u32(s_f + buf * kSF + p)), "l"(sp), "r"(ok ? 4 : 0) : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // the tiles of the block's next kWgBufs - 1 grids are in flight while
  // this grid's products run (one group of copies per step, empty past
  // the last grid); the staging areas are rounded into bfloat16 (the
  // gradient also summed for the bias gradient) at the start of a step
  for (int k = 0; k < kWgBufs - 1; ++k) {
    const int nk = (int)blockIdx.y + k * kWgradSplitTc;
    if (nk < n_grids) copy(nk, k);
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int buf = 0;
  for (int n = blockIdx.y; n < n_grids; n += kWgradSplitTc) {
    asm volatile("cp.async.wait_group %0;" :: "n"(kWgBufs - 2) : "memory");   // this grid's group is done
    __syncthreads();                                         // its tiles are in; the buffer of the last step is free
    uint8_t* sx = smb + buf * (kXB + kGB);
    uint8_t* sg = sx + kXB;
    if constexpr (!GBF || CIN == 1) {
      if constexpr (!GBF) {                                  // one channel: a compact bfloat16 array
        for (int p = threadIdx.x; p < TZ * TY * TX; p += kWgThreads) {
          const float v = s_f[buf * kSF + p];
          bsum.x += v;
          reinterpret_cast<__nv_bfloat16*>(sg)[p] = __float2bfloat16_rn(v);
        }
      }
      if constexpr (CIN == 1)                                // the halo as an array of bfloat16 values
        for (int p = threadIdx.x; p < HZ * HY * HX; p += kWgThreads)
          reinterpret_cast<__nv_bfloat16*>(sx)[p] = __float2bfloat16_rn(s_h[buf * kSH + p]);
      __syncthreads();                                       // rounded
    }
    {
      const int nn = n + (kWgBufs - 1) * kWgradSplitTc, nb = (buf + kWgBufs - 1) % kWgBufs;
      if (nn < n_grids) copy(nn, nb);
      else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if constexpr (CIN == 1) compute_taps(reinterpret_cast<const uint16_t*>(sx), smem_u32(sg));
    else if constexpr (TAPS_N) compute_taps_n(smem_u32(sx), reinterpret_cast<const uint16_t*>(sg));
    else compute(smem_u32(sx), smem_u32(sg));
    buf = (buf + 1) % kWgBufs;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");     // (only empty groups remain)
  if constexpr (CIN == 1) {
    // the warps' sums (acc[mt][0][nt]: taps 16 mt + g4 (+ 8), channels
    // 8 nt + 2 t4 (+ 1)) added through shared memory, one add per weight
    __syncthreads();
    float* s_red = reinterpret_cast<float*>(smb);            // kWgWarps x 32 taps x 32 channels
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int t = 16 * mt + g4 + 8 * h, co = 8 * nt + 2 * t4;
          s_red[(warp * 32 + t) * 32 + co] = acc[mt][0][nt][2 * h];
          s_red[(warp * 32 + t) * 32 + co + 1] = acc[mt][0][nt][2 * h + 1];
        }
    __syncthreads();
    for (int e = threadIdx.x; e < 27 * COUT; e += kWgThreads) {
      float t = 0.0f;
      for (int w = 0; w < kWgWarps; ++w) t += s_red[w * 32 * 32 + e];
      atomicAdd(&dW[e], t);                                  // dW[t][0][co] at t * COUT + co
    }
  } else if constexpr (TAPS_N) {
    // the warps' sums (accn[mt][nt]: channels 16 mt + g4 (+ 8), taps
    // 8 nt + 2 t4 (+ 1)) added through shared memory, one add per weight
    __syncthreads();
    float* s_red = reinterpret_cast<float*>(smb);            // kWgWarps x 32 taps x 32 channels
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int ci = 16 * mt + g4 + 8 * h, t = 8 * nt + 2 * t4;
          s_red[(warp * 32 + t) * 32 + ci] = accn[mt][nt][2 * h];
          s_red[(warp * 32 + t + 1) * 32 + ci] = accn[mt][nt][2 * h + 1];
        }
    __syncthreads();
    for (int e = threadIdx.x; e < 27 * CIN; e += kWgThreads) {
      float t = 0.0f;
      for (int w = 0; w < kWgWarps; ++w) t += s_red[w * 32 * 32 + e];
      atomicAdd(&dW[e], t);                                  // dW[t][ci][0] at t * CIN + ci
    }
  } else {
#pragma unroll
  for (int j = 0; j < kTapsPerWarp; ++j) {
    const int t = warp + kWgWarps * j;
    if (t >= 27) break;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ci = 16 * mt + g4 + 8 * h;
        if (ci >= CIN) continue;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int co = 8 * nt + 2 * t4;
          if (co < COUT) atomicAdd(&dW[(t * CIN + ci) * COUT + co], acc[j][mt][nt][2 * h]);
          if (co + 1 < COUT) atomicAdd(&dW[(t * CIN + ci) * COUT + co + 1], acc[j][mt][nt][2 * h + 1]);
        }
      }
  }
  }
  // bias gradient of the one output channel: the threads' sums, then one
  // add per block (a 32-channel gradient's bias gradient is summed by the
  // input-gradient pass that makes it)
  if constexpr (!GBF) {
    __syncthreads();
    float* s_red = reinterpret_cast<float*>(smb);
    s_red[threadIdx.x] = bsum.x;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int q = 0; q < kWgThreads; ++q) t += s_red[q];
      atomicAdd(&db[0], t);
    }
  }
}

// kWgBufs buffers of rows and the binary32 staging areas of the one-channel sides
template <int CIN, int COUT>
constexpr size_t wgrad_mma_smem() {
  return ((size_t)(HZ * HY * HX + TZ * TY * TX) * kRowB + (COUT == 1 ? (size_t)TZ * TY * TX * 4 : 0) +
          (CIN == 1 ? (size_t)HZ * HY * HX * 4 : 0)) * kWgBufs;
}
static_assert(wgrad_mma_smem<1, HID>() <= 227 * 1024 && wgrad_mma_smem<HID, 1>() <= 227 * 1024 &&
              wgrad_mma_smem<HID, HID>() <= 227 * 1024, "weight-gradient buffers fit a block's shared memory");

// ------------------------------------------------------ weight gradients

// ----------------------------------------------------------------- loss
// g[v] = 2 (y[v] - t[v]) / N over the N voxels of all grids; loss += sum of
// squares / N (block partial sums added once per block).
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, size_t n, float inv_n,
                            float* __restrict__ g, float* __restrict__ loss) {
  __shared__ float s_part[32];
  float part = 0.0f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = 2.0f * d * inv_n;
    part = fmaf(d, d, part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    float s = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += s_part[q];
    atomicAdd(loss, s * inv_n);
  }
}

// ------------------------------------------------------------ parameters
// The effective weights: each W rounded to bfloat16 (nearest even), biases
// as they are, and the bfloat16 rows of the tensor-core convolutions:
// forward wf[tap][co][ci] and input gradient wd[26 - tap][ci][co] (=
// W[tap][ci][co]), rows of 32 input channels; layer 0 has one real input
// channel per row, layer 3 one real output row of 16 per tap.
__global__ void refresh_kernel(const float* __restrict__ P, float* __restrict__ Pq, __nv_bfloat16* __restrict__ wf0,
                               __nv_bfloat16* __restrict__ wf1, __nv_bfloat16* __restrict__ wf2,
                               __nv_bfloat16* __restrict__ wf3, __nv_bfloat16* __restrict__ wd1,
                               __nv_bfloat16* __restrict__ wd2, __nv_bfloat16* __restrict__ wd3) {
  const int woff[4] = {kWOff[0], kWOff[1], kWOff[2], kWOff[3]}, boff[4] = {kBOff[0], kBOff[1], kBOff[2], kBOff[3]};
  const int cin[4] = {kCin[0], kCin[1], kCin[2], kCin[3]}, cout[4] = {kCout[0], kCout[1], kCout[2], kCout[3]};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RO_MC_PARAMS; i += gridDim.x * blockDim.x) {
    int layer = 3;
    while (layer > 0 && i < woff[layer]) --layer;
    const bool is_w = i < boff[layer];
    const float q = is_w ? __bfloat162float(__float2bfloat16_rn(P[i])) : P[i];
    Pq[i] = q;
    if (is_w) {
      const int ci_n = cin[layer], co_n = cout[layer];
      const int r = i - woff[layer];
      const int t = r / (ci_n * co_n), ci = (r / co_n) % ci_n, co = r % co_n;
      const __nv_bfloat16 h = __float2bfloat16_rn(q);
      if (layer == 0) {                     // 1 -> 32: rows of 32 input channels, the first one real
        wf0[(t * HID + co) * HID] = h;
      } else if (layer == 3) {              // 32 -> 1: row 0 of 16 per tap; input gradient 1 -> 32
        wf3[(t * 16) * HID + ci] = h;
        wd3[((26 - t) * HID + ci) * HID] = h;
      } else {
        (layer == 1 ? wf1 : wf2)[(t * co_n + co) * ci_n + ci] = h;
        (layer == 1 ? wd1 : wd2)[((26 - t) * ci_n + ci) * co_n + co] = h;
      }
    }
  }
}

// Adam on the binary32 parameters (bias corrections folded into lr_t and
// eps_t by the host).
__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                            const float* __restrict__ G, float lr_t, float eps_t) {
  // each constant the binary32 value nearest to its decimal (1 - 0.999f
  // would be 1.3e-5 away from 0.001)
  const float b1 = 0.9f, b2 = 0.999f, c1 = 0.1f, c2 = 0.001f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RO_MC_PARAMS; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = fmaf(b1, M[i], c1 * g);
    const float v = fmaf(b2, V[i], c2 * g * g);
    M[i] = m;
    V[i] = v;
    P[i] -= lr_t * m / (sqrtf(v) + eps_t);
  }
}

}  // namespace

// ================================================================ host side

struct ro_mc {
  ro_mc_desc desc;
  cudaStream_t stream = nullptr;
  float *P, *Pq, *M, *V, *G;          // parameters, effective copy, Adam moments, gradients
  // tensor-core rows of the layers: forward wf0..wf3, input gradient wd1..wd3
  // (layers 0 and 3 padded: one real input channel, one real output row)
  __nv_bfloat16 *wf0, *wf1, *wf2, *wf3, *wd1, *wd2, *wd3;
  __nv_bfloat16 *a1, *a2, *a3;        // hidden activations (after ReLU), n * NV * 32, bfloat16
  __nv_bfloat16 *ga, *gb, *gc;        // hidden gradients, n * NV * 32, bfloat16
  float *g4, *y;                      // output gradient and output, n * NV
  float* loss;                        // scratch loss when the caller passes none
  uint32_t* flag;                     // set by a tensor-core wait that gave up (latched)
  uint32_t step = 0;
  cudaStream_t side = nullptr;        // weight gradients, beside the input gradients
  cudaEvent_t ev[5] = {};             // fork and join points between the two streams
  ~ro_mc() {
    for (cudaEvent_t& x : ev)
      if (x) cudaEventDestroy(x);
    if (side) cudaStreamDestroy(side);
  }
};

namespace {

constexpr uint64_t kMcAlign = 256;
uint64_t mc_align(uint64_t v) { return (v + kMcAlign - 1) / kMcAlign * kMcAlign; }

struct McLayout {
  uint64_t P, Pq, M, V, G, flag, wf0, wf1, wf2, wf3, wd1, wd2, wd3, wend, a1, a2, a3, ga, gb, gc, g4, y, loss,
      total;
};

McLayout mc_layout(uint32_t nb) {
  McLayout L{};
  uint64_t o = 0;
  auto take = [&](uint64_t bytes) { const uint64_t at = o; o = mc_align(o + bytes); return at; };
  const uint64_t pb = (uint64_t)RO_MC_PARAMS * 4, act = (uint64_t)nb * NV * HID * 2, one = (uint64_t)nb * NV * 4;
  L.P = take(pb); L.Pq = take(pb); L.M = take(pb); L.V = take(pb); L.G = take(pb); L.flag = take(4);
  L.wf0 = take(27ull * HID * HID * 2); L.wf1 = take(27ull * HID * HID * 2); L.wf2 = take(27ull * HID * HID * 2);
  L.wf3 = take(27ull * 16 * HID * 2);
  L.wd1 = take(27ull * HID * HID * 2); L.wd2 = take(27ull * HID * HID * 2); L.wd3 = take(27ull * HID * HID * 2);
  L.wend = o;
  L.a1 = take(act); L.a2 = take(act); L.a3 = take(act); L.ga = take(act); L.gb = take(act); L.gc = take(act);
  L.g4 = take(one); L.y = take(one); L.loss = take(4);
  L.total = o;
  return L;
}

template <int EPI, int CIN, int COUT, bool INBF>
cudaError_t conv_tc(const void* in, const __nv_bfloat16* wb, const float* b, void* out, const void* aux, uint32_t n,
                    uint32_t* flag, cudaStream_t s, float* db = nullptr) {
  auto k = conv_tz_kernel<EPI, CIN, COUT, INBF>;
  constexpr size_t sm = TzShape<CIN, COUT>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // persistent: two blocks per SM (the shared memory and tensor memory of
  // a block are sized for two; the carveout gives the SM's shared memory to
  // them), each at least kTzMinShare output slices.  Blocks never wait for
  // one another, so a block that finds no room simply starts later.
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint32_t total = n * (uint32_t)(kTzMTiles * EG);
  const uint32_t blocks = std::min((uint32_t)(kTzBlocksPerSm * sms), (total + kTzMinShare - 1) / kTzMinShare);
  k<<<blocks, kTzThreads, sm, s>>>(in, wb, b, out, aux, n, db, flag);
  return cudaGetLastError();
}

template <int CIN, int COUT, bool INBF>
cudaError_t wgrad_tc(const void* in, const void* g, uint32_t n, float* dW, float* db, cudaStream_t s) {
  constexpr size_t sm = wgrad_mma_smem<CIN, COUT>();
  auto k = wgrad_mma_kernel<CIN, COUT, INBF>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<dim3(kTilesX * kTilesY * kTilesZ, kWgradSplitTc), kWgThreads, sm, s>>>(in, g, (int)n, dW, db);
  return cudaGetLastError();
}


ro_status mc_err(cudaError_t e) { return e == cudaSuccess ? RO_OK : RO_ERR_CUDA; }

// y = x0 + f(x0); keeps the hidden activations for a backward pass
cudaError_t mc_forward(ro_mc* m, uint32_t n, const float* x0, float* y) {
  cudaStream_t s = m->stream;
  const float* Pq = m->Pq;
  cudaError_t e = conv_tc<kEpiRelu, 1, HID, false>(x0, m->wf0, Pq + kBOff[0], m->a1, nullptr, n, m->flag, s);
  if (e == cudaSuccess) e = conv_tc<kEpiRelu, HID, HID, true>(m->a1, m->wf1, Pq + kBOff[1], m->a2, nullptr, n, m->flag, s);
  if (e == cudaSuccess) e = conv_tc<kEpiRelu, HID, HID, true>(m->a2, m->wf2, Pq + kBOff[2], m->a3, nullptr, n, m->flag, s);
  if (e == cudaSuccess) e = conv_tc<kEpiResidual, HID, 1, true>(m->a3, m->wf3, Pq + kBOff[3], y, x0, n, m->flag, s);
  return e;
}

// loss and gradients into G (zeroed first)
cudaError_t mc_backward(ro_mc* m, uint32_t n, const float* x0, const float* target, float* G, float* loss) {
  cudaStream_t s = m->stream;
  cudaError_t e = mc_forward(m, n, x0, m->y);
  if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, (size_t)RO_MC_PARAMS * 4, s);
  if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, 4, s);
  const size_t nv = (size_t)n * NV;
  if (e == cudaSuccess) {
    loss_kernel<<<152 * 4, 256, 0, s>>>(m->y, target, nv, 1.0f / (float)nv, m->g4, loss);
    e = cudaGetLastError();
  }
  const float* zero_bias = nullptr;
  // The weight gradients of a layer and the input gradients through it read
  // the same output gradient and write different buffers: the weight
  // gradients run on the side stream.  Each output gradient has a buffer of
  // its own (ga, gb, gc), so neither stream waits for the other until the
  // main stream joins the side stream at the end.
  cudaStream_t s2 = m->side;
  auto fork = [&](int k) {
    cudaError_t r = cudaEventRecord(m->ev[k], s);
    return r == cudaSuccess ? cudaStreamWaitEvent(s2, m->ev[k], 0) : r;
  };
  // layer 4 (32 -> 1)
  if (e == cudaSuccess) e = fork(0);
  if (e == cudaSuccess) e = wgrad_tc<HID, 1, true>(m->a3, m->g4, n, G + kWOff[3], G + kBOff[3], s2);
  if (e == cudaSuccess)
    e = conv_tc<kEpiMask, 1, HID, false>(m->g4, m->wd3, zero_bias, m->ga, m->a3, n, m->flag, s, G + kBOff[2]);
  // layer 3 (32 -> 32)
  if (e == cudaSuccess) e = fork(1);
  if (e == cudaSuccess) e = wgrad_tc<HID, HID, true>(m->a2, m->ga, n, G + kWOff[2], G + kBOff[2], s2);
  if (e == cudaSuccess)
    e = conv_tc<kEpiMask, HID, HID, true>(m->ga, m->wd2, zero_bias, m->gb, m->a2, n, m->flag, s, G + kBOff[1]);
  // layer 2 (32 -> 32)
  if (e == cudaSuccess) e = fork(3);
  if (e == cudaSuccess) e = wgrad_tc<HID, HID, true>(m->a1, m->gb, n, G + kWOff[1], G + kBOff[1], s2);
  if (e == cudaSuccess)
    e = conv_tc<kEpiMask, HID, HID, true>(m->gb, m->wd1, zero_bias, m->gc, m->a1, n, m->flag, s, G + kBOff[0]);
  // layer 1 (1 -> 32)
  if (e == cudaSuccess) e = wgrad_tc<1, HID, false>(x0, m->gc, n, G + kWOff[0], G + kBOff[0], s);
  if (e == cudaSuccess) e = cudaEventRecord(m->ev[4], s2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev[4], 0);
  return e;
}

cudaError_t mc_refresh(ro_mc* m) {
  refresh_kernel<<<64, 256, 0, m->stream>>>(m->P, m->Pq, m->wf0, m->wf1, m->wf2, m->wf3, m->wd1, m->wd2, m->wd3);
  return cudaGetLastError();
}

}  // namespace

ro_status ro_mc_query_bytes(const ro_mc_desc* d, uint64_t* bytes) {
  if (!d || !bytes || d->max_batch < 1) return RO_ERR_INVALID_ARG;
  *bytes = mc_layout(d->max_batch).total;
  return RO_OK;
}

ro_status ro_mc_create(const ro_mc_desc* d, void* arena, uint64_t arena_bytes, void* stream, ro_mc** out) {
  if (!out) return RO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d || d->max_batch < 1 || !arena || reinterpret_cast<uintptr_t>(arena) % kMcAlign) return RO_ERR_INVALID_ARG;
  const McLayout L = mc_layout(d->max_batch);
  if (arena_bytes < L.total) return RO_ERR_CAPACITY;
  ro_mc* m = new (std::nothrow) ro_mc();
  if (!m) return RO_ERR_CAPACITY;
  m->desc = *d;
  m->stream = static_cast<cudaStream_t>(stream);
  uint8_t* b = static_cast<uint8_t*>(arena);
  auto f = [&](uint64_t off) { return reinterpret_cast<float*>(b + off); };
  m->P = f(L.P); m->Pq = f(L.Pq); m->M = f(L.M); m->V = f(L.V); m->G = f(L.G);
  auto h = [&](uint64_t off) { return reinterpret_cast<__nv_bfloat16*>(b + off); };
  m->wf0 = h(L.wf0); m->wf1 = h(L.wf1); m->wf2 = h(L.wf2); m->wf3 = h(L.wf3);
  m->wd1 = h(L.wd1); m->wd2 = h(L.wd2); m->wd3 = h(L.wd3);
  m->a1 = h(L.a1); m->a2 = h(L.a2); m->a3 = h(L.a3); m->ga = h(L.ga); m->gb = h(L.gb); m->gc = h(L.gc);
  m->g4 = f(L.g4); m->y = f(L.y); m->loss = f(L.loss);
  m->flag = reinterpret_cast<uint32_t*>(b + L.flag);
  cudaError_t e = cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking);
  for (cudaEvent_t& x : m->ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  // parameters, copies, moments, gradients, flag and the tensor-core rows
  // (whose padding stays zero)
  if (e == cudaSuccess) e = cudaMemsetAsync(arena, 0, L.wend, m->stream);
  if (e == cudaSuccess) e = mc_refresh(m);
  if (e != cudaSuccess) {
    delete m;
    return RO_ERR_CUDA;
  }
  *out = m;
  return RO_OK;
}

ro_status ro_mc_destroy(ro_mc* m) {
  if (!m) return RO_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(m->stream);
  const cudaError_t e2 = cudaStreamSynchronize(m->side);
  if (e == cudaSuccess) e = e2;
  delete m;
  return mc_err(e);
}

ro_status ro_mc_set_params(ro_mc* m, const float* host) {
  if (!m || !host) return RO_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(m->P, host, (size_t)RO_MC_PARAMS * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->M, 0, (size_t)RO_MC_PARAMS * 4, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->V, 0, (size_t)RO_MC_PARAMS * 4, m->stream);
  if (e == cudaSuccess) e = mc_refresh(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);   // the host buffer may be reused at once
  m->step = 0;
  return mc_err(e);
}

ro_status ro_mc_get_params(ro_mc* m, float* host) {
  if (!m || !host) return RO_ERR_INVALID_ARG;
  uint32_t flag = 0;
  cudaError_t e = cudaMemcpyAsync(host, m->P, (size_t)RO_MC_PARAMS * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, m->flag, 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess && flag) return RO_ERR_INTERNAL;
  return mc_err(e);
}

ro_status ro_mc_upsample(ro_mc* m, uint32_t n, const uint16_t* slots, const uint32_t* octants, float* x0) {
  if (!m || !slots || !octants || !x0 || n < 1 || n > m->desc.max_batch) return RO_ERR_INVALID_ARG;
  upsample_kernel<<<dim3(n, kGridBlocks), 256, 0, m->stream>>>(reinterpret_cast<const uint8_t*>(slots), (size_t)NV * 2,
                                                                nullptr, octants, x0);
  return mc_err(cudaGetLastError());
}

ro_status ro_mc_forward(ro_mc* m, uint32_t n, const float* x0, float* y) {
  if (!m || !x0 || !y || n < 1 || n > m->desc.max_batch) return RO_ERR_INVALID_ARG;
  return mc_err(mc_forward(m, n, x0, y));
}

ro_status ro_mc_gradients(ro_mc* m, uint32_t n, const float* x0, const float* target, float* grads, float* loss) {
  if (!m || !x0 || !target || !grads || n < 1 || n > m->desc.max_batch) return RO_ERR_INVALID_ARG;
  return mc_err(mc_backward(m, n, x0, target, grads, loss));
}

namespace {

// Adam step m->step + 1 on the gradients G (device), then the refreshed
// bfloat16 copies.  The bias corrections of Kingma and Ba's Algorithm 1 are
// folded into the step size and epsilon: lr_t = lr sqrt(1 - b2^t) / (1 -
// b1^t), eps_t = eps sqrt(1 - b2^t) (their Sec. 2), so that
// lr_t m / (sqrt(v) + eps_t) = lr m_hat / (sqrt(v_hat) + eps).
cudaError_t mc_adam(ro_mc* m, const float* G, float lr) {
  ++m->step;
  const double c1 = 1.0 - std::pow(0.9, (double)m->step), c2 = 1.0 - std::pow(0.999, (double)m->step);
  const float lr_t = (float)(lr * std::sqrt(c2) / c1), eps_t = (float)(1e-8 * std::sqrt(c2));
  adam_kernel<<<64, 256, 0, m->stream>>>(m->P, m->M, m->V, G, lr_t, eps_t);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = mc_refresh(m);
  return e;
}

}  // namespace

ro_status ro_mc_train_step(ro_mc* m, uint32_t n, const float* x0, const float* target, float lr, float* loss) {
  if (!m || !x0 || !target || n < 1 || n > m->desc.max_batch || !(lr > 0.0f)) return RO_ERR_INVALID_ARG;
  cudaError_t e = mc_backward(m, n, x0, target, m->G, loss);
  if (e == cudaSuccess) e = mc_adam(m, m->G, lr);
  return mc_err(e);
}

ro_status ro_mc_apply_gradients(ro_mc* m, const float* grads, float lr) {
  if (!m || !grads || !(lr > 0.0f)) return RO_ERR_INVALID_ARG;
  return mc_err(mc_adam(m, grads, lr));
}

ro_status ro_mc_get_moments(ro_mc* m, float* host_m, float* host_v, uint32_t* step) {
  if (!m || !host_m || !host_v) return RO_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(host_m, m->M, (size_t)RO_MC_PARAMS * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_v, m->V, (size_t)RO_MC_PARAMS * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (step) *step = m->step;
  return mc_err(e);
}

namespace ro {

uint32_t mc_max_batch(const ::ro_mc* m) { return m ? m->desc.max_batch : 0; }

// x0 goes to the compensator's output-gradient buffer (unused outside
// training), y to its output buffer; the work runs on the caller's stream.
cudaError_t mc_synthesize(::ro_mc* m, uint32_t n, const uint8_t* cache, uint32_t pitch, const uint32_t* parent_slots,
                          const uint32_t* octants, uint8_t* out, uint32_t out_pitch, cudaStream_t s) {
  if (!m || n < 1 || n > m->desc.max_batch) return cudaErrorInvalidValue;
  cudaStream_t keep = m->stream;
  m->stream = s;
  upsample_kernel<<<dim3(n, kGridBlocks), 256, 0, s>>>(cache, pitch, parent_slots, octants, m->g4);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = mc_forward(m, n, m->g4, m->y);
  if (e == cudaSuccess) {
    to_raw_kernel<<<dim3(n, kGridBlocks), 256, 0, s>>>(m->y, out, out_pitch);
    e = cudaGetLastError();
  }
  m->stream = keep;
  return e;
}

}  // namespace ro
