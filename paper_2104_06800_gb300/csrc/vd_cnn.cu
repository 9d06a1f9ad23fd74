// Learned initialiser of the EM state (no counterpart in the paper): six 3x3
// convolutions, 32 channels, bfloat16 weights and activations, float32
// accumulation, from the N flow fields to an initial inverse depth and
// rigidness.
//
// Convolutions are implicit GEMMs on the 5th-generation tensor cores:
// D[pixel][c_out] = sum_k A[pixel][k] B[c_out][k], k = (ky * 3 + kx) * C_in + c_in.
// Activations are stored pixel-major, [H][W][C] bf16 with C = 16 or 32
// channels (32 or 64 bytes per pixel).  A tile is R image rows of 128
// consecutive pixels.  No im2col matrix is built: one TMA box loads the
// tile's halo (R + 2 rows of 130 pixels, every channel, zero outside the
// image) into [row][x][C] with the 32- or 64-byte swizzle, whose rows of
// one pixel each are the K-major swizzled operand layout (8-row groups 8
// pixels apart), so tap (ky, kx) of output row r is the same tile with its
// start address moved by ((r + ky) * 130 + kx) pixels, and the second 16
// input channels by 32 bytes.  Each box row is a whole pixel and each halo
// row one contiguous run of 130 pixels in global memory.  The weights, stored pre-tiled in that layout (LBO = 128 B,
// SBO = 16 K bytes), arrive by one bulk copy.  One thread issues
// R * 9 * C_in / 16 tcgen05.mma (kind::f16, bf16 x bf16 -> f32) into R
// tensor-memory accumulators of N columns and commits them to an mbarrier;
// each warp reads its 32 accumulator lanes with tcgen05.ld.  The backward
// data gradient is the same GEMM on dL/dz with the weights flipped by 180
// degrees and transposed; the weight gradient is a float32 reduction over
// pixels on the CUDA cores, in a fixed order.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "vd_device.cuh"

#define CNN_L 6
#define CNN_WIDTH 32
#define CNN_TILE 128               // output pixels of a row per tile (the MMA's M)
#define CNN_HALO_X (CNN_TILE + 2)
#ifndef CNN_ROWS
#define CNN_ROWS 4                 // output rows per tile
#endif
#ifndef CNN_STAGES
#define CNN_STAGES 3               // halo tiles in flight per CTA
#endif
#define CNN_WAIT_LIMIT (1 << 22)   // mbarrier polls before a wait gives up

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t vd_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t vd_umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Shared-memory matrix descriptor of a K-major operand in a swizzled layout
// (rows of `row_bytes` = 32 or 64 bytes, 16-byte chunks permuted by the
// smem address bits above the row: the layout the tensor copy writes with
// the same swizzle): SBO = 8 rows, LBO unused (one K step fits a row),
// swizzle mode 6 (32 B) or 4 (64 B) in bits 61-63; the base-offset field
// (bits 49-51) carries the start's phase in the pattern when VD_SW_PHASE.
#ifndef VD_SW_PHASE
#define VD_SW_PHASE 0
#endif
__device__ __forceinline__ uint64_t vd_umma_desc_sw(uint32_t saddr, uint32_t row_bytes) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                                   // LBO (unused)
  d |= (uint64_t)(((8u * row_bytes) >> 4) & 0x3FFFu) << 32;  // SBO
  d |= (uint64_t)1 << 46;
  if (VD_SW_PHASE) d |= (uint64_t)((saddr >> 7) & 7u) << 49;
  d |= (uint64_t)(row_bytes == 64 ? 4u : 6u) << 61;
  return d;
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t vd_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void vd_tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(vd_smem_u32(dst)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void vd_tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void vd_umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b,
                                             uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void vd_umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   vd_smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void vd_mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(vd_smem_u32(m)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool vd_mbar_try_wait(uint64_t* m, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(vd_smem_u32(m)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within the poll limit.
__device__ __forceinline__ bool vd_mbar_wait_bounded(uint64_t* m, uint32_t phase) {
  for (int i = 0; i < CNN_WAIT_LIMIT; ++i)
    if (vd_mbar_try_wait(m, phase)) return true;
  return false;
}

__device__ __forceinline__ void vd_mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vd_smem_u32(m)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void vd_mbar_arrive(uint64_t* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(vd_smem_u32(m)) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// into shared memory, completing on the mbarrier's transaction count.
__device__ __forceinline__ void vd_bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                             uint64_t* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(vd_smem_u32(m))
      : "memory");
}

// Tiled TMA load of one box of a rank-4 tensor map at (c0, c1, c2, c3); c0
// (the innermost coordinate) must be a multiple of 16 bytes' worth of
// elements.
// Tiled TMA load of one box of a rank-3 tensor map at (c0, c1, c2); c0 (the
// innermost coordinate) must be a multiple of 16 bytes' worth of elements.
__device__ __forceinline__ void vd_tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0,
                                               int c1, int c2, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(vd_smem_u32(m))
      : "memory");
}

__device__ __forceinline__ void vd_tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0,
                                               int c1, int c2, int c3, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(vd_smem_u32(m))
      : "memory");
}

__device__ __forceinline__ void vd_tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void vd_tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive f32 columns of this warp's 32 accumulator lanes.
__device__ __forceinline__ void vd_tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void vd_tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// The convolution GEMM.  X (through the tensor map `xmap`): bf16 [H][W][C_in]
// with C_in = K / 9 = 16 or 32 channels, dims {C_in, W, H}, box
// {C_in, 130, R + 2}, swizzled.  Wt: the N x K weights
// pre-tiled (vd_tile_index).  Epilogues:
//   EPI_RELU  out = bf16 [HW][N]: relu(D + bias)
//   EPI_LAST  out = f32 [HW][16]: D + bias for the nout real channels, 0 after
//   EPI_DGRAD out = bf16 [HW][N]: D where mask ([HW][N]) > 0, else 0
// ---------------------------------------------------------------------------
enum { EPI_RELU = 0, EPI_LAST = 1, EPI_DGRAD = 2 };

// Element (n, k) of an N x K operand in the K-major no-swizzle layout with
// LBO = 128 B and SBO = 16 K bytes.
__host__ __device__ constexpr size_t vd_tile_index(int n, int k, int K) {
  return (size_t)(n >> 3) * (K * 8) + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
}

__host__ __device__ constexpr uint32_t vd_round128(uint32_t b) { return (b + 127u) & ~127u; }

__host__ __device__ constexpr uint32_t vd_round1024(uint32_t b) { return (b + 1023u) & ~1023u; }

template <int K, int N, int R, int NS>
struct VdConvShape {
  static constexpr int CIN = K / 9;
  static constexpr uint32_t PIX = (uint32_t)CIN * 2;        // bytes of one pixel (one A row)
  static constexpr uint32_t B_BYTES = (uint32_t)N * K * 2;
  static constexpr uint32_t BOX = (uint32_t)(R + 2) * CNN_HALO_X * PIX;   // one halo tile
  // stages start on 1024-byte boundaries (the swizzle pattern's phase is
  // then that of the tile's first pixel)
  static constexpr uint32_t STAGE = vd_round1024(BOX);
  static constexpr uint32_t A_OFF = vd_round1024(B_BYTES);
  static constexpr uint32_t ACC = (uint32_t)R * N;          // columns of one accumulator
  // tensor-memory columns: two accumulators, as a power of two >= 32
  static constexpr uint32_t NCOLS = 2 * ACC <= 32 ? 32 : 2 * ACC <= 64 ? 64 : 2 * ACC <= 128 ? 128
                                  : 2 * ACC <= 256 ? 256 : 512;
  // shared memory: weights, NS halo stages, 1024 B of alignment slack, and
  // at least enough that no more CTAs share an SM than its 512 tensor-memory
  // columns hold (228 KB per SM, 1 KB reserved per CTA)
  static constexpr uint32_t NEED = A_OFF + NS * STAGE + 1024;
  static constexpr uint32_t FLOOR = 233472u / (512u / NCOLS + 1u) - 1024u + 16u;
  static constexpr uint32_t SMEM = NEED > FLOOR ? NEED : FLOOR;
};

// Bounded wait that also gives up once another role of the CTA has set
// `abort` (checked every 256 polls).
__device__ __forceinline__ bool vd_mbar_wait_or_abort(uint64_t* m, uint32_t phase,
                                                      volatile int* abort,
                                                      int limit = CNN_WAIT_LIMIT) {
  for (int i = 0; i < limit; ++i) {
    if (vd_mbar_try_wait(m, phase)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  return false;
}

// Self-test of that failure path: one thread waits on a barrier that
// nothing completes, gives up after `polls` polls and sets the error flag,
// as a role of the convolution does; the host reads the flag.
__global__ void k_wait_probe(int polls, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort;
  if (threadIdx.x != 0) return;
  abort = 0;
  vd_mbar_init(&bar, 1);
  if (!vd_mbar_wait_or_abort(&bar, 0, &abort, polls)) *err = 1;
}

// Persistent, warp-specialised: CTA b takes tiles b, b + gridDim.x, ...
// (tile = x-tile + tiles_x * row block).  Warp 4 loads halo tiles into a ring
// of NS stages (the weights with the first); one thread of warp 5 issues a
// tile's MMAs into one of two tensor-memory accumulators and commits them to
// the stage's `empty` barrier and the accumulator's `full` barrier; the
// other 4 * CNN_EPI_SPLIT warps run the epilogue (warp w reads tensor-memory
// lanes 32 (w % 4) .. 32 (w % 4) + 31, the warps of one lane quarter take
// the tile's rows in turn) and release the accumulator.  So tile i + 1's
// MMAs run under tile i's epilogue and the loads of the tiles after it.
// Every wait is bounded; a role that gives up flags the error and the
// abort, the others stop at their next wait, and before the CTA ends the
// loads and MMAs it issued are waited for.
#ifndef CNN_EPI_SPLIT
#define CNN_EPI_SPLIT 2
#endif
constexpr int CNN_CONV_THREADS = 32 * (4 * CNN_EPI_SPLIT + 2);
template <int K, int N, int EPI, int R, int NS>
__global__ void __launch_bounds__(CNN_CONV_THREADS, 1)
k_conv_tc(const __grid_constant__ CUtensorMap xmap, int Wimg, int Himg, int tiles_x, int n_tiles,
          const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
          void* __restrict__ out, const __nv_bfloat16* __restrict__ mask, int nout,
          int* __restrict__ err) {
  using S = VdConvShape<K, N, R, NS>;
  static_assert(K % 144 == 0 && (N == 16 || N == 32), "shapes of this network");
  static_assert(S::NCOLS <= 512 && R + 2 <= 256 && NS >= 2, "tile");
  constexpr int CIN = S::CIN;
  extern __shared__ uint8_t smem[];
  __shared__ uint64_t full[NS], empty[NS], accfull[2], accempty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort = &s_abort;
  if (warp == 0) vd_tmem_alloc(&tmem_base, S::NCOLS);
  if (tid == 32) {
    for (int s = 0; s < NS; ++s) {
      vd_mbar_init(&full[s], 1);
      vd_mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      vd_mbar_init(&accfull[a], 1);
      vd_mbar_init(&accempty[a], 4 * CNN_EPI_SPLIT);
    }
    vd_mbar_init(&fin, 1);
    s_abort = 0;
  }
  vd_tc_fence_before();
  __syncthreads();
  vd_tc_fence_after();
  const uint32_t dt = tmem_base;
  const uint32_t sB = (vd_smem_u32(smem) + 1023u) & ~1023u, sA = sB + S::A_OFF;
  const int my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (warp == 4) {
    if (lane == 0) {   // producer
      int issued = 0;
      for (int i = 0; i < my_tiles && !*abort; ++i) {
        const int s = i % NS;
        if (i >= NS && !vd_mbar_wait_or_abort(&empty[s], ((i / NS) - 1) & 1, abort)) {
          atomicExch(err, 1);
          *abort = 1;
          break;
        }
        const int tile = blockIdx.x + i * gridDim.x;
        const int x0 = (tile % tiles_x) * CNN_TILE, y0 = (tile / tiles_x) * R;
        vd_mbar_expect_tx(&full[s], S::BOX + (i == 0 ? S::B_BYTES : 0u));
        if (i == 0) vd_bulk_load(sB, Wt, S::B_BYTES, &full[0]);
        // halo rows y0 - 1 .. y0 + R, pixels x0 - 1 .. x0 + 128, every channel
        vd_tma_load_3d(sA + s * S::STAGE, &xmap, 0, x0 - 1, y0 - 1, &full[s]);
        issued = i + 1;
      }
      // the loads in flight land before the CTA ends
      for (int i = issued > NS ? issued - NS : 0; i < issued; ++i)
        vd_mbar_wait_bounded(&full[i % NS], (i / NS) & 1);
    }
  } else if (warp == 5) {
    if (lane == 0) {   // MMA issuer
      bool any = false;
      constexpr uint32_t idesc = vd_idesc_bf16(CNN_TILE, N);
      for (int i = 0; i < my_tiles && !*abort; ++i) {
        const int s = i % NS, a = i & 1;
        if (!vd_mbar_wait_or_abort(&full[s], (i / NS) & 1, abort) ||
            (i >= 2 && !vd_mbar_wait_or_abort(&accempty[a], ((i >> 1) - 1) & 1, abort))) {
          atomicExch(err, 1);
          *abort = 1;
          break;
        }
        vd_tc_fence_after();
        const uint32_t a0 = sA + s * S::STAGE, d0 = dt + a * S::ACC;
        // the descriptors of the stage's first pixel and of the weights; an
        // operand at byte offset o has the descriptor + o / 16 (the start
        // field is the shared address / 16, 14 bits, and every address of
        // the CTA's shared memory fits it without a carry)
        static_assert(VD_SW_PHASE == 0, "offset descriptors need a fixed base-offset field");
        const uint64_t dA0 = vd_umma_desc_sw(a0, S::PIX), dB0 = vd_umma_desc(sB, 128, K * 16);
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
          const uint64_t dAr = dA0 + (uint64_t)((r * CNN_HALO_X * S::PIX) >> 4);
#pragma unroll
          for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int j = 0; j < CIN / 16; ++j) {   // 16 input channels (32 bytes) per MMA
              const uint32_t oa = (((t / 3) * CNN_HALO_X + t % 3) * S::PIX + 32 * j) >> 4;
              const uint32_t ob = (((t * CIN + 16 * j) >> 3) * 128) >> 4;
              vd_umma_bf16(d0 + r * N, dAr + oa, dB0 + ob, idesc, (t | j) ? 1u : 0u);
            }
        }
        vd_umma_commit(&empty[s]);     // the stage is free once these MMAs are done
        vd_umma_commit(&accfull[a]);   // and the accumulator is ready
        any = true;
      }
      if (any) {   // every MMA issued has finished before the memory is freed
        vd_umma_commit(&fin);
        vd_mbar_wait_bounded(&fin, 0);
      }
    }
  } else {   // epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31
    // warps 0..3 take rows 0, CNN_EPI_SPLIT, ...; warps 6..9 (lane quarters
    // 2, 3, 0, 1) rows 1, 1 + CNN_EPI_SPLIT, ...
    static_assert(CNN_EPI_SPLIT == 1 || CNN_EPI_SPLIT == 2, "epilogue warps");
    const int quarter = warp & 3, part = warp < 4 ? 0 : 1;
    const uint32_t tl = dt + ((uint32_t)(quarter * 32) << 16);
    for (int i = 0; i < my_tiles; ++i) {
      const int a = i & 1;
      int ok = 0;
      if (lane == 0) ok = vd_mbar_wait_or_abort(&accfull[a], (i >> 1) & 1, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicExch(err, 1);
          *abort = 1;
        }
        break;
      }
      vd_tc_fence_after();
      const int tile = blockIdx.x + i * gridDim.x;
      const int x = (tile % tiles_x) * CNN_TILE + quarter * 32 + lane, y0 = (tile / tiles_x) * R;
#pragma unroll 1
      for (int r = part; r < R; r += CNN_EPI_SPLIT) {
        const int y = y0 + r;
        if (y >= Himg) break;   // warp-uniform
        float v[N];
        if (N == 32)
          vd_tmem_ld32(tl + a * S::ACC + r * N, v);
        else
          vd_tmem_ld16(tl + a * S::ACC + r * N, v);
        if (x >= Wimg) continue;
        const size_t p = (size_t)y * Wimg + x;
        if (EPI == EPI_LAST) {
          float* dst = reinterpret_cast<float*>(out) + p * 16;
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            *reinterpret_cast<float4*>(dst + c) =
                make_float4(c + 0 < nout ? v[c + 0] + bias[c + 0] : 0.0f,
                            c + 1 < nout ? v[c + 1] + bias[c + 1] : 0.0f,
                            c + 2 < nout ? v[c + 2] + bias[c + 2] : 0.0f,
                            c + 3 < nout ? v[c + 3] + bias[c + 3] : 0.0f);
        } else {
          __align__(16) __nv_bfloat16 o[N];
          if (EPI == EPI_RELU) {
#pragma unroll
            for (int c = 0; c < N; ++c) o[c] = __float2bfloat16_rn(fmaxf(v[c] + bias[c], 0.0f));
          } else {
            __align__(16) __nv_bfloat16 mk[N];
#pragma unroll
            for (int c = 0; c < N; c += 8)
              *reinterpret_cast<uint4*>(mk + c) =
                  *reinterpret_cast<const uint4*>(mask + p * N + c);
#pragma unroll
            for (int c = 0; c < N; ++c)
              o[c] = __float2bfloat16_rn(__bfloat162float(mk[c]) > 0.0f ? v[c] : 0.0f);
          }
          __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(out);
#pragma unroll
          for (int c = 0; c < N; c += 8)   // channels c .. c + 7 of pixel p
            *reinterpret_cast<uint4*>(dst + p * N + c) = *reinterpret_cast<const uint4*>(o + c);
        }
      }
      vd_tc_fence_before();
      __syncwarp();
      if (lane == 0) vd_mbar_arrive(&accempty[a]);
    }
  }
  vd_tc_fence_before();
  __syncthreads();
  if (warp == 0) vd_tmem_dealloc(dt, S::NCOLS);
}

// ---------------------------------------------------------------------------
// Input planes: flow [N][H][W][2] -> bf16 [H][W][C0].
// ---------------------------------------------------------------------------
// Geometry planes 2N .. 2N+3 (zero without a pose): the flow that the
// rotation of T_1 alone gives pixel (u, v), and the extra flow of a point at
// inverse depth GEO_RHO (units of |tau_1|) under the whole T_1, both / 32 px.
#define GEO_RHO 0.1f

__global__ void k_cnn_input(const float2* __restrict__ flow, int N, int Wimg, int HW, int C0,
                            const double* __restrict__ G1, float fx, float fy, float cx,
                            float cy, __nv_bfloat16* __restrict__ a0) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  float geo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (G1) {
    const float u = (float)(p % Wimg), v = (float)(p / Wimg);
    const float rx = (u - cx) / fx, ry = (v - cy) / fy;
    float h[3], d[3];
    for (int r = 0; r < 3; ++r) {
      h[r] = (float)G1[4 * r] * rx + (float)G1[4 * r + 1] * ry + (float)G1[4 * r + 2];
      d[r] = h[r] + GEO_RHO * (float)G1[4 * r + 3];
    }
    if (h[2] > 1e-6f && d[2] > 1e-6f) {
      const float x0 = fx * h[0] / h[2] + cx, y0 = fy * h[1] / h[2] + cy;
      const float x1 = fx * d[0] / d[2] + cx, y1 = fy * d[1] / d[2] + cy;
      geo[0] = (x0 - u) * (1.0f / 32.0f);
      geo[1] = (y0 - v) * (1.0f / 32.0f);
      geo[2] = (x1 - x0) * (1.0f / 32.0f);
      geo[3] = (y1 - y0) * (1.0f / 32.0f);
    }
  }
  for (int g = 0; g < C0 / 8; ++g) {   // channels 8 g .. 8 g + 7 of pixel p, 16 bytes
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = 8 * g + k;
      float v = 0.0f;
      if (c < 2 * N) {
        const float2 f = flow[(size_t)(c >> 1) * HW + p];
        v = ((c & 1) ? f.y : f.x) * (1.0f / 32.0f);
      } else if (c < 2 * N + 4) {
        v = geo[c - 2 * N];
      }
      o[k] = __float2bfloat16_rn(v);
    }
    *reinterpret_cast<uint4*>(a0 + (size_t)p * C0 + 8 * g) = *reinterpret_cast<uint4*>(o);
  }
}

// ---------------------------------------------------------------------------
// Heads, loss and dL/dz of the last layer (z: f32 [HW][16], channel 0 the
// inverse depth, 1..N the rigidness of each flow; dz: bf16 [HW][16]).
// Per-block partial sums of the loss.
// ---------------------------------------------------------------------------
__global__ void k_cnn_heads(const float* __restrict__ z, int HW, int N, float rho_min,
                            float rho_max, float* __restrict__ rho, float* __restrict__ q) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const float* v = z + (size_t)p * 16;
  if (rho) rho[p] = fminf(fmaxf(sqrtf(rho_min * rho_max) * __expf(v[0]), rho_min), rho_max);
  if (q)
    for (int t = 0; t < N; ++t) q[(size_t)t * HW + p] = 1.0f / (1.0f + __expf(-v[1 + t]));
}

__global__ void k_cnn_loss(const float* __restrict__ z, int HW, int N,
                           const float* __restrict__ rho_t, const float* __restrict__ q_t,
                           const unsigned char* __restrict__ mask, float rho_min, float rho_max,
                           float w_q, const int* __restrict__ nmask,
                           __nv_bfloat16* __restrict__ dz, double* __restrict__ partial) {
  __shared__ double s_l[256];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (p < HW) {
    const float* v = z + (size_t)p * 16;
    const float m = mask[p] ? 1.0f : 0.0f;
    const float inv_n = 1.0f / (float)max(*nmask, 1);
    const float wq_n = w_q / (float)N;
    // log error of the inverse-depth head
    const float r = v[0] + 0.5f * logf(rho_min * rho_max) - logf(rho_t[p]);
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
    o[0] = __float2bfloat16_rn(m * 2.0f * r * inv_n);
    float bce = 0.0f;
    for (int t = 0; t < N; ++t) {
      const float s = 1.0f / (1.0f + __expf(-v[1 + t]));
      const float qt = q_t[(size_t)t * HW + p];
      bce += -(qt * __logf(fmaxf(s, 1e-12f)) + (1.0f - qt) * __logf(fmaxf(1.0f - s, 1e-12f)));
      o[1 + t] = __float2bfloat16_rn(wq_n * m * (s - qt) * inv_n);
    }
    l = (double)(m * (r * r + wq_n * bce));
    *reinterpret_cast<uint4*>(dz + (size_t)p * 16) = *reinterpret_cast<uint4*>(o);
    *reinterpret_cast<uint4*>(dz + (size_t)p * 16 + 8) = *reinterpret_cast<uint4*>(o + 8);
  }
  s_l[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_l[threadIdx.x] += s_l[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s_l[0];
}

// Pixels inside the mask (integer atomics: the count does not depend on the
// order of the blocks); *n is zero on entry.
__global__ void k_cnn_count(const unsigned char* __restrict__ mask, int HW, int* __restrict__ n) {
  __shared__ int s[256];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  s[threadIdx.x] = p < HW && mask[p] ? 1 : 0;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && s[0]) atomicAdd(n, s[0]);
}

// Mean loss: the per-block partials summed by one block of 1024 threads in
// a fixed order (strided per thread, then a tree), divided by the count.
__global__ void k_cnn_sum(const double* __restrict__ partial, int n, const int* __restrict__ nmask,
                          double* __restrict__ out) {
  __shared__ double s[1024];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] / (double)max(*nmask, 1);
}

// ---------------------------------------------------------------------------
// Weight gradient on the CUDA cores: dW[co][tap * CIN + ci] =
// sum_p dz[p][co] X[p + offset(tap)][ci], db[co] = sum_p dz[p][co].  dz: bf16
// [HW][COUT]; X: bf16 [HW][CIN].
// The image is cut into tiles of WG_ROWS rows x WG_COLS pixels; block b
// takes tiles b, b + gridDim.x, ... in order.  A block stages a tile's
// input halo and dz in shared memory; thread (co8, ci) holds dW for 8
// output channels x 9 taps of input channel ci in registers and walks the
// tile's pixels row by row, sliding its 3 x 3 window of X along the row (3
// new values, one 16-byte dz load and 72 FMAs per pixel).  The block's sums
// go to partial[b][co][k] (and partial_b[b][co]); k_cnn_wgrad_reduce adds
// the blocks in index order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
#ifndef WG_BLOCKS
#define WG_BLOCKS 608
#endif
#define WG_ROWS 4
#define WG_COLS 64

template <int CIN, int COUT>
__global__ void __launch_bounds__(COUT / 8 * CIN)
k_cnn_wgrad(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ dz, int Wimg,
            int Himg, float* __restrict__ partial, float* __restrict__ partial_b) {
  constexpr int K = 9 * CIN, NT = COUT / 8 * CIN;
  constexpr int HR = WG_ROWS + 2, HC = WG_COLS + 2;
  __shared__ __align__(16) __nv_bfloat16 sX[HR * HC * CIN];
  __shared__ __align__(16) __nv_bfloat16 sD[WG_ROWS * WG_COLS * COUT];
  const int tid = threadIdx.x, ci = tid % CIN, co8 = tid / CIN;
  const int tiles_x = (Wimg + WG_COLS - 1) / WG_COLS;
  const int n_tiles = tiles_x * ((Himg + WG_ROWS - 1) / WG_ROWS);
  float acc[8][9];
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[c][t] = 0.0f;
  float accb = 0.0f;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int y0 = tile / tiles_x * WG_ROWS, x0 = tile % tiles_x * WG_COLS;
    __syncthreads();   // the previous tile's values are no longer read
    for (int i = tid; i < HR * HC * (CIN / 8); i += NT) {   // pixels fastest: coalesced
      const int g = i / (HR * HC), px = i - g * (HR * HC);
      const int yy = y0 - 1 + px / HC, xx = x0 - 1 + px % HC;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (yy >= 0 && yy < Himg && xx >= 0 && xx < Wimg)
        v = *reinterpret_cast<const uint4*>(X + ((size_t)yy * Wimg + xx) * CIN + 8 * g);
      *reinterpret_cast<uint4*>(sX + (size_t)px * CIN + 8 * g) = v;
    }
    for (int i = tid; i < WG_ROWS * WG_COLS * (COUT / 8); i += NT) {
      const int g = i / (WG_ROWS * WG_COLS), px = i - g * (WG_ROWS * WG_COLS);
      const int yy = y0 + px / WG_COLS, xx = x0 + px % WG_COLS;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (yy < Himg && xx < Wimg)
        v = *reinterpret_cast<const uint4*>(dz + ((size_t)yy * Wimg + xx) * COUT + 8 * g);
      *reinterpret_cast<uint4*>(sD + (size_t)px * COUT + 8 * g) = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < WG_ROWS; ++r) {
      float w[3][3];   // X at rows r .. r + 2, columns x .. x + 2 of the halo
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        w[dy][0] = __bfloat162float(sX[((r + dy) * HC + 0) * CIN + ci]);
        w[dy][1] = __bfloat162float(sX[((r + dy) * HC + 1) * CIN + ci]);
      }
#pragma unroll 2
      for (int x = 0; x < WG_COLS; ++x) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
          w[dy][2] = __bfloat162float(sX[((r + dy) * HC + x + 2) * CIN + ci]);
        const __nv_bfloat16* d = sD + (size_t)(r * WG_COLS + x) * COUT + co8 * 8;
        const uint4 dv = *reinterpret_cast<const uint4*>(d);
        const __nv_bfloat162* d2 = reinterpret_cast<const __nv_bfloat162*>(&dv);
        float dzv[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 f = __bfloat1622float2(d2[c]);
          dzv[2 * c] = f.x;
          dzv[2 * c + 1] = f.y;
        }
        accb += __bfloat162float(d[ci & 7]);
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
              acc[c][dy * 3 + dx] = fmaf(dzv[c], w[dy][dx], acc[c][dy * 3 + dx]);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          w[dy][0] = w[dy][1];
          w[dy][1] = w[dy][2];
        }
      }
    }
  }
  float* out = partial + (size_t)blockIdx.x * COUT * K;
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) out[(size_t)(co8 * 8 + c) * K + t * CIN + ci] = acc[c][t];
  if (ci < 8) partial_b[blockIdx.x * COUT + co8 * 8 + ci] = accb;
}

// Sum of the blocks' partials.  The partials hold `stride` values per block
// (COUT_P padded rows); the first nout are the real ones.  A CTA of 8 warps
// takes 32 outputs: warp w adds blocks w, w + 8, ... in order, then warp 0
// adds the 8 warps' sums in order.  CTA 0 also sums the bias partials.
__global__ void __launch_bounds__(256)
k_cnn_wgrad_reduce(const float* __restrict__ partial, const float* __restrict__ partial_b,
                   int nblk, int stride, int nout, int stride_b, int cout,
                   float* __restrict__ gW, float* __restrict__ gb) {
  __shared__ float s[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  float v = 0.0f;
  if (o < nout)
#pragma unroll 4
    for (int b = w; b < nblk; b += 8) v += partial[(size_t)b * stride + o];
  s[w][lane] = v;
  __syncthreads();
  if (w == 0 && o < nout) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += s[i][lane];
    gW[o] = t;
  }
  if (blockIdx.x != 0) return;
  __syncthreads();
  v = 0.0f;
  if (lane < cout)
    for (int b = w; b < nblk; b += 8) v += partial_b[b * stride_b + lane];
  s[w][lane] = v;
  __syncthreads();
  if (w == 0 && lane < cout) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += s[i][lane];
    gb[lane] = t;
  }
}

// ---------------------------------------------------------------------------
// Adam on the float32 master parameters, then the bf16 copies the GEMMs
// read, both pre-tiled (vd_tile_index): forward Wt[co][k] (rows padded to
// NPAD) and data-gradient Wd[ci][tap' * COUT_P + co] = W[co][8 - tap'][ci]
// (COUT padded to COUT_P).
// ---------------------------------------------------------------------------
__global__ void k_cnn_adam(float* __restrict__ theta, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ g, int n, float lr,
                           float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

__global__ void k_cnn_pack(const float* __restrict__ W, int cout, int cin, int npad, int coutp,
                           __nv_bfloat16* __restrict__ Wt, __nv_bfloat16* __restrict__ Wd) {
  const int K = 9 * cin;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // forward copy: npad x K
  if (i < npad * K) {
    const int co = i / K, k = i - co * K;
    Wt[vd_tile_index(co, k, K)] = __float2bfloat16_rn(co < cout ? W[(size_t)co * K + k] : 0.0f);
  }
  // data-gradient copy: cin x 9 coutp
  if (Wd && i < cin * 9 * coutp) {
    const int ci = i / (9 * coutp), r = i - ci * (9 * coutp);
    const int tp = r / coutp, co = r - tp * coutp;
    const int tap = 8 - tp;
    Wd[vd_tile_index(ci, r, 9 * coutp)] =
        __float2bfloat16_rn(co < cout ? W[(size_t)co * K + tap * cin + ci] : 0.0f);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct vd_cnn {
  int N;               // flows
  int cin[CNN_L], cout[CNN_L];
  size_t woff[CNN_L], boff[CNN_L];   // offsets of W_l, b_l in the parameter vector
  size_t nparam;
  float* theta;        // master parameters (f32)
  float* mom1;
  float* mom2;
  float* grad;
  __nv_bfloat16* wt[CNN_L];   // forward weights npad x K, pre-tiled
  __nv_bfloat16* wd[CNN_L];   // data-gradient weights cin x 9 coutp, pre-tiled
  int step;
  // per-image buffers (grown on demand)
  int cap_hw;
  __nv_bfloat16* act[CNN_L];  // a_0 .. a_5 (NHWC bf16)
  __nv_bfloat16* g0;          // dL/dz ping-pong (bf16, 32 channels)
  __nv_bfloat16* g1;
  float* zlast;        // [HW][16] f32
  float* wg_partial;
  float* wg_partial_b;
  double* loss_partial;
  double* loss;
  int* nmask;          // pixels inside the training mask
  double* geo;         // [12] T_1 given to the host-API calls
  int* err;
};

static void cnn_free_images(vd_cnn* n) {
  for (int l = 0; l < CNN_L; ++l)
    if (n->act[l]) cudaFree(n->act[l]), n->act[l] = nullptr;
  void* p[] = {n->g0, n->g1, n->zlast, n->loss_partial};
  for (void* q : p)
    if (q) cudaFree(q);
  n->g0 = n->g1 = nullptr;
  n->zlast = nullptr;
  n->loss_partial = nullptr;
  n->cap_hw = 0;
}

static cudaError_t cnn_reserve(vd_cnn* n, int HW) {
  if (HW <= n->cap_hw) return cudaSuccess;
  cnn_free_images(n);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < CNN_L && e == cudaSuccess; ++l)
    e = cudaMalloc(&n->act[l], sizeof(__nv_bfloat16) * (size_t)HW * n->cin[l]);
  if (e == cudaSuccess) e = cudaMalloc(&n->g0, sizeof(__nv_bfloat16) * (size_t)HW * CNN_WIDTH);
  if (e == cudaSuccess) e = cudaMalloc(&n->g1, sizeof(__nv_bfloat16) * (size_t)HW * CNN_WIDTH);
  if (e == cudaSuccess) e = cudaMalloc(&n->zlast, sizeof(float) * 16 * (size_t)HW);
  if (e == cudaSuccess) e = cudaMalloc(&n->loss_partial, sizeof(double) * ((HW + 255) / 256));
  if (e == cudaSuccess) n->cap_hw = HW;
  return e;
}

// cuTensorMapEncodeTiled from the CUDA driver API (libcuda), looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 vd_encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// Tensor map of a bf16 image with cin = 16 or 32 channels per pixel
// ([H][W][cin]): dims {cin, W, H}, box {cin, 130, rows + 2}, zero fill
// outside the image, 32- or 64-byte swizzle (one pixel is one swizzle row,
// the layout vd_umma_desc_sw reads).
static cudaError_t vd_halo_map(CUtensorMap* m, const void* X, int cin, int W, int H, int rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = vd_encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) || (cin != 16 && cin != 32))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[2] = {(cuuint64_t)cin * 2, (cuuint64_t)W * cin * 2};
  const cuuint32_t box[3] = {(cuuint32_t)cin, CNN_HALO_X, (cuuint32_t)rows + 2};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(X), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         cin == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int K, int N, int EPI>
static cudaError_t launch_conv(const __nv_bfloat16* X, int W, int H, const __nv_bfloat16* Wt,
                               const float* b, void* out, const __nv_bfloat16* mask, int* err,
                               cudaStream_t s, int nout = N) {
  constexpr int R = CNN_ROWS, NS = CNN_STAGES;
  using S = VdConvShape<K, N, R, NS>;
  auto kern = k_conv_tc<K, N, EPI, R, NS>;
  // persistent grid: every CTA that fits on the device at once (set up once)
  static int slots = 0;
  if (!slots) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CNN_CONV_THREADS, S::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    slots = sms * per_sm;
  }
  CUtensorMap map;
  cudaError_t e = vd_halo_map(&map, X, K / 9, W, H, R);
  if (e != cudaSuccess) return e;
  if (reinterpret_cast<uintptr_t>(Wt) & 15u) return cudaErrorInvalidValue;
  const int tiles_x = (W + CNN_TILE - 1) / CNN_TILE;
  const int n_tiles = tiles_x * ((H + R - 1) / R);
  kern<<<min(n_tiles, slots), CNN_CONV_THREADS, S::SMEM, s>>>(map, W, H, tiles_x, n_tiles, Wt, b, out, mask,
                                                 nout, err);
  return cudaGetLastError();
}

// Forward pass of the whole network on flow [N][H][W][2] (device); keeps the
// activations for a backward pass.
// Geometry of the input planes: intrinsics and T_1 (device, 12 doubles) or
// none (zero planes).
struct VdCnnGeo {
  const double* G1;
  float fx, fy, cx, cy;
};

static cudaError_t cnn_forward(vd_cnn* n, const float* flow, int W, int H, cudaStream_t s,
                               VdCnnGeo g) {
  const int HW = W * H;
  cudaError_t e = cnn_reserve(n, HW);
  if (e != cudaSuccess) return e;
  k_cnn_input<<<(HW + 255) / 256, 256, 0, s>>>((const float2*)flow, n->N, W, HW, n->cin[0],
                                               g.G1, g.fx, g.fy, g.cx, g.cy, n->act[0]);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int l = 0; l < CNN_L; ++l) {
    const float* b = n->theta + n->boff[l];
    const int K = 9 * n->cin[l];
    if (l == CNN_L - 1) {
      e = launch_conv<288, 16, EPI_LAST>(n->act[l], W, H, n->wt[l], b, n->zlast, nullptr, n->err,
                                         s, n->cout[l]);
    } else if (K == 144) {
      e = launch_conv<144, 32, EPI_RELU>(n->act[l], W, H, n->wt[l], b, n->act[l + 1], nullptr,
                                         n->err, s);
    } else {
      e = launch_conv<288, 32, EPI_RELU>(n->act[l], W, H, n->wt[l], b, n->act[l + 1], nullptr,
                                         n->err, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Gradients of the loss with respect to every parameter, after cnn_forward
// on the same image; dz of the last layer comes from k_cnn_loss (in g0 with
// 16 channels).
template <int CIN, int COUT>
static cudaError_t launch_wgrad(vd_cnn* n, int l, const __nv_bfloat16* dz, int W, int H,
                                cudaStream_t s) {
  k_cnn_wgrad<CIN, COUT><<<WG_BLOCKS, COUT / 8 * CIN, 0, s>>>(n->act[l], dz, W, H,
                                                                   n->wg_partial,
                                                                   n->wg_partial_b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int stride = COUT * 9 * CIN, nout = n->cout[l] * 9 * CIN;
  k_cnn_wgrad_reduce<<<(nout + 31) / 32, 256, 0, s>>>(
      n->wg_partial, n->wg_partial_b, WG_BLOCKS, stride, nout, COUT, n->cout[l],
      n->grad + n->woff[l], n->grad + n->boff[l]);
  return cudaGetLastError();
}

static cudaError_t cnn_backward(vd_cnn* n, int W, int H, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  __nv_bfloat16* dz = n->g0;    // dL/dz of layer l
  __nv_bfloat16* nxt = n->g1;
  for (int l = CNN_L - 1; l >= 0 && e == cudaSuccess; --l) {
    if (l == CNN_L - 1)
      e = launch_wgrad<32, 16>(n, l, dz, W, H, s);   // 1 + N of 16 rows used
    else if (l == 0 && n->cin[0] == 16)
      e = launch_wgrad<16, 32>(n, l, dz, W, H, s);   // 16 input planes (2N + 4 <= 16)
    else
      e = launch_wgrad<32, 32>(n, l, dz, W, H, s);
    if (e != cudaSuccess || l == 0) break;
    // dL/dz_{l-1} = (W_l^T * dL/dz_l) where a_l > 0
    if (l == CNN_L - 1)
      e = launch_conv<144, 32, EPI_DGRAD>(dz, W, H, n->wd[l], nullptr, nxt, n->act[l], n->err, s);
    else
      e = launch_conv<288, 32, EPI_DGRAD>(dz, W, H, n->wd[l], nullptr, nxt, n->act[l], n->err, s);
    __nv_bfloat16* t = dz;
    dz = nxt;
    nxt = t;
  }
  return e;
}

static cudaError_t cnn_pack_all(vd_cnn* n, cudaStream_t s) {
  for (int l = 0; l < CNN_L; ++l) {
    const int cin = n->cin[l], cout = n->cout[l];
    const int npad = cout < 16 ? 16 : cout;
    const int coutp = cout < 16 ? 16 : cout;
    const int cnt = max(npad * 9 * cin, cin * 9 * coutp);
    k_cnn_pack<<<(cnt + 255) / 256, 256, 0, s>>>(n->theta + n->woff[l], cout, cin, npad, coutp,
                                                 n->wt[l], l > 0 ? n->wd[l] : nullptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static vd_status cnn_check_err(vd_cnn* n, cudaStream_t s) {
  int h = 0;
  VD_CU(cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  VD_CU(cudaStreamSynchronize(s));
  if (h) {
    vd_set_error("a tensor-core wait gave up");
    return VD_ERR_TIMEOUT;
  }
  return VD_OK;
}

extern "C" vd_status vd_check_bounded_wait(int polls, void* cuda_stream) {
  if (polls < 1 || polls > (1 << 20)) return VD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  int h = 0;
  cudaError_t e = cudaMallocAsync((void**)&d, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_probe<<<1, 32, 0, s>>>(polls, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (d) cudaFreeAsync(d, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  if (h) {
    vd_set_error("a tensor-core wait gave up");
    return VD_ERR_TIMEOUT;
  }
  return VD_OK;
}

extern "C" vd_status vd_cnn_create(int n_flows, unsigned long long seed, vd_cnn** out) {
  if (!out || n_flows < 1 || n_flows > 8) return VD_ERR_ARG;
  *out = nullptr;
  vd_cnn* n = new vd_cnn();
  memset((void*)n, 0, sizeof *n);
  n->N = n_flows;
  // input planes: 2N flow planes and 4 geometry planes, padded to 16 or 32
  // (the GEMM tiles take 16 or 32 input channels)
  const int c0p = 2 * n_flows + 4 <= 16 ? 16 : 32;
  size_t off = 0;
  for (int l = 0; l < CNN_L; ++l) {
    n->cin[l] = l == 0 ? c0p : CNN_WIDTH;
    n->cout[l] = l == CNN_L - 1 ? 1 + n_flows : CNN_WIDTH;
    n->woff[l] = off;
    off += (size_t)n->cout[l] * 9 * n->cin[l];
    n->boff[l] = off;
    off += n->cout[l];
  }
  n->nparam = off;
  // He-normal weights (std sqrt(2 / fan_in)) from a host generator seeded by
  // `seed` (Box-Muller on a 64-bit LCG); zero biases.  Padding channels of
  // the input layer get zero weights.
  std::vector<float> h(off, 0.0f);
  unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto u01 = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < CNN_L; ++l) {
    const int cin_real = l == 0 ? 2 * n_flows + 4 : n->cin[l];
    const double sd = sqrt(2.0 / (9.0 * cin_real));
    for (int co = 0; co < n->cout[l]; ++co)
      for (int t = 0; t < 9; ++t)
        for (int ci = 0; ci < n->cin[l]; ++ci) {
          const double g = sqrt(-2.0 * log(u01())) * cos(6.283185307179586 * u01());
          h[n->woff[l] + ((size_t)co * 9 + t) * n->cin[l] + ci] =
              ci < cin_real ? (float)(g * sd) : 0.0f;
        }
  }
  cudaError_t e = cudaMalloc(&n->theta, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMalloc(&n->mom1, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMalloc(&n->mom2, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMalloc(&n->grad, sizeof(float) * off);
  for (int l = 0; l < CNN_L && e == cudaSuccess; ++l) {
    const int npad = n->cout[l] < 16 ? 16 : n->cout[l];
    e = cudaMalloc(&n->wt[l], sizeof(__nv_bfloat16) * npad * 9 * n->cin[l]);
    if (e == cudaSuccess && l > 0)
      e = cudaMalloc(&n->wd[l], sizeof(__nv_bfloat16) * n->cin[l] * 9 * npad);
  }
  if (e == cudaSuccess)
    e = cudaMalloc(&n->wg_partial, sizeof(float) * WG_BLOCKS * CNN_WIDTH * 9 * CNN_WIDTH);
  if (e == cudaSuccess) e = cudaMalloc(&n->wg_partial_b, sizeof(float) * WG_BLOCKS * CNN_WIDTH);
  if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&n->nmask, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&n->geo, sizeof(double) * 12);
  if (e == cudaSuccess) e = cudaMemcpy(n->theta, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->mom1, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(n->mom2, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cnn_pack_all(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    vd_cnn_destroy(n);
    return e == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA;
  }
  *out = n;
  return VD_OK;
}

extern "C" vd_status vd_cnn_destroy(vd_cnn* n) {
  if (!n) return VD_ERR_ARG;
  cudaDeviceSynchronize();
  cnn_free_images(n);
  void* p[] = {n->theta, n->mom1, n->mom2, n->grad, n->wg_partial, n->wg_partial_b,
               n->loss, n->nmask, n->err, n->geo};
  for (void* q : p)
    if (q) cudaFree(q);
  for (int l = 0; l < CNN_L; ++l) {
    if (n->wt[l]) cudaFree(n->wt[l]);
    if (n->wd[l]) cudaFree(n->wd[l]);
  }
  delete n;
  return VD_OK;
}

extern "C" vd_status vd_cnn_layout(vd_cnn* n, int* n_params, int* cin, int* cout, long* woff,
                                   long* boff) {
  if (!n || !n_params) return VD_ERR_ARG;
  *n_params = (int)n->nparam;
  for (int l = 0; l < CNN_L; ++l) {
    if (cin) cin[l] = n->cin[l];
    if (cout) cout[l] = n->cout[l];
    if (woff) woff[l] = (long)n->woff[l];
    if (boff) boff[l] = (long)n->boff[l];
  }
  return VD_OK;
}

extern "C" vd_status vd_cnn_get_params(vd_cnn* n, float* out) {
  if (!n || !out) return VD_ERR_ARG;
  VD_CU(cudaMemcpy(out, n->theta, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
  return VD_OK;
}

extern "C" vd_status vd_cnn_set_params(vd_cnn* n, const float* in) {
  if (!n || !in) return VD_ERR_ARG;
  for (size_t i = 0; i < n->nparam; ++i)
    if (!isfinite(in[i])) return VD_ERR_ARG;
  VD_CU(cudaMemcpy(n->theta, in, sizeof(float) * n->nparam, cudaMemcpyHostToDevice));
  VD_CU(cudaMemset(n->mom1, 0, sizeof(float) * n->nparam));
  VD_CU(cudaMemset(n->mom2, 0, sizeof(float) * n->nparam));
  n->step = 0;
  VD_CU(cnn_pack_all(n, 0));
  VD_CU(cudaDeviceSynchronize());
  return VD_OK;
}

extern "C" vd_status vd_cnn_get_grads(vd_cnn* n, float* out) {
  if (!n || !out) return VD_ERR_ARG;
  VD_CU(cudaMemcpy(out, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost));
  return VD_OK;
}

extern "C" vd_status vd_cnn_get_activation(vd_cnn* n, int layer, float* out, int width,
                                           int height) {
  if (!n || !out || layer < 0 || layer > CNN_L || width * height > n->cap_hw) return VD_ERR_ARG;
  const size_t HW = (size_t)width * height;
  if (layer == CNN_L) {   // z of the last layer, [HW][16]
    VD_CU(cudaMemcpy(out, n->zlast, sizeof(float) * 16 * HW, cudaMemcpyDeviceToHost));
    return VD_OK;
  }
  const int C = n->cin[layer];
  std::vector<__nv_bfloat16> h(HW * C);   // [HW][C] on the device
  VD_CU(cudaMemcpy(h.data(), n->act[layer], sizeof(__nv_bfloat16) * h.size(),
                   cudaMemcpyDeviceToHost));
  for (size_t p = 0; p < HW; ++p)
    for (int c = 0; c < C; ++c)
      out[p * C + c] = __bfloat162float(h[p * C + c]);
  return VD_OK;
}

// Host-given geometry: T_1 copied to the network's device slot.
static cudaError_t cnn_host_geo(vd_cnn* n, const vd_cnn_geometry* g, cudaStream_t s,
                                VdCnnGeo* out) {
  *out = VdCnnGeo{nullptr, 1.0f, 1.0f, 0.0f, 0.0f};
  if (!g) return cudaSuccess;
  out->G1 = n->geo;
  out->fx = (float)g->fx;
  out->fy = (float)g->fy;
  out->cx = (float)g->cx;
  out->cy = (float)g->cy;
  return cudaMemcpyAsync(n->geo, g->T1, sizeof(double) * 12, cudaMemcpyHostToDevice, s);
}

static bool geo_ok(const vd_cnn_geometry* g) {
  if (!g) return true;
  if (!(g->fx > 0) || !(g->fy > 0) || !isfinite(g->cx) || !isfinite(g->cy)) return false;
  for (int i = 0; i < 12; ++i)
    if (!isfinite(g->T1[i])) return false;
  return true;
}

extern "C" vd_status vd_cnn_forward(vd_cnn* n, const float* flow, int width, int height,
                                    const vd_cnn_geometry* geom, float rho_min, float rho_max,
                                    float* rho_out, float* q_out, void* stream) {
  if (!n || !flow || width < 1 || height < 1 || !(rho_max > rho_min) || !geo_ok(geom))
    return VD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  VD_CU(cudaMemsetAsync(n->err, 0, sizeof(int), s));
  VdCnnGeo g;
  VD_CU(cnn_host_geo(n, geom, s, &g));
  VD_CU(cnn_forward(n, flow, width, height, s, g));
  const int HW = width * height;
  if (rho_out || q_out) {
    k_cnn_heads<<<(HW + 255) / 256, 256, 0, s>>>(n->zlast, HW, n->N, rho_min, rho_max, rho_out,
                                                 q_out);
    VD_CU(cudaGetLastError());
  }
  return cnn_check_err(n, s);
}

extern "C" vd_status vd_cnn_train_step(vd_cnn* n, const float* flow, int width, int height,
                                       const vd_cnn_geometry* geom, const float* rho_t,
                                       const float* q_t, const unsigned char* mask,
                                       float rho_min, float rho_max, float w_q, float lr,
                                       int update, double* loss_out, void* stream) {
  if (!n || !flow || !rho_t || !q_t || !mask || width < 1 || height < 1 ||
      !(rho_max > rho_min) || !(lr >= 0.0f) || !geo_ok(geom))
    return VD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int HW = width * height;
  VD_CU(cudaMemsetAsync(n->err, 0, sizeof(int), s));
  VdCnnGeo g;
  VD_CU(cnn_host_geo(n, geom, s, &g));
  VD_CU(cnn_forward(n, flow, width, height, s, g));
  const int nb = (HW + 255) / 256;
  VD_CU(cudaMemsetAsync(n->nmask, 0, sizeof(int), s));
  k_cnn_count<<<nb, 256, 0, s>>>(mask, HW, n->nmask);
  k_cnn_loss<<<nb, 256, 0, s>>>(n->zlast, HW, n->N, rho_t, q_t, mask, rho_min, rho_max, w_q,
                                n->nmask, n->g0, n->loss_partial);
  k_cnn_sum<<<1, 1024, 0, s>>>(n->loss_partial, nb, n->nmask, n->loss);
  VD_CU(cudaGetLastError());
  VD_CU(cnn_backward(n, width, height, s));
  if (update) {
    n->step += 1;
    const float bc1 = (float)(1.0 - pow(0.9, n->step)), bc2 = (float)(1.0 - pow(0.999, n->step));
    k_cnn_adam<<<(int)((n->nparam + 255) / 256), 256, 0, s>>>(n->theta, n->mom1, n->mom2, n->grad,
                                                              (int)n->nparam, lr, bc1, bc2);
    VD_CU(cudaGetLastError());
    VD_CU(cnn_pack_all(n, s));
  }
  if (loss_out) VD_CU(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  return cnn_check_err(n, s);
}

// ---------------------------------------------------------------------------
// Initial EM state of a context from the network: rho (in the context's
// range) into rho_dst and the rigidness of every flow into q_dst.
int vd_cnn_flows(const vd_cnn* n) { return n->N; }

cudaError_t launch_cnn_init(vd_cnn* n, vd_ctx* c, float* rho_dst, float* q_dst) {
  cudaError_t e = cudaMemsetAsync(n->err, 0, sizeof(int), c->stream);
  // geometry from the context's current T_1 (the 8-point bootstrap's, or
  // the poses it was given)
  const VdCnnGeo g{c->G + 12, (float)c->desc.fx, (float)c->desc.fy, (float)c->desc.cx,
                   (float)c->desc.cy};
  if (e == cudaSuccess) e = cnn_forward(n, (const float*)c->flow, c->W, c->H, c->stream, g);
  if (e != cudaSuccess) return e;
  const int HW = c->W * c->H;
  k_cnn_heads<<<(HW + 255) / 256, 256, 0, c->stream>>>(n->zlast, HW, n->N, c->prm.rho_min,
                                                       c->prm.rho_max, rho_dst, q_dst);
  return cudaGetLastError();
}

int* vd_cnn_err_flag(vd_cnn* n) { return n->err; }

VD_CHECK_ACCESSOR(cnn)
