// 3x3 convolutions of the warm-start U-Net on the fifth-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory, operands staged
// in shared memory by the tensor memory accelerator.
//
// The convolution is an implicit GEMM.  One CTA computes a tile of M = 128
// output pixels (R image rows of TW pixels, R TW = 128) times NT output
// channels; K runs over the 9 taps and the input channels, 16 channels (one
// K = 16 MMA) per tap and chunk.  Operands use the K-major layout without
// swizzling, whose unit is the core matrix: 8 rows (pixels, or output
// channels) of 16 bytes (8 channels) stored contiguously.
//
//   A (pixels x channels): the input halo tile is loaded by TMA from a 3-D
//   tensor map over the activation view (channels, x, y), one box of 8
//   channels per channel group, so shared memory holds [row][pixel][8 ch],
//   16 bytes per pixel.  A tap's operand is a window of that tile: with one
//   image row per tile (R = 1) the box spans TW + 2 pixels and a tap's
//   shift (dy, dx) moves the descriptor's start by dy rows and dx pixels
//   (16 bytes each); with R > 1 rows a pixel shift would wrap between rows,
//   so three boxes are loaded, each already shifted by its dx, and a tap
//   moves the start by dy rows only.  Out-of-image pixels are zero-filled by
//   the TMA unit, which is the convolution's zero padding.
//   B (output channels x channels): weights pre-packed (k_pack_conv_weights)
//   into the exact shared-memory image of a chunk, copied by one bulk copy.
//
// Consecutive convolutions are programmatic dependent launches (the next
// kernel's set-up overlaps the previous one's tail).  The CTAs are
// persistent and loop over tiles.  One thread issues the TMA
// loads and another the MMAs (a pipeline of 2-3 stages on mbarriers: full =
// data landed, empty = the MMAs reading a stage are done, signalled by
// tcgen05.commit); four epilogue warps read the accumulator from tensor
// memory (warp w owns lanes 32 w .. 32 w + 31, i.e. pixels) and apply bias
// and ReLU, while the next tile accumulates into a second accumulator.
// Every wait is bounded: a wait that gives up sets a flag in mapped host
// memory and the CTA skips the rest of its work.
//
// The weight gradient (k_conv3x3_wgrad_tc, below) is a GEMM over pixels
// whose operands come MN-major straight from TMA boxes of the same
// [pixel][8 channels] form.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "ibm_internal.h"
#include "nn_internal.h"

namespace ibm {
namespace nn {

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 192;  // warps 0-3: epilogue; warp 4: TMA loads; warp 5: MMAs
constexpr int TC_STAGES_MAX = 4;
constexpr int TC_SMEM_MAX = 200 * 1024;  // dynamic shared memory a launch may ask for
constexpr int SM_SMEM = 228 * 1024;      // shared memory of one SM
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about 2 s at the SM clock

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// waits for the phase with the given parity to complete; false if it has
// not completed within TC_WAIT_CYCLES
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor, K-major without swizzling: start address,
// leading byte offset (between the two core matrices of a K = 16 slice),
// stride byte offset (between 8-row groups), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Geometry of one launch (host-computed).
struct TcGeom {
  int TW, R;           // pixels per tile row, rows per tile (TW R = 128)
  int copies, boxw;    // A boxes per channel group (1 or 3), pixels per box row
  int a_region;        // bytes of one A box in shared memory (padded to 128)
  int a_bytes, b_bytes, stage_bytes, tx_bytes, stages;
  int NT, tmem_cols, nchunks;
  int tiles_x, tiles_z, ntiles;  // tiles: TW-pixel columns x R-row bands x NT-channel groups
};

// waits for the phase with the given parity of an mbarrier unless the CTA
// has given up; gives up (sets *abort) after TC_WAIT_CYCLES
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > TC_WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Persistent: CTA b computes tiles b, b + gridDim.x, ...  Warps 0-3 drain
// the accumulators (TMEM lanes 0-127 = the tile's pixels) and write the
// outputs; lane 0 of warp 4 issues the loads (a ring of G.stages stages over
// the sequence of (tile, chunk) pairs), lane 0 of warp 5 the MMAs.  Two accumulators in
// tensor memory alternate between tiles, so the MMAs of a tile run while
// the previous tile's epilogue reads the other one.
template <bool RELU>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv3x3_tc(const __grid_constant__ CUtensorMap tmX, const bf16* __restrict__ wpk, const float* __restrict__ bias,
                 bf16* __restrict__ Y, int ldy, int offy, float* __restrict__ yf, int H, int W, int Cout, TcGeom G,
                 unsigned int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_full[TC_STAGES_MAX], bar_empty[TC_STAGES_MAX];
  __shared__ __align__(8) unsigned long long bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nmine = (int)blockIdx.x < G.ntiles ? (G.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t half_cols = (uint32_t)G.tmem_cols / 2;  // column of the second accumulator
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(G.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < G.stages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_tfull[b]), 1);
      mbar_init(smem_u32(&bar_tempty[b]), 4);  // one arrival per epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // Launched as a programmatic dependent of the previous kernel on the
  // stream: the set-up above (tensor memory, barriers) overlaps that
  // kernel's tail, and no thread touches global memory before the previous
  // kernel has completed and its writes are visible (griddepcontrol.wait);
  // then the next launch may be scheduled.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  auto coords = [&](int li, int& x0, int& y0, int& z) {
    int t = (int)blockIdx.x + li * (int)gridDim.x;
    z = t % G.tiles_z;
    t /= G.tiles_z;
    x0 = (t % G.tiles_x) * G.TW;
    y0 = (t / G.tiles_x) * G.R;
  };

  const int nc = G.nchunks, S = G.stages, nq = nmine * nc;
  if (warp == 4) {
    // TMA producer: the ring of stages over the sequence of (tile, chunk)
    // pairs q = li nc + ch; a stage is reloaded once the MMAs that read it
    // have completed (empty barrier, committed by the MMA thread)
    if (lane == 0) {
      const size_t wchunk = (size_t)2 * 9 * G.NT * 8;  // bf16 elements of one chunk's weights
      int issued = 0;
      for (int q = 0; q < nq; ++q) {
        const int li = q / nc, ch = q % nc, s = q % S;
        if (q >= S && !wait_or_abort(smem_u32(&bar_empty[s]), (uint32_t)(q / S - 1) & 1u, abort)) break;
        int x0, y0, z;
        coords(li, x0, y0, z);
        const uint32_t st = sbase + s * G.stage_bytes, bar = smem_u32(&bar_full[s]);
        mbar_expect_tx(bar, G.tx_bytes);
        for (int cp = 0; cp < G.copies; ++cp)
          for (int g = 0; g < 2; ++g)
            tma_load_3d(st + (cp * 2 + g) * G.a_region, &tmX, ch * 16 + g * 8, G.copies == 1 ? x0 - 1 : x0 + cp - 1,
                        y0 - 1, bar);
        bulk_load(st + G.a_bytes, wpk + ((size_t)z * nc + ch) * wchunk, G.b_bytes, bar);
        issued = q + 1;
      }
      if (*abort && issued > 0)  // the last load issued has landed (bounded) before the CTA may exit
        mbar_wait(smem_u32(&bar_full[(issued - 1) % S]), (uint32_t)((issued - 1) / S) & 1u);
    }
    __syncwarp();
  } else if (warp == 5) {
    // MMA issuer: never waits for its own MMAs, only for data (full) and for
    // the epilogue to have drained an accumulator (tempty)
    if (lane == 0) {
      const uint32_t idesc = instr_desc(G.NT);
      int done = 0;
      for (int q = 0; q < nq; ++q) {
        const int li = q / nc, ch = q % nc, s = q % S, buf = li & 1;
        if (ch == 0 && li >= 2 && !wait_or_abort(smem_u32(&bar_tempty[buf]), (uint32_t)((li >> 1) - 1) & 1u, abort))
          break;
        if (!wait_or_abort(smem_u32(&bar_full[s]), (uint32_t)(q / S) & 1u, abort)) break;
        tc_fence_after();
        const uint32_t st = sbase + s * G.stage_bytes, d = tmem + (uint32_t)buf * half_cols;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
          const uint32_t a =
              G.copies == 1 ? st + (dy * G.boxw + dx) * 16 : st + dx * 2 * G.a_region + dy * G.TW * 16;
          // B: [tap][8-row group of output channels][channel group][8 rows][16 bytes]
          const uint32_t b = st + G.a_bytes + tap * G.NT * 32;
          tc_mma(d, smem_desc(a, G.a_region, 128), smem_desc(b, 128, 256), idesc, (ch | tap) != 0);
        }
        tc_commit(smem_u32(&bar_empty[s]));
        if (ch == nc - 1) tc_commit(smem_u32(&bar_tfull[buf]));
        done = q + 1;
      }
      if (*abort) {
        // the MMAs issued have completed (bounded) before the accumulators are freed
        if (done > 0) mbar_wait(smem_u32(&bar_empty[(done - 1) % S]), (uint32_t)((done - 1) / S) & 1u);
        atomicOr_system(err, 1u);
      }
    }
    __syncwarp();
  } else {
    const int m = warp * 32 + lane;
    for (int li = 0; li < nmine; ++li) {
      const int buf = li & 1;
      if (!wait_or_abort(smem_u32(&bar_tfull[buf]), (uint32_t)(li >> 1) & 1u, abort)) {
        if (lane == 0) atomicOr_system(err, 1u);
        break;
      }
      tc_fence_after();
      int x0, y0, z;
      coords(li, x0, y0, z);
      const int y = y0 + m / G.TW, x = x0 + m % G.TW, n0 = z * G.NT;
      const bool valid = x < W && y < H;
      const size_t p = (size_t)y * W + x;
      for (int c0 = 0; c0 < G.NT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)buf * half_cols + (uint32_t)c0, v);
        const int co = n0 + c0;
        if (!valid || co >= Cout) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float t = v[j] + (bias ? bias[co + j] : 0.f);
          v[j] = RELU ? fmaxf(t, 0.f) : t;
        }
        uint4 o[2];
        uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          ow[j] = *reinterpret_cast<uint32_t*>(&h);
        }
        uint4* dst = reinterpret_cast<uint4*>(Y + p * ldy + offy + co);
        dst[0] = o[0];
        dst[1] = o[1];
        if (yf) {
          float4* f = reinterpret_cast<float4*>(yf + p * Cout + co);
#pragma unroll
          for (int j = 0; j < 4; ++j) f[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[buf]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.tmem_cols) : "memory");
  }
}

// ------------------------------------------------------- weight gradient
//
// dW[co][tap][ci] += sum over pixels p of G[p][co] X[p + shift(tap)][ci], a
// GEMM per tap with M = 128 output channels (a tile of them; rows beyond
// Cout zero), N = NT
// input channels, K = pixels.  Both operands come as TMA boxes of [pixel][8
// channels], i.e. MN-major: a core matrix is 8 pixels (K) x 8 channels (MN),
// 16 bytes per pixel; K groups of 8 pixels are 128 bytes apart, MN groups of
// 8 channels one box apart.  A CTA owns one tap row dy (taps 3 dy .. 3 dy + 2,
// one accumulator of NT columns each), one NT-channel tile and a range of
// pixel chunks (P pixels of one image row); the X box of a chunk spans P + 2
// pixels of row y + dy, and tap dx reads it dx pixels further.  After its
// chunks the CTA adds its accumulators to dW (vector atomics).
struct WgGeom {
  int P;                // pixels per chunk (a multiple of 16, <= 128)
  int NT, ntiles_ci;    // input channels per tile, tiles
  int co_tiles;         // tiles of 128 output channels
  int a_region, b_region, a_bytes, b_bytes, stage_bytes, stages;
  int tmem_cols, chunks_x, nchunks, ksplit;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv3x3_wgrad_tc(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmX, int Cin,
                       int Cout, float* __restrict__ dW, WgGeom G, unsigned int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_full[TC_STAGES_MAX], bar_empty[TC_STAGES_MAX], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work unit: blockIdx.x = (ksplit part, tap row, input-channel tile,
  // output-channel tile)
  const int part = blockIdx.x % G.ksplit;
  int rest = blockIdx.x / G.ksplit;
  const int dy = rest % 3;
  rest /= 3;
  const int zt = rest % G.ntiles_ci, co0 = (rest / G.ntiles_ci) * 128;
  const int cog = (Cout - co0) / 8 < 16 ? (Cout - co0) / 8 : 16;  // 8-channel groups of G in this tile
  const int tx_bytes = cog * G.P * 16 + (G.NT / 8) * (G.P + 2) * 16;
  const int c_begin = (int)((long)G.nchunks * part / G.ksplit), c_end = (int)((long)G.nchunks * (part + 1) / G.ksplit);
  const int nq = c_end - c_begin, S = G.stages;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(G.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the MN groups of A beyond Cout are never loaded: zero them in every stage
  const int zero_bytes = (16 - cog) * G.a_region;
  for (int s = 0; s < S; ++s) {
    uint4* z = reinterpret_cast<uint4*>(smem_raw + (sbase - smem_u32(smem_raw)) + s * G.stage_bytes +
                                        cog * G.a_region);
    for (int k = threadIdx.x; k < zero_bytes / 16; k += blockDim.x) z[k] = make_uint4(0, 0, 0, 0);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes seen by the tensor cores
  if (threadIdx.x == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_acc), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (warp == 4) {
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < nq; ++q) {
        const int s = q % S, c = c_begin + q;
        if (q >= S && !wait_or_abort(smem_u32(&bar_empty[s]), (uint32_t)(q / S - 1) & 1u, abort)) break;
        const int x0 = (c % G.chunks_x) * G.P, y = c / G.chunks_x;
        const uint32_t st = sbase + s * G.stage_bytes, bar = smem_u32(&bar_full[s]);
        mbar_expect_tx(bar, tx_bytes);
        for (int g = 0; g < cog; ++g) tma_load_3d(st + g * G.a_region, &tmG, co0 + 8 * g, x0, y, bar);
        for (int g = 0; g < G.NT / 8; ++g)
          tma_load_3d(st + G.a_bytes + g * G.b_region, &tmX, zt * G.NT + 8 * g, x0 - 1, y + dy - 1, bar);
        issued = q + 1;
      }
      if (*abort && issued > 0) mbar_wait(smem_u32(&bar_full[(issued - 1) % S]), (uint32_t)((issued - 1) / S) & 1u);
    }
    __syncwarp();
  } else if (warp == 5) {
    if (lane == 0) {
      // both operands MN-major (transpose bits), N = NT, M = 128
      const uint32_t idesc = instr_desc(G.NT) | (1u << 15) | (1u << 16);
      int done = 0;
      for (int q = 0; q < nq; ++q) {
        const int s = q % S;
        if (!wait_or_abort(smem_u32(&bar_full[s]), (uint32_t)(q / S) & 1u, abort)) break;
        tc_fence_after();
        const uint32_t st = sbase + s * G.stage_bytes;
        for (int ks = 0; ks < G.P / 16; ++ks) {
          const uint64_t a = smem_desc(st + ks * 256, 128, G.a_region);
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const uint64_t b = smem_desc(st + G.a_bytes + (ks * 16 + t) * 16, 128, G.b_region);
            tc_mma(tmem + (uint32_t)(t * G.NT), a, b, idesc, (q | ks) != 0);
          }
        }
        tc_commit(smem_u32(&bar_empty[s]));
        done = q + 1;
      }
      tc_commit(smem_u32(&bar_acc));
      if (*abort) {
        if (done > 0) mbar_wait(smem_u32(&bar_empty[(done - 1) % S]), (uint32_t)((done - 1) / S) & 1u);
        atomicOr_system(err, 1u);
      }
    }
    __syncwarp();
  } else if (nq > 0) {
    // epilogue: lane = output channel co, 16 input channels per load
    if (wait_or_abort(smem_u32(&bar_acc), 0u, abort)) {
      tc_fence_after();
      const int co = co0 + warp * 32 + lane;
      for (int t = 0; t < 3; ++t)
        for (int c0 = 0; c0 < G.NT; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * G.NT + c0), v);
          if (co >= Cout || zt * G.NT + c0 >= Cin) continue;
          float4* dst = reinterpret_cast<float4*>(dW + ((size_t)co * 9 + 3 * dy + t) * Cin + zt * G.NT + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) atomicAdd(dst + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
        }
    } else if (lane == 0) {
      atomicOr_system(err, 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.tmem_cols) : "memory");
  }
}

// Packed weights of a convolution with Cin input and Cout output channels:
// for output-channel tile t (NT channels) and input-channel chunk ch (16
// channels), the chunk's shared-memory image
//   [tap 9][8-row group NT/8][channel group 2][row 8][8 channels]
// of W'[co][tap][ci], zero for co >= Cout.  W' is the layer's weights
// w[Cout][9][Cin]; with flip it is the data-gradient operator of a layer
// whose weights are w[Cin][9][Cout]: W'[co][tap][ci] = w[ci][8 - tap][co].
// One launch packs every job (blockIdx.y = job).
__global__ void k_pack_conv_weights(const PackJob* __restrict__ jobs) {
  const PackJob J = jobs[blockIdx.y];
  const int Cin = J.cin, Cout = J.cout, NT = J.nt, nchunks = Cin / 16;
  const long n = (long)J.ntiles * nchunks * 9 * NT * 16;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const int e = (int)(k & 7), row = (int)((k >> 3) & 7), g = (int)((k >> 6) & 1);
    long r = k >> 7;
    const int ngrp = (int)(r % (NT / 8));
    r /= NT / 8;
    const int tap = (int)(r % 9);
    r /= 9;
    const int ch = (int)(r % nchunks), t = (int)(r / nchunks);
    const int co = t * NT + ngrp * 8 + row, ci = ch * 16 + g * 8 + e;
    bf16 v = __float2bfloat16_rn(0.f);
    if (co < Cout)
      v = J.flip ? J.w[((size_t)ci * 9 + (8 - tap)) * Cout + co] : J.w[((size_t)co * 9 + tap) * Cin + ci];
    J.wpk[k] = v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// a flag the kernels set (system-scope atomic) when a wait gives up; mapped
// host memory, so the host reads it without a device synchronisation
unsigned int* error_flag(unsigned int** dev) {
  static unsigned int* host = nullptr;
  static unsigned int* devp = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    if (cudaHostAlloc(&h, sizeof(unsigned int), cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
      host = static_cast<unsigned int*>(h);
      *host = 0u;
      void* d = nullptr;
      if (cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess) devp = static_cast<unsigned int*>(d);
    }
  });
  *dev = devp;
  return host;
}

// Least dynamic shared memory per CTA such that the CTAs that fit on one SM
// by shared memory (1 KB static and 1 KB reserved each) hold no more than the
// SM's 512 tensor-memory columns: then an allocation never waits for
// another CTA's.
int tmem_min_smem(int cols) {
  const int k = 512 / cols;  // CTAs whose columns fit
  return SM_SMEM / (k + 1) - 2048 + 1;
}

// kernel attributes (shared memory size and carveout) are set once per device
bool first_use_on_device(int which) {
  static std::mutex mu;
  static unsigned long long done[2] = {0ull, 0ull};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return true;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long bit = 1ull << dev;
  if (done[which] & bit) return false;
  done[which] |= bit;
  return true;
}

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

int conv_tile_channels(int Cout) { return Cout <= 128 ? Cout : 128; }

size_t packed_conv_weights(int Cin, int Cout) {
  const int NT = conv_tile_channels(Cout), ntiles = (Cout + NT - 1) / NT;
  return (size_t)ntiles * NT * 9 * Cin;
}

PackJob pack_job(int Cin, int Cout, const bf16* w, bf16* wpk, bool flip) {
  PackJob j{};
  j.cin = Cin;
  j.cout = Cout;
  j.nt = conv_tile_channels(Cout);
  j.ntiles = (Cout + j.nt - 1) / j.nt;
  j.flip = flip ? 1 : 0;
  j.w = w;
  j.wpk = wpk;
  return j;
}

void pack_conv_weights(cudaStream_t s, const PackJob* jobs_dev, int njobs, long max_elems) {
  long b = (max_elems + 255) / 256;
  k_pack_conv_weights<<<dim3((unsigned)(b > 1024 ? 1024 : b), (unsigned)njobs), 256, 0, s>>>(jobs_dev);
}

int conv3x3_wgrad(cudaStream_t s, int H, int W, int Cin, int Cout, const bf16* Gd, int ldg, int offg, const bf16* X,
                   int ldx, int offx, float* dW) {
  // channel counts and slices were checked by the forward convolutions of the same layer
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  unsigned int* err_dev = nullptr;
  error_flag(&err_dev);
  if (!enc || !err_dev || Cin % 16 || Cout % 16) {
    set_last_error("weight gradient: unsupported channel counts or no tensor-map encoder");
    return -1;
  }
  WgGeom G{};
  G.P = W >= 128 ? 128 : (pow2_at_least(W) < 16 ? 16 : pow2_at_least(W));
  G.NT = Cin <= 128 ? Cin : 128;
  G.ntiles_ci = (Cin + G.NT - 1) / G.NT;
  G.co_tiles = (Cout + 127) / 128;
  G.a_region = G.P * 16;
  G.a_bytes = 16 * G.a_region;
  G.b_region = ((G.P + 2) * 16 + 127) / 128 * 128;
  G.b_bytes = (G.NT / 8) * G.b_region;
  G.stage_bytes = (G.a_bytes + G.b_bytes + 1023) / 1024 * 1024;
  G.stages = 3 * G.stage_bytes + 1024 <= TC_SMEM_MAX ? 3 : 2;
  G.tmem_cols = pow2_at_least(3 * G.NT < 32 ? 32 : 3 * G.NT);
  G.chunks_x = (W + G.P - 1) / G.P;
  G.nchunks = H * G.chunks_x;
  int smem = G.stages * G.stage_bytes + 1024;
  const int smem_tmem = tmem_min_smem(G.tmem_cols);
  if (smem < smem_tmem) smem = smem_tmem;
  if (smem > TC_SMEM_MAX) {
    set_last_error("weight-gradient tile does not fit in shared memory");
    return -1;
  }
  CUtensorMap mg, mx;
  cuuint32_t estr[3] = {1, 1, 1};
  {
    cuuint64_t dims[3] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H};
    cuuint64_t strides[2] = {(cuuint64_t)ldg * 2, (cuuint64_t)W * ldg * 2};
    cuuint32_t box[3] = {8, (cuuint32_t)G.P, 1};
    if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(Gd + offg), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_last_error("cuTensorMapEncodeTiled rejected a gradient view");
      return -1;
    }
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H};
    cuuint64_t strides[2] = {(cuuint64_t)ldx * 2, (cuuint64_t)W * ldx * 2};
    cuuint32_t box[3] = {8, (cuuint32_t)(G.P + 2), 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(X + offx), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_last_error("cuTensorMapEncodeTiled rejected an activation view");
      return -1;
    }
  }
  if (first_use_on_device(1)) {
    cudaFuncSetAttribute(k_conv3x3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
    cudaFuncSetAttribute(k_conv3x3_wgrad_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = SM_SMEM / (smem + 2048);
  if (per_sm > 2048 / TC_THREADS) per_sm = 2048 / TC_THREADS;
  if (per_sm > 512 / G.tmem_cols) per_sm = 512 / G.tmem_cols;
  if (per_sm < 1) per_sm = 1;
  // split the pixel chunks so that the CTAs fill the device once
  const int units = 3 * G.ntiles_ci * G.co_tiles;
  G.ksplit = (int)((long)nsm * per_sm / units);
  if (G.ksplit < 1) G.ksplit = 1;
  if (G.ksplit > G.nchunks) G.ksplit = G.nchunks;
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(units * G.ksplit);
  lc.blockDim = dim3(TC_THREADS);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  if (cudaLaunchKernelEx(&lc, k_conv3x3_wgrad_tc, mg, mx, Cin, Cout, dW, G, err_dev) != cudaSuccess) {
    set_last_error("weight-gradient launch failed");
    return -1;
  }
  return 0;
}

bool conv_tc_failed() {
  unsigned int* dev = nullptr;
  unsigned int* host = error_flag(&dev);
  return host && *reinterpret_cast<volatile unsigned int*>(host) != 0u;
}

int conv3x3(cudaStream_t s, int H, int W, int Cin, int Cout, const bf16* X, int ldx, int offx, const bf16* wpk,
            const float* bias, bf16* Y, int ldy, int offy, bool relu, float* yf) {
  if (Cin % 16 || Cout % 16 || ldx % 8 || offx % 8 || ldy % 8 || offy % 8) {
    set_last_error("convolution channel counts and slices must be multiples of 16 and 8");
    return -1;
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  unsigned int* err_dev = nullptr;
  error_flag(&err_dev);
  if (!enc || !err_dev) {
    set_last_error("cuTensorMapEncodeTiled or the mapped error flag is unavailable");
    return -1;
  }
  TcGeom G{};
  G.TW = W >= TC_M ? TC_M : (pow2_at_least(W) < 8 ? 8 : pow2_at_least(W));
  G.R = TC_M / G.TW;
  G.copies = G.R == 1 ? 1 : 3;
  G.boxw = G.R == 1 ? G.TW + 2 : G.TW;
  const int rows = G.R + 2;
  G.a_region = (rows * G.boxw * 16 + 127) / 128 * 128;
  G.a_bytes = G.copies * 2 * G.a_region;
  G.NT = conv_tile_channels(Cout);
  G.b_bytes = 9 * G.NT * 32;
  G.stage_bytes = (G.a_bytes + G.b_bytes + 1023) / 1024 * 1024;
  G.tx_bytes = G.copies * 2 * rows * G.boxw * 16 + G.b_bytes;
  G.tmem_cols = pow2_at_least(2 * G.NT < 64 ? 64 : 2 * G.NT);  // two accumulators, each at least 32 columns
  G.nchunks = Cin / 16;
  G.stages = 3 * G.stage_bytes + 1024 <= TC_SMEM_MAX ? 3 : 2;
  G.tiles_x = (W + G.TW - 1) / G.TW;
  G.tiles_z = (Cout + G.NT - 1) / G.NT;
  G.ntiles = G.tiles_x * ((H + G.R - 1) / G.R) * G.tiles_z;
  // dynamic shared memory: the stages plus alignment slack, at least
  // tmem_min_smem
  int smem = G.stages * G.stage_bytes + 1024;
  const int smem_tmem = tmem_min_smem(G.tmem_cols);
  if (smem < smem_tmem) smem = smem_tmem;
  if (smem > TC_SMEM_MAX) {
    set_last_error("convolution tile does not fit in shared memory");
    return -1;
  }
  CUtensorMap map;
  cuuint64_t dims[3] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[2] = {(cuuint64_t)ldx * 2, (cuuint64_t)W * ldx * 2};
  cuuint32_t box[3] = {8, (cuuint32_t)G.boxw, (cuuint32_t)rows};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(X + offx), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled rejected an activation view");
    return -1;
  }
  if (first_use_on_device(0)) {
    // the largest shared-memory carveout, so that several CTAs fit on an SM
    for (auto k : {k_conv3x3_tc<true>, k_conv3x3_tc<false>}) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
      cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    }
  }
  // persistent CTAs: as many as fit on the device at once (shared memory,
  // with 1 KB static and 1 KB reserved per CTA; threads; tensor-memory
  // columns), at most one per tile
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  auto kern = relu ? k_conv3x3_tc<true> : k_conv3x3_tc<false>;
  int per_sm = SM_SMEM / (smem + 2048);
  if (per_sm > 2048 / TC_THREADS) per_sm = 2048 / TC_THREADS;
  if (per_sm > 512 / G.tmem_cols) per_sm = 512 / G.tmem_cols;
  if (per_sm < 1) per_sm = 1;
  const long slots = (long)nsm * per_sm;
  const int grid = (int)(G.ntiles < slots ? G.ntiles : slots);
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(TC_THREADS);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  if (cudaLaunchKernelEx(&lc, kern, map, wpk, bias, Y, ldy, offy, yf, H, W, Cout, G, err_dev) != cudaSuccess) {
    set_last_error("convolution launch failed");
    return -1;
  }
  return 0;
}

}  // namespace nn
}  // namespace ibm
