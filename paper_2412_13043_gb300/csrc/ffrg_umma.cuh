// Tensor-core (tcgen05 / UMMA) pieces of the FP64-faithful sliced contraction
// used for the finite-T sums over many loop-side states (see ffrg_ozaki.cu).
//
// Operands are BF16 slices holding small integers (at most 32 in magnitude),
// so every product is an integer below 2^10 in magnitude and any sum of up to
// 2^14 of them is an integer below 2^24: the FP32 accumulator in tensor memory
// holds it exactly.  One CTA computes one pass: a 128 x 256 output tile of one
// slice pair over one K range, D = A_i^T-tile x B_j-tile, and writes the exact
// FP32 sums to global memory.
//
// Shared-memory operand layout (no swizzle, K-major, the canonical
// "interleaved" form of the UMMA shared-memory descriptor): a tile of R rows x
// kBK K-elements (BF16) is made of 8 x 8 core matrices of 128 contiguous bytes
// (8 rows of 16 bytes); core matrices adjacent in the row direction are 128
// bytes apart (stride byte offset, SBO) and those adjacent in K are R x 16
// bytes apart (leading byte offset, LBO).  Global memory holds the slices
// already in this tile order, so one bulk copy moves a whole tile.
//
// Roles of the 4 warps: warp 0 lane 0 issues the bulk copies of each K-tile
// (A: 8 KB, B: 16 KB) into a 4-stage ring; warp 1 allocates 256 columns of
// tensor memory and lane 0 issues the MMAs (M = 128, N = 256, K = 16 each, two
// per K-tile) and commits each stage back to the producer; after the last
// commit all 4 warps read their 32 accumulator lanes (tcgen05.ld) and store
// the rows.  Every wait is bounded; a wait that gives up sets the status word
// and the CTA unwinds (remaining waits bounded too, tensor memory freed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ffrg {
namespace umma {

constexpr int kBM = 128;          // output rows per tile (A rows)
constexpr int kBN = 256;          // output columns per tile (B rows: states)
constexpr int kBK = 32;           // K-elements per stage
constexpr int kStages = 4;
constexpr int kTileA = kBM * kBK * 2;   // 8 KB
constexpr int kTileB = kBN * kBK * 2;   // 16 KB
constexpr int kStageBytes = kTileA + kTileB;
constexpr int kSmemBytes = kStages * kStageBytes;   // 96 KB: two CTAs per SM
constexpr int kTmemCols = 256;
constexpr int kThreadsGemm = 128;
constexpr int kMaxExactK = 16384;  // K-elements whose slice products sum exactly in FP32
constexpr unsigned kStatusTimeoutBit = 2u;
constexpr long long kWaitLimit = 4000000000LL;   // clock cycles (about 2 s)

// element offset of (row r, K-element k) inside a rows x kBK tile
__host__ __device__ inline int tile_offset(int r, int k, int rows) {
  return (k >> 3) * (rows * 8) + (r >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

struct GemmArgs {
  const uint16_t *A;   // BF16 bits, slices [nsl][m_tiles][k_tiles][128 x kBK tile]
  const uint16_t *B;   // BF16 bits, slices [nsl][n_tiles][k_tiles][256 x kBK tile]
  float *part;         // [passes][m_tiles * 128][n_tiles * 256], exact sums per pass
  const int4 *pass_tab; // per CTA z: slice pair (i, j), output pass, K range
  int m_tiles, n_tiles, k_tiles;
  int kt_per_chunk, n_chunks;  // K-tiles per pass and K ranges per slice pair
  unsigned *status;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a barrier phase; false (and the status bit) when it gives up
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, unsigned *status) {
  const long long t0 = clock64();
  while (!bar_try(bar, parity)) {
    if (clock64() - t0 > kWaitLimit) {
      if (status) atomicOr(status, kStatusTimeoutBit);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// shared-memory matrix descriptor: no swizzle, byte offsets in 16-byte units,
// descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// arrive on `bar` once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns of 32-bit accumulators: this thread's lane, 32 columns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One pass per CTA: blockIdx.x = output column tile, blockIdx.y = output row
// tile, blockIdx.z = slot of the pass table (slice pair, its output pass and
// K range; slots that run together share an A slice).
__global__ void __launch_bounds__(kThreadsGemm, 1) slice_pair_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued, consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = blockIdx.x, tm = blockIdx.y;
  const int4 pt = g.pass_tab[blockIdx.z];
  const int2 ij = make_int2(pt.x, pt.y);
  const int pass = pt.z, chunk = pt.w;
  const int kt0 = chunk * g.kt_per_chunk;
  const int nkt = min(g.kt_per_chunk, g.k_tiles - kt0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    bar_init(&done, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  const uint16_t *Ab = g.A + ((size_t)(ij.x * g.m_tiles + tm) * g.k_tiles) * (kBM * kBK);
  const uint16_t *Bb = g.B + ((size_t)(ij.y * g.n_tiles + tn) * g.k_tiles) * (kBN * kBK);

  if (warp == 0 && lane == 0) {
    // producer: K-tile t goes to stage t % 2; the stage's previous MMAs must have completed
    for (int t = 0; t < nkt; ++t) {
      const int s = t % kStages;
      const uint32_t ph = (uint32_t)(t / kStages) & 1u;
      if (!bar_wait(&empty[s], ph ^ 1u, g.status)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*(volatile int *)&abort_flag) break;
      unsigned char *st = smem + s * kStageBytes;
      bar_expect_tx(&full[s], kStageBytes);
      bulk_load(st, Ab + (size_t)(kt0 + t) * (kBM * kBK), kTileA, &full[s]);
      bulk_load(st + kTileA, Bb + (size_t)(kt0 + t) * (kBN * kBK), kTileB, &full[s]);
      issued = t + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int t = 0; t < nkt; ++t) {
      const int s = t % kStages;
      const uint32_t ph = (uint32_t)(t / kStages) & 1u;
      if (!bar_wait(&full[s], ph, g.status) || *(volatile int *)&abort_flag) {
        atomicExch(&abort_flag, 1);
        break;
      }
      fence_after();
      const uint32_t a0 = su32(smem + s * kStageBytes), b0 = a0 + kTileA;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K = 16 spans two core matrices in K: 2 x LBO bytes per step
        const uint64_t ad = smem_desc(a0 + kk * 2 * (kBM * 16), kBM * 16, 128);
        const uint64_t bd = smem_desc(b0 + kk * 2 * (kBN * 16), kBN * 16, 128);
        mma_bf16(tmem, ad, bd, (t > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
      consumed = t + 1;
    }
    mma_commit(&done);   // after every MMA issued above
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) {
    // an unwinding CTA first waits (bounded) for its own copies still in flight
    for (int t = consumed; t < issued; ++t)
      bar_wait(&full[t % kStages], (uint32_t)(t / kStages) & 1u, nullptr);
  }

  // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w + 31
  const bool ok = bar_wait(&done, 0, g.status) && !*(volatile int *)&abort_flag;
  fence_after();
  if (ok && nkt > 0) {
    const int row = tm * kBM + warp * 32 + lane;
    const size_t ld = (size_t)g.n_tiles * kBN;
    float *dst = g.part + ((size_t)pass * g.m_tiles * kBM + row) * ld + (size_t)tn * kBN;
#pragma unroll 1
    for (int c = 0; c < kBN / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
      float4 *d4 = reinterpret_cast<float4 *>(dst + c * 32);
      // streaming stores: the pass sums are read once, by the combine kernel;
      // evict-first keeps the operand slices in L2 for the other passes
#pragma unroll
      for (int q = 0; q < 8; ++q)
        __stcs(d4 + q, make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                   __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace umma
}  // namespace ffrg
