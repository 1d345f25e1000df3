// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M, N] = A[M, K] * B[N, K]^T   (A and B row-major, K contiguous; FP32 accumulate)
// One CTA of 128 threads computes a 128 x 128 tile of C:
//  * warp 0 allocates 128 TMEM columns (128 lanes x 128 FP32 accumulators);
//  * per K chunk of 64, all threads copy the A and B tiles into shared memory in
//    the canonical no-swizzle K-major layout (8-row x 16-byte core matrices,
//    core matrices adjacent in K 128 B apart, 8-row groups 1024 B apart), then
//    fence the writes to the async proxy;
//  * one thread issues four tcgen05.mma (M=128, N=128, K=16 each) and commits
//    them to an mbarrier, on which every thread waits (bounded) before the
//    buffer is reused;
//  * epilogue: each warp reads its 32 TMEM lanes (= 32 rows of C) with
//    tcgen05.ld, applies the epilogue functor and stores.
// Requirements: M % 128 == 0, N % 128 == 0, K % 64 == 0, 16-byte aligned rows.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace nrpf {

constexpr int kGemmBM = 128, kGemmBN = 128, kGemmBK = 64;
constexpr int kGemmThreads = 128;
constexpr uint32_t kTmemCols = 128;
// spin limit of the MMA-completion wait; the kernel reports a timeout in
// *err instead of waiting forever
constexpr uint32_t kMbarSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle, K-major): start address,
// leading byte offset (between core matrices adjacent in K), stride byte
// offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;  // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy a [rows x 64] BF16 tile (row stride ld elements) into the canonical
// layout: element (r, k) at byte (r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2.
template <int ROWS>
__device__ __forceinline__ void load_tile_kmajor(uint8_t* s, const __nv_bfloat16* __restrict__ g, int64_t ld,
                                                 int tid) {
  constexpr int chunks = ROWS * 8;  // 16-byte chunks
#pragma unroll 4
  for (int c = tid; c < chunks; c += kGemmThreads) {
    const int r = c >> 3, k8 = c & 7;
    const uint4 v = *reinterpret_cast<const uint4*>(g + (int64_t)r * ld + k8 * 8);
    *reinterpret_cast<uint4*>(s + (r >> 3) * 1024 + k8 * 128 + (r & 7) * 16) = v;
  }
}

// Epilogue functor interface: op(row, col, value) for one C element.
template <class Epi>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(const __nv_bfloat16* __restrict__ A,
                                                          const __nv_bfloat16* __restrict__ B, int M, int N, int K,
                                                          Epi epi, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                            // 128 x 64 BF16 = 16 KB
  uint8_t* sB = smem + kGemmBM * kGemmBK * 2;    // 128 x 64 BF16 = 16 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * kGemmBN;
  if (warp == 0) tmem_alloc(&tmem_holder, kTmemCols);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  constexpr uint32_t idesc = make_idesc_bf16(kGemmBM, kGemmBN);
  const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
  uint32_t phase = 0;
  bool timed_out = false;
  const int nk = K / kGemmBK;
  for (int kc = 0; kc < nk; ++kc) {
    load_tile_kmajor<kGemmBM>(sA, A + (int64_t)m0 * K + kc * kGemmBK, K, tid);
    load_tile_kmajor<kGemmBN>(sB, B + (int64_t)n0 * K + kc * kGemmBK, K, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kGemmBK / 16; ++kk) {
        const uint64_t ad = make_sdesc(aaddr + kk * 256, 128, 1024);
        const uint64_t bd = make_sdesc(baddr + kk * 256, 128, 1024);
        umma_bf16(tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&mbar);
    }
    // wait for the MMAs of this chunk before the tiles are overwritten
    uint32_t spins = 0;
    while (!mbar_try_wait(&mbar, phase)) {
      if (++spins > kMbarSpinLimit) {
        timed_out = true;
        break;
      }
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) atomicExch(err, 1);
      // give the MMAs in flight a second bounded wait before TMEM is freed
      uint32_t again = 0;
      while (!mbar_try_wait(&mbar, phase ^ 1) && ++again < kMbarSpinLimit) {
      }
      timed_out = true;
      break;
    }
  }
  if (!timed_out) {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kGemmBN; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) epi(row, n0 + c0 + j, v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Dynamic shared memory per CTA: the two 16 KB tiles, rounded up to 64 KB so
// that at most three CTAs share an SM and their TMEM (3 x 128 of 512 columns)
// never has to wait for another CTA's deallocation.
constexpr size_t kGemmSmem = 64 * 1024;

}  // namespace nrpf

// ---------------------------------------------------------------------------
// Pipelined variant: TMA (cp.async.bulk.tensor) fills a ring of kStages
// shared-memory stages with 128-byte-swizzled tiles; thread 0 of warp 0
// produces (expect-tx + two TMA loads per stage), thread 0 of warp 1 issues
// the MMAs of each stage as soon as its bytes have landed and commits them to
// the stage's "empty" barrier, which releases the stage to the producer.  The
// accumulator is complete when a final commit arrives on "done"; then all four
// warps run the same epilogue as k_gemm_tc.  Every wait is bounded.
// ---------------------------------------------------------------------------
namespace nrpf {

constexpr int kStages = 4;
constexpr uint32_t kStageBytes = (kGemmBM + kGemmBN) * kGemmBK * 2;  // 32 KB
constexpr size_t kGemmTmaSmem = (size_t)kStages * kStageBytes + 1024;

// Shared-memory descriptor, K-major with 128-byte swizzle: 8-row atoms of
// 1024 B (stride byte offset), leading byte offset unused (1), layout type 2.
__device__ __forceinline__ uint64_t make_sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < kMbarSpinLimit; ++spins)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <class Epi, class TMap>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tma(const __grid_constant__ TMap tmA,
                                                           const __grid_constant__ TMap tmB, int M, int N, int K,
                                                           Epi epi, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_holder;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * kGemmBN;
  const int nk = K / kGemmBK;
  if (warp == 0) tmem_alloc(&tmem_holder, kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  const uint32_t base = smem_u32(smem);
  if (warp == 0 && lane == 0) {
    // producer
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kStages;
      if (kc >= kStages && !mbar_wait(&empty[s], ((kc / kStages) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      const uint32_t sa = base + s * kStageBytes, sb = sa + kGemmBM * kGemmBK * 2;
      mbar_expect_tx(&full[s], kStageBytes);
      tma_load_2d(sa, &tmA, kc * kGemmBK, m0, &full[s]);
      tma_load_2d(sb, &tmB, kc * kGemmBK, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = make_idesc_bf16(kGemmBM, kGemmBN);
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kStages;
      if (!mbar_wait(&full[s], (kc / kStages) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + s * kStageBytes, sb = sa + kGemmBM * kGemmBK * 2;
#pragma unroll
      for (int kk = 0; kk < kGemmBK / 16; ++kk)
        umma_bf16(tmem, make_sdesc_sw128(sa + kk * 32), make_sdesc_sw128(sb + kk * 32), idesc,
                  (kc > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    if (!ok) s_fail = 1;
    umma_commit(&done);  // arrives once every MMA issued above has completed
  }
  const bool got = mbar_wait(&done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool fail = !got || s_fail;
  if (fail) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kGemmBN; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) epi(row, n0 + c0 + j, v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace nrpf
