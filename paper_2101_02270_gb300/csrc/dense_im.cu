// Instance-major dense block for the FP32 LU (Sec. 4.3: the serial tail of the
// column DAG, factorised as one dense matrix per instance).
//
// In the interleaved layout every lane of a warp is its own instance, so the
// 32 threads of a warp never share an operand and the trailing update can
// only reuse data through a per-thread register tile.  Here instance b's
// dense block is its own column-major ndp x ndp matrix,
//   element (r, c) at lu + ((b / 32) * NLU + NS) * 32 + (b % 32) * ndp^2 + c * ndp + r,
// inside the same per-tile LU array (only the order of the dense part
// changes; ndp is a multiple of 64).  The factorisation is blocked, without
// pivoting, and left-looking by outer panels (blocked Crout).  Outer panel j
// at column kj = 128 j, of width 128 (64 for the last one when ndp % 128 ==
// 64):
//   k_im_gemm          : (j > 0) its block column and row, rows [kj, ndp) x
//                        columns [kj, kj+128) and rows [kj, kj+128) x columns
//                        [kj+128, ndp), minus the products of all earlier
//                        panels in one pass of depth kj: one 128 x 128 tile
//                        of C per CTA, operand chunks of depth 32 loaded by
//                        TMA into a two-stage shared-memory ring, an 8 x 8
//                        register tile per thread updated with packed
//                        two-wide FP32 FMAs;
//   k_im_diag  (step 0): LU of the 64 x 64 diagonal block at (kj, kj), and the
//                        inverses U11^-1, L11^-1 of its factors;
//   k_im_panel (step 0): L21 = A21 U11^-1 for the rows below and
//                        U12 = L11^-1 A12 for the columns to the right, as
//                        register-tiled products on 128 x 64 tiles;
//   k_im_diag  (step 1): block (kj+64, kj+64) minus L(., kj:kj+64) U(kj:kj+64, .),
//                        then its LU and inverses;
//   k_im_panel (step 1): rows below / columns right of kj+128, each first minus
//                        its product with step 0's L or U, then multiplied by
//                        the inverse.
// Every entry of the block is read and written by k_im_gemm once per
// refactorisation (a right-looking order would rewrite the trailing block
// after every outer panel), and each entry still takes its subtractions in
// ascending pivot order, as the interleaved kernels do.  The panel multiplies
// by the explicit inverses of the 64 x 64 diagonal factors (the LU is the
// FP32 inner solve of an inexact Newton step whose mismatch and update stay
// FP64).
#include <cfloat>
#include <cstdint>

#include "dense_im.h"

namespace nrpf {

namespace {

constexpr int kImOuter = 128;               // outer panel width
constexpr int kImTile = 128;                // GEMM tile (rows and columns of C)
constexpr int kImKc = 32;                   // GEMM depth per stage
constexpr int kImStages = 2;
// column groups of 32 per warp in the block update (four columns of each per
// thread): 2 (an 8 x 8 register tile, 8 warps per CTA) or 4 (8 x 16, 4 warps).
// The wider tile needs fewer shared-memory wavefronts per FMA but leaves half
// the warps; measured on the 9,000-bus update it is 1 % slower, so the 8 x 8
// tile is used.
constexpr int kImGC = 2;
// packed two-wide FP32 FMA (fma.rn.f32x2) in the trailing update: each
// instruction updates two rows of a column; the B chunk is negated while it is
// transposed, so acc + a (-b) rounds exactly as fmaf(-a, b, acc)
constexpr bool kImPacked = true;
constexpr int kImGemmThreads = 32 * 4 * (4 / kImGC);
constexpr uint32_t kImABytes = kImKc * kImTile * 4;  // 16 KB: [32 columns][128 rows]
constexpr uint32_t kImBBytes = kImTile * kImKc * 4;  // 16 KB: [128 columns][32 rows], swizzled
constexpr uint32_t kImStageBytes = kImABytes + kImBBytes;
// two TMA stages, the double-buffered transposed B chunk, 1024-byte alignment slack
constexpr size_t kImGemmSmem = (size_t)kImStages * kImStageBytes + 2 * (size_t)kImKc * kImTile * 4 + 1024;
// bounded wait on the TMA completion barriers (each try_wait also suspends
// for a hardware-defined time window)
constexpr uint32_t kImSpinLimit = 1u << 20;

constexpr int kImDiagThreads = 512;
constexpr int kImSolveThreads = 256;
constexpr int kPitch = 68;  // shared row pitch (floats) of 64-wide blocks: rows stay 16-byte aligned

__device__ __forceinline__ float* im_block(const DevPlan& P, const DevState& S, int b) {
  return reinterpret_cast<float*>(S.lu) + ((size_t)(b >> 5) * (size_t)P.NLU + (size_t)P.NS) * kTile +
         (size_t)(b & 31) * (size_t)P.ndp * (size_t)P.ndp;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared (no register staging)
__device__ __forceinline__ void cp16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp16_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < kImSpinLimit; ++spins) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                       uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ float comp(const float4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// Update C -= A B of one 128 x 128 tile of one instance, over the depth of the
// pivot columns k .. k + 32 nkc - 1, the tile held in registers throughout.
// Per chunk of depth 32, TMA lands the A chunk (As[kk][i] = A(i0 + i, k + 32 kc
// + kk), 512 bytes per kk) and the B chunk as 128 rows of 128 bytes (row j =
// B(k + 32 kc + 0..31, j0 + j), 16-byte chunk q stored at chunk q ^ (j % 8):
// TMA 128-byte swizzle) in a two-stage ring.  The CTA first transposes the B
// chunk into Bt[kk][j] (double-buffered, so one barrier per chunk suffices),
// then every thread runs the register-tiled product: per kk two 16-byte loads
// of A and two of B feed 64 FMAs, the next kk's fragments loaded while the
// current ones are used.
// Warp w = (wy, wx), wy = w % 4, wx = w / 4, owns the 32 x (32 kImGC) block at
// rows 32 wy, columns 32 kImGC wx of the tile; its lane (lx, ly), lx = lane % 8,
// ly = lane / 8, owns rows 32 wy + ly*4 + 16h + q and columns 32 kImGC wx +
// lx*4 + 32g + r (h < 2, g < kImGC; q, r < 4).  Every shared load of a warp then touches four
// (A) or eight (B) distinct 16-byte words of one 128-byte row: one wavefront.
// A tile whose rows (columns) run past ndp has 64 of them; the warps outside
// skip the arithmetic (the TMA box past ndp is filled with zeros, unused).
// Returns the chunk whose wait ran out, or -1.
// ---------------------------------------------------------------------------

// TMA copies of GEMM chunk kc (A: 128 rows x 32 columns, B: 32 rows x 128
// columns of instance (tile_b, lane_b)) into stage kc % kImStages
__device__ __forceinline__ void issue_chunk(uint8_t* sm, uint64_t* full, const CUtensorMap* tmA,
                                            const CUtensorMap* tmB, int kc, int i0, int j0, int k, int lane_b,
                                            int tile_b) {
  const int s = kc % kImStages;
  const uint32_t sa = su32(sm) + (uint32_t)s * kImStageBytes;
  // order the generic-proxy reads of this stage before the async-proxy writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(&full[s], kImStageBytes);
  tma_4d(sa, tmA, i0, k + kc * kImKc, lane_b, tile_b, &full[s]);
  tma_4d(sa + kImABytes, tmB, k + kc * kImKc, j0, lane_b, tile_b, &full[s]);
}

__device__ __forceinline__ void fma_kk(float (&acc)[2][kImGC][4][4], const float4 (&a)[2],
                                       const float4 (&b)[kImGC]) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < kImGC; ++g)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float bv = comp(b[g], r);
        float* d = acc[h][g][r];
        d[0] = fmaf(-a[h].x, bv, d[0]);
        d[1] = fmaf(-a[h].y, bv, d[1]);
        d[2] = fmaf(-a[h].z, bv, d[2]);
        d[3] = fmaf(-a[h].w, bv, d[3]);
      }
}

// the same update on packed pairs: acc2[h][g][r][p] = rows 2p, 2p+1 of the
// thread's 4-row group h, column g, r; b holds -B
__device__ __forceinline__ void fma_kk2(float2 (&acc)[2][kImGC][4][2], const float4 (&a)[2],
                                        const float4 (&b)[kImGC]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 a01 = make_float2(a[h].x, a[h].y), a23 = make_float2(a[h].z, a[h].w);
#pragma unroll
    for (int g = 0; g < kImGC; ++g)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float bv = comp(b[g], r);
        const float2 b2 = make_float2(bv, bv);
        acc[h][g][r][0] = __ffma2_rn(a01, b2, acc[h][g][r][0]);
        acc[h][g][r][1] = __ffma2_rn(a23, b2, acc[h][g][r][1]);
      }
  }
}

__device__ __forceinline__ int gemm_tile(float* __restrict__ C, int ld, int i0, int j0, int k, int nkc, uint8_t* sm,
                                         uint64_t* full, const CUtensorMap* tmA, const CUtensorMap* tmB, int lane_b,
                                         int tile_b, bool active, int rw, int cw, int lx, int ly) {
  // acc[h][g][r][q] (acc2: the same as pairs of q): row rw + ly*4 + 16h + q,
  // column cw + lx*4 + 32g + r
  float acc[2][kImGC][4][4];
  float2 acc2[2][kImGC][4][2];
  const size_t cstride = (size_t)ld;
  if (active) {
    const float* __restrict__ Ct = C + (size_t)(j0 + cw + lx * 4) * ld + i0 + rw + ly * 4;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < kImGC; ++g)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 v = *reinterpret_cast<const float4*>(Ct + (size_t)(32 * g + r) * cstride + 16 * h);
          if constexpr (kImPacked) {
            acc2[h][g][r][0] = make_float2(v.x, v.y);
            acc2[h][g][r][1] = make_float2(v.z, v.w);
          } else {
            acc[h][g][r][0] = v.x;
            acc[h][g][r][1] = v.y;
            acc[h][g][r][2] = v.z;
            acc[h][g][r][3] = v.w;
          }
        }
  }
  float* Bt0 = reinterpret_cast<float*>(sm + (size_t)kImStages * kImStageBytes);
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int kc = 0; kc < nkc; ++kc) {
    const int s = kc % kImStages;
    const bool ok = bar_wait(&full[s], (uint32_t)(kc / kImStages) & 1u);
    // transpose the B chunk: thread tid takes column j = tid % 128 and the
    // 16-byte words q = tid / 128, tid / 128 + 2, ... of its row
    float* Bt = Bt0 + (kc & 1) * (kImKc * kImTile);
    {
      const uint8_t* Bs = sm + (size_t)s * kImStageBytes + kImABytes;
      const int j = tid & (kImTile - 1);
#pragma unroll
      for (int q = tid >> 7; q < kImKc / 4; q += kImGemmThreads / kImTile) {
        const float4 v = *reinterpret_cast<const float4*>(Bs + j * 128 + ((q ^ (j & 7)) << 4));
        const float sg = kImPacked ? -1.f : 1.f;
        Bt[(4 * q) * kImTile + j] = sg * v.x;
        Bt[(4 * q + 1) * kImTile + j] = sg * v.y;
        Bt[(4 * q + 2) * kImTile + j] = sg * v.z;
        Bt[(4 * q + 3) * kImTile + j] = sg * v.w;
      }
    }
    // one barrier: the chunk has landed for everyone, Bt is complete, and
    // every warp is done with chunk kc - 1 (its stage may be refilled)
    if (__syncthreads_or(!ok)) return kc;
    if (kc >= 1 && kc + 1 < nkc && tid == 0)
      issue_chunk(sm, full, tmA, tmB, kc + 1, i0, j0, k, lane_b, tile_b);
    if (active) {
      const float* As = reinterpret_cast<const float*>(sm + (size_t)s * kImStageBytes) + rw + ly * 4;
      const float* Bq = Bt + cw + lx * 4;
      float4 a[2], b[kImGC];
      a[0] = *reinterpret_cast<const float4*>(As);
      a[1] = *reinterpret_cast<const float4*>(As + 16);
#pragma unroll
      for (int g = 0; g < kImGC; ++g) b[g] = *reinterpret_cast<const float4*>(Bq + 32 * g);
#pragma unroll 8
      for (int kk = 0; kk < kImKc - 1; ++kk) {
        float4 an[2], bn[kImGC];
        an[0] = *reinterpret_cast<const float4*>(As + (kk + 1) * kImTile);
        an[1] = *reinterpret_cast<const float4*>(As + (kk + 1) * kImTile + 16);
#pragma unroll
        for (int g = 0; g < kImGC; ++g) bn[g] = *reinterpret_cast<const float4*>(Bq + (kk + 1) * kImTile + 32 * g);
        if constexpr (kImPacked) fma_kk2(acc2, a, b);
        else fma_kk(acc, a, b);
        a[0] = an[0];
        a[1] = an[1];
#pragma unroll
        for (int g = 0; g < kImGC; ++g) b[g] = bn[g];
      }
      if constexpr (kImPacked) fma_kk2(acc2, a, b);
      else fma_kk(acc, a, b);
    }
  }
  if (active) {
    float* __restrict__ Ct = C + (size_t)(j0 + cw + lx * 4) * ld + i0 + rw + ly * 4;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < kImGC; ++g)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          *reinterpret_cast<float4*>(Ct + (size_t)(32 * g + r) * cstride + 16 * h) =
              kImPacked ? make_float4(acc2[h][g][r][0].x, acc2[h][g][r][0].y, acc2[h][g][r][1].x, acc2[h][g][r][1].y)
                        : make_float4(acc[h][g][r][0], acc[h][g][r][1], acc[h][g][r][2], acc[h][g][r][3]);
  }
  return -1;
}

// The block column and row of the outer panel at r0: tiles of 128 over rows
// [r0, ld) x columns [r0, r0+128) and rows [r0, r0+128) x columns [r0+128,
// ld), 2 ntc - 1 of them (ntc = tiles across [r0, ld)), each minus the
// products over pivot columns 0 .. r0-1 (r0 / 32 chunks).  grid: Bp * (2 ntc
// - 1) CTAs, tile-fastest within an instance, so that the CTAs resident at
// one time share their instance's operand panels in L2.
__global__ void __launch_bounds__(kImGemmThreads, 2)
    k_im_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, DevPlan P,
              DevState S, int r0, int ntc, const int32_t* __restrict__ gate) {
  extern __shared__ uint8_t im_smem_raw[];
  __shared__ __align__(8) uint64_t full[kImStages];
  if (gate && *gate == 0) return;
  const int ntile = 2 * ntc - 1;
  const int b = (int)(blockIdx.x / (unsigned)ntile);
  const int t = (int)(blockIdx.x - (unsigned)b * (unsigned)ntile);
  if (!S.active[b]) return;
  const int ld = P.ndp;
  const int k = 0, nkc = r0 / kImKc;
  const int i0 = r0 + (t < ntc ? t : 0) * kImTile, j0 = r0 + (t < ntc ? 0 : t - ntc + 1) * kImTile;
  // 1024-byte alignment for the swizzled B chunks (offset arithmetic on the
  // shared array keeps the pointer in the shared address space)
  uint8_t* sm = im_smem_raw + ((1024u - (su32(im_smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rw = (warp & 3) * 32, cw = (warp >> 2) * 32 * kImGC;
  const int lane_b = b & 31, tile_b = b >> 5;
  if (tid == 0) {
    for (int s = 0; s < kImStages; ++s) bar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int kc = 0; kc < kImStages && kc < nkc; ++kc)
      issue_chunk(sm, full, &tmA, &tmB, kc, i0, j0, k, lane_b, tile_b);
  // rows (columns) of this tile inside the block: 128, or 64 at the edge
  const int mrows = ld - i0 < kImTile ? ld - i0 : kImTile;
  const int ncols = ld - j0 < kImTile ? ld - j0 : kImTile;
  const bool active = rw < mrows && cw < ncols;
  const int fail = gemm_tile(im_block(P, S, b), ld, i0, j0, k, nkc, sm, full, &tmA, &tmB, lane_b, tile_b, active, rw, cw,
                             lane & 7, lane >> 3);
  if (fail >= 0 && tid == 0) {
    // a copy did not land in time: the instance is marked failed (its step
    // is discarded) and the CTA waits, bounded, for the copies it issued
    // (chunks up to fail + 1: one chunk ahead of the one consumed)
    S.bad[b] = 1;
    const int issued = fail + 2 < nkc ? fail + 2 : nkc;
    for (int kc = fail; kc < issued; ++kc) bar_wait(&full[kc % kImStages], (uint32_t)(kc / kImStages) & 1u);
  }
}

// ---------------------------------------------------------------------------
// LU of the 64 x 64 diagonal block at (ki, ki), one CTA per instance, and the
// inverses of its factors.  With PRE, the block first receives the product
// L(ki:ki+64, k:k+64) U(k:k+64, ki:ki+64) of the outer panel's first step.
// Unblocked right-looking elimination: the pivot column is scaled by the
// reciprocal of the pivot, then the trailing block takes the rank-1 update,
// and the same row operations on an identity block give L11^-1.  A backward
// sweep over the rows of [U | I] then gives U11^-1.  Both go to the instance's
// slot of S.inv as
//   ui[q * 64 + c] = U11^-1(q, c),  li[q * 64 + r] = L11^-1(r, q)
// (zero outside the triangles), the operands the panel kernel multiplies by.
// Thread (tr, tc) = (tid / R, tid % R), R = 8 threads per row, holds in
// registers the entries of row tr in the columns c = tc + R i (i < 64 / R) of
// D, of L11^-1 and of U11^-1.  Per pivot p the threads of row p publish their
// row to a double-buffered shared row (one barrier per pivot), the multiplier
// of row tr comes from its owner by a shuffle among the row's R lanes, and
// every update is unrolled.  Measured on the 9,000-bus block: R = 4 (256
// threads) 184 ms per step, stalled on instruction fetch (the unrolled pivot
// loops); R = 8 179 ms; R = 16 304 ms; a pivot loop not unrolled, 558 ms.
// Shared memory (dynamic, PRE only): W1[q][r] = L(ki + r, k + q), W2[c][q] =
// U(k + q, ki + c).
// ---------------------------------------------------------------------------
constexpr size_t kImDiagSmemPre = 2 * 64 * kPitch * sizeof(float);

template <bool PRE>
__global__ void __launch_bounds__(kImDiagThreads, 2) k_im_diag(DevPlan P, DevState S, int k, int ki,
                                                                        const int32_t* __restrict__ gate) {
  constexpr int R = kImDiagThreads / 64;  // threads per row
  constexpr int NC = 64 / R;              // columns per thread
  extern __shared__ __align__(16) float diag_smem[];
  __shared__ float prow[2][64], pli[2][64], invd[64];
  if (gate && *gate == 0) return;
  const int b = blockIdx.x;
  if (!S.active[b]) return;
  const int ld = P.ndp, tid = threadIdx.x, tc = tid % R, tr = tid / R;
  const int src0 = tid & 31 & ~(R - 1);  // lane of (tr, 0)
  float* __restrict__ A = im_block(P, S, b);
  float d[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) d[i] = A[(size_t)(ki + tc + R * i) * ld + ki + tr];
  if (PRE) {
    float(*W1)[kPitch] = reinterpret_cast<float(*)[kPitch]>(diag_smem);
    float(*W2)[kPitch] = reinterpret_cast<float(*)[kPitch]>(diag_smem + 64 * kPitch);
#pragma unroll
    for (int j = 0; j < 64 * 16 / kImDiagThreads; ++j) {
      const int e = tid + j * kImDiagThreads, c = e >> 4, r4 = 4 * (e & 15);
      cp16(&W1[c][r4], A + (size_t)(k + c) * ld + ki + r4);
      cp16(&W2[c][r4], A + (size_t)(ki + c) * ld + k + r4);
    }
    cp16_wait_all();
    __syncthreads();
    // D(tr, c) minus the products in ascending q
#pragma unroll 1
    for (int q = 0; q < 64; q += 4) {
      const float l0 = W1[q][tr], l1 = W1[q + 1][tr], l2 = W1[q + 2][tr], l3 = W1[q + 3][tr];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const float4 u = *reinterpret_cast<const float4*>(&W2[tc + R * i][q]);
        d[i] = fmaf(-l0, u.x, d[i]);
        d[i] = fmaf(-l1, u.y, d[i]);
        d[i] = fmaf(-l2, u.z, d[i]);
        d[i] = fmaf(-l3, u.w, d[i]);
      }
    }
  }
  float li[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) li[i] = (tc + R * i == tr) ? 1.f : 0.f;
#pragma unroll
  for (int p = 0; p < 64; ++p) {
    const int buf = p & 1;
    if (tr == p) {
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        prow[buf][tc + R * i] = d[i];
        pli[buf][tc + R * i] = li[i];
      }
    }
    __syncthreads();
    const float lraw = __shfl_sync(0xffffffffu, d[p / R], src0 | (p % R));  // D(tr, p)
    if (tr > p) {
      const float inv = 1.f / prow[buf][p];
      const float l = lraw * inv;
      if (tc == p % R) d[p / R] = l;
#pragma unroll
      for (int i = 0; i < NC; ++i)
        if (tc + R * i > p) d[i] = fmaf(-l, prow[buf][tc + R * i], d[i]);
#pragma unroll
      for (int i = 0; i < NC; ++i)
        if (tc + R * i <= p) li[i] = fmaf(-l, pli[buf][tc + R * i], li[i]);
    }
  }
  float* __restrict__ inv_out = reinterpret_cast<float*>(S.inv) + (size_t)b * 8192;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    A[(size_t)(ki + tc + R * i) * ld + ki + tr] = d[i];
    inv_out[4096 + (tc + R * i) * 64 + tr] = li[i];  // li[q][r] = L11^-1(r, q)
    if (tc + R * i == tr) invd[tr] = 1.f / d[i];
  }
  float ui[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) ui[i] = (tc + R * i == tr) ? 1.f : 0.f;
  __syncthreads();
  // row p of [U | I], still unscaled, goes to the rows above it; then row p
  // is scaled by 1 / U(p, p)
#pragma unroll
  for (int p = 63; p >= 0; --p) {
    const int buf = p & 1;
    if (tr == p) {
#pragma unroll
      for (int i = 0; i < NC; ++i) prow[buf][tc + R * i] = ui[i];
    }
    __syncthreads();
    const float uraw = __shfl_sync(0xffffffffu, d[p / R], src0 | (p % R));  // U(tr, p)
    if (tr < p) {
      const float u = uraw * invd[p];
#pragma unroll
      for (int i = 0; i < NC; ++i)
        if (tc + R * i >= p) ui[i] = fmaf(-u, prow[buf][tc + R * i], ui[i]);
    } else if (tr == p) {
#pragma unroll
      for (int i = 0; i < NC; ++i)
        if (tc + R * i >= p) ui[i] *= invd[p];
    }
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) inv_out[tr * 64 + tc + R * i] = ui[i];  // ui[q][c] = U11^-1(q, c)
}

// ---------------------------------------------------------------------------
// Panel of the step at ki (the diagonal block factorised, its inverses in
// S.inv): tasks 0 .. nch-1 take 128 rows each of L21 (rows ki+64 ..), tasks
// nch .. 2nch-1 128 columns each of U12 (columns ki+64 ..).  Both are products
// on a 128 x 64 tile T whose long side m runs over the task's rows (columns)
// and whose short side n over the 64 columns (rows) of the step:
//   rows   : T(m, n) = A(i, ki + n),  L21(i, .) = [T - L(i, k:k+64) U(k:k+64, ki:ki+64)] U11^-1
//   columns: T(m, n) = A(ki + n, j),  U12(., j) = L11^-1 [T - L(ki:ki+64, k:k+64) U(k:k+64, j)]
// (the bracketed product only with PRE, the second step of an outer panel).
// All operands sit in shared memory k-major: P[q][m], Q[q][n].  Warp w =
// (wm, wn), wm = w % 2, wn = w / 2, owns m in [64 wm, 64 wm + 64) and n in
// [32 wn, 32 wn + 32); lane (lx, ly), lx = lane % 4, ly = lane / 4, owns m =
// 64 wm + ly*4 + 32h + q and n = 32 wn + lx*4 + 16g + r (h, g < 2; q, r < 4):
// per q two 16-byte loads of P and two of Q feed 64 FMAs (packed in pairs of
// m).  The inverse is triangular, so the second product stops at q < 32 (wn +
// 1).
// ---------------------------------------------------------------------------
constexpr int kImPanelThreads2 = 128;
// row pitches (floats) of Pk / T2 and of Qk: with 132 and 68 the stores that
// transpose (a quarter warp's 16-byte stores of four rows n = no + 16g + r of
// T2; scalar stores of four rows 4 q4 + c of Pk or Qk) meet 2-way bank
// conflicts instead of 4-way
constexpr int kT2Pitch = 132;
constexpr int kQkPitch = 68;
// Pk (reused for T2 once the left-looking product is done), Q2, Qk
constexpr size_t kImPanelSmemPre = (size_t)(64 * kT2Pitch + 64 * 64 + 64 * kQkPitch) * sizeof(float);
constexpr size_t kImPanelSmem = (size_t)(64 * kT2Pitch + 64 * 64) * sizeof(float);


// acc[h][g][r][p] holds rows (2p, 2p+1) of the thread's 4-row group h,
// column (g, r); one packed two-wide FMA per pair (same rounding as fmaf)
__device__ __forceinline__ void fma_q(float2 (&acc)[2][2][4][2], const float4 (&a)[2], const float4 (&b)[2],
                                      float sign) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 a01 = make_float2(a[h].x, a[h].y), a23 = make_float2(a[h].z, a[h].w);
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float bv = sign * comp(b[g], r);
        const float2 b2 = make_float2(bv, bv);
        acc[h][g][r][0] = __ffma2_rn(a01, b2, acc[h][g][r][0]);
        acc[h][g][r][1] = __ffma2_rn(a23, b2, acc[h][g][r][1]);
      }
  }
}

__device__ __forceinline__ float& el(float2 (&acc)[2][2][4][2], int h, int g, int r, int q) {
  return (q & 1) ? acc[h][g][r][q >> 1].y : acc[h][g][r][q >> 1].x;
}

template <bool PRE>
__global__ void __launch_bounds__(kImPanelThreads2, 3) k_im_panel(DevPlan P, DevState S, int k, int ki, int nch,
                                                               const int32_t* __restrict__ gate) {
  extern __shared__ __align__(16) float pan_smem[];
  float* Pk = pan_smem;                           // PRE: [64 q][kT2Pitch]
  float* T2 = pan_smem;                           // [64 n][kT2Pitch]: the first result, k-major (over Pk)
  float* Q2 = pan_smem + 64 * kT2Pitch;           // [64 q][64 n]: the inverse factor
  float* Qk = Q2 + 64 * 64;                       // PRE: [64 q][kQkPitch]
  if (gate && *gate == 0) return;
  const int per = 2 * nch;
  const int b = (int)(blockIdx.x / (unsigned)per);
  const int task = (int)(blockIdx.x - (unsigned)b * (unsigned)per);
  if (!S.active[b]) return;
  const int ld = P.ndp, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 1, wn = warp >> 1, lx = lane & 3, ly = lane >> 2;
  const int mo = wm * 64 + ly * 4, no = wn * 32 + lx * 4;
  float* __restrict__ A = im_block(P, S, b);
  const bool rows = task < nch;
  const int base = ki + 64 + (rows ? task : task - nch) * 128;  // first row (rows) or column (columns)
  const int mvalid = min(128, ld - base);
  const bool active = wm * 64 < mvalid;
  // operands: contiguous 16-byte words by asynchronous copies, all in flight
  // together; the transposed ones through registers, fully unrolled
  {
    const float* src = reinterpret_cast<const float*>(S.inv) + (size_t)b * 8192 + (rows ? 0 : 4096);
#pragma unroll
    for (int j = 0; j < 64 * 16 / kImPanelThreads2; ++j) {
      const int e = tid + j * kImPanelThreads2;
      cp16(Q2 + 4 * e, src + 4 * e);
    }
  }
  // The transposed operands are read four 16-byte words of one column per
  // four lanes (64-byte segments): lanes (c4 = lane % 4, the column from the
  // rest), word q4 = c4 + 4 (j % 4).
  if (PRE) {
    if (rows) {
      // Pk[q][m] = L(base + m, k + q); Qk[q][n] = U(k + q, ki + n)
#pragma unroll
      for (int j = 0; j < 64 * 32 / kImPanelThreads2; ++j) {
        const int e = tid + j * kImPanelThreads2, q = e >> 5, m4 = e & 31;
        if (4 * m4 < mvalid) cp16(Pk + q * kT2Pitch + 4 * m4, A + (size_t)(k + q) * ld + base + 4 * m4);
      }
#pragma unroll
      for (int j = 0; j < 64 * 16 / kImPanelThreads2; ++j) {
        const int n = (tid >> 2) + 32 * (j >> 2), q4 = (tid & 3) + 4 * (j & 3);
        const float4 v = *reinterpret_cast<const float4*>(A + (size_t)(ki + n) * ld + k + 4 * q4);
        Qk[(4 * q4) * kQkPitch + n] = v.x;
        Qk[(4 * q4 + 1) * kQkPitch + n] = v.y;
        Qk[(4 * q4 + 2) * kQkPitch + n] = v.z;
        Qk[(4 * q4 + 3) * kQkPitch + n] = v.w;
      }
    } else {
      // Pk[q][m] = U(k + q, base + m); Qk[q][n] = L(ki + n, k + q)
#pragma unroll
      for (int j = 0; j < 64 * 16 / kImPanelThreads2; ++j) {
        const int e = tid + j * kImPanelThreads2, q = e >> 4, n4 = e & 15;
        cp16(Qk + q * kQkPitch + 4 * n4, A + (size_t)(k + q) * ld + ki + 4 * n4);
      }
#pragma unroll
      for (int j = 0; j < 128 * 16 / kImPanelThreads2; ++j) {
        const int m = (tid >> 2) + 32 * (j >> 2), q4 = (tid & 3) + 4 * (j & 3);
        if (m < mvalid) {
          const float4 v = *reinterpret_cast<const float4*>(A + (size_t)(base + m) * ld + k + 4 * q4);
          Pk[(4 * q4) * kT2Pitch + m] = v.x;
          Pk[(4 * q4 + 1) * kT2Pitch + m] = v.y;
          Pk[(4 * q4 + 2) * kT2Pitch + m] = v.z;
          Pk[(4 * q4 + 3) * kT2Pitch + m] = v.w;
        }
      }
    }
  }
  // el(acc, h, g, r, q) = T(m = mo + 32h + q, n = no + 16g + r); pairs of q packed
  float2 acc[2][2][4][2];
  if (active) {
    if (rows) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float4 v =
                *reinterpret_cast<const float4*>(A + (size_t)(ki + no + 16 * g + r) * ld + base + mo + 32 * h);
            acc[h][g][r][0] = make_float2(v.x, v.y);
            acc[h][g][r][1] = make_float2(v.z, v.w);
          }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const float4 v =
                *reinterpret_cast<const float4*>(A + (size_t)(base + mo + 32 * h + q) * ld + ki + no + 16 * g);
            el(acc, h, g, 0, q) = v.x;
            el(acc, h, g, 1, q) = v.y;
            el(acc, h, g, 2, q) = v.z;
            el(acc, h, g, 3, q) = v.w;
          }
    }
  }
  cp16_wait_all();
  __syncthreads();
  if (PRE && active) {
#pragma unroll 4
    for (int q = 0; q < 64; ++q) {
      const float4 a[2] = {*reinterpret_cast<const float4*>(Pk + q * kT2Pitch + mo),
                           *reinterpret_cast<const float4*>(Pk + q * kT2Pitch + mo + 32)};
      const float4 bq[2] = {*reinterpret_cast<const float4*>(Qk + q * kQkPitch + no),
                            *reinterpret_cast<const float4*>(Qk + q * kQkPitch + no + 16)};
      fma_q(acc, a, bq, -1.f);
    }
  }
  if (PRE) __syncthreads();  // T2 overwrites Pk
  if (active) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          *reinterpret_cast<float4*>(T2 + (no + 16 * g + r) * kT2Pitch + mo + 32 * h) =
              make_float4(acc[h][g][r][0].x, acc[h][g][r][0].y, acc[h][g][r][1].x, acc[h][g][r][1].y);
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[h][g][r][0] = make_float2(0.f, 0.f);
        acc[h][g][r][1] = make_float2(0.f, 0.f);
      }
  const int qend = 32 * (wn + 1);
#pragma unroll 4
  for (int q = 0; q < qend; ++q) {
    const float4 a[2] = {*reinterpret_cast<const float4*>(T2 + q * kT2Pitch + mo),
                         *reinterpret_cast<const float4*>(T2 + q * kT2Pitch + mo + 32)};
    const float4 bq[2] = {*reinterpret_cast<const float4*>(Q2 + q * 64 + no),
                          *reinterpret_cast<const float4*>(Q2 + q * 64 + no + 16)};
    fma_q(acc, a, bq, 1.f);
  }
  if (rows) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          *reinterpret_cast<float4*>(A + (size_t)(ki + no + 16 * g + r) * ld + base + mo + 32 * h) =
              make_float4(acc[h][g][r][0].x, acc[h][g][r][0].y, acc[h][g][r][1].x, acc[h][g][r][1].y);
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int g = 0; g < 2; ++g)
          *reinterpret_cast<float4*>(A + (size_t)(base + mo + 32 * h + q) * ld + ki + no + 16 * g) =
              make_float4(el(acc, h, g, 0, q), el(acc, h, g, 1, q), el(acc, h, g, 2, q), el(acc, h, g, 3, q));
  }
}

// ---------------------------------------------------------------------------
// Dense forward (unit lower L) and backward (upper U) substitution, one CTA
// per instance, the right-hand side in shared memory.  Per block of 64
// columns: the 64 x 64 triangle is copied to shared memory and solved by one
// warp (two rows per lane, the solved entry broadcast by a shuffle); then every
// thread updates its rows below (above) the block with the block's 64
// entries, reading the matrix columns contiguously across the CTA.  The solve
// reads each instance's block once and is bound by how many loads are in
// flight: at most 40 registers per thread let six CTAs (six instances) run on
// an SM instead of four, which halved its time on the 9,000-bus block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kImSolveThreads, 6) k_im_dsolve(DevPlan P, DevState S,
                                                              const int32_t* __restrict__ gate) {
  extern __shared__ float xs[];                  // [ndp]
  __shared__ float T[64][65];                    // T[c][r]
  if (gate && *gate == 0) return;
  const int b = blockIdx.x;
  if (!S.active[b]) return;
  const int ld = P.ndp, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* __restrict__ A = im_block(P, S, b);
  float* __restrict__ X = reinterpret_cast<float*>(S.x) + ((size_t)(b >> 5) * P.mp + P.s) * kTile + (b & 31);
  for (int r = tid; r < ld; r += kImSolveThreads) xs[r] = X[(size_t)r * kTile];
  __syncthreads();
  for (int kb = 0; kb < ld; kb += 64) {
    for (int e = tid; e < 64 * 64; e += kImSolveThreads) {
      const int c = e >> 6, r = e & 63;
      T[c][r] = A[(size_t)(kb + c) * ld + kb + r];
    }
    __syncthreads();
    if (warp == 0) {
      float v0 = xs[kb + lane], v1 = xs[kb + 32 + lane];
#pragma unroll 8
      for (int c = 0; c < 64; ++c) {
        const float xc = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31);
        if (lane > c) v0 = fmaf(-T[c][lane], xc, v0);
        if (32 + lane > c) v1 = fmaf(-T[c][32 + lane], xc, v1);
      }
      xs[kb + lane] = v0;
      xs[kb + 32 + lane] = v1;
    }
    __syncthreads();
    for (int r = kb + 64 + tid; r < ld; r += kImSolveThreads) {
      float acc = xs[r];
#pragma unroll 8
      for (int c = 0; c < 64; ++c) acc = fmaf(-A[(size_t)(kb + c) * ld + r], xs[kb + c], acc);
      xs[r] = acc;
    }
    __syncthreads();
  }
  for (int kb = ld - 64; kb >= 0; kb -= 64) {
    for (int e = tid; e < 64 * 64; e += kImSolveThreads) {
      const int c = e >> 6, r = e & 63;
      T[c][r] = A[(size_t)(kb + c) * ld + kb + r];
    }
    __syncthreads();
    if (warp == 0) {
      float v0 = xs[kb + lane], v1 = xs[kb + 32 + lane];
#pragma unroll 8
      for (int c = 63; c >= 0; --c) {
        if (c >= 32) {
          if (lane == c - 32) v1 = v1 * (1.f / T[c][c]);
        } else if (lane == c) {
          v0 = v0 * (1.f / T[c][c]);
        }
        const float xc = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31);
        if (lane < c) v0 = fmaf(-T[c][lane], xc, v0);
        if (32 + lane < c) v1 = fmaf(-T[c][32 + lane], xc, v1);
      }
      xs[kb + lane] = v0;
      xs[kb + 32 + lane] = v1;
    }
    __syncthreads();
    for (int r = tid; r < kb; r += kImSolveThreads) {
      float acc = xs[r];
#pragma unroll 8
      for (int c = 0; c < 64; ++c) acc = fmaf(-A[(size_t)(kb + c) * ld + r], xs[kb + c], acc);
      xs[r] = acc;
    }
    __syncthreads();
  }
  for (int r = tid; r < ld; r += kImSolveThreads) X[(size_t)r * kTile] = xs[r];
}

// Padding of the dense block, one CTA per instance: columns nd .. ndp-1 are
// identity columns (contiguous in the instance-major layout), and the
// right-hand side's padding rows m .. m+n_one-1 are zero, so that no stale
// value leaks into real rows during the substitutions.
__global__ void __launch_bounds__(256) k_im_set_ones(DevPlan P, DevState S, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int b = blockIdx.x;
  const int ld = P.ndp;
  float* __restrict__ A = im_block(P, S, b) + (size_t)P.nd * ld;
  const int n = P.n_one * ld;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int c = e / ld, r = e - c * ld;
    A[e] = r == P.nd + c ? 1.f : 0.f;
  }
  float* __restrict__ X = reinterpret_cast<float*>(S.x) + (size_t)(b >> 5) * P.mp * kTile + (b & 31);
  for (int t = threadIdx.x; t < P.n_one; t += blockDim.x) X[(size_t)(P.m + t) * kTile] = 0.f;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn im_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

bool make_dense_im_maps(const DevPlan& P, void* lu, int Bp, DenseImMaps* out) {
  EncodeTiledFn fn = im_encode_fn();
  if (!fn || !lu || Bp <= 0 || Bp % kTile || P.ndp <= 0 || P.ndp % 64) return false;
  const cuuint64_t ld = (cuuint64_t)P.ndp;
  void* base = reinterpret_cast<float*>(lu) + (size_t)P.NS * kTile;
  const cuuint64_t dims[4] = {ld, ld, (cuuint64_t)kTile, (cuuint64_t)(Bp / kTile)};
  const cuuint64_t strides[3] = {ld * 4, ld * ld * 4, (cuuint64_t)P.NLU * kTile * 4};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const cuuint32_t box_a[4] = {(cuuint32_t)kImTile, (cuuint32_t)kImKc, 1, 1};
  const cuuint32_t box_b[4] = {(cuuint32_t)kImKc, (cuuint32_t)kImTile, 1, 1};
  if (fn(&out->a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box_a, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return fn(&out->b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box_b, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_dense_im_factor(const DevPlan& P, const DevState& S, const DenseImMaps& maps, const int32_t* gate,
                            cudaStream_t st, Recorder* rec) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_im_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kImGemmSmem);
    cudaFuncSetAttribute(k_im_diag<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kImDiagSmemPre);
    cudaFuncSetAttribute(k_im_panel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kImPanelSmem);
    cudaFuncSetAttribute(k_im_panel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kImPanelSmemPre);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const unsigned Bp = (unsigned)S.Bp;
  const int ld = P.ndp;
  // the two 64-wide steps of the outer panel at k
  auto outer = [&](int k) {
    NRPF_LAUNCH(rec, K_DENSE_DIAG, st,
                k_im_diag<false><<<Bp, kImDiagThreads, 0, st>>>(P, S, k, k, gate));
    int nr = ld - k - 64;
    if (nr > 0) {
      const int nch = (nr + 127) / 128;
      NRPF_LAUNCH(rec, K_DENSE_PANEL, st,
                  k_im_panel<false><<<Bp * 2 * nch, kImPanelThreads2, kImPanelSmem, st>>>(P, S, k, k, nch, gate));
    }
    if (ld - k < kImOuter) return;  // a last outer panel of 64
    NRPF_LAUNCH(rec, K_DENSE_DIAG, st,
                k_im_diag<true><<<Bp, kImDiagThreads, kImDiagSmemPre, st>>>(P, S, k, k + 64, gate));
    nr = ld - k - kImOuter;
    if (nr > 0) {
      const int nch = (nr + 127) / 128;
      NRPF_LAUNCH(rec, K_DENSE_PANEL, st,
                  k_im_panel<true><<<Bp * 2 * nch, kImPanelThreads2, kImPanelSmemPre, st>>>(P, S, k, k + 64, nch,
                                                                                          gate));
    }
  };
  // block column and row of the outer panel at r0 minus the products of the
  // panels before it
  auto gemm = [&](int r0) {
    const int ntc = (ld - r0 + kImTile - 1) / kImTile;
    NRPF_LAUNCH(rec, K_DENSE_UPDATE, st,
                k_im_gemm<<<Bp * (unsigned)(2 * ntc - 1), kImGemmThreads, kImGemmSmem, st>>>(maps.a, maps.b, P, S,
                                                                                            r0, ntc, gate));
  };
  // Left-looking by outer panels: panel j's block column and row first take
  // the products of panels 0 .. j-1 (depth kj, each entry's subtractions in
  // ascending pivot order, as in the right-looking form), then it is factorised.
  for (int kj = 0; kj < ld; kj += kImOuter) {
    if (kj > 0) gemm(kj);
    outer(kj);
  }
}

void launch_dense_im_set_ones(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                              Recorder* rec) {
  NRPF_LAUNCH(rec, K_ONES, st, k_im_set_ones<<<(unsigned)S.Bp, 256, 0, st>>>(P, S, gate));
}

void launch_dense_im_solve(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                           Recorder* rec) {
  const size_t smem = (size_t)P.ndp * sizeof(float);
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_im_dsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  NRPF_LAUNCH(rec, K_DENSE_SOLVE, st,
              k_im_dsolve<<<(unsigned)S.Bp, kImSolveThreads, smem, st>>>(P, S, gate));
}

}  // namespace nrpf
