// Batched Newton-Raphson kernels (sm_103a).  Every kernel works on tiles of
// kTile = 32 interleaved instances: lane = instance within the tile, so all
// plan indices are warp-uniform (broadcast loads) and all value accesses are
// contiguous across the warp.
#include <cfloat>
#include <cstdint>
#include <vector>

#include "dense_im.h"
#include "device.h"
#include "kernels.h"

namespace nrpf {

namespace {

__device__ __forceinline__ size_t sidx(int tile, int64_t E, int64_t e, int lane) {
  return ((size_t)tile * (size_t)E + (size_t)e) * kTile + lane;
}

__device__ __forceinline__ bool tile_active(const DevState& S, int tile, int lane) {
  return __any_sync(0xffffffffu, S.active[tile * kTile + lane] != 0);
}

// Layout of the dense block inside a tile's LU array.  FP64: element (r, c)
// of the ndp x ndp block at (c * ndp + r) * 32 + lane.  FP32: four
// consecutive rows of a column stay together per lane,
// (c * ndp + (r & ~3)) * 32 + lane * 4 + (r & 3), so a lane reads rows
// r..r+3 (r % 4 == 0) as one 16-byte vector and a warp's access is still one
// contiguous 512-byte segment.  ndp is a multiple of the panel width (>= 4).
template <typename T>
struct DenseGroup {
  static constexpr int G = sizeof(T) == 4 ? 4 : 1;
};

template <typename T>
__device__ __forceinline__ size_t dense_off(int r, int c, int ld, int lane) {
  constexpr int G = DenseGroup<T>::G;
  return ((size_t)c * ld + (r & ~(G - 1))) * kTile + (size_t)lane * G + (r & (G - 1));
}

// offset of LU position p of lane `lane` within its tile's array (positions
// >= NS are in the dense block: interleaved, grouped by four rows in FP32, or
// instance-major when P.dim is set, lane l's block then at NS * 32 + l * ndp^2)
template <typename T>
__device__ __forceinline__ size_t lu_off(const DevPlan& P, int64_t p, int lane) {
  constexpr int G = DenseGroup<T>::G;
  const int64_t NS = P.NS;
  if (p < NS) return (size_t)p * kTile + lane;
  const int64_t q = p - NS;
  if (P.dim) return (size_t)NS * kTile + (size_t)lane * (size_t)P.ndp * (size_t)P.ndp + (size_t)q;
  if (G == 1) return (size_t)p * kTile + lane;
  return (size_t)NS * kTile + (size_t)(q & ~(int64_t)(G - 1)) * kTile + (size_t)lane * G + (size_t)(q & (G - 1));
}

// ---------------------------------------------------------------------------
// Input / output transposes: user [B, n] complex128 <-> interleaved tiles
// (the paper's "transpose to batch" step on the device, Sec. 3.2).
// Block (32, 8): a 32-bus x 32-instance tile through shared memory.
// ---------------------------------------------------------------------------
__global__ void k_load(DevPlan P, DevState S, int B, const double2* __restrict__ sbus,
                       const double2* __restrict__ v0) {
  __shared__ double2 ss[32][33];
  __shared__ double2 sv[32][33];
  const int tile = blockIdx.y;
  const int i0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    int b = tile * kTile + r;
    int i = i0 + tx;
    double2 s = make_double2(0.0, 0.0), v = make_double2(1.0, 0.0);
    if (b < B && i < P.n) {
      s = sbus[(size_t)b * P.n + i];
      v = v0[(size_t)b * P.n + i];
    }
    ss[r][tx] = s;
    sv[r][tx] = v;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    int i = i0 + c;
    if (i >= P.n) continue;
    double2 s = ss[tx][c], v = sv[tx][c];
    size_t o = sidx(tile, P.n, i, tx);
    // a start on the positive real axis (flat start) needs no FP64 sqrt or
    // atan2: |V| is the real part itself and the angle 0
    const bool real = v.y == 0.0 && v.x > 0.0;
    double vm = real ? v.x : sqrt(v.x * v.x + v.y * v.y);
    S.psp[o] = s.x;
    S.qsp[o] = s.y;
    S.vm[o] = vm;
    S.va[o] = real ? 0.0 : atan2(v.y, v.x);
    S.ve[o] = v.x;
    S.vf[o] = v.y;
    S.vinv[o] = 1.0 / vm;
  }
  if (blockIdx.x == 0 && ty == 0) {
    int b = tile * kTile + tx;
    S.iters[b] = 0;
    S.status[b] = NRPF_MAXIT_CODE;
    S.active[b] = b < B ? 1 : 0;
    S.bad[b] = 0;
    S.norm[b] = 0ull;
  }
}

__global__ void k_store(DevPlan P, DevState S, int B, double2* __restrict__ v_out,
                        int32_t* __restrict__ iters, uint8_t* __restrict__ status) {
  __shared__ double2 sv[32][33];
  const int tile = blockIdx.y;
  const int i0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int c = ty; c < 32; c += 8) {
    int i = i0 + c;
    if (i >= P.n) continue;
    size_t o = sidx(tile, P.n, i, tx);
    sv[tx][c] = make_double2(S.ve[o], S.vf[o]);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int b = tile * kTile + r;
    int i = i0 + tx;
    if (b < B && i < P.n) v_out[(size_t)b * P.n + i] = sv[r][tx];
  }
  if (blockIdx.x == 0 && ty == 0) {
    int b = tile * kTile + tx;
    if (b < B) {
      iters[b] = S.iters[b];
      status[b] = (uint8_t)S.status[b];
    }
  }
}

// ---------------------------------------------------------------------------
// Nodal power mismatch (Eq. 1, Alg. 1) fused with the Jacobian refill straight
// into the permuted LU workspace (Sec. 3.1.2, static lookup jmap).
// Rectangular voltages e + jf avoid a sine/cosine per admittance entry:
//   I_i = sum_k Y_ik V_k,  S_i = V_i conj(I_i)
//   W_ik = V_i conj(Y_ik V_k)          (k != i)
//   dP_i/dth_k = Im W_ik, dQ_i/dth_k = -Re W_ik,
//   dP_i/d|V_k| = Re W_ik / |V_k|, dQ_i/d|V_k| = Im W_ik / |V_k|
//   dP_i/dth_i = -Q_i - B_ii |V_i|^2,  dQ_i/dth_i = P_i - G_ii |V_i|^2
//   dP_i/d|V_i| = P_i/|V_i| + G_ii |V_i|, dQ_i/d|V_i| = Q_i/|V_i| - B_ii |V_i|
// Block: 32 lanes x kWarps warps; each warp walks kBusPerWarp buses.
// The right-hand side receives -F at the permuted row of each equation.
// ---------------------------------------------------------------------------
constexpr int kMWarps = 8;
constexpr int kBusPerWarp = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kMWarps) k_mismatch_jac(DevPlan P, DevState S, int jac,
                                                               const int32_t* __restrict__ gate) {
  __shared__ double red[kMWarps][32];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tile = blockIdx.y;
  if (gate && *gate == 0) return;
  T* __restrict__ LU = reinterpret_cast<T*>(S.lu) + (size_t)tile * P.NLU * kTile;
  T* __restrict__ X = reinterpret_cast<T*>(S.x) + (size_t)tile * P.mp * kTile;
  const double* __restrict__ ve = S.ve + (size_t)tile * P.n * kTile;
  const double* __restrict__ vf = S.vf + (size_t)tile * P.n * kTile;
  const double* __restrict__ vinv = S.vinv + (size_t)tile * P.n * kTile;
  // per-instance admittances (interleaved like every per-instance array) or
  // the plan's shared ones; the choice is uniform over the launch
  const double2* __restrict__ Yv = S.yv ? S.yv + (size_t)tile * P.nnzY * kTile + lane : nullptr;
  auto yval = [&](int d, double& G, double& Bv) {
    if (Yv) {
      const double2 y = Yv[(size_t)d * kTile];
      G = y.x;
      Bv = y.y;
    } else {
      G = P.yre[d];
      Bv = P.yim[d];
    }
  };
  double nrm = 0.0;
  const int ibeg = (blockIdx.x * kMWarps + warp) * kBusPerWarp;
  for (int ii = 0; ii < kBusPerWarp; ++ii) {
    const int i = ibeg + ii;
    if (i >= P.n) break;
    const int bt = P.bus_type[i];
    if (bt == 3) continue;
    const double ei = ve[i * kTile + lane], fi = vf[i * kTile + lane];
    double Ir = 0.0, Ii = 0.0;
    const int d0 = P.rowptr[i], d1 = P.rowptr[i + 1];
    for (int d = d0; d < d1; ++d) {
      const int k = P.colidx[d];
      double G, Bv;
      yval(d, G, Bv);
      const double ek = ve[k * kTile + lane], fk = vf[k * kTile + lane];
      const double yr = G * ek - Bv * fk;
      const double yi = G * fk + Bv * ek;
      Ir += yr;
      Ii += yi;
      if (jac && k != i) {
        const int4 jm = reinterpret_cast<const int4*>(P.jmap)[d];
        if (jm.x >= 0) {
          // off-diagonal Jacobian entries, formed in the LU precision (they
          // are stored in it; the mismatch above stays FP64)
          const T Wr = (T)ei * (T)yr + (T)fi * (T)yi;
          const T Wi = (T)fi * (T)yr - (T)ei * (T)yi;
          const T ik = (T)vinv[k * kTile + lane];
          LU[lu_off<T>(P, jm.x, lane)] = Wi;
          if (jm.y >= 0) LU[lu_off<T>(P, jm.y, lane)] = Wr * ik;
          if (jm.z >= 0) LU[lu_off<T>(P, jm.z, lane)] = -Wr;
          if (jm.w >= 0) LU[lu_off<T>(P, jm.w, lane)] = Wi * ik;
        }
      }
    }
    const double Pc = ei * Ir + fi * Ii;
    const double Qc = fi * Ir - ei * Ii;
    const size_t o = (size_t)i * kTile + lane;
    const size_t so = (size_t)tile * P.n * kTile + o;
    const double dP = Pc - S.psp[so];
    double a = fabs(dP);
    X[(size_t)P.rhs_p[i] * kTile + lane] = (T)(-dP);
    if (bt == 1) {
      const double dQ = Qc - S.qsp[so];
      X[(size_t)P.rhs_q[i] * kTile + lane] = (T)(-dQ);
      const double q = fabs(dQ);
      a = (q > a || q != q) ? q : a;
    }
    nrm = (a > nrm || a != a) ? a : nrm;
    if (jac) {
      const int dd = P.ydiag[i];
      const int4 jm = reinterpret_cast<const int4*>(P.jmap)[dd];
      double G, Bv;
      yval(dd, G, Bv);
      const double vm2 = ei * ei + fi * fi;
      const double ivm = vinv[o];
      const double vm = vm2 * ivm;
      LU[lu_off<T>(P, jm.x, lane)] = (T)(-Qc - Bv * vm2);
      if (jm.y >= 0) LU[lu_off<T>(P, jm.y, lane)] = (T)(Pc * ivm + G * vm);
      if (jm.z >= 0) LU[lu_off<T>(P, jm.z, lane)] = (T)(Pc - G * vm2);
      if (jm.w >= 0) LU[lu_off<T>(P, jm.w, lane)] = (T)(Qc * ivm - Bv * vm);
    }
  }
  // NaN -> +inf so that the unsigned-integer max keeps it
  if (!(nrm <= DBL_MAX)) nrm = __longlong_as_double(0x7ff0000000000000ll);
  red[warp][lane] = nrm;
  __syncthreads();
  if (warp == 0) {
    double r = red[0][lane];
    for (int w = 1; w < kMWarps; ++w) r = fmax(r, red[w][lane]);
    atomicMax(&S.norm[tile * kTile + lane], (unsigned long long)__double_as_longlong(r));
  }
}

// Per-instance Ybus values: user [B, nnzY] complex -> interleaved tiles,
// through a 32-entry x 32-instance tile in shared memory (block (32, 8)).
__global__ void k_load_y(int nnzY, int B, const double2* __restrict__ y, double2* __restrict__ yv) {
  __shared__ double2 t[32][33];
  const int d0 = blockIdx.x * 32, tile = blockIdx.y;
  for (int r = threadIdx.y; r < 32; r += 8) {  // r = instance within the tile
    const int b = tile * kTile + r, d = d0 + threadIdx.x;
    t[r][threadIdx.x] = (b < B && d < nnzY) ? y[(size_t)b * nnzY + d] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += 8) {  // c = entry within the block
    const int d = d0 + c;
    if (d < nnzY) yv[((size_t)tile * nnzY + d) * kTile + threadIdx.x] = t[threadIdx.x][c];
  }
}

// Outage cases built on the device: every instance starts from the plan's
// base admittances (interleaved layout), then loses the stamps of its outaged
// branches (repeated indices of one instance count once).
__global__ void k_base_y(DevPlan P, double2* __restrict__ yv, int tiles) {
  const int lane = threadIdx.x;
  const int64_t q = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;  // (tile, entry)
  if (q >= (int64_t)tiles * P.nnzY) return;
  const int d = (int)(q % P.nnzY);
  yv[q * kTile + lane] = make_double2(P.yre[d], P.yim[d]);
}

__global__ void k_outage_y(int nnzY, int B, int k, const int32_t* __restrict__ outages,
                           const int4* __restrict__ bpos, const double* __restrict__ bval, int nbr,
                           double2* __restrict__ yv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double2* y = yv + (size_t)(b / kTile) * nnzY * kTile + (b % kTile);
  for (int a = 0; a < k; ++a) {
    const int e = outages[(size_t)b * k + a];
    if (e < 0 || e >= nbr) continue;
    bool seen = false;
    for (int c = 0; c < a; ++c) seen = seen || outages[(size_t)b * k + c] == e;
    if (seen) continue;
    const int4 ps = bpos[e];
    const double gs = bval[3 * e], bs = bval[3 * e + 1], bh = bval[3 * e + 2];
    y[(size_t)ps.x * kTile].x -= gs;
    y[(size_t)ps.x * kTile].y -= bs + bh;
    y[(size_t)ps.y * kTile].x -= gs;
    y[(size_t)ps.y * kTile].y -= bs + bh;
    y[(size_t)ps.z * kTile].x += gs;
    y[(size_t)ps.z * kTile].y += bs;
    y[(size_t)ps.w * kTile].x += gs;
    y[(size_t)ps.w * kTile].y += bs;
  }
}

// Convergence test and per-instance bookkeeping, one thread per instance.
// it = number of updates performed so far.
__global__ void k_check(DevState S, int Bp) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Bp) return;
  const int it = S.ctl->it, maxit = S.ctl->maxit;
  const double tol = S.ctl->tol;
  int32_t* counter = &S.ctl->cur;
  const double nrm = __longlong_as_double((long long)S.norm[b]);
  S.norm[b] = 0ull;
  if (!S.active[b]) return;
  int keep = 0;
  if (S.bad[b]) {  // the previous step was not finite: it does not count
    S.status[b] = NRPF_FAILED_CODE;
    S.iters[b] = it - 1;
  } else if (!(nrm <= DBL_MAX)) {
    S.status[b] = NRPF_FAILED_CODE;
    S.iters[b] = it;
  } else if (nrm < tol) {
    S.status[b] = NRPF_CONVERGED_CODE;
    S.iters[b] = it;
  } else if (it >= maxit) {
    S.status[b] = NRPF_MAXIT_CODE;
    S.iters[b] = it;
  } else {
    keep = 1;
    S.iters[b] = it + 1;
  }
  S.active[b] = keep;
  const unsigned mask = __ballot_sync(__activemask(), keep);
  if (keep && (threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(counter, __popc(mask));
}

__global__ void k_ctl_init(SolveCtl* c, int maxit, double tol) {
  c->prev = 1;
  c->cur = 0;
  c->it = 0;
  c->maxit = maxit;
  c->tol = tol;
}

// One thread.  The check of this iteration has finished (stream order), so
// cur is final.
__global__ void k_iter_tail(SolveCtl* c, cudaGraphConditionalHandle cond, int graph) {
  const int cur = c->cur;
  c->prev = cur;
  c->cur = 0;
  c->it += 1;
  if (graph) {
    c->graph_iters += 1;
    cudaGraphSetConditional(cond, (cur > 0 && c->it < c->maxit) ? 1u : 0u);
  }
}

// Zero a buffer (16-byte stores, grid-stride), skipped once no instance is
// active.
// Zero the first n16 16-byte words of each of `tiles` arrays spaced stride16
// words apart (the LU arrays of the tiles: whole, or their sparse segments).
__global__ void k_zero16(uint4* __restrict__ p, size_t n16, size_t stride16, int tiles,
                         const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  const size_t total = n16 * (size_t)tiles;
  if (n16 == stride16) {  // the whole per-tile arrays: one contiguous range
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
      p[i] = z;
    return;
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    p[(i / n16) * stride16 + i % n16] = z;
}

// Identity on the padding of the dense block, and zero right-hand side on
// its padding rows (m .. s+ndp-1): no other kernel writes those rows, and a
// stale non-finite value there would leak into real rows as 0 * NaN during
// the backward substitution.
template <typename T>
__global__ void k_set_ones(DevPlan P, DevState S, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int tile = blockIdx.y, lane = threadIdx.x;
  T* LU = reinterpret_cast<T*>(S.lu) + (size_t)tile * P.NLU * kTile;
  T* X = reinterpret_cast<T*>(S.x) + (size_t)tile * P.mp * kTile;
  // padding columns nd .. ndp-1 of the dense block: whole identity columns
  // (the refactorisation does not zero the dense block)
  for (int q = threadIdx.y; q < P.n_one * P.ndp; q += blockDim.y) {
    const int t = q / P.ndp, r = q % P.ndp;
    LU[lu_off<T>(P, P.NS + (int64_t)(P.nd + t) * P.ndp + r, lane)] = (T)(r == P.nd + t ? 1 : 0);
  }
  for (int t = threadIdx.y; t < P.n_one; t += blockDim.y) X[(size_t)(P.m + t) * kTile + lane] = (T)0;
}

// ---------------------------------------------------------------------------
// Sparse left-looking refactorisation, one level of the column schedule
// (Alg. 2 / Alg. 3 stage 1: every column of a level in parallel, one lane per
// instance).  Column j: for each finished column k with U(k,j) != 0, in
// ascending k:  col_j[rows of L(:,k)] -= U(k,j) * L(:,k);  then, for a sparse
// column, L(:,j) /= U(j,j).  Dense-block columns only receive the updates of
// the sparse columns (their Schur complement), and are finished later.
// ---------------------------------------------------------------------------
constexpr int kLWarps = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kLWarps) k_lu_sparse_level(DevPlan P, DevState S, int c0, int c1,
                                                                  const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int ci = c0 + blockIdx.x * kLWarps + threadIdx.y;
  const int tile = blockIdx.y;
  if (ci >= c1) return;
  if (!tile_active(S, tile, lane)) return;
  T* __restrict__ LUb = reinterpret_cast<T*>(S.lu) + (size_t)tile * P.NLU * kTile;  // tile base
  T* __restrict__ LU = LUb + lane;  // sparse positions (< NS): p * 32
  const int j = P.lu_cols[ci];
  const int u0 = P.col_upd_ptr[j], u1 = P.col_upd_ptr[j + 1];
  for (int u = u0; u < u1; ++u) {
    const DevUpd up = P.upd[u];
    const T x = LU[(size_t)up.ukj * kTile];
    const int32_t* __restrict__ dst = P.dst + up.dst_off;
    const T* __restrict__ src = LU + (size_t)up.lsrc * kTile;
    int q = 0;
    for (; q + 4 <= up.llen; q += 4) {
      const size_t o0 = lu_off<T>(P, dst[q], lane), o1 = lu_off<T>(P, dst[q + 1], lane);
      const size_t o2 = lu_off<T>(P, dst[q + 2], lane), o3 = lu_off<T>(P, dst[q + 3], lane);
      const T s0 = src[(size_t)q * kTile], s1 = src[(size_t)(q + 1) * kTile];
      const T s2 = src[(size_t)(q + 2) * kTile], s3 = src[(size_t)(q + 3) * kTile];
      const T a0 = LUb[o0], a1 = LUb[o1];
      const T a2 = LUb[o2], a3 = LUb[o3];
      LUb[o0] = a0 - x * s0;
      LUb[o1] = a1 - x * s1;
      LUb[o2] = a2 - x * s2;
      LUb[o3] = a3 - x * s3;
    }
    for (; q < up.llen; ++q) LUb[lu_off<T>(P, dst[q], lane)] -= x * src[(size_t)q * kTile];
  }
  const int dpj = P.dp[j];
  if (dpj >= 0) {
    const T inv = (T)1 / LU[(size_t)dpj * kTile];
    const int64_t e = P.ce[j];
    for (int64_t p = dpj + 1; p < e; ++p) LU[(size_t)p * kTile] *= inv;
  }
}

// Schur complement of the sparse columns into the dense block, after the
// sparse levels (every U(k, j) is then final).  A warp per (dense column j,
// chunk of 32 dense rows) and tile: the rows live in shared memory (one
// column of 32 rows per lane) while the products L(i, k) U(k, j) of all
// sparse columns k are applied, then go back once.  The warp reads 32 entries
// with one coalesced load and hands them out by shuffles, so the L and U loads
// of eight entries are in flight together.
//   FP64 (bound by the FP64 pipe): each row starts from A(i, j) and takes the
//   subtractions, in the order of the sparse columns as a left-looking
//   column does; no separate subtraction pass.  At most 72 registers: 7 CTAs
//   per SM, the shared-memory limit.
//   FP32 (bound by load latency): each row starts from 0, sums the products
//   and is subtracted from A(i, j) at the end, which keeps the register count
//   and so the warps per SM up (at most 48 registers: ten CTAs per SM).
constexpr int kSchurWarps = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kSchurWarps, sizeof(T) == 8 ? 7 : 10) k_schur(DevPlan P, DevState S, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ T acc[kSchurWarps][32][33];  // [row of the chunk][lane], padded: a row of one lane is read across the warp
  const int lane = threadIdx.x, w = threadIdx.y;
  const int t = blockIdx.x * kSchurWarps + w;
  const int tile = blockIdx.y;
  if (t >= P.n_schur) return;
  if (!tile_active(S, tile, lane)) return;
  T* __restrict__ LUb = reinterpret_cast<T*>(S.lu) + (size_t)tile * P.NLU * kTile;
  const T* __restrict__ LU = LUb + lane;  // sparse positions (< NS): p * 32
  T(*a)[33] = acc[w];
  const int4 task = P.schur_task[t];
  // A(i, j) = J(i, j) where J has an entry, else 0: the block is not zeroed
  // before the refactorisation; the Jacobian fill has written its entries
  const uint32_t jm = P.schur_jmask[t];
  constexpr bool kSeeded = DenseGroup<T>::G != 4;
  if constexpr (kSeeded) {
    const int64_t col = P.NS + (int64_t)task.x * P.ndp + 32 * task.y;
    const int nr = min(32, P.ndp - 32 * task.y);
#pragma unroll 4
    for (int r = 0; r < 32; ++r)
      a[r][lane] = (r < nr && (jm >> r & 1u)) ? LUb[lu_off<T>(P, col + r, lane)] : (T)0;
  } else {
#pragma unroll
    for (int r = 0; r < 32; ++r) a[r][lane] = (T)0;
  }
  for (int eb = task.z; eb < task.w; eb += 32) {
    const int cnt = min(32, task.w - eb);
    const int32_t xl = lane < cnt ? P.schur_ent[eb + lane] : 0;
    const int32_t ul = lane < cnt ? P.schur_u[eb + lane] : 0;
    for (int i = 0; i < cnt; i += 8) {
      T l[8], u[8];
      int r[8];
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        const int32_t x = __shfl_sync(0xffffffffu, xl, i + z);
        const int32_t up = __shfl_sync(0xffffffffu, ul, i + z);
        r[z] = x & 31;
        const bool ok = i + z < cnt;
        l[z] = ok ? LU[(size_t)(x >> 5) * kTile] : (T)0;
        u[z] = ok ? LU[(size_t)up * kTile] : (T)0;
      }
      // entries of one task keep their order (the sparse columns ascending)
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (i + z < cnt) {
          if constexpr (kSeeded) a[r[z]][lane] -= l[z] * u[z];
          else a[r[z]][lane] += l[z] * u[z];
        }
    }
  }
  // every row of the chunk below the padded size is written back
  if constexpr (!kSeeded) {
    if (P.dim) {
      // instance-major block: instance l's 32 rows of column task.x are one
      // contiguous 128-byte line, written by the whole warp (lane = row)
      __syncwarp();
      const int nr = min(32, P.ndp - 32 * task.y);
      const bool jrow = (jm >> lane) & 1u;
      float* __restrict__ col = LUb + (size_t)P.NS * kTile + (size_t)task.x * P.ndp + 32 * task.y + lane;
      const size_t bstride = (size_t)P.ndp * (size_t)P.ndp;
      if (lane < nr) {
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          float* q = col + (size_t)l * bstride;
          const float sum = a[lane][l];
          *q = jrow ? *q - sum : -sum;
        }
      }
      return;
    }
    // FP32 grouped interleaved block: rows 4g .. 4g+3 of the chunk are one
    // 16-byte word per lane; A(i, j) minus the sum
    float4* __restrict__ A4 = reinterpret_cast<float4*>(LUb + (size_t)P.NS * kTile);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int r0 = 32 * task.y + 4 * g;
      if (r0 >= P.ndp) break;
      float4* q = A4 + ((size_t)task.x * P.ndp + r0) * 8 + lane;
      const uint32_t jb = jm >> (4 * g) & 0xFu;
      float4 v = jb ? *q : make_float4(0.f, 0.f, 0.f, 0.f);
      v.x = (jb & 1u) ? v.x - a[4 * g][lane] : -a[4 * g][lane];
      v.y = (jb & 2u) ? v.y - a[4 * g + 1][lane] : -a[4 * g + 1][lane];
      v.z = (jb & 4u) ? v.z - a[4 * g + 2][lane] : -a[4 * g + 2][lane];
      v.w = (jb & 8u) ? v.w - a[4 * g + 3][lane] : -a[4 * g + 3][lane];
      *q = v;
    }
  } else {
    const int64_t col = P.NS + (int64_t)task.x * P.ndp + 32 * task.y;
    const int nr = min(32, P.ndp - 32 * task.y);
#pragma unroll 4
    for (int r = 0; r < nr; ++r) LUb[lu_off<T>(P, col + r, lane)] = a[r][lane];
  }
}

// ---------------------------------------------------------------------------
// Dense trailing block: right-looking blocked LU without pivoting, panel width
// kb, on every instance's ndp x ndp column-major block (Sec. 4.3: the serial
// tail of the column DAG, where few columns remain per level, is handled as
// one dense matrix whose updates are independent multiply-adds).
//   (a) k_dense_diag   : factor the kb x kb diagonal block, store 1/pivots
//   (b) k_dense_panel  : L21 = A21 U11^-1 (rows) and U12 = L11^-1 A12 (cols),
//                        four rows or four columns per thread
//   (c) k_dense_update : A22 -= L21 U12, a register tile per thread (4x4 FP64, 8x8 FP32)
// ---------------------------------------------------------------------------
template <typename T, int KB>
__global__ void k_dense_diag(DevPlan P, DevState S, int k, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int tile = blockIdx.x * blockDim.y + threadIdx.y;
  if (tile * kTile >= S.Bp) return;
  if (!tile_active(S, tile, lane)) return;
  T* __restrict__ A = reinterpret_cast<T*>(S.lu) + ((size_t)tile * P.NLU + P.NS) * kTile;  // dense block
  T* __restrict__ inv = reinterpret_cast<T*>(S.inv) + (size_t)tile * KB * kTile + lane;
  const int ld = P.ndp;
  T D[KB][KB];
#pragma unroll
  for (int c = 0; c < KB; ++c)
#pragma unroll
    for (int r = 0; r < KB; ++r) D[r][c] = A[dense_off<T>(k + r, k + c, ld, lane)];
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    const T ip = (T)1 / D[c][c];
    inv[c * kTile] = ip;
#pragma unroll
    for (int r = c + 1; r < KB; ++r) D[r][c] *= ip;
#pragma unroll
    for (int cc = c + 1; cc < KB; ++cc)
#pragma unroll
      for (int r = c + 1; r < KB; ++r) D[r][cc] -= D[r][c] * D[c][cc];
  }
#pragma unroll
  for (int c = 0; c < KB; ++c)
#pragma unroll
    for (int r = 0; r < KB; ++r) A[dense_off<T>(k + r, k + c, ld, lane)] = D[r][c];
}

// four consecutive rows r .. r+3 (r a multiple of 4) of dense column c for
// this lane: one 16-byte load in the grouped FP32 layout, four loads in FP64
template <typename T>
__device__ __forceinline__ void ld4(const T* __restrict__ A, int r, int c, int ld, int lane, T (&v)[4]) {
  if constexpr (DenseGroup<T>::G == 4) {
    const float4 q = reinterpret_cast<const float4*>(A)[((size_t)c * ld + r) * 8 + lane];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = A[dense_off<T>(r + i, c, ld, lane)];
  }
}

template <typename T>
__device__ __forceinline__ void st4(T* __restrict__ A, int r, int c, int ld, int lane, const T (&v)[4]) {
  if constexpr (DenseGroup<T>::G == 4) {
    reinterpret_cast<float4*>(A)[((size_t)c * ld + r) * 8 + lane] = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) A[dense_off<T>(r + i, c, ld, lane)] = v[i];
  }
}

// y <- L^-1 y for NC columns held in registers, L the NR x NR unit-lower
// block at dense (k, k): column-oriented forward elimination, the
// subtractions into each y[c] in ascending p
template <typename T, int NR, int NC>
__device__ __forceinline__ void unit_lower_solve(const T* __restrict__ A, int k, int ld, int lane, T (&y)[NC][NR]) {
#pragma unroll
  for (int p = 0; p < NR - 1; ++p)
#pragma unroll
    for (int q = (p + 1) / 4; q < NR / 4; ++q) {
      T l[4];
      ld4(A, k + 4 * q, k + p, ld, lane, l);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (4 * q + i > p) {
#pragma unroll
          for (int t = 0; t < NC; ++t) y[t][4 * q + i] -= l[i] * y[t][p];
        }
    }
}

template <typename T, int KB>
__global__ void k_dense_panel(DevPlan P, DevState S, int k, int cend, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int tile = blockIdx.y;
  if (!tile_active(S, tile, lane)) return;
  const int ld = P.ndp;
  const int r0 = k + KB;              // first trailing row/column
  const int ngrp = (ld - r0) / 4;     // groups of four rows (down to ld)
  const int ngc = (cend - r0) / 4;    // groups of four columns (up to cend)
  const int g = blockIdx.x * blockDim.y + threadIdx.y;
  if (g >= ngrp + ngc) return;
  T* __restrict__ A = reinterpret_cast<T*>(S.lu) + ((size_t)tile * P.NLU + P.NS) * kTile;  // dense block
  const T* __restrict__ inv = reinterpret_cast<const T*>(S.inv) + (size_t)tile * KB * kTile + lane;
  if (g < ngrp) {
    // rows i0..i0+3: x U11 = a  (U11 upper, pivots inverted), column by
    // column; the subtractions into x[c] in ascending p
    const int i0 = r0 + 4 * g;
    T x[KB][4];
#pragma unroll
    for (int c = 0; c < KB; ++c) ld4(A, i0, k + c, ld, lane, x[c]);
#pragma unroll
    for (int c = 0; c < KB; ++c) {
#pragma unroll
      for (int q = 0; q < KB / 4; ++q) {
        if (4 * q >= c) break;
        T u[4];
        ld4(A, k + 4 * q, k + c, ld, lane, u);  // U(k+4q .. k+4q+3, k+c)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (4 * q + i < c) {
#pragma unroll
            for (int t = 0; t < 4; ++t) x[c][t] -= x[4 * q + i][t] * u[i];
          }
      }
      const T ip = inv[c * kTile];
#pragma unroll
      for (int t = 0; t < 4; ++t) x[c][t] *= ip;
    }
#pragma unroll
    for (int c = 0; c < KB; ++c) st4(A, i0, k + c, ld, lane, x[c]);
  } else {
    // columns j0..j0+3: L11 y = a  (L11 unit lower)
    const int j0 = r0 + 4 * (g - ngrp);
    T y[4][KB];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int q = 0; q < KB / 4; ++q) {
        T v[4];
        ld4(A, k + 4 * q, j0 + t, ld, lane, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) y[t][4 * q + i] = v[i];
      }
    unit_lower_solve<T, KB, 4>(A, k, ld, lane, y);
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int q = 0; q < KB / 4; ++q) {
        const T v[4] = {y[t][4 * q], y[t][4 * q + 1], y[t][4 * q + 2], y[t][4 * q + 3]};
        st4(A, k + 4 * q, j0 + t, ld, lane, v);
      }
  }
}

// occupancy hint: 128-thread CTAs, at least kUpdMinBlocks resident per SM
// (the 8x8 FP32 tile is latency-bound when registers limit residency)
template <typename T, int TS>
struct UpdOcc {
  static constexpr int value = (sizeof(T) == 4 && TS == 8) ? 2 : 6;
};

// The updated region is the trailing block [r0, ld) x [r0, ld) without its
// part [kend, ld) x [kend, ld): kend = ld for a one-level panel (the whole
// trailing block); kend = the end of the outer panel for an inner step of a
// two-level panel (the outer panel's own columns, and its rows to the right).
template <typename T, int KB, int TS>
__global__ void __launch_bounds__(128, UpdOcc<T, TS>::value) k_dense_update(DevPlan P, DevState S, int k, int kend,
                                                                           int cend, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int tile = blockIdx.y;
  if (!tile_active(S, tile, lane)) return;
  const int ld = P.ndp;
  const int r0 = k + KB;
  const int nbr = (ld - r0) / TS, nbk = (kend - r0) / TS, nbx = (cend - kend) / TS;
  const int n1 = nbr * nbk;  // columns [r0, kend), all rows
  const int t = blockIdx.x * blockDim.y + threadIdx.y;
  if (t >= n1 + nbk * nbx) return;
  int i0, j0;
  if (t < n1) {
    i0 = r0 + TS * (t % nbr);
    j0 = r0 + TS * (t / nbr);
  } else {  // rows [r0, kend), columns [kend, ld)
    i0 = r0 + TS * ((t - n1) % nbk);
    j0 = kend + TS * ((t - n1) / nbk);
  }
  T* __restrict__ Ab = reinterpret_cast<T*>(S.lu) + ((size_t)tile * P.NLU + P.NS) * kTile;  // dense block
  T acc[TS][TS];
  if constexpr (DenseGroup<T>::G == 4 && TS == 8) {
    // FP32, grouped rows: rows r..r+3 of column c for this lane are the
    // float4 at index (c * ld + r) * 8 + lane.  acc2[p][c] holds rows 2p,
    // 2p+1 of column c: one packed two-wide FMA (fma.rn.f32x2) per pair, with
    // -b, which rounds as acc - a b in one step
    float4* __restrict__ A4 = reinterpret_cast<float4*>(Ab);
    float2 acc2[4][TS];
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 v = A4[((size_t)(j0 + c) * ld + i0 + 4 * h) * 8 + lane];
        acc2[2 * h][c] = make_float2(v.x, v.y);
        acc2[2 * h + 1][c] = make_float2(v.z, v.w);
      }
#pragma unroll(KB > 16 ? 2 : KB / 4)
    for (int pp = 0; pp < KB / 4; ++pp) {
      float4 bq[TS];  // rows k+4pp .. k+4pp+3 of columns j0 .. j0+7 (U12)
#pragma unroll
      for (int c = 0; c < TS; ++c) bq[c] = A4[((size_t)(j0 + c) * ld + k + 4 * pp) * 8 + lane];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = 4 * pp + q;
        const float4 a0 = A4[((size_t)(k + p) * ld + i0) * 8 + lane];  // rows i0..i0+7 of column k+p (L21)
        const float4 a1 = A4[((size_t)(k + p) * ld + i0 + 4) * 8 + lane];
        const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                              make_float2(a1.z, a1.w)};
#pragma unroll
        for (int c = 0; c < TS; ++c) {
          const float nb = -(q == 0 ? bq[c].x : q == 1 ? bq[c].y : q == 2 ? bq[c].z : bq[c].w);
          const float2 b2 = make_float2(nb, nb);
#pragma unroll
          for (int r = 0; r < 4; ++r) acc2[r][c] = __ffma2_rn(ap[r], b2, acc2[r][c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        A4[((size_t)(j0 + c) * ld + i0 + 4 * h) * 8 + lane] =
            make_float4(acc2[2 * h][c].x, acc2[2 * h][c].y, acc2[2 * h + 1][c].x, acc2[2 * h + 1][c].y);
  } else if constexpr (DenseGroup<T>::G == 1) {
    // element (r, c) is Ab[(c * ld + r) * 32 + lane]: a column pointer plus a
    // compile-time offset for every access
    T* __restrict__ A = Ab + lane;
    const size_t cstride = (size_t)ld * kTile;
    T* __restrict__ cj = A + (size_t)j0 * cstride + (size_t)i0 * kTile;      // (i0, j0)
    const T* __restrict__ pa = A + (size_t)k * cstride + (size_t)i0 * kTile;  // (i0, k)
    const T* __restrict__ pb = A + (size_t)j0 * cstride + (size_t)k * kTile;  // (k, j0)
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int r = 0; r < TS; ++r) acc[r][c] = cj[c * cstride + r * kTile];
#pragma unroll(KB > 16 ? 8 : KB)
    for (int p = 0; p < KB; ++p) {
      T a[TS], b[TS];
#pragma unroll
      for (int r = 0; r < TS; ++r) a[r] = pa[p * cstride + r * kTile];
#pragma unroll
      for (int c = 0; c < TS; ++c) b[c] = pb[c * cstride + p * kTile];
#pragma unroll
      for (int c = 0; c < TS; ++c)
#pragma unroll
        for (int r = 0; r < TS; ++r) acc[r][c] -= a[r] * b[c];
    }
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int r = 0; r < TS; ++r) cj[c * cstride + r * kTile] = acc[r][c];
  } else {
    // grouped layout with a 4x4 tile (FP32 with panel 4): element by element
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int r = 0; r < TS; ++r) acc[r][c] = Ab[dense_off<T>(i0 + r, j0 + c, ld, lane)];
#pragma unroll(KB > 16 ? 8 : KB)
    for (int p = 0; p < KB; ++p) {
      T a[TS], b[TS];
#pragma unroll
      for (int r = 0; r < TS; ++r) a[r] = Ab[dense_off<T>(i0 + r, k + p, ld, lane)];
#pragma unroll
      for (int c = 0; c < TS; ++c) b[c] = Ab[dense_off<T>(k + p, j0 + c, ld, lane)];
#pragma unroll
      for (int c = 0; c < TS; ++c)
#pragma unroll
        for (int r = 0; r < TS; ++r) acc[r][c] -= a[r] * b[c];
    }
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int r = 0; r < TS; ++r) Ab[dense_off<T>(i0 + r, j0 + c, ld, lane)] = acc[r][c];
  }
}

// ---------------------------------------------------------------------------
// Forward / backward substitution (Sec. 4.3.3).  Row-oriented gathers per
// level instead of the paper's atomicAdd scatter: every row writes only its
// own entry, so the result is deterministic.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fwd_level(DevPlan P, DevState S, int r0, int r1, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int ri = r0 + blockIdx.x * blockDim.y + threadIdx.y;
  const int tile = blockIdx.y;
  if (ri >= r1) return;
  if (!tile_active(S, tile, lane)) return;
  const T* __restrict__ LU = reinterpret_cast<const T*>(S.lu) + (size_t)tile * P.NLU * kTile + lane;
  T* __restrict__ X = reinterpret_cast<T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
  const int i = P.fw_rows[ri];
  T acc = X[(size_t)i * kTile];
  const int e0 = P.fw_ptr[ri], e1 = P.fw_ptr[ri + 1];
  for (int e = e0; e < e1; ++e) acc -= LU[(size_t)P.fw_pos[e] * kTile] * X[(size_t)P.fw_col[e] * kTile];
  X[(size_t)i * kTile] = acc;
}

template <typename T>
__global__ void k_bwd_level(DevPlan P, DevState S, int r0, int r1, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int ri = r0 + blockIdx.x * blockDim.y + threadIdx.y;
  const int tile = blockIdx.y;
  if (ri >= r1) return;
  if (!tile_active(S, tile, lane)) return;
  const T* __restrict__ LU = reinterpret_cast<const T*>(S.lu) + (size_t)tile * P.NLU * kTile + lane;
  T* __restrict__ X = reinterpret_cast<T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
  const int i = P.bw_rows[ri];
  T acc = X[(size_t)i * kTile];
  const int e0 = P.bw_ptr[ri], e1 = P.bw_ptr[ri + 1];
  for (int e = e0; e < e1; ++e) acc -= LU[(size_t)P.bw_pos[e] * kTile] * X[(size_t)P.bw_col[e] * kTile];
  X[(size_t)i * kTile] = acc / LU[(size_t)P.dp[i] * kTile];
}


// Dense block solves with one tile's right-hand side held in shared memory.
// CTA = one tile (32 instances) x kSolveWarps warps.  Forward (unit lower) and
// backward (upper) substitution by blocks of SB columns: warp 0 solves the
// SB x SB diagonal block, then every warp updates its share of the remaining
// rows with SB multiply-adds each (the row updates of a block are independent).
constexpr int kSolveWarps = 8;

template <typename T, int SB, bool SMEM>
__global__ void __launch_bounds__(32 * kSolveWarps) k_dense_solve_smem(DevPlan P, DevState S,
                                                                       const int32_t* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tile = blockIdx.x;
  if (!__syncthreads_or(S.active[tile * kTile + lane])) return;
  const T* __restrict__ Ab = reinterpret_cast<const T*>(S.lu) + ((size_t)tile * P.NLU + P.NS) * kTile;
  const size_t cstride = (size_t)P.ndp * kTile;
  auto A = [&](int r, int c) -> T {
    if constexpr (DenseGroup<T>::G == 1)
      return Ab[(size_t)c * cstride + (size_t)r * kTile + lane];
    else
      return Ab[dense_off<T>(r, c, P.ndp, lane)];
  };
  T* __restrict__ X = reinterpret_cast<T*>(S.x) + ((size_t)tile * P.mp + P.s) * kTile + lane;
  const int ld = P.ndp;
  // the tile's right-hand side: in shared memory when it fits, else in place
  // in global memory (same blocked algorithm, L2-resident per tile)
  T* xs = SMEM ? reinterpret_cast<T*>(smem_raw) : X - lane;  // xs[r * 32 + lane]
  if (SMEM) {
    for (int r = warp; r < ld; r += kSolveWarps) xs[r * kTile + lane] = X[(size_t)r * kTile];
    __syncthreads();
  }
  for (int k0 = 0; k0 < ld; k0 += SB) {
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        const T xc = xs[(k0 + c) * kTile + lane];
#pragma unroll
        for (int r = c + 1; r < SB; ++r)
          xs[(k0 + r) * kTile + lane] -= A(k0 + r, k0 + c) * xc;
      }
    }
    __syncthreads();
    T xb[SB];
#pragma unroll
    for (int c = 0; c < SB; ++c) xb[c] = xs[(k0 + c) * kTile + lane];
    for (int r = k0 + SB + warp; r < ld; r += kSolveWarps) {
      T acc = xs[r * kTile + lane];
#pragma unroll
      for (int c = 0; c < SB; ++c) acc -= A(r, k0 + c) * xb[c];
      xs[r * kTile + lane] = acc;
    }
    __syncthreads();
  }
  for (int k0 = ld - SB; k0 >= 0; k0 -= SB) {
    if (warp == 0) {
#pragma unroll
      for (int c = SB - 1; c >= 0; --c) {
        const T xc = xs[(k0 + c) * kTile + lane] / A(k0 + c, k0 + c);
        xs[(k0 + c) * kTile + lane] = xc;
#pragma unroll
        for (int r = 0; r < c; ++r) xs[(k0 + r) * kTile + lane] -= A(k0 + r, k0 + c) * xc;
      }
    }
    __syncthreads();
    T xb[SB];
#pragma unroll
    for (int c = 0; c < SB; ++c) xb[c] = xs[(k0 + c) * kTile + lane];
    for (int r = warp; r < k0; r += kSolveWarps) {
      T acc = xs[r * kTile + lane];
#pragma unroll
      for (int c = 0; c < SB; ++c) acc -= A(r, k0 + c) * xb[c];
      xs[r * kTile + lane] = acc;
    }
    __syncthreads();
  }
  if (SMEM)
    for (int r = warp; r < ld; r += kSolveWarps) X[(size_t)r * kTile] = xs[r * kTile + lane];
}

// ---------------------------------------------------------------------------
// Voltage update (Sec. 3, step 4): th[PV+PQ] += dx, |V|[PQ] += dx, then the
// rectangular form and 1/|V| for the next mismatch.  Inactive instances keep
// their voltages.  A non-finite step marks the instance failed.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_update(DevPlan P, DevState S, const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x;
  const int tile = blockIdx.y;
  const int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= P.n) return;
  const int b = tile * kTile + lane;
  if (!S.active[b]) return;
  const int bt = P.bus_type[i];
  if (bt == 3) return;
  const T* __restrict__ X = reinterpret_cast<const T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
  const size_t o = sidx(tile, P.n, i, lane);
  const double dth = (double)X[(size_t)P.rhs_p[i] * kTile];
  double va = S.va[o] + dth;
  double vm = S.vm[o];
  bool ok = fabs(dth) <= DBL_MAX;
  if (bt == 1) {
    const double dvm = (double)X[(size_t)P.rhs_q[i] * kTile];
    ok = ok && fabs(dvm) <= DBL_MAX;
    vm += dvm;
  }
  if (!ok) {
    S.bad[b] = 1;
    return;
  }
  double sn, cs;
  sincos(va, &sn, &cs);
  S.va[o] = va;
  S.vm[o] = vm;
  S.ve[o] = vm * cs;
  S.vf[o] = vm * sn;
  S.vinv[o] = 1.0 / vm;
}

// Scatter a user right-hand side [B, m] (J row order) into the permuted rhs,
// and gather the solution back into J column order.
template <typename T>
__global__ void k_rhs_in(DevPlan P, DevState S, int B, const double* __restrict__ rhs) {
  const int lane = threadIdx.x, tile = blockIdx.y;
  const int u = blockIdx.x * blockDim.y + threadIdx.y;
  if (u >= P.m) return;
  const int b = tile * kTile + lane;
  T* X = reinterpret_cast<T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
  X[(size_t)P.unk_pos[u] * kTile] = b < B ? (T)rhs[(size_t)b * P.m + u] : (T)0;
}

template <typename T>
__global__ void k_rhs_out(DevPlan P, DevState S, int B, double* __restrict__ dx) {
  const int lane = threadIdx.x, tile = blockIdx.y;
  const int u = blockIdx.x * blockDim.y + threadIdx.y;
  if (u >= P.m) return;
  const int b = tile * kTile + lane;
  const T* X = reinterpret_cast<const T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
  if (b < B) dx[(size_t)b * P.m + u] = (double)X[(size_t)P.unk_pos[u] * kTile];
}

// F in J row order and the norm, for the mismatch stage entry point.
template <typename T>
__global__ void k_f_out(DevPlan P, DevState S, int B, double* __restrict__ F, double* __restrict__ norm) {
  const int lane = threadIdx.x, tile = blockIdx.y;
  const int u = blockIdx.x * blockDim.y + threadIdx.y;
  const int b = tile * kTile + lane;
  if (b >= B) return;
  if (u < P.m) {
    const T* X = reinterpret_cast<const T*>(S.x) + (size_t)tile * P.mp * kTile + lane;
    F[(size_t)b * P.m + u] = -(double)X[(size_t)P.unk_pos[u] * kTile];
  }
  if (u == 0) norm[b] = __longlong_as_double((long long)S.norm[b]);
}

// LU values of the pattern (CCS order of pf_plan_get_pattern) out to [B, nnz].
template <typename T>
__global__ void k_lu_out(DevPlan P, DevState S, int B, const int64_t* __restrict__ map, int64_t nnz,
                         double* __restrict__ out) {
  const int lane = threadIdx.x, tile = blockIdx.y;
  const int64_t q = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  if (q >= nnz) return;
  const int b = tile * kTile + lane;
  if (b >= B) return;
  const T* LU = reinterpret_cast<const T*>(S.lu) + (size_t)tile * P.NLU * kTile;
  out[(size_t)b * nnz + q] = (double)LU[lu_off<T>(P, map[q], lane)];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launchers (every launch goes through NRPF_LAUNCH for counting and
// optional per-class CUDA-event timing)
// ---------------------------------------------------------------------------
static inline dim3 grid2(int64_t items, int per_block, int tiles) {
  return dim3((unsigned)((items + per_block - 1) / per_block), (unsigned)tiles);
}

void launch_load(const DevPlan& P, const DevState& S, int B, const double* sbus, const double* v0,
                 cudaStream_t st, Recorder* rec) {
  dim3 g((P.n + 31) / 32, S.Bp / kTile);
  NRPF_LAUNCH(rec, K_LOAD, st,
              k_load<<<g, dim3(32, 8), 0, st>>>(P, S, B, reinterpret_cast<const double2*>(sbus),
                                                reinterpret_cast<const double2*>(v0)));
}

void launch_store(const DevPlan& P, const DevState& S, int B, double* v_out, int32_t* iters,
                  uint8_t* status, cudaStream_t st, Recorder* rec) {
  dim3 g((P.n + 31) / 32, S.Bp / kTile);
  NRPF_LAUNCH(rec, K_STORE, st,
              k_store<<<g, dim3(32, 8), 0, st>>>(P, S, B, reinterpret_cast<double2*>(v_out), iters, status));
}

template <typename T>
void launch_mismatch(const DevPlan& P, const DevState& S, int jac, const int32_t* gate, cudaStream_t st,
                     Recorder* rec) {
  dim3 g((P.n + kMWarps * kBusPerWarp - 1) / (kMWarps * kBusPerWarp), S.Bp / kTile);
  NRPF_LAUNCH(rec, K_MISMATCH, st, k_mismatch_jac<T><<<g, dim3(32, kMWarps), 0, st>>>(P, S, jac, gate));
}

void launch_load_y(const DevPlan& P, const DevState& S, int B, const double* y, cudaStream_t st, Recorder* rec) {
  dim3 g((P.nnzY + 31) / 32, S.Bp / kTile);
  NRPF_LAUNCH(rec, K_LOAD, st,
              k_load_y<<<g, dim3(32, 8), 0, st>>>(P.nnzY, B, reinterpret_cast<const double2*>(y),
                                                  const_cast<double2*>(S.yv)));
}

void launch_outage_y(const DevPlan& P, const DevState& S, int B, const int32_t* outages, int k, const int4* bpos,
                     const double* bval, int nbr, cudaStream_t st, Recorder* rec) {
  const int tiles = S.Bp / kTile;
  double2* yv = const_cast<double2*>(S.yv);
  NRPF_LAUNCH(rec, K_LOAD, st,
              k_base_y<<<grid2((int64_t)tiles * P.nnzY, 8, 1), dim3(32, 8), 0, st>>>(P, yv, tiles));
  if (k > 0)
    NRPF_LAUNCH(rec, K_LOAD, st,
                k_outage_y<<<(B + 127) / 128, 128, 0, st>>>(P.nnzY, B, k, outages, bpos, bval, nbr, yv));
}

void launch_ctl_init(const DevState& S, int maxit, double tol, cudaStream_t st, Recorder* rec) {
  NRPF_LAUNCH(rec, K_AUX, st, k_ctl_init<<<1, 1, 0, st>>>(S.ctl, maxit, tol));
}

void launch_check(const DevState& S, cudaStream_t st, Recorder* rec) {
  NRPF_LAUNCH(rec, K_CHECK, st, k_check<<<(S.Bp + 255) / 256, 256, 0, st>>>(S, S.Bp));
}

void launch_iter_tail(const DevState& S, cudaGraphConditionalHandle cond, int graph, cudaStream_t st,
                      Recorder* rec) {
  NRPF_LAUNCH(rec, K_AUX, st, k_iter_tail<<<1, 1, 0, st>>>(S.ctl, cond, graph));
}

template <typename T>
void launch_prepare_lu(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                       Recorder* rec, bool whole) {
  // per tile, NLU * 32 values; the sparse segments are the first NS * 32
  // (both multiples of 128 bytes).  The dense block is left alone unless
  // `whole`: the Schur tasks then write every position of it.
  const size_t stride16 = (size_t)P.NLU * kTile * sizeof(T) / 16;
  const size_t n16 = (whole || P.nd == 0) ? stride16 : (size_t)P.NS * kTile * sizeof(T) / 16;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  NRPF_LAUNCH(rec, K_ZERO, st,
              k_zero16<<<sms * 8, 256, 0, st>>>(reinterpret_cast<uint4*>(S.lu), n16, stride16, S.Bp / kTile, gate));
  if (P.n_one > 0) {
    if (sizeof(T) == 4 && P.dim)
      launch_dense_im_set_ones(P, S, gate, st, rec);
    else
      NRPF_LAUNCH(rec, K_ONES, st, k_set_ones<T><<<dim3(1, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, gate));
  }
}

// one panel step of width KB at column k.  The column part of the panel
// covers columns < cend; the update covers the trailing block's columns
// [r0, kend) and, for rows [r0, kend), columns [kend, cend)
// (kend = cend = ld: the whole trailing block).
template <typename T, int KB>
static void launch_dense_step(const DevPlan& P, const DevState& S, int k, int kend, int cend, const int32_t* gate,
                              cudaStream_t st, Recorder* rec) {
  const int tiles = S.Bp / kTile;
  const int rows = P.ndp - k - KB;
  NRPF_LAUNCH(rec, K_DENSE_DIAG, st,
              k_dense_diag<T, KB><<<(tiles + 3) / 4, dim3(32, 4), 0, st>>>(P, S, k, gate));
  if (rows > 0) {
    const int cols = cend - k - KB;
    NRPF_LAUNCH(rec, K_DENSE_PANEL, st,
                k_dense_panel<T, KB><<<grid2(rows / 4 + cols / 4, 4, tiles), dim3(32, 4), 0, st>>>(P, S, k, cend,
                                                                                                  gate));
    // register tile: 4 x 4 for FP64 (the FP64 pipe is the bound), 8 x 8 for
    // FP32 (halves the loads per multiply-add; FP32 is load-bound)
    constexpr int TS = (sizeof(T) == 4 && KB >= 8) ? 8 : 4;
    const int64_t nk = (kend - k - KB) / TS;
    const int64_t ntiles = (rows / TS) * nk + nk * ((cend - kend) / TS);
    if (ntiles > 0) {
      NRPF_LAUNCH(rec, K_DENSE_UPDATE, st,
                  k_dense_update<T, KB, TS><<<grid2(ntiles, 4, tiles), dim3(32, 4), 0, st>>>(P, S, k, kend, cend,
                                                                                            gate));
    }
  }
}

// Outer panel of width KBO (two-level blocking): 16-wide steps factorise the
// outer panel's columns and its rows to the right (U12), each step updating
// only that L-shaped region; then one trailing update of depth KBO (one pass
// over the trailing block per KBO columns instead of per 16).
template <typename T, int KBO>
static void launch_dense_outer(const DevPlan& P, const DevState& S, int k, const int32_t* gate, cudaStream_t st,
                               Recorder* rec) {
  const int tiles = S.Bp / kTile;
  for (int ki = k; ki < k + KBO; ki += 16) launch_dense_step<T, 16>(P, S, ki, k + KBO, P.ndp, gate, st, rec);
  const int rest = P.ndp - k - KBO;
  if (rest > 0) {
    constexpr int TS = sizeof(T) == 4 ? 8 : 4;
    NRPF_LAUNCH(rec, K_DENSE_UPDATE, st,
                k_dense_update<T, KBO, TS><<<grid2((int64_t)(rest / TS) * (rest / TS), 4, tiles), dim3(32, 4), 0,
                                             st>>>(P, S, k, P.ndp, P.ndp, gate));
  }
}

template <typename T>
void launch_factor(const DevPlan& P, const DevState& S, const std::vector<int32_t>& lvl_ptr,
                   const int32_t* gate, cudaStream_t st, Recorder* rec) {
  const int tiles = S.Bp / kTile;
  for (size_t l = 0; l + 1 < lvl_ptr.size(); ++l) {
    int c0 = lvl_ptr[l], c1 = lvl_ptr[l + 1];
    if (c1 <= c0) continue;
    NRPF_LAUNCH(rec, K_LU_SPARSE, st,
                k_lu_sparse_level<T><<<grid2(c1 - c0, kLWarps, tiles), dim3(32, kLWarps), 0, st>>>(P, S, c0, c1,
                                                                                                  gate));
  }
  if (P.n_schur > 0)
    NRPF_LAUNCH(rec, K_SCHUR, st,
                k_schur<T><<<grid2(P.n_schur, kSchurWarps, tiles), dim3(32, kSchurWarps), 0, st>>>(P, S, gate));
  if constexpr (sizeof(T) == 4) {
    if (P.dim) {
      if (P.ndp > 0) launch_dense_im_factor(P, S, *reinterpret_cast<const DenseImMaps*>(S.im_maps), gate, st, rec);
      return;
    }
  }
  for (int k = 0; k < P.ndp; k += P.kb) {
    if (P.kb == 4) launch_dense_step<T, 4>(P, S, k, P.ndp, P.ndp, gate, st, rec);
    else if (P.kb == 8) launch_dense_step<T, 8>(P, S, k, P.ndp, P.ndp, gate, st, rec);
    else if (P.kb == 16) launch_dense_step<T, 16>(P, S, k, P.ndp, P.ndp, gate, st, rec);
    else if (P.kb == 32) launch_dense_outer<T, 32>(P, S, k, gate, st, rec);
    else launch_dense_outer<T, 64>(P, S, k, gate, st, rec);
  }
}

// Dense solve with the tile's right-hand side in shared memory, when it fits.
constexpr size_t kSolveSmemMax = 200 * 1024;

template <typename T, int SB>
static void launch_dense_solve_smem(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                                    Recorder* rec, size_t smem) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_dense_solve_smem<T, SB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSolveSmemMax);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  if (smem <= kSolveSmemMax)
    NRPF_LAUNCH(rec, K_DENSE_SOLVE, st,
                k_dense_solve_smem<T, SB, true><<<S.Bp / kTile, dim3(32, kSolveWarps), smem, st>>>(P, S, gate));
  else
    NRPF_LAUNCH(rec, K_DENSE_SOLVE, st,
                k_dense_solve_smem<T, SB, false><<<S.Bp / kTile, dim3(32, kSolveWarps), 0, st>>>(P, S, gate));
}

template <typename T>
void launch_solve(const DevPlan& P, const DevState& S, const std::vector<int32_t>& fw_lvl,
                  const std::vector<int32_t>& bw_lvl, const int32_t* gate, cudaStream_t st, Recorder* rec) {
  const int tiles = S.Bp / kTile;
  for (size_t l = 0; l + 1 < fw_lvl.size(); ++l) {
    int r0 = fw_lvl[l], r1 = fw_lvl[l + 1];
    if (r1 > r0)
      NRPF_LAUNCH(rec, K_FWD, st,
                  k_fwd_level<T><<<grid2(r1 - r0, 4, tiles), dim3(32, 4), 0, st>>>(P, S, r0, r1, gate));
  }
  if (sizeof(T) == 4 && P.dim) {
    if (P.ndp > 0) launch_dense_im_solve(P, S, gate, st, rec);
  } else if (P.ndp > 0) {
    const size_t smem = (size_t)P.ndp * kTile * sizeof(T);
    if (P.ndp % 8 == 0)
      launch_dense_solve_smem<T, 8>(P, S, gate, st, rec, smem);
    else
      launch_dense_solve_smem<T, 4>(P, S, gate, st, rec, smem);
  }
  for (size_t l = 0; l + 1 < bw_lvl.size(); ++l) {
    int r0 = bw_lvl[l], r1 = bw_lvl[l + 1];
    if (r1 > r0)
      NRPF_LAUNCH(rec, K_BWD, st,
                  k_bwd_level<T><<<grid2(r1 - r0, 4, tiles), dim3(32, 4), 0, st>>>(P, S, r0, r1, gate));
  }
}

template <typename T>
void launch_update(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st, Recorder* rec) {
  NRPF_LAUNCH(rec, K_UPDATE, st, k_update<T><<<grid2(P.n, 8, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, gate));
}

template <typename T>
void launch_rhs_in(const DevPlan& P, const DevState& S, int B, const double* rhs, cudaStream_t st) {
  cudaMemsetAsync(S.x, 0, (size_t)P.mp * S.Bp * sizeof(T), st);
  if (P.m > 0) k_rhs_in<T><<<grid2(P.m, 8, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, B, rhs);
}

template <typename T>
void launch_rhs_out(const DevPlan& P, const DevState& S, int B, double* dx, cudaStream_t st) {
  if (P.m > 0) k_rhs_out<T><<<grid2(P.m, 8, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, B, dx);
}

template <typename T>
void launch_f_out(const DevPlan& P, const DevState& S, int B, double* F, double* norm, cudaStream_t st) {
  k_f_out<T><<<grid2(P.m > 0 ? P.m : 1, 8, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, B, F, norm);
}

template <typename T>
void launch_lu_out(const DevPlan& P, const DevState& S, int B, const int64_t* map, int64_t nnz, double* out,
                   cudaStream_t st) {
  if (nnz > 0) k_lu_out<T><<<grid2(nnz, 8, S.Bp / kTile), dim3(32, 8), 0, st>>>(P, S, B, map, nnz, out);
}

#define NRPF_INST(T)                                                                                          \
  template void launch_mismatch<T>(const DevPlan&, const DevState&, int, const int32_t*, cudaStream_t,       \
                                   Recorder*);                                                               \
  template void launch_prepare_lu<T>(const DevPlan&, const DevState&, const int32_t*, cudaStream_t,          \
                                     Recorder*, bool);                                                       \
  template void launch_factor<T>(const DevPlan&, const DevState&, const std::vector<int32_t>&,               \
                                 const int32_t*, cudaStream_t, Recorder*);                                   \
  template void launch_solve<T>(const DevPlan&, const DevState&, const std::vector<int32_t>&,                \
                                const std::vector<int32_t>&, const int32_t*, cudaStream_t, Recorder*);       \
  template void launch_update<T>(const DevPlan&, const DevState&, const int32_t*, cudaStream_t, Recorder*);  \
  template void launch_rhs_in<T>(const DevPlan&, const DevState&, int, const double*, cudaStream_t);         \
  template void launch_rhs_out<T>(const DevPlan&, const DevState&, int, double*, cudaStream_t);              \
  template void launch_f_out<T>(const DevPlan&, const DevState&, int, double*, double*, cudaStream_t);       \
  template void launch_lu_out<T>(const DevPlan&, const DevState&, int, const int64_t*, int64_t, double*,     \
                                 cudaStream_t);

NRPF_INST(double)
NRPF_INST(float)

}  // namespace nrpf
