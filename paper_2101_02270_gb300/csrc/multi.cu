// Uneven batching: grids of different sizes and patterns (one plan each) and
// different scenario counts solved by ONE persistent kernel.  Work items are
// (plan, tile of up to S scenarios), sorted by decreasing work; every CTA
// pulls items from an atomic counter and runs the whole Newton loop of its
// item (Sec. 3 steps 1-4).  Lane l of a warp serves scenario l % S of the
// item as worker warp * (32 / S) + l / S: the workers split the buses of the
// mismatch and update, the columns of each refactor level and the rows of
// each FS/BS level, with a CTA barrier between phases.  Element e of
// scenario s sits at e * S + s.  The item's state (voltages, injections,
// right-hand side, LU values) lives in shared memory when it fits the
// launch's dynamic shared memory, otherwise in a private global slot.  The
// memset of the counter and the kernel are captured once in a CUDA graph and
// replayed.  Plans must have no dense block (create them with dense_frac >= 1).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nrpf.h"
#include "handle.h"
#include "kernels.h"

namespace {

using nrpf::DevPlan;
using nrpf::DevUpd;
using nrpf::kTile;

constexpr int kMaxWarps = 16;
// dynamic shared memory a CTA may use for its item's state
constexpr size_t kMultiSmemMax = 200 * 1024;

struct Item {
  int32_t plan;  // plan index
  int32_t b0;    // first scenario of the tile within the plan's batch
  int32_t nb;    // scenarios in the tile (<= S)
  int32_t smem;  // 1: the state fits the launch's shared memory
};

struct DevMulti {
  const DevPlan* plans;     // [k]
  const int64_t* in_off;    // [k] first complex element of plan f in sbus/v0/v_out
  const int64_t* inst_off;  // [k] first instance of plan f in iters/status
  const Item* items;        // [n_items]
  int n_items;
  int* next;                // work counter (zeroed before every launch)
  char* ws;                 // slots
  size_t slot_bytes;
  int log_s;                // S = 1 << log_s scenarios per item
};

// Bytes of an item's state for S scenarios: 7 FP64 bus arrays, then the
// right-hand side and the LU values in the LU precision.
inline size_t state_bytes(const nrpf::HostPlan& h, int S, size_t w) {
  const size_t b = (size_t)S * ((size_t)7 * h.n * 8 + (size_t)(h.s + h.ndp + h.NLU) * w);
  return (b + 255) / 256 * 256;
}

// One item's whole Newton loop.  base: its state (shared or global memory).
template <typename T>
__device__ __forceinline__ void run_item(const DevMulti& M, const Item& it, char* base, const double2* __restrict__ sbus,
                                         const double2* __restrict__ v0, double tol, int maxit,
                                         double2* __restrict__ vout, int32_t* __restrict__ iters_out,
                                         uint8_t* __restrict__ status_out, double* s_red, int* s_bad) {
  const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
  const int tid = warp * 32 + lane, nthr = 32 * W;
  const int ls = M.log_s, S = 1 << ls;
  const int sc = lane & (S - 1);                       // scenario of this lane
  const int wk = warp * (32 >> ls) + (lane >> ls);     // worker index
  const int nw = W * (32 >> ls);                       // workers per scenario
  const DevPlan& P = M.plans[it.plan];
  const int n = P.n;
  double* vm = reinterpret_cast<double*>(base);
  double* va = vm + (size_t)n * S;
  double* ve = va + (size_t)n * S;
  double* vf = ve + (size_t)n * S;
  double* vinv = vf + (size_t)n * S;
  double* psp = vinv + (size_t)n * S;
  double* qsp = psp + (size_t)n * S;
  T* X = reinterpret_cast<T*>(qsp + (size_t)n * S);
  T* LU = X + (size_t)P.mp * S;
  auto at = [&](int64_t e) -> int64_t { return (e << ls) + sc; };
  const bool valid = sc < it.nb;
  const int64_t gbase = M.in_off[it.plan] + (int64_t)(it.b0 + sc) * n;
  // ---- load (user layout -> item layout) ----
  for (int i = wk; i < n; i += nw) {
    double2 s = make_double2(0.0, 0.0), v = make_double2(1.0, 0.0);
    if (valid) {
      s = sbus[gbase + i];
      v = v0[gbase + i];
    }
    // a start on the positive real axis (flat start) needs no FP64 sqrt or
    // atan2
    const bool real = v.y == 0.0 && v.x > 0.0;
    const double mag = real ? v.x : sqrt(v.x * v.x + v.y * v.y);
    const int64_t o = at(i);
    psp[o] = s.x;
    qsp[o] = s.y;
    vm[o] = mag;
    va[o] = real ? 0.0 : atan2(v.y, v.x);
    ve[o] = v.x;
    vf[o] = v.y;
    vinv[o] = 1.0 / mag;
  }
  if (tid < 32) s_bad[tid] = 0;
  int act = valid ? 1 : 0, my_iters = 0, my_status = NRPF_MAXIT_CODE;
  __syncthreads();
  for (int itn = 0;; ++itn) {
    // ---- zero the LU values, then mismatch + Jacobian (Alg. 1, Sec. 3.1.2) ----
    for (int64_t e = tid; e < P.NLU * S; e += nthr) LU[e] = (T)0;
    __syncthreads();
    double nrm = 0.0;
    for (int i = wk; i < n; i += nw) {
      const int bt = P.bus_type[i];
      if (bt == 3) continue;
      const double ei = ve[at(i)], fi = vf[at(i)];
      double Ir = 0.0, Ii = 0.0;
      for (int d = P.rowptr[i]; d < P.rowptr[i + 1]; ++d) {
        const int k = P.colidx[d];
        const double G = P.yre[d], Bv = P.yim[d];
        const double ek = ve[at(k)], fk = vf[at(k)];
        const double yr = G * ek - Bv * fk, yi = G * fk + Bv * ek;
        Ir += yr;
        Ii += yi;
        if (k != i) {
          const int4 jm = reinterpret_cast<const int4*>(P.jmap)[d];
          if (jm.x >= 0) {
            // off-diagonal Jacobian entries in the LU precision (stored in
            // it); the mismatch stays FP64
            const T Wr = (T)ei * (T)yr + (T)fi * (T)yi, Wi = (T)fi * (T)yr - (T)ei * (T)yi;
            const T ik = (T)vinv[at(k)];
            LU[at(jm.x)] = Wi;
            if (jm.y >= 0) LU[at(jm.y)] = Wr * ik;
            if (jm.z >= 0) LU[at(jm.z)] = -Wr;
            if (jm.w >= 0) LU[at(jm.w)] = Wi * ik;
          }
        }
      }
      const double Pc = ei * Ir + fi * Ii, Qc = fi * Ir - ei * Ii;
      const int64_t o = at(i);
      const double dP = Pc - psp[o];
      double a = fabs(dP);
      X[at(P.rhs_p[i])] = (T)(-dP);
      if (bt == 1) {
        const double dQ = Qc - qsp[o];
        X[at(P.rhs_q[i])] = (T)(-dQ);
        const double q = fabs(dQ);
        a = (q > a || q != q) ? q : a;
      }
      nrm = (a > nrm || a != a) ? a : nrm;
      const int dd = P.ydiag[i];
      const int4 jm = reinterpret_cast<const int4*>(P.jmap)[dd];
      const double G = P.yre[dd], Bv = P.yim[dd];
      const double vm2 = ei * ei + fi * fi, ivm = vinv[o], mg = vm2 * ivm;
      LU[at(jm.x)] = (T)(-Qc - Bv * vm2);
      if (jm.y >= 0) LU[at(jm.y)] = (T)(Pc * ivm + G * mg);
      if (jm.z >= 0) LU[at(jm.z)] = (T)(Pc - G * vm2);
      if (jm.w >= 0) LU[at(jm.w)] = (T)(Qc * ivm - Bv * mg);
    }
    if (!(nrm <= DBL_MAX)) nrm = __longlong_as_double(0x7ff0000000000000ll);
    // max over the workers of each scenario: within the warp (lanes of the
    // same scenario differ in the bits above log S), then across warps
    for (int off = S; off < 32; off <<= 1) {
      const double o2 = __shfl_xor_sync(0xffffffffu, nrm, off);
      nrm = (o2 > nrm || o2 != o2) ? o2 : nrm;
    }
    if (lane < S) s_red[warp * 32 + lane] = nrm;
    __syncthreads();
    // ---- convergence test (every thread computes its scenario's outcome) ----
    double tot = s_red[sc];
    for (int w = 1; w < W; ++w) {
      const double o2 = s_red[w * 32 + sc];
      tot = (o2 > tot || o2 != o2) ? o2 : tot;
    }
    if (act) {
      if (s_bad[sc]) {
        my_status = NRPF_FAILED_CODE;
        my_iters = itn - 1;
        act = 0;
      } else if (!(tot <= DBL_MAX)) {
        my_status = NRPF_FAILED_CODE;
        my_iters = itn;
        act = 0;
      } else if (tot < tol) {
        my_status = NRPF_CONVERGED_CODE;
        my_iters = itn;
        act = 0;
      } else if (itn >= maxit) {
        my_status = NRPF_MAXIT_CODE;
        my_iters = itn;
        act = 0;
      } else {
        my_iters = itn + 1;
      }
    }
    if (!__syncthreads_or(act)) break;
    // ---- sparse left-looking refactor, level by level ----
    for (int l = 0; l < P.n_lu_lvl; ++l) {
      const int c0 = P.lu_lvl_ptr[l], c1 = P.lu_lvl_ptr[l + 1];
      for (int ci = c0 + wk; ci < c1; ci += nw) {
        const int j = P.lu_cols[ci];
        for (int u = P.col_upd_ptr[j]; u < P.col_upd_ptr[j + 1]; ++u) {
          const DevUpd up = P.upd[u];
          const T x = LU[at(up.ukj)];
          const int32_t* dst = P.dst + up.dst_off;
          for (int q = 0; q < up.llen; ++q) LU[at(dst[q])] -= x * LU[at(up.lsrc + q)];
        }
        const int dpj = P.dp[j];
        if (dpj >= 0) {
          const T inv = (T)1 / LU[at(dpj)];
          for (int64_t p = dpj + 1; p < P.ce[j]; ++p) LU[at(p)] *= inv;
        }
      }
      __syncthreads();
    }
    // ---- forward / backward substitution ----
    for (int l = 0; l < P.n_fw_lvl; ++l) {
      const int r0 = P.fw_lvl_ptr[l], r1 = P.fw_lvl_ptr[l + 1];
      for (int ri = r0 + wk; ri < r1; ri += nw) {
        const int i = P.fw_rows[ri];
        T acc = X[at(i)];
        for (int e = P.fw_ptr[ri]; e < P.fw_ptr[ri + 1]; ++e) acc -= LU[at(P.fw_pos[e])] * X[at(P.fw_col[e])];
        X[at(i)] = acc;
      }
      __syncthreads();
    }
    for (int l = 0; l < P.n_bw_lvl; ++l) {
      const int r0 = P.bw_lvl_ptr[l], r1 = P.bw_lvl_ptr[l + 1];
      for (int ri = r0 + wk; ri < r1; ri += nw) {
        const int i = P.bw_rows[ri];
        T acc = X[at(i)];
        for (int e = P.bw_ptr[ri]; e < P.bw_ptr[ri + 1]; ++e) acc -= LU[at(P.bw_pos[e])] * X[at(P.bw_col[e])];
        X[at(i)] = acc / LU[at(P.dp[i])];
      }
      __syncthreads();
    }
    // ---- voltage update (Sec. 3 step 4) ----
    if (act) {
      for (int i = wk; i < n; i += nw) {
        const int bt = P.bus_type[i];
        if (bt == 3) continue;
        const int64_t o = at(i);
        const double dth = (double)X[at(P.rhs_p[i])];
        double a = va[o] + dth, g = vm[o];
        bool ok = fabs(dth) <= DBL_MAX;
        if (bt == 1) {
          const double dv = (double)X[at(P.rhs_q[i])];
          ok = ok && fabs(dv) <= DBL_MAX;
          g += dv;
        }
        if (!ok) {
          s_bad[sc] = 1;
          continue;
        }
        double sn, cs;
        sincos(a, &sn, &cs);
        va[o] = a;
        vm[o] = g;
        ve[o] = g * cs;
        vf[o] = g * sn;
        vinv[o] = 1.0 / g;
      }
    }
    __syncthreads();
  }
  // ---- store ----
  if (valid) {
    for (int i = wk; i < n; i += nw) vout[gbase + i] = make_double2(ve[at(i)], vf[at(i)]);
    if (wk == 0) {
      const int64_t g = M.inst_off[it.plan] + it.b0 + sc;
      iters_out[g] = my_iters;
      status_out[g] = (uint8_t)my_status;
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(32 * kMaxWarps) k_multi(DevMulti M, const double2* __restrict__ sbus,
                                                          const double2* __restrict__ v0, double tol, int maxit,
                                                          double2* __restrict__ vout, int32_t* __restrict__ iters_out,
                                                          uint8_t* __restrict__ status_out) {
  extern __shared__ __align__(16) unsigned char msm[];
  __shared__ int s_item;
  __shared__ double s_red[kMaxWarps * 32];
  __shared__ int s_bad[32];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  char* slot = M.ws + (size_t)blockIdx.x * M.slot_bytes;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(M.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= M.n_items) break;
    const Item it = M.items[item];
    if (it.smem)
      run_item<T>(M, it, reinterpret_cast<char*>(msm), sbus, v0, tol, maxit, vout, iters_out, status_out, s_red,
                  s_bad);
    else
      run_item<T>(M, it, slot, sbus, v0, tol, maxit, vout, iters_out, status_out, s_red, s_bad);
  }
}

}  // namespace

struct pf_multi {
  int k = 0;
  int lu_precision = NRPF_LU_FP64;
  int device = 0;
  int warps = 4;
  int blocks_per_sm = 4;
  int scen = kTile;       // scenarios per item (a power of two, <= 32)
  int use_smem = 0;       // 1: items whose state fits kMultiSmemMax run in shared memory
  size_t smem_bytes = 0;  // dynamic shared memory per CTA (largest state of an item in it)
  int smem_items = 0;
  int sms = 0;
  int64_t total_instances = 0;
  size_t slot_bytes = 0;
  std::vector<const pf_plan*> plans;
  std::vector<int32_t> batch;
  std::vector<void*> allocs;
  void* d_items = nullptr;
  size_t items_cap = 0;
  DevMulti dm{};
  void* ws = nullptr;
  size_t ws_slots = 0;
  // captured graph of (memset counter, kernel) for the last argument set
  cudaGraphExec_t gexec = nullptr;
  const void* g_args[7] = {};
  double g_tol = -1;
  int g_maxit = -1, g_warps = -1, g_bps = -1;
  cudaStream_t g_stream = nullptr;
};

namespace {

int ensure_slots(pf_multi* mp, size_t slots) {
  if (slots <= mp->ws_slots && mp->dm.slot_bytes == mp->slot_bytes) return NRPF_OK;
  if (mp->ws) {
    cudaDeviceSynchronize();
    cudaFree(mp->ws);
    mp->ws = nullptr;
    mp->ws_slots = 0;
  }
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, std::max<size_t>(slots * mp->slot_bytes, 256));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
  mp->ws = d;
  mp->ws_slots = slots;
  mp->dm.ws = reinterpret_cast<char*>(d);
  mp->dm.slot_bytes = mp->slot_bytes;
  return NRPF_OK;
}

void drop_graph(pf_multi* mp) {
  if (mp->gexec) cudaGraphExecDestroy(mp->gexec);
  mp->gexec = nullptr;
}

// Work items for S scenarios per item: (plan, tile of <= S scenarios), sorted
// by decreasing estimated work; with use_smem, the items of every plan whose
// state fits kMultiSmemMax run in shared memory (sized for the largest), the
// others in global slots.
int build_items(pf_multi* mp, int S, int use_smem) {
  const size_t w = mp->lu_precision == NRPF_LU_FP32 ? 4 : 8;
  size_t smem = 0;
  if (use_smem)
    for (const pf_plan* p : mp->plans) {
      const size_t b = state_bytes(p->hp, S, w);
      if (b <= kMultiSmemMax) smem = std::max(smem, b);
    }
  size_t slot = 256;
  std::vector<std::pair<double, Item>> items;
  int in_smem = 0;
  for (int f = 0; f < mp->k; ++f) {
    const nrpf::HostPlan& h = mp->plans[f]->hp;
    const size_t b = state_bytes(h, S, w);
    const int sm = smem > 0 && b <= smem;
    if (!sm) slot = std::max(slot, b);
    const double work = h.lu_fma + h.solve_fma + 16.0 * (double)h.colidx.size();
    for (int b0 = 0; b0 < mp->batch[f]; b0 += S) {
      Item it{f, b0, std::min(S, mp->batch[f] - b0), sm};
      items.push_back({work * it.nb, it});
      in_smem += sm;
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<double, Item>& a, const std::pair<double, Item>& b) { return a.first > b.first; });
  std::vector<Item> its(items.size());
  for (size_t i = 0; i < items.size(); ++i) its[i] = items[i].second;
  if (its.size() > mp->items_cap) {
    if (mp->d_items) {
      cudaDeviceSynchronize();
      cudaFree(mp->d_items);
      mp->d_items = nullptr;
    }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, std::max<size_t>(its.size(), 1) * sizeof(Item));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
    mp->d_items = d;
    mp->items_cap = its.size();
  } else if (mp->d_items) {
    cudaDeviceSynchronize();  // a running launch may still read the old list
  }
  if (!its.empty() &&
      cudaMemcpy(mp->d_items, its.data(), its.size() * sizeof(Item), cudaMemcpyHostToDevice) != cudaSuccess)
    return NRPF_ERR_CUDA;
  drop_graph(mp);
  int ls = 0;
  while ((1 << ls) < S) ++ls;
  mp->scen = S;
  mp->use_smem = use_smem;
  mp->smem_bytes = smem;
  mp->smem_items = in_smem;
  mp->slot_bytes = slot;
  mp->dm.items = reinterpret_cast<const Item*>(mp->d_items);
  mp->dm.n_items = (int)its.size();
  mp->dm.log_s = ls;
  cudaError_t e = mp->lu_precision == NRPF_LU_FP32
                      ? cudaFuncSetAttribute(k_multi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_multi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return NRPF_ERR_CUDA;
  return ensure_slots(mp, (size_t)mp->sms * mp->blocks_per_sm);
}

template <typename T>
int launch_multi(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                 int32_t* iters, uint8_t* status, cudaStream_t st) {
  const unsigned grid = (unsigned)(mp->sms * mp->blocks_per_sm);
  cudaMemsetAsync(mp->dm.next, 0, sizeof(int), st);
  k_multi<T><<<grid, dim3(32, mp->warps), mp->smem_bytes, st>>>(mp->dm, reinterpret_cast<const double2*>(sbus),
                                                               reinterpret_cast<const double2*>(v0), tol, maxit,
                                                               reinterpret_cast<double2*>(v_out), iters, status);
  return NRPF_OK;
}

}  // namespace

extern "C" {

int pf_multi_create(int k, pf_plan* const* plans, const int32_t* batch, pf_multi** out) {
  if (!out || k <= 0 || !plans || !batch) return NRPF_ERR_ARG;
  *out = nullptr;
  const int prec = plans[0] ? plans[0]->lu_precision : 0;
  int64_t inst = 0, cin = 0;
  std::vector<nrpf::DevPlan> dps(k);
  std::vector<int64_t> in_off(k), inst_off(k);
  for (int f = 0; f < k; ++f) {
    const pf_plan* p = plans[f];
    if (!p || p->host_only || batch[f] < 0) return NRPF_ERR_ARG;
    if (p->lu_precision != prec || p->hp.nd != 0) return NRPF_ERR_ARG;
    dps[f] = p->dp;
    in_off[f] = cin;
    inst_off[f] = inst;
    cin += (int64_t)batch[f] * p->hp.n;
    inst += batch[f];
  }
  pf_multi* mp = new (std::nothrow) pf_multi();
  if (!mp) return NRPF_ERR_NOMEM;
  mp->k = k;
  mp->lu_precision = prec;
  mp->total_instances = inst;
  mp->plans.assign(plans, plans + k);
  mp->batch.assign(batch, batch + k);
  cudaGetDevice(&mp->device);
  cudaDeviceGetAttribute(&mp->sms, cudaDevAttrMultiProcessorCount, mp->device);
  auto up = [&](const void* src, size_t bytes, void** dst) -> int {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
    mp->allocs.push_back(d);
    if (bytes && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return NRPF_ERR_CUDA;
    *dst = d;
    return NRPF_OK;
  };
  void *d_plans, *d_in, *d_inst, *d_next;
  int zero = 0;
  int rc;
  if ((rc = up(dps.data(), dps.size() * sizeof(nrpf::DevPlan), &d_plans)) ||
      (rc = up(in_off.data(), in_off.size() * 8, &d_in)) || (rc = up(inst_off.data(), inst_off.size() * 8, &d_inst)) ||
      (rc = up(&zero, sizeof(int), &d_next))) {
    pf_multi_destroy(mp);
    return rc;
  }
  mp->dm.plans = reinterpret_cast<const nrpf::DevPlan*>(d_plans);
  mp->dm.in_off = reinterpret_cast<const int64_t*>(d_in);
  mp->dm.inst_off = reinterpret_cast<const int64_t*>(d_inst);
  mp->dm.next = reinterpret_cast<int*>(d_next);
  if ((rc = build_items(mp, kTile, 0))) {
    pf_multi_destroy(mp);
    return rc;
  }
  *out = mp;
  return NRPF_OK;
}

int pf_multi_set_scenarios(pf_multi* mp, int per_item, int use_smem) {
  if (!mp || per_item < 1 || per_item > kTile || (per_item & (per_item - 1)) || (use_smem != 0 && use_smem != 1))
    return NRPF_ERR_ARG;
  return build_items(mp, per_item, use_smem);
}

int pf_multi_get_scenarios(const pf_multi* mp, int* per_item, int* use_smem, int64_t* smem_bytes, int* smem_items) {
  if (!mp) return NRPF_ERR_ARG;
  if (per_item) *per_item = mp->scen;
  if (use_smem) *use_smem = mp->use_smem;
  if (smem_bytes) *smem_bytes = (int64_t)mp->smem_bytes;
  if (smem_items) *smem_items = mp->smem_items;
  return NRPF_OK;
}

int pf_multi_set_config(pf_multi* mp, int warps, int blocks_per_sm) {
  if (!mp || warps < 1 || warps > kMaxWarps || blocks_per_sm < 1 || blocks_per_sm > 32) return NRPF_ERR_ARG;
  int rc = ensure_slots(mp, (size_t)mp->sms * blocks_per_sm);
  if (rc) return rc;
  mp->warps = warps;
  mp->blocks_per_sm = blocks_per_sm;
  return NRPF_OK;
}

int pf_multi_get_config(const pf_multi* mp, int* warps, int* blocks_per_sm, int64_t* instances, int* items) {
  if (!mp) return NRPF_ERR_ARG;
  if (warps) *warps = mp->warps;
  if (blocks_per_sm) *blocks_per_sm = mp->blocks_per_sm;
  if (instances) *instances = mp->total_instances;
  if (items) *items = mp->dm.n_items;
  return NRPF_OK;
}

int pf_multi_solve(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                   int32_t* iters, uint8_t* status, void* stream) {
  if (!mp || maxit < 0 || !(tol >= 0) || !std::isfinite(tol)) return NRPF_ERR_ARG;
  if (mp->total_instances == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const void* args[7] = {sbus, v0, v_out, iters, status, nullptr, nullptr};
  const bool same = mp->gexec && mp->g_tol == tol && mp->g_maxit == maxit && mp->g_warps == mp->warps &&
                    mp->g_bps == mp->blocks_per_sm && mp->g_stream == st &&
                    std::equal(args, args + 5, mp->g_args);
  if (!same) {
    drop_graph(mp);
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return NRPF_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (mp->lu_precision == NRPF_LU_FP32)
      launch_multi<float>(mp, sbus, v0, tol, maxit, v_out, iters, status, cap);
    else
      launch_multi<double>(mp, sbus, v0, tol, maxit, v_out, iters, status, cap);
    const cudaError_t el = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (el != cudaSuccess) e = el;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || !g) return NRPF_ERR_CUDA;
    e = cudaGraphInstantiate(&mp->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      mp->gexec = nullptr;
      return NRPF_ERR_CUDA;
    }
    std::copy(args, args + 7, mp->g_args);
    mp->g_tol = tol;
    mp->g_maxit = maxit;
    mp->g_warps = mp->warps;
    mp->g_bps = mp->blocks_per_sm;
    mp->g_stream = st;
  }
  if (cudaGraphLaunch(mp->gexec, st) != cudaSuccess) return NRPF_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_multi_autotune(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                      int32_t* iters, uint8_t* status, void* stream, double* best_ms) {
  if (!mp) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int bw = mp->warps, bb = mp->blocks_per_sm, bs = mp->scen, bm = mp->use_smem;
  const int warps_c[] = {1, 2, 4, 8, 16};
  const int bps_c[] = {1, 2, 4, 8, 16};
  // scenarios per item with the state in global slots (32, 16, 8) or, where
  // it fits, in shared memory (32 .. 2)
  const int scen_c[][2] = {{32, 0}, {16, 0}, {8, 0}, {32, 1}, {16, 1}, {8, 1}, {4, 1}, {2, 1}};
  int rc = NRPF_OK;
  for (const auto& sc : scen_c) {
    if ((rc = pf_multi_set_scenarios(mp, sc[0], sc[1]))) break;
    if (sc[1] && mp->smem_items == 0) continue;  // nothing fits: same as global slots
    for (int w : warps_c)
      for (int b : bps_c) {
        if (w * b > 64) continue;  // at most 2048 threads per SM
        if (mp->smem_bytes * b > 228 * 1024) continue;  // CTAs that could not be resident together
        if ((rc = pf_multi_set_config(mp, w, b))) break;
        if ((rc = pf_multi_solve(mp, sbus, v0, tol, maxit, v_out, iters, status, stream))) break;
        float ms_min = 1e30f;
        for (int r = 0; r < 2; ++r) {
          cudaEventRecord(e0, st);
          pf_multi_solve(mp, sbus, v0, tol, maxit, v_out, iters, status, stream);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best) {
          best = ms_min;
          bw = w;
          bb = b;
          bs = sc[0];
          bm = sc[1];
        }
      }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best_ms) *best_ms = best;
  if ((rc = pf_multi_set_scenarios(mp, bs, bm))) return rc;
  return pf_multi_set_config(mp, bw, bb);
}

void pf_multi_destroy(pf_multi* mp) {
  if (!mp) return;
  cudaDeviceSynchronize();
  drop_graph(mp);
  if (mp->ws) cudaFree(mp->ws);
  if (mp->d_items) cudaFree(mp->d_items);
  for (void* a : mp->allocs) cudaFree(a);
  delete mp;
}

}  // extern "C"
