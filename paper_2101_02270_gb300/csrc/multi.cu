// Uneven batching: grids of different sizes and patterns (one plan each) and
// different scenario counts solved by ONE persistent kernel.  Work items are
// (plan, tile of up to 32 scenarios), sorted by decreasing work; every CTA
// pulls items from an atomic counter and runs the whole Newton loop of its
// item (Sec. 3 steps 1-4) with the item's data in a private workspace slot:
// lanes = scenarios of the tile, warps = threads per instance, splitting the
// buses of the mismatch and update, the columns of each refactor level and
// the rows of each FS/BS level, with a CTA barrier between phases.  The memset
// of the counter and the kernel are captured once in a CUDA graph and
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

struct Item {
  int32_t plan;  // plan index
  int32_t b0;    // first scenario of the tile within the plan's batch
  int32_t nb;    // scenarios in the tile (<= 32)
  int32_t pad;
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
};

template <typename T>
__global__ void __launch_bounds__(32 * kMaxWarps) k_multi(DevMulti M, const double2* __restrict__ sbus,
                                                          const double2* __restrict__ v0, double tol, int maxit,
                                                          double2* __restrict__ vout, int32_t* __restrict__ iters_out,
                                                          uint8_t* __restrict__ status_out) {
  __shared__ int s_item;
  __shared__ double s_red[kMaxWarps][32];
  __shared__ int s_bad[32];
  const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
  const int tid = warp * 32 + lane, nthr = 32 * W;
  char* slot = M.ws + (size_t)blockIdx.x * M.slot_bytes;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(M.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= M.n_items) break;
    const Item it = M.items[item];
    const DevPlan& P = M.plans[it.plan];
    const int n = P.n;
    double* vm = reinterpret_cast<double*>(slot);
    double* va = vm + (size_t)n * kTile;
    double* ve = va + (size_t)n * kTile;
    double* vf = ve + (size_t)n * kTile;
    double* vinv = vf + (size_t)n * kTile;
    double* psp = vinv + (size_t)n * kTile;
    double* qsp = psp + (size_t)n * kTile;
    T* X = reinterpret_cast<T*>(qsp + (size_t)n * kTile);
    T* LU = X + (size_t)P.mp * kTile;
    const bool valid = lane < it.nb;
    const int64_t base = M.in_off[it.plan] + (int64_t)(it.b0 + lane) * n;
    // ---- load (user layout -> interleaved slot) ----
    for (int i = warp; i < n; i += W) {
      double2 s = make_double2(0.0, 0.0), v = make_double2(1.0, 0.0);
      if (valid) {
        s = sbus[base + i];
        v = v0[base + i];
      }
      // a start on the positive real axis (flat start) needs no FP64 sqrt
      // or atan2
      const bool real = v.y == 0.0 && v.x > 0.0;
      const double mag = real ? v.x : sqrt(v.x * v.x + v.y * v.y);
      const int o = i * kTile + lane;
      psp[o] = s.x;
      qsp[o] = s.y;
      vm[o] = mag;
      va[o] = real ? 0.0 : atan2(v.y, v.x);
      ve[o] = v.x;
      vf[o] = v.y;
      vinv[o] = 1.0 / mag;
    }
    if (warp == 0) s_bad[lane] = 0;
    int act = valid ? 1 : 0, my_iters = 0, my_status = NRPF_MAXIT_CODE;
    __syncthreads();
    for (int itn = 0;; ++itn) {
      // ---- zero the LU workspace, then mismatch + Jacobian (Alg. 1, Sec. 3.1.2) ----
      for (int64_t e = tid; e < P.NLU * kTile; e += nthr) LU[e] = (T)0;
      __syncthreads();
      double nrm = 0.0;
      for (int i = warp; i < n; i += W) {
        const int bt = P.bus_type[i];
        if (bt == 3) continue;
        const double ei = ve[i * kTile + lane], fi = vf[i * kTile + lane];
        double Ir = 0.0, Ii = 0.0;
        for (int d = P.rowptr[i]; d < P.rowptr[i + 1]; ++d) {
          const int k = P.colidx[d];
          const double G = P.yre[d], Bv = P.yim[d];
          const double ek = ve[k * kTile + lane], fk = vf[k * kTile + lane];
          const double yr = G * ek - Bv * fk, yi = G * fk + Bv * ek;
          Ir += yr;
          Ii += yi;
          if (k != i) {
            const int4 jm = reinterpret_cast<const int4*>(P.jmap)[d];
            if (jm.x >= 0) {
              // off-diagonal Jacobian entries in the LU precision (stored in
              // it); the mismatch stays FP64
              const T Wr = (T)ei * (T)yr + (T)fi * (T)yi, Wi = (T)fi * (T)yr - (T)ei * (T)yi;
              const T ik = (T)vinv[k * kTile + lane];
              LU[(size_t)jm.x * kTile + lane] = Wi;
              if (jm.y >= 0) LU[(size_t)jm.y * kTile + lane] = Wr * ik;
              if (jm.z >= 0) LU[(size_t)jm.z * kTile + lane] = -Wr;
              if (jm.w >= 0) LU[(size_t)jm.w * kTile + lane] = Wi * ik;
            }
          }
        }
        const double Pc = ei * Ir + fi * Ii, Qc = fi * Ir - ei * Ii;
        const int o = i * kTile + lane;
        const double dP = Pc - psp[o];
        double a = fabs(dP);
        X[(size_t)P.rhs_p[i] * kTile + lane] = (T)(-dP);
        if (bt == 1) {
          const double dQ = Qc - qsp[o];
          X[(size_t)P.rhs_q[i] * kTile + lane] = (T)(-dQ);
          const double q = fabs(dQ);
          a = (q > a || q != q) ? q : a;
        }
        nrm = (a > nrm || a != a) ? a : nrm;
        const int dd = P.ydiag[i];
        const int4 jm = reinterpret_cast<const int4*>(P.jmap)[dd];
        const double G = P.yre[dd], Bv = P.yim[dd];
        const double vm2 = ei * ei + fi * fi, ivm = vinv[o], mg = vm2 * ivm;
        LU[(size_t)jm.x * kTile + lane] = (T)(-Qc - Bv * vm2);
        if (jm.y >= 0) LU[(size_t)jm.y * kTile + lane] = (T)(Pc * ivm + G * mg);
        if (jm.z >= 0) LU[(size_t)jm.z * kTile + lane] = (T)(Pc - G * vm2);
        if (jm.w >= 0) LU[(size_t)jm.w * kTile + lane] = (T)(Qc * ivm - Bv * mg);
      }
      if (!(nrm <= DBL_MAX)) nrm = __longlong_as_double(0x7ff0000000000000ll);
      s_red[warp][lane] = nrm;
      __syncthreads();
      // ---- convergence test (every thread computes its lane's outcome) ----
      double tot = s_red[0][lane];
      for (int w = 1; w < W; ++w) tot = fmax(tot, s_red[w][lane]);
      if (act) {
        if (s_bad[lane]) {
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
        for (int ci = c0 + warp; ci < c1; ci += W) {
          const int j = P.lu_cols[ci];
          for (int u = P.col_upd_ptr[j]; u < P.col_upd_ptr[j + 1]; ++u) {
            const DevUpd up = P.upd[u];
            const T x = LU[(size_t)up.ukj * kTile + lane];
            const int32_t* dst = P.dst + up.dst_off;
            const T* src = LU + (size_t)up.lsrc * kTile + lane;
            for (int q = 0; q < up.llen; ++q) LU[(size_t)dst[q] * kTile + lane] -= x * src[(size_t)q * kTile];
          }
          const int dpj = P.dp[j];
          if (dpj >= 0) {
            const T inv = (T)1 / LU[(size_t)dpj * kTile + lane];
            for (int64_t p = dpj + 1; p < P.ce[j]; ++p) LU[(size_t)p * kTile + lane] *= inv;
          }
        }
        __syncthreads();
      }
      // ---- forward / backward substitution ----
      for (int l = 0; l < P.n_fw_lvl; ++l) {
        const int r0 = P.fw_lvl_ptr[l], r1 = P.fw_lvl_ptr[l + 1];
        for (int ri = r0 + warp; ri < r1; ri += W) {
          const int i = P.fw_rows[ri];
          T acc = X[(size_t)i * kTile + lane];
          for (int e = P.fw_ptr[ri]; e < P.fw_ptr[ri + 1]; ++e)
            acc -= LU[(size_t)P.fw_pos[e] * kTile + lane] * X[(size_t)P.fw_col[e] * kTile + lane];
          X[(size_t)i * kTile + lane] = acc;
        }
        __syncthreads();
      }
      for (int l = 0; l < P.n_bw_lvl; ++l) {
        const int r0 = P.bw_lvl_ptr[l], r1 = P.bw_lvl_ptr[l + 1];
        for (int ri = r0 + warp; ri < r1; ri += W) {
          const int i = P.bw_rows[ri];
          T acc = X[(size_t)i * kTile + lane];
          for (int e = P.bw_ptr[ri]; e < P.bw_ptr[ri + 1]; ++e)
            acc -= LU[(size_t)P.bw_pos[e] * kTile + lane] * X[(size_t)P.bw_col[e] * kTile + lane];
          X[(size_t)i * kTile + lane] = acc / LU[(size_t)P.dp[i] * kTile + lane];
        }
        __syncthreads();
      }
      // ---- voltage update (Sec. 3 step 4) ----
      if (act) {
        for (int i = warp; i < n; i += W) {
          const int bt = P.bus_type[i];
          if (bt == 3) continue;
          const int o = i * kTile + lane;
          const double dth = (double)X[(size_t)P.rhs_p[i] * kTile + lane];
          double a = va[o] + dth, g = vm[o];
          bool ok = fabs(dth) <= DBL_MAX;
          if (bt == 1) {
            const double dv = (double)X[(size_t)P.rhs_q[i] * kTile + lane];
            ok = ok && fabs(dv) <= DBL_MAX;
            g += dv;
          }
          if (!ok) {
            s_bad[lane] = 1;
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
      for (int i = warp; i < n; i += W) vout[base + i] = make_double2(ve[i * kTile + lane], vf[i * kTile + lane]);
      if (warp == 0) {
        const int64_t g = M.inst_off[it.plan] + it.b0 + lane;
        iters_out[g] = my_iters;
        status_out[g] = (uint8_t)my_status;
      }
    }
    __syncthreads();
  }
}

}  // namespace

struct pf_multi {
  int k = 0;
  int lu_precision = NRPF_LU_FP64;
  int device = 0;
  int warps = 4;
  int blocks_per_sm = 4;
  int sms = 0;
  int64_t total_instances = 0;
  size_t slot_bytes = 0;
  std::vector<void*> allocs;
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
  if (slots <= mp->ws_slots) return NRPF_OK;
  if (mp->ws) {
    cudaDeviceSynchronize();
    cudaFree(mp->ws);
    mp->ws = nullptr;
    mp->ws_slots = 0;
  }
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, slots * mp->slot_bytes);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
  mp->ws = d;
  mp->ws_slots = slots;
  mp->dm.ws = reinterpret_cast<char*>(d);
  mp->dm.slot_bytes = mp->slot_bytes;
  return NRPF_OK;
}

template <typename T>
void launch_multi(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                  int32_t* iters, uint8_t* status, cudaStream_t st) {
  const unsigned grid = (unsigned)(mp->sms * mp->blocks_per_sm);
  cudaMemsetAsync(mp->dm.next, 0, sizeof(int), st);
  k_multi<T><<<grid, dim3(32, mp->warps), 0, st>>>(mp->dm, reinterpret_cast<const double2*>(sbus),
                                                   reinterpret_cast<const double2*>(v0), tol, maxit,
                                                   reinterpret_cast<double2*>(v_out), iters, status);
}

void drop_graph(pf_multi* mp) {
  if (mp->gexec) cudaGraphExecDestroy(mp->gexec);
  mp->gexec = nullptr;
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
  std::vector<std::pair<double, Item>> items;
  size_t slot = 0;
  for (int f = 0; f < k; ++f) {
    const pf_plan* p = plans[f];
    if (!p || p->host_only || batch[f] < 0) return NRPF_ERR_ARG;
    if (p->lu_precision != prec || p->hp.nd != 0) return NRPF_ERR_ARG;
    dps[f] = p->dp;
    in_off[f] = cin;
    inst_off[f] = inst;
    cin += (int64_t)batch[f] * p->hp.n;
    inst += batch[f];
    const double work = p->hp.lu_fma + p->hp.solve_fma + 16.0 * (double)p->hp.colidx.size();
    for (int b0 = 0; b0 < batch[f]; b0 += kTile) {
      Item it{f, b0, std::min(kTile, batch[f] - b0), 0};
      items.push_back({work * it.nb, it});
    }
    const size_t w = prec == NRPF_LU_FP32 ? 4 : 8;
    const size_t bytes = ((size_t)7 * p->hp.n * 8 + (size_t)(p->hp.s + p->hp.ndp + p->hp.NLU) * w) * kTile;
    slot = std::max(slot, (bytes + 255) / 256 * 256);
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<double, Item>& a, const std::pair<double, Item>& b) { return a.first > b.first; });
  std::vector<Item> its(items.size());
  for (size_t i = 0; i < items.size(); ++i) its[i] = items[i].second;
  pf_multi* mp = new (std::nothrow) pf_multi();
  if (!mp) return NRPF_ERR_NOMEM;
  mp->k = k;
  mp->lu_precision = prec;
  mp->total_instances = inst;
  mp->slot_bytes = std::max<size_t>(slot, 256);
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
  void *d_plans, *d_in, *d_inst, *d_items, *d_next;
  int zero = 0;
  int rc;
  if ((rc = up(dps.data(), dps.size() * sizeof(nrpf::DevPlan), &d_plans)) ||
      (rc = up(in_off.data(), in_off.size() * 8, &d_in)) || (rc = up(inst_off.data(), inst_off.size() * 8, &d_inst)) ||
      (rc = up(its.data(), its.size() * sizeof(Item), &d_items)) || (rc = up(&zero, sizeof(int), &d_next))) {
    pf_multi_destroy(mp);
    return rc;
  }
  mp->dm.plans = reinterpret_cast<const nrpf::DevPlan*>(d_plans);
  mp->dm.in_off = reinterpret_cast<const int64_t*>(d_in);
  mp->dm.inst_off = reinterpret_cast<const int64_t*>(d_inst);
  mp->dm.items = reinterpret_cast<const Item*>(d_items);
  mp->dm.n_items = (int)its.size();
  mp->dm.next = reinterpret_cast<int*>(d_next);
  if ((rc = ensure_slots(mp, (size_t)mp->sms * mp->blocks_per_sm))) {
    pf_multi_destroy(mp);
    return rc;
  }
  *out = mp;
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
    cudaError_t e = cudaStreamEndCapture(cap, &g);
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
  int bw = mp->warps, bb = mp->blocks_per_sm;
  const int warps_c[] = {1, 2, 4, 8, 16};
  const int bps_c[] = {1, 2, 4, 8, 16};
  int rc = NRPF_OK;
  for (int w : warps_c)
    for (int b : bps_c) {
      if (w * b > 64) continue;  // at most 2048 threads per SM
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
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best_ms) *best_ms = best;
  return pf_multi_set_config(mp, bw, bb);
}

void pf_multi_destroy(pf_multi* mp) {
  if (!mp) return;
  cudaDeviceSynchronize();
  drop_graph(mp);
  if (mp->ws) cudaFree(mp->ws);
  for (void* a : mp->allocs) cudaFree(a);
  delete mp;
}

}  // extern "C"
