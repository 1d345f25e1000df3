// C ABI of the batched Newton-Raphson power-flow library (include/nrpf.h).
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nrpf.h"
#include "device.h"
#include "handle.h"
#include "kernels.h"
#include "plan.h"

using nrpf::DevPlan;
using nrpf::DevState;
using nrpf::HostPlan;
using nrpf::kTile;


namespace {

// seeded minimum-degree tie-breaks tried per plan when pf_options.order_tries
// is 0: 128 up to 4,000 buses, fewer above so that the orderings take about
// as long as the rest of the symbolic analysis, never fewer than 8
int default_order_tries(int n) { return std::max(8, std::min(128, 512000 / std::max(n, 1))); }
constexpr double kSparseWeightFp64 = 1.5;
constexpr double kSparseWeightFp32 = 15.0;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      return e_ == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA; \
    }                                              \
  } while (0)

template <typename T>
int upload(pf_plan* p, const std::vector<T>& v, const T** out) {
  if (v.empty()) { *out = nullptr; return NRPF_OK; }
  void* d = nullptr;
  CK(cudaMalloc(&d, v.size() * sizeof(T)));
  p->plan_allocs.push_back(d);
  CK(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = reinterpret_cast<const T*>(d);
  return NRPF_OK;
}

// Fold the launches made by loop graphs (one body's launches x bodies run)
// into the counters and zero the device count.  Synchronises the device.
void fold_graph_launches(pf_plan* p) {
  if (!p->st.ctl) return;
  cudaDeviceSynchronize();
  long long gi = 0;
  char* f = reinterpret_cast<char*>(p->st.ctl) + offsetof(nrpf::SolveCtl, graph_iters);
  if (cudaMemcpy(&gi, f, sizeof(gi), cudaMemcpyDeviceToHost) != cudaSuccess) return;
  for (int c = 0; c < nrpf::K_NCLASS; ++c) p->rec.launches[c] += p->body_launches[c] * gi;
  const long long zero = 0;
  cudaMemcpy(f, &zero, sizeof(zero), cudaMemcpyHostToDevice);
}

void destroy_loop_graphs(pf_plan* p) {
  for (auto& kv : p->loops) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  p->loops.clear();
}

void free_ws(pf_plan* p) {
  fold_graph_launches(p);
  destroy_loop_graphs(p);
  if (p->yv_mem) cudaFree(p->yv_mem);
  p->yv_mem = nullptr;
  p->yv_cap = 0;
  for (void* a : p->ws_allocs) cudaFree(a);
  p->ws_allocs.clear();
  p->capacity = 0;
  p->st = DevState{};
}

int ensure_capacity(pf_plan* p, int B) {
  const int Bp = (B + kTile - 1) / kTile * kTile;
  if (Bp <= p->capacity) return NRPF_OK;
  // The new workspace replaces the old one: wait for work still using it.
  CK(cudaDeviceSynchronize());
  free_ws(p);
  const HostPlan& h = p->hp;
  const size_t w = p->lu_precision == NRPF_LU_FP32 ? 4 : 8;
  auto alloc = [&](size_t bytes, void** out) -> int {
    void* d = nullptr;
    CK(cudaMalloc(&d, std::max<size_t>(bytes, 256)));
    p->ws_allocs.push_back(d);
    *out = d;
    return NRPF_OK;
  };
  DevState s{};
  s.Bp = Bp;
  int rc = NRPF_OK;
  const size_t nb = (size_t)h.n * Bp * sizeof(double);
  void* t = nullptr;
#define AL(bytes, field, type)            \
  if ((rc = alloc((bytes), &t))) { free_ws(p); return rc; } \
  s.field = reinterpret_cast<type>(t);
  AL(nb, vm, double*);
  AL(nb, va, double*);
  AL(nb, ve, double*);
  AL(nb, vf, double*);
  AL(nb, vinv, double*);
  AL(nb, psp, double*);
  AL(nb, qsp, double*);
  AL((size_t)(h.s + h.ndp) * Bp * w, x, void*);
  AL((size_t)h.NLU * Bp * w, lu, void*);
  // inverse pivots of the current diagonal block (interleaved dense block),
  // or U11^-1 and L11^-1 of the current 64 x 64 block (instance-major)
  AL(p->dp.dim ? (size_t)2 * 64 * 64 * Bp * sizeof(float) : (size_t)std::max(h.kb, 1) * Bp * w, inv, void*);
  AL((size_t)Bp * sizeof(unsigned long long), norm, unsigned long long*);
  AL((size_t)Bp * 4, iters, int32_t*);
  AL((size_t)Bp * 4, status, int32_t*);
  AL((size_t)Bp * 4, active, int32_t*);
  AL((size_t)Bp * 4, bad, int32_t*);
  AL(sizeof(nrpf::SolveCtl), ctl, nrpf::SolveCtl*);
#undef AL
  CK(cudaMemset(s.ctl, 0, sizeof(nrpf::SolveCtl)));
  if (p->dp.dim && h.ndp > 0) {
    // TMA descriptors of this workspace's dense blocks
    if (!nrpf::make_dense_im_maps(p->dp, s.lu, Bp, &p->im_maps)) {
      free_ws(p);
      return NRPF_ERR_CUDA;
    }
    s.im_maps = &p->im_maps;
  }
  if (!p->h_prev) CK(cudaHostAlloc(reinterpret_cast<void**>(&p->h_prev), sizeof(int32_t), cudaHostAllocDefault));
  p->st = s;
  p->capacity = Bp;
  return NRPF_OK;
}

// One Newton iteration (Alg. 1 loop body): LU preparation and mismatch +
// Jacobian (gated by the previous check), the convergence test, then
// refactorisation, FS/BS and update (gated by this check), and the tail that
// advances the loop control.
template <typename T>
void enqueue_body(pf_plan* p, const DevState& S, cudaStream_t st, nrpf::Recorder* rec,
                  cudaGraphConditionalHandle cond, int graph) {
  const DevPlan& P = p->dp;
  const HostPlan& h = p->hp;
  const int32_t* prev = nrpf::ctl_prev(S);
  const int32_t* cur = nrpf::ctl_cur(S);
  nrpf::launch_prepare_lu<T>(P, S, prev, st, rec, false);
  nrpf::launch_mismatch<T>(P, S, 1, prev, st, rec);
  nrpf::launch_check(S, st, rec);
  nrpf::launch_factor<T>(P, S, h.lu_lvl_ptr, cur, st, rec);
  nrpf::launch_solve<T>(P, S, h.fw_lvl_ptr, h.bw_lvl_ptr, cur, st, rec);
  nrpf::launch_update<T>(P, S, cur, st, rec);
  nrpf::launch_iter_tail(S, cond, graph, st, rec);
}

// The loop graph: a WHILE node whose body is one iteration, captured once per
// workspace and padded batch size; the iteration's tail kernel sets the
// condition, so the loop ends on the device as soon as no instance is active
// (or at maxit).
template <typename T>
int ensure_loop_graph(pf_plan* p, const DevState& S, cudaGraphExec_t* out) {
  const int key = 2 * S.Bp + (S.yv ? 1 : 0);
  auto it = p->loops.find(key);
  if (it != p->loops.end()) {
    *out = it->second.exec;
    return NRPF_OK;
  }
  if (!p->capture_stream) CK(cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  auto fail = [&](cudaError_t e) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
  };
  cudaGraphConditionalHandle cond = 0;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e);
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) return fail(e);
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(p->capture_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(e);
  nrpf::Recorder count;  // launches of one body, by class
  enqueue_body<T>(p, S, p->capture_stream, &count, cond, 1);
  cudaGraph_t captured = nullptr;
  const cudaError_t el = cudaGetLastError();
  e = cudaStreamEndCapture(p->capture_stream, &captured);
  if (el != cudaSuccess) return fail(el);
  if (e != cudaSuccess) return fail(e);
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess) return fail(e);
  p->loops[key] = pf_plan::LoopGraph{g, exec};
  for (int c = 0; c < nrpf::K_NCLASS; ++c) p->body_launches[c] = count.launches[c];
  *out = exec;
  return NRPF_OK;
}

// workspace array of per-instance Ybus values for the current capacity
int ensure_yv(pf_plan* p) {
  if (p->yv_mem && p->yv_cap >= p->capacity) return NRPF_OK;
  if (p->yv_mem) {
    CK(cudaDeviceSynchronize());
    cudaFree(p->yv_mem);
    p->yv_mem = nullptr;
    p->yv_cap = 0;
  }
  CK(cudaMalloc(&p->yv_mem, std::max<size_t>((size_t)p->capacity * p->dp.nnzY * 16, 256)));
  p->yv_cap = p->capacity;
  return NRPF_OK;
}

// ybus: per-instance [B, nnzY] complex device values, or null for the plan's;
// outages (device [B, k], with ybus null): per-instance admittances built on
// the device from the plan's base values and branch stamps
template <typename T>
int enqueue_solve(pf_plan* p, int B, const double* ybus, const double* sbus, const double* v0, double tol,
                  int maxit, double* v_out, int32_t* iters, uint8_t* status, cudaStream_t st,
                  const int32_t* outages = nullptr, int k = 0) {
  const DevPlan& P = p->dp;
  // grids cover this batch's tiles only (tiles are contiguous per array, so
  // the first Bp of the workspace's capacity serve)
  DevState S = p->st;
  S.Bp = (B + kTile - 1) / kTile * kTile;
  nrpf::Recorder* rec = &p->rec;
  if (ybus || outages) {
    int rc = ensure_yv(p);
    if (rc) return rc;
    S.yv = reinterpret_cast<const double2*>(p->yv_mem);
    if (ybus)
      nrpf::launch_load_y(P, S, B, ybus, st, rec);
    else
      nrpf::launch_outage_y(P, S, B, outages, k, p->d_bpos, p->d_bval, p->nbr, st, rec);
  }
  nrpf::launch_load(P, S, B, sbus, v0, st, rec);
  nrpf::launch_ctl_init(S, maxit, tol, st, rec);
  if (P.m > 0 && maxit > 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      // the caller captures this stream: maxit iterations, instances that
      // have finished skip through the gates
      for (int it = 0; it < maxit; ++it) enqueue_body<T>(p, S, st, rec, 0, 0);
    } else if (rec->time_mask) {
      // profiled solve (per-launch events): the host ends the loop
      for (int it = 0; it < maxit; ++it) {
        enqueue_body<T>(p, S, st, rec, 0, 0);
        CK(cudaMemcpyAsync(p->h_prev, nrpf::ctl_prev(S), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*p->h_prev == 0) break;
      }
    } else {
      cudaGraphExec_t exec = nullptr;
      int rc = ensure_loop_graph<T>(p, S, &exec);
      if (rc) return rc;
      CK(cudaGraphLaunch(exec, st));
    }
  }
  // the last convergence test (iteration ctl->it; nothing is active after an
  // early exit): the mismatch only, no Jacobian
  if (P.m > 0) nrpf::launch_mismatch<T>(P, S, 0, nrpf::ctl_prev(S), st, rec);
  nrpf::launch_check(S, st, rec);
  nrpf::launch_store(P, S, B, v_out, iters, status, st, rec);
  return NRPF_OK;
}

int build_pattern_map(pf_plan* p) {
  if (p->d_pattern_map) return NRPF_OK;
  const HostPlan& h = p->hp;
  std::vector<int64_t> map;
  map.reserve((size_t)h.nnz_pattern);
  for (int j = 0; j < h.m; ++j) {
    for (int64_t q = h.cs[j]; q < h.ce[j]; ++q) map.push_back(q);
    if (j >= h.s)
      for (int r = h.s; r < h.m; ++r) map.push_back(h.NS + (int64_t)(j - h.s) * h.ndp + (r - h.s));
  }
  p->pattern_nnz = (int64_t)map.size();
  if (map.empty()) return NRPF_OK;
  void* d = nullptr;
  CK(cudaMalloc(&d, map.size() * sizeof(int64_t)));
  CK(cudaMemcpy(d, map.data(), map.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  p->d_pattern_map = reinterpret_cast<int64_t*>(d);
  return NRPF_OK;
}

template <typename T>
void enqueue_factor(pf_plan* p, int factor, cudaStream_t st) {
  nrpf::launch_prepare_lu<T>(p->dp, p->st, nullptr, st);
  nrpf::launch_mismatch<T>(p->dp, p->st, 1, nullptr, st);
  if (factor) nrpf::launch_factor<T>(p->dp, p->st, p->hp.lu_lvl_ptr, nullptr, st);
}

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NRPF_OK;
  return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
}

}  // namespace

extern "C" {

int pf_options_default(pf_options* opt) {
  if (!opt) return NRPF_ERR_ARG;
  opt->lu_precision = NRPF_LU_FP64;
  opt->ordering = NRPF_ORDER_AMD;
  opt->dense_frac = 0.0;  /* chosen by precision at plan creation */
  opt->panel = 0;  /* chosen by precision at plan creation */
  opt->max_batch = 0;
  opt->host_only = 0;
  opt->order_tries = 0;  /* default at plan creation */
  opt->dense_layout = NRPF_DENSE_AUTO;
  return NRPF_OK;
}

int pf_ybus_from_branches(int n, int nbr, const int32_t* f, const int32_t* t, const double* r,
                          const double* x, const double* b, int32_t* rowptr, int32_t* colidx,
                          double* y_re, double* y_im, int64_t cap, int64_t* nnz_out) {
  if (n <= 0 || nbr < 0 || !rowptr || !nnz_out) return NRPF_ERR_ARG;
  if (nbr > 0 && (!f || !t || !r || !x || !b)) return NRPF_ERR_ARG;
  // pi model: ys = 1/(r + jx); Y_ff += ys + jb/2, Y_tt += ys + jb/2, Y_ft -= ys, Y_tf -= ys
  std::vector<std::map<int, std::pair<double, double>>> rows(n);
  for (int i = 0; i < n; ++i) rows[i][i] = {0.0, 0.0};
  for (int e = 0; e < nbr; ++e) {
    const int a = f[e], c = t[e];
    if (a < 0 || a >= n || c < 0 || c >= n) return NRPF_ERR_ARG;
    const double den = r[e] * r[e] + x[e] * x[e];
    if (!(den > 0.0) || !std::isfinite(den) || !std::isfinite(b[e])) return NRPF_ERR_ARG;
    const double gs = r[e] / den, bs = -x[e] / den;
    auto add = [&](int i, int k, double gr, double gi) {
      auto& v = rows[i][k];
      v.first += gr;
      v.second += gi;
    };
    add(a, a, gs, bs + 0.5 * b[e]);
    add(c, c, gs, bs + 0.5 * b[e]);
    add(a, c, -gs, -bs);
    add(c, a, -gs, -bs);
  }
  int64_t nnz = 0;
  for (auto& row : rows) nnz += (int64_t)row.size();
  *nnz_out = nnz;
  if (nnz > cap || !colidx || !y_re || !y_im) return NRPF_ERR_ARG;
  int64_t q = 0;
  rowptr[0] = 0;
  for (int i = 0; i < n; ++i) {
    for (auto& kv : rows[i]) {
      colidx[q] = kv.first;
      y_re[q] = kv.second.first;
      y_im[q] = kv.second.second;
      ++q;
    }
    rowptr[i + 1] = (int32_t)q;
  }
  return NRPF_OK;
}

int pf_plan_create(int n, const int32_t* rowptr, const int32_t* colidx, const double* y_re,
                   const double* y_im, const int8_t* bus_type, const pf_options* opt, pf_plan** out) {
  if (!out) return NRPF_ERR_ARG;
  *out = nullptr;
  pf_options o;
  pf_options_default(&o);
  if (opt) o = *opt;
  if (o.dense_layout < NRPF_DENSE_AUTO || o.dense_layout > NRPF_DENSE_INSTANCE_MAJOR) return NRPF_ERR_ARG;
  // the instance-major kernels take FP32 blocks padded to a multiple of 64
  if (o.dense_layout == NRPF_DENSE_INSTANCE_MAJOR &&
      (o.lu_precision != NRPF_LU_FP32 || (o.panel != 0 && o.panel != 64)))
    return NRPF_ERR_ARG;
  const bool im_ok = o.lu_precision == NRPF_LU_FP32 && (o.panel == 0 || o.panel == 64);
  // default panel width by precision: FP32 needs the wider panel to feed its
  // FMA pipes with fewer passes over the trailing block
  if (o.panel == 0) o.panel = o.lu_precision == NRPF_LU_FP32 ? 64 : 8;
  // default dense cut by LU precision: an FMA of the sparse phase costs about
  // twice a dense-block FMA in FP64 (the FP64 pipe bounds both) but about 13x
  // in FP32 (the dense block runs at FP32 rate, the sparse phase does not),
  // so the FP32 path hands more of the matrix to the dense block
  if (o.dense_frac == 0.0) o.dense_frac = o.lu_precision == NRPF_LU_FP32 ? 0.3 : 0.7;
  if (o.order_tries == 0) o.order_tries = default_order_tries(n);
  if (o.lu_precision != NRPF_LU_FP64 && o.lu_precision != NRPF_LU_FP32) return NRPF_ERR_ARG;
  if (o.ordering != NRPF_ORDER_AMD && o.ordering != NRPF_ORDER_NATURAL) return NRPF_ERR_ARG;
  if (!(o.dense_frac > 0.0) || o.max_batch < 0 || o.order_tries < 0) return NRPF_ERR_ARG;
  // relative time of a multiply-add of the sparse phase (level schedule and
  // Schur tasks) to one of the dense block, from the kernels' measured times
  // per multiply-add on the 2,000-bus meshed grid
  const double sparse_weight = o.lu_precision == NRPF_LU_FP32 ? kSparseWeightFp32 : kSparseWeightFp64;
  pf_plan* p = new (std::nothrow) pf_plan();
  if (!p) return NRPF_ERR_NOMEM;
  std::string err;
  int rc;
  try {
    rc = nrpf::build_plan(n, rowptr, colidx, y_re, y_im, bus_type, o.ordering, o.dense_frac, o.panel,
                          o.order_tries, sparse_weight, p->hp, err);
  } catch (const std::bad_alloc&) {
    rc = NRPF_ERR_NOMEM;
  } catch (...) {
    rc = NRPF_ERR_ARG;
  }
  if (rc) {
    delete p;
    return rc;
  }
  p->lu_precision = o.lu_precision;
  p->host_only = o.host_only != 0;
  // instance-major dense block: FP32 blocks large enough for the CTA-tiled
  // kernels to pay (a 128 x 128 tile of C per CTA)
  p->dp.dim = o.dense_layout == NRPF_DENSE_INSTANCE_MAJOR ||
              (o.dense_layout == NRPF_DENSE_AUTO && im_ok && p->hp.nd >= NRPF_DENSE_IM_MIN);
  if (p->host_only) {
    *out = p;
    return NRPF_OK;
  }
  cudaGetDevice(&p->device);
  const HostPlan& h = p->hp;
  DevPlan& d = p->dp;
  d.n = h.n; d.m = h.m; d.s = h.s; d.nd = h.nd; d.ndp = h.ndp; d.kb = h.kb; d.mp = h.s + h.ndp;
  d.NS = h.NS; d.NLU = h.NLU; d.nnzY = (int)h.colidx.size();
  d.n_one = (int)h.one_pos.size();
  d.n_lu_lvl = (int)h.lu_lvl_ptr.size() - 1;
  d.n_fw_lvl = (int)h.fw_lvl_ptr.size() - 1;
  d.n_bw_lvl = (int)h.bw_lvl_ptr.size() - 1;
  std::vector<int32_t> ydiag(h.n);
  for (int i = 0; i < h.n; ++i)
    for (int q = h.rowptr[i]; q < h.rowptr[i + 1]; ++q)
      if (h.colidx[q] == i) ydiag[i] = q;
  std::vector<nrpf::DevUpd> upd(h.upd.size());
  for (size_t u = 0; u < h.upd.size(); ++u)
    upd[u] = nrpf::DevUpd{h.upd[u].ukj, h.upd[u].lsrc, h.upd[u].llen, h.upd[u].dst_off};
  if ((rc = upload(p, h.rowptr, &d.rowptr)) || (rc = upload(p, h.colidx, &d.colidx)) ||
      (rc = upload(p, h.yre, &d.yre)) || (rc = upload(p, h.yim, &d.yim)) ||
      (rc = upload(p, ydiag, &d.ydiag)) || (rc = upload(p, h.bus_type, &d.bus_type)) ||
      (rc = upload(p, h.jmap, &d.jmap)) || (rc = upload(p, h.rhs_pos_p, &d.rhs_p)) ||
      (rc = upload(p, h.rhs_pos_q, &d.rhs_q)) || (rc = upload(p, h.one_pos, &d.one_pos)) ||
      (rc = upload(p, h.lu_lvl_cols, &d.lu_cols)) || (rc = upload(p, h.col_upd_ptr, &d.col_upd_ptr)) ||
      (rc = upload(p, upd, &d.upd)) || (rc = upload(p, h.dst, &d.dst)) || (rc = upload(p, h.dp, &d.dp)) ||
      (rc = upload(p, h.ce, &d.ce)) || (rc = upload(p, h.fw_rows, &d.fw_rows)) ||
      (rc = upload(p, h.fw_ptr, &d.fw_ptr)) || (rc = upload(p, h.fw_pos, &d.fw_pos)) ||
      (rc = upload(p, h.fw_col, &d.fw_col)) || (rc = upload(p, h.bw_rows, &d.bw_rows)) ||
      (rc = upload(p, h.bw_ptr, &d.bw_ptr)) || (rc = upload(p, h.bw_pos, &d.bw_pos)) ||
      (rc = upload(p, h.bw_col, &d.bw_col)) || (rc = upload(p, h.unk_pos, &d.unk_pos)) ||
      (rc = upload(p, h.lu_lvl_ptr, &d.lu_lvl_ptr)) || (rc = upload(p, h.fw_lvl_ptr, &d.fw_lvl_ptr)) ||
      (rc = upload(p, h.bw_lvl_ptr, &d.bw_lvl_ptr)) || (rc = upload(p, h.schur_u, &d.schur_u)) ||
      (rc = upload(p, h.schur_ent, &d.schur_ent))) {
    pf_plan_destroy(p);
    return rc;
  }
  {
    const int32_t* tasks = nullptr;
    if ((rc = upload(p, h.schur_task, &tasks)) || (rc = upload(p, h.schur_jmask, &d.schur_jmask))) {
      pf_plan_destroy(p);
      return rc;
    }
    d.schur_task = reinterpret_cast<const int4*>(tasks);
    d.n_schur = (int)(h.schur_task.size() / 4);
  }
  if (o.max_batch > 0 && (rc = ensure_capacity(p, o.max_batch))) {
    pf_plan_destroy(p);
    return rc;
  }
  *out = p;
  return NRPF_OK;
}

int pf_plan_get_info(const pf_plan* p, pf_plan_info* info) {
  if (!p || !info) return NRPF_ERR_ARG;
  const HostPlan& h = p->hp;
  info->n = h.n;
  info->m = h.m;
  info->n_pv = h.npv;
  info->n_pq = h.npq;
  info->n_slack = h.nslack;
  info->nnz_ybus = (int64_t)h.colidx.size();
  info->nnz_j = h.nnz_j;
  info->nnz_lu = h.NLU;
  info->sparse_cols = h.s;
  info->dense_dim = h.nd;
  info->dense_pad = h.ndp;
  info->lu_levels = (int)h.lu_lvl_ptr.size() - 1;
  info->fwd_levels = (int)h.fw_lvl_ptr.size() - 1;
  info->bwd_levels = (int)h.bw_lvl_ptr.size() - 1;
  info->lu_fma = h.lu_fma;
  info->solve_fma = h.solve_fma;
  info->capacity = p->capacity;
  info->lu_precision = p->lu_precision;
  info->panel = h.kb;
  info->order_seed = (int)h.order_seed;
  info->order_key = h.order_key;
  info->dense_layout = p->dp.dim ? NRPF_DENSE_INSTANCE_MAJOR : NRPF_DENSE_INTERLEAVED;
  return NRPF_OK;
}

int pf_plan_get_pattern(const pf_plan* p, int32_t* pos_of_unknown, int64_t* colptr, int32_t* rowidx,
                        int64_t* nnz_out) {
  if (!p) return NRPF_ERR_ARG;
  const HostPlan& h = p->hp;
  if (pos_of_unknown) std::copy(h.unk_pos.begin(), h.unk_pos.end(), pos_of_unknown);
  int64_t q = 0;
  if (colptr) colptr[0] = 0;
  for (int j = 0; j < h.m; ++j) {
    for (int64_t e = h.cs[j]; e < h.ce[j]; ++e) {
      if (rowidx) rowidx[q] = h.seg_row[e];
      ++q;
    }
    if (j >= h.s)
      for (int r = h.s; r < h.m; ++r) {
        if (rowidx) rowidx[q] = r;
        ++q;
      }
    if (colptr) colptr[j + 1] = q;
  }
  if (nnz_out) *nnz_out = q;
  return NRPF_OK;
}

int pf_solve_batch(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                   double* v_out, int32_t* iters, uint8_t* status, void* stream) {
  if (!p || p->host_only || B < 0 || maxit < 0 || !std::isfinite(tol) || tol < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (p->lu_precision == NRPF_LU_FP32)
    rc = enqueue_solve<float>(p, B, nullptr, sbus, v0, tol, maxit, v_out, iters, status, st);
  else
    rc = enqueue_solve<double>(p, B, nullptr, sbus, v0, tol, maxit, v_out, iters, status, st);
  if (rc) return rc;
  return check_launch();
}

int pf_solve_batch_y(pf_plan* p, int B, const double* ybus, const double* sbus, const double* v0, double tol,
                     int maxit, double* v_out, int32_t* iters, uint8_t* status, void* stream) {
  if (!p || p->host_only || B < 0 || maxit < 0 || !std::isfinite(tol) || tol < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!ybus || !sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (p->lu_precision == NRPF_LU_FP32)
    rc = enqueue_solve<float>(p, B, ybus, sbus, v0, tol, maxit, v_out, iters, status, st);
  else
    rc = enqueue_solve<double>(p, B, ybus, sbus, v0, tol, maxit, v_out, iters, status, st);
  if (rc) return rc;
  return check_launch();
}

int pf_plan_set_branches(pf_plan* p, int nbr, const int32_t* f, const int32_t* t, const double* r, const double* x,
                         const double* b) {
  if (!p || p->host_only || nbr < 0 || (nbr > 0 && (!f || !t || !r || !x || !b))) return NRPF_ERR_ARG;
  const HostPlan& h = p->hp;
  auto find = [&](int i, int k) -> int {
    const int32_t* lo = h.colidx.data() + h.rowptr[i];
    const int32_t* hi = h.colidx.data() + h.rowptr[i + 1];
    const int32_t* q = std::lower_bound(lo, hi, k);
    return (q != hi && *q == k) ? (int)(q - h.colidx.data()) : -1;
  };
  std::vector<int4> pos(nbr);
  std::vector<double> val((size_t)nbr * 3);
  for (int e = 0; e < nbr; ++e) {
    const int a = f[e], c = t[e];
    if (a < 0 || a >= h.n || c < 0 || c >= h.n) return NRPF_ERR_ARG;
    const double den = r[e] * r[e] + x[e] * x[e];
    if (!(den > 0.0) || !std::isfinite(den) || !std::isfinite(b[e])) return NRPF_ERR_ARG;
    pos[e] = make_int4(find(a, a), find(c, c), find(a, c), find(c, a));
    if (pos[e].x < 0 || pos[e].y < 0 || pos[e].z < 0 || pos[e].w < 0) return NRPF_ERR_PATTERN;
    val[3 * e] = r[e] / den;
    val[3 * e + 1] = -x[e] / den;
    val[3 * e + 2] = 0.5 * b[e];
  }
  CK(cudaDeviceSynchronize());
  if (p->d_bpos) cudaFree(p->d_bpos);
  if (p->d_bval) cudaFree(p->d_bval);
  p->d_bpos = nullptr;
  p->d_bval = nullptr;
  p->nbr = 0;
  CK(cudaMalloc(&p->d_bpos, std::max<size_t>(pos.size() * sizeof(int4), 16)));
  CK(cudaMalloc(&p->d_bval, std::max<size_t>(val.size() * sizeof(double), 16)));
  if (nbr > 0) {
    CK(cudaMemcpy(p->d_bpos, pos.data(), pos.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_bval, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  p->nbr = nbr;
  return NRPF_OK;
}

int pf_solve_batch_outages(pf_plan* p, int B, const int32_t* outages, int k, const double* sbus, const double* v0,
                           double tol, int maxit, double* v_out, int32_t* iters, uint8_t* status, void* stream) {
  if (!p || p->host_only || B < 0 || k < 0 || maxit < 0 || !std::isfinite(tol) || tol < 0 || !p->d_bpos)
    return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if ((k > 0 && !outages) || !sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (p->lu_precision == NRPF_LU_FP32)
    rc = enqueue_solve<float>(p, B, nullptr, sbus, v0, tol, maxit, v_out, iters, status, st, outages, k);
  else
    rc = enqueue_solve<double>(p, B, nullptr, sbus, v0, tol, maxit, v_out, iters, status, st, outages, k);
  if (rc) return rc;
  return check_launch();
}

int pf_ybus_values(int n, int nbr, const int32_t* f, const int32_t* t, const double* r, const double* x,
                   const double* b, int B, const uint8_t* in_service, const int32_t* rowptr,
                   const int32_t* colidx, double* y) {
  if (n <= 0 || nbr < 0 || B < 0 || !rowptr || !y) return NRPF_ERR_ARG;
  if (nbr > 0 && (!f || !t || !r || !x || !b)) return NRPF_ERR_ARG;
  const int64_t nnz = rowptr[n];
  if (rowptr[0] != 0 || nnz < 0 || (nnz > 0 && !colidx)) return NRPF_ERR_ARG;
  // pattern position of (i, k): binary search in row i's sorted columns
  auto find = [&](int i, int k) -> int64_t {
    const int32_t* lo = colidx + rowptr[i];
    const int32_t* hi = colidx + rowptr[i + 1];
    const int32_t* q = std::lower_bound(lo, hi, k);
    return (q != hi && *q == k) ? (int64_t)(q - colidx) : -1;
  };
  struct Stamp {
    int64_t ff, tt, ft, tf;
    double gs, bs, bh;
  };
  std::vector<Stamp> st(nbr);
  for (int e = 0; e < nbr; ++e) {
    const int a = f[e], c = t[e];
    if (a < 0 || a >= n || c < 0 || c >= n) return NRPF_ERR_ARG;
    const double den = r[e] * r[e] + x[e] * x[e];
    if (!(den > 0.0) || !std::isfinite(den) || !std::isfinite(b[e])) return NRPF_ERR_ARG;
    Stamp s{find(a, a), find(c, c), find(a, c), find(c, a), r[e] / den, -x[e] / den, 0.5 * b[e]};
    if (s.ff < 0 || s.tt < 0 || s.ft < 0 || s.tf < 0) return NRPF_ERR_PATTERN;
    st[e] = s;
  }
  for (int k = 0; k < B; ++k) {
    double* yk = y + (size_t)k * nnz * 2;
    std::fill(yk, yk + nnz * 2, 0.0);
    const uint8_t* ins = in_service ? in_service + (size_t)k * nbr : nullptr;
    for (int e = 0; e < nbr; ++e) {
      if (ins && !ins[e]) continue;
      const Stamp& s = st[e];
      yk[2 * s.ff] += s.gs;
      yk[2 * s.ff + 1] += s.bs + s.bh;
      yk[2 * s.tt] += s.gs;
      yk[2 * s.tt + 1] += s.bs + s.bh;
      yk[2 * s.ft] -= s.gs;
      yk[2 * s.ft + 1] -= s.bs;
      yk[2 * s.tf] -= s.gs;
      yk[2 * s.tf + 1] -= s.bs;
    }
  }
  return NRPF_OK;
}

int pf_solve_batch_host(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                        double* v_out, int32_t* iters, uint8_t* status, int chunk, void* stream) {
  if (!p || p->host_only || B < 0 || maxit < 0 || chunk < 0 || !std::isfinite(tol) || tol < 0)
    return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  if (chunk == 0 || chunk > B) chunk = B;
  const int n = p->hp.n;
  int rc = ensure_capacity(p, chunk);
  if (rc) return rc;
  // staging slot layout: sbus, v0, v_out [chunk, n] complex; iters [chunk]; status [chunk]
  const size_t cplx = (size_t)n * 16;
  auto slot_bytes = [&](int c) { return (size_t)c * (3 * cplx + 4 + 1) + 256; };
  if (chunk > p->stage_cap) {
    CK(cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i) {
      if (p->stage_mem[i]) cudaFree(p->stage_mem[i]);
      p->stage_mem[i] = nullptr;
    }
    p->stage_cap = 0;
    p->slot_used[0] = p->slot_used[1] = false;
    for (int i = 0; i < 2; ++i) CK(cudaMalloc(&p->stage_mem[i], slot_bytes(chunk)));
    p->stage_cap = chunk;
  }
  if (!p->in_stream) {
    CK(cudaStreamCreateWithFlags(&p->in_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&p->out_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CK(cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->ev_out[i], cudaEventDisableTiming));
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t is = p->in_stream, os = p->out_stream;
  const size_t cap = (size_t)p->stage_cap;
  struct Slot {
    double *s, *v0, *v;
    int32_t* it;
    uint8_t* st;
  } slot[2];
  for (int i = 0; i < 2; ++i) {
    char* base = reinterpret_cast<char*>(p->stage_mem[i]);
    slot[i] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + cap * cplx),
               reinterpret_cast<double*>(base + 2 * cap * cplx), reinterpret_cast<int32_t*>(base + 3 * cap * cplx),
               reinterpret_cast<uint8_t*>(base + 3 * cap * cplx + cap * 4)};
  }
  const int nch = (B + chunk - 1) / chunk;
  auto first = [&](int c) { return (size_t)c * chunk; };
  auto count = [&](int c) { return (int)std::min<size_t>(chunk, B - first(c)); };
  // chunk c's inputs into staging slot i (copy-in stream), once the chunk
  // that used the slot before has been copied out
  auto copy_in = [&](int c, int i) -> cudaError_t {
    const Slot& d = slot[i];
    cudaError_t e = cudaSuccess;
    if (p->slot_used[i]) e = cudaStreamWaitEvent(is, p->ev_out[i], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d.s, sbus + first(c) * 2 * n, count(c) * cplx, cudaMemcpyHostToDevice, is);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d.v0, v0 + first(c) * 2 * n, count(c) * cplx, cudaMemcpyHostToDevice, is);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[i], is);
    return e;
  };
  int i = p->slot_next;
  CK(copy_in(0, i));
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) CK(copy_in(c + 1, i ^ 1));
    CK(cudaStreamWaitEvent(st, p->ev_in[i], 0));
    const Slot& d = slot[i];
    if (p->lu_precision == NRPF_LU_FP32)
      rc = enqueue_solve<float>(p, count(c), nullptr, d.s, d.v0, tol, maxit, d.v, d.it, d.st, st);
    else
      rc = enqueue_solve<double>(p, count(c), nullptr, d.s, d.v0, tol, maxit, d.v, d.it, d.st, st);
    if (rc) return rc;
    CK(cudaEventRecord(p->ev_done[i], st));
    CK(cudaStreamWaitEvent(os, p->ev_done[i], 0));
    CK(cudaMemcpyAsync(v_out + first(c) * 2 * n, d.v, count(c) * cplx, cudaMemcpyDeviceToHost, os));
    CK(cudaMemcpyAsync(iters + first(c), d.it, count(c) * 4, cudaMemcpyDeviceToHost, os));
    CK(cudaMemcpyAsync(status + first(c), d.st, count(c), cudaMemcpyDeviceToHost, os));
    CK(cudaEventRecord(p->ev_out[i], os));
    p->slot_used[i] = true;
    i ^= 1;
  }
  p->slot_next = i;
  // later work on the caller's stream follows the last copy out (the copy-out
  // stream is in order, so this covers every chunk)
  CK(cudaStreamWaitEvent(st, p->ev_out[i ^ 1], 0));
  return check_launch();
}

int pf_stage_mismatch(pf_plan* p, int B, const double* sbus, const double* v, double* F, double* norm,
                      void* stream) {
  if (!p || p->host_only || B < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v || !F || !norm) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  nrpf::launch_load(p->dp, p->st, B, sbus, v, st);
  if (p->lu_precision == NRPF_LU_FP32) {
    nrpf::launch_mismatch<float>(p->dp, p->st, 0, nullptr, st);
    nrpf::launch_f_out<float>(p->dp, p->st, B, F, norm, st);
  } else {
    nrpf::launch_mismatch<double>(p->dp, p->st, 0, nullptr, st);
    nrpf::launch_f_out<double>(p->dp, p->st, B, F, norm, st);
  }
  return check_launch();
}

int pf_stage_factor(pf_plan* p, int B, const double* v, int factor, double* lu_out, void* stream) {
  if (!p || p->host_only || B < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!v || !lu_out) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  if ((rc = build_pattern_map(p))) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the specified injections do not enter J: reuse v as a harmless sbus
  nrpf::launch_load(p->dp, p->st, B, v, v, st);
  if (p->hp.m == 0) return check_launch();
  if (p->lu_precision == NRPF_LU_FP32) {
    enqueue_factor<float>(p, factor, st);
    nrpf::launch_lu_out<float>(p->dp, p->st, B, p->d_pattern_map, p->pattern_nnz, lu_out, st);
  } else {
    enqueue_factor<double>(p, factor, st);
    nrpf::launch_lu_out<double>(p->dp, p->st, B, p->d_pattern_map, p->pattern_nnz, lu_out, st);
  }
  return check_launch();
}

int pf_stage_linear_solve(pf_plan* p, int B, const double* v, const double* rhs, double* dx, void* stream) {
  if (!p || p->host_only || B < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!v || !rhs || !dx) return NRPF_ERR_ARG;
  int rc = ensure_capacity(p, B);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  nrpf::launch_load(p->dp, p->st, B, v, v, st);
  if (p->hp.m == 0) return check_launch();
  if (p->lu_precision == NRPF_LU_FP32) {
    enqueue_factor<float>(p, 1, st);
    nrpf::launch_rhs_in<float>(p->dp, p->st, B, rhs, st);
    nrpf::launch_solve<float>(p->dp, p->st, p->hp.fw_lvl_ptr, p->hp.bw_lvl_ptr, nullptr, st);
    nrpf::launch_rhs_out<float>(p->dp, p->st, B, dx, st);
  } else {
    enqueue_factor<double>(p, 1, st);
    nrpf::launch_rhs_in<double>(p->dp, p->st, B, rhs, st);
    nrpf::launch_solve<double>(p->dp, p->st, p->hp.fw_lvl_ptr, p->hp.bw_lvl_ptr, nullptr, st);
    nrpf::launch_rhs_out<double>(p->dp, p->st, B, dx, st);
  }
  return check_launch();
}

int pf_profile_start(pf_plan* p, uint32_t time_mask) {
  if (!p || p->host_only) return NRPF_ERR_ARG;
  fold_graph_launches(p);
  p->rec.reset(time_mask);
  return NRPF_OK;
}

int pf_profile_read(pf_plan* p, pf_profile* out) {
  if (!p || !out || p->host_only) return NRPF_ERR_ARG;
  p->rec.drain();
  fold_graph_launches(p);
  static_assert(nrpf::K_NCLASS <= NRPF_KCLASSES, "kernel class table too small");
  for (int c = 0; c < NRPF_KCLASSES; ++c) {
    out->launches[c] = c < nrpf::K_NCLASS ? p->rec.launches[c] : 0;
    out->timed[c] = c < nrpf::K_NCLASS ? p->rec.timed[c] : 0;
    out->ms[c] = c < nrpf::K_NCLASS ? p->rec.ms[c] : 0.0;
  }
  return check_launch();
}

const char* pf_kernel_class_name(int c) {
  static const char* names[] = {"load", "store", "mismatch_jacobian", "check", "zero_lu", "set_ones",
                                "lu_sparse_level", "dense_diag", "dense_panel", "dense_update", "fwd_level",
                                "dense_solve", "bwd_level", "update", "aux", "lu_schur"};
  if (c < 0 || c >= nrpf::K_NCLASS) return "unknown";
  return names[c];
}

void pf_plan_destroy(pf_plan* p) {
  if (!p) return;
  if (p->host_only) {
    delete p;
    return;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  free_ws(p);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  if (p->yv_mem) cudaFree(p->yv_mem);
  if (p->d_bpos) cudaFree(p->d_bpos);
  if (p->d_bval) cudaFree(p->d_bval);
  for (int i = 0; i < 2; ++i) {
    if (p->stage_mem[i]) cudaFree(p->stage_mem[i]);
    if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
    if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
    if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
  }
  if (p->in_stream) cudaStreamDestroy(p->in_stream);
  if (p->out_stream) cudaStreamDestroy(p->out_stream);
  if (p->h_prev) cudaFreeHost(p->h_prev);
  for (void* a : p->plan_allocs) cudaFree(a);
  if (p->d_pattern_map) cudaFree(p->d_pattern_map);
  if (cur != p->device) cudaSetDevice(cur);
  delete p;
}

const char* pf_status_str(int code) {
  switch (code) {
    case NRPF_OK: return "ok";
    case NRPF_ERR_ARG: return "invalid argument";
    case NRPF_ERR_PATTERN: return "invalid Ybus pattern or bus types";
    case NRPF_ERR_NOMEM: return "out of memory";
    case NRPF_ERR_CUDA: return "CUDA runtime error";
    case NRPF_ERR_CAPACITY: return "batch exceeds plan capacity";
    default: return "unknown";
  }
}

}  // extern "C"
