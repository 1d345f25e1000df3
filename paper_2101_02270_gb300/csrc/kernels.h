// Launchers of the batched Newton-Raphson kernels (kernels.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "device.h"
#include "recorder.h"

#define NRPF_CONVERGED_CODE 0
#define NRPF_MAXIT_CODE 1
#define NRPF_FAILED_CODE 2

namespace nrpf {

void launch_load(const DevPlan& P, const DevState& S, int B, const double* sbus, const double* v0,
                 cudaStream_t st, Recorder* rec = nullptr);
void launch_store(const DevPlan& P, const DevState& S, int B, double* v_out, int32_t* iters,
                  uint8_t* status, cudaStream_t st, Recorder* rec = nullptr);
// gates of the Newton loop (addresses inside the device control block)
inline const int32_t* ctl_prev(const DevState& S) {
  return reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(S.ctl) + offsetof(SolveCtl, prev));
}
inline const int32_t* ctl_cur(const DevState& S) {
  return reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(S.ctl) + offsetof(SolveCtl, cur));
}

// Per-instance Ybus values [B, nnzY] complex into S.yv (interleaved).
void launch_load_y(const DevPlan& P, const DevState& S, int B, const double* y, cudaStream_t st,
                   Recorder* rec = nullptr);

// Per-instance Ybus values of outage cases into S.yv: the plan's base values
// minus the stamps of each instance's outaged branches (outages [B, k]).
void launch_outage_y(const DevPlan& P, const DevState& S, int B, const int32_t* outages, int k, const int4* bpos,
                     const double* bval, int nbr, cudaStream_t st, Recorder* rec = nullptr);

// Reset the loop control (prev = 1, cur = 0, it = 0) with the tolerance and
// iteration limit of this solve.
void launch_ctl_init(const DevState& S, int maxit, double tol, cudaStream_t st, Recorder* rec = nullptr);
// Convergence test of iteration ctl->it: counts the instances still active
// into ctl->cur.
void launch_check(const DevState& S, cudaStream_t st, Recorder* rec = nullptr);
// End of one iteration: prev = cur, cur = 0, it += 1; with a graph handle
// (graph != 0), also sets the loop's condition to (cur > 0 && it < maxit).
void launch_iter_tail(const DevState& S, cudaGraphConditionalHandle cond, int graph, cudaStream_t st,
                      Recorder* rec = nullptr);

template <typename T>
void launch_mismatch(const DevPlan& P, const DevState& S, int jac, const int32_t* gate, cudaStream_t st,
                     Recorder* rec = nullptr);
template <typename T>
// Zero the LU workspace (whole = false: only the sparse segments; the
// refactorisation then writes every position of the dense block) and set the
// identity padding of the dense block.
void launch_prepare_lu(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                       Recorder* rec = nullptr, bool whole = true);
template <typename T>
void launch_factor(const DevPlan& P, const DevState& S, const std::vector<int32_t>& lvl_ptr,
                   const int32_t* gate, cudaStream_t st, Recorder* rec = nullptr);
template <typename T>
void launch_solve(const DevPlan& P, const DevState& S, const std::vector<int32_t>& fw_lvl,
                  const std::vector<int32_t>& bw_lvl, const int32_t* gate, cudaStream_t st,
                  Recorder* rec = nullptr);
template <typename T>
void launch_update(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                   Recorder* rec = nullptr);
template <typename T>
void launch_rhs_in(const DevPlan& P, const DevState& S, int B, const double* rhs, cudaStream_t st);
template <typename T>
void launch_rhs_out(const DevPlan& P, const DevState& S, int B, double* dx, cudaStream_t st);
template <typename T>
void launch_f_out(const DevPlan& P, const DevState& S, int B, double* F, double* norm, cudaStream_t st);
template <typename T>
void launch_lu_out(const DevPlan& P, const DevState& S, int B, const int64_t* map, int64_t nnz, double* out,
                   cudaStream_t st);

}  // namespace nrpf
