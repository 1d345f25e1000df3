// Launchers of the batched Newton-Raphson kernels (kernels.cu).
#pragma once
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
void launch_check(const DevState& S, int it, int maxit, double tol, int32_t* counter, cudaStream_t st,
                  Recorder* rec = nullptr);

template <typename T>
void launch_mismatch(const DevPlan& P, const DevState& S, int jac, const int32_t* gate, cudaStream_t st,
                     Recorder* rec = nullptr);
template <typename T>
void launch_prepare_lu(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                       Recorder* rec = nullptr);
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
