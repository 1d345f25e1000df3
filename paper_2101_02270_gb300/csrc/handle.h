// The opaque plan handle of the C ABI (internal definition, shared by the
// translation units that implement entry points).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/nrpf.h"
#include "device.h"
#include "plan.h"
#include "recorder.h"

struct pf_plan {
  nrpf::HostPlan hp;
  nrpf::DevPlan dp{};
  nrpf::DevState st{};
  int capacity = 0;  // instances (multiple of kTile)
  int lu_precision = NRPF_LU_FP64;
  int device = 0;
  int host_only = 0;
  std::vector<void*> plan_allocs;
  std::vector<void*> ws_allocs;
  int64_t* d_pattern_map = nullptr;  // CCS pattern -> LU element
  int64_t pattern_nnz = 0;
  nrpf::Recorder rec;
  // Newton loop as a graph: one iteration captured as the body of a WHILE
  // node whose condition the iteration's last kernel sets (built per
  // workspace; launches of one body by kernel class, for the counters)
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  int64_t body_launches[nrpf::K_NCLASS] = {};
  int32_t* h_prev = nullptr;  // pinned: ctl->prev read back by profiled solves
};
