// The opaque plan handle of the C ABI (internal definition, shared by the
// translation units that implement entry points).
#pragma once
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/nrpf.h"
#include "dense_im.h"
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
  nrpf::DenseImMaps im_maps{};       // TMA descriptors of the workspace (instance-major dense block)
  int64_t pattern_nnz = 0;
  nrpf::Recorder rec;
  // Newton loop as a graph: one iteration captured as the body of a WHILE
  // node whose condition the iteration's last kernel sets (built per
  // workspace; launches of one body by kernel class, for the counters)
  struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  std::map<int, LoopGraph> loops;  // by 2 x padded batch + per-instance Ybus flag
  cudaStream_t capture_stream = nullptr;
  int64_t body_launches[nrpf::K_NCLASS] = {};
  int32_t* h_prev = nullptr;  // pinned: ctl->prev read back by profiled solves
  // host-resident batches: two device staging slots of stage_cap instances,
  // a copy stream and the events that order copies and solves
  int stage_cap = 0;
  void* stage_mem[2] = {nullptr, nullptr};
  cudaStream_t in_stream = nullptr;   // copies host -> device
  cudaStream_t out_stream = nullptr;  // copies device -> host
  cudaEvent_t ev_in[2] = {nullptr, nullptr};     // slot's inputs copied in
  cudaEvent_t ev_done[2] = {nullptr, nullptr};   // slot's chunk solved
  cudaEvent_t ev_out[2] = {nullptr, nullptr};    // slot's results copied out
  void* yv_mem = nullptr;  // per-instance Ybus values, capacity x nnzY complex
  // branch stamps for device-built outage cases: per branch the pattern
  // positions of (f,f), (t,t), (f,t), (t,f) and (series G, series B, half
  // charging)
  int nbr = 0;
  int4* d_bpos = nullptr;
  double* d_bval = nullptr;  // [nbr * 3]
  int yv_cap = 0;
  int slot_next = 0;                            // staging slot of the next chunk
  bool slot_used[2] = {false, false};           // slot holds a chunk whose copy-out was enqueued
};
