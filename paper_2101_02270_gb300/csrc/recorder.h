// Launch bookkeeping: counts every kernel the library enqueues and, for the
// kernel classes selected by a mask, brackets each launch with CUDA events on
// the launching stream so that per-kernel device time can be read back.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace nrpf {

enum KClass : int {
  K_LOAD = 0, K_STORE, K_MISMATCH, K_CHECK, K_ZERO, K_ONES, K_LU_SPARSE, K_DENSE_DIAG,
  K_DENSE_PANEL, K_DENSE_UPDATE, K_FWD, K_DENSE_SOLVE, K_BWD, K_UPDATE, K_AUX, K_SCHUR, K_NCLASS
};

struct Recorder {
  int64_t launches[K_NCLASS] = {};
  int64_t timed[K_NCLASS] = {};
  double ms[K_NCLASS] = {};
  uint32_t time_mask = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;

  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void pre(int c, cudaStream_t st) {
    launches[c]++;
    if (time_mask >> c & 1u) {
      cudaEvent_t a = get(), b = get();
      cudaEventRecord(a, st);
      pending.push_back({c, {a, b}});
    }
  }
  void post(int c, cudaStream_t st) {
    if (time_mask >> c & 1u) cudaEventRecord(pending.back().second.second, st);
  }
  // Wait for the recorded events and fold their times into ms[].
  void drain() {
    for (auto& p : pending) {
      cudaEventSynchronize(p.second.second);
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) {
        ms[p.first] += t;
        timed[p.first]++;
      }
    }
    pending.clear();
    used = 0;
  }
  void reset(uint32_t mask) {
    drain();
    for (int c = 0; c < K_NCLASS; ++c) { launches[c] = 0; timed[c] = 0; ms[c] = 0.0; }
    time_mask = mask;
  }
  ~Recorder() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// Bracket one launch statement.
#define NRPF_LAUNCH(rec, cls, st, ...) \
  do {                                 \
    if (rec) (rec)->pre((cls), (st));  \
    __VA_ARGS__;                       \
    if (rec) (rec)->post((cls), (st)); \
  } while (0)

}  // namespace nrpf
