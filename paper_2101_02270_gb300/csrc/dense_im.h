// Instance-major dense block (FP32 LU): the trailing dense block of every
// instance stored as its own column-major ndp x ndp matrix, factorised by
// per-instance kernels whose trailing update is a CTA-tiled product with
// operand tiles staged in shared memory by TMA (dense_im.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "device.h"
#include "recorder.h"

namespace nrpf {

// TMA descriptors of one workspace's dense blocks, viewed as a 4-D tensor
// (row, column, lane, tile) of float32 with strides (4 B, 4 ndp B,
// 4 ndp^2 B, 128 NLU B).  a: boxes of 128 rows x 32 columns (no swizzle),
// the L21 operand; b: boxes of 32 rows x 128 columns with 128-byte swizzle,
// the U12 operand.
struct DenseImMaps {
  CUtensorMap a;
  CUtensorMap b;
};

// Encode the maps for the dense blocks of a workspace of Bp instances
// (lu = the workspace's LU array).  Returns false when the driver's tensor-map
// encoder is unavailable or rejects the shape.
bool make_dense_im_maps(const DevPlan& P, void* lu, int Bp, DenseImMaps* out);

// Blocked LU without pivoting of every active instance's dense block, left-
// looking by outer panels of 128: each panel's block column and row first
// take the products of all earlier panels (one update of depth 128 j for
// panel j), then the panel is factorised in two 64-wide steps.
void launch_dense_im_factor(const DevPlan& P, const DevState& S, const DenseImMaps& maps, const int32_t* gate,
                            cudaStream_t st, Recorder* rec);

// Identity on the padding columns nd .. ndp-1 of every instance's dense block
// and zero right-hand side on its padding rows (one CTA per instance).
void launch_dense_im_set_ones(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                              Recorder* rec);

// Forward (unit lower) and backward (upper) substitution of the dense block,
// one CTA per instance, right-hand side rows s .. s+ndp-1 of S.x.
void launch_dense_im_solve(const DevPlan& P, const DevState& S, const int32_t* gate, cudaStream_t st,
                           Recorder* rec);

}  // namespace nrpf
