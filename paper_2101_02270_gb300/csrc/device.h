// Device-side plan and per-solve state shared by the kernels and the C ABI.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace nrpf {

// Instances are interleaved in tiles of kTile (Sec. 3.1, Fig. 1d: element-major,
// batch contiguous): element e of instance b lives at
//   ((b / kTile) * E + e) * kTile + (b % kTile)
// for an array holding E elements per instance.  A warp of 32 lanes covers one
// tile, so every per-element access of a warp is one contiguous 256-byte
// (float64) or 128-byte (float32) segment.
constexpr int kTile = 32;

struct DevUpd {
  int32_t ukj, lsrc, llen, dst_off;
};

// Read-only plan arrays on the device (copied once by pf_plan_create).
struct DevPlan {
  int n, m, s, nd, ndp, kb, mp;  // mp = s + ndp (rhs length incl. padding)
  int dim;  // 1: instance-major dense block (FP32 LU; see dense_im.h), 0: interleaved
  int64_t NS, NLU;
  int nnzY;
  const int32_t* rowptr;   // [n+1]
  const int32_t* colidx;   // [nnzY]
  const double* yre;       // [nnzY]
  const double* yim;       // [nnzY]
  const int32_t* ydiag;    // [n] index of the diagonal entry in row i
  const int8_t* bus_type;  // [n]
  const int32_t* jmap;     // [nnzY*4]
  const int32_t* rhs_p;    // [n] A row of the P equation (-1 for slack)
  const int32_t* rhs_q;    // [n] A row of the Q equation (-1 unless PQ)
  const int32_t* one_pos;  // [ndp-nd]
  int n_one;
  // sparse refactor
  const int32_t* lu_cols;      // columns grouped by level
  const int32_t* col_upd_ptr;  // [m+1]
  const DevUpd* upd;
  const int32_t* dst;
  const int32_t* dp;           // [m] diagonal position (-1 for dense columns)
  const int64_t* ce;           // [m] segment end
  // Schur complement of the sparse columns into the dense block
  const int4* schur_task;     // {dense column, 32-row chunk, first entry, end}
  const int32_t* schur_ent;   // (L(i, k) position << 5) | row in chunk
  const int32_t* schur_u;     // U(k, j) position of the entry
  const uint32_t* schur_jmask; // rows of the chunk holding a Jacobian entry
  int n_schur;
  // FS/BS
  const int32_t* fw_rows; const int32_t* fw_ptr; const int32_t* fw_pos; const int32_t* fw_col;
  const int32_t* bw_rows; const int32_t* bw_ptr; const int32_t* bw_pos; const int32_t* bw_col;
  const int32_t* unk_pos;  // [m]
  // level boundaries of the schedules (device copies, for fused kernels)
  const int32_t* lu_lvl_ptr; int n_lu_lvl;
  const int32_t* fw_lvl_ptr; int n_fw_lvl;
  const int32_t* bw_lvl_ptr; int n_bw_lvl;
};

// Per-solve workspace (capacity Bp instances, a multiple of kTile).
// Device-resident control of the Newton loop, so that one iteration can run
// unchanged from a graph: every kernel of an iteration reads its gate and the
// iteration number here.
struct SolveCtl {
  int32_t prev;     // instances active after the previous check: gate of the
                    // LU preparation and mismatch (nonzero before the first)
  int32_t cur;      // instances active after this iteration's check: gate of
                    // factorisation, FS/BS and update
  int32_t it;       // Newton iteration of the check
  int32_t maxit;
  double tol;
  long long graph_iters;  // loop bodies run by the graph since the last reset
};

struct DevState {
  int Bp;
  double* vm;    // [n] magnitudes
  double* va;    // [n] angles
  double* ve;    // [n] real part
  double* vf;    // [n] imaginary part
  double* vinv;  // [n] 1/|V|
  double* psp;   // [n] specified P
  double* qsp;   // [n] specified Q
  void* x;       // [mp] right-hand side / solution (LU precision)
  void* lu;      // [NLU] LU values (LU precision)
  void* inv;     // [kb] inverse pivots of the current dense diagonal block
  unsigned long long* norm;  // [Bp] max |F| as float64 bits
  int32_t* iters;   // [Bp]
  int32_t* status;  // [Bp]
  int32_t* active;  // [Bp]
  int32_t* bad;     // [Bp] non-finite step detected
  SolveCtl* ctl;  // Newton loop control (one per workspace)
  const double2* yv;  // [nnzY] per-instance Ybus values (re, im), or null: the plan's shared values
  const void* im_maps;  // host pointer to the workspace's DenseImMaps (instance-major plans), never read on the device
};

}  // namespace nrpf
