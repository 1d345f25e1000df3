// Host-side symbolic plan: everything that depends only on the Ybus sparsity
// pattern and the bus types, built once (Sec. 3.2 "initialization", Sec. 4.1).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace nrpf {

// One left-looking update of column j by a finished column k (Alg. 2 / Alg. 3
// inner loop): LU[dst[dst_off + q]] -= LU[ukj] * LU[lsrc + q], q < llen.
struct Upd {
  int32_t ukj;      // position of U(k, j)
  int32_t lsrc;     // position of the first strictly-lower entry of column k
  int32_t llen;     // number of strictly-lower entries of column k
  int32_t dst_off;  // offset into HostPlan::dst
};

struct HostPlan {
  // ---- problem ----
  int n = 0, m = 0, npv = 0, npq = 0, nslack = 0;
  std::vector<int32_t> rowptr, colidx;     // Ybus CRS
  std::vector<double> yre, yim;
  std::vector<int8_t> bus_type;
  // ---- unknowns: position in A = P J P^T of each bus's angle / magnitude ----
  std::vector<int32_t> th_pos, vm_pos;     // [n], -1 when the bus has none
  std::vector<int32_t> unk_pos;            // [m]: J order (angles of PV+PQ asc, |V| of PQ asc) -> A position
  // ---- LU storage (per instance) ----
  // Columns j < s are "sparse": their whole column (U part, diagonal, L part)
  // is a contiguous segment [cs[j], ce[j]) with ascending rows; dp[j] is the
  // diagonal.  Columns j >= s keep only their rows < s in the segment; rows
  // and columns >= s form a dense block of side ndp (nd rounded up to the
  // panel width kb, padded with an identity) stored column-major at NS.
  int s = 0, nd = 0, ndp = 0, kb = 8;
  std::vector<int64_t> cs, ce;
  std::vector<int32_t> dp;
  std::vector<int32_t> seg_row;            // [NS] row of each segment entry
  int64_t NS = 0, NLU = 0;
  // ---- static lookup Ybus entry -> up to four A positions (Sec. 3.1.2) ----
  std::vector<int32_t> jmap;               // [nnzY*4]: dP/dth, dP/d|V|, dQ/dth, dQ/d|V|
  std::vector<int32_t> one_pos;            // identity padding of the dense block
  std::vector<int32_t> rhs_pos_p, rhs_pos_q;  // [n]: A row of the P / Q equation (-1: none)
  // ---- sparse refactor schedule ----
  std::vector<int32_t> lu_lvl_ptr, lu_lvl_cols;  // columns grouped by level
  std::vector<int32_t> col_upd_ptr;              // [m+1] into upd
  std::vector<Upd> upd;
  std::vector<int32_t> dst;
  // ---- Schur complement of the sparse columns into the dense block ----
  // The updates of a dense column j by sparse columns k keep only their rows
  // < s in the level schedule (they finish U(k, j)); the rows >= s are applied
  // afterwards, all dense columns at once, by tasks of (dense column, chunk of
  // 32 dense rows), one per chunk of every real dense column, in that order:
  // schur_task[4t..] = {j - s, chunk, first entry, end};
  // entry e: schur_ent[e] = (position of L(i, k) << 5) | (i - s - 32 chunk),
  // schur_u[e] = position of U(k, j).  A task writes every row of its chunk
  // (below the padded size): the row's Jacobian value, or 0, minus its sum.
  std::vector<int32_t> schur_task, schur_ent, schur_u;
  std::vector<uint32_t> schur_jmask;  // [tasks] rows of the chunk holding a Jacobian entry
  // ---- forward / backward substitution schedules (row-oriented) ----
  std::vector<int32_t> fw_lvl_ptr, fw_rows, fw_ptr, fw_pos, fw_col;
  std::vector<int32_t> bw_lvl_ptr, bw_rows, bw_ptr, bw_pos, bw_col;
  // ---- counts ----
  int64_t nnz_j = 0, nnz_pattern = 0;
  double lu_fma = 0, solve_fma = 0;
  uint64_t order_seed = 0;                  // tie-break seed of the AMD ordering kept
  int order_key = 0;                        // its key: 0 minimum degree, 1 mean local fill

  int64_t pos(int r, int c) const;  // A position of (r, c); -1 if not stored
};

// Build the plan.  With the AMD ordering and order_tries > 1, seeds
// 0 .. order_tries-1 of each elimination key (minimum degree, mean local fill)
// are tried and the ordering of least estimated refactor time kept:
// dense-block multiply-adds plus sparse_weight times the sparse ones.  One try
// is minimum degree with seed 0.  Returns 0 or a negative NRPF_ERR_* code with
// a message.
int build_plan(int n, const int32_t* rowptr, const int32_t* colidx, const double* yre,
               const double* yim, const int8_t* bus_type, int ordering, double dense_frac,
               int kb, int order_tries, double sparse_weight, HostPlan& out, std::string& err);

}  // namespace nrpf
