/*
 * nrpf.h - batched Newton-Raphson AC power flow on one GPU (C ABI).
 *
 * Many power flows whose admittance matrices share one sparsity pattern are
 * solved at once (Wang, Wende-von Berg & Braun, "Fast Parallel Newton-Raphson
 * Power Flow Solver for Large Number of System Calculations with CPU and GPU",
 * Sec. 3).  A plan does the symbolic work once per pattern (Sec. 4.1: ordering,
 * fill-in pattern, static lookup, level schedules); each solve then runs, per
 * Newton iteration and for the whole batch, the nodal power mismatch (Alg. 1),
 * the Jacobian refill straight into the permuted LU workspace (Sec. 3.1.2),
 * the LU refactorisation without pivoting (Sec. 4.3, Eq. 3), forward/backward
 * substitution (Sec. 4.3.3, Eq. 2) and the voltage update (Sec. 3, step 4).
 *
 * Conventions shared by every entry point:
 *  - All functions return an int status: NRPF_OK (0) or a negative NRPF_ERR_*
 *    code; pf_status_str() names it.  No function throws or aborts.
 *  - "host" pointers are ordinary CPU memory read during the call; "device"
 *    pointers are CUDA global memory of the current device, owned by the
 *    caller, and are accessed asynchronously on the caller's stream.
 *  - Complex arrays are interleaved (re, im) float64 pairs, row-major [B, n]:
 *    element (b, i) is at offset 2*(b*n + i).
 *  - Bus-type codes follow MATPOWER: 3 = slack, 2 = PV, 1 = PQ.
 *  - Per-instance status codes: 0 converged, 1 reached maxit, 2 numerical
 *    failure (zero or non-finite pivot, non-finite mismatch or step).
 */
#ifndef NRPF_H
#define NRPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define NRPF_OK 0
#define NRPF_ERR_ARG (-1)        /* null pointer, bad size, bad option       */
#define NRPF_ERR_PATTERN (-2)    /* invalid Ybus pattern or bus types        */
#define NRPF_ERR_NOMEM (-3)      /* host or device allocation failed         */
#define NRPF_ERR_CUDA (-4)       /* a CUDA runtime call failed               */
#define NRPF_ERR_CAPACITY (-5)   /* batch larger than the plan's capacity    */

/* ---- per-instance outcomes ---- */
#define NRPF_CONVERGED 0
#define NRPF_MAXIT 1
#define NRPF_FAILED 2

/* ---- options ---- */
#define NRPF_LU_FP64 0           /* LU refactor and FS/BS in float64           */
#define NRPF_LU_FP32 1           /* LU refactor and FS/BS in float32 (inexact
                                    Newton step; mismatch/update stay float64) */
#define NRPF_ORDER_AMD 0         /* approximate minimum degree on the bus graph */
#define NRPF_ORDER_NATURAL 1     /* bus order as given (tests)                  */
#define NRPF_DENSE_AUTO 0        /* instance-major for FP32 LU with a dense block
                                    of at least NRPF_DENSE_IM_MIN unknowns and
                                    panel 64, interleaved otherwise            */
#define NRPF_DENSE_INTERLEAVED 1 /* dense block interleaved across the 32
                                    instances of a tile (one lane each)        */
#define NRPF_DENSE_INSTANCE_MAJOR 2 /* each instance's dense block its own
                                    column-major matrix, factorised by CTA-tiled
                                    kernels, left-looking by outer panels of
                                    128 (FP32 LU only, panel 64)                */
#define NRPF_DENSE_IM_MIN 512

typedef struct pf_options {
  int lu_precision;    /* NRPF_LU_FP64 | NRPF_LU_FP32                              */
  int ordering;        /* NRPF_ORDER_AMD | NRPF_ORDER_NATURAL                      */
  double dense_frac;   /* AMD stops once the cheapest vertex touches this share of
                          the remaining unknowns; the rest is one dense block.
                          0 selects the default (0.7 for FP64 LU, 0.3 for FP32
                          LU); >= 1 disables the block. */
  int panel;           /* dense-block panel width: 4, 8 or 16 (one trailing
                          update per panel), or 32 / 64 (an outer panel
                          factorised in steps of 16, then one trailing update
                          per outer panel); 0 = default (8 for FP64 LU, 64 for
                          FP32 LU)                                               */
  int max_batch;       /* batch capacity to allocate at plan creation; 0 = grow on
                          first solve (that call then allocates device memory)    */
  int host_only;       /* 1: symbolic analysis only, no device memory; the plan
                          answers pf_plan_get_info / pf_plan_get_pattern and every
                          solve or stage call on it returns NRPF_ERR_ARG          */
  int order_tries;     /* AMD only: minimum degree leaves ties between vertices of
                          equal degree open.  With order_tries = T > 1 the plan
                          tries T seeded tie-breaks (seed 0: lowest bus index
                          first) of each of two elimination keys (minimum
                          degree; mean local fill) and keeps the ordering of
                          least estimated refactor time (dense-block
                          multiply-adds plus a precision-dependent weight times
                          the sparse ones).  0 = default (T = 128 up to 4,000
                          buses, 512,000 / n above, at least 8); 1 = minimum
                          degree with seed 0 only                                */
  int dense_layout;    /* NRPF_DENSE_AUTO | NRPF_DENSE_INTERLEAVED |
                          NRPF_DENSE_INSTANCE_MAJOR (storage and kernels of the
                          dense block; results differ only by rounding)          */
} pf_options;

typedef struct pf_plan pf_plan;   /* opaque; owns its device arrays and workspace */

typedef struct pf_plan_info {
  int n;               /* buses                                                  */
  int m;               /* unknowns = dim J = n_pv + 2 n_pq                         */
  int n_pv, n_pq, n_slack;
  int64_t nnz_ybus;
  int64_t nnz_j;       /* structural nonzeros of J                               */
  int64_t nnz_lu;      /* stored LU values per instance (incl. dense block pad)  */
  int sparse_cols;     /* columns factorised by the sparse phase (first s)       */
  int dense_dim;       /* unknowns in the trailing dense block (nd)              */
  int dense_pad;       /* nd rounded up to the panel width                       */
  int lu_levels;       /* level count of the sparse refactor schedule            */
  int fwd_levels, bwd_levels;
  double lu_fma;       /* multiply-adds of one refactorisation, one instance     */
  double solve_fma;    /* multiply-adds of one FS/BS, one instance                */
  int capacity;        /* batch capacity currently allocated                     */
  int lu_precision;
  int panel;           /* dense-block panel width in use                          */
  int order_seed;      /* tie-break seed of the ordering kept (0 for NATURAL)     */
  int order_key;       /* its elimination key: 0 minimum degree, 1 mean local fill */
  int dense_layout;    /* NRPF_DENSE_INTERLEAVED or NRPF_DENSE_INSTANCE_MAJOR     */
} pf_plan_info;

/* Fill pf_options with the defaults (AMD ordering, FP64 LU, dense_frac and
 * panel chosen by precision, grow-on-demand workspace, device upload). */
int pf_options_default(pf_options* opt);

/* Assemble Ybus (MATPOWER pi-model convention, Sec. 3) from branch data.
 * host in : n buses, nbr branches, f/t [nbr] bus indices, r/x/b [nbr] series
 *           resistance, series reactance, total line charging (p.u.).
 * host out: rowptr [n+1], colidx [cap], y_re/y_im [cap] as CRS with sorted
 *           columns and every diagonal present; *nnz_out = entries written.
 * Errors: NRPF_ERR_ARG for bad sizes/indices or cap too small (then *nnz_out
 * holds the required capacity). */
int pf_ybus_from_branches(int n, int nbr, const int32_t* f, const int32_t* t, const double* r,
                          const double* x, const double* b, int32_t* rowptr, int32_t* colidx,
                          double* y_re, double* y_im, int64_t cap, int64_t* nnz_out);

/* Symbolic analysis, done once per sparsity pattern (Sec. 3.2 "initialization",
 * Sec. 4.1): bus maps, Jacobian pattern, fill-reducing ordering, LU fill,
 * static lookup Ybus entry -> LU slots (Sec. 3.1.2), level schedules (Sec.
 * 4.3.1); uploads everything to the current device.
 * host in : Ybus CRS (rowptr [n+1], colidx [nnz], sorted, diagonal present,
 *           structurally symmetric), values y_re/y_im [nnz] shared by every
 *           instance, bus_type [n] (at least one slack).
 * out     : *out receives a plan to be released with pf_plan_destroy.
 * Errors: NRPF_ERR_ARG, NRPF_ERR_PATTERN, NRPF_ERR_NOMEM, NRPF_ERR_CUDA. */
int pf_plan_create(int n, const int32_t* rowptr, const int32_t* colidx, const double* y_re,
                   const double* y_im, const int8_t* bus_type, const pf_options* opt,
                   pf_plan** out);

/* Sizes and work counts of a plan (host out). */
int pf_plan_get_info(const pf_plan* p, pf_plan_info* info);

/* Permutation and pattern of the factorised matrix A = P J P^T (Eq. 3).
 * host out: pos_of_unknown [m]: position in A of J row/column u (rows and
 *           columns share the permutation); colptr [m+1], rowidx [nnz]: CCS
 *           pattern of L+U-I with sorted rows (the dense block listed in full);
 *           any output pointer may be NULL.  *nnz_out = pattern size. */
int pf_plan_get_pattern(const pf_plan* p, int32_t* pos_of_unknown, int64_t* colptr,
                        int32_t* rowidx, int64_t* nnz_out);

/* Solve B power flows (Sec. 3, steps 1-4, until max |mismatch| < tol or maxit
 * Newton updates).
 * device in : sbus [B,n] complex specified injections (generation - load, p.u.);
 *             v0 [B,n] complex start; slack voltages and PV magnitudes are
 *             held at their v0 values.
 * device out: v_out [B,n] complex (may alias v0), iters [B] Newton updates
 *             performed, status [B] per-instance outcome (NRPF_CONVERGED ...).
 *             v_out of an NRPF_FAILED instance is unspecified: a bus whose
 *             step was not finite keeps its previous value while the other
 *             buses of the instance take theirs, so it mixes two iterates
 *             (the second chance, pf_retry_failed, starts again from v0).
 * stream    : cudaStream_t of the caller (NULL = legacy default stream).
 * Asynchronous: returns after enqueueing.  Grows the workspace (device
 * allocation, synchronous) when B exceeds the plan's capacity.
 * The Newton loop ends on the device: one iteration is captured once per
 * padded batch size as the body of a CUDA graph WHILE node, and the
 * iteration's last kernel clears the condition when no instance is active
 * (or at maxit).  Inside a caller's stream capture the loop is enqueued as
 * maxit iterations instead (finished instances skip through their gates);
 * with per-kernel timing on (pf_profile_start with a nonzero mask) the host
 * ends the loop after each iteration.  All three give identical results.
 * Calls on one plan share its workspace: serialise them (one stream).
 * Errors: NRPF_ERR_ARG (B < 0, tol not finite, maxit < 0, null pointers),
 * NRPF_ERR_NOMEM, NRPF_ERR_CUDA.  B == 0 is a no-op. */
int pf_solve_batch(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                   double* v_out, int32_t* iters, uint8_t* status, void* stream);

/* Per-instance admittance values on the plan's pattern: many Ybus that share
 * one sparsity pattern, e.g. static N-1 contingency analysis, where each
 * instance removes a branch (the paper's profile variant with one Ybus per
 * case and a shared pattern, Sec. 3.2).  The pattern is the plan's (an
 * outaged branch keeps its entries, with zero admittance).
 * device in : ybus [B, nnz] complex values in the plan's CRS order (nnz =
 *             rowptr[n] of pf_plan_create), sbus / v0 [B, n] complex.
 * device out: as pf_solve_batch.
 * The values are copied into a workspace array interleaved by instance
 * (allocated on first use, grown with the batch capacity).
 * Errors: as pf_solve_batch. */
int pf_solve_batch_y(pf_plan* p, int B, const double* ybus, const double* sbus, const double* v0, double tol,
                     int maxit, double* v_out, int32_t* iters, uint8_t* status, void* stream);

/* Branch outages on the device (static N-1 / N-k analysis without building
 * admittance arrays on the host).  pf_plan_set_branches keeps the branch
 * data of the plan's grid (pi model, as pf_ybus_from_branches; every branch
 * must have its entries in the plan's pattern); pf_solve_batch_outages then
 * solves B instances whose admittances are the plan's base values minus the
 * stamps of their outaged branches, built on the device.
 * pf_plan_set_branches: host in nbr, f/t/r/x/b [nbr].  Errors: NRPF_ERR_ARG,
 * NRPF_ERR_PATTERN (a branch entry missing from the pattern), NRPF_ERR_NOMEM.
 * pf_solve_batch_outages: device in outages [B, k] branch indices (-1 = none;
 * repeated indices are removed once), sbus / v0 [B, n]; device out as
 * pf_solve_batch.  Errors: as pf_solve_batch; NRPF_ERR_ARG also when no
 * branches were set or k < 0. */
int pf_plan_set_branches(pf_plan* p, int nbr, const int32_t* f, const int32_t* t, const double* r, const double* x,
                         const double* b);
int pf_solve_batch_outages(pf_plan* p, int B, const int32_t* outages, int k, const double* sbus, const double* v0,
                           double tol, int maxit, double* v_out, int32_t* iters, uint8_t* status, void* stream);

/* Host helper for pf_solve_batch_y: Ybus values of B branch-status cases on a
 * given pattern (MATPOWER pi model as pf_ybus_from_branches; branches out of
 * service contribute nothing).
 * host in : n buses, nbr branches f/t/r/x/b [nbr]; in_service [B, nbr]
 *           (nonzero = in service; NULL = all in service); rowptr [n+1],
 *           colidx [nnz] with sorted columns per row.
 * host out: y [B, nnz] complex (re, im interleaved).
 * Errors: NRPF_ERR_ARG (bad sizes or indices, zero series impedance),
 * NRPF_ERR_PATTERN (a branch entry missing from the pattern). */
int pf_ybus_values(int n, int nbr, const int32_t* f, const int32_t* t, const double* r, const double* x,
                   const double* b, int B, const uint8_t* in_service, const int32_t* rowptr,
                   const int32_t* colidx, double* y);

/* Batched Newton-Raphson on the host cores (the paper's CPU solver: SIMD
 * across instances, threads across mini-batches, Sec. 4).  Same plan, same
 * arithmetic and conventions as pf_solve_batch in FP64 (up to summation
 * order): instances in mini-batches of 8 interleaved lanes, left-looking
 * sparse refactor in column order, the sparse columns' updates of the dense
 * block, dense LU of the trailing block, FS/BS, polar update.
 * host in : sbus / v0 [B, n] complex; host out: v_out [B, n], iters [B],
 * status [B].  threads: host threads (0 = all hardware threads).  Works on
 * host-only plans.  Synchronous.  Errors: NRPF_ERR_ARG. */
int pf_solve_batch_cpu(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                       double* v_out, int32_t* iters, uint8_t* status, int threads);

/* Second chance for failed instances (Sec. 3.2: cases whose refactorisation
 * without pivoting breaks down are solved again with a pivoting
 * factorisation).  Newton-Raphson on the host cores with a left-looking
 * sparse LU that picks each pivot row among the rows not yet pivoted
 * (threshold 0.1 towards the diagonal) in the plan's column order; same
 * tolerance, iteration and status conventions as pf_solve_batch.
 *
 * pf_solve_pivoting_host: host in sbus / v0 [B, n] complex; host out v_out
 * [B, n], iters [B], status [B].  Works on host-only plans.  Synchronous.
 *
 * pf_retry_failed: after a pf_solve_batch on `stream` (device arrays of that
 * call), synchronises the stream, re-solves from v0 every instance whose
 * status is NRPF_FAILED and writes its v_out / iters / status back to the
 * device; *n_retried (may be NULL) receives the count.  Synchronous.
 * Errors: NRPF_ERR_ARG, NRPF_ERR_CUDA. */
int pf_solve_pivoting_host(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                           double* v_out, int32_t* iters, uint8_t* status);
int pf_retry_failed(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                    double* v_out, int32_t* iters, uint8_t* status, int* n_retried, void* stream);

/* Branch power flows of solved batches (post-processing after convergence,
 * Sec. 3.2): the complex power entering each branch at its from end (sf) and
 * at its to end (st), pi model as pf_ybus_from_branches; sf + st is the
 * branch's loss.
 * device in : f, t [nbr] bus indices, r, x, b [nbr] branch data;
 *             in_service [B, nbr] (nonzero = in service; NULL = all; a branch
 *             out of service carries zero flow); v [B, n] complex voltages.
 * device out: sf, st [B, nbr] complex.
 * Asynchronous on `stream`.  Errors: NRPF_ERR_ARG, NRPF_ERR_CUDA. */
int pf_branch_flows(int n, int nbr, const int32_t* f, const int32_t* t, const double* r, const double* x,
                    const double* b, int B, const uint8_t* in_service, const double* v, double* sf, double* st,
                    void* stream);

/* pf_solve_batch for a batch held in host memory (the paper's stream study,
 * Sec. 3.2 / Sec. 5: copies overlapped with computation).  The batch is cut
 * into chunks of `chunk` instances (0 = the whole batch).  Each chunk goes
 * through one of two device staging slots owned by the plan, used in turn
 * across chunks and across calls: its inputs are copied in on a copy-in
 * stream owned by the plan, it is solved on `stream`, and its results are
 * copied out on a copy-out stream owned by the plan.  A copy-in waits only
 * for its slot to be free (the copy-out of the chunk that used it before),
 * so it overlaps the solve of the previous chunk or of the previous call.
 * host in : sbus [B,n], v0 [B,n] complex (page-locked memory lets the copies
 *           run asynchronously; pageable memory works but serialises them).
 *           They are read at some time after the call: do not modify them
 *           until `stream` has completed the call's work.
 * host out: v_out [B,n] complex, iters [B], status [B] (as pf_solve_batch).
 * stream  : the caller's stream; the solves are ordered after the work
 *           already on it, and work enqueued on it later runs after the last
 *           result has reached host memory.  Asynchronous: synchronise
 *           `stream` before reading the outputs.
 * The workspace is sized for one chunk (grown as in pf_solve_batch); the
 * staging slots grow (synchronously) when a larger chunk is asked for.
 * Errors: as pf_solve_batch; NRPF_ERR_ARG also for chunk < 0. */
int pf_solve_batch_host(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                        double* v_out, int32_t* iters, uint8_t* status, int chunk, void* stream);

/* ---- single stages, for tests and profiling (same layouts as above) ---- */

/* Alg. 1 at voltages v: F [B,m] float64 in J row order (dP of the PV buses,
 * then dP of the PQ buses, then dQ of the PQ buses, each group in ascending
 * bus order; J columns follow the same order for angles and magnitudes),
 * norm [B] = max |F|. */
int pf_stage_mismatch(pf_plan* p, int B, const double* sbus, const double* v, double* F,
                      double* norm, void* stream);

/* Jacobian at v scattered into the permuted LU workspace (Sec. 3.1.2), then,
 * if factor != 0, refactorised in place (Sec. 4.3).  lu_out [B, nnz] float64 in
 * the order of pf_plan_get_pattern (CCS of A, or of L+U-I when factorised;
 * L is unit lower and its diagonal is not stored). */
int pf_stage_factor(pf_plan* p, int B, const double* v, int factor, double* lu_out, void* stream);

/* One linear solve J(v) dx = rhs (refill, refactor, FS/BS).
 * device in: v [B,n] complex, rhs [B,m] float64 in J row order.
 * device out: dx [B,m] float64 in J column order. */
int pf_stage_linear_solve(pf_plan* p, int B, const double* v, const double* rhs, double* dx,
                          void* stream);

/* ---- uneven batching: many plans, one persistent launch ----
 * Grids of different sizes and sparsity patterns (one plan each, all with the
 * same LU precision and no dense block, i.e. created with dense_frac >= 1) and
 * different scenario counts are solved together by one persistent kernel
 * (the paper's remark on imbalanced batches across streams/GPUs, Sec. 5,
 * motivates it).  Work items are (plan, tile of up to S scenarios), sorted
 * by decreasing work and pulled from a device counter; each item runs the
 * full Newton loop of Sec. 3, the S scenarios of the item sharing each warp
 * (32 / S workers per scenario and warp).  Its state (voltages, injections,
 * right-hand side, LU values) sits in the CTA's shared memory when it fits
 * (pf_multi_set_scenarios with use_smem), otherwise in a private global
 * slot.  The launch is captured in a CUDA graph and replayed while arguments
 * are unchanged. */
typedef struct pf_multi pf_multi;

/* host in: k plans (kept alive by the caller while the group exists) and
 * batch[k] scenario counts.  Inputs and outputs of pf_multi_solve are the
 * plans' [B_f, n_f] blocks concatenated in plan order; iters/status are
 * concatenated [B_f] blocks.  Allocates the group's device tables and slots.
 * Errors: NRPF_ERR_ARG (mixed precision, a plan with a dense block, host-only
 * plan), NRPF_ERR_NOMEM, NRPF_ERR_CUDA. */
int pf_multi_create(int k, pf_plan* const* plans, const int32_t* batch, pf_multi** out);

/* Solve every scenario of the group (same semantics and outputs as
 * pf_solve_batch, concatenated).  Asynchronous on stream. */
int pf_multi_solve(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                   int32_t* iters, uint8_t* status, void* stream);

/* Launch shape: warps per item (threads per instance, 1..16) and resident
 * CTAs per SM (1..32); may grow the slot pool (allocation). */
int pf_multi_set_config(pf_multi* mp, int warps, int blocks_per_sm);
int pf_multi_get_config(const pf_multi* mp, int* warps, int* blocks_per_sm, int64_t* instances, int* items);

/* Scenarios per work item S (1, 2, 4, ..., 32; default 32) and whether item
 * states that fit 200 KB go to shared memory (use_smem 1; the launch then
 * takes the largest such state as its dynamic shared memory per CTA).
 * Rebuilds the item list; may grow the slot pool (allocation, synchronous).
 * Errors: NRPF_ERR_ARG (S not a power of two in [1, 32], use_smem not 0/1),
 * NRPF_ERR_NOMEM, NRPF_ERR_CUDA. */
int pf_multi_set_scenarios(pf_multi* mp, int per_item, int use_smem);
/* Current S, use_smem, dynamic shared memory per CTA (bytes) and the number of
 * items whose state is in shared memory. */
int pf_multi_get_scenarios(const pf_multi* mp, int* per_item, int* use_smem, int64_t* smem_bytes, int* smem_items);

/* Autotuner: times the real solve for every (S, use_smem) in {(32, 0), (16, 0),
 * (8, 0), (32, 1), (16, 1), (8, 1), (4, 1), (2, 1)} and (warps, CTAs per SM) pair in
 * {1,2,4,8,16}^2 with at most 2048 threads and 228 KB of dynamic shared
 * memory per SM, keeps the fastest and reports its time (host-blocking;
 * outputs hold the last solve). */
int pf_multi_autotune(pf_multi* mp, const double* sbus, const double* v0, double tol, int maxit, double* v_out,
                      int32_t* iters, uint8_t* status, void* stream, double* best_ms);

void pf_multi_destroy(pf_multi* mp);

/* ---- learned warm start (BF16 tensor-core MLP) ----
 * The paper motivates fast repeated power flows with the training of neural
 * networks on many solutions (Sec. 1); here the solver also feeds one: an
 * MLP maps per-bus injections to an initial voltage guess, and Newton then
 * runs from that guess to the same tolerance (flat start as fallback).
 * Network: h1 = GELU(x W1^T + b1), h2 = GELU(h1 W2^T + b2), y = h2 W3^T + b3,
 * exact erf-GELU, weights [out][in] FP32 master copies, BF16 tensor-core
 * GEMMs (tcgen05, FP32 accumulate) in the forward and backward passes, loss =
 * mean squared error on standardised inputs and targets, AdamW (beta 0.9 /
 * 0.999, eps 1e-8, decoupled weight decay). */
typedef struct pf_mlp pf_mlp;

/* nh1, nh2 must be multiples of 128; bmax = largest batch of any call.
 * Weights uniform(+-1/sqrt(fan_in)) from a seeded generator, biases zero. */
int pf_mlp_create(int nin, int nh1, int nh2, int nout, int bmax, uint64_t seed, pf_mlp** out);

/* host in: per-feature means and standard deviations (nonzero) of the inputs
 * [nin] and targets [nout] used to standardise them. */
int pf_mlp_set_norm(pf_mlp* p, const float* mux, const float* sdx, const float* muy, const float* sdy);

/* Standardisation fitted on a training set: per-column mean and standard
 * deviation of x [B, nin] and t [B, nout] (device, FP32); constant columns
 * keep scale 1. */
int pf_mlp_fit_norm(pf_mlp* p, int64_t B, const float* X, const float* T, void* stream);

/* set != 0: load the 6 host arrays W1 [nh1*nin], b1, W2, b2, W3, b3 (and reset
 * the optimiser); set == 0: copy them out.  Synchronous. */
int pf_mlp_params(pf_mlp* p, int set, float* const* host);

/* Gradients of the last pf_mlp_train_step, same 6-array layout (host out). */
int pf_mlp_grads(pf_mlp* p, float* const* host);

/* device in: x [B, nin] FP32 (raw units); device out: y [B, nout] FP32 (raw
 * units).  Errors: NRPF_ERR_CAPACITY when B > bmax. */
int pf_mlp_predict(pf_mlp* p, int B, const float* x, float* y, void* stream);

/* One training step on a minibatch: forward, loss, backward, and (update != 0)
 * an AdamW update with learning rate lr and weight decay wd.
 * device in: x [B, nin], t [B, nout] FP32 raw units; device out: *loss_out
 * (FP32, may be NULL) = mean squared standardised error. */
int pf_mlp_train_step(pf_mlp* p, int B, const float* x, const float* t, float lr, float wd, int update,
                      float* loss_out, void* stream);

/* 1 if a tensor-core kernel gave up waiting for its MMAs (bounded wait). */
int pf_mlp_error(pf_mlp* p);

void pf_mlp_destroy(pf_mlp* p);

/* Standalone tensor-core GEMM: C[M,N] FP32 = A[M,K] B[N,K]^T with A, B BF16
 * row-major on the device; M, N multiples of 128, K of 64.  variant 0: tiles
 * copied by the CTA then multiplied (one stage); variant 1: TMA-filled
 * four-stage ring with a producer thread and an MMA-issuing thread.
 * *err (device int) is set to 1 when a kernel gives up a bounded wait. */
int pf_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, int variant, int* err,
                 void* stream);

/* GEMM variant used by the network (default 1; 0 when the TMA encoder is
 * unavailable). */
int pf_gemm_set_variant(int variant);

/* Warm-start glue (device in/out):
 * features: X [B, 2n] = [P_0..P_{n-1}, Q_0..Q_{n-1}] of sbus [B, n];
 * targets : T [B, 2 nns] = [|V|, angle] of the nns non-slack buses of V [B, n],
 *           nsidx [n] = rank of a bus among the non-slack buses, -1 for slack;
 * v0      : start voltages from a prediction Y [B, 2 nns]: slack buses keep
 *           v_flat, PV buses keep |v_flat| with the predicted angle, PQ buses
 *           take the predicted magnitude and angle. */
int pf_warmstart_features(int n, int B, const double* sbus, float* X, void* stream);
int pf_warmstart_targets(int n, int B, const int32_t* nsidx, int nns, const double* v, float* T, void* stream);
int pf_warmstart_v0(int n, int B, const int32_t* nsidx, const int8_t* bus_type, int nns, const float* Y,
                    const double* v_flat, double* v0, void* stream);

/* Screen of warm-started results (device in/out).  Newton from a guess can
 * converge to another root of the power-flow equations than the one reached
 * from flat start (a low-voltage solution).  The reading taken: the correct
 * result is the flat-start solution, so a warm-started instance is redone
 * from flat start when redo[b] = 1: status[b] != 0, a non-finite voltage, or
 * min_i |v[b, i]| < vmin (p.u., >= 0).  v [B, n] complex128, status [B]
 * (pf_solve_batch codes), redo [B] uint8.  No counterpart in the paper, which
 * always starts from flat start (Sec. 3). */
int pf_warmstart_screen(int n, int B, const double* v, const uint8_t* status, double vmin, uint8_t* redo,
                        void* stream);

/* ---- launch accounting and per-kernel device time ----
 * Kernel classes (index into the pf_profile arrays): 0 load (input transpose),
 * 1 store, 2 mismatch_jacobian, 3 check, 4 zero_lu, 5 set_ones,
 * 6 lu_sparse_level, 7 dense_diag, 8 dense_panel, 9 dense_update, 10 fwd_level,
 * 11 dense_solve, 12 bwd_level, 13 update, 14 aux, 15 lu_schur (the sparse
 * columns' updates of the dense block). */
#define NRPF_KCLASSES 16
typedef struct pf_profile {
  int64_t launches[NRPF_KCLASSES];  /* kernels enqueued by pf_solve_batch        */
  int64_t timed[NRPF_KCLASSES];     /* launches bracketed by CUDA events          */
  double ms[NRPF_KCLASSES];         /* summed event time of the timed launches    */
} pf_profile;

/* Reset the counters of a plan.  Every later launch of a class whose bit is set
 * in time_mask is bracketed by two CUDA events recorded on the launching
 * stream (adds two event records per launch).  Not thread-safe. */
int pf_profile_start(pf_plan* p, uint32_t time_mask);

/* Wait for the recorded events (host-blocking) and report counts and times. */
int pf_profile_read(pf_plan* p, pf_profile* out);

/* Static name of a kernel class, or "unknown". */
const char* pf_kernel_class_name(int c);

/* Measured FP64 and FP32 fused-multiply-add throughput of the current device
 * (TFLOP/s, 2 flop per FMA), the arithmetic roofline against which the
 * solver's FP-bound kernels are reported.  The paper has no counterpart: it
 * is a measurement aid.  Runs a few hundred milliseconds of synchronous work
 * on the given stream and allocates a small scratch buffer. */
int pf_fma_peak(double* fp64_tflops, double* fp32_tflops, void* stream);

/* Mismatch and max|F| of a batch without allocating device memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc when they evaluate the mismatch - code whose device memory is
 * owned entirely by another allocator (a framework's caching pool holding the
 * GPU), or a real-time loop that must not take cudaMalloc's latency and its
 * implicit device-wide synchronisation.  pf_stage_mismatch computes the same
 * values but stages them through the plan's workspace, which it grows with
 * cudaMalloc when the batch exceeds the plan's capacity.
 * Here the only scratch (the running per-instance maxima of the cross-block
 * reduction and an arrival counter) lives in one static device array of
 * NRPF_NOALLOC_MAX_BATCH + 32 eight-byte words (about 512 KB), which every GPU
 * that loads the library holds until the process exits.
 * device in : sbus, v [B,n] complex as in pf_solve_batch.
 * device out: F [B,m] float64, row r = the equation at position r of
 *             A = P J P^T (pf_plan_get_pattern's pos_of_unknown maps J row u to
 *             position pos_of_unknown[u]); norm [B] = max |F| (a non-finite
 *             entry gives +inf).  F and norm are float64 arithmetic and
 *             float64 results for plans of either LU precision.  (The staged
 *             pf_stage_mismatch of an FP32-LU plan reads F back from its FP32
 *             right-hand side, so its F is rounded to float32; its norm is the
 *             float64 one.)
 * The first call on a device looks up the array's device address (a runtime
 * query, once per device, with that device current); make that first call
 * before any stream capture begins.  The address is kept for the life of the
 * process: it does not survive cudaDeviceReset, after which this entry point
 * must not be called again in the same process.  Each call clears the part of the array it
 * uses (stream-ordered memsets) and then runs one kernel.  All calls share the
 * array, so calls that overlap on the GPU (different streams, or threads)
 * race and give wrong norms: serialise them.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 * Errors: NRPF_ERR_ARG (null pointers, host-only plan, B < 0),
 * NRPF_ERR_CAPACITY (B > NRPF_NOALLOC_MAX_BATCH), NRPF_ERR_CUDA.
 * B == 0 is a no-op. */
#define NRPF_NOALLOC_MAX_BATCH 65536
int pf_stage_mismatch_noalloc(const pf_plan* p, int B, const double* sbus, const double* v, double* F,
                              double* norm, void* stream);

void pf_plan_destroy(pf_plan* p);

/* Static string naming a return code (or "unknown"). */
const char* pf_status_str(int code);

#ifdef __cplusplus
}
#endif

#endif /* NRPF_H */
