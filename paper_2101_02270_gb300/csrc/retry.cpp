// Second chance for instances that fail on the GPU (Sec. 3.2: a case whose
// refactorisation without pivoting breaks down is solved again with a
// factorisation that pivots).  Newton-Raphson on the host, one instance at a
// time, with a left-looking sparse LU (Gilbert-Peierls) that chooses each
// pivot row among the rows not yet pivoted (threshold partial pivoting,
// preferring the diagonal) and keeps the plan's fill-reducing column order.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nrpf.h"
#include "handle.h"
#include "plan.h"

namespace {

using cd = std::complex<double>;

// J in compressed columns; rows and columns in J order (angles of PV then PQ
// buses, then magnitudes of PQ buses; equations likewise P then Q).
struct JPattern {
  int m = 0;
  std::vector<int> colptr, rowind;
  // per Ybus entry d: CSC positions of dP/dth, dP/d|V|, dQ/dth, dQ/d|V| (-1: none)
  std::vector<int> pos;
  std::vector<int> jth, jvm;  // bus -> J index of its angle / magnitude (-1: none)
  std::vector<int> colorder;  // LU column order (the plan's elimination order)
};

void build_pattern(const nrpf::HostPlan& h, JPattern& J) {
  const int n = h.n;
  J.jth.assign(n, -1);
  J.jvm.assign(n, -1);
  int u = 0;
  for (int i = 0; i < n; ++i) if (h.bus_type[i] == 2) J.jth[i] = u++;
  for (int i = 0; i < n; ++i) if (h.bus_type[i] == 1) J.jth[i] = u++;
  for (int i = 0; i < n; ++i) if (h.bus_type[i] == 1) J.jvm[i] = u++;
  J.m = u;
  std::vector<std::vector<std::pair<int, int>>> cols(J.m);  // (row, entry id)
  const int nnzY = h.rowptr[n];
  J.pos.assign((size_t)nnzY * 4, -1);
  for (int i = 0; i < n; ++i)
    for (int d = h.rowptr[i]; d < h.rowptr[i + 1]; ++d) {
      const int k = h.colidx[d];
      const int rp = J.jth[i], rq = J.jvm[i], ct = J.jth[k], cv = J.jvm[k];
      if (rp >= 0 && ct >= 0) cols[ct].push_back({rp, 4 * d + 0});
      if (rp >= 0 && cv >= 0) cols[cv].push_back({rp, 4 * d + 1});
      if (rq >= 0 && ct >= 0) cols[ct].push_back({rq, 4 * d + 2});
      if (rq >= 0 && cv >= 0) cols[cv].push_back({rq, 4 * d + 3});
    }
  J.colptr.assign(J.m + 1, 0);
  J.rowind.clear();
  for (int c = 0; c < J.m; ++c) {
    std::sort(cols[c].begin(), cols[c].end());
    for (auto& e : cols[c]) {
      J.pos[e.second] = (int)J.rowind.size();
      J.rowind.push_back(e.first);
    }
    J.colptr[c + 1] = (int)J.rowind.size();
  }
  // column order: by position in the plan's permuted matrix A = P J P^T
  J.colorder.resize(J.m);
  for (int c = 0; c < J.m; ++c) J.colorder[c] = c;
  std::sort(J.colorder.begin(), J.colorder.end(), [&](int a, int b) { return h.unk_pos[a] < h.unk_pos[b]; });
}

struct SparseLU {
  std::vector<int> Lp, Li, Up, Ui, pinv, prow;
  std::vector<double> Lx, Ux;
};

// Left-looking LU of the m x m CSC matrix (colptr, rowind, val) with columns
// taken in `q` order.  Returns false on a zero or non-finite pivot column.
bool factor(int m, const std::vector<int>& colptr, const std::vector<int>& rowind, const std::vector<double>& val,
            const std::vector<int>& q, double thresh, SparseLU& F) {
  F.Lp.assign(1, 0);
  F.Up.assign(1, 0);
  F.Li.clear(); F.Lx.clear(); F.Ui.clear(); F.Ux.clear();
  F.pinv.assign(m, -1);
  F.prow.assign(m, -1);
  std::vector<double> x(m, 0.0);
  std::vector<int> mark(m, -1), topo, stack, next;
  topo.reserve(m);
  for (int k = 0; k < m; ++k) {
    const int c = q[k];
    // rows reachable from A(:, c) through the columns of L: depth-first
    // search, rows recorded on completion (reverse topological order)
    topo.clear();
    for (int p = colptr[c]; p < colptr[c + 1]; ++p) {
      const int r0 = rowind[p];
      if (mark[r0] == k) continue;
      mark[r0] = k;
      stack.assign(1, r0);
      next.assign(1, 0);
      while (!stack.empty()) {
        const int r = stack.back();
        const int j = F.pinv[r];
        int& it = next.back();
        bool pushed = false;
        if (j >= 0) {
          while (F.Lp[j] + it < F.Lp[j + 1]) {
            const int w = F.Li[F.Lp[j] + it];
            ++it;
            if (mark[w] != k) {
              mark[w] = k;
              stack.push_back(w);
              next.push_back(0);
              pushed = true;
              break;
            }
          }
        }
        if (!pushed) {
          topo.push_back(r);
          stack.pop_back();
          next.pop_back();
        }
      }
    }
    for (int p = colptr[c]; p < colptr[c + 1]; ++p) x[rowind[p]] = val[p];
    // x = L^-1 A(:, c) over the reached rows, in topological order
    for (auto it = topo.rbegin(); it != topo.rend(); ++it) {
      const int r = *it, j = F.pinv[r];
      if (j < 0) continue;
      const double xr = x[r];
      for (int p = F.Lp[j]; p < F.Lp[j + 1]; ++p) x[F.Li[p]] -= F.Lx[p] * xr;
    }
    // pivot among the rows not yet pivoted; the diagonal row if it is within
    // the threshold of the largest
    int piv = -1;
    double amax = 0.0;
    for (int r : topo)
      if (F.pinv[r] < 0 && std::fabs(x[r]) > amax) {
        amax = std::fabs(x[r]);
        piv = r;
      }
    if (piv < 0 || !(amax > 0.0) || !std::isfinite(amax)) {
      for (int r : topo) x[r] = 0.0;
      return false;
    }
    if (F.pinv[c] < 0 && mark[c] == k && std::fabs(x[c]) >= thresh * amax) piv = c;
    const double pv = x[piv];
    for (int r : topo) {
      const int j = F.pinv[r];
      if (j >= 0) {
        F.Ui.push_back(j);
        F.Ux.push_back(x[r]);
      } else if (r != piv) {
        F.Li.push_back(r);
        F.Lx.push_back(x[r] / pv);
      }
      x[r] = 0.0;
    }
    F.Ui.push_back(k);  // diagonal last in the column
    F.Ux.push_back(pv);
    F.Up.push_back((int)F.Ui.size());
    F.Lp.push_back((int)F.Li.size());
    F.pinv[piv] = k;
    F.prow[k] = piv;
  }
  return true;
}

// x = A^-1 b with the factors of `factor` (b in row order, x in column order)
void solve(int m, const SparseLU& F, const std::vector<int>& q, std::vector<double>& b, std::vector<double>& out) {
  std::vector<double> y(m);
  for (int k = 0; k < m; ++k) {
    const double yk = b[F.prow[k]];
    y[k] = yk;
    for (int p = F.Lp[k]; p < F.Lp[k + 1]; ++p) b[F.Li[p]] -= F.Lx[p] * yk;
  }
  for (int k = m - 1; k >= 0; --k) {
    const int pd = F.Up[k + 1] - 1;  // diagonal
    const double zk = y[k] / F.Ux[pd];
    y[k] = zk;
    for (int p = F.Up[k]; p < pd; ++p) y[F.Ui[p]] -= F.Ux[p] * zk;
  }
  out.assign(m, 0.0);
  for (int k = 0; k < m; ++k) out[q[k]] = y[k];
}

// Newton-Raphson of one instance (Sec. 3, steps 1-4) with the pivoting LU;
// same conventions as the GPU solve: strict tol on max |F|, iters = updates,
// status 0 / 1 / 2.
void newton(const nrpf::HostPlan& h, const JPattern& J, const cd* S, const cd* V0, double tol, int maxit, cd* Vout,
            int32_t* iters, uint8_t* status) {
  const int n = h.n, m = J.m;
  std::vector<double> vm(n), va(n);
  std::vector<cd> V(V0, V0 + n), I(n);
  for (int i = 0; i < n; ++i) {
    vm[i] = std::abs(V[i]);
    va[i] = std::arg(V[i]);
  }
  std::vector<double> F(m), val(J.rowind.size()), rhs(m), dx;
  SparseLU lu;
  *status = NRPF_FAILED;
  *iters = 0;
  for (int it = 0;; ++it) {
    // mismatch (Eq. 1, Alg. 1)
    for (int i = 0; i < n; ++i) {
      cd acc = 0.0;
      for (int d = h.rowptr[i]; d < h.rowptr[i + 1]; ++d) acc += cd(h.yre[d], h.yim[d]) * V[h.colidx[d]];
      I[i] = acc;
    }
    double nrm = 0.0;
    bool finite = true;
    for (int i = 0; i < n; ++i) {
      const cd Sc = V[i] * std::conj(I[i]);
      if (J.jth[i] >= 0) F[J.jth[i]] = Sc.real() - S[i].real();
      if (J.jvm[i] >= 0) F[J.jvm[i]] = Sc.imag() - S[i].imag();
    }
    for (int u = 0; u < m; ++u) {
      if (!std::isfinite(F[u])) finite = false;
      nrm = std::max(nrm, std::fabs(F[u]));
    }
    *iters = it;
    if (!finite) { *status = NRPF_FAILED; break; }
    if (nrm < tol) { *status = NRPF_CONVERGED; break; }
    if (it >= maxit) { *status = NRPF_MAXIT; break; }
    // Jacobian: dS/dth = j diag(V) conj(diag(I) - Y diag(V)),
    //           dS/d|V| = diag(V) conj(Y diag(V/|V|)) + conj(diag(I)) diag(V/|V|)
    std::fill(val.begin(), val.end(), 0.0);
    for (int i = 0; i < n; ++i)
      for (int d = h.rowptr[i]; d < h.rowptr[i + 1]; ++d) {
        const int k = h.colidx[d];
        const cd y(h.yre[d], h.yim[d]);
        const cd uk = V[k] / vm[k];
        cd dth = cd(0, 1) * V[i] * std::conj(-y * V[k]);
        cd dvm = V[i] * std::conj(y * uk);
        if (k == i) {
          dth += cd(0, 1) * V[i] * std::conj(I[i]);
          dvm += std::conj(I[i]) * uk;
        }
        const int* p = &J.pos[(size_t)4 * d];
        if (p[0] >= 0) val[p[0]] += dth.real();
        if (p[1] >= 0) val[p[1]] += dvm.real();
        if (p[2] >= 0) val[p[2]] += dth.imag();
        if (p[3] >= 0) val[p[3]] += dvm.imag();
      }
    if (!factor(m, J.colptr, J.rowind, val, J.colorder, 0.1, lu)) { *status = NRPF_FAILED; break; }
    for (int u = 0; u < m; ++u) rhs[u] = -F[u];
    solve(m, lu, J.colorder, rhs, dx);
    bool ok = true;
    for (double v : dx) ok = ok && std::isfinite(v);
    if (!ok) { *status = NRPF_FAILED; break; }
    for (int i = 0; i < n; ++i) {
      if (J.jth[i] >= 0) va[i] += dx[J.jth[i]];
      if (J.jvm[i] >= 0) vm[i] += dx[J.jvm[i]];
      if (J.jth[i] >= 0) V[i] = std::polar(vm[i], va[i]);
    }
  }
  std::copy(V.begin(), V.end(), Vout);
}

// solve instances idx[] of the host arrays, spread over host threads
void solve_many(const pf_plan* p, const std::vector<int>& idx, const cd* S, const cd* V0, double tol, int maxit,
                cd* Vout, int32_t* iters, uint8_t* status) {
  JPattern J;
  build_pattern(p->hp, J);
  const int n = p->hp.n;
  const int nt = (int)std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)idx.size()));
  std::vector<std::thread> th;
  for (int w = 0; w < nt; ++w)
    th.emplace_back([&, w] {
      for (size_t k = w; k < idx.size(); k += nt) {
        const int b = idx[k];
        newton(p->hp, J, S + (size_t)b * n, V0 + (size_t)b * n, tol, maxit, Vout + (size_t)b * n, iters + b,
               status + b);
      }
    });
  for (auto& t : th) t.join();
}

}  // namespace

extern "C" int pf_solve_pivoting_host(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                                      double* v_out, int32_t* iters, uint8_t* status) {
  if (!p || B < 0 || maxit < 0 || !std::isfinite(tol) || tol < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  std::vector<int> idx(B);
  for (int b = 0; b < B; ++b) idx[b] = b;
  solve_many(p, idx, reinterpret_cast<const cd*>(sbus), reinterpret_cast<const cd*>(v0), tol, maxit,
             reinterpret_cast<cd*>(v_out), iters, status);
  return NRPF_OK;
}

extern "C" int pf_retry_failed(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                               double* v_out, int32_t* iters, uint8_t* status, int* n_retried, void* stream) {
  if (!p || p->host_only || B < 0 || maxit < 0 || !std::isfinite(tol) || tol < 0) return NRPF_ERR_ARG;
  if (n_retried) *n_retried = 0;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return NRPF_ERR_CUDA;
  std::vector<uint8_t> sth(B);
  if (cudaMemcpy(sth.data(), status, B, cudaMemcpyDeviceToHost) != cudaSuccess) return NRPF_ERR_CUDA;
  std::vector<int> failed;
  for (int b = 0; b < B; ++b) if (sth[b] == NRPF_FAILED) failed.push_back(b);
  if (failed.empty()) return NRPF_OK;
  const int n = p->hp.n;
  const size_t row = (size_t)n * sizeof(cd);
  const int nf = (int)failed.size();
  std::vector<cd> S((size_t)nf * n), V0((size_t)nf * n), V((size_t)nf * n);
  for (int k = 0; k < nf; ++k) {
    const size_t off = (size_t)failed[k] * n * 2;
    if (cudaMemcpy(&S[(size_t)k * n], sbus + off, row, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&V0[(size_t)k * n], v0 + off, row, cudaMemcpyDeviceToHost) != cudaSuccess)
      return NRPF_ERR_CUDA;
  }
  std::vector<int32_t> it(nf);
  std::vector<uint8_t> stt(nf);
  std::vector<int> local(nf);
  for (int k = 0; k < nf; ++k) local[k] = k;
  solve_many(p, local, S.data(), V0.data(), tol, maxit, V.data(), it.data(), stt.data());
  for (int k = 0; k < nf; ++k) {
    const int b = failed[k];
    if (cudaMemcpy(v_out + (size_t)b * n * 2, &V[(size_t)k * n], row, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(iters + b, &it[k], 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(status + b, &stt[k], 1, cudaMemcpyHostToDevice) != cudaSuccess)
      return NRPF_ERR_CUDA;
  }
  if (n_retried) *n_retried = nf;
  return NRPF_OK;
}
