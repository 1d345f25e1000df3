// Batched Newton-Raphson on the host cores (the paper's CPU solver, Sec. 4:
// instances in SIMD lanes, mini-batches spread over hardware threads).  It
// runs the same plan as the GPU path: the fused mismatch + Jacobian refill
// through the static Ybus -> LU lookup, the left-looking sparse refactor in
// column order, the sparse columns' updates of the dense block, a dense LU of
// the trailing block, FS/BS and the polar update.  Data of a mini-batch are
// interleaved by kLanes instances, so every inner loop runs over the lanes
// and is left to the compiler's vectoriser (no target-specific intrinsics).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/nrpf.h"
#include "handle.h"
#include "plan.h"

namespace {

constexpr int kLanes = 8;
constexpr int kPanel = 8;  // dense LU panel width

// one mini-batch of up to kLanes instances (instances b0 .. b0+nb-1)
void solve_group(const nrpf::HostPlan& h, int nb, const double* sbus, const double* v0, double tol, int maxit,
                 double* v_out, int32_t* iters, uint8_t* status, std::vector<double>& lu, std::vector<double>& x) {
  const int n = h.n, m = h.m, s = h.s, ndp = h.ndp;
  const int64_t NS = h.NS, NLU = h.NLU;
  const int mp = s + ndp;
  constexpr int W = kLanes;
  lu.assign((size_t)NLU * W, 0.0);
  x.assign((size_t)mp * W, 0.0);
  std::vector<double> ve((size_t)n * W), vf((size_t)n * W), vm((size_t)n * W), va((size_t)n * W),
      ps((size_t)n * W), qs((size_t)n * W);
  bool active[W], bad[W];
  for (int l = 0; l < W; ++l) {
    active[l] = l < nb;
    bad[l] = false;
  }
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < W; ++l) {
      const int b = l < nb ? l : 0;
      const double re = v0[((size_t)b * n + i) * 2], im = v0[((size_t)b * n + i) * 2 + 1];
      const size_t o = (size_t)i * W + l;
      ve[o] = re;
      vf[o] = im;
      vm[o] = std::sqrt(re * re + im * im);
      va[o] = std::atan2(im, re);
      ps[o] = sbus[((size_t)b * n + i) * 2];
      qs[o] = sbus[((size_t)b * n + i) * 2 + 1];
    }
  auto L = [&](int64_t p) { return &lu[(size_t)p * W]; };
  auto X = [&](int64_t r) { return &x[(size_t)r * W]; };
  for (int it = 0;; ++it) {
    // ---- LU preparation, mismatch and Jacobian (Eq. 1, Alg. 1, Sec. 3.1.2)
    std::fill(lu.begin(), lu.end(), 0.0);
    for (int32_t q : h.one_pos) std::fill(L(q), L(q) + W, 1.0);
    std::fill(x.begin(), x.end(), 0.0);
    double nrm[W] = {};
    for (int i = 0; i < n; ++i) {
      const int bt = h.bus_type[i];
      if (bt == 3) continue;
      double Ir[W] = {}, Ii[W] = {};
      const double* ei = &ve[(size_t)i * W];
      const double* fi = &vf[(size_t)i * W];
      int dd = -1;
      for (int d = h.rowptr[i]; d < h.rowptr[i + 1]; ++d) {
        const int k = h.colidx[d];
        if (k == i) dd = d;
        const double G = h.yre[d], Bv = h.yim[d];
        const double* ek = &ve[(size_t)k * W];
        const double* fk = &vf[(size_t)k * W];
        double yr[W], yi[W];
        for (int l = 0; l < W; ++l) {
          yr[l] = G * ek[l] - Bv * fk[l];
          yi[l] = G * fk[l] + Bv * ek[l];
          Ir[l] += yr[l];
          Ii[l] += yi[l];
        }
        if (k != i) {
          const int32_t* jm = &h.jmap[(size_t)d * 4];
          if (jm[0] >= 0) {
            const double* ivk = &vm[(size_t)k * W];
            double* a0 = L(jm[0]);
            double* a1 = jm[1] >= 0 ? L(jm[1]) : nullptr;
            double* a2 = jm[2] >= 0 ? L(jm[2]) : nullptr;
            double* a3 = jm[3] >= 0 ? L(jm[3]) : nullptr;
            for (int l = 0; l < W; ++l) {
              const double Wr = ei[l] * yr[l] + fi[l] * yi[l];
              const double Wi = fi[l] * yr[l] - ei[l] * yi[l];
              a0[l] = Wi;
              if (a1) a1[l] = Wr / ivk[l];
              if (a2) a2[l] = -Wr;
              if (a3) a3[l] = Wi / ivk[l];
            }
          }
        }
      }
      double* xp = X(h.rhs_pos_p[i]);
      double* xq = bt == 1 ? X(h.rhs_pos_q[i]) : nullptr;
      double Pc[W], Qc[W];
      for (int l = 0; l < W; ++l) {
        const size_t o = (size_t)i * W + l;
        Pc[l] = ei[l] * Ir[l] + fi[l] * Ii[l];
        Qc[l] = fi[l] * Ir[l] - ei[l] * Ii[l];
        const double dP = Pc[l] - ps[o];
        double a = std::fabs(dP);
        xp[l] = -dP;
        if (xq) {
          const double dQ = Qc[l] - qs[o];
          xq[l] = -dQ;
          const double q = std::fabs(dQ);
          a = (q > a || q != q) ? q : a;
        }
        nrm[l] = (a > nrm[l] || a != a) ? a : nrm[l];
      }
      const int32_t* jm = &h.jmap[(size_t)dd * 4];
      const double G = h.yre[dd], Bv = h.yim[dd];
      for (int l = 0; l < W; ++l) {
        const size_t o = (size_t)i * W + l;
        const double vm2 = ei[l] * ei[l] + fi[l] * fi[l];
        const double ivm = 1.0 / vm[o];
        const double vmag = vm2 * ivm;
        L(jm[0])[l] = -Qc[l] - Bv * vm2;
        if (jm[1] >= 0) L(jm[1])[l] = Pc[l] * ivm + G * vmag;
        if (jm[2] >= 0) L(jm[2])[l] = Pc[l] - G * vm2;
        if (jm[3] >= 0) L(jm[3])[l] = Qc[l] * ivm - Bv * vmag;
      }
    }
    // ---- convergence test (strict tol, iteration = updates performed)
    bool any = false;
    for (int l = 0; l < nb; ++l) {
      if (!active[l]) continue;
      int keep = 0;
      if (bad[l]) {
        status[l] = NRPF_FAILED;
        iters[l] = it - 1;
      } else if (!(nrm[l] <= 1.7976931348623157e308)) {
        status[l] = NRPF_FAILED;
        iters[l] = it;
      } else if (nrm[l] < tol) {
        status[l] = NRPF_CONVERGED;
        iters[l] = it;
      } else if (it >= maxit) {
        status[l] = NRPF_MAXIT;
        iters[l] = it;
      } else {
        keep = 1;
      }
      active[l] = keep;
      any = any || keep;
    }
    if (!any) break;
    // ---- sparse left-looking refactor in column order (Alg. 2)
    for (int j = 0; j < m; ++j) {
      for (int u = h.col_upd_ptr[j]; u < h.col_upd_ptr[j + 1]; ++u) {
        const nrpf::Upd& up = h.upd[u];
        const double* ukj = L(up.ukj);
        double xv[W];
        std::copy(ukj, ukj + W, xv);
        const int32_t* dst = &h.dst[up.dst_off];
        for (int q = 0; q < up.llen; ++q) {
          double* a = L(dst[q]);
          const double* sv = L(up.lsrc + q);
          for (int l = 0; l < W; ++l) a[l] -= xv[l] * sv[l];
        }
      }
      const int dpj = h.dp[j];
      if (dpj >= 0) {
        double inv[W];
        const double* pv = L(dpj);
        for (int l = 0; l < W; ++l) inv[l] = 1.0 / pv[l];
        for (int64_t p = dpj + 1; p < h.ce[j]; ++p) {
          double* a = L(p);
          for (int l = 0; l < W; ++l) a[l] *= inv[l];
        }
      }
    }
    // ---- the sparse columns' updates of the dense block
    const size_t ntask = h.schur_task.size() / 4;
    for (size_t t = 0; t < ntask; ++t) {
      const int jc = h.schur_task[4 * t], c = h.schur_task[4 * t + 1];
      const int e0 = h.schur_task[4 * t + 2], e1 = h.schur_task[4 * t + 3];
      const int64_t col = NS + (int64_t)jc * ndp + 32 * c;
      for (int e = e0; e < e1; ++e) {
        const int32_t xe = h.schur_ent[e];
        const double* lv = L(xe >> 5);
        const double* uv = L(h.schur_u[e]);
        double* a = L(col + (xe & 31));
        for (int l = 0; l < W; ++l) a[l] -= lv[l] * uv[l];
      }
    }
    // ---- dense trailing block: right-looking LU without pivoting, blocked
    // by panels of kPanel columns: the panel's columns and its rows to the
    // right first, then one pass over the trailing block per panel
    auto A = [&](int r, int c) { return L(NS + (int64_t)c * ndp + r); };
    for (int k = 0; k < ndp; k += kPanel) {
      const int ke = std::min(ndp, k + kPanel);
      for (int kk = k; kk < ke; ++kk) {
        double inv[W];
        const double* akk = A(kk, kk);
        for (int l = 0; l < W; ++l) inv[l] = 1.0 / akk[l];
        double* ck = A(0, kk);
        for (int r = kk + 1; r < ndp; ++r)
          for (int l = 0; l < W; ++l) ck[(size_t)r * W + l] *= inv[l];
        for (int c = kk + 1; c < ke; ++c) {  // the rest of the panel
          const double* u = A(kk, c);
          double* cc = A(0, c);
          for (int r = kk + 1; r < ndp; ++r)
            for (int l = 0; l < W; ++l) cc[(size_t)r * W + l] -= ck[(size_t)r * W + l] * u[l];
        }
      }
      for (int c = ke; c < ndp; ++c) {
        double* cc = A(0, c);
        // U12: rows k .. ke-1 of column c (unit lower L11)
        for (int kk = k; kk < ke; ++kk)
          for (int r = kk + 1; r < ke; ++r)
            for (int l = 0; l < W; ++l) cc[(size_t)r * W + l] -= A(r, kk)[l] * cc[(size_t)kk * W + l];
        // trailing rows of column c: one pass, kPanel multiply-adds per entry
        double u[kPanel][W];
        const int kw = ke - k;
        for (int q = 0; q < kw; ++q)
          for (int l = 0; l < W; ++l) u[q][l] = cc[(size_t)(k + q) * W + l];
        for (int r = ke; r < ndp; ++r) {
          double acc[W];
          for (int l = 0; l < W; ++l) acc[l] = cc[(size_t)r * W + l];
          for (int q = 0; q < kw; ++q) {
            const double* lr = A(r, k + q);
            for (int l = 0; l < W; ++l) acc[l] -= lr[l] * u[q][l];
          }
          for (int l = 0; l < W; ++l) cc[(size_t)r * W + l] = acc[l];
        }
      }
    }
    // ---- FS/BS (Sec. 4.3.3): sparse forward rows, dense forward and
    // backward, sparse backward rows
    for (size_t ri = 0; ri < h.fw_rows.size(); ++ri) {
      double* xi = X(h.fw_rows[ri]);
      for (int e = h.fw_ptr[ri]; e < h.fw_ptr[ri + 1]; ++e) {
        const double* lv = L(h.fw_pos[e]);
        const double* xk = X(h.fw_col[e]);
        for (int l = 0; l < W; ++l) xi[l] -= lv[l] * xk[l];
      }
    }
    for (int k = 0; k < ndp; ++k) {
      const double* xk = X(s + k);
      for (int r = k + 1; r < ndp; ++r) {
        const double* lv = L(NS + (int64_t)k * ndp + r);
        double* xr = X(s + r);
        for (int l = 0; l < W; ++l) xr[l] -= lv[l] * xk[l];
      }
    }
    for (int k = ndp - 1; k >= 0; --k) {
      double* xk = X(s + k);
      const double* pv = L(NS + (int64_t)k * ndp + k);
      for (int l = 0; l < W; ++l) xk[l] /= pv[l];
      for (int r = 0; r < k; ++r) {
        const double* uv = L(NS + (int64_t)k * ndp + r);
        double* xr = X(s + r);
        for (int l = 0; l < W; ++l) xr[l] -= uv[l] * xk[l];
      }
    }
    for (size_t ri = 0; ri < h.bw_rows.size(); ++ri) {
      const int i = h.bw_rows[ri];
      double* xi = X(i);
      for (int e = h.bw_ptr[ri]; e < h.bw_ptr[ri + 1]; ++e) {
        const double* uv = L(h.bw_pos[e]);
        const double* xj = X(h.bw_col[e]);
        for (int l = 0; l < W; ++l) xi[l] -= uv[l] * xj[l];
      }
      const double* pv = L(h.dp[i]);
      for (int l = 0; l < W; ++l) xi[l] /= pv[l];
    }
    // ---- update (Sec. 3 step 4), active lanes only
    for (int i = 0; i < n; ++i) {
      const int bt = h.bus_type[i];
      if (bt == 3) continue;
      const double* dth = X(h.rhs_pos_p[i]);
      const double* dvm = bt == 1 ? X(h.rhs_pos_q[i]) : nullptr;
      for (int l = 0; l < nb; ++l) {
        if (!active[l]) continue;
        const size_t o = (size_t)i * W + l;
        const double a = va[o] + dth[l];
        const double mg = vm[o] + (dvm ? dvm[l] : 0.0);
        if (!std::isfinite(a) || !std::isfinite(mg)) {
          bad[l] = true;
          continue;
        }
        va[o] = a;
        vm[o] = mg;
        ve[o] = mg * std::cos(a);
        vf[o] = mg * std::sin(a);
      }
    }
  }
  for (int l = 0; l < nb; ++l)
    for (int i = 0; i < n; ++i) {
      const size_t o = (size_t)i * W + l;
      v_out[((size_t)l * n + i) * 2] = ve[o];
      v_out[((size_t)l * n + i) * 2 + 1] = vf[o];
    }
}

}  // namespace

extern "C" int pf_solve_batch_cpu(pf_plan* p, int B, const double* sbus, const double* v0, double tol, int maxit,
                                  double* v_out, int32_t* iters, uint8_t* status, int threads) {
  if (!p || B < 0 || maxit < 0 || threads < 0 || !std::isfinite(tol) || tol < 0) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v0 || !v_out || !iters || !status) return NRPF_ERR_ARG;
  const nrpf::HostPlan& h = p->hp;
  const int n = h.n;
  const int groups = (B + kLanes - 1) / kLanes;
  int nt = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::min(nt, groups);
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  for (int w = 0; w < nt; ++w)
    pool.emplace_back([&] {
      std::vector<double> lu, x;
      for (int g; (g = next.fetch_add(1)) < groups;) {
        const int b0 = g * kLanes, nb = std::min(kLanes, B - b0);
        solve_group(h, nb, sbus + (size_t)b0 * n * 2, v0 + (size_t)b0 * n * 2, tol, maxit,
                    v_out + (size_t)b0 * n * 2, iters + b0, status + b0, lu, x);
      }
    });
  for (auto& t : pool) t.join();
  return NRPF_OK;
}
