// Symbolic analysis for the batched Newton-Raphson solver (host side, once per
// sparsity pattern): input validation, bus maps, Jacobian pattern, bus-level
// fill-reducing ordering, LU fill pattern with a trailing dense block, static
// Ybus -> LU lookup and the level schedules of the refactor and of FS/BS.
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <set>
#include <thread>

#include "../../include/nrpf.h"
#include "ordering.h"

namespace nrpf {

int64_t HostPlan::pos(int r, int c) const {
  if (r < 0 || c < 0 || r >= m || c >= m) return -1;
  if (c >= s && r >= s) return NS + (int64_t)(c - s) * ndp + (r - s);
  const int32_t* b = seg_row.data() + cs[c];
  const int32_t* e = seg_row.data() + ce[c];
  const int32_t* it = std::lower_bound(b, e, r);
  if (it == e || *it != r) return -1;
  return cs[c] + (it - b);
}

namespace {

int validate(int n, const int32_t* rowptr, const int32_t* colidx, const double* yre,
             const double* yim, const int8_t* bt, std::string& err) {
  if (n <= 0) { err = "n must be positive"; return NRPF_ERR_ARG; }
  if (!rowptr || !colidx || !yre || !yim || !bt) { err = "null input"; return NRPF_ERR_ARG; }
  if (rowptr[0] != 0) { err = "rowptr[0] != 0"; return NRPF_ERR_PATTERN; }
  for (int i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) { err = "rowptr not monotone"; return NRPF_ERR_PATTERN; }
    bool diag = false;
    for (int d = rowptr[i]; d < rowptr[i + 1]; ++d) {
      int c = colidx[d];
      if (c < 0 || c >= n) { err = "column index out of range"; return NRPF_ERR_PATTERN; }
      if (d > rowptr[i] && colidx[d - 1] >= c) { err = "columns not strictly ascending"; return NRPF_ERR_PATTERN; }
      if (c == i) diag = true;
      if (!std::isfinite(yre[d]) || !std::isfinite(yim[d])) { err = "non-finite admittance"; return NRPF_ERR_ARG; }
    }
    if (!diag) { err = "missing diagonal"; return NRPF_ERR_PATTERN; }
  }
  // structural symmetry
  for (int i = 0; i < n; ++i)
    for (int d = rowptr[i]; d < rowptr[i + 1]; ++d) {
      int c = colidx[d];
      const int32_t* b = colidx + rowptr[c];
      const int32_t* e = colidx + rowptr[c + 1];
      if (!std::binary_search(b, e, i)) { err = "pattern not symmetric"; return NRPF_ERR_PATTERN; }
    }
  int nslack = 0;
  for (int i = 0; i < n; ++i) {
    if (bt[i] != 1 && bt[i] != 2 && bt[i] != 3) { err = "bus type not in {1,2,3}"; return NRPF_ERR_PATTERN; }
    nslack += bt[i] == 3;
  }
  if (nslack == 0) { err = "no slack bus"; return NRPF_ERR_PATTERN; }
  return NRPF_OK;
}

}  // namespace

int build_plan(int n, const int32_t* rowptr, const int32_t* colidx, const double* yre,
               const double* yim, const int8_t* bt, int ordering, double dense_frac, int kb,
               int order_tries, double sparse_weight, HostPlan& P, std::string& err) {
  int rc = validate(n, rowptr, colidx, yre, yim, bt, err);
  if (rc) return rc;
  if (kb != 4 && kb != 8 && kb != 16 && kb != 32 && kb != 64) {
    err = "panel must be 4, 8, 16, 32 or 64";
    return NRPF_ERR_ARG;
  }
  if (order_tries < 1 || !(sparse_weight >= 0.0)) {
    err = "order_tries must be >= 1 and sparse_weight >= 0";
    return NRPF_ERR_ARG;
  }
  const int nnzY = rowptr[n];
  P.n = n;
  P.kb = kb;
  P.rowptr.assign(rowptr, rowptr + n + 1);
  P.colidx.assign(colidx, colidx + nnzY);
  P.yre.assign(yre, yre + nnzY);
  P.yim.assign(yim, yim + nnzY);
  P.bus_type.assign(bt, bt + n);

  // ---- vertices of the ordering: non-slack buses, weight = unknowns ----
  std::vector<int> vbus, vid(n, -1), w;
  for (int i = 0; i < n; ++i) {
    if (bt[i] == 3) { P.nslack++; continue; }
    vid[i] = (int)vbus.size();
    vbus.push_back(i);
    w.push_back(bt[i] == 1 ? 2 : 1);
    if (bt[i] == 1) P.npq++; else P.npv++;
  }
  const int nv = (int)vbus.size();
  P.m = P.npv + 2 * P.npq;
  const int m = P.m;
  std::vector<std::vector<int>> adj(nv);
  for (int v = 0; v < nv; ++v) {
    int i = vbus[v];
    for (int d = rowptr[i]; d < rowptr[i + 1]; ++d) {
      int c = colidx[d];
      if (c != i && vid[c] >= 0) adj[v].push_back(vid[c]);
    }
  }
  Ordering ord;
  if (ordering == NRPF_ORDER_NATURAL) {
    ord = natural_order(nv, adj, w);
  } else {
    // one try: minimum degree, seed 0; more: seeds 0 .. order_tries-1 with
    // each key (try t: key t / order_tries, seed t % order_tries).  The tries
    // are independent: they run on the host's threads, and the ordering kept
    // is the cheapest, the lowest try among equal costs, for any thread count
    const int ntries = order_tries > 1 ? 2 * order_tries : 1;
    auto key_of = [&](int t) { return t < order_tries ? OrderKey::kDegree : OrderKey::kMeanFill; };
    std::vector<double> cost(ntries, 0.0);
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::min(ntries, (int)std::min(16u, hw));
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    auto work = [&] {
      try {
        for (int t; (t = next.fetch_add(1)) < ntries;) {
          const Ordering o = amd_order(nv, adj, w, dense_frac, (uint64_t)(t % order_tries), key_of(t));
          const OrderingCost c = ordering_cost(o, w, kb);
          cost[t] = c.dense_fma + sparse_weight * c.sparse_fma;
        }
      } catch (...) {
        failed = true;
      }
    };
    if (nt <= 1) {
      work();
    } else {
      // a thread that cannot be created leaves its share to the others and
      // to this thread; the threads started are always joined
      std::vector<std::thread> pool;
      pool.reserve(nt);
      for (int i = 0; i < nt; ++i) {
        try {
          pool.emplace_back(work);
        } catch (...) {
          break;
        }
      }
      work();
      for (auto& th : pool) th.join();
    }
    if (failed) { err = "out of host memory while ordering"; return NRPF_ERR_NOMEM; }
    int best = 0;
    for (int t = 1; t < ntries; ++t)
      if (cost[t] < cost[best]) best = t;
    ord = amd_order(nv, adj, w, dense_frac, (uint64_t)(best % order_tries), key_of(best));
    P.order_seed = (uint64_t)(best % order_tries);
    P.order_key = (int)key_of(best);
  }

  // ---- scalar positions: per bus in elimination order, angle then |V| ----
  P.th_pos.assign(n, -1);
  P.vm_pos.assign(n, -1);
  std::vector<int> qbase(nv + 1, 0);
  for (int q = 0; q < nv; ++q) {
    int bus = vbus[ord.order[q]];
    qbase[q + 1] = qbase[q] + (bt[bus] == 1 ? 2 : 1);
    P.th_pos[bus] = qbase[q];
    if (bt[bus] == 1) P.vm_pos[bus] = qbase[q] + 1;
  }
  // J order (rows and columns alike): angles / P equations of the PV buses,
  // then of the PQ buses, then magnitudes / Q equations of the PQ buses, each
  // group in ascending bus order.
  P.unk_pos.clear();
  for (int i = 0; i < n; ++i) if (bt[i] == 2) P.unk_pos.push_back(P.th_pos[i]);
  for (int i = 0; i < n; ++i) if (bt[i] == 1) P.unk_pos.push_back(P.th_pos[i]);
  for (int i = 0; i < n; ++i) if (bt[i] == 1) P.unk_pos.push_back(P.vm_pos[i]);
  P.s = ord.dense_start < nv ? qbase[ord.dense_start] : m;
  P.nd = m - P.s;
  P.ndp = P.nd ? (P.nd + kb - 1) / kb * kb : 0;
  const int s = P.s;

  // ---- scalar L pattern of the sparse columns (rows > j, ascending) ----
  std::vector<std::vector<int>> Lpat(s);
  for (int q = 0; q < ord.dense_start && q < nv; ++q) {
    int bus = vbus[ord.order[q]];
    std::vector<int> rows;
    for (int r : ord.lstruct[q])
      for (int t = qbase[r]; t < qbase[r + 1]; ++t) rows.push_back(t);
    int j0 = qbase[q];
    if (bt[bus] == 1) {
      Lpat[j0].push_back(j0 + 1);
      Lpat[j0].insert(Lpat[j0].end(), rows.begin(), rows.end());
      Lpat[j0 + 1] = rows;
    } else {
      Lpat[j0] = rows;
    }
  }
  // U row structure of every column: k < j with j in Lpat(k), k < s.
  std::vector<std::vector<int>> Ustr(m);
  for (int k = 0; k < s; ++k)
    for (int i : Lpat[k]) Ustr[i].push_back(k);  // ascending k by construction

  // ---- segments ----
  P.cs.assign(m, 0);
  P.ce.assign(m, 0);
  P.dp.assign(m, -1);
  P.seg_row.clear();
  for (int j = 0; j < m; ++j) {
    P.cs[j] = (int64_t)P.seg_row.size();
    for (int k : Ustr[j]) P.seg_row.push_back(k);
    if (j < s) {
      P.dp[j] = (int32_t)P.seg_row.size();
      P.seg_row.push_back(j);
      for (int i : Lpat[j]) P.seg_row.push_back(i);
    }
    P.ce[j] = (int64_t)P.seg_row.size();
  }
  P.NS = (int64_t)P.seg_row.size();
  P.NLU = P.NS + (int64_t)P.ndp * P.ndp;
  if (P.NLU >= (int64_t)1 << 31) { err = "LU too large for 32-bit positions"; return NRPF_ERR_NOMEM; }
  P.nnz_pattern = P.NS + (int64_t)P.nd * P.nd;

  // ---- static lookup: Ybus entry -> A positions ----
  P.jmap.assign((size_t)nnzY * 4, -1);
  P.nnz_j = 0;
  for (int i = 0; i < n; ++i)
    for (int d = rowptr[i]; d < rowptr[i + 1]; ++d) {
      int k = colidx[d];
      if (bt[i] == 3 || bt[k] == 3) continue;
      int32_t* jm = &P.jmap[(size_t)d * 4];
      int64_t p0 = P.pos(P.th_pos[i], P.th_pos[k]);
      int64_t p1 = bt[k] == 1 ? P.pos(P.th_pos[i], P.vm_pos[k]) : -2;
      int64_t p2 = bt[i] == 1 ? P.pos(P.vm_pos[i], P.th_pos[k]) : -2;
      int64_t p3 = (bt[i] == 1 && bt[k] == 1) ? P.pos(P.vm_pos[i], P.vm_pos[k]) : -2;
      if (p0 == -1 || p1 == -1 || p2 == -1 || p3 == -1) { err = "internal: J entry outside LU pattern"; return NRPF_ERR_PATTERN; }
      jm[0] = (int32_t)p0;
      jm[1] = (int32_t)std::max<int64_t>(p1, -1);
      jm[2] = (int32_t)std::max<int64_t>(p2, -1);
      jm[3] = (int32_t)std::max<int64_t>(p3, -1);
      for (int t = 0; t < 4; ++t) P.nnz_j += jm[t] >= 0;
    }
  P.one_pos.clear();
  // (the Schur tasks' Jacobian-row masks are filled after the tasks exist)
  for (int t = P.nd; t < P.ndp; ++t) P.one_pos.push_back((int32_t)(P.NS + (int64_t)t * P.ndp + t));
  P.rhs_pos_p.assign(n, -1);
  P.rhs_pos_q.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    if (bt[i] != 3) P.rhs_pos_p[i] = P.th_pos[i];
    if (bt[i] == 1) P.rhs_pos_q[i] = P.vm_pos[i];
  }

  // ---- left-looking refactor updates and levels ----
  std::vector<int> level(m, 0);
  P.col_upd_ptr.assign(m + 1, 0);
  P.upd.clear();
  P.dst.clear();
  double fma = 0;
  for (int k = 0; k < s; ++k)
    if (!std::is_sorted(Lpat[k].begin(), Lpat[k].end())) { err = "internal: L pattern not sorted"; return NRPF_ERR_PATTERN; }
  P.schur_task.clear(); P.schur_ent.clear(); P.schur_u.clear(); P.schur_jmask.clear();
  for (int j = 0; j < m; ++j) {
    int lv = 0;
    for (int k : Ustr[j]) {  // k < s, ascending
      lv = std::max(lv, level[k] + 1);
      // rows of L(:, k) below s go to the level schedule; for a dense column
      // the rows >= s (ascending, after them) go to the Schur tasks
      int nsp = (int)Lpat[k].size();
      if (j >= s) nsp = (int)(std::lower_bound(Lpat[k].begin(), Lpat[k].end(), s) - Lpat[k].begin());
      fma += (double)Lpat[k].size();
      if (nsp == 0) continue;
      Upd u;
      u.ukj = (int32_t)P.pos(k, j);
      u.lsrc = P.dp[k] + 1;
      u.llen = nsp;
      u.dst_off = (int32_t)P.dst.size();
      if (P.dst.size() + nsp >= ((size_t)1 << 31)) {
        err = "refactor schedule exceeds 2^31 updates (use the AMD ordering)";
        return NRPF_ERR_NOMEM;
      }
      for (int q = 0; q < nsp; ++q) {
        int64_t pp = P.pos(Lpat[k][q], j);
        if (pp < 0) { err = "internal: fill pattern not closed"; return NRPF_ERR_PATTERN; }
        P.dst.push_back((int32_t)pp);
      }
      P.upd.push_back(u);
    }
    if (j >= s && P.nd > 0) {
      const int nch = (P.ndp + 31) / 32;
      for (int c = 0; c < nch; ++c) {
        const int e0 = (int)P.schur_ent.size();
        for (int k : Ustr[j]) {
          const int32_t ukj = (int32_t)P.pos(k, j);
          auto it = std::lower_bound(Lpat[k].begin(), Lpat[k].end(), s + 32 * c);
          for (; it != Lpat[k].end() && *it < s + 32 * c + 32; ++it) {
            const int64_t lpos = P.dp[k] + 1 + (it - Lpat[k].begin());
            if (lpos >= ((int64_t)1 << 26)) { err = "LU too large for the Schur task encoding"; return NRPF_ERR_NOMEM; }
            const int r = *it - s - 32 * c;
            P.schur_ent.push_back((int32_t)((lpos << 5) | r));
            P.schur_u.push_back(ukj);
          }
        }
        if (P.schur_ent.size() >= ((size_t)1 << 31)) { err = "Schur task list exceeds 2^31 entries"; return NRPF_ERR_NOMEM; }
        P.schur_task.insert(P.schur_task.end(), {j - s, c, e0, (int32_t)P.schur_ent.size()});
        P.schur_jmask.push_back(0u);
      }
    }
    level[j] = lv;
    P.col_upd_ptr[j + 1] = (int32_t)P.upd.size();
  }
  // Sparse columns need a task (normalisation) even without updates; dense
  // columns only when they receive updates from the sparse part.
  int nlv = 0;
  for (int j = 0; j < m; ++j)
    if (j < s || P.col_upd_ptr[j + 1] > P.col_upd_ptr[j]) nlv = std::max(nlv, level[j] + 1);
  P.lu_lvl_ptr.assign(nlv + 1, 0);
  P.lu_lvl_cols.clear();
  for (int l = 0; l < nlv; ++l) {
    for (int j = 0; j < m; ++j)
      if (level[j] == l && (j < s || P.col_upd_ptr[j + 1] > P.col_upd_ptr[j])) P.lu_lvl_cols.push_back(j);
    P.lu_lvl_ptr[l + 1] = (int32_t)P.lu_lvl_cols.size();
  }
  // rows of each Schur task's chunk that hold a Jacobian entry
  if (P.nd > 0) {
    const int nch = (P.ndp + 31) / 32;
    for (int32_t q : P.jmap) {
      if (q < P.NS) continue;
      const int64_t d = q - P.NS;
      const int col = (int)(d / P.ndp), row = (int)(d % P.ndp);
      P.schur_jmask[(size_t)col * nch + row / 32] |= 1u << (row % 32);
    }
  }
  for (int j = 0; j < s; ++j) fma += (double)(P.ce[j] - P.dp[j] - 1);  // normalisation
  for (int k = 0; k < P.ndp; ++k) {
    double r = P.ndp - k - 1;
    fma += r + r * r;
  }
  P.lu_fma = fma;

  // ---- forward substitution (unit L), rows by level; all rows gather the
  //      contributions of sparse columns, the dense block follows ----
  {
    std::vector<std::vector<std::pair<int, int>>> rowent(m);  // (pos, k)
    for (int k = 0; k < s; ++k)
      for (int64_t p = P.dp[k] + 1; p < P.ce[k]; ++p) rowent[P.seg_row[p]].push_back({(int)p, k});
    std::vector<int> fl(m, 0);
    int nl = 0;
    for (int i = 0; i < m; ++i) {
      int lv = 0;
      for (auto& e : rowent[i]) lv = std::max(lv, fl[e.second] + 1);
      fl[i] = lv;
      if (i < s || !rowent[i].empty()) nl = std::max(nl, lv + 1);
    }
    // rows with nothing to gather need no task
    P.fw_ptr.assign(1, 0);
    P.fw_lvl_ptr.assign(1, 0);
    P.fw_rows.clear(); P.fw_pos.clear(); P.fw_col.clear();
    std::vector<int> rowslot;
    for (int l = 0; l < nl; ++l) {
      for (int i = 0; i < m; ++i) {
        if (fl[i] != l || rowent[i].empty()) continue;
        P.fw_rows.push_back(i);
        for (auto& e : rowent[i]) { P.fw_pos.push_back(e.first); P.fw_col.push_back(e.second); }
        P.fw_ptr.push_back((int32_t)P.fw_pos.size());
      }
      P.fw_lvl_ptr.push_back((int32_t)P.fw_rows.size());
    }
    // drop empty trailing levels
    while (P.fw_lvl_ptr.size() > 1 && P.fw_lvl_ptr[P.fw_lvl_ptr.size() - 1] == P.fw_lvl_ptr[P.fw_lvl_ptr.size() - 2])
      P.fw_lvl_ptr.pop_back();
  }
  // ---- backward substitution: rows i < s, x_i = (y_i - sum U(i,j) x_j) / U(i,i) ----
  {
    std::vector<std::vector<std::pair<int, int>>> rowent(s);  // (pos of U(i,j), j)
    for (int j = 0; j < m; ++j)
      for (int64_t p = P.cs[j]; p < (j < s ? P.dp[j] : P.ce[j]); ++p) rowent[P.seg_row[p]].push_back({(int)p, j});
    std::vector<int> bl(m, -1);
    int nl = 0;
    for (int i = s - 1; i >= 0; --i) {
      int lv = 0;
      for (auto& e : rowent[i]) if (e.second < s) lv = std::max(lv, bl[e.second] + 1);
      bl[i] = lv;
      nl = std::max(nl, lv + 1);
    }
    P.bw_ptr.assign(1, 0);
    P.bw_lvl_ptr.assign(1, 0);
    P.bw_rows.clear(); P.bw_pos.clear(); P.bw_col.clear();
    for (int l = 0; l < nl; ++l) {
      for (int i = 0; i < s; ++i) {
        if (bl[i] != l) continue;
        P.bw_rows.push_back(i);
        for (auto& e : rowent[i]) { P.bw_pos.push_back(e.first); P.bw_col.push_back(e.second); }
        P.bw_ptr.push_back((int32_t)P.bw_pos.size());
      }
      P.bw_lvl_ptr.push_back((int32_t)P.bw_rows.size());
    }
  }
  P.solve_fma = (double)P.fw_pos.size() + (double)P.bw_pos.size() + (double)s +
                (double)P.ndp * P.ndp;
  return NRPF_OK;
}

}  // namespace nrpf
