// Fill-reducing ordering on the bus graph (Sec. 4.1: AMD pre-ordering, done
// once per sparsity pattern) and the bus-level column structure of L that the
// elimination produces.
#include "ordering.h"

#include <algorithm>
#include <numeric>
#include <set>
#include <utility>

namespace nrpf {

namespace {

Ordering eliminate(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w,
                   double dense_frac, bool use_degree) {
  std::vector<std::vector<int>> A(adj);   // variable -> adjacent live variables
  std::vector<std::vector<int>> E(nv);    // variable -> adjacent live elements
  std::vector<std::vector<int>> Le(nv);   // element -> boundary variables
  std::vector<long> Lw(nv, 0);            // weighted size of Le
  std::vector<char> elim(nv, 0), absorbed(nv, 0);
  std::vector<long> deg(nv, 0);
  std::vector<int> mark(nv, -1), we_mark(nv, -1);
  std::vector<long> we(nv, 0);
  std::vector<std::vector<int>> lst(nv);  // per vertex: L column structure (vertices)
  long remaining_w = 0;
  for (int i = 0; i < nv; ++i) remaining_w += w[i];
  std::set<std::pair<long, int>> heap;
  if (use_degree) {
    for (int i = 0; i < nv; ++i) {
      long d = 0;
      for (int j : A[i]) d += w[j];
      deg[i] = d;
      heap.insert({d, i});
    }
  }
  Ordering out;
  out.order.reserve(nv);
  int k = 0;
  std::vector<int> Lp;
  for (; k < nv; ++k) {
    int p;
    if (use_degree) {
      p = heap.begin()->second;
      if (dense_frac < 1.0 && nv - k > 1 &&
          (double)deg[p] >= dense_frac * (double)(remaining_w - w[p])) {
        break;  // remaining graph is dense: stop here
      }
      heap.erase(heap.begin());
    } else {
      p = k;
    }
    elim[p] = 1;
    remaining_w -= w[p];
    out.order.push_back(p);
    // Boundary of the new element p: live neighbours reached directly or
    // through p's adjacent elements, which are absorbed.
    Lp.clear();
    const int stamp = k;
    for (int j : A[p])
      if (!elim[j] && mark[j] != stamp) { mark[j] = stamp; Lp.push_back(j); }
    for (int e : E[p]) {
      if (absorbed[e]) continue;
      for (int j : Le[e])
        if (!elim[j] && mark[j] != stamp) { mark[j] = stamp; Lp.push_back(j); }
      absorbed[e] = 1;
      std::vector<int>().swap(Le[e]);
    }
    std::vector<int>().swap(A[p]);
    std::vector<int>().swap(E[p]);
    long lpw = 0;
    for (int j : Lp) lpw += w[j];
    Le[p] = Lp;
    Lw[p] = lpw;
    lst[p] = Lp;
    for (int i : Lp) {
      auto& Ei = E[i];
      Ei.erase(std::remove_if(Ei.begin(), Ei.end(), [&](int e) { return absorbed[e] != 0; }), Ei.end());
      Ei.push_back(p);
      auto& Ai = A[i];
      Ai.erase(std::remove_if(Ai.begin(), Ai.end(), [&](int j) { return elim[j] || mark[j] == stamp; }),
               Ai.end());
    }
    if (!use_degree) continue;
    // Approximate external degrees of the boundary variables.
    for (int i : Lp)
      for (int e : E[i]) {
        if (e == p) continue;
        if (we_mark[e] != stamp) { we_mark[e] = stamp; we[e] = Lw[e]; }
        we[e] -= w[i];
      }
    for (int i : Lp) {
      long ext = lpw - w[i];
      for (int j : A[i]) ext += w[j];
      for (int e : E[i])
        if (e != p) ext += std::max(we[e], 0L);
      long d = std::min({remaining_w - w[i], deg[i] + lpw - w[i], ext});
      if (d != deg[i]) {
        heap.erase({deg[i], i});
        deg[i] = d;
        heap.insert({d, i});
      }
    }
  }
  out.dense_start = k;
  if (k < nv) {
    // Dense tail: remaining variables in ascending degree order.
    std::vector<int> rest;
    for (auto& pr : heap) rest.push_back(pr.second);
    for (int v : rest) out.order.push_back(v);
  }
  std::vector<int> pos(nv);
  for (int i = 0; i < nv; ++i) pos[out.order[i]] = i;
  out.lstruct.assign(nv, {});
  for (int q = 0; q < nv; ++q) {
    auto& dst = out.lstruct[q];
    if (q < out.dense_start) {
      for (int v : lst[out.order[q]]) dst.push_back(pos[v]);
      std::sort(dst.begin(), dst.end());
    } else {
      for (int r = q + 1; r < nv; ++r) dst.push_back(r);
    }
  }
  return out;
}

}  // namespace

Ordering amd_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w,
                   double dense_frac) {
  return eliminate(nv, adj, w, dense_frac, true);
}

Ordering natural_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w) {
  Ordering o = eliminate(nv, adj, w, 1.0, false);
  o.dense_start = nv;
  return o;
}

}  // namespace nrpf
