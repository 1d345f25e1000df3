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

// splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the tie-break ranks of a seeded ordering.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// rank[v] breaks ties between vertices of equal approximate degree: seed 0
// keeps the vertex order, any other seed a Fisher-Yates shuffle of it.
std::vector<int> tie_ranks(int nv, uint64_t seed) {
  std::vector<int> rank(nv);
  std::iota(rank.begin(), rank.end(), 0);
  if (seed == 0) return rank;
  uint64_t x = seed;
  for (int i = nv - 1; i > 0; --i) {
    const int j = (int)(splitmix64(x) % (uint64_t)(i + 1));
    std::swap(rank[i], rank[j]);
  }
  return rank;
}

Ordering eliminate(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w,
                   double dense_frac, bool use_degree, uint64_t seed, OrderKey okey) {
  std::vector<std::vector<int>> A(adj);   // variable -> adjacent live variables
  std::vector<std::vector<int>> E(nv);    // variable -> adjacent live elements
  std::vector<std::vector<int>> Le(nv);   // element -> boundary variables
  std::vector<long> Lw(nv, 0);            // weighted size of Le
  std::vector<char> elim(nv, 0), absorbed(nv, 0);
  std::vector<long> deg(nv, 0), key(nv, 0);
  // heap key of a variable of approximate external degree d whose newest
  // element leaves c of those unknowns already connected to each other
  auto score = [&](int i, long d, long c) -> long {
    if (okey == OrderKey::kDegree) return d;
    // mean local fill: the new pairs among the d neighbours, (d^2 - c^2)/2,
    // over the unknowns of the vertex (its weight)
    return (d * d - c * c) / w[i];
  };
  std::vector<int> mark(nv, -1), we_mark(nv, -1);
  std::vector<long> we(nv, 0);
  std::vector<std::vector<int>> lst(nv);  // per vertex: L column structure (vertices)
  long remaining_w = 0;
  for (int i = 0; i < nv; ++i) remaining_w += w[i];
  // (key, tie-break rank); byrank maps a rank back to its vertex
  std::set<std::pair<long, int>> heap;
  const std::vector<int> rank = tie_ranks(nv, seed);
  std::vector<int> byrank(nv);
  for (int i = 0; i < nv; ++i) byrank[rank[i]] = i;
  if (use_degree) {
    for (int i = 0; i < nv; ++i) {
      long d = 0;
      for (int j : A[i]) d += w[j];
      deg[i] = d;
      key[i] = score(i, d, 0);
      heap.insert({key[i], rank[i]});
    }
  }
  Ordering out;
  out.order.reserve(nv);
  int k = 0;
  std::vector<int> Lp;
  for (; k < nv; ++k) {
    int p;
    if (use_degree) {
      p = byrank[heap.begin()->second];
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
      const long kk = score(i, d, lpw - w[i]);
      if (kk != key[i]) {
        heap.erase({key[i], rank[i]});
        key[i] = kk;
        heap.insert({kk, rank[i]});
      }
      deg[i] = d;
    }
  }
  out.dense_start = k;
  if (k < nv) {
    // Dense tail: remaining variables in ascending key order.
    std::vector<int> rest;
    for (auto& pr : heap) rest.push_back(byrank[pr.second]);
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
                   double dense_frac, uint64_t seed, OrderKey key) {
  return eliminate(nv, adj, w, dense_frac, true, seed, key);
}

Ordering natural_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w) {
  Ordering o = eliminate(nv, adj, w, 1.0, false, 0, OrderKey::kDegree);
  o.dense_start = nv;
  return o;
}

OrderingCost ordering_cost(const Ordering& o, const std::vector<int>& w, int panel) {
  OrderingCost c;
  const int nv = (int)o.order.size();
  // scalar L column of the t-th unknown of the vertex at position q: the
  // vertex's later unknowns plus every unknown of the vertices in lstruct[q];
  // a left-looking refactor spends r (scaling) + r^2 (updates) multiply-adds
  // on a column with r entries below the diagonal (symmetric pattern)
  int nd = 0;
  for (int q = 0; q < nv; ++q) {
    const int wq = w[o.order[q]];
    if (q >= o.dense_start) { nd += wq; continue; }
    double ext = 0;
    for (int r : o.lstruct[q]) ext += w[o.order[r]];
    for (int t = 0; t < wq; ++t) {
      const double r = (double)(wq - 1 - t) + ext;
      c.sparse_fma += r + r * r;
    }
  }
  const int ndp = nd ? (nd + panel - 1) / panel * panel : 0;
  for (int k = 0; k < ndp; ++k) {
    const double r = ndp - k - 1;
    c.dense_fma += r + r * r;
  }
  return c;
}

}  // namespace nrpf
