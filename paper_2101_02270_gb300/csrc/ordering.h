// Fill-reducing symmetric ordering and bus-level symbolic factorisation.
#pragma once
#include <cstdint>
#include <vector>

namespace nrpf {

// Result of ordering a weighted undirected graph (vertex v carries w[v] scalar
// unknowns).  order[k] is the vertex eliminated k-th; lstruct[k] lists the
// elimination positions (> k) of the vertices in the k-th vertex's column of L
// (ascending).  Vertices at positions >= dense_start form a trailing block that
// is treated as completely dense.
struct Ordering {
  std::vector<int> order;
  std::vector<std::vector<int>> lstruct;
  int dense_start = 0;
};

// Approximate-minimum-degree elimination on a quotient graph (Amestoy, Davis &
// Duff, "An approximate minimum degree ordering algorithm", SIMAX 1996), with
// element absorption and weighted (scalar) external degrees.  Elimination stops
// once the cheapest remaining vertex is adjacent to at least `dense_frac` of the
// remaining scalar unknowns; the rest is ordered by ascending degree and marked
// dense.  adj must be symmetric without self loops.
//
// key picks the vertex eliminated next:
//  - kDegree: least approximate external degree d (minimum degree);
//  - kMeanFill: least mean local fill, (d^2 - c^2) / w[v], where c counts the
//    unknowns among the d that the newest element adjacent to v already
//    connects to each other.  This is the idea of the approximate minimum mean
//    local fill heuristic (Ng & Raghavan, "Performance of greedy ordering
//    heuristics for sparse Cholesky factorization", SIMAX 1999), in the
//    simplified form that only the newest element is subtracted.
// Ties between equal keys go to the lower vertex index when seed is 0, else to
// the lower rank in a seeded random permutation of the vertices.  Minimum
// degree leaves the tie-break open; on meshed grids it moves the fill by
// about 10%.
enum class OrderKey { kDegree = 0, kMeanFill = 1 };
Ordering amd_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w,
                   double dense_frac, uint64_t seed = 0, OrderKey key = OrderKey::kDegree);

// Multiply-adds of one LU refactorisation under an ordering (one instance),
// split into the columns eliminated sparsely (including their updates of the
// dense block) and the dense block itself padded to `panel`.
struct OrderingCost {
  double sparse_fma = 0;
  double dense_fma = 0;
};
OrderingCost ordering_cost(const Ordering& o, const std::vector<int>& w, int panel);

// Natural order (identity), same symbolic output: used by tests.
Ordering natural_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w);

}  // namespace nrpf
