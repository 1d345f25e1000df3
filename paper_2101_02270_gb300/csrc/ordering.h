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
Ordering amd_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w,
                   double dense_frac);

// Natural order (identity), same symbolic output: used by tests.
Ordering natural_order(int nv, const std::vector<std::vector<int>>& adj, const std::vector<int>& w);

}  // namespace nrpf
