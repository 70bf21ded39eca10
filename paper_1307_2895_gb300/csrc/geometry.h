// Host geometry of the nested-dissection tree (Section 3.1, 3.2) and the
// index sets of cells and fronts at each level.
#pragma once
#include <cstdint>
#include <vector>

namespace hif {

struct Geometry {
  int dim = 2, n = 0, m = 0, L = 0, leaf = 8;
  int64_t N = 0;
  // cls[l][x], x = 0..n: interval index (>= 0) of coordinate x among the
  // level-l cells, or -(ordinal+1) when x is the ordinal-th level-l separator.
  std::vector<std::vector<int>> cls;
  std::vector<int> ncell;   // cells per axis at level l (2^(L-l))

  void init(int dim_, int n_, int leaf_);
  inline void coords(int64_t g, int x[3]) const {
    x[0] = (int)(g % m) + 1;
    x[1] = (int)((g / m) % m) + 1;
    x[2] = dim == 3 ? (int)(g / ((int64_t)m * m)) + 1 : 1;
  }
  inline int ncells(int l) const {
    int c = 1;
    for (int a = 0; a < dim; ++a) c *= ncell[l];
    return c;
  }
};

// Index sets of one level: cells (interior I, boundary B) and, after the
// interiors are eliminated, fronts (strict interiors of edges / faces).
struct HostCell {
  std::vector<int> I, B;
  int child[8];
};

struct HostFront {
  int axis = 0, P1 = -1, P2 = -1;
  std::vector<int> c;           // front DOFs, ascending
  std::vector<int> N;           // neighbours, ascending
  std::vector<int> pos1, pos2;  // positions in B_P1 / B_P2 of [c ; N] (-1 absent)
};

// Cells of level l from the alive DOFs (ascending list).
void build_cells(const Geometry& G, int l, const std::vector<int>& alive, std::vector<HostCell>& cells);

// Child maps of level-l cells into the level-(l-1) boundaries:
// out[(a) * 8 + s] for the frontal index a of cell P (I then B) and child slot s.
void build_child_map(const Geometry& G, int l, const HostCell& P, int cell_lin,
                     const std::vector<HostCell>& prev, std::vector<int>& out, int child[8]);
void build_child_map(const Geometry& G, int l, const HostCell& P, int cell_lin,
                     const std::vector<HostCell>& prev, int* out, int child[8]);

// Fronts of level l + 1/2 from the DOFs alive after the level-l elimination.
void build_fronts(const Geometry& G, int l, const std::vector<int>& alive,
                  const std::vector<HostCell>& cells, std::vector<HostFront>& fronts,
                  std::vector<int>& scratch_mark);

}  // namespace hif
