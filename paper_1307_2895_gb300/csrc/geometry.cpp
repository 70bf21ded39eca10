// Host tree and block-index builder.
//
// Separators (Section 3.1): for n = 2^L m the level-l separators sit every
// 2^l m grid lines.  For other n the separator positions are round(i n / 2^L),
// i = 1..2^L-1 (half up), and level l keeps every 2^l-th of them, so the
// levels still nest.  L = max(1, round(log2(n / leaf))).
//
// Fronts (Section 4.3, accelerated compression): the DOFs with exactly one
// coordinate on a level-l separator, grouped by that separator and the cell
// intervals of the other coordinates (the strict interior of a 2D edge or a
// 3D face).  DOFs with two or more separator coordinates (2D corners, 3D cell
// edges and corners) belong to no front.
#include "geometry.h"

#include <algorithm>
#include <cmath>

namespace hif {

void Geometry::init(int dim_, int n_, int leaf_) {
  dim = dim_;
  n = n_;
  leaf = leaf_ > 0 ? leaf_ : 8;
  m = n - 1;
  N = 1;
  for (int a = 0; a < dim; ++a) N *= m;
  L = (int)std::lround(std::log2((double)n / (double)leaf));
  if (L < 1) L = 1;
  const int P = 1 << L;
  std::vector<int> sep(P);            // sep[i], i = 1..P-1
  for (int i = 1; i < P; ++i) sep[i] = (int)((2LL * i * n + P) / (2LL * P));
  // top[x]: highest level at which x is a separator (-1: never); separator i
  // belongs to the levels l with 2^l dividing i.
  std::vector<int> top(n + 1, -1);
  for (int i = 1; i < P; ++i) {
    int t = 0;
    while (((i >> t) & 1) == 0) ++t;
    top[sep[i]] = t;
  }
  cls.assign(L + 1, std::vector<int>(n + 1, 0));
  ncell.assign(L + 1, 1);
  for (int l = 0; l <= L; ++l) {
    ncell[l] = 1 << (L - l);
    std::vector<int>& c = cls[l];
    int ord = 0;
    for (int x = 0; x <= n; ++x) {
      const bool on = top[x] >= l;
      if (on) { c[x] = -(ord + 1); ++ord; }
      else c[x] = ord;                // number of level-l separators below x
    }
  }
}

static inline int lin_index(const int iv[3], int dim, int nc) {
  int lin = 0;
  for (int a = dim - 1; a >= 0; --a) lin = lin * nc + iv[a];
  return lin;
}

void build_cells(const Geometry& G, int l, const std::vector<int>& alive, std::vector<HostCell>& cells) {
  const int nc = G.ncell[l];
  const int ncells = G.ncells(l);
  cells.assign(ncells, HostCell{});
  const std::vector<int>& cl = G.cls[l];
  for (int g : alive) {
    int x[3];
    G.coords(g, x);
    int lo[3], hi[3];
    bool interior = true;
    for (int a = 0; a < 3; ++a) {
      if (a >= G.dim) { lo[a] = hi[a] = 0; continue; }
      const int c = cl[x[a]];
      if (c >= 0) { lo[a] = hi[a] = c; }
      else { lo[a] = -c - 1; hi[a] = -c; interior = false; }
    }
    if (interior) {
      cells[lin_index(lo, G.dim, nc)].I.push_back(g);
      continue;
    }
    int iv[3];
    for (iv[2] = lo[2]; iv[2] <= hi[2]; ++iv[2])
      for (iv[1] = lo[1]; iv[1] <= hi[1]; ++iv[1])
        for (iv[0] = lo[0]; iv[0] <= hi[0]; ++iv[0])
          cells[lin_index(iv, G.dim, nc)].B.push_back(g);
  }
}

void build_child_map(const Geometry& G, int l, const HostCell& P, int cell_lin,
                     const std::vector<HostCell>& prev, std::vector<int>& out, int child[8]) {
  const int nc = G.ncell[l], ncp = G.ncell[l - 1];
  const int nchild = 1 << G.dim;
  int iv[3] = {0, 0, 0};
  {
    int t = cell_lin;
    for (int a = 0; a < G.dim; ++a) { iv[a] = t % nc; t /= nc; }
  }
  for (int s = 0; s < 8; ++s) child[s] = -1;
  for (int s = 0; s < nchild; ++s) {
    int civ[3] = {0, 0, 0};
    for (int a = 0; a < G.dim; ++a) civ[a] = 2 * iv[a] + ((s >> a) & 1);
    child[s] = lin_index(civ, G.dim, ncp);
  }
  const int nF = (int)(P.I.size() + P.B.size());
  out.assign((size_t)nF * 8, -1);
  for (int s = 0; s < nchild; ++s) {
    const std::vector<int>& cb = prev[child[s]].B;
    // both lists ascending: merge-walk I and B separately
    for (int part = 0; part < 2; ++part) {
      const std::vector<int>& v = part == 0 ? P.I : P.B;
      const int base = part == 0 ? 0 : (int)P.I.size();
      size_t j = 0;
      for (size_t i = 0; i < v.size(); ++i) {
        while (j < cb.size() && cb[j] < v[i]) ++j;
        if (j < cb.size() && cb[j] == v[i]) out[(size_t)(base + i) * 8 + s] = (int)j;
      }
    }
  }
}

void build_fronts(const Geometry& G, int l, const std::vector<int>& alive,
                  const std::vector<HostCell>& cells, std::vector<HostFront>& fronts,
                  std::vector<int>& mark) {
  const int nc = G.ncell[l];
  const int nsep = nc - 1;
  const std::vector<int>& cl = G.cls[l];
  int per_axis = nsep;
  for (int a = 1; a < G.dim; ++a) per_axis *= nc;
  fronts.assign((size_t)per_axis * G.dim, HostFront{});
  for (int g : alive) {
    int x[3];
    G.coords(g, x);
    int non = 0, axis = -1;
    for (int a = 0; a < G.dim; ++a)
      if (cl[x[a]] < 0) { ++non; axis = a; }
    if (non != 1) continue;
    const int ord = -cl[x[axis]] - 1;
    int other = 0;
    for (int a = G.dim - 1; a >= 0; --a)
      if (a != axis) other = other * nc + cl[x[a]];
    const int f = axis * per_axis + ord + nsep * other;
    HostFront& F = fronts[f];
    if (F.c.empty()) {
      F.axis = axis;
      int iv[3] = {0, 0, 0};
      for (int a = 0; a < G.dim; ++a) iv[a] = (a == axis) ? ord : cl[x[a]];
      F.P1 = lin_index(iv, G.dim, nc);
      iv[axis] = ord + 1;
      F.P2 = lin_index(iv, G.dim, nc);
    }
    F.c.push_back(g);
  }
  // drop empty fronts
  std::vector<HostFront> kept;
  kept.reserve(fronts.size());
  for (auto& F : fronts)
    if (!F.c.empty()) kept.push_back(std::move(F));
  fronts.swap(kept);
  if ((int64_t)mark.size() < G.N) mark.assign(G.N, -1);
  for (size_t f = 0; f < fronts.size(); ++f) {
    HostFront& F = fronts[f];
    for (int g : F.c) mark[g] = (int)f;
    const std::vector<int>& b1 = cells[F.P1].B;
    const std::vector<int>& b2 = cells[F.P2].B;
    std::vector<int> c1(F.c.size(), -1), c2(F.c.size(), -1);
    std::vector<int> n1, n2;
    size_t i = 0, j = 0, ci = 0;
    while (i < b1.size() || j < b2.size()) {
      int g;
      int p1 = -1, p2 = -1;
      if (j >= b2.size() || (i < b1.size() && b1[i] < b2[j])) { g = b1[i]; p1 = (int)i++; }
      else if (i >= b1.size() || b2[j] < b1[i]) { g = b2[j]; p2 = (int)j++; }
      else { g = b1[i]; p1 = (int)i++; p2 = (int)j++; }
      if (mark[g] == (int)f) {
        c1[ci] = p1;
        c2[ci] = p2;
        ++ci;
      } else {
        F.N.push_back(g);
        n1.push_back(p1);
        n2.push_back(p2);
      }
    }
    F.pos1 = c1;
    F.pos1.insert(F.pos1.end(), n1.begin(), n1.end());
    F.pos2 = c2;
    F.pos2.insert(F.pos2.end(), n2.begin(), n2.end());
    for (int g : F.c) mark[g] = -1;
  }
}

}  // namespace hif
