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

#include "host_pool.h"

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

// Cells touched by the alive DOF g at level l: interior DOFs belong to one
// cell (I), separator DOFs to the 2^(#separator coordinates) adjacent cells (B).
struct CellSpan {
  int lo[3], hi[3];
  bool interior;
};

static inline CellSpan cell_span(const Geometry& G, const std::vector<int>& cl, int g) {
  int x[3];
  G.coords(g, x);
  CellSpan s;
  s.interior = true;
  for (int a = 0; a < 3; ++a) {
    if (a >= G.dim) { s.lo[a] = s.hi[a] = 0; continue; }
    const int c = cl[x[a]];
    if (c >= 0) { s.lo[a] = s.hi[a] = c; }
    else { s.lo[a] = -c - 1; s.hi[a] = -c; s.interior = false; }
  }
  return s;
}

void build_cells(const Geometry& G, int l, const std::vector<int>& alive, std::vector<HostCell>& cells) {
  const int nc = G.ncell[l];
  const int ncells = G.ncells(l);
  cells.resize(ncells);
  const std::vector<int>& cl = G.cls[l];
  // count, size every list once, then fill.  alive is ascending and cut into
  // contiguous ranges, one per task; a task writes its DOFs of a cell after
  // those of the tasks before it, so I and B come out ascending, exactly as
  // one pass over alive would make them.
  const int64_t na = (int64_t)alive.size();
  const int T = task_count(na, 4096);
  std::vector<std::vector<int>> nI(T, std::vector<int>(ncells, 0)), nB(T, std::vector<int>(ncells, 0));
  auto each = [&](int t, auto&& on_interior, auto&& on_boundary) {
    int64_t lo, hi;
    task_range(na, T, t, lo, hi);
    for (int64_t e = lo; e < hi; ++e) {
      const int g = alive[e];
      const CellSpan sp = cell_span(G, cl, g);
      if (sp.interior) { on_interior(lin_index(sp.lo, G.dim, nc), g); continue; }
      int iv[3];
      for (iv[2] = sp.lo[2]; iv[2] <= sp.hi[2]; ++iv[2])
        for (iv[1] = sp.lo[1]; iv[1] <= sp.hi[1]; ++iv[1])
          for (iv[0] = sp.lo[0]; iv[0] <= sp.hi[0]; ++iv[0]) on_boundary(lin_index(iv, G.dim, nc), g);
    }
  };
  parallel_tasks(T, [&](int t) {
    std::vector<int>& ci = nI[t];
    std::vector<int>& cb = nB[t];
    each(t, [&](int c, int) { ++ci[c]; }, [&](int c, int) { ++cb[c]; });
  });
  for (int c = 0; c < ncells; ++c) {   // counts -> each task's first position
    int si = 0, sb = 0;
    for (int t = 0; t < T; ++t) {
      const int a = nI[t][c], b = nB[t][c];
      nI[t][c] = si;
      nB[t][c] = sb;
      si += a;
      sb += b;
    }
    cells[c].I.resize(si);
    cells[c].B.resize(sb);
  }
  parallel_tasks(T, [&](int t) {
    std::vector<int>& ci = nI[t];
    std::vector<int>& cb = nB[t];
    each(t, [&](int c, int g) { cells[c].I[ci[c]++] = g; }, [&](int c, int g) { cells[c].B[cb[c]++] = g; });
  });
}

void build_child_map(const Geometry& G, int l, const HostCell& P, int cell_lin,
                     const std::vector<HostCell>& prev, std::vector<int>& out, int child[8]) {
  out.resize((P.I.size() + P.B.size()) * 8);
  build_child_map(G, l, P, cell_lin, prev, out.data(), child);
}

void build_child_map(const Geometry& G, int l, const HostCell& P, int cell_lin,
                     const std::vector<HostCell>& prev, int* out, int child[8]) {
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
  std::fill(out, out + (size_t)nF * 8, -1);
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
  const int nslot = per_axis * G.dim;
  // slot of an alive DOF with exactly one separator coordinate, else -1
  auto slot_of = [&](int g, int& axis, int& ord, int x[3]) {
    G.coords(g, x);
    int non = 0;
    axis = -1;
    for (int a = 0; a < G.dim; ++a)
      if (cl[x[a]] < 0) { ++non; axis = a; }
    if (non != 1) return -1;
    ord = -cl[x[axis]] - 1;
    int other = 0;
    for (int a = G.dim - 1; a >= 0; --a)
      if (a != axis) other = other * nc + cl[x[a]];
    return axis * per_axis + ord + nsep * other;
  };
  // count per slot; the non-empty slots become the fronts (in slot order).
  // As in build_cells: contiguous ranges of alive per task, positions
  // assigned in task order, so every F.c is ascending.
  const int64_t na = (int64_t)alive.size();
  const int T = task_count(na, 4096);
  std::vector<std::vector<int>> cnt(T, std::vector<int>(nslot, 0));
  parallel_tasks(T, [&](int t) {
    int64_t lo, hi;
    task_range(na, T, t, lo, hi);
    std::vector<int>& ct = cnt[t];
    for (int64_t e = lo; e < hi; ++e) {
      int axis, ord, x[3];
      const int f = slot_of(alive[e], axis, ord, x);
      if (f >= 0) ++ct[f];
    }
  });
  std::vector<int> fid(nslot, -1), fsize;
  int nf = 0;
  for (int f = 0; f < nslot; ++f) {   // counts -> each task's first position
    int tot = 0;
    for (int t = 0; t < T; ++t) {
      const int a = cnt[t][f];
      cnt[t][f] = tot;
      tot += a;
    }
    if (tot > 0) {
      fid[f] = nf++;
      fsize.push_back(tot);
    }
  }
  fronts.assign(nf, HostFront{});
  for (int f = 0; f < nf; ++f) fronts[f].c.resize(fsize[f]);
  parallel_tasks(T, [&](int t) {
    int64_t lo, hi;
    task_range(na, T, t, lo, hi);
    std::vector<int>& ct = cnt[t];
    for (int64_t e = lo; e < hi; ++e) {
      const int g = alive[e];
      int axis, ord, x[3];
      const int f = slot_of(g, axis, ord, x);
      if (f < 0) continue;
      HostFront& F = fronts[fid[f]];
      const int pos = ct[f]++;
      if (pos == 0) {    // the front's first DOF: its axis and the two cells
        F.axis = axis;
        int iv[3] = {0, 0, 0};
        for (int a = 0; a < G.dim; ++a) iv[a] = (a == axis) ? ord : cl[x[a]];
        F.P1 = lin_index(iv, G.dim, nc);
        iv[axis] = ord + 1;
        F.P2 = lin_index(iv, G.dim, nc);
      }
      F.c[pos] = g;
    }
  });
  if ((int64_t)mark.size() < G.N) mark.assign(G.N, -1);
  // neighbour lists: the fronts partition the DOFs, so each front marks and
  // unmarks its own entries of `mark`
  const int TF = task_count(nf, 64);
  parallel_tasks(TF, [&](int t) {
    int64_t f0, f1;
    task_range(nf, TF, t, f0, f1);
    for (int64_t f = f0; f < f1; ++f) {
      HostFront& F = fronts[f];
      for (int g : F.c) mark[g] = (int)f;
      const std::vector<int>& b1 = cells[F.P1].B;
      const std::vector<int>& b2 = cells[F.P2].B;
      const size_t ncf = F.c.size(), bound = b1.size() + b2.size();
      F.pos1.assign(ncf + bound, -1);
      F.pos2.assign(ncf + bound, -1);
      F.N.resize(bound);
      size_t i = 0, j = 0, ci = 0, ni = 0;
      while (i < b1.size() || j < b2.size()) {
        int g;
        int p1 = -1, p2 = -1;
        if (j >= b2.size() || (i < b1.size() && b1[i] < b2[j])) { g = b1[i]; p1 = (int)i++; }
        else if (i >= b1.size() || b2[j] < b1[i]) { g = b2[j]; p2 = (int)j++; }
        else { g = b1[i]; p1 = (int)i++; p2 = (int)j++; }
        if (mark[g] == (int)f) {            // c in ascending order, as F.c
          F.pos1[ci] = p1;
          F.pos2[ci] = p2;
          ++ci;
        } else {
          F.N[ni] = g;
          F.pos1[ncf + ni] = p1;
          F.pos2[ncf + ni] = p2;
          ++ni;
        }
      }
      F.N.resize(ni);
      F.pos1.resize(ncf + ni);
      F.pos2.resize(ncf + ni);
      for (int g : F.c) mark[g] = -1;
    }
  });
}

}  // namespace hif
