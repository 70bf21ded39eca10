// Test harness (CPU, no CUDA): runs the host tree builder (build_cells,
// build_fronts, build_child_map) on an alive set read from a file and writes
// the index lists, for tests/test_host_builder.py to check against their
// definitions.
//
// usage: builder_check dim n level alive.bin out.bin [prev_alive.bin]
// alive.bin: int32 count, then count ascending DOF ids (the active DOFs before
// the level's cells are eliminated).  out.bin (int32 stream):
//   ncells, then per cell: nI, I..., nB, B...
//   nfronts, then per front: axis, P1, P2, nc, c..., nN, N..., pos1[nc+nN], pos2[nc+nN]
// With prev_alive.bin (the level below's alive set), the child maps of every
// cell are appended: per cell: 8 child ids, then (nI + nB) * 8 positions.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "geometry.h"

using namespace hif;

static std::vector<int> read_ids(const char* path) {
  std::vector<int> v;
  FILE* f = std::fopen(path, "rb");
  if (!f) return v;
  int32_t n = 0;
  if (std::fread(&n, 4, 1, f) == 1 && n > 0) {
    v.resize(n);
    if (std::fread(v.data(), 4, n, f) != (size_t)n) v.clear();
  }
  std::fclose(f);
  return v;
}

static void put(std::vector<int32_t>& o, const std::vector<int>& v) {
  o.push_back((int32_t)v.size());
  o.insert(o.end(), v.begin(), v.end());
}

int main(int argc, char** argv) {
  if (argc < 6) return 2;
  const int dim = std::atoi(argv[1]), n = std::atoi(argv[2]), l = std::atoi(argv[3]);
  Geometry G;
  G.init(dim, n, 8);
  if (l < 0 || l >= G.L) return 3;
  const std::vector<int> alive = read_ids(argv[4]);
  std::vector<HostCell> cells;
  build_cells(G, l, alive, cells);
  std::vector<int> after;   // alive after the cells' interiors leave
  {
    std::vector<char> dead(G.N, 0);
    for (const HostCell& c : cells)
      for (int g : c.I) dead[g] = 1;
    for (int g : alive)
      if (!dead[g]) after.push_back(g);
  }
  std::vector<HostFront> fronts;
  std::vector<int> mark;
  build_fronts(G, l, after, cells, fronts, mark);
  std::vector<int32_t> o;
  o.push_back((int32_t)cells.size());
  for (const HostCell& c : cells) {
    put(o, c.I);
    put(o, c.B);
  }
  o.push_back((int32_t)fronts.size());
  for (const HostFront& F : fronts) {
    o.push_back(F.axis);
    o.push_back(F.P1);
    o.push_back(F.P2);
    put(o, F.c);
    put(o, F.N);
    o.insert(o.end(), F.pos1.begin(), F.pos1.end());
    o.insert(o.end(), F.pos2.begin(), F.pos2.end());
  }
  if (argc > 6 && l > 0) {   // child maps into the level below's boundaries
    const std::vector<int> prev_alive = read_ids(argv[6]);
    std::vector<HostCell> prev;
    build_cells(G, l - 1, prev_alive, prev);
    for (size_t i = 0; i < cells.size(); ++i) {
      std::vector<int> map;
      int child[8];
      build_child_map(G, l, cells[i], (int)i, prev, map, child);
      o.insert(o.end(), child, child + 8);
      o.insert(o.end(), map.begin(), map.end());
    }
  }
  FILE* f = std::fopen(argv[5], "wb");
  if (!f) return 4;
  std::fwrite(o.data(), 4, o.size(), f);
  std::fclose(f);
  return 0;
}
