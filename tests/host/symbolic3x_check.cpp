// Test harness (CPU, no CUDA): drives the host symbolic stage of HIF-DE in
// 3D with edge skeletonization (Symbolic3x) through every level with the
// skeletons that a factorization chose, and writes the index sets it builds,
// for tests/test_host_symbolic3x.py to compare with that factorization's.
//
// usage: symbolic3x_check n leaf edge_start skel.bin out.bin
// skel.bin (int32 stream), per level l: the face groups' skeletons
// (G, then per group: ns, s...), then, when l >= edge_start, the edge
// groups' skeletons in the same form.
// out.bin (int32 stream), per level: ncells, per cell: np, p..., nq, q...;
// nfaces, per face: nc, c..., nN, N... (c^N before any group of the level
// is skeletonized); when l >= edge_start, nedges, per edge: the same; at the
// end: nroot, root....  On a group-count mismatch or a
// rejected skeleton, what was built so far is written and the exit code is 4.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "symbolic3x.h"

using namespace hif;

static void put(std::vector<int32_t>& o, const std::vector<int>& v) {
  o.push_back((int32_t)v.size());
  o.insert(o.end(), v.begin(), v.end());
}

static int write_out(const char* path, const std::vector<int32_t>& o, int rc) {
  FILE* f = std::fopen(path, "wb");
  if (!f) return 3;
  std::fwrite(o.data(), 4, o.size(), f);
  std::fclose(f);
  return rc;
}

int main(int argc, char** argv) {
  if (argc < 6) return 2;
  const int n = std::atoi(argv[1]), leaf = std::atoi(argv[2]), edge_start = std::atoi(argv[3]);
  std::vector<int32_t> in;
  {
    FILE* f = std::fopen(argv[4], "rb");
    if (!f) return 3;
    int32_t v;
    while (std::fread(&v, 4, 1, f) == 1) in.push_back(v);
    std::fclose(f);
  }
  size_t k = 0;
  auto take = [&]() -> int { return k < in.size() ? in[k++] : -1; };
  Symbolic3x S(n, leaf);
  std::vector<int32_t> o;
  for (int l = 0; l < S.levels(); ++l) {
    const std::vector<std::vector<int>> cells = S.cells(l);
    o.push_back((int32_t)cells.size());
    for (const std::vector<int>& p : cells) {
      put(o, p);
      put(o, S.neighbors(p));
      S.eliminate(p);
    }
    for (int kind = 1; kind <= 2; ++kind) {
      if (kind == 2 && l < edge_start) break;
      const std::vector<std::vector<int>> g = S.groups(l, kind);
      o.push_back((int32_t)g.size());
      for (const std::vector<int>& c : g) {   // all IDs of a fractional level see the same A
        put(o, c);
        put(o, S.neighbors(c));
      }
      if (take() != (int)g.size()) return write_out(argv[5], o, 4);
      for (const std::vector<int>& c : g) {
        const int ns = take();
        if (ns < 0) return write_out(argv[5], o, 4);
        std::vector<int> s(ns);
        for (int& v : s) v = take();
        if (S.skeletonize(c, s) == -2) return write_out(argv[5], o, 4);
      }
    }
  }
  put(o, S.active());
  return write_out(argv[5], o, 0);
}
