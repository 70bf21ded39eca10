// Test shim (CPU, no CUDA): a C interface to the host symbolic stage of
// HIF-DE in 3D with edge skeletonization (Symbolic3x) for ctypes, so that
// tests/test_host_clique_plan.py can drive it step by step next to a model
// of the clique matrices.  A call that produces index lists leaves them in
// the handle; s3x_count / s3x_size / s3x_copy read them back.
#include <cstdint>
#include <vector>

#include "symbolic3x.h"

using hif::Symbolic3x;

namespace {
struct Handle {
  Symbolic3x S;
  std::vector<std::vector<int>> last;
  Handle(int n, int leaf, bool implicit) : S(n, leaf, implicit) {}
};
std::vector<int> ids(const int* p, int k) { return std::vector<int>(p, p + k); }
}  // namespace

extern "C" {

void* s3x_new(int n, int leaf, int implicit_stencil) { return new Handle(n, leaf, implicit_stencil != 0); }
void s3x_free(void* h) { delete static_cast<Handle*>(h); }
int s3x_levels(void* h) { return static_cast<Handle*>(h)->S.levels(); }

int s3x_count(void* h) { return (int)static_cast<Handle*>(h)->last.size(); }
int s3x_size(void* h, int i) { return (int)static_cast<Handle*>(h)->last[i].size(); }
void s3x_copy(void* h, int i, int* out) {
  const std::vector<int>& v = static_cast<Handle*>(h)->last[i];
  for (size_t k = 0; k < v.size(); ++k) out[k] = v[k];
}

int s3x_add_clique(void* h, const int* m, int k) { return static_cast<Handle*>(h)->S.add_clique(ids(m, k)); }
void s3x_cells(void* h, int l) {
  Handle* H = static_cast<Handle*>(h);
  H->last = H->S.cells(l);
}
void s3x_groups(void* h, int l, int kind) {
  Handle* H = static_cast<Handle*>(h);
  H->last = H->S.groups(l, kind);
}
void s3x_neighbors(void* h, const int* c, int k) {
  Handle* H = static_cast<Handle*>(h);
  H->last = {H->S.neighbors(ids(c, k))};
}
void s3x_touching(void* h, const int* c, int k) {
  Handle* H = static_cast<Handle*>(h);
  H->last = {H->S.touching(ids(c, k))};
}
void s3x_members(void* h, int id) {
  Handle* H = static_cast<Handle*>(h);
  H->last = {H->S.members(id)};
}
void s3x_active(void* h) {
  Handle* H = static_cast<Handle*>(h);
  H->last = {H->S.active()};
}
// Gather plan of nt targets given flattened key and order lists (offsets of
// nt + 1 entries); leaves dim, start, clique, map_start, map as the lists.
int s3x_gather_plan(void* h, int nt, const int* keys, const int* key_off, const int* order, const int* ord_off) {
  Handle* H = static_cast<Handle*>(h);
  std::vector<std::vector<int>> K(nt), O(nt);
  for (int t = 0; t < nt; ++t) {
    K[t].assign(keys + key_off[t], keys + key_off[t + 1]);
    O[t].assign(order + ord_off[t], order + ord_off[t + 1]);
  }
  hif::GatherPlan g;
  const bool ok = H->S.gather_plan(K, O, g);
  H->last = {g.dim, g.start, g.clique, g.map_start, g.map};
  return ok ? 1 : 0;
}
int s3x_eliminate(void* h, const int* p, int k) { return static_cast<Handle*>(h)->S.eliminate(ids(p, k)); }
int s3x_skeletonize(void* h, const int* c, int kc, const int* s, int ks) {
  return static_cast<Handle*>(h)->S.skeletonize(ids(c, kc), ids(s, ks));
}

}  // extern "C"
