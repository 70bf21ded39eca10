// Host symbolic stage of HIF-DE in 3D with edge skeletonization
// (Section 4.5, Algorithm 4.2): the sparsity pattern of the active matrix
// A_l and the index sets of every level built from it.
//
// Pattern.  Two active DOFs are coupled when a live clique of two or more
// members holds both, or (with the implicit stencil) when they are 7-point
// stencil neighbours.  The elimination of a set p (Lemma 2.1) absorbs every
// clique touching p (each lies in p and its neighbours q = p^N) into one
// clique on q (B_qq is dense) and removes p; the skeletonization of a group
// c with skeleton s (Lemma 2.4) removes the redundant DOFs r = c \ s from
// every clique (their couplings outside c are dropped with the ID's
// residual) and adds a clique on s (the update of A_ss).  No coupling
// between two active DOFs is ever removed.
//
// Cliques have identities and ordered members, so that A_l can be held as a
// sum of dense matrices, one per live clique (the stencil's bonds and
// diagonal included, as cliques of two and one): eliminate returns the id of
// the clique that replaces the absorbed ones, skeletonize that of the new
// skeleton clique, and a clique that loses members keeps the others in
// their order.
//
// Index sets of level l (S = 2^l m, K = 2^(L-l) cells per axis; distances
// exact in doubled grid units; a DOF with two or more nearest centers joins
// no set):
//   * cells: Voronoi cells of the active DOFs about the cell centers
//     ((j - 1/2) S per axis, j = 1..K), then, cell by cell in ascending
//     linear index (x fastest) and DOF by DOF in ascending index, every DOF
//     coupled to a DOF that is at that moment in another cell leaves its
//     cell;
//   * faces (kind 1): Voronoi cells about the face centers (j S on the
//     normal axis, j = 1..K-1, (j - 1/2) S on the other two; the x-, y-,
//     z-normal faces are families 0, 1, 2);
//   * edges (kind 2): the same about the edge centers ((j - 1/2) S along the
//     edge, j S on the other two; edges along x, y, z are families 0, 1, 2).
// Which DOFs a group keeps comes from the numerical ID and is an input.
//
// One object serves one factorization; its calls share scratch state and
// must not run concurrently (cells and groups use the host thread pool
// internally).
#pragma once
#include <cstdint>
#include <vector>

namespace hif {

// Flat description of one batch of gathers (a launch's worth of blocks):
// target t's dense block, of side dim[t], is the sum over its contributions
// k in [start[t], start[t+1]) of the matrix of clique clique[k], whose
// member i lands on row and column map[map_start[k] + i] of the block.
struct GatherPlan {
  std::vector<int> dim, start, clique, map_start, map;
};

class Symbolic3x {
 public:
  // Grid of n intervals per axis, N = (n-1)^3 DOFs (x fastest); L = the
  // nearest integer to log2(n / leaf), at least 1; m = floor(n / 2^L).
  // implicit_stencil: the 7-point couplings belong to the pattern without
  // cliques (pattern-only use); otherwise every coupling comes from cliques
  // the caller adds.
  Symbolic3x(int n, int leaf, bool implicit_stencil = true);

  int levels() const { return L_; }
  int leaf_width() const { return m_; }
  int dofs() const { return N_; }
  bool is_active(int i) const { return active_[i] != 0; }
  // Active DOFs, ascending.
  const std::vector<int>& active();

  // Level l's cells after peeling, each ascending, in ascending linear cell
  // index (empty cells omitted).
  std::vector<std::vector<int>> cells(int l);
  // Face (kind 1) or edge (kind 2) groups of level l, each ascending, in
  // ascending (family, x index, y index, z index) order.
  std::vector<std::vector<int>> groups(int l, int kind);
  // c^N: active DOFs outside c coupled to a DOF of c, ascending.
  std::vector<int> neighbors(const std::vector<int>& c) const;

  // A clique on the given active DOFs, in the order given; returns its id.
  int add_clique(const std::vector<int>& members);
  // Ids of the live cliques with a member in c, ascending.
  std::vector<int> touching(const std::vector<int>& c) const;
  // Members of clique id in their order (empty once it is dead).
  const std::vector<int>& members(int id) const { return clique_[id]; }
  bool live(int id) const { return clique_live_[id] != 0; }

  // The gathers of a batch: for target t, the live cliques touching keys[t]
  // (ascending ids), each member placed at its position in order[t].
  // Returns false (out unspecified) when a member of such a clique is not in
  // order[t]: the block would not hold the clique.
  bool gather_plan(const std::vector<std::vector<int>>& keys, const std::vector<std::vector<int>>& order,
                   GatherPlan& out) const;

  // Lemma 2.1 on the active set p: the cliques touching p die and one clique
  // on q = p^N (ascending) replaces them.  Returns its id, or -1 (q empty).
  int eliminate(const std::vector<int>& p);
  // Lemma 2.4 on group c with skeleton s (a subset of c): r = c \ s leaves
  // every clique (a clique left empty dies); when r and s are both
  // non-empty a clique on s (in the order given) is added and its id
  // returned, else -1.  Returns -2, changing nothing, when c holds an
  // inactive DOF or s is not in c.
  int skeletonize(const std::vector<int>& c, const std::vector<int>& s);

 private:
  struct Key {
    int fam, i[3];
  };
  // Nearest center of the union of families (per family, a list of
  // positions per axis, doubled units); false on a tie.
  bool voronoi(int g, const std::vector<std::vector<int>>* fams, int nfam, Key& k) const;
  void remove(const std::vector<int>& dofs);

  int n_, m_, L_, N_;
  bool implicit_;
  std::vector<char> active_;
  std::vector<int> active_list_;
  bool active_dirty_ = false;
  std::vector<std::vector<int>> clique_;   // active members (compacted on removal)
  std::vector<char> clique_live_;
  std::vector<std::vector<int>> of_;       // cliques holding each DOF (may list dead ones)
  std::vector<int> mark_;                  // scratch: a DOF's current cell during the peel, or -1
  mutable std::vector<int> pos_;           // scratch: position of a DOF in a block's order, or -1
  mutable std::vector<int> seen_;
  mutable std::vector<int> clique_seen_;   // scratch stamps per clique
  mutable int stamp_ = 0;
};

}  // namespace hif
