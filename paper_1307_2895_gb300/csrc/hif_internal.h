// Internal types shared by the host driver and the kernels.
//
// Storage model (unassembled multifrontal form of the active matrix A_l):
//   A_l restricted to the separators is the sum, over the cells of the
//   previous level, of one dense "update matrix" per cell over the cell's
//   boundary DOFs (Lemma 2.1: B_qq of that cell).  Original stencil entries
//   between separator DOFs are given to exactly one leaf cell (the lowest
//   linear index among the cells whose closure holds both DOFs), so the sum
//   is A_l exactly.  A front (2D edge / 3D face interior) lies on the boundary
//   of exactly two cells P1 < P2; its skeletonized block B_ss is written back
//   to P1's update matrix and P2's copy is zeroed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hif {

constexpr int kMaxChild = 8;   // 2^dim children per cell

// One cell (level l) or the root (level L, nB == 0).
// Offsets are element offsets into the level's pools.
struct CellDesc {
  int nI, nB;          // interior (eliminated) and boundary (c^N) sizes
  int64_t ids;         // int pool: ids_I[nI] then ids_B[nB] (global DOF ids, ascending)
  int64_t F;           // work pool: F_II[nI*nI] | F_BI[nB*nI] | F_BB[nB*nB]   (row-major)
  int64_t fac;         // factor pool: Linv[nI*nI] | L[nI*nI] | G[nB*nI]      (row-major)
  int64_t cmap;        // int pool: (nI+nB) x kMaxChild positions in each child's B (-1 absent)
  int child[kMaxChild];// child cell index at the previous level (-1 absent)
  int cell_lin;        // linear cell index (x fastest) at this level
};

// One front (edge or face interior) at a fractional level l + 1/2.
struct FrontDesc {
  int nc, nN;          // |c| and |c^N|
  int P1, P2;          // adjacent cells (indices into the level's cell array)
  int64_t ids;         // int pool: ids_c[nc] | pos1[nc+nN] | pos2[nc+nN]  (c first, then N)
  int64_t work;        // work pool: M[nN*nc] (column-major) | A_cc[nc*nc] | 3 scratch nc*nc
  int64_t fac;         // factor pool: T[nc*nc] | Linv[nc*nc] | L[nc*nc] | G[nc*nc]
  int64_t out;         // int pool (outputs): k | perm[nc] | ids_sr[nc]
};

// Block of the factor as the apply sweeps see it.  Cell: p = I, q = B.
// Front: p = redundant set r, q = skeleton set s, with T (nq x np).
// All matrices row-major: Linv, L (np x np), G (nq x np), T (nq x np).
struct ApplyDesc {
  int np, nq;
  int64_t ids;         // int pool: ids_p[np] then ids_q[nq]
  int64_t Linv, L, G, T;   // factor pool offsets (T = -1 for cells)
};

// Process-wide count of kernel launches issued by the library.
void note_launches(long long n);

// Message returned by hif_last_error() on the calling thread.
void set_last_error(const char* msg);

struct GridInfo {
  int dim, n, m;       // m = n - 1 nodes per axis
  double inv_h2;
};

}  // namespace hif
