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
  int64_t F;           // work pool: F_II[nI*nI] | F_BI[nB*nI] | F_BB[nB*nB] | X[nI*nI] (row-major)
  int64_t fac;         // factor pool: Linv (packed) | G[nB*nI] | L (packed), see fac_layout
  int64_t cmap;        // int pool: (nI+nB) x kMaxChild positions in each child's B (-1 absent)
  int child[kMaxChild];// child cell index at the previous level (-1 absent)
  int cell_lin;        // linear cell index (x fastest) at this level
  // two-sided (unsymmetric) factorization only, -1 otherwise: work pool
  // offset of F_IB[nI*nB] (row-major) followed by 2 nI*nI scratch, and factor
  // pool offset of the second set Linv2 = U^-T (packed) | G2 = (L^-1 F_IB)^T
  // [nB*nI] | L2 = U^T (packed), see cell_fac2_size
  int64_t FIB = -1;
  int64_t fac2 = -1;
};

// One front (edge or face interior) at a fractional level l + 1/2.
struct FrontDesc {
  int nc, nN;          // |c| and |c^N|
  int P1, P2;          // adjacent cells (indices into the level's cell array)
  int64_t ids;         // int pool: ids_c[nc] | pos1[nc+nN] | pos2[nc+nN] (c first, then N) | ids_N[nN]
  int64_t work;        // work pool: M[nN*nc] (column-major) | A_cc[nc*nc] | 3 scratch nc*nc
  int64_t fac;         // factor pool (capacity for nc): Linv (packed) | G | T | L (packed)
  int64_t out;         // output buffer: k | perm[nc] | ids_sr[nc]
  int64_t fac2 = -1;   // two-sided: factor pool offset of Linv2 | G2 | L2 (capacity nc), else -1
};

// A dense elimination problem for the tiled kernels (Lemma 2.1 on
// [F_II F_BI^T; F_BI F_BB]): a large cell, or the redundant block of a large
// front after its ID (F_II = B_rr, F_BI = B_sr, F_BB = A_ss, Lemma 2.4).
// Offsets of the row-major blocks into the work pool (F_II: nI x nI, F_BI:
// nB x nI, F_BB: nB x nB, X: cell_x_elems(nI) scratch) and of the outputs
// into the factor pool (Linv and L packed by rows, G = F_BI L^-T: nB x nI).
struct TDesc {
  int nI, nB;
  int64_t FII, FBI, FBB, X;
  int64_t Linv, G, Lp, S;   // S: the diagonal block's signs (all +1 on this path)
};

// Block of the factor as the apply sweeps see it.  Cell: p = I, q = B.
// Front: p = redundant set r, q = skeleton set s, with T (nq x np); or, for
// a front skeletonized by the SVD (Section 4.4), p = the dropped directions
// and q = the kept ones in the slots of the front's DOFs (q first), with the
// rotation V ((nq + np) x (nq + np), row-major, rows by slot, columns by
// direction) in the place of T: x_c <- V^T x_c before the elimination of
// the up sweep, x_c <- V x_c after that of the down sweep.
// Linv and L are lower triangular, packed by rows (entry (i, t), t <= i, at
// i (i + 1) / 2 + t); G and T are row-major nq x np.  Every region starts on
// a 16-byte boundary (sizes rounded up to 4 elements).
// A_pp = L D L^T with D = diag(S) (+1 / -1, Section 5's LDL^T of an
// indefinite diagonal block; all +1 when A_pp is SPD); L^-1 is stored, G is
// A_qp L^-T D (so that x_q -= G y with y = L^-1 x_p), and the up sweep stores
// D y as the block's p values.
struct ApplyDesc {
  int np, nq;
  int64_t ids;         // int pool: ids_p[np] then ids_q[nq]
  int64_t Linv, L, G, T;   // factor pool offsets (T = -1 for cells)
  int64_t S;           // factor pool offset of the signs (np values)
  int64_t cslot;       // cells: row of x_q's first contribution in the level's
                       // contribution buffer (the deterministic scatter)
  int64_t V = -1;      // SVD fronts: factor pool offset of V (-1: none)
  // two-sided (unsymmetric) blocks, A_pp = L U (L unit lower): Linv = L^-1,
  // G = A_qp U^-1 and L (unit lower) as above; the down sweep and the
  // forward operator read Linv2 = U^-T, G2 = (L^-1 A_pq)^T (nq x np) and
  // L2 = U^T (packed lower) instead of Linv, G and L (-1: the symmetric
  // block, where they coincide)
  int64_t Linv2 = -1, G2 = -1, L2 = -1;
};

// Gaussian stream of the randomized ID (Section 4.3) at one fractional level
// l: front c's sketch matrix is Phi[r][j] = normal(key_c, r * nglob + j) for
// sketch row r and global DOF id j of a row of A_{N,c}, with key_c the
// splitmix64 output number level_base + c_0 + 1 of the stream seeded with
// `seed` (level_base = l * nglob, c_0 = the front's smallest DOF id, nglob =
// N) and normal(key, e) the Box-Muller cosine branch, in FP64, of the
// uniforms (top 53 bits) of outputs 2e + 1 and 2e + 2 of the stream seeded
// with key.  Indexed by DOF ids, so Phi A_{N,c} does not depend on the order
// of N or on rows that are structurally zero.  power: power iterations on
// the sketch, Y = Phi A (A^T A)^power.
struct SketchStream {
  uint64_t seed, level_base, nglob;
  int power;
};

// Rank-prediction MLP: kFeat input features per front, hidden width kHid.
constexpr int kFeat = 10;
constexpr int kHid = 64;
constexpr int kMlpParams = kHid * kFeat + kHid + kHid * kHid + kHid + kHid + 1;

// Process-wide count of kernel launches issued by the library.
void note_launches(long long n);

// Message returned by hif_last_error() on the calling thread.
void set_last_error(const char* msg);

// Factor-pool sizes (elements, rounded up to 4 so every region is 16-byte aligned).
__host__ __device__ inline int64_t pad4(int64_t x) { return (x + 3) & ~int64_t(3); }
__host__ __device__ inline int64_t packed_size(int64_t n) { return pad4(n * (n + 1) / 2); }
// cell: Linv | G | L | S
__host__ __device__ inline int64_t cell_fac_G(int nI) { return packed_size(nI); }
__host__ __device__ inline int64_t cell_fac_L(int nI, int nB) { return packed_size(nI) + pad4((int64_t)nB * nI); }
__host__ __device__ inline int64_t cell_fac_S(int nI, int nB) { return 2 * packed_size(nI) + pad4((int64_t)nB * nI); }
__host__ __device__ inline int64_t cell_fac_size(int nI, int nB) {
  return 2 * packed_size(nI) + pad4((int64_t)nB * nI) + pad4(nI);
}
// Largest grid of the reducing vector kernels (8 blocks of 256 threads per
// SM of a 152-SM GB300: enough loads in flight to stream HBM); the solver's
// partial-sum buffer holds 4 values per block and right-hand side.
constexpr int kVecBlocksMax = 1216;

// Tile edge of the multi-block elimination of large cells, and the size of a
// cell's X region of the work pool: room for Linv in the single-block kernel,
// or for the diagonal-tile inverses plus the original diagonal in the tiled one.
constexpr int kTile = 64;
// Smallest front of the multi-block skeletonization: its work layout gives the
// elimination scratch |c|^2 elements, which covers cell_x_elems(|c|) from
// |c| = 105 on.
constexpr int kBigFrontMin = 128;
__host__ __device__ inline int64_t cell_x_elems(int nI) {
  const int64_t t = (int64_t)((nI + kTile - 1) / kTile) * kTile * kTile + nI;
  const int64_t s = (int64_t)nI * nI;
  return pad4(s > t ? s : t);
}
// front with capacity nc: Linv | G | T | L | S
__host__ __device__ inline int64_t front_fac_G(int nc) { return packed_size(nc); }
__host__ __device__ inline int64_t front_fac_T(int nc) { return packed_size(nc) + pad4((int64_t)nc * nc); }
__host__ __device__ inline int64_t front_fac_L(int nc) { return packed_size(nc) + 2 * pad4((int64_t)nc * nc); }
__host__ __device__ inline int64_t front_fac_S(int nc) { return 2 * packed_size(nc) + 2 * pad4((int64_t)nc * nc); }
__host__ __device__ inline int64_t front_fac_size(int nc) {
  return 2 * packed_size(nc) + 2 * pad4((int64_t)nc * nc) + pad4(nc);
}

// Two-sided factorization: the second factor set of a cell or front
// (Linv2 packed | G2 | L2 packed) and a cell's extra work (F_IB, 2 scratch).
__host__ __device__ inline int64_t cell_fac2_size(int nI, int nB) {
  return 2 * packed_size(nI) + pad4((int64_t)nB * nI);
}
__host__ __device__ inline int64_t cell_work2_size(int nI, int nB) {
  return (int64_t)nI * nB + 2 * (int64_t)nI * nI;
}
__host__ __device__ inline int64_t front_fac2_size(int nc) { return 2 * packed_size(nc) + pad4((int64_t)nc * nc); }

struct GridInfo {
  int dim, n, m;       // m = n - 1 nodes per axis
  double inv_h2;
};

}  // namespace hif
