// Factorization kernels: frontal assembly, interior elimination (Lemma 2.1)
// and front skeletonization (Lemma 2.2 ID + Lemma 2.4).  One thread block
// per cell or front; every block of one level goes in one launch.
#include <algorithm>

#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"
#include "front_common.cuh"

namespace hif {

// ---------------------------------------------------------------------------
// Stencil entries (Section 3.1 / 3.2) and the leaf frontal matrices
// ---------------------------------------------------------------------------

struct LeafGeom {
  GridInfo g;
  const double* a_stag;
  const double* bnode;
  const int* cls;      // cls[x], x = 0..n: interval index (>= 0) or -(ordinal+1) on a separator
  int ncell;           // leaf cells per axis
  double conv[3];      // beta_e / 2h of a convection term beta . grad u (zero: none)
};

__device__ __forceinline__ void dof_coords(int gid, int m, int dim, int x[3]) {
  x[0] = gid % m + 1;
  x[1] = (gid / m) % m + 1;
  x[2] = (dim == 3) ? gid / (m * m) + 1 : 1;
}

// a at the bond between node jlo and jlo + e_axis (jlo[axis] in 0..n-1).
__device__ __forceinline__ double bond(const LeafGeom& L, int axis, const int j[3]) {
  const int n = L.g.n, m = L.g.m;
  if (L.g.dim == 2) {
    if (axis == 0) return L.a_stag[(int64_t)(j[1] - 1) * n + j[0]];
    return L.a_stag[(int64_t)n * m + (int64_t)j[1] * m + (j[0] - 1)];
  }
  const int64_t blk = (int64_t)n * m * m;
  if (axis == 0) return L.a_stag[((int64_t)(j[2] - 1) * m + (j[1] - 1)) * n + j[0]];
  if (axis == 1) return L.a_stag[blk + ((int64_t)(j[2] - 1) * n + j[1]) * m + (j[0] - 1)];
  return L.a_stag[2 * blk + ((int64_t)j[2] * m + (j[1] - 1)) * m + (j[0] - 1)];
}

// Does the cell with interval coordinates civ own the entry between nodes xa
// and xb?  Owner = lowest linear index among cells whose closure holds both,
// i.e. per axis the smallest interval common to both nodes.
__device__ __forceinline__ bool owns(const LeafGeom& L, const int civ[3], const int xa[3], const int xb[3]) {
  for (int a = 0; a < L.g.dim; ++a) {
    const int ca = L.cls[xa[a]], cb = L.cls[xb[a]];
    const int alo = ca >= 0 ? ca : -ca - 1, ahi = ca >= 0 ? ca : -ca;
    const int blo = cb >= 0 ? cb : -cb - 1, bhi = cb >= 0 ? cb : -cb;
    const int lo = alo > blo ? alo : blo, hi = ahi < bhi ? ahi : bhi;
    if (lo > hi || lo != civ[a]) return false;
  }
  return true;
}

template <typename T>
__global__ void k_leaf_assemble(const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                                T* __restrict__ work, LeafGeom L) {
  const CellDesc cd = cells[blockIdx.x];
  const int nI = cd.nI, nB = cd.nB, nF = nI + nB, dim = L.g.dim, m = L.g.m;
  const int* ids = ipool + cd.ids;
  T* FII = work + cd.F;
  T* FBI = FII + (int64_t)nI * nI;
  T* FBB = FBI + (int64_t)nB * nI;
  int civ[3];
  {
    int t = cd.cell_lin;
    for (int a = 0; a < 3; ++a) { civ[a] = t % L.ncell; t /= L.ncell; }
  }
  T* FIB = cd.FIB >= 0 ? work + cd.FIB : nullptr;   // two-sided only: F_IB stored too
  for (int64_t e = threadIdx.x; e < (int64_t)nF * nF; e += blockDim.x) {
    const int a = (int)(e / nF), b = (int)(e % nF);
    if (a < nI && b >= nI && !FIB) continue;   // F_IB: the transpose of F_BI, not stored
    const int ga = ids[a], gb = ids[b];
    int xa[3], xb[3];
    dof_coords(ga, m, dim, xa);
    dof_coords(gb, m, dim, xb);
    const bool inner = (a < nI) || (b < nI);
    double v = 0.0;
    if (ga == gb) {
      if (inner || owns(L, civ, xa, xa)) {
        v = L.bnode[ga];
        for (int ax = 0; ax < dim; ++ax) {
          int j[3] = {xa[0], xa[1], xa[2]};
          double s = bond(L, ax, j);          // upper bond (j + e/2)
          j[ax] -= 1;
          s += bond(L, ax, j);                // lower bond (j - e/2)
          v += s * L.g.inv_h2;
        }
      }
    } else {
      int ndiff = 0, axd = -1, d = 0;
      for (int ax = 0; ax < dim; ++ax)
        if (xa[ax] != xb[ax]) { ++ndiff; axd = ax; d = xb[ax] - xa[ax]; }
      if (ndiff == 1 && (d == 1 || d == -1) && (inner || owns(L, civ, xa, xb))) {
        int j[3] = {xa[0], xa[1], xa[2]};
        if (d < 0) j[axd] = xb[axd];
        v = -bond(L, axd, j) * L.g.inv_h2;
        if (L.conv[axd] != 0.0) v += d * L.conv[axd];   // (beta_e / 2h)(u_{j+e} - u_{j-e})
      }
    }
    T* dst;
    if (a < nI && b >= nI) dst = FIB + (int64_t)a * nB + (b - nI);
    else if (a < nI) dst = FII + (int64_t)a * nI + b;
    else if (b < nI) dst = FBI + (int64_t)(a - nI) * nI + b;
    else dst = FBB + (int64_t)(a - nI) * nB + (b - nI);
    *dst = (T)v;
  }
}

// ---------------------------------------------------------------------------
// Extend-add: F_P = sum over children of their update matrices (restricted
// to the surviving DOFs), in child-slot order.
// ---------------------------------------------------------------------------
template <typename TU, typename TF>
__global__ void k_extend_add(const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                             TF* __restrict__ work, const CellDesc* __restrict__ pcells,
                             const TU* __restrict__ pwork, int nchild) {
  const CellDesc cd = cells[blockIdx.x];
  const int64_t nF2 = (int64_t)(cd.nI + cd.nB) * (cd.nI + cd.nB);
  const int64_t e0 = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if ((int64_t)blockIdx.y * blockDim.x >= nF2) return;
  const int nI = cd.nI, nB = cd.nB, nF = nI + nB;
  const int* cmap = ipool + cd.cmap;
  TF* FII = work + cd.F;
  TF* FBI = FII + (int64_t)nI * nI;
  TF* FBB = FBI + (int64_t)nB * nI;
  __shared__ const TU* sU[kMaxChild];
  __shared__ int sld[kMaxChild];
  if (threadIdx.x < kMaxChild) {
    const int s = threadIdx.x;
    const int c = (s < nchild) ? cd.child[s] : -1;
    if (c >= 0) {
      const CellDesc pc = pcells[c];
      sU[s] = pwork + pc.F + (int64_t)pc.nI * pc.nI + (int64_t)pc.nB * pc.nI;
      sld[s] = pc.nB;
    } else {
      sU[s] = nullptr;
      sld[s] = 0;
    }
  }
  __syncthreads();
  TF* FIB = cd.FIB >= 0 ? work + cd.FIB : nullptr;   // two-sided only
  for (int64_t e = e0; e < nF2; e += (int64_t)gridDim.y * blockDim.x) {
    const int a = (int)(e / nF), b = (int)(e % nF);
    if (a < nI && b >= nI && !FIB) continue;
    const int* ca = cmap + (int64_t)a * kMaxChild;
    const int* cb = cmap + (int64_t)b * kMaxChild;
    TF s = TF(0);
    for (int c = 0; c < nchild; ++c) {
      const int pa = ca[c], pb = cb[c];
      if (pa >= 0 && pb >= 0) s += (TF)sU[c][(int64_t)pa * sld[c] + pb];
    }
    TF* dst;
    if (a < nI && b >= nI) dst = FIB + (int64_t)a * nB + (b - nI);
    else if (a < nI) dst = FII + (int64_t)a * nI + b;
    else if (b < nI) dst = FBI + (int64_t)(a - nI) * nI + b;
    else dst = FBB + (int64_t)(a - nI) * nB + (b - nI);
    *dst = s;
  }
}

// ---------------------------------------------------------------------------
// Interior elimination (Lemma 2.1): F_II = L L^T, Linv = L^{-1},
// G = F_BI L^{-T}, U = F_BB - G G^T (in place: U becomes the cell's update).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_cell_factor(const CellDesc* __restrict__ cells, const int* __restrict__ sel,
                              T* __restrict__ work, T* __restrict__ fac, int* status, int smem_elems, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const CellDesc cd = cells[sel ? sel[blockIdx.x] : blockIdx.x];
  const int nI = cd.nI, nB = cd.nB;
  T* FII = work + cd.F;
  T* FBI = FII + (int64_t)nI * nI;
  T* FBB = FBI + (int64_t)nB * nI;
  T* Xg = FBB + (int64_t)nB * nB;           // global room for Linv when smem is short
  T* Linv = fac + cd.fac;
  T* G = fac + cd.fac + cell_fac_G(nI);
  T* Lp = fac + cd.fac + cell_fac_L(nI, nB);
  T* Sg = fac + cd.fac + cell_fac_S(nI, nB);   // signs of D (LDL^T of an indefinite F_II)
  const int64_t n2 = (int64_t)nI * nI;
  T* A = FII;
  T* X = Xg;
  T* W = G;                                  // W = F_BI L^-T, in shared memory when it fits
  if (2 * n2 + (int64_t)nB * nI <= smem_elems) {
    A = sm;
    X = sm + n2;
    W = sm + 2 * n2;
  } else if (2 * n2 <= smem_elems) {
    A = sm;
    X = sm + n2;
  } else if (n2 <= smem_elems) {
    A = sm;
  }
  if (A != FII) blk_copy(FII, nI, A, nI, nI, nI);
  const bool neg = blk_cholesky(A, nI, nI, status, tau, (const T*)nullptr, Sg);
  blk_tri_inverse(A, nI, nI, X, nI);
  blk_pack_lower(A, nI, Lp, nI);
  blk_pack_lower(X, nI, Linv, nI);
  if (nB > 0) {
    blk_mul_linvT(FBI, nI, X, nI, nB, nI, W, nI);          // W = F_BI L^-T
    blk_syrk_sub(FBB, nB, W, nI, nB, nI, neg ? Sg : (const T*)nullptr);   // F_BB -= W D W^T
    if (neg) blk_scale_cols(W, nI, nB, nI, Sg);           // the stored G is W D
    if (W != G) blk_copy(W, nI, G, nI, nB, nI);
  }
}

// ---------------------------------------------------------------------------
// Front skeletonization: ID of A_{N,c} (column-pivoted Householder QR,
// Lemma 2.2 and Section 2.2) then Lemma 2.4 and the elimination of the
// redundant DOFs.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_front(const FrontDesc* __restrict__ fronts, const CellDesc* __restrict__ cells,
                        const int* __restrict__ ipool, int* __restrict__ obuf, T* __restrict__ fwork,
                        T* __restrict__ fac, T* __restrict__ cwork, double eps, int* status, T tau,
                        const int* __restrict__ sketch, SketchStream ss, const int* __restrict__ sel) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fi = sel ? sel[blockIdx.x] : (int)blockIdx.x;
  const FrontDesc fd = fronts[fi];
  const int nc = fd.nc, nN = fd.nN;
  const int* idc = ipool + fd.ids;
  const int* pos1 = idc + nc;
  const int* pos2 = pos1 + nc + nN;
  int* out = obuf + fd.out;
  const CellDesc P1 = cells[fd.P1], P2 = cells[fd.P2];
  T* U1 = cwork + P1.F + (int64_t)P1.nI * P1.nI + (int64_t)P1.nB * P1.nI;
  T* U2 = cwork + P2.F + (int64_t)P2.nI * P2.nI + (int64_t)P2.nB * P2.nI;
  const int ld1 = P1.nB, ld2 = P2.nB;

  double* sq = reinterpret_cast<double*>(smem_raw);          // nc
  double* v = sq + nc;                                        // nN
  int* perm = reinterpret_cast<int*>(v + nN);                 // nc
  int* chosen = perm + nc;                                    // nc
  __shared__ double s_e2[32], s_m2[32];

  T* M = fwork + fd.work;                 // nN x nc, column-major
  T* Acc = M + (int64_t)nN * nc;          // nc x nc
  T* S1 = Acc + (int64_t)nc * nc;
  T* S2 = S1 + (int64_t)nc * nc;
  T* S3 = S2 + (int64_t)nc * nc;
  T* PH = S3 + (int64_t)nc * nc;          // sketch matrix (ell x nN), ell < nc

  // ---- assemble A_{N,c} and A_cc
  for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) {
    const int j = (int)(e / nN), i = (int)(e % nN);
    M[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, nc + i, j);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {
    const int i = (int)(e / nc), j = (int)(e % nc);
    Acc[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, i, j);
  }
  __syncthreads();

  T* Linvp = fac + fd.fac;                 // packed nR x nR
  T* G = fac + fd.fac + front_fac_G(nc);   // k x nR
  T* Tm = fac + fd.fac + front_fac_T(nc);  // k x nR
  T* Lp = fac + fd.fac + front_fac_L(nc);  // packed nR x nR

  // ---- ID: from a Gaussian sketch Y = Phi A_{N,c} (Section 4.3) when a
  // sketch size is given: the skeletons of the pivoted QR of Y (rank rule at
  // kSketchRankTol * eps), T by least squares on A_{N,c}, accepted only if
  // every column of A_r - A_s T has norm <= eps max_j ||A_j||; otherwise (or
  // without a sketch) the pivoted QR of A_{N,c} itself.
  const int ell = sketch ? sketch[fi] : 0;
  int k = -1;
  if (ell > 0 && ell < nc && ell < nN) {
    const uint64_t key0 = sketch_key(ss, idc[0]);
    const int* idN = pos2 + nc + nN;       // global ids of the rows of A_{N,c}
    for (int64_t e = threadIdx.x; e < (int64_t)ell * nN; e += blockDim.x) {
      const int r = (int)(e / nN), i = (int)(e % nN);
      PH[e] = (T)sketch_normal(key0, (uint64_t)r * ss.nglob + (uint64_t)idN[i]);
    }
    __syncthreads();
    T* Y = S3;                             // ell x nc, column-major (ld ell)
    for (int64_t e = threadIdx.x; e < (int64_t)ell * nc; e += blockDim.x) {
      const int j = (int)(e / ell), r = (int)(e % ell);
      const T* ph = PH + (int64_t)r * nN;
      const T* mc = M + (int64_t)j * nN;
      T a = T(0);
      for (int i = 0; i < nN; ++i) a += ph[i] * mc[i];
      Y[e] = a;
    }
    __syncthreads();
    // power iterations Y <- (Y M^T) M, Z = Y M^T in PH (ell x nN, row-major)
    for (int g = 0; g < ss.power; ++g) {
      for (int64_t e = threadIdx.x; e < (int64_t)ell * nN; e += blockDim.x) {
        const int r = (int)(e / nN), i = (int)(e % nN);
        T a = T(0);
        for (int j = 0; j < nc; ++j) a += Y[(int64_t)j * ell + r] * M[(int64_t)j * nN + i];
        PH[e] = a;
      }
      __syncthreads();
      for (int64_t e = threadIdx.x; e < (int64_t)ell * nc; e += blockDim.x) {
        const int j = (int)(e / ell), r = (int)(e % ell);
        const T* ph = PH + (int64_t)r * nN;
        const T* mc = M + (int64_t)j * nN;
        T a = T(0);
        for (int i = 0; i < nN; ++i) a += ph[i] * mc[i];
        Y[e] = a;
      }
      __syncthreads();
    }
    int ks = blk_pivoted_qr(Y, ell, nc, sketch_rank_tol(eps, ss.power), status, false, sq, v, perm, chosen);
    bool ok = false;
    if (ks < ell) {
      // accept when every residual column |M_r - M_s T|_j <= eps max_j |M_j|
      // (the pivoted QR's stopping rule for the sketch's skeletons), T by
      // least squares on a copy of M in PH (free once Y is formed)
      T* C = PH;
      for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) C[e] = M[e];
      __syncthreads();
      double e2 = blk_ls_id(C, nN, nc, perm, ks, chosen, v, Tm);
      if (e2 < 0.0) e2 = INFINITY;
      double m2 = 0.0;
      for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const T* mc = M + (int64_t)c * nN;
        double cs = 0.0;
        for (int i = 0; i < nN; ++i) cs += (double)mc[i] * (double)mc[i];
        m2 = fmax(m2, cs);
      }
      for (int o = 16; o > 0; o >>= 1) {
        e2 = fmax(e2, __shfl_xor_sync(0xffffffffu, e2, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
      }
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (lane == 0) { s_e2[warp] = e2; s_m2[warp] = m2; }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = fmax(a, s_e2[w]); b = fmax(b, s_m2[w]); }
        s_e2[0] = a;
        s_m2[0] = b;
      }
      __syncthreads();
      ok = s_e2[0] <= eps * eps * s_m2[0];
      __syncthreads();
    }
    if (ok) {
      k = ks;
      if (threadIdx.x == 0) atomicAdd(status + 2, 1);
    } else if (threadIdx.x == 0) {
      atomicAdd(status + 3, 1);
    }
  }
  if (k < 0) {
    k = blk_pivoted_qr(M, nN, nc, eps, status, true, sq, v, perm, chosen);
    blk_id_T(M, nN, perm, k, nc, Tm);
  }
  const int nR = nc - k;

  // ---- Lemma 2.4: W = A_ss T (S1), B_sr = A_sr - W (S2), B_rr (S3)
  for (int64_t e = threadIdx.x; e < (int64_t)k * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    const T* arow = Acc + (int64_t)perm[i] * nc;
    T s = T(0);
    for (int t = 0; t < k; ++t) s += arow[perm[t]] * Tm[(int64_t)t * nR + j];
    S1[e] = s;
    S2[e] = arow[perm[k + j]] - s;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)nR * (nR + 1) / 2; e += blockDim.x) {
    int i, j;
    tri_decode(e, i, j);                   // j <= i
    T x1 = T(0), x2 = T(0), y = T(0);
    for (int t = 0; t < k; ++t) {
      const T* at = Acc + (int64_t)perm[t] * nc;
      const T ti = Tm[(int64_t)t * nR + i], tj = Tm[(int64_t)t * nR + j];
      x1 += at[perm[k + i]] * tj;        // (A_sr^T T)_{ij}
      x2 += at[perm[k + j]] * ti;        // (A_sr^T T)_{ji}
      y += ti * S1[(int64_t)t * nR + j]; // (T^T A_ss T)_{ij}
    }
    const T b = Acc[(int64_t)perm[k + i] * nc + perm[k + j]] - x1 - x2 + y;
    S3[(int64_t)i * nR + j] = b;
    S3[(int64_t)j * nR + i] = b;
  }
  __syncthreads();
  if (nR > 0) {
    T* Sg = fac + fd.fac + front_fac_S(nc);   // signs of D (LDL^T of an indefinite B_rr)
    const bool neg = blk_cholesky(S3, nR, nR, status, tau, (const T*)nullptr, Sg);
    T* X = S1;                             // W is no longer needed
    blk_tri_inverse(S3, nR, nR, X, nR);
    blk_pack_lower(S3, nR, Lp, nR);
    blk_pack_lower(X, nR, Linvp, nR);
    if (k > 0) {
      blk_mul_linvT(S2, nR, X, nR, k, nR, G, nR);
      // B_ss = A_ss - G D G^T -> P1's update (skeleton block), zero in P2's
      for (int64_t e = threadIdx.x; e < (int64_t)k * (k + 1) / 2; e += blockDim.x) {
        int i, j;
        tri_decode(e, i, j);               // j <= i; B_ss is symmetric
        const T* gi = G + (int64_t)i * nR;
        const T* gj = G + (int64_t)j * nR;
        T s = T(0);
        if (neg)
          for (int t = 0; t < nR; ++t) s += (gi[t] * Sg[t]) * gj[t];
        else
          for (int t = 0; t < nR; ++t) s += gi[t] * gj[t];
        const int ci = perm[i], cj = perm[j];
        const T b = Acc[(int64_t)ci * nc + cj] - s;
        U1[(int64_t)pos1[ci] * ld1 + pos1[cj]] = b;
        U1[(int64_t)pos1[cj] * ld1 + pos1[ci]] = b;
        if (pos2[ci] >= 0 && pos2[cj] >= 0) {   // (no second cell in the assembled upper levels)
          U2[(int64_t)pos2[ci] * ld2 + pos2[cj]] = T(0);
          U2[(int64_t)pos2[cj] * ld2 + pos2[ci]] = T(0);
        }
      }
      __syncthreads();
      if (neg) blk_scale_cols(G, nR, k, nR, Sg);          // the stored G is B_sr L^-T D
    }
  }
  // ---- outputs
  if (threadIdx.x == 0) out[0] = k;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    out[1 + t] = perm[t];
    out[1 + nc + t] = idc[perm[t]];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_leaf_assemble(const CellDesc* cells, int ncells, const int* ipool, T* work,
                          GridInfo g, const double* a_stag, const double* bnode, const int* cls,
                          int ncell_axis, const double* beta, cudaStream_t st) {
  LeafGeom L{g, a_stag, bnode, cls, ncell_axis, {0.0, 0.0, 0.0}};
  for (int a = 0; a < g.dim && beta; ++a) L.conv[a] = beta[a] * g.n / 2.0;   // 1 / 2h = n / 2
  note_launches(1);
  k_leaf_assemble<T><<<ncells, 256, 0, st>>>(cells, ipool, work, L);
}

template <typename TU, typename TF>
void launch_extend_add(const CellDesc* cells, int ncells, const int* ipool, TF* work,
                       const CellDesc* pcells, const TU* pwork, int nchild, int max_nF, cudaStream_t st) {
  if (ncells == 0) return;
  // one block per cell for the small cells; large cells spread over up to
  // 4096 blocks of 256 threads (one 256-entry chunk per block and pass)
  const int64_t f2 = (int64_t)max_nF * max_nF;
  int chunks = (int)std::min<int64_t>((f2 + 256 * 16 - 1) / (256 * 16), 4096);
  if (chunks < 1) chunks = 1;
  note_launches(1);
  k_extend_add<TU, TF><<<dim3(ncells, chunks), 256, 0, st>>>(cells, ipool, work, pcells, pwork, nchild);
}

template <typename T>
void launch_cell_factor(const CellDesc* cells, const int* sel, int ncells, T* work, T* fac, int* status,
                        int max_nI, int max_nB, double tau, cudaStream_t st) {
  if (ncells == 0) return;
  const int cap_bytes = 200 * 1024;
  // L, L^-1 and W = F_BI L^-T in shared memory when they fit (the Schur
  // update then reads W's rows from shared memory), else L and L^-1, else L.
  // W only when it is large: the many small leaf cells run faster with more
  // blocks resident per SM than with W's rows in shared memory.
  const bool w_smem = (int64_t)max_nB * max_nI * (int64_t)sizeof(T) > 16 * 1024;
  int64_t need = (2LL * max_nI * max_nI + (w_smem ? (int64_t)max_nB * max_nI : 0)) * (int64_t)sizeof(T);
  if (need > cap_bytes) need = 2LL * max_nI * max_nI * (int64_t)sizeof(T);
  if (need > cap_bytes) need = (int64_t)max_nI * max_nI * (int64_t)sizeof(T);
  if (need > cap_bytes) need = 0;
  const int smem = (int)need;
  if (smem > 48 * 1024)
    raise_smem_limit(k_cell_factor<T>);
  note_launches(1);
  k_cell_factor<T><<<ncells, 256, smem, st>>>(cells, sel, work, fac, status, smem / (int)sizeof(T), (T)tau);
}

template <typename T>
void launch_front(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                  T* fwork,
                  T* fac, T* cwork, double eps, int* status, int max_nc, int max_nN, double tau,
                  const int* sketch, SketchStream ss, const int* sel, cudaStream_t st) {
  if (nfronts == 0) return;
  const int smem = (int)(sizeof(double) * (max_nc + max_nN) + sizeof(int) * 2 * max_nc + 64);
  if (smem > 48 * 1024)
    raise_smem_limit(k_front<T>);
  note_launches(1);
  k_front<T><<<nfronts, 256, smem, st>>>(fronts, cells, ipool, obuf, fwork, fac, cwork, eps, status, (T)tau,
                                         sketch, ss, sel);
}

template void launch_leaf_assemble<double>(const CellDesc*, int, const int*, double*, GridInfo,
                                           const double*, const double*, const int*, int, const double*,
                                           cudaStream_t);
template void launch_leaf_assemble<float>(const CellDesc*, int, const int*, float*, GridInfo,
                                          const double*, const double*, const int*, int, const double*,
                                          cudaStream_t);
template void launch_extend_add<double, double>(const CellDesc*, int, const int*, double*,
                                                const CellDesc*, const double*, int, int, cudaStream_t);
template void launch_extend_add<float, float>(const CellDesc*, int, const int*, float*,
                                              const CellDesc*, const float*, int, int, cudaStream_t);
template void launch_extend_add<float, double>(const CellDesc*, int, const int*, double*,
                                               const CellDesc*, const float*, int, int, cudaStream_t);
template void launch_cell_factor<double>(const CellDesc*, const int*, int, double*, double*, int*, int, int,
                                         double, cudaStream_t);
template void launch_cell_factor<float>(const CellDesc*, const int*, int, float*, float*, int*, int, int, double,
                                        cudaStream_t);
template void launch_front<double>(const FrontDesc*, int, const CellDesc*, const int*, int*, double*, double*,
                                   double*, double, int*, int, int, double, const int*, SketchStream, const int*,
                                   cudaStream_t);
template void launch_front<float>(const FrontDesc*, int, const CellDesc*, const int*, int*, float*, float*,
                                  float*, double, int*, int, int, double, const int*, SketchStream, const int*,
                                  cudaStream_t);

// ---------------------------------------------------------------------------
// Features of each front for the rank predictor: level, log2 |c|, log2 |N|,
// log10 eps, and min / max / mean / std / spread of log10 a over the stencil
// couplings of the front's DOFs, and the dimension.
// ---------------------------------------------------------------------------
__global__ void k_front_features(const FrontDesc* __restrict__ fronts, const int* __restrict__ ipool,
                                 const double* __restrict__ W, int dim, int n, int level, double eps,
                                 float* __restrict__ feats) {
  const FrontDesc fd = fronts[blockIdx.x];
  const int* idc = ipool + fd.ids;
  const int ns = 2 * dim + 1;
  const double h2 = 1.0 / ((double)n * (double)n);
  double mn = 1e300, mx = -1e300, sm = 0.0, s2 = 0.0, cnt = 0.0;
  for (int e = threadIdx.x; e < fd.nc * 2 * dim; e += blockDim.x) {
    const int i = e / (2 * dim), kk = e % (2 * dim);
    const double w = W[(int64_t)idc[i] * ns + 1 + kk];
    if (w < 0.0) {
      const double la = log10(-w * h2);
      mn = fmin(mn, la);
      mx = fmax(mx, la);
      sm += la;
      s2 += la * la;
      cnt += 1.0;
    }
  }
  __shared__ double r[5][32];
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sm += __shfl_xor_sync(0xffffffffu, sm, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) { r[0][warp] = mn; r[1][warp] = mx; r[2][warp] = sm; r[3][warp] = s2; r[4][warp] = cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      mn = fmin(mn, r[0][w]); mx = fmax(mx, r[1][w]); sm += r[2][w]; s2 += r[3][w]; cnt += r[4][w];
    }
    mn = r[0][0] < mn ? r[0][0] : mn;
    float* f = feats + (int64_t)blockIdx.x * kFeat;
    const double mean = cnt > 0 ? sm / cnt : 0.0;
    const double var = cnt > 0 ? fmax(s2 / cnt - mean * mean, 0.0) : 0.0;
    if (cnt == 0) { mn = 0.0; mx = 0.0; }
    f[0] = (float)level;
    f[1] = (float)log2((double)fd.nc);
    f[2] = (float)log2((double)(fd.nN > 0 ? fd.nN : 1));
    f[3] = (float)log10(eps);
    f[4] = (float)mn;
    f[5] = (float)mx;
    f[6] = (float)mean;
    f[7] = (float)sqrt(var);
    f[8] = (float)(mx - mn);
    f[9] = (float)dim;
  }
}

// Sketch rows per front: learned (mode 2) k_hat = ceil(exp(pred) - 1), or the
// model-free guess k_hat = ceil(|c| / 2) (mode 1); ell = k_hat + oversample,
// 0 (pivoted QR directly) when ell would not be smaller than the block.
__global__ void k_sketch_sizes(const FrontDesc* __restrict__ fronts, int nf, const float* __restrict__ pred,
                               int mode, int oversample, int* __restrict__ sketch) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const FrontDesc fd = fronts[f];
  int kh;
  if (mode == 2 && pred) {
    const float p = fminf(fmaxf(pred[f], 0.f), 12.f);
    kh = (int)ceilf(expm1f(p));
  } else {
    kh = (fd.nc + 1) / 2;
  }
  kh = kh < 1 ? 1 : kh;
  int ell = kh + oversample;
  const int lim = fd.nc < fd.nN ? fd.nc : fd.nN;
  sketch[f] = ell < lim ? ell : 0;
}

void launch_front_features(const FrontDesc* fronts, int nfronts, const int* ipool, const double* stencil_w,
                           int dim, int n, int level, double eps, float* feats, cudaStream_t st) {
  if (nfronts == 0) return;
  note_launches(1);
  k_front_features<<<nfronts, 64, 0, st>>>(fronts, ipool, stencil_w, dim, n, level, eps, feats);
}

void launch_sketch_sizes(const FrontDesc* fronts, int nfronts, const float* pred, int mode, int oversample,
                         int* sketch, cudaStream_t st) {
  if (nfronts == 0) return;
  note_launches(1);
  k_sketch_sizes<<<(nfronts + 127) / 128, 128, 0, st>>>(fronts, nfronts, pred, mode, oversample, sketch);
}

}  // namespace hif
