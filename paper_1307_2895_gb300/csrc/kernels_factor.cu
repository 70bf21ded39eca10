// Factorization kernels: frontal assembly, interior elimination (Lemma 2.1)
// and front skeletonization (Lemma 2.2 ID + Lemma 2.4).  One thread block
// per cell or front; every block of one level goes in one launch.
#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"

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
  for (int64_t e = threadIdx.x; e < (int64_t)nF * nF; e += blockDim.x) {
    const int a = (int)(e / nF), b = (int)(e % nF);
    if (a < nI && b >= nI) continue;            // F_IB is never stored
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
      }
    }
    T* dst;
    if (a < nI) dst = FII + (int64_t)a * nI + b;
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
  for (int64_t e = threadIdx.x; e < (int64_t)nF * nF; e += blockDim.x) {
    const int a = (int)(e / nF), b = (int)(e % nF);
    if (a < nI && b >= nI) continue;
    const int* ca = cmap + (int64_t)a * kMaxChild;
    const int* cb = cmap + (int64_t)b * kMaxChild;
    TF s = TF(0);
    for (int c = 0; c < nchild; ++c) {
      const int pa = ca[c], pb = cb[c];
      if (pa >= 0 && pb >= 0) s += (TF)sU[c][(int64_t)pa * sld[c] + pb];
    }
    TF* dst;
    if (a < nI) dst = FII + (int64_t)a * nI + b;
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
__global__ void k_cell_factor(const CellDesc* __restrict__ cells, T* __restrict__ work,
                              T* __restrict__ fac, int* status, int smem_elems, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const CellDesc cd = cells[blockIdx.x];
  const int nI = cd.nI, nB = cd.nB;
  T* FII = work + cd.F;
  T* FBI = FII + (int64_t)nI * nI;
  T* FBB = FBI + (int64_t)nB * nI;
  T* Xg = FBB + (int64_t)nB * nB;           // global room for Linv when smem is short
  T* Linv = fac + cd.fac;
  T* G = fac + cd.fac + cell_fac_G(nI);
  T* Lp = fac + cd.fac + cell_fac_L(nI, nB);
  const int64_t n2 = (int64_t)nI * nI;
  T* A = FII;
  T* X = Xg;
  if (2 * n2 <= smem_elems) {
    A = sm;
    X = sm + n2;
  } else if (n2 <= smem_elems) {
    A = sm;
  }
  if (A != FII) blk_copy(FII, nI, A, nI, nI, nI);
  blk_cholesky(A, nI, nI, status, tau);
  blk_tri_inverse(A, nI, nI, X, nI);
  blk_pack_lower(A, nI, Lp, nI);
  blk_pack_lower(X, nI, Linv, nI);
  if (nB > 0) {
    blk_mul_linvT(FBI, nI, X, nI, nB, nI, G, nI);
    blk_syrk_sub(FBB, nB, G, nI, nB, nI);
  }
}

// ---------------------------------------------------------------------------
// Front skeletonization: ID of A_{N,c} (column-pivoted Householder QR,
// Lemma 2.2 and Section 2.2) then Lemma 2.4 and the elimination of the
// redundant DOFs.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T front_entry(const T* U1, int ld1, const T* U2, int ld2,
                                         const int* pos1, const int* pos2, int x, int y) {
  T v = T(0);
  const int a1 = pos1[x], b1 = pos1[y];
  if (a1 >= 0 && b1 >= 0) v += U1[(int64_t)a1 * ld1 + b1];
  const int a2 = pos2[x], b2 = pos2[y];
  if (a2 >= 0 && b2 >= 0) v += U2[(int64_t)a2 * ld2 + b2];
  return v;
}

template <typename T>
__global__ void k_front(const FrontDesc* __restrict__ fronts, const CellDesc* __restrict__ cells,
                        const int* __restrict__ ipool, int* __restrict__ obuf, T* __restrict__ fwork,
                        T* __restrict__ fac,
                        T* __restrict__ cwork, double eps, int* status, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FrontDesc fd = fronts[blockIdx.x];
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
  __shared__ double s_mx, s_vv, s_alpha;
  __shared__ int s_piv, s_stop, s_k;

  T* M = fwork + fd.work;                 // nN x nc, column-major
  T* Acc = M + (int64_t)nN * nc;          // nc x nc
  T* S1 = Acc + (int64_t)nc * nc;
  T* S2 = S1 + (int64_t)nc * nc;
  T* S3 = S2 + (int64_t)nc * nc;

  // ---- assemble A_{N,c} and A_cc
  for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) {
    const int j = (int)(e / nN), i = (int)(e % nN);
    M[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, nc + i, j);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {
    const int i = (int)(e / nc), j = (int)(e % nc);
    Acc[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, i, j);
  }
  for (int j = threadIdx.x; j < nc; j += blockDim.x) chosen[j] = 0;
  if (threadIdx.x == 0) { s_k = 0; s_stop = 0; }
  __syncthreads();

  // ---- column-pivoted Householder QR with recomputed norms
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  double nu1sq = 0.0;
  const int kmax = nN < nc ? nN : nc;
  for (int i = 0; i < kmax; ++i) {
    for (int j = warp; j < nc; j += nwarps) {
      if (chosen[j]) continue;
      const T* col = M + (int64_t)j * nN;
      double acc = 0.0;
      for (int r = i + lane; r < nN; r += 32) { const double x = (double)col[r]; acc += x * x; }
      acc = warp_sum(acc);
      if (lane == 0) sq[j] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      double mx = -1.0;
      for (int j = lane; j < nc; j += 32) if (!chosen[j] && sq[j] > mx) mx = sq[j];
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int piv = 0x7fffffff;
      for (int j = lane; j < nc; j += 32)
        if (!chosen[j] && sq[j] >= (1.0 - 1e-10) * mx) { piv = j; break; }
      for (int o = 16; o > 0; o >>= 1) piv = min(piv, __shfl_xor_sync(0xffffffffu, piv, o));
      if (lane == 0) {
        if (i == 0) s_mx = mx; // nu1^2
        const double nu = (i == 0) ? mx : s_mx;
        const double ratio = (nu > 0.0) ? sqrt(mx / nu) : 0.0;
        if (fabs(ratio - eps) <= 1e-8 * eps) atomicOr(status, 2);
        int stop = (mx <= 0.0) || (i > 0 && mx <= eps * eps * nu);
        s_stop = stop;
        if (!stop) {
          s_piv = piv;
          const double x0 = (double)M[(int64_t)piv * nN + i];
          const double alpha = (x0 >= 0.0) ? -sqrt(mx) : sqrt(mx);
          // use the pivot's own squared norm for the reflector
          const double sp = sq[piv];
          const double a2 = (x0 >= 0.0) ? -sqrt(sp) : sqrt(sp);
          s_alpha = a2;
          s_vv = sp - x0 * x0 + (x0 - a2) * (x0 - a2);
          (void)alpha;
          perm[s_k] = piv;
          chosen[piv] = 1;
          s_k = s_k + 1;
        }
      }
    }
    __syncthreads();
    if (i == 0) nu1sq = s_mx;
    if (s_stop) break;
    const int piv = s_piv;
    const double alpha = s_alpha, vv = s_vv;
    T* pc = M + (int64_t)piv * nN;
    for (int r = i + threadIdx.x; r < nN; r += blockDim.x) v[r] = (double)pc[r] - (r == i ? alpha : 0.0);
    __syncthreads();
    if (vv > 0.0) {
      for (int j = warp; j < nc; j += nwarps) {
        if (chosen[j]) continue;
        T* col = M + (int64_t)j * nN;
        double s = 0.0;
        for (int r = i + lane; r < nN; r += 32) s += v[r] * (double)col[r];
        s = warp_sum(s);
        const double f = 2.0 * s / vv;
        for (int r = i + lane; r < nN; r += 32) col[r] = (T)((double)col[r] - f * v[r]);
      }
    }
    for (int r = i + threadIdx.x; r < nN; r += blockDim.x) pc[r] = (r == i) ? (T)alpha : T(0);
    __syncthreads();
  }
  (void)nu1sq;
  const int k = s_k;
  const int nR = nc - k;
  // redundant columns in ascending order after the skeletons
  if (threadIdx.x == 0) {
    int t = k;
    for (int j = 0; j < nc; ++j) if (!chosen[j]) perm[t++] = j;
  }
  __syncthreads();

  T* Linvp = fac + fd.fac;                 // packed nR x nR
  T* G = fac + fd.fac + front_fac_G(nc);   // k x nR
  T* Tm = fac + fd.fac + front_fac_T(nc);  // k x nR
  T* Lp = fac + fd.fac + front_fac_L(nc);  // packed nR x nR

  // ---- T = R11^{-1} R12 (back substitution, one thread per column)
  for (int c = threadIdx.x; c < nR; c += blockDim.x) {
    const T* r12 = M + (int64_t)perm[k + c] * nN;
    for (int t = k - 1; t >= 0; --t) {
      T s = r12[t];
      for (int u = t + 1; u < k; ++u) s -= M[(int64_t)perm[u] * nN + t] * Tm[(int64_t)u * nR + c];
      Tm[(int64_t)t * nR + c] = s / M[(int64_t)perm[t] * nN + t];
    }
  }
  __syncthreads();

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
  for (int64_t e = threadIdx.x; e < (int64_t)nR * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    if (j > i) continue;
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
    blk_cholesky(S3, nR, nR, status, tau);
    T* X = S1;                             // W is no longer needed
    blk_tri_inverse(S3, nR, nR, X, nR);
    blk_pack_lower(S3, nR, Lp, nR);
    blk_pack_lower(X, nR, Linvp, nR);
    if (k > 0) {
      blk_mul_linvT(S2, nR, X, nR, k, nR, G, nR);
      // B_ss = A_ss - G G^T -> P1's update (skeleton block), zero in P2's
      for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        const T* gi = G + (int64_t)i * nR;
        const T* gj = G + (int64_t)j * nR;
        T s = T(0);
        for (int t = 0; t < nR; ++t) s += gi[t] * gj[t];
        const int ci = perm[i], cj = perm[j];
        const T b = Acc[(int64_t)ci * nc + cj] - s;
        U1[(int64_t)pos1[ci] * ld1 + pos1[cj]] = b;
        U2[(int64_t)pos2[ci] * ld2 + pos2[cj]] = T(0);
      }
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
                          int ncell_axis, cudaStream_t st) {
  LeafGeom L{g, a_stag, bnode, cls, ncell_axis};
  note_launches(1);
  k_leaf_assemble<T><<<ncells, 256, 0, st>>>(cells, ipool, work, L);
}

template <typename TU, typename TF>
void launch_extend_add(const CellDesc* cells, int ncells, const int* ipool, TF* work,
                       const CellDesc* pcells, const TU* pwork, int nchild, cudaStream_t st) {
  note_launches(1);
  k_extend_add<TU, TF><<<ncells, 256, 0, st>>>(cells, ipool, work, pcells, pwork, nchild);
}

template <typename T>
void launch_cell_factor(const CellDesc* cells, int ncells, T* work, T* fac, int* status,
                        int max_nI, double tau, cudaStream_t st) {
  const int cap_bytes = 200 * 1024;
  int64_t need = 2LL * max_nI * max_nI * (int64_t)sizeof(T);
  if (need > cap_bytes) need = (int64_t)max_nI * max_nI * (int64_t)sizeof(T);
  if (need > cap_bytes) need = 0;
  const int smem = (int)need;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_cell_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  note_launches(1);
  k_cell_factor<T><<<ncells, 256, smem, st>>>(cells, work, fac, status, smem / (int)sizeof(T), (T)tau);
}

template <typename T>
void launch_front(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                  T* fwork,
                  T* fac, T* cwork, double eps, int* status, int max_nc, int max_nN, double tau,
                  cudaStream_t st) {
  const int smem = (int)(sizeof(double) * (max_nc + max_nN) + sizeof(int) * 2 * max_nc + 64);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_front<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  note_launches(1);
  k_front<T><<<nfronts, 256, smem, st>>>(fronts, cells, ipool, obuf, fwork, fac, cwork, eps, status, (T)tau);
}

template void launch_leaf_assemble<double>(const CellDesc*, int, const int*, double*, GridInfo,
                                           const double*, const double*, const int*, int, cudaStream_t);
template void launch_leaf_assemble<float>(const CellDesc*, int, const int*, float*, GridInfo,
                                          const double*, const double*, const int*, int, cudaStream_t);
template void launch_extend_add<double, double>(const CellDesc*, int, const int*, double*,
                                                const CellDesc*, const double*, int, cudaStream_t);
template void launch_extend_add<float, float>(const CellDesc*, int, const int*, float*,
                                              const CellDesc*, const float*, int, cudaStream_t);
template void launch_extend_add<float, double>(const CellDesc*, int, const int*, double*,
                                               const CellDesc*, const float*, int, cudaStream_t);
template void launch_cell_factor<double>(const CellDesc*, int, double*, double*, int*, int, double, cudaStream_t);
template void launch_cell_factor<float>(const CellDesc*, int, float*, float*, int*, int, double, cudaStream_t);
template void launch_front<double>(const FrontDesc*, int, const CellDesc*, const int*, int*, double*, double*,
                                   double*, double, int*, int, int, double, cudaStream_t);
template void launch_front<float>(const FrontDesc*, int, const CellDesc*, const int*, int*, float*, float*,
                                  float*, double, int*, int, int, double, cudaStream_t);

}  // namespace hif
