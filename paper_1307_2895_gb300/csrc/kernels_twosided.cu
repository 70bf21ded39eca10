// The two-sided (unsymmetric) factorization, the generalization of the
// paper's Section 6: the operators R_p and S_p of Lemma 2.1 from A_pp = L U
// (LU without pivoting, L unit lower), and front skeletons from one ID of
// the stacked [A_{N,c}; A_{c,N}^T], whose T serves rows and columns.
//
// Factor of a block (p eliminated against q), as the sweeps read it:
//   Linv = L^-1, G = A_qp U^-1, L (unit lower)        up sweep, F's down sweep
//   Linv2 = U^-T, G2 = (L^-1 A_pq)^T, L2 = U^T          down sweep, F's up sweep
// so that the symmetric sweep kernels apply R_p^T (up) and S_p (down) with
// the second set in the place of the first.  B_qq = A_qq - G G2^T.
#include "hif_internal.h"
#include "blockops.cuh"
#include "front_common.cuh"
#include "kernels.h"

namespace hif {

// Lf = the unit lower factor of an in-place LU (n x n), Ut = U^T (lower).
template <typename T>
__device__ void split_lu(const T* A, int n, T* Lf, T* Ut) {
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    Lf[e] = (j < i) ? A[e] : (j == i ? T(1) : T(0));
    Ut[e] = (j <= i) ? A[(int64_t)j * n + i] : T(0);
  }
  __syncthreads();
}

// G2 (m x n, row-major) with G2[i][j] = sum_{t <= j} B[t][i] X[j][t]:
// (X B)^T for X = L^-1 (n x n lower) and B (n x m, row-major).
template <typename T>
__device__ void mul_linv_b_t(const T* B, int m, const T* X, int n, T* G2) {
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const T* x = X + (int64_t)j * n;
    T s = T(0);
    for (int t = 0; t <= j; ++t) s += B[(int64_t)t * m + i] * x[t];
    G2[e] = s;
  }
  __syncthreads();
}

// Interior elimination of one cell: F_II = L U, the two factor sets, and
// F_BB <- F_BB - F_BI F_II^-1 F_IB.
template <typename T>
__global__ void __launch_bounds__(256) k_cell_lu(const CellDesc* __restrict__ cells, const int* __restrict__ sel,
                                                 T* __restrict__ work, T* __restrict__ fac, int* status) {
  const CellDesc cd = cells[sel ? sel[blockIdx.x] : blockIdx.x];
  const int nI = cd.nI, nB = cd.nB;
  T* FII = work + cd.F;
  T* FBI = FII + (int64_t)nI * nI;
  T* FBB = FBI + (int64_t)nB * nI;
  T* X = FBB + (int64_t)nB * nB;           // cell_x_elems(nI) >= nI^2
  const T* FIB = work + cd.FIB;            // nI x nB, then 2 nI^2 scratch
  T* Lf = work + cd.FIB + (int64_t)nI * nB;
  T* Ut = Lf + (int64_t)nI * nI;
  T* Linv = fac + cd.fac;
  T* G = fac + cd.fac + cell_fac_G(nI);
  T* Lp = fac + cd.fac + cell_fac_L(nI, nB);
  T* Sg = fac + cd.fac + cell_fac_S(nI, nB);
  T* Linv2 = fac + cd.fac2;
  T* G2 = Linv2 + packed_size(nI);
  T* L2 = G2 + pad4((int64_t)nB * nI);
  blk_lu_nopivot(FII, nI, nI, status);
  split_lu(FII, nI, Lf, Ut);
  blk_tri_inverse(Lf, nI, nI, X, nI);      // L^-1
  blk_pack_lower(Lf, nI, Lp, nI);
  blk_pack_lower(X, nI, Linv, nI);
  blk_tri_inverse(Ut, nI, nI, FII, nI);    // (U^T)^-1 = U^-T, over the factored F_II
  blk_pack_lower(Ut, nI, L2, nI);
  blk_pack_lower(FII, nI, Linv2, nI);
  for (int i = threadIdx.x; i < nI; i += blockDim.x) Sg[i] = T(1);
  if (nB > 0) {
    blk_mul_linvT(FBI, nI, FII, nI, nB, nI, G, nI);   // G = F_BI U^-1
    mul_linv_b_t(FIB, nB, X, nI, G2);                  // G2 = (L^-1 F_IB)^T
    for (int64_t e = threadIdx.x; e < (int64_t)nB * nB; e += blockDim.x) {
      const int i = (int)(e / nB), j = (int)(e % nB);
      const T* gi = G + (int64_t)i * nI;
      const T* hj = G2 + (int64_t)j * nI;
      T s = T(0);
      for (int t = 0; t < nI; ++t) s += gi[t] * hj[t];
      FBB[e] -= s;
    }
  }
}

// One front: the ID of [A_{N,c}; A_{c,N}^T] (column-pivoted QR of Section
// 2.2), then Q_c^T A Q_c and the two-sided elimination of the redundant
// DOFs; B_ss written back to P1's update matrix (P2's copy zeroed).
// Work: M (2|N| x |c|, column-major) | A_cc | six |c|^2 scratch blocks.
template <typename T>
__global__ void __launch_bounds__(256) k_front_lu(const FrontDesc* __restrict__ fronts,
                                                  const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                                                  int* __restrict__ obuf, T* __restrict__ fwork, T* __restrict__ fac,
                                                  T* __restrict__ cwork, double eps, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FrontDesc fd = fronts[blockIdx.x];
  const int nc = fd.nc, nN = fd.nN, m2 = 2 * fd.nN;
  const int* idc = ipool + fd.ids;
  const int* pos1 = idc + nc;
  const int* pos2 = pos1 + nc + nN;
  int* out = obuf + fd.out;
  const CellDesc P1 = cells[fd.P1], P2 = cells[fd.P2];
  T* U1 = cwork + P1.F + (int64_t)P1.nI * P1.nI + (int64_t)P1.nB * P1.nI;
  T* U2 = cwork + P2.F + (int64_t)P2.nI * P2.nI + (int64_t)P2.nB * P2.nI;
  const int ld1 = P1.nB, ld2 = P2.nB;
  double* sq = reinterpret_cast<double*>(smem_raw);   // nc
  double* v = sq + nc;                                 // 2 nN
  int* perm = reinterpret_cast<int*>(v + m2);          // nc
  int* chosen = perm + nc;                             // nc

  const int64_t c2 = (int64_t)nc * nc;
  T* M = fwork + fd.work;
  T* Acc = M + (int64_t)m2 * nc;
  T* S1 = Acc + c2;
  T* S2 = S1 + c2;
  T* S3 = S2 + c2;
  T* S4 = S3 + c2;
  T* S5 = S4 + c2;
  T* S6 = S5 + c2;
  T* Linvp = fac + fd.fac;
  T* G = fac + fd.fac + front_fac_G(nc);
  T* Tm = fac + fd.fac + front_fac_T(nc);
  T* Lp = fac + fd.fac + front_fac_L(nc);
  T* Sg = fac + fd.fac + front_fac_S(nc);
  T* Linv2p = fac + fd.fac2;
  T* G2 = Linv2p + packed_size(nc);
  T* L2p = G2 + pad4(c2);

  for (int64_t e = threadIdx.x; e < (int64_t)m2 * nc; e += blockDim.x) {
    const int j = (int)(e / m2), i = (int)(e % m2);
    M[e] = (i < nN) ? front_entry<T>(U1, ld1, U2, ld2, pos1, pos2, nc + i, j)           // A_{N,c}
                    : front_entry<T>(U1, ld1, U2, ld2, pos1, pos2, j, nc + (i - nN));  // A_{c,N}^T
  }
  for (int64_t e = threadIdx.x; e < c2; e += blockDim.x) {
    const int i = (int)(e / nc), j = (int)(e % nc);
    Acc[e] = front_entry<T>(U1, ld1, U2, ld2, pos1, pos2, i, j);
  }
  __syncthreads();
  const int k = blk_pivoted_qr(M, m2, nc, eps, status, true, sq, v, perm, chosen);
  blk_id_T(M, m2, perm, k, nc, Tm);
  const int nR = nc - k;

  // ---- Q_c^T A Q_c: W = A_ss T (S1), B_sr (S2), W2 = T^T A_ss (S5), B_rs (S4), B_rr (S3)
  for (int64_t e = threadIdx.x; e < (int64_t)k * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    const T* arow = Acc + (int64_t)perm[i] * nc;
    T s = T(0);
    for (int t = 0; t < k; ++t) s += arow[perm[t]] * Tm[(int64_t)t * nR + j];
    S1[e] = s;
    S2[e] = arow[perm[k + j]] - s;
  }
  for (int64_t e = threadIdx.x; e < (int64_t)nR * k; e += blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    T s = T(0);
    for (int t = 0; t < k; ++t) s += Tm[(int64_t)t * nR + i] * Acc[(int64_t)perm[t] * nc + perm[j]];
    S5[e] = s;
    S4[e] = Acc[(int64_t)perm[k + i] * nc + perm[j]] - s;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)nR * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    const int ri = perm[k + i], rj = perm[k + j];
    T b = Acc[(int64_t)ri * nc + rj];
    for (int t = 0; t < k; ++t) {
      const int st = perm[t];
      const T ti = Tm[(int64_t)t * nR + i], tj = Tm[(int64_t)t * nR + j];
      b -= ti * Acc[(int64_t)st * nc + rj] + Acc[(int64_t)ri * nc + st] * tj;
      b += ti * S1[(int64_t)t * nR + j];
    }
    S3[e] = b;
  }
  __syncthreads();
  if (nR > 0) {
    blk_lu_nopivot(S3, nR, nR, status);
    split_lu(S3, nR, S1, S5);                // W and W2 are no longer needed
    blk_tri_inverse(S1, nR, nR, S6, nR);     // L^-1
    blk_pack_lower(S1, nR, Lp, nR);
    blk_pack_lower(S6, nR, Linvp, nR);
    blk_tri_inverse(S5, nR, nR, S3, nR);     // U^-T
    blk_pack_lower(S5, nR, L2p, nR);
    blk_pack_lower(S3, nR, Linv2p, nR);
    for (int i = threadIdx.x; i < nR; i += blockDim.x) Sg[i] = T(1);
    if (k > 0) {
      blk_mul_linvT(S2, nR, S3, nR, k, nR, G, nR);   // G = B_sr U^-1
      mul_linv_b_t(S4, k, S6, nR, G2);              // G2 = (L^-1 B_rs)^T
      for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        const T* gi = G + (int64_t)i * nR;
        const T* hj = G2 + (int64_t)j * nR;
        T s = T(0);
        for (int t = 0; t < nR; ++t) s += gi[t] * hj[t];
        const int ci = perm[i], cj = perm[j];
        U1[(int64_t)pos1[ci] * ld1 + pos1[cj]] = Acc[(int64_t)ci * nc + cj] - s;
        if (pos2[ci] >= 0 && pos2[cj] >= 0) U2[(int64_t)pos2[ci] * ld2 + pos2[cj]] = T(0);
      }
    }
  }
  if (threadIdx.x == 0) out[0] = k;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    out[1 + t] = perm[t];
    out[1 + nc + t] = idc[perm[t]];
  }
}

template <typename T>
void launch_cell_lu(const CellDesc* cells, const int* sel, int ncells, T* work, T* fac, int* status,
                    cudaStream_t st) {
  if (ncells == 0) return;
  note_launches(1);
  k_cell_lu<T><<<ncells, 256, 0, st>>>(cells, sel, work, fac, status);
}

template <typename T>
void launch_front_lu(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                     T* fwork, T* fac, T* cwork, double eps, int* status, int max_nc, int max_nN, cudaStream_t st) {
  if (nfronts == 0) return;
  const int smem = (int)(sizeof(double) * ((size_t)max_nc + 2 * (size_t)max_nN) + sizeof(int) * 2 * (size_t)max_nc +
                         64);
  if (smem > 48 * 1024) raise_smem_limit(k_front_lu<T>);
  note_launches(1);
  k_front_lu<T><<<nfronts, 256, smem, st>>>(fronts, cells, ipool, obuf, fwork, fac, cwork, eps, status);
}

template void launch_cell_lu<double>(const CellDesc*, const int*, int, double*, double*, int*, cudaStream_t);
template void launch_cell_lu<float>(const CellDesc*, const int*, int, float*, float*, int*, cudaStream_t);
template void launch_front_lu<double>(const FrontDesc*, int, const CellDesc*, const int*, int*, double*, double*,
                                      double*, double, int*, int, int, cudaStream_t);
template void launch_front_lu<float>(const FrontDesc*, int, const CellDesc*, const int*, int*, float*, float*,
                                     float*, double, int*, int, int, cudaStream_t);

}  // namespace hif
