// Front skeletonization by the SVD (Section 4.4): A_{N,c} = U Sigma V^T,
// Q_c = diag(V, I), the directions with sigma <= eps sigma_1 eliminated
// (Lemma 2.1 on B_p1p1 of B = V^T A_cc V) with their interactions dropped,
// the k kept directions left in the slots of the first k DOFs of c with
// interactions A_{N,c} V_2.
//
// Two launches per fractional level.  k_front_svd (one thread block per
// front) takes the SVD of A_{N,c} as the cells' update matrices hold it
// before the level, by one-sided Jacobi (Hestenes: pairs of columns of
// A_{N,c} rotated until orthogonal, V accumulating the rotations, pairs in
// round-robin order so that each warp rotates its own disjoint pairs), and
// forms the front's factor (V, Linv, L, G, the signs) and the kept block
// B~_p2p2.  k_svd_rotate (one thread block per cell that borders a
// skeletonized front) then applies every such front's rotation to the
// cell's update matrix, U <- Q^T U Q (columns, then rows: the rotations of
// different fronts act on disjoint slots and commute), and writes B~_p2p2
// (the first cell of the front) or zero (the second) on the kept slots.
// No rotation is made when nothing or everything is dropped (k = 0 or
// k = |c|): the factorization does not depend on the basis of a block that
// is wholly kept or wholly eliminated.
#include <algorithm>

#include "hif_internal.h"
#include "blockops.cuh"
#include "front_common.cuh"
#include "kernels.h"

namespace hif {

// Round-robin pairing of n2 (even) players: round r, match m; player 0 stays,
// the others turn by one place per round, so that every pair meets once in
// n2 - 1 rounds.
__device__ __forceinline__ int rr_player(int pos, int r, int n2) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (n2 - 1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_front_svd(const FrontDesc* __restrict__ fronts,
                                                   const CellDesc* __restrict__ cells,
                                                   const int* __restrict__ ipool, int* __restrict__ obuf,
                                                   T* __restrict__ fwork, T* __restrict__ fac,
                                                   const T* __restrict__ cwork, double eps, int* status, T tau,
                                                   int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FrontDesc fd = fronts[blockIdx.x];
  const int nc = fd.nc, nN = fd.nN;
  const int* idc = ipool + fd.ids;
  const int* pos1 = idc + nc;
  const int* pos2 = pos1 + nc + nN;
  int* out = obuf + fd.out;
  const CellDesc P1 = cells[fd.P1], P2 = cells[fd.P2];
  const T* U1 = cwork + P1.F + (int64_t)P1.nI * P1.nI + (int64_t)P1.nB * P1.nI;
  const T* U2 = cwork + P2.F + (int64_t)P2.nI * P2.nI + (int64_t)P2.nB * P2.nI;
  const int ld1 = P1.nB, ld2 = P2.nB;
  double* sig = reinterpret_cast<double*>(smem_raw);   // nc column norms
  int* order = reinterpret_cast<int*>(sig + nc);       // nc: columns by descending norm
  __shared__ int s_rot, s_k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;

  T* M = fwork + fd.work;                 // nN x nc, column-major
  T* Acc = M + (int64_t)nN * nc;          // nc x nc
  T* S1 = Acc + (int64_t)nc * nc;
  T* S2 = S1 + (int64_t)nc * nc;
  T* S3 = S2 + (int64_t)nc * nc;
  T* Linvp = fac + fd.fac;
  T* G = fac + fd.fac + front_fac_G(nc);
  T* Vf = fac + fd.fac + front_fac_T(nc);  // V, nc x nc row-major (the ID's T slot)
  T* Lp = fac + fd.fac + front_fac_L(nc);
  T* Sg = fac + fd.fac + front_fac_S(nc);

  for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) {
    const int j = (int)(e / nN), i = (int)(e % nN);
    M[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, nc + i, j);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {
    const int i = (int)(e / nc), j = (int)(e % nc);
    Acc[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, i, j);
    S1[e] = (i == j) ? T(1) : T(0);       // V = I
  }
  __syncthreads();

  // ---- one-sided Jacobi: rotate column pairs (a, b) of M while
  // |m_a . m_b| > tol |m_a| |m_b|; V <- V J for each rotation J.  Columns of
  // squared norm below 1e-31 ||M||_F^2 (rounding residue, below every rank
  // threshold) are left alone, or their pairs would turn forever.
  const double tol = 4.0 * 2.220446049250313e-16 * sqrt((double)(nN > 1 ? nN : 1));
  __shared__ double s_fro2;
  if (threadIdx.x == 0) s_fro2 = 0.0;
  __syncthreads();
  {
    double f = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) f += (double)M[e] * (double)M[e];
    f = warp_sum(f);
    if (lane == 0) atomicAdd(&s_fro2, f);
  }
  __syncthreads();
  const double floor2 = 1e-31 * s_fro2;
  const int n2 = nc + (nc & 1);
  for (int sweep = 0; sweep < max_sweeps && nN > 0; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < n2 - 1; ++r) {
      for (int m = warp; m < n2 / 2; m += nwarps) {
        int a = rr_player(m, r, n2), b = rr_player(n2 - 1 - m, r, n2);
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= nc) continue;                      // the idle player of an odd count
        T* ca = M + (int64_t)a * nN;
        T* cb = M + (int64_t)b * nN;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < nN; i += 32) {
          const double x = (double)ca[i], y = (double)cb[i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fmin(al, be) > floor2 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int i = lane; i < nN; i += 32) {
            const double x = (double)ca[i], y = (double)cb[i];
            ca[i] = (T)(c * x - s * y);
            cb[i] = (T)(s * x + c * y);
          }
          for (int i = lane; i < nc; i += 32) {
            T* vr = S1 + (int64_t)i * nc;
            const double x = (double)vr[a], y = (double)vr[b];
            vr[a] = (T)(c * x - s * y);
            vr[b] = (T)(s * x + c * y);
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }

  // ---- singular values (column norms), descending order (ties: position)
  for (int j = warp; j < nc; j += nwarps) {
    const T* cj = M + (int64_t)j * nN;
    double acc = 0.0;
    for (int i = lane; i < nN; i += 32) acc += (double)cj[i] * (double)cj[i];
    acc = warp_sum(acc);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < nc; ++i) r += (sig[i] > sig[j] || (sig[i] == sig[j] && i < j)) ? 1 : 0;
    order[r] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double smax = nc > 0 ? sig[order[0]] : 0.0;
    int k = 0;
    if (smax > 0.0) {
      for (int r = 0; r < nc; ++r) {
        const double ratio = sig[order[r]] / smax;
        if (ratio > eps) ++k;
        if (fabs(ratio - eps) <= 1e-8 * eps) atomicOr(status, 2);
      }
    }
    s_k = k < nN ? k : nN;                 // at most min(|N|, |c|) singular values exist
  }
  __syncthreads();
  const int k = s_k;
  const int nR = nc - k;
  const bool rotate = k > 0 && k < nc;

  // ---- V (sorted) to the factor; B = V^T A_cc V in S1 (or A_cc unrotated)
  if (rotate) {
    for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {
      const int t = (int)(e / nc), j = (int)(e % nc);
      Vf[e] = S1[(int64_t)t * nc + order[j]];
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {   // W = A_cc V
      const int i = (int)(e / nc), j = (int)(e % nc);
      const T* ar = Acc + (int64_t)i * nc;
      T s = T(0);
      for (int t = 0; t < nc; ++t) s += ar[t] * Vf[(int64_t)t * nc + j];
      S3[e] = s;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) {   // B = V^T W
      const int i = (int)(e / nc), j = (int)(e % nc);
      T s = T(0);
      for (int t = 0; t < nc; ++t) s += Vf[(int64_t)t * nc + i] * S3[(int64_t)t * nc + j];
      S1[e] = s;
    }
  } else {
    for (int64_t e = threadIdx.x; e < (int64_t)nc * nc; e += blockDim.x) S1[e] = Acc[e];
  }
  __syncthreads();

  // ---- Lemma 2.1 on p1 = [k, nc) against p2 = [0, k): B_p1p1 in S3,
  // B_p2p1 in Acc (k x nR), B_p2p2 read from S1 (ld nc)
  for (int64_t e = threadIdx.x; e < (int64_t)nR * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    S3[e] = S1[(int64_t)(k + i) * nc + k + j];
  }
  for (int64_t e = threadIdx.x; e < (int64_t)k * nR; e += blockDim.x) {
    const int i = (int)(e / nR), j = (int)(e % nR);
    Acc[e] = S1[(int64_t)i * nc + k + j];
  }
  __syncthreads();
  T* Bt = M;                               // B~_p2p2, k x k row-major (k^2 <= nN nc)
  if (nR > 0) {
    const bool neg = blk_cholesky(S3, nR, nR, status, tau, (const T*)nullptr, Sg);
    T* X = S2;
    blk_tri_inverse(S3, nR, nR, X, nR);
    blk_pack_lower(S3, nR, Lp, nR);
    blk_pack_lower(X, nR, Linvp, nR);
    if (k > 0) {
      blk_mul_linvT(Acc, nR, X, nR, k, nR, G, nR);     // G = B_p2p1 L^-T
      for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        const T* gi = G + (int64_t)i * nR;
        const T* gj = G + (int64_t)j * nR;
        T s = T(0);
        if (neg)
          for (int t = 0; t < nR; ++t) s += (gi[t] * Sg[t]) * gj[t];
        else
          for (int t = 0; t < nR; ++t) s += gi[t] * gj[t];
        Bt[e] = S1[(int64_t)i * nc + j] - s;
      }
      __syncthreads();
      if (neg) blk_scale_cols(G, nR, k, nR, Sg);       // the stored G is B_p2p1 L^-T D
    }
  }
  // ---- outputs: the kept slots first, in place
  if (threadIdx.x == 0) out[0] = k;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    out[1 + t] = t;
    out[1 + nc + t] = idc[t];
  }
}

// U <- Q^T U Q on the update matrix of one cell for each of its skeletonized
// fronts (list cptr / clist: (front, side) pairs, side 1 or 2 = the cell is
// the front's P1 or P2), then the kept block.  tile: rt x max_nc elements of
// dynamic shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_svd_rotate(const int* __restrict__ ccell, const int* __restrict__ cptr,
                                                    const int* __restrict__ clist,
                                                    const FrontDesc* __restrict__ fronts,
                                                    const CellDesc* __restrict__ cells,
                                                    const int* __restrict__ ipool, const int* __restrict__ obuf,
                                                    const T* __restrict__ fwork, const T* __restrict__ fac,
                                                    T* __restrict__ cwork, int rt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  const CellDesc P = cells[ccell[blockIdx.x]];
  const int nB = P.nB;
  T* U = cwork + P.F + (int64_t)P.nI * P.nI + (int64_t)P.nB * P.nI;
  for (int e = cptr[blockIdx.x]; e < cptr[blockIdx.x + 1]; ++e) {
    const int f = clist[2 * e], side = clist[2 * e + 1];
    const FrontDesc fd = fronts[f];
    const int nc = fd.nc;
    const int k = obuf[fd.out];
    if (k <= 0 || k >= nc) continue;      // no rotation
    const int* pos = ipool + fd.ids + nc + (side == 2 ? nc + fd.nN : 0);   // slots of c in this cell
    const T* V = fac + fd.fac + front_fac_T(nc);
    for (int r0 = 0; r0 < nB; r0 += rt) {   // columns: U[:, c] <- U[:, c] V
      const int rn = (nB - r0) < rt ? (nB - r0) : rt;
      for (int x = threadIdx.x; x < rn * nc; x += blockDim.x) {
        const int rr = x / nc, t = x % nc;
        tile[x] = U[(int64_t)(r0 + rr) * nB + pos[t]];
      }
      __syncthreads();
      for (int x = threadIdx.x; x < rn * nc; x += blockDim.x) {
        const int rr = x / nc, j = x % nc;
        const T* tr = tile + (int64_t)rr * nc;
        T s = T(0);
        for (int t = 0; t < nc; ++t) s += tr[t] * V[(int64_t)t * nc + j];
        U[(int64_t)(r0 + rr) * nB + pos[j]] = s;
      }
      __syncthreads();
    }
    for (int c0 = 0; c0 < nB; c0 += rt) {   // rows: U[c, :] <- V^T U[c, :]
      const int cn = (nB - c0) < rt ? (nB - c0) : rt;
      for (int x = threadIdx.x; x < cn * nc; x += blockDim.x) {
        const int t = x / cn, cc = x % cn;
        tile[x] = U[(int64_t)pos[t] * nB + c0 + cc];
      }
      __syncthreads();
      for (int x = threadIdx.x; x < cn * nc; x += blockDim.x) {
        const int j = x / cn, cc = x % cn;
        T s = T(0);
        for (int t = 0; t < nc; ++t) s += V[(int64_t)t * nc + j] * tile[(int64_t)t * cn + cc];
        U[(int64_t)pos[j] * nB + c0 + cc] = s;
      }
      __syncthreads();
    }
    const T* Bt = fwork + fd.work;
    for (int x = threadIdx.x; x < k * k; x += blockDim.x) {
      const int a = x / k, b = x % k;
      U[(int64_t)pos[a] * nB + pos[b]] = (side == 1) ? Bt[x] : T(0);
    }
    __syncthreads();
  }
}

constexpr int kJacobiMaxSweeps = 40;

template <typename T>
void launch_front_svd(const FrontDesc* fronts, int nfronts, const CellDesc* cells, const int* ipool, int* obuf,
                      T* fwork, T* fac, const T* cwork, double eps, int* status, int max_nc, double tau,
                      cudaStream_t st) {
  if (nfronts == 0) return;
  const int smem = (int)((sizeof(double) + sizeof(int)) * (size_t)max_nc + 64);
  if (smem > 48 * 1024) raise_smem_limit(k_front_svd<T>);
  note_launches(1);
  k_front_svd<T><<<nfronts, 256, smem, st>>>(fronts, cells, ipool, obuf, fwork, fac, cwork, eps, status, (T)tau,
                                             kJacobiMaxSweeps);
}

template <typename T>
void launch_svd_rotate(const int* ccell, const int* cptr, const int* clist, int ncells, const FrontDesc* fronts,
                       const CellDesc* cells, const int* ipool, const int* obuf, const T* fwork, const T* fac,
                       T* cwork, int max_nc, cudaStream_t st) {
  if (ncells == 0 || max_nc <= 0) return;
  int rt = (int)((96 * 1024) / ((size_t)max_nc * sizeof(T)));
  rt = std::max(1, std::min(rt, 64));
  const int smem = (int)((size_t)rt * max_nc * sizeof(T));
  if (smem > 48 * 1024) raise_smem_limit(k_svd_rotate<T>);
  note_launches(1);
  k_svd_rotate<T><<<ncells, 256, smem, st>>>(ccell, cptr, clist, fronts, cells, ipool, obuf, fwork, fac, cwork, rt);
}

template void launch_front_svd<double>(const FrontDesc*, int, const CellDesc*, const int*, int*, double*, double*,
                                       const double*, double, int*, int, double, cudaStream_t);
template void launch_front_svd<float>(const FrontDesc*, int, const CellDesc*, const int*, int*, float*, float*,
                                      const float*, double, int*, int, double, cudaStream_t);
template void launch_svd_rotate<double>(const int*, const int*, const int*, int, const FrontDesc*, const CellDesc*,
                                        const int*, const int*, const double*, const double*, double*, int,
                                        cudaStream_t);
template void launch_svd_rotate<float>(const int*, const int*, const int*, int, const FrontDesc*, const CellDesc*,
                                       const int*, const int*, const float*, const float*, float*, int,
                                       cudaStream_t);

}  // namespace hif
