// Skeletonization of large fronts (the ID of Section 2.2 / 4.3 and the
// elimination of Lemma 2.4) spread over many thread blocks per front.  The
// one-block kernel (k_front) runs every step of a front on one SM, which at
// the top levels of a 3D tree leaves the GPU nearly idle for seconds; here
// every dense product of the fronts of a level is one launch over 64 x 64
// tiles of all of them:
//
//   M = A_{N,c}, A_cc from the adjacent cells' update matrices (k_bf_assemble)
//   ID:  Y = Phi M (k_bf_sketch, Phi generated on the fly), pivoted QR of Y
//        and T from its R (k_bf_id), accepted when every column of
//        M_r - M_s T has norm <= eps max_j ||M_j|| (k_bf_colmax, k_bf_resid,
//        k_bf_check); otherwise, and in the
//        pivoted-QR mode, the pivoted QR of M itself (k_bf_id, one block)
//   B_sr = A_sr - A_ss T, B_rr = A_rr - A_sr^T T - T^T B_sr (k_bf_form_*)
//   L L^T = B_rr, G = B_sr L^-T, B_ss = A_ss - G G^T by the tiled
//   elimination of large cells (kernels_tiled.cu) on [B_rr; B_sr; A_ss]
//   B_ss into the first cell's update matrix, zeros into the second's
//   (k_bf_scatter).
//
// Work layout of a large front (from fd.work in the level's front pool):
//   M (nN x nc, column-major) | A_cc (nc x nc) | F: B_rr (nR x nR) | B_sr
//   (k x nR) | A_ss (k x k) (<= nc^2) | X (elimination scratch, <= nc^2) |
//   Y (the sketch, ell x nc column-major, <= nc^2).
#include <algorithm>
#include <vector>

#include "hif_internal.h"
#include "blockops.cuh"
#include "front_common.cuh"
#include "kernels.h"
#include "tile_mma.cuh"

namespace hif {

struct BfView {
  int nc, nN;
  int64_t M, Acc, F, X, Y;
};

__device__ __forceinline__ BfView bf_view(const FrontDesc& fd) {
  BfView v;
  v.nc = fd.nc;
  v.nN = fd.nN;
  v.M = fd.work;
  v.Acc = v.M + (int64_t)fd.nN * fd.nc;
  v.F = v.Acc + (int64_t)fd.nc * fd.nc;
  v.X = v.F + (int64_t)fd.nc * fd.nc;
  v.Y = v.X + (int64_t)fd.nc * fd.nc;
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_part[32];
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_part[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
  __syncthreads();
  return t;   // valid in thread 0
}

// ---- assembly: M and A_cc
template <typename T>
__global__ void k_bf_assemble(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                              const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                              const T* __restrict__ cwork, T* __restrict__ fwork) {
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int* idc = ipool + fd.ids;
  const int* pos1 = idc + nc;
  const int* pos2 = pos1 + nc + nN;
  const CellDesc P1 = cells[fd.P1], P2 = cells[fd.P2];
  const T* U1 = cwork + P1.F + (int64_t)P1.nI * P1.nI + (int64_t)P1.nB * P1.nI;
  const T* U2 = cwork + P2.F + (int64_t)P2.nI * P2.nI + (int64_t)P2.nB * P2.nI;
  const int ld1 = P1.nB, ld2 = P2.nB;
  T* M = fwork + v.M;
  T* Acc = fwork + v.Acc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nN * nc; e += stride) {
    const int j = (int)(e / nN), i = (int)(e % nN);
    M[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, nc + i, j);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nc * nc; e += stride) {
    const int i = (int)(e / nc), j = (int)(e % nc);
    Acc[e] = front_entry(U1, ld1, U2, ld2, pos1, pos2, i, j);
  }
}

// ---- largest squared column norm of M: one warp per column, block maxima
template <typename T>
__global__ void k_bf_colmax(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                            const T* __restrict__ fwork, double* __restrict__ m2part) {
  __shared__ double s_mx[8];
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + warp;
  double s = 0.0;
  if (c < fd.nc) {
    const T* col = fwork + v.M + (int64_t)c * fd.nN;
    for (int i = lane; i < fd.nN; i += 32) s += (double)col[i] * (double)col[i];
  }
  s = warp_sum(s);
  if (lane == 0) s_mx[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < 8; ++w) mx = fmax(mx, s_mx[w]);
    m2part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = mx;
  }
}

// ---- sketch: Y = Phi M (ell x nc), Phi from the front's stream (SketchStream)
template <typename T>
__global__ void __launch_bounds__(TT) k_bf_sketch(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                  const int* __restrict__ sketch, const int* __restrict__ ipool,
                                                  T* __restrict__ fwork, SketchStream ss) {
  __shared__ TileSmem<T> sm;
  const int f = big[blockIdx.y];
  const FrontDesc fd = fronts[f];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int ell = sketch ? sketch[f] : 0;
  if (ell <= 0 || ell >= nc || ell >= nN) return;
  const int tcn = (nc + TB - 1) / TB;
  if ((int)blockIdx.x >= ((ell + TB - 1) / TB) * tcn) return;
  const int r0 = (blockIdx.x / tcn) * TB, c0 = (blockIdx.x % tcn) * TB;
  const int* idc = ipool + fd.ids;
  const int* idN = idc + nc + 2 * (nc + nN);     // global ids of the rows of M
  const uint64_t key0 = sketch_key(ss, idc[0]);
  const T* M = fwork + v.M;
  T* Y = fwork + v.Y;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, true>(
      sm, acc, nN,
      [&](int r, int k) {
        return (r0 + r < ell) ? (T)sketch_normal(key0, (uint64_t)(r0 + r) * ss.nglob + (uint64_t)idN[k]) : T(0);
      },
      [&](int k, int c) { return (c0 + c < nc) ? M[(int64_t)(c0 + c) * nN + k] : T(0); });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < ell && c < nc) Y[(int64_t)c * ell + r] = acc[i][j];
    }
}

// ---- power iteration on the sketch: Z = Y M^T (ell x nN, row-major, in the
// spare region after Y), then Y = Z M (ell x nc, column-major)
template <typename T>
__global__ void __launch_bounds__(TT) k_bf_power_z(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                   const int* __restrict__ sketch, T* __restrict__ fwork) {
  __shared__ TileSmem<T> sm;
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int ell = sketch ? sketch[big[blockIdx.y]] : 0;
  if (ell <= 0 || ell >= nc || ell >= nN) return;
  const int tcn = (nN + TB - 1) / TB;
  if ((int)blockIdx.x >= ((ell + TB - 1) / TB) * tcn) return;
  const int r0 = (blockIdx.x / tcn) * TB, c0 = (blockIdx.x % tcn) * TB;
  const T* M = fwork + v.M;
  const T* Y = fwork + v.Y;
  T* Z = fwork + v.Y + (int64_t)nc * nc;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, false>(
      sm, acc, nc, [&](int r, int j) { return (r0 + r < ell) ? Y[(int64_t)j * ell + r0 + r] : T(0); },
      [&](int j, int i) { return (c0 + i < nN) ? M[(int64_t)j * nN + c0 + i] : T(0); });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < ell && c < nN) Z[(int64_t)r * nN + c] = acc[i][j];
    }
}

template <typename T>
__global__ void __launch_bounds__(TT) k_bf_power_y(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                   const int* __restrict__ sketch, T* __restrict__ fwork) {
  __shared__ TileSmem<T> sm;
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int ell = sketch ? sketch[big[blockIdx.y]] : 0;
  if (ell <= 0 || ell >= nc || ell >= nN) return;
  const int tcn = (nc + TB - 1) / TB;
  if ((int)blockIdx.x >= ((ell + TB - 1) / TB) * tcn) return;
  const int r0 = (blockIdx.x / tcn) * TB, c0 = (blockIdx.x % tcn) * TB;
  const T* M = fwork + v.M;
  const T* Z = fwork + v.Y + (int64_t)nc * nc;
  T* Y = fwork + v.Y;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, true>(
      sm, acc, nN, [&](int r, int i) { return (r0 + r < ell) ? Z[(int64_t)(r0 + r) * nN + i] : T(0); },
      [&](int i, int c) { return (c0 + c < nc) ? M[(int64_t)(c0 + c) * nN + i] : T(0); });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < ell && c < nc) Y[(int64_t)c * ell + r] = acc[i][j];
    }
}

// ---- the ID, one thread block per front.
// pass 0: fronts with a valid sketch size take the pivoted QR of Y (rank
// rule at kSketchRankTol * eps), then T by least squares on a copy of M
// (blk_ls_id, in the spare region after Y), accepted (state 0) when every
// residual column norm is at most eps times the largest column norm of M
// (m2part: the partial maxima of k_bf_colmax), else left in state 2 (also
// when the sketch saturated, k = ell); the other fronts take the pivoted QR
// of M (state 0), or are left in state 2 for the multi-block QR (defer_qr).
// pass 1: fronts in state 2 take the pivoted QR of M (state 0).  Writes T
// (k x nR) to the front's factor, and k | perm | ids (pivot order) to its
// output slot.
template <typename T>
__global__ void k_bf_id(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                        const int* __restrict__ sketch, const int* __restrict__ ipool, T* __restrict__ fwork,
                        T* __restrict__ fac, int* __restrict__ obuf, int* __restrict__ state, double eps,
                        int* status, int pass, int defer_qr, const double* __restrict__ m2part, int nm,
                        int power) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int f = big[blockIdx.x];
  const FrontDesc fd = fronts[f];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int ell = sketch ? sketch[f] : 0;
  const bool use_sketch = pass == 0 && ell > 0 && ell < nc && ell < nN;
  if (pass == 1 && state[blockIdx.x] != 2) return;
  if (!use_sketch && defer_qr) {                 // the pivoted QR of M goes to k_bf_qr_coop
    if (threadIdx.x == 0) state[blockIdx.x] = 2;
    return;
  }
  const int m = use_sketch ? ell : nN;
  double* sq = reinterpret_cast<double*>(smem_raw);            // nc
  double* vv = sq + nc;                                         // nN (m <= nN)
  int* perm = reinterpret_cast<int*>(vv + nN);                  // nc
  int* chosen = perm + nc;                                      // nc
  T* A = fwork + (use_sketch ? v.Y : v.M);
  T* Tm = fac + fd.fac + front_fac_T(nc);
  const int k = blk_pivoted_qr(A, m, nc, use_sketch ? sketch_rank_tol(eps, power) : eps, status, !use_sketch, sq,
                               vv, perm, chosen);
  if (use_sketch && k >= ell) {                                 // saturated: fall back
    if (threadIdx.x == 0) {
      state[blockIdx.x] = 2;
      atomicAdd(status + 3, 1);
    }
    return;
  }
  if (use_sketch) {
    T* C = fwork + v.Y + (int64_t)nc * nc;                      // spare: nN x nc
    const T* M = fwork + v.M;
    for (int64_t e = threadIdx.x; e < (int64_t)nN * nc; e += blockDim.x) C[e] = M[e];
    __syncthreads();
    const double e2 = blk_ls_id(C, nN, nc, perm, k, chosen, vv, Tm);
    double m2 = 0.0;
    for (int i = 0; i < nm; ++i) m2 = fmax(m2, m2part[(int64_t)blockIdx.x * nm + i]);
    if (!(e2 >= 0.0 && e2 <= eps * eps * m2)) {
      if (threadIdx.x == 0) {
        state[blockIdx.x] = 2;
        atomicAdd(status + 3, 1);
      }
      return;
    }
    if (threadIdx.x == 0) atomicAdd(status + 2, 1);
  } else {
    blk_id_T(A, m, perm, k, nc, Tm);
  }
  int* out = obuf + fd.out;
  const int* idc = ipool + fd.ids;
  if (threadIdx.x == 0) {
    out[0] = k;
    state[blockIdx.x] = 0;
  }
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    out[1 + t] = perm[t];
    out[1 + nc + t] = idc[perm[t]];
  }
}

// ---- Lemma 2.4 blocks in the elimination layout.  F_BI (k x nR) = B_sr =
// A_sr - A_ss T; F_BB (k x k) = A_ss.
template <typename T>
__global__ void __launch_bounds__(TT) k_bf_form_sr(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                   const int* __restrict__ obuf, T* __restrict__ fwork,
                                                   const T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc;
  const int* out = obuf + fd.out;
  const int k = out[0], nR = nc - k;
  const int* perm = out + 1;
  if (k == 0 || nR == 0) return;
  const int tcn = (nR + TB - 1) / TB;
  if ((int)blockIdx.x >= ((k + TB - 1) / TB) * tcn) return;
  const int i0 = (blockIdx.x / tcn) * TB, j0 = (blockIdx.x % tcn) * TB;
  const T* Acc = fwork + v.Acc;
  const T* Tm = fac + fd.fac + front_fac_T(nc);
  T* FBI = fwork + v.F + (int64_t)nR * nR;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, false>(
      sm, acc, k,
      [&](int r, int t) { return (i0 + r < k) ? Acc[(int64_t)perm[i0 + r] * nc + perm[t]] : T(0); },
      [&](int t, int c) { return (j0 + c < nR) ? Tm[(int64_t)t * nR + j0 + c] : T(0); });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
      if (r < k && c < nR) FBI[(int64_t)r * nR + c] = Acc[(int64_t)perm[r] * nc + perm[k + c]] - acc[i][j];
    }
}

template <typename T>
__global__ void k_bf_form_ss(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                             const int* __restrict__ obuf, T* __restrict__ fwork) {
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc;
  const int* out = obuf + fd.out;
  const int k = out[0], nR = nc - k;
  const int* perm = out + 1;
  if (nR == 0) return;
  const T* Acc = fwork + v.Acc;
  T* FBB = fwork + v.F + (int64_t)nR * nR + (int64_t)k * nR;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    FBB[e] = Acc[(int64_t)perm[i] * nc + perm[j]];
  }
}

// F_II (nR x nR) = B_rr = A_rr - A_sr^T T - T^T B_sr, lower tiles only (the
// elimination reads the lower triangle).
template <typename T>
__global__ void __launch_bounds__(TT) k_bf_form_rr(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                   const int* __restrict__ obuf, T* __restrict__ fwork,
                                                   const T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc;
  const int* out = obuf + fd.out;
  const int k = out[0], nR = nc - k;
  const int* perm = out + 1;
  const int P = (nR + TB - 1) / TB;
  const int64_t t = blockIdx.x;
  if (nR == 0 || t >= (int64_t)P * (P + 1) / 2) return;
  int a, b;
  tri_decode(t, a, b);
  const int i0 = a * TB, j0 = b * TB;
  const T* Acc = fwork + v.Acc;
  const T* Tm = fac + fd.fac + front_fac_T(nc);
  const T* Bsr = fwork + v.F + (int64_t)nR * nR;
  T* FII = fwork + v.F;
  T acc[4][4];
  zero_acc(acc);
  if (k > 0) {
    tile_mma<T, false>(
        sm, acc, k,
        [&](int r, int s) { return (i0 + r < nR) ? Acc[(int64_t)perm[s] * nc + perm[k + i0 + r]] : T(0); },
        [&](int s, int c) { return (j0 + c < nR) ? Tm[(int64_t)s * nR + j0 + c] : T(0); });
    tile_mma<T, false>(
        sm, acc, k, [&](int r, int s) { return (i0 + r < nR) ? Tm[(int64_t)s * nR + i0 + r] : T(0); },
        [&](int s, int c) { return (j0 + c < nR) ? Bsr[(int64_t)s * nR + j0 + c] : T(0); });
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
      if (r < nR && c < nR)
        FII[(int64_t)r * nR + c] = Acc[(int64_t)perm[k + r] * nc + perm[k + c]] - acc[i][j];
    }
}

// ---- B_ss (F_BB after the elimination) into the first adjacent cell's
// update matrix, zeros into the second's
template <typename T>
__global__ void k_bf_scatter(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                             const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                             const int* __restrict__ obuf, const T* __restrict__ fwork, T* __restrict__ cwork) {
  const FrontDesc fd = fronts[big[blockIdx.y]];
  const BfView v = bf_view(fd);
  const int nc = fd.nc, nN = fd.nN;
  const int* out = obuf + fd.out;
  const int k = out[0], nR = nc - k;
  const int* perm = out + 1;
  if (k == 0 || nR == 0) return;
  const int* idc = ipool + fd.ids;
  const int* pos1 = idc + nc;
  const int* pos2 = pos1 + nc + nN;
  const CellDesc P1 = cells[fd.P1], P2 = cells[fd.P2];
  T* U1 = cwork + P1.F + (int64_t)P1.nI * P1.nI + (int64_t)P1.nB * P1.nI;
  T* U2 = cwork + P2.F + (int64_t)P2.nI * P2.nI + (int64_t)P2.nB * P2.nI;
  const int ld1 = P1.nB, ld2 = P2.nB;
  const T* FBB = fwork + v.F + (int64_t)nR * nR + (int64_t)k * nR;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    const int ci = perm[i], cj = perm[j];
    U1[(int64_t)pos1[ci] * ld1 + pos1[cj]] = FBB[e];
    if (pos2[ci] >= 0 && pos2[cj] >= 0) U2[(int64_t)pos2[ci] * ld2 + pos2[cj]] = T(0);
  }
}

// ---- pivoted QR of M by a group of co-resident thread blocks per front.
// Block g of G owns the columns [g nc / G, (g+1) nc / G).  Every step: each
// block writes the squared residual norms of its unchosen columns (parity
// buffer of the front's scratch), one group barrier, then every block takes
// the same pivot from all norms (tie rule and rank rule of blk_pivoted_qr),
// builds the reflector from the pivot column and applies it to its own
// columns.  The pivot column itself is never rewritten (its diagonal R_ii
// goes to diagR), so blocks still reading it are never raced.  The norms
// and dot products are the warp-per-column reductions of blk_pivoted_qr, so
// pivots, R and T are those of the one-block kernel bit for bit.
// Scratch per front: sq[2][nc] | diagR[nc] (double) | chosen[nc] (int) |
// barrier[2] (unsigned), zeroed before the launch.
__device__ bool group_barrier(unsigned* bar, int G, int* err, long polls = 1L << 22) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == (unsigned)(G - 1)) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (*vgen == gen) {
        if (++it > polls) {        // ~0.1-1 s: a member never arrived
          atomicOr(err, 16);
          s_ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- check of the bounded wait: one block of a group of two (the other
// never arrives) waits at the group barrier with `polls` polls; the wait
// gives up, sets bit 4 of *err and returns.  bar: two zeroed unsigned.
__global__ void k_wait_test_group(unsigned* bar, int* err, long polls) { group_barrier(bar, 2, err, polls); }

void launch_wait_test_group(unsigned* bar, int* err, long polls, cudaStream_t st) {
  note_launches(1);
  k_wait_test_group<<<1, 64, 0, st>>>(bar, err, polls);
}

__host__ __device__ inline int64_t coop_scratch_elems(int nc) { return 3 * (int64_t)nc + ((int64_t)nc + 4) / 2 + 2; }

template <typename T>
__global__ void __launch_bounds__(256) k_bf_qr_coop(const FrontDesc* __restrict__ fronts, const int* __restrict__ big,
                                                    const int4* __restrict__ ctas, double* __restrict__ scratch,
                                                    const int64_t* __restrict__ soff, const int* __restrict__ ipool,
                                                    T* __restrict__ fwork, T* __restrict__ fac, int* __restrict__ obuf,
                                                    int* __restrict__ state, double eps, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* v = reinterpret_cast<double*>(smem_raw);   // m
  __shared__ double s_alpha, s_vv, s_nu;
  __shared__ int s_piv, s_stop, s_k;
  const int4 cd = ctas[blockIdx.x];
  const int b = cd.x, g = cd.y, G = cd.z;
  if (state[b] != 2) return;                          // the same for the whole group
  const FrontDesc fd = fronts[big[b]];
  const BfView bv = bf_view(fd);
  const int nc = fd.nc, m = fd.nN;
  T* A = fwork + bv.M;
  double* sq2 = scratch + soff[b];
  double* diagR = sq2 + 2 * nc;
  int* chosen = reinterpret_cast<int*>(diagR + nc);
  unsigned* bar = reinterpret_cast<unsigned*>(scratch + soff[b] + coop_scratch_elems(nc) - 2);
  int* out = obuf + fd.out;
  const int c0 = (int)((int64_t)g * nc / G), c1 = (int)((int64_t)(g + 1) * nc / G);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) { s_k = 0; s_stop = 0; }
  const int kmax = m < nc ? m : nc;
  for (int i = 0; i < kmax; ++i) {
    double* sq = sq2 + (i & 1) * nc;
    for (int j = c0 + warp; j < c1; j += nwarps) {
      if (__ldcg(chosen + j)) {
        if (lane == 0) sq[j] = -1.0;
        continue;
      }
      const T* col = A + (int64_t)j * m;
      double acc = 0.0;
      for (int r = i + lane; r < m; r += 32) { const double x = (double)col[r]; acc += x * x; }
      acc = warp_sum(acc);
      if (lane == 0) sq[j] = acc;
    }
    if (!group_barrier(bar, G, status)) return;
    // The pivot is taken from this step's norm snapshot alone, in which the
    // owners marked their chosen columns -1 before the barrier: chosen[] may
    // change during this step (the owner of this step's pivot marks it), the
    // snapshot cannot until every block has passed the next barrier.  Data
    // written by other blocks of the group is read through L2.
    if (warp == 0) {
      double mx = -1.0;
      for (int j = lane; j < nc; j += 32) {
        const double sj = __ldcg(sq + j);
        if (sj > mx) mx = sj;
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int piv = 0x7fffffff;
      for (int j = lane; j < nc; j += 32)
        if (__ldcg(sq + j) >= (1.0 - 1e-10) * mx) { piv = j; break; }
      for (int o = 16; o > 0; o >>= 1) piv = min(piv, __shfl_xor_sync(0xffffffffu, piv, o));
      if (lane == 0) {
        if (i == 0) s_nu = mx;
        const double nu = s_nu;
        const double ratio = (nu > 0.0) ? sqrt(mx / nu) : 0.0;
        if (g == 0 && fabs(ratio - eps) <= 1e-8 * eps) atomicOr(status, 2);
        const int stop = (mx <= 0.0) || (i > 0 && mx <= eps * eps * nu);
        s_stop = stop;
        if (!stop) {
          s_piv = piv;
          const double x0 = (double)__ldcg(A + (int64_t)piv * m + i);
          const double sp = __ldcg(sq + piv);
          const double a2 = (x0 >= 0.0) ? -sqrt(sp) : sqrt(sp);
          s_alpha = a2;
          s_vv = sp - x0 * x0 + (x0 - a2) * (x0 - a2);
          s_k = i + 1;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int piv = s_piv;
    const double alpha = s_alpha, vv = s_vv;
    const T* pc = A + (int64_t)piv * m;
    for (int r = i + threadIdx.x; r < m; r += blockDim.x) v[r] = (double)__ldcg(pc + r) - (r == i ? alpha : 0.0);
    if (threadIdx.x == 0) {
      if (g == 0) {
        out[1 + i] = piv;
        diagR[i] = (double)(T)alpha;
      }
      if (piv >= c0 && piv < c1) chosen[piv] = 1;
    }
    __syncthreads();
    if (vv > 0.0) {
      for (int j = c0 + warp; j < c1; j += nwarps) {
        if (j == piv || __ldcg(chosen + j)) continue;
        T* col = A + (int64_t)j * m;
        double s = 0.0;
        for (int r = i + lane; r < m; r += 32) s += v[r] * (double)col[r];
        s = warp_sum(s);
        const double f = 2.0 * s / vv;
        for (int r = i + lane; r < m; r += 32) col[r] = (T)((double)col[r] - f * v[r]);
      }
    }
    __syncthreads();
  }
  const int k = s_k;
  if (!group_barrier(bar, G, status)) return;
  // redundant columns in ascending order: index of this block's first one
  __shared__ int s_base, s_own;
  if (threadIdx.x == 0) {
    int cnt = 0, own = 0;
    for (int j = 0; j < c0; ++j) cnt += !__ldcg(chosen + j);
    for (int j = c0; j < c1; ++j) own += !__ldcg(chosen + j);
    s_base = cnt;
    s_own = own;
  }
  __syncthreads();
  const int nR = nc - k;
  T* Tm = fac + fd.fac + front_fac_T(nc);
  const int* idc = ipool + fd.ids;
  if (threadIdx.x == 0) {
    int idx = s_base;
    for (int j = c0; j < c1 && idx < nR; ++j)      // (idx < nR holds when the group agrees on k)
      if (!__ldcg(chosen + j)) {
        out[1 + k + idx] = j;
        out[1 + nc + k + idx] = idc[j];
        ++idx;
      }
  }
  __syncthreads();
  // T = R11^-1 R12 for this block's redundant columns (blk_id_T's arithmetic)
  for (int c = s_base + threadIdx.x; c < s_base + s_own && c < nR; c += blockDim.x) {
    const int col = out[1 + k + c];
    const T* r12 = A + (int64_t)col * m;
    for (int t = k - 1; t >= 0; --t) {
      T sum = r12[t];
      for (int u = t + 1; u < k; ++u)
        sum -= __ldcg(A + (int64_t)__ldcg(out + 1 + u) * m + t) * Tm[(int64_t)u * nR + c];
      Tm[(int64_t)t * nR + c] = sum / (T)__ldcg(diagR + t);
    }
  }
  if (g == 0) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) out[1 + nc + t] = idc[__ldcg(out + 1 + t)];
    if (threadIdx.x == 0) {
      out[0] = k;
      state[b] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
static int chunk_blocks(int64_t n, int cap) {
  const int64_t b = (n + 256 * 8 - 1) / (256 * 8);
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
void launch_bigfront_id(const FrontDesc* fronts, const int* big, int nbig, const CellDesc* cells, const int* ipool,
                        const T* cwork, T* fwork, T* fac, int* obuf, const int* sketch, SketchStream ss, double eps,
                        int* status, int* state, double* m2part, int nm, int max_nc,
                        int max_nN, int max_ell, const int* h_nc, const int* h_nN, bool coop_ok, cudaStream_t st) {
  if (nbig == 0) return;
  long long nl = 0;
  k_bf_assemble<T><<<dim3(chunk_blocks((int64_t)max_nc * (max_nN + max_nc), 2048), nbig), 256, 0, st>>>(
      fronts, big, cells, ipool, cwork, fwork);
  ++nl;
  const bool sk = sketch && max_ell > 0;
  if (sk) {
    k_bf_colmax<T><<<dim3(nm, nbig), 256, 0, st>>>(fronts, big, fwork, m2part);
    ++nl;
    const int tiles = ((max_ell + TB - 1) / TB) * ((max_nc + TB - 1) / TB);
    k_bf_sketch<T><<<dim3(tiles, nbig), TT, 0, st>>>(fronts, big, sketch, ipool, fwork, ss);
    ++nl;
    const int ztiles = ((max_ell + TB - 1) / TB) * ((max_nN + TB - 1) / TB);
    for (int g = 0; g < ss.power; ++g) {
      k_bf_power_z<T><<<dim3(ztiles, nbig), TT, 0, st>>>(fronts, big, sketch, fwork);
      k_bf_power_y<T><<<dim3(tiles, nbig), TT, 0, st>>>(fronts, big, sketch, fwork);
      nl += 2;
    }
  }
  const int smem = (int)(sizeof(double) * (max_nc + max_nN) + sizeof(int) * 2 * max_nc + 64);
  if (smem > 48 * 1024)
    raise_smem_limit(k_bf_id<T>);
  // groups of the multi-block QR: blocks per front in proportion to its QR
  // work (|N| |c|^2), at least 32 columns per block, all co-resident
  const int csmem = (int)(sizeof(double) * max_nN + 64);
  bool coop = coop_ok && csmem <= 200 * 1024;
  std::vector<int4> ctas;
  std::vector<int64_t> soff(nbig);
  int64_t sc_elems = 0;
  if (coop) {
    if (csmem > 48 * 1024)
      raise_smem_limit(k_bf_qr_coop<T>);
    int nb = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bf_qr_coop<T>, 256, csmem) != cudaSuccess) {
      cudaGetLastError();
      nb = 0;
    }
    const int cap = nb * nsm;
    double wsum = 0.0;
    for (int b = 0; b < nbig; ++b) wsum += (double)h_nN[b] * h_nc[b] * h_nc[b];
    std::vector<int> G(nbig, 1);
    int tot = nbig;
    if (cap >= nbig) {
      tot = 0;
      for (int b = 0; b < nbig; ++b) {
        const double w = (double)h_nN[b] * h_nc[b] * h_nc[b];
        int g = (int)((double)(cap - nbig) * w / (wsum > 0 ? wsum : 1.0)) + 1;
        g = std::min(g, std::max(1, h_nc[b] / 32));
        G[b] = g;
        tot += g;
      }
    }
    coop = cap >= nbig && tot <= cap;
    if (coop) {
      for (int b = 0; b < nbig; ++b) {
        soff[b] = sc_elems;
        sc_elems += (coop_scratch_elems(h_nc[b]) + 3) & ~int64_t(3);
        for (int g = 0; g < G[b]; ++g) ctas.push_back(make_int4(b, g, G[b], 0));
      }
    }
  }
  k_bf_id<T><<<nbig, 256, smem, st>>>(fronts, big, sketch, ipool, fwork, fac, obuf, state, eps, status, 0,
                                      coop ? 1 : 0, m2part, nm, ss.power);
  ++nl;
  bool done = false;
  if (coop) {
    // descriptors and the zeroed scratch live in one stream-ordered buffer
    const size_t cbytes = sizeof(int4) * ctas.size(), obytes = sizeof(int64_t) * soff.size();
    const size_t off_s = (cbytes + obytes + 255) & ~size_t(255);
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, off_s + sizeof(double) * (size_t)sc_elems, st) == cudaSuccess) {
      char* cb = static_cast<char*>(buf);
      cudaMemcpyAsync(cb, ctas.data(), cbytes, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(cb + cbytes, soff.data(), obytes, cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(cb + off_s, 0, sizeof(double) * (size_t)sc_elems, st);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)ctas.size());
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = csmem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, k_bf_qr_coop<T>, fronts, big,
                                               reinterpret_cast<const int4*>(cb),
                                               reinterpret_cast<double*>(cb + off_s),
                                               reinterpret_cast<const int64_t*>(cb + cbytes), ipool, fwork, fac,
                                               obuf, state, eps, status);
      cudaFreeAsync(buf, st);
      if (e == cudaSuccess) {
        done = true;
        ++nl;
      } else {
        cudaGetLastError();
      }
    } else {
      cudaGetLastError();
    }
  }
  if (!done && (sk || coop)) {
    k_bf_id<T><<<nbig, 256, smem, st>>>(fronts, big, sketch, ipool, fwork, fac, obuf, state, eps, status, 1, 0,
                                        m2part, nm, ss.power);
    ++nl;
  }
  note_launches(nl);
}

template <typename T>
void launch_bigfront_form(const FrontDesc* fronts, const int* big, int nbig, const int* obuf, T* fwork,
                          const T* fac, int max_k, int max_nR, cudaStream_t st) {
  if (nbig == 0) return;
  long long nl = 0;
  if (max_k > 0 && max_nR > 0) {
    const int tiles = ((max_k + TB - 1) / TB) * ((max_nR + TB - 1) / TB);
    k_bf_form_sr<T><<<dim3(tiles, nbig), TT, 0, st>>>(fronts, big, obuf, fwork, fac);
    k_bf_form_ss<T><<<dim3(chunk_blocks((int64_t)max_k * max_k, 1024), nbig), 256, 0, st>>>(fronts, big, obuf,
                                                                                           fwork);
    nl += 2;
  }
  if (max_nR > 0) {
    const int P = (max_nR + TB - 1) / TB;
    k_bf_form_rr<T><<<dim3(P * (P + 1) / 2, nbig), TT, 0, st>>>(fronts, big, obuf, fwork, fac);
    ++nl;
  }
  note_launches(nl);
}

template <typename T>
void launch_bigfront_scatter(const FrontDesc* fronts, const int* big, int nbig, const CellDesc* cells,
                             const int* ipool, const int* obuf, const T* fwork, T* cwork, int max_k,
                             cudaStream_t st) {
  if (nbig == 0 || max_k == 0) return;
  note_launches(1);
  k_bf_scatter<T><<<dim3(chunk_blocks((int64_t)max_k * max_k, 1024), nbig), 256, 0, st>>>(fronts, big, cells, ipool,
                                                                                        obuf, fwork, cwork);
}

int bigfront_colmax_blocks(int max_nc) { return (max_nc + 7) / 8; }

#define HIF_BF_INST(T)                                                                                          \
  template void launch_bigfront_id<T>(const FrontDesc*, const int*, int, const CellDesc*, const int*, const T*, \
                                      T*, T*, int*, const int*, SketchStream, double, int*, int*, double*, int, \
                                      int, int, int, const int*, const int*, bool, cudaStream_t);               \
  template void launch_bigfront_form<T>(const FrontDesc*, const int*, int, const int*, T*, const T*, int, int,  \
                                        cudaStream_t);                                                           \
  template void launch_bigfront_scatter<T>(const FrontDesc*, const int*, int, const CellDesc*, const int*,      \
                                           const int*, const T*, T*, int, cudaStream_t);
HIF_BF_INST(double)
HIF_BF_INST(float)
#undef HIF_BF_INST

}  // namespace hif
