// Interior elimination (Lemma 2.1) of large cells, tiled over many thread
// blocks.  The single-block kernel (k_cell_factor) leaves all but a few SMs
// idle at the top levels of the tree, where a handful of cells carry
// thousands of interior DOFs; here every cell of such a level is cut into
// 64 x 64 tiles and each step of a blocked right-looking Cholesky runs as one
// launch over the tiles of all the level's large cells:
//
//   for each panel p:  A_pp = L_pp S_p L_pp^T, D_p = L_pp^{-1}      (k_tl_potrf)
//                      [A; F_BI]_{i,p} <- [A; F_BI]_{i,p} D_p^T S_p (k_tl_trsm)
//                      A_ij, F_BI,j -= L_ip S_p L_jp^T  (j > p)     (k_tl_update)
//   U = F_BB - G S G^T with G = F_BI L^{-T} S (the stacked panels)  (k_tl_syrk)
//   Linv_ij = -D_i sum_{k=j}^{i-1} L_ik Linv_kj  (row block i)      (k_tl_linv)
//   pack L and G into the factor                                    (k_tl_pack)
//
// S = diag(+-1) holds the signs of the pivots: all +1 (Cholesky) on a
// positive definite block; an indefinite one (the Helmholtz operator's) gets
// the signed LDL^T of blk_cholesky, 1 x 1 pivots in order, with the signs
// written to the factor by k_tl_potrf.  The mixed mode's safeguarded pivots
// are positive, so its tensor-core panels carry no signs.
// Results are those of k_cell_factor up to rounding order: the same L, Linv,
// S, G and Schur complement.  Scratch (the D_p tiles and the original diagonal
// for the pivot safeguard) lives in the problem's X region of the work pool.
// Each problem is described by a TDesc (a large cell, or the redundant block
// of a large front).
#include <atomic>
#include <type_traits>

#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"
#include "tile_mma.cuh"

namespace hif {


// original diagonal of F_II (pivot safeguard of the mixed mode)
template <typename T>
__global__ void k_tl_init(const TDesc* __restrict__ td, T* __restrict__ work) {
  const TCell c = tcell(td[blockIdx.y]);
  T* d0 = work + c.X + (int64_t)c.P * TB * TB;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.nI; i += gridDim.x * blockDim.x)
    d0[i] = work[c.FII + (int64_t)i * c.nI + i];
}

// Panel p: Cholesky of the diagonal tile and its inverse D_p (written to the
// scratch tile, zero-padded to 64 x 64, and to Linv's diagonal tile).
template <typename T>
__global__ void k_tl_potrf(const TDesc* __restrict__ td, int p,
                           T* __restrict__ work, T* __restrict__ fac, int* status, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);   // TB x TB
  T* X = A + TB * TB;                      // TB x TB
  const TCell c = tcell(td[blockIdx.x]);
  if (p >= c.P) return;
  const int o = p * TB, w = min(TB, c.nI - o);
  T* FII = work + c.FII;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e / TB, q = e % TB;
    A[e] = (r < w && q < w) ? FII[(int64_t)(o + r) * c.nI + o + q] : T(0);
  }
  __syncthreads();
  const T* d0 = (tau > T(0)) ? work + c.X + (int64_t)c.P * TB * TB + o : nullptr;
  blk_cholesky(A, w, TB, status, tau, d0, fac + c.S + o);   // signs of the panel's pivots
  blk_tri_inverse(A, w, TB, X, TB);
  T* D = work + c.X + (int64_t)p * TB * TB;
  T* Linv = fac + c.Linv;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e / TB, q = e % TB;
    const bool in = (r < w && q < w);
    D[e] = in ? X[r * TB + q] : T(0);
    if (in && q <= r) {
      FII[(int64_t)(o + r) * c.nI + o + q] = A[r * TB + q];
      Linv[tri64(o + r) + o + q] = X[r * TB + q];
    }
  }
}

// Panel p: row tiles below the diagonal (F_II rows, then F_BI rows) times D_p^T.
template <typename T>
__global__ void __launch_bounds__(TT) k_tl_trsm(const TDesc* __restrict__ td,
                                                int p, T* __restrict__ work, const T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const TCell c = tcell(td[blockIdx.y]);
  if (p >= c.P) return;
  const int below = c.P - p - 1;
  const int t = blockIdx.x;
  if (t >= below + c.RB) return;
  const int o = p * TB, w = min(TB, c.nI - o);
  T* M;          // first row of the tile
  int rows;
  if (t < below) {
    const int r0 = (p + 1 + t) * TB;
    M = work + c.FII + (int64_t)r0 * c.nI;
    rows = min(TB, c.nI - r0);
  } else {
    const int r0 = (t - below) * TB;
    M = work + c.FBI + (int64_t)r0 * c.nI;
    rows = min(TB, c.nB - r0);
  }
  const T* D = work + c.X + (int64_t)p * TB * TB;
  const T* sg = fac + c.S + o;
  const int ld = c.nI;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, true>(
      sm, acc, w, [&](int r, int k) { return r < rows ? M[(int64_t)r * ld + o + k] : T(0); },
      [&](int k, int q) { return D[q * TB + k]; });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, q = tx + 16 * j;
      if (r < rows && q < w) M[(int64_t)r * ld + o + q] = acc[i][j] * sg[q];
    }
}

// Panel p: trailing update of column tiles j > p: lower tiles of F_II, then
// all row tiles of F_BI.
template <typename T>
__global__ void __launch_bounds__(TT) k_tl_update(const TDesc* __restrict__ td,
                                                  int p, T* __restrict__ work, const T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const TCell c = tcell(td[blockIdx.y]);
  if (p >= c.P) return;
  const int m = c.P - p - 1;
  const int64_t nlow = (int64_t)m * (m + 1) / 2;
  const int64_t t = blockIdx.x;
  if (m <= 0 || t >= nlow + (int64_t)c.RB * m) return;
  const int o = p * TB, w = min(TB, c.nI - o);
  const int ld = c.nI;
  const T* Lrow;   // left operand rows (panel columns o .. o + w)
  T* Out;
  int rows, j;
  if (t < nlow) {
    int a, b;
    tri_decode(t, a, b);
    const int i = p + 1 + a;
    j = p + 1 + b;
    Lrow = work + c.FII + (int64_t)i * TB * ld;
    Out = work + c.FII + (int64_t)i * TB * ld;
    rows = min(TB, c.nI - i * TB);
  } else {
    const int64_t u = t - nlow;
    const int rb = (int)(u / m);
    j = p + 1 + (int)(u % m);
    Lrow = work + c.FBI + (int64_t)rb * TB * ld;
    Out = work + c.FBI + (int64_t)rb * TB * ld;
    rows = min(TB, c.nB - rb * TB);
  }
  const T* Lcol = work + c.FII + (int64_t)j * TB * ld;
  const T* sg = fac + c.S + o;
  const int cols = min(TB, c.nI - j * TB);
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, true>(
      sm, acc, w, [&](int r, int k) { return r < rows ? Lrow[(int64_t)r * ld + o + k] * sg[k] : T(0); },
      [&](int k, int q) { return q < cols ? Lcol[(int64_t)q * ld + o + k] : T(0); });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int oc = j * TB;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int r = ty + 16 * i, q = tx + 16 * jj;
      if (r < rows && q < cols) Out[(int64_t)r * ld + oc + q] -= acc[i][jj];
    }
}

// U = F_BB - G S G^T (G = F_BI after the panels), tile (i, j >= ... ) with
// i >= j, mirrored into (j, i).
template <typename T>
__global__ void __launch_bounds__(TT) k_tl_syrk(const TDesc* __restrict__ td,
                                                T* __restrict__ work, const T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const TCell c = tcell(td[blockIdx.y]);
  const int64_t t = blockIdx.x;
  if (t >= (int64_t)c.RB * (c.RB + 1) / 2) return;
  int a, b;
  tri_decode(t, a, b);
  const int ld = c.nI;
  const T* Gi = work + c.FBI + (int64_t)a * TB * ld;
  const T* Gj = work + c.FBI + (int64_t)b * TB * ld;
  const int ri = min(TB, c.nB - a * TB), rj = min(TB, c.nB - b * TB);
  const T* sg = fac + c.S;
  T acc[4][4];
  zero_acc(acc);
  tile_mma<T, true>(
      sm, acc, c.nI, [&](int r, int k) { return r < ri ? Gi[(int64_t)r * ld + k] * sg[k] : T(0); },
      [&](int k, int q) { return q < rj ? Gj[(int64_t)q * ld + k] : T(0); });
  T* U = work + c.FBB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int r = ty + 16 * i, q = tx + 16 * jj;
      if (r < ri && q < rj) {
        const int64_t R = a * TB + r, Q = b * TB + q;
        const T v = U[R * c.nB + Q] - acc[i][jj];
        U[R * c.nB + Q] = v;
        if (a != b) U[Q * c.nB + R] = v;
      }
    }
}

// Row block i of Linv: tiles (i, j), j < i.
template <typename T>
__global__ void __launch_bounds__(TT) k_tl_linv(const TDesc* __restrict__ td,
                                                int i, const T* __restrict__ work, T* __restrict__ fac) {
  __shared__ TileSmem<T> sm;
  const TCell c = tcell(td[blockIdx.y]);
  const int j = blockIdx.x;
  if (i >= c.P || j >= i) return;
  const int ld = c.nI;
  const int r0 = i * TB, c0 = j * TB;
  const int rows = min(TB, c.nI - r0);
  const T* Lr = work + c.FII + (int64_t)r0 * ld;
  T* Linv = fac + c.Linv;
  T acc[4][4];
  zero_acc(acc);
  // tmp = sum_{k=j}^{i-1} L_ik Linv_kj  (k runs over columns c0 .. r0 of L)
  tile_mma<T, false>(
      sm, acc, r0 - c0, [&](int r, int k) { return r < rows ? Lr[(int64_t)r * ld + c0 + k] : T(0); },
      [&](int k, int q) {
        const int64_t R = c0 + k, Q = c0 + q;
        return Q <= R ? Linv[tri64(R) + Q] : T(0);
      });
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = ty + 16 * a, q = tx + 16 * b;
      if (r < rows) Linv[tri64(r0 + r) + c0 + q] = acc[a][b];
    }
  __syncthreads();
  const T* D = work + c.X + (int64_t)i * TB * TB;
  T acc2[4][4];
  zero_acc(acc2);
  tile_mma<T, false>(
      sm, acc2, rows, [&](int r, int k) { return D[r * TB + k]; },
      [&](int k, int q) { return Linv[tri64(r0 + k) + c0 + q]; });
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = ty + 16 * a, q = tx + 16 * b;
      if (r < rows) Linv[tri64(r0 + r) + c0 + q] = -acc2[a][b];
    }
}

// L (lower F_II, packed by rows) and G (= F_BI) into the factor.
template <typename T>
__global__ void k_tl_pack(const TDesc* __restrict__ td,
                          const T* __restrict__ work, T* __restrict__ fac) {
  const TCell c = tcell(td[blockIdx.y]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = blockIdx.x * (blockDim.x >> 5) + warp; r < c.nI + c.nB; r += gridDim.x * (blockDim.x >> 5)) {
    if (r < c.nI) {
      const T* src = work + c.FII + (int64_t)r * c.nI;
      T* dst = fac + c.Lp + tri64(r);
      for (int q = lane; q <= r; q += 32) dst[q] = src[q];
    } else {
      const T* src = work + c.FBI + (int64_t)(r - c.nI) * c.nI;
      T* dst = fac + c.G + (int64_t)(r - c.nI) * c.nI;
      for (int q = lane; q < c.nI; q += 32) dst[q] = src[q];
    }
  }
}

template <typename T>
void launch_tiled_elim(const TDesc* td, int nsel, int max_nI, int max_nB, T* work, T* fac, int* status,
                       double tau, cudaStream_t st, int tc_split) {
  // FP32 with tc_split > 0: the panel solves, trailing updates and the Schur
  // complement run on the tensor cores (kernels_tc.cu), each operand split
  // into tc_split TF32 parts
  const bool tc = std::is_same<T, float>::value && tc_split > 0;
  if (nsel == 0 || max_nI == 0) return;
  const int P = (max_nI + TB - 1) / TB, RB = (max_nB + TB - 1) / TB;
  const int psmem = 2 * TB * TB * (int)sizeof(T);
  static std::atomic<bool> attr{false};
  if (!attr) {
    cudaFuncSetAttribute(k_tl_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * TB * TB * 8);
    cudaFuncSetAttribute(k_tl_potrf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * TB * TB * 4);
    attr = true;
  }
  long long nl = 0;
  if (tau > 0.0) {
    k_tl_init<T><<<dim3((max_nI + 255) / 256, nsel), 256, 0, st>>>(td, work);
    ++nl;
  }
  for (int p = 0; p < P; ++p) {
    k_tl_potrf<T><<<nsel, TT, psmem, st>>>(td, p, work, fac, status, (T)tau);
    ++nl;
    if (tc) {
      nl += tc_panel(td, nsel, p, P, max_nI, max_nB, reinterpret_cast<float*>(work), tc_split, status, st);
      continue;
    }
    const int below = P - p - 1;
    if (below + RB > 0) k_tl_trsm<T><<<dim3(below + RB, nsel), TT, 0, st>>>(td, p, work, fac);
    const int64_t nup = (int64_t)below * (below + 1) / 2 + (int64_t)RB * below;
    if (nup > 0) k_tl_update<T><<<dim3((unsigned)nup, nsel), TT, 0, st>>>(td, p, work, fac);
    nl += (below + RB > 0) + (nup > 0);
  }
  if (tc) {
    nl += tc_syrk(td, nsel, max_nB, reinterpret_cast<float*>(work), tc_split, status, st);
  } else if (RB > 0) {
    k_tl_syrk<T><<<dim3((unsigned)((int64_t)RB * (RB + 1) / 2), nsel), TT, 0, st>>>(td, work, fac);
    ++nl;
  }
  for (int i = 1; i < P; ++i) {
    k_tl_linv<T><<<dim3(i, nsel), TT, 0, st>>>(td, i, work, fac);
    ++nl;
  }
  const int rows = max_nI + max_nB;
  k_tl_pack<T><<<dim3((rows + 7) / 8 < 4096 ? (rows + 7) / 8 : 4096, nsel), 256, 0, st>>>(td, work, fac);
  ++nl;
  note_launches(nl);
}

template void launch_tiled_elim<double>(const TDesc*, int, int, int, double*, double*, int*, double, cudaStream_t,
                                        int);
template void launch_tiled_elim<float>(const TDesc*, int, int, int, float*, float*, int*, double, cudaStream_t, int);

}  // namespace hif
