// The assembled upper levels of HIF-DE in 3D with edge skeletonization
// (Section 4.5, Algorithm 4.2).  From the first edge level on, the cells of
// a level are Voronoi cells of the active DOFs (peeled so that no two cells
// are coupled) and the faces and edges are Voronoi groups; a cell's
// neighbours reach into other cells' neighbourhoods, so the per-cell update
// matrices of the lower levels cannot hold A_l.  Here A_l is one dense
// matrix over the DOFs active at the hand-over (row-major, side n_act,
// global DOF g at row map[g]); rows of DOFs that leave are never read again.
//
//   hand-over: A = sum over the last box cells of their update matrices
//              (k_dense_from_cells, atomic adds: cells share boundaries);
//   cells:     F_II = A_pp, F_BI = A_qp, F_BB = 0 (k_dense_gather_cells);
//              the cell kernels then leave -A_qp A_pp^-1 A_pq in F_BB, which
//              is added to A_qq (k_dense_scatter_cells).  Cells of a level
//              are uncoupled, so no cell reads a column another one writes,
//              and the additions commute (Lemma 2.1 for each cell);
//   groups:    the front kernels read A_{N,c} and A_cc through a one-cell
//              view of A (pos1 = map of [c ; N], no second cell) and write
//              the new A_ss over the old (Lemma 2.4);
//   root:      D = A restricted to the DOFs still active (k_dense_gather_root).
#include <cstdint>

#include "hif_internal.h"
#include "kernels.h"

namespace hif {

template <typename TU, typename TA>
__global__ void k_dense_from_cells(const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                                   const TU* __restrict__ work, const int* __restrict__ map, TA* __restrict__ A,
                                   int64_t n_act) {
  const CellDesc c = cells[blockIdx.y];
  const int nB = c.nB;
  const int* idB = ipool + c.ids + c.nI;
  const TU* U = work + c.F + (int64_t)c.nI * c.nI + (int64_t)nB * c.nI;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nB * nB; e += stride) {
    const int i = (int)(e / nB), j = (int)(e % nB);
    const int di = map[idB[i]], dj = map[idB[j]];
    if (di >= 0 && dj >= 0) atomicAdd(A + di * n_act + dj, (TA)U[e]);
  }
}

template <typename T>
__global__ void k_dense_gather_cells(const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                                     const int* __restrict__ map, const T* __restrict__ A, int64_t n_act,
                                     T* __restrict__ work) {
  const CellDesc c = cells[blockIdx.y];
  const int nI = c.nI, nB = c.nB;
  const int* idp = ipool + c.ids;
  const int* idq = idp + nI;
  T* FII = work + c.F;
  T* FBI = FII + (int64_t)nI * nI;
  T* FBB = FBI + (int64_t)nB * nI;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t e = t0; e < (int64_t)nI * nI; e += stride) {
    const int i = (int)(e / nI), j = (int)(e % nI);
    FII[e] = A[map[idp[i]] * n_act + map[idp[j]]];
  }
  for (int64_t e = t0; e < (int64_t)nB * nI; e += stride) {
    const int i = (int)(e / nI), j = (int)(e % nI);
    FBI[e] = A[map[idq[i]] * n_act + map[idp[j]]];
  }
  for (int64_t e = t0; e < (int64_t)nB * nB; e += stride) FBB[e] = T(0);
}

template <typename T>
__global__ void k_dense_scatter_cells(const CellDesc* __restrict__ cells, const int* __restrict__ ipool,
                                      const int* __restrict__ map, T* __restrict__ A, int64_t n_act,
                                      const T* __restrict__ work) {
  const CellDesc c = cells[blockIdx.y];
  const int nI = c.nI, nB = c.nB;
  const int* idq = ipool + c.ids + nI;
  const T* FBB = work + c.F + (int64_t)nI * nI + (int64_t)nB * nI;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nB * nB; e += stride) {
    const int i = (int)(e / nB), j = (int)(e % nB);
    atomicAdd(A + map[idq[i]] * n_act + map[idq[j]], FBB[e]);
  }
}

template <typename TA, typename TD>
__global__ void k_dense_gather_root(const int* __restrict__ ids, int n, const int* __restrict__ map,
                                    const TA* __restrict__ A, int64_t n_act, TD* __restrict__ D) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n; e += stride) {
    const int i = (int)(e / n), j = (int)(e % n);
    D[e] = (TD)A[map[ids[i]] * n_act + map[ids[j]]];
  }
}

static inline int dense_blocks(int64_t elems, int cap) {
  const int64_t b = (elems + 256 * 4 - 1) / (256 * 4);
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename TU, typename TA>
void launch_dense_from_cells(const CellDesc* cells, int ncells, const int* ipool, const TU* work, int max_nB,
                             const int* map, TA* A, int64_t n_act, cudaStream_t st) {
  if (ncells == 0 || max_nB == 0) return;
  note_launches(1);
  k_dense_from_cells<TU, TA><<<dim3(dense_blocks((int64_t)max_nB * max_nB, 256), ncells), 256, 0, st>>>(
      cells, ipool, work, map, A, n_act);
}

template <typename T>
void launch_dense_cells(int phase, const CellDesc* cells, int ncells, const int* ipool, int max_nF,
                        const int* map, T* A, int64_t n_act, T* work, cudaStream_t st) {
  if (ncells == 0 || max_nF == 0) return;
  note_launches(1);
  const dim3 grid(dense_blocks((int64_t)max_nF * max_nF, 256), ncells);
  if (phase == 0)
    k_dense_gather_cells<T><<<grid, 256, 0, st>>>(cells, ipool, map, A, n_act, work);
  else
    k_dense_scatter_cells<T><<<grid, 256, 0, st>>>(cells, ipool, map, A, n_act, work);
}

template <typename TA, typename TD>
void launch_dense_gather_root(const int* ids, int n, const int* map, const TA* A, int64_t n_act, TD* D,
                              cudaStream_t st) {
  if (n == 0) return;
  note_launches(1);
  k_dense_gather_root<TA, TD><<<dense_blocks((int64_t)n * n, 2048), 256, 0, st>>>(ids, n, map, A, n_act, D);
}

template void launch_dense_from_cells<double, double>(const CellDesc*, int, const int*, const double*, int,
                                                      const int*, double*, int64_t, cudaStream_t);
template void launch_dense_from_cells<float, float>(const CellDesc*, int, const int*, const float*, int,
                                                    const int*, float*, int64_t, cudaStream_t);
template void launch_dense_cells<double>(int, const CellDesc*, int, const int*, int, const int*, double*, int64_t,
                                         double*, cudaStream_t);
template void launch_dense_cells<float>(int, const CellDesc*, int, const int*, int, const int*, float*, int64_t,
                                        float*, cudaStream_t);
template void launch_dense_gather_root<double, double>(const int*, int, const int*, const double*, int64_t,
                                                       double*, cudaStream_t);
template void launch_dense_gather_root<float, double>(const int*, int, const int*, const float*, int64_t,
                                                      double*, cudaStream_t);

}  // namespace hif
