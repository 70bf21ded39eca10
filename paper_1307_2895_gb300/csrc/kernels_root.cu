// D^-1 of a large root (Eq. 4.2's middle factor) by the whole GPU.  The
// root D = L S L^T (S = diag(sgn), all +1 when D is SPD) is stored as L^-1,
// lower triangular and packed by rows (row i at i (i + 1) / 2), and sgn.
// The sweep kernel applies a block with one thread block, which for a 3D
// root of thousands of DOFs leaves one SM streaming megabytes; here
// D^-1 x = L^-T S (L^-1 x) is three launches over all SMs:
//   k_root_lower:   y = S L^-1 x_root, one warp per row (coalesced row reads,
//                   lane-strided dot products, warp sums); also zeroes z;
//   k_root_upper:   z = L^-T y as column strips: a block takes 64 columns and
//                   256 rows, reads each row's 64 entries in one coalesced
//                   load, sums its four row groups and adds to z atomically;
//   k_root_scatter: x_root = z.
// In the deterministic mode the column strips write their partial sums
// (one per block of 256 rows) instead of adding them to z, and the scatter
// adds them in row-block order.
#include <cstdint>

#include "hif_internal.h"
#include "kernels.h"

namespace hif {

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_root_lower(int np, const int* __restrict__ ids, const T* __restrict__ Linv,
                                                    const T* __restrict__ sgn, const T* __restrict__ x, int nr,
                                                    int ldx, T* __restrict__ y, T* __restrict__ z) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t e = gt; e < (int64_t)np * R; e += (int64_t)gridDim.x * blockDim.x) z[e] = T(0);
  const int i = (int)(gt >> 5), lane = threadIdx.x & 31;
  if (i >= np) return;
  const T* l = Linv + (int64_t)i * (i + 1) / 2;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  for (int t = lane; t <= i; t += 32) {
    const T lv = l[t];
    const T* xr = x + (int64_t)ids[t] * ldx;
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] += lv * (c < nr ? xr[c] : T(0));
  }
  const T sg = sgn[i];                            // D = diag(sgn) (LDL^T of an indefinite root)
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const T s = warp_sum_t(acc[c]);
    if (lane == c) y[(int64_t)i * R + c] = sg * s;
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_root_upper(int np, const T* __restrict__ Linv, const T* __restrict__ y,
                                                    T* __restrict__ z, T* __restrict__ rpart) {
  __shared__ T part[4][64][R];
  const int j0 = blockIdx.x * 64, i0 = blockIdx.y * 256;
  if (j0 >= i0 + 256 || j0 >= np) return;        // rows i < j hold no entry of column j
  const int jj = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int j = j0 + jj;
  const int i1 = (i0 + 256 < np) ? i0 + 256 : np;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  if (j < np) {
    for (int i = i0 + rg; i < i1; i += 4) {
      if (i < j) continue;
      const T lv = Linv[(int64_t)i * (i + 1) / 2 + j];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] += lv * y[(int64_t)i * R + c];
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c) part[rg][jj][c] = acc[c];
  __syncthreads();
  if (rg == 0 && j < np) {
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const T s = part[0][jj][c] + part[1][jj][c] + part[2][jj][c] + part[3][jj][c];
      if (rpart) rpart[((int64_t)blockIdx.y * np + j) * R + c] = s;
      else atomicAdd(z + (int64_t)j * R + c, s);
    }
  }
}

// rpart (deterministic mode): column j's partial of row block rb at
// rpart[(rb np + j) R + c], written by every row block whose rows reach the
// column's strip (rb >= (64 floor(j / 64)) / 256)
template <typename T, int R>
__global__ void k_root_scatter(int np, const int* __restrict__ ids, const T* __restrict__ z, T* __restrict__ x,
                               int nr, int ldx, const T* __restrict__ rpart) {
  const int nrb = (np + 255) / 256;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)np * nr;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nr), c = (int)(e % nr);
    T v;
    if (rpart) {
      v = T(0);
      for (int rb = ((i / 64) * 64) / 256; rb < nrb; ++rb) v += rpart[((int64_t)rb * np + i) * R + c];
    } else {
      v = z[(int64_t)i * R + c];
    }
    x[(int64_t)ids[i] * ldx + c] = v;
  }
}

template <typename T, int R>
static void root_chunk(int np, const int* ids, const T* Linv, const T* sgn, T* x, int nr, int ldx, T* y, T* z,
                       T* rpart, cudaStream_t st) {
  const int lower_blocks = (int)(((int64_t)np * 32 + 255) / 256);
  k_root_lower<T, R><<<lower_blocks, 256, 0, st>>>(np, ids, Linv, sgn, x, nr, ldx, y, z);
  k_root_upper<T, R><<<dim3((np + 63) / 64, (np + 255) / 256), 256, 0, st>>>(np, Linv, y, z, rpart);
  const int64_t n = (int64_t)np * nr;
  const int sb = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
  k_root_scatter<T, R><<<sb, 256, 0, st>>>(np, ids, z, x, nr, ldx, rpart);
  note_launches(3);
}

int64_t root_scratch_elems(int np, bool det) {
  return (int64_t)np * kRootChunk * (2 + (det ? (np + 255) / 256 : 0));
}

template <typename T>
int launch_root_apply(int np, const int* ids, const T* Linv, const T* sgn, T* x, int nrhs, int ldx, T* scratch,
                      bool det, cudaStream_t st) {
  if (np <= 0 || nrhs <= 0) return 0;
  int launches = 0;
  for (int r0 = 0; r0 < nrhs; r0 += kRootChunk) {
    const int nr = (nrhs - r0) < kRootChunk ? (nrhs - r0) : kRootChunk;
    T* y = scratch;
    T* z = scratch + (int64_t)np * kRootChunk;
    T* rp = det ? scratch + 2 * (int64_t)np * kRootChunk : nullptr;
    if (nr > 4) root_chunk<T, 8>(np, ids, Linv, sgn, x + r0, nr, ldx, y, z, rp, st);
    else if (nr > 2) root_chunk<T, 4>(np, ids, Linv, sgn, x + r0, nr, ldx, y, z, rp, st);
    else if (nr > 1) root_chunk<T, 2>(np, ids, Linv, sgn, x + r0, nr, ldx, y, z, rp, st);
    else root_chunk<T, 1>(np, ids, Linv, sgn, x + r0, nr, ldx, y, z, rp, st);
    launches += 3;
  }
  return launches;
}

template int launch_root_apply<double>(int, const int*, const double*, const double*, double*, int, int, double*,
                                       bool, cudaStream_t);
template int launch_root_apply<float>(int, const int*, const float*, const float*, float*, int, int, float*,
                                      bool, cudaStream_t);

}  // namespace hif
