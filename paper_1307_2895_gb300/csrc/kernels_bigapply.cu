// F^-1 sweeps (Eq. 4.2) of the large blocks of a level by many thread
// blocks each.  The one-block sweep kernels give a block one CTA; a 3D
// upper-level cell or face of a few thousand DOFs then streams tens of
// megabytes through one SM while the others wait.  Here the blocks of a level
// above a size threshold are applied as a few launches over all SMs (grid y:
// the block, grid x: its rows or column strips), in the pattern of the
// multi-block root apply (kernels_root.cu):
//
//   up   [front] acc = T^T x_q            column strips, atomics into acc
//        y = Linv (x_p - acc)             one warp per row of Linv
//        x_q -= G y; x_p = S y            one warp per row of G (and of x_p)
//   down acc = G^T x_q                    column strips, atomics into acc
//        z = Linv^T (x_p - acc)           column strips, atomics into z
//        x_p = z; [front] x_q -= T z      one warp per row of T (and of x_p)
//
// (G, T: nq x np row-major; Linv: np x np lower, packed by rows; S: the
// signs of D_p.)  Each block has 2 np kBigChunk elements of scratch at
// bb.scr: acc, then y (or z); the caller zeroes them before a direction.
// The results equal the one-block kernels' up to rounding order.
#include <cstdint>

#include "hif_internal.h"
#include "kernels.h"

namespace hif {

template <typename T>
__device__ __forceinline__ T warp_sum_b(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int64_t tri_b(int64_t i) { return i * (i + 1) / 2; }

// acc[i][c] += sum_s M[s][i] x[idq[s]][c] for a strip of 64 columns i and a
// chunk of 256 rows s of one block (M = T or G, nq x np row-major).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_tmv(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                 const T* __restrict__ fac, int use_t, const T* __restrict__ x,
                                                 int nr, int ldx, T* __restrict__ scratch) {
  __shared__ T part[4][64][R];
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np, nq = bb.d.nq;
  const int strips = (np + 63) / 64;
  const int j0 = (int)(blockIdx.x % strips) * 64, s0 = (int)(blockIdx.x / strips) * 256;
  if (j0 >= np || s0 >= nq) return;
  const int* idq = ipool + bb.d.ids + np;
  const T* M = fac + (use_t ? bb.d.T : bb.d.G);
  const int jj = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int j = j0 + jj;
  const int s1 = (s0 + 256 < nq) ? s0 + 256 : nq;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  if (j < np) {
    for (int s = s0 + rg; s < s1; s += 4) {
      const T m = M[(int64_t)s * np + j];
      const T* xr = x + (int64_t)idq[s] * ldx;
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] += m * (c < nr ? xr[c] : T(0));
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c) part[rg][jj][c] = acc[c];
  __syncthreads();
  if (rg == 0 && j < np) {
    T* a = scratch + bb.scr + (int64_t)j * R;
#pragma unroll
    for (int c = 0; c < R; ++c) atomicAdd(a + c, part[0][jj][c] + part[1][jj][c] + part[2][jj][c] + part[3][jj][c]);
  }
}

// up: y_i = sum_{t <= i} Linv[i][t] (x_p[t] - acc[t]), one warp per row.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_lower(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                   const T* __restrict__ fac, const T* __restrict__ x, int nr,
                                                   int ldx, T* __restrict__ scratch) {
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np;
  const int i = (int)blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= np) return;
  const int* idp = ipool + bb.d.ids;
  const T* l = fac + bb.d.Linv + tri_b(i);
  const T* accv = scratch + bb.scr;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  for (int t = lane; t <= i; t += 32) {
    const T lv = l[t];
    const T* xr = x + (int64_t)idp[t] * ldx;
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] += lv * ((c < nr ? xr[c] : T(0)) - accv[(int64_t)t * R + c]);
  }
  T* y = scratch + bb.scr + (int64_t)np * kBigChunk + (int64_t)i * R;
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const T s = warp_sum_b(acc[c]);
    if (lane == c) y[c] = s;
  }
}

// up: x_q -= G y (fronts own x_q: stored; cells share it: atomics), and
// x_p = S y; warp w takes row w of G and row w of x_p.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_gy(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                const T* __restrict__ fac, int is_front, T* __restrict__ x, int nr,
                                                int ldx, const T* __restrict__ scratch) {
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np, nq = bb.d.nq;
  const int w = (int)blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int* idp = ipool + bb.d.ids;
  const int* idq = idp + np;
  const T* y = scratch + bb.scr + (int64_t)np * kBigChunk;
  if (w < np && lane < nr) x[(int64_t)idp[w] * ldx + lane] = fac[bb.d.S + w] * y[(int64_t)w * R + lane];
  if (w >= nq) return;
  const T* g = fac + bb.d.G + (int64_t)w * np;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  for (int t = lane; t < np; t += 32) {
    const T gv = g[t];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] += gv * y[(int64_t)t * R + c];
  }
  T* xr = x + (int64_t)idq[w] * ldx;
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const T s = warp_sum_b(acc[c]);
    if (lane == c && c < nr) {
      if (is_front) xr[c] = xr[c] - s;
      else atomicAdd(xr + c, -s);
    }
  }
}

// down: z_j += sum_{i >= j} Linv[i][j] (x_p[i] - acc[i]) for a strip of 64
// columns j and a block of 256 rows i (blocks entirely above the diagonal
// return at once).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_upper(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                   const T* __restrict__ fac, const T* __restrict__ x, int nr,
                                                   int ldx, T* __restrict__ scratch) {
  __shared__ T part[4][64][R];
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np;
  const int strips = (np + 63) / 64;
  const int j0 = (int)(blockIdx.x % strips) * 64, i0 = (int)(blockIdx.x / strips) * 256;
  if (j0 >= np || i0 >= np || j0 >= i0 + 256) return;
  const int* idp = ipool + bb.d.ids;
  const T* Linv = fac + bb.d.Linv;
  const T* accv = scratch + bb.scr;
  const int jj = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int j = j0 + jj;
  const int i1 = (i0 + 256 < np) ? i0 + 256 : np;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  if (j < np) {
    for (int i = i0 + rg; i < i1; i += 4) {
      if (i < j) continue;
      const T lv = Linv[tri_b(i) + j];
      const T* xr = x + (int64_t)idp[i] * ldx;
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] += lv * ((c < nr ? xr[c] : T(0)) - accv[(int64_t)i * R + c]);
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c) part[rg][jj][c] = acc[c];
  __syncthreads();
  if (rg == 0 && j < np) {
    T* z = scratch + bb.scr + (int64_t)np * kBigChunk + (int64_t)j * R;
#pragma unroll
    for (int c = 0; c < R; ++c) atomicAdd(z + c, part[0][jj][c] + part[1][jj][c] + part[2][jj][c] + part[3][jj][c]);
  }
}

// down: x_p = z, and (fronts) x_q -= T z; warp w takes row w of x_p and of T.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_tz(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                const T* __restrict__ fac, int is_front, T* __restrict__ x, int nr,
                                                int ldx, const T* __restrict__ scratch) {
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np, nq = bb.d.nq;
  const int w = (int)blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int* idp = ipool + bb.d.ids;
  const int* idq = idp + np;
  const T* z = scratch + bb.scr + (int64_t)np * kBigChunk;
  if (w < np && lane < nr) x[(int64_t)idp[w] * ldx + lane] = z[(int64_t)w * R + lane];
  if (!is_front || w >= nq) return;
  const T* tr = fac + bb.d.T + (int64_t)w * np;
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  for (int t = lane; t < np; t += 32) {
    const T tv = tr[t];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] += tv * z[(int64_t)t * R + c];
  }
  T* xr = x + (int64_t)idq[w] * ldx;
#pragma unroll
  for (int c = 0; c < R; ++c) {
    const T s = warp_sum_b(acc[c]);
    if (lane == c && c < nr) xr[c] = xr[c] - s;
  }
}

template <typename T, int R>
static int big_chunk(int dir, const BigBlock* bbs, int nbig, int max_np, int max_nq, int is_front, const int* ipool,
                     const T* fac, T* x, int nr, int ldx, T* scratch, int64_t scratch_elems, cudaStream_t st) {
  int nl = 0;
  cudaMemsetAsync(scratch, 0, sizeof(T) * (size_t)scratch_elems, st);
  const unsigned strips = (unsigned)((max_np + 63) / 64);
  const unsigned rows8 = (unsigned)((max_np + 7) / 8);
  const int mx = max_np > max_nq ? max_np : max_nq;
  const unsigned both8 = (unsigned)((mx + 7) / 8);
  if (dir == 0) {
    if (is_front && max_nq > 0) {
      const unsigned gx = strips * (unsigned)((max_nq + 255) / 256);
      k_big_tmv<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, 1, x, nr, ldx, scratch);
      ++nl;
    }
    k_big_lower<T, R><<<dim3(rows8, nbig), 256, 0, st>>>(bbs, ipool, fac, x, nr, ldx, scratch);
    k_big_gy<T, R><<<dim3(both8, nbig), 256, 0, st>>>(bbs, ipool, fac, is_front, x, nr, ldx, scratch);
    nl += 2;
  } else {
    if (max_nq > 0) {
      const unsigned gx = strips * (unsigned)((max_nq + 255) / 256);
      k_big_tmv<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, 0, x, nr, ldx, scratch);
      ++nl;
    }
    const unsigned gx = strips * (unsigned)((max_np + 255) / 256);
    k_big_upper<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, x, nr, ldx, scratch);
    k_big_tz<T, R><<<dim3(both8, nbig), 256, 0, st>>>(bbs, ipool, fac, is_front, x, nr, ldx, scratch);
    nl += 2;
  }
  note_launches(nl);
  return nl;
}

template <typename T>
int launch_big_sweep(int dir, const BigBlock* bbs, int nbig, int max_np, int max_nq, int is_front, const int* ipool,
                     const T* fac, T* x, int nrhs, int ldx, T* scratch, int64_t scratch_elems, cudaStream_t st) {
  if (nbig <= 0 || max_np <= 0 || nrhs <= 0) return 0;
  int nl = 0;
  for (int r0 = 0; r0 < nrhs; r0 += kBigChunk) {
    const int nr = (nrhs - r0) < kBigChunk ? (nrhs - r0) : kBigChunk;
    T* xr = x + r0;
    if (nr > 4)
      nl += big_chunk<T, 8>(dir, bbs, nbig, max_np, max_nq, is_front, ipool, fac, xr, nr, ldx, scratch,
                            scratch_elems, st);
    else if (nr > 2)
      nl += big_chunk<T, 4>(dir, bbs, nbig, max_np, max_nq, is_front, ipool, fac, xr, nr, ldx, scratch,
                            scratch_elems, st);
    else if (nr > 1)
      nl += big_chunk<T, 2>(dir, bbs, nbig, max_np, max_nq, is_front, ipool, fac, xr, nr, ldx, scratch,
                            scratch_elems, st);
    else
      nl += big_chunk<T, 1>(dir, bbs, nbig, max_np, max_nq, is_front, ipool, fac, xr, nr, ldx, scratch,
                            scratch_elems, st);
  }
  return nl;
}

template int launch_big_sweep<double>(int, const BigBlock*, int, int, int, int, const int*, const double*, double*,
                                      int, int, double*, int64_t, cudaStream_t);
template int launch_big_sweep<float>(int, const BigBlock*, int, int, int, int, const int*, const float*, float*,
                                     int, int, float*, int64_t, cudaStream_t);

}  // namespace hif
