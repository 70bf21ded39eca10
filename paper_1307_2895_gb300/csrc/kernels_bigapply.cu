// F^-1 sweeps (Eq. 4.2) of the large blocks of a level by many thread
// blocks each.  The one-block sweep kernels give a block one CTA; a 3D
// upper-level cell or face of a few thousand DOFs then streams tens of
// megabytes through one SM while the others wait.  Here the blocks of a level
// above a size threshold are applied as a few launches over all SMs (grid y:
// the block, grid x: its rows or column strips), in the pattern of the
// multi-block root apply (kernels_root.cu):
//
//   up   [front] acc = T^T x_q            column strips, atomics into acc
//        y = Linv (x_p - acc)             32-row x 256-column tiles, atomics into y
//        x_q -= G y; x_p = S y            tiles of G, atomics into x_q
//   down acc = G^T x_q                    column strips, atomics into acc
//        z = Linv^T (x_p - acc)           column strips, atomics into z
//        x_p = z; [front] x_q -= T z      tiles of T, atomics into x_q
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
#pragma unroll 4
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

// Row-times-vector products over one tile of M: the CTA's 32 rows (warp w:
// rows r0 + 8k + w, k < 4) and the columns [t0, t1).  acc[k][c] =
// sum_t M[i][t] v[t][c], over t <= i when M is the packed lower Linv and over
// all t when M is nq x np row-major, summed across the warp.  v (produced
// element-wise by stage(t, c)) is staged in shared memory, read once by the
// CTA, and each staged v[t] is loaded into registers once for the warp's four
// rows.  The kernels below give each tile its own CTA (grid x: row blocks ×
// column chunks) and add the partial sums atomically.
constexpr int kRowsPerCta = 32;
constexpr int kRowsPerWarp = kRowsPerCta / 8;
constexpr int kRowChunk = 256;
template <typename T, int R, typename Stage>
__device__ __forceinline__ void staged_rows(T (*ws)[R], const T* __restrict__ M, bool lower, int np, int nrows,
                                            int r0, int t0, int t1, Stage stage, T (&acc)[kRowsPerWarp][R]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < (t1 - t0) * R; e += blockDim.x) ws[e / R][e % R] = stage(t0 + e / R, e % R);
  const T* rowp[kRowsPerWarp];
  int rlen[kRowsPerWarp];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) {
    const int i = r0 + k * 8 + warp;
    rowp[k] = M + (lower ? tri_b(i) : (int64_t)i * np);
    rlen[k] = (i < nrows) ? (lower ? (i + 1 < t1 ? i + 1 : t1) : t1) : 0;
#pragma unroll
    for (int c = 0; c < R; ++c) acc[k][c] = T(0);
  }
  __syncthreads();
  for (int t = t0 + lane; t < t1; t += 32) {
    T v[R];
#pragma unroll
    for (int c = 0; c < R; ++c) v[c] = ws[t - t0][c];
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
      if (t < rlen[k]) {
        const T m = rowp[k][t];
#pragma unroll
        for (int c = 0; c < R; ++c) acc[k][c] += m * v[c];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[k][c] = warp_sum_b(acc[k][c]);
}

// up: y_i += sum_{t0 <= t < t1, t <= i} Linv[i][t] (x_p[t] - acc[t]) for one
// tile (tiles wholly above the diagonal return at once).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_lower(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                   const T* __restrict__ fac, const T* __restrict__ x, int nr,
                                                   int ldx, T* __restrict__ scratch) {
  __shared__ T ws[kRowChunk][R];
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np;
  const int nrb = (np + kRowsPerCta - 1) / kRowsPerCta, ncb = (np + kRowChunk - 1) / kRowChunk;
  const int rb = (int)(blockIdx.x % nrb), cb = (int)(blockIdx.x / nrb);
  if (cb >= ncb) return;
  const int r0 = rb * kRowsPerCta, t0 = cb * kRowChunk;
  const int rend = (r0 + kRowsPerCta < np) ? r0 + kRowsPerCta : np;
  if (t0 >= rend) return;
  const int t1 = (t0 + kRowChunk < rend) ? t0 + kRowChunk : rend;
  const int* idp = ipool + bb.d.ids;
  const T* accv = scratch + bb.scr;
  T acc[kRowsPerWarp][R];
  staged_rows<T, R>(ws, fac + bb.d.Linv, true, np, np, r0, t0, t1,
                    [&](int t, int c) { return (c < nr ? x[(int64_t)idp[t] * ldx + c] : T(0)) - accv[(int64_t)t * R + c]; },
                    acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) {
    const int i = r0 + k * 8 + warp;
    if (i >= np) continue;
    T* y = scratch + bb.scr + (int64_t)np * kBigChunk + (int64_t)i * R;
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (lane == c) atomicAdd(y + c, acc[k][c]);
  }
}

// up: x_q -= G y over one tile of G, and (first column chunk) x_p = S y for
// the tile's rows.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_gy(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx,
                                                const T* __restrict__ scratch) {
  __shared__ T ws[kRowChunk][R];
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np, nq = bb.d.nq;
  const int mrows = np > nq ? np : nq;
  const int nrb = (mrows + kRowsPerCta - 1) / kRowsPerCta, ncb = (np + kRowChunk - 1) / kRowChunk;
  const int rb = (int)(blockIdx.x % nrb), cb = (int)(blockIdx.x / nrb);
  if (cb >= ncb) return;
  const int r0 = rb * kRowsPerCta, t0 = cb * kRowChunk;
  const int t1 = (t0 + kRowChunk < np) ? t0 + kRowChunk : np;
  const int* idp = ipool + bb.d.ids;
  const int* idq = idp + np;
  const T* y = scratch + bb.scr + (int64_t)np * kBigChunk;
  if (cb == 0) {
    for (int e = threadIdx.x; e < kRowsPerCta * R; e += blockDim.x) {
      const int r = r0 + e / R, c = e % R;
      if (r < np && c < nr) x[(int64_t)idp[r] * ldx + c] = fac[bb.d.S + r] * y[(int64_t)r * R + c];
    }
  }
  if (r0 >= nq) return;
  T acc[kRowsPerWarp][R];
  staged_rows<T, R>(ws, fac + bb.d.G, false, np, nq, r0, t0, t1, [&](int t, int c) { return y[(int64_t)t * R + c]; },
                    acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) {
    const int w = r0 + k * 8 + warp;
    if (w >= nq) continue;
    T* xr = x + (int64_t)idq[w] * ldx;
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (lane == c && c < nr) atomicAdd(xr + c, -acc[k][c]);
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
  __shared__ T wsu[256][R];   // w = x_p - acc on the block's 256 rows, read once
  const int jj = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int j = j0 + jj;
  const int i1 = (i0 + 256 < np) ? i0 + 256 : np;
  for (int e = threadIdx.x; e < (i1 - i0) * R; e += blockDim.x) {
    const int i = i0 + e / R, c = e % R;
    wsu[e / R][c] = (c < nr ? x[(int64_t)idp[i] * ldx + c] : T(0)) - accv[(int64_t)i * R + c];
  }
  __syncthreads();
  T acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = T(0);
  if (j < np) {
    int i = i0 + rg;
    if (i < j) i += ((j - i + 3) >> 2) << 2;   // the first row i >= j of this thread's rows
#pragma unroll 4
    for (; i < i1; i += 4) {
      const T lv = Linv[tri_b(i) + j];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] += lv * wsu[i - i0][c];
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

// down: x_p = z for the tile's rows (first column chunk), and (fronts)
// x_q -= T z over one tile of T.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_big_tz(const BigBlock* __restrict__ bbs, const int* __restrict__ ipool,
                                                const T* __restrict__ fac, int is_front, T* __restrict__ x, int nr,
                                                int ldx, const T* __restrict__ scratch) {
  __shared__ T ws[kRowChunk][R];
  const BigBlock bb = bbs[blockIdx.y];
  const int np = bb.d.np, nq = bb.d.nq;
  const int mrows = np > nq ? np : nq;
  const int nrb = (mrows + kRowsPerCta - 1) / kRowsPerCta, ncb = (np + kRowChunk - 1) / kRowChunk;
  const int rb = (int)(blockIdx.x % nrb), cb = (int)(blockIdx.x / nrb);
  if (cb >= ncb) return;
  const int r0 = rb * kRowsPerCta, t0 = cb * kRowChunk;
  const int t1 = (t0 + kRowChunk < np) ? t0 + kRowChunk : np;
  const int* idp = ipool + bb.d.ids;
  const int* idq = idp + np;
  const T* z = scratch + bb.scr + (int64_t)np * kBigChunk;
  if (cb == 0) {
    for (int e = threadIdx.x; e < kRowsPerCta * R; e += blockDim.x) {
      const int r = r0 + e / R, c = e % R;
      if (r < np && c < nr) x[(int64_t)idp[r] * ldx + c] = z[(int64_t)r * R + c];
    }
  }
  if (!is_front || r0 >= nq) return;
  T acc[kRowsPerWarp][R];
  staged_rows<T, R>(ws, fac + bb.d.T, false, np, nq, r0, t0, t1, [&](int t, int c) { return z[(int64_t)t * R + c]; },
                    acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) {
    const int w = r0 + k * 8 + warp;
    if (w >= nq) continue;
    T* xr = x + (int64_t)idq[w] * ldx;
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (lane == c && c < nr) atomicAdd(xr + c, -acc[k][c]);
  }
}

template <typename T, int R>
static int big_chunk(int dir, const BigBlock* bbs, int nbig, int max_np, int max_nq, int is_front, const int* ipool,
                     const T* fac, T* x, int nr, int ldx, T* scratch, int64_t scratch_elems, cudaStream_t st) {
  int nl = 0;
  cudaMemsetAsync(scratch, 0, sizeof(T) * (size_t)scratch_elems, st);
  const unsigned strips = (unsigned)((max_np + 63) / 64);
  const unsigned cchunks = (unsigned)((max_np + kRowChunk - 1) / kRowChunk);
  const unsigned tiles_p = (unsigned)((max_np + kRowsPerCta - 1) / kRowsPerCta) * cchunks;
  const int mx = max_np > max_nq ? max_np : max_nq;
  const unsigned tiles_pq = (unsigned)((mx + kRowsPerCta - 1) / kRowsPerCta) * cchunks;
  if (dir == 0) {
    if (is_front && max_nq > 0) {
      const unsigned gx = strips * (unsigned)((max_nq + 255) / 256);
      k_big_tmv<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, 1, x, nr, ldx, scratch);
      ++nl;
    }
    k_big_lower<T, R><<<dim3(tiles_p, nbig), 256, 0, st>>>(bbs, ipool, fac, x, nr, ldx, scratch);
    k_big_gy<T, R><<<dim3(tiles_pq, nbig), 256, 0, st>>>(bbs, ipool, fac, x, nr, ldx, scratch);
    nl += 2;
  } else {
    if (max_nq > 0) {
      const unsigned gx = strips * (unsigned)((max_nq + 255) / 256);
      k_big_tmv<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, 0, x, nr, ldx, scratch);
      ++nl;
    }
    const unsigned gx = strips * (unsigned)((max_np + 255) / 256);
    k_big_upper<T, R><<<dim3(gx, nbig), 256, 0, st>>>(bbs, ipool, fac, x, nr, ldx, scratch);
    k_big_tz<T, R><<<dim3(tiles_pq, nbig), 256, 0, st>>>(bbs, ipool, fac, is_front, x, nr, ldx, scratch);
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
