// 64 x 64 output tiles computed by one thread block of 256 threads (16 x 16,
// 4 x 4 outputs each) from operands staged through shared memory in k-chunks
// of 32; the operands are read through functors, so gathers, permutations
// and generated matrices need no copies.  Used by the tiled elimination of
// large cells and by the skeletonization of large fronts.
#pragma once
#include <cstdint>

#include "hif_internal.h"

namespace hif {

constexpr int TB = kTile;   // tile edge
constexpr int TK = 32;      // k-chunk staged in shared memory
constexpr int TT = 256;     // threads per block

__device__ __forceinline__ int64_t tri64(int64_t r) { return r * (r + 1) / 2; }

// acc[i][j] += sum_{k < K} fa(ty + 16 i, k) * fb(k, tx + 16 j).
// fa(r, k) / fb(k, c) return 0 outside their operands.  BKC: the right
// operand is stored with k contiguous (load it k-fastest for coalescing).
template <typename T>
struct TileSmem {
  T a[TB][TK + 1];
  T b[TK][TB + 1];
};

template <typename T, bool BKC, typename FA, typename FB>
__device__ __forceinline__ void tile_mma(TileSmem<T>& sm, T (&acc)[4][4], int K, FA fa, FB fb) {
  T (*sA)[TK + 1] = sm.a;
  T (*sB)[TB + 1] = sm.b;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TB * TK; e += TT) {
      const int r = e / TK, kk = e % TK;
      sA[r][kk] = (k0 + kk < K) ? fa(r, k0 + kk) : T(0);
    }
    if (BKC) {
      for (int e = threadIdx.x; e < TB * TK; e += TT) {
        const int c = e / TK, kk = e % TK;
        sB[kk][c] = (k0 + kk < K) ? fb(k0 + kk, c) : T(0);
      }
    } else {
      for (int e = threadIdx.x; e < TK * TB; e += TT) {
        const int kk = e / TB, c = e % TB;
        sB[kk][c] = (k0 + kk < K) ? fb(k0 + kk, c) : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// One tiled elimination problem (a large cell, or the redundant block of a
// large front) with its tile counts: P panels of F_II, RB row tiles of F_BI.
struct TCell {
  int nI, nB, P, RB;
  int64_t FII, FBI, FBB, X, Linv, G, Lp, S;
};

__device__ __forceinline__ TCell tcell(const TDesc& d) {
  TCell c;
  c.nI = d.nI;
  c.nB = d.nB;
  c.P = (d.nI + TB - 1) / TB;
  c.RB = (d.nB + TB - 1) / TB;
  c.FII = d.FII;
  c.FBI = d.FBI;
  c.FBB = d.FBB;
  c.X = d.X;
  c.Linv = d.Linv;
  c.G = d.G;
  c.Lp = d.Lp;
  c.S = d.S;
  return c;
}

template <typename T>
__device__ __forceinline__ void zero_acc(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}

}  // namespace hif
