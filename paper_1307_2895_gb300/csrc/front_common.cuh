// Device pieces shared by the one-block front kernel and the multi-block
// skeletonization of large fronts: the entries of a front's blocks from the
// two adjacent cells' update matrices, the column-pivoted QR with the rank
// rule of Section 2.2, T = R11^-1 R12 (Lemma 2.2) and the counter-based
// Gaussian stream of the randomized ID (Section 4.3).
#pragma once
#include <cstdint>

#include "blockops.cuh"
#include "hif_internal.h"

namespace hif {

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

// Column-pivoted Householder QR of A (m x nc, column-major, ld m), in place,
// with residual norms recomputed every step (FP64 accumulation), the pivot
// tie rule (smallest position within a factor 1 - 1e-10 of the largest
// squared norm) and the rank rule (stop when |R_ii| <= eps |R_11|).
// perm[0..k) = skeleton columns in pivot order, perm[k..nc) = the others in
// ascending order.  Returns k.  flag_near marks pivot ratios within 1e-8 of
// eps in bit 1 of *status.
template <typename T>
__device__ int blk_pivoted_qr(T* A, int m, int nc, double eps, int* status, bool flag_near, double* sq,
                              double* v, int* perm, int* chosen) {
  __shared__ double s_mx, s_vv, s_alpha;
  __shared__ int s_piv, s_stop, s_k;
  for (int j = threadIdx.x; j < nc; j += blockDim.x) chosen[j] = 0;
  if (threadIdx.x == 0) { s_k = 0; s_stop = 0; }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int kmax = m < nc ? m : nc;
  for (int i = 0; i < kmax; ++i) {
    for (int j = warp; j < nc; j += nwarps) {
      if (chosen[j]) continue;
      const T* col = A + (int64_t)j * m;
      double acc = 0.0;
      for (int r = i + lane; r < m; r += 32) { const double x = (double)col[r]; acc += x * x; }
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
        if (i == 0) s_mx = mx;  // |R_11|^2
        const double nu = (i == 0) ? mx : s_mx;
        const double ratio = (nu > 0.0) ? sqrt(mx / nu) : 0.0;
        if (flag_near && fabs(ratio - eps) <= 1e-8 * eps) atomicOr(status, 2);
        const int stop = (mx <= 0.0) || (i > 0 && mx <= eps * eps * nu);
        s_stop = stop;
        if (!stop) {
          s_piv = piv;
          const double x0 = (double)A[(int64_t)piv * m + i];
          const double sp = sq[piv];      // the pivot's own squared norm builds the reflector
          const double a2 = (x0 >= 0.0) ? -sqrt(sp) : sqrt(sp);
          s_alpha = a2;
          s_vv = sp - x0 * x0 + (x0 - a2) * (x0 - a2);
          perm[s_k] = piv;
          chosen[piv] = 1;
          s_k = s_k + 1;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int piv = s_piv;
    const double alpha = s_alpha, vv = s_vv;
    T* pc = A + (int64_t)piv * m;
    for (int r = i + threadIdx.x; r < m; r += blockDim.x) v[r] = (double)pc[r] - (r == i ? alpha : 0.0);
    __syncthreads();
    if (vv > 0.0) {
      for (int j = warp; j < nc; j += nwarps) {
        if (chosen[j]) continue;
        T* col = A + (int64_t)j * m;
        double s = 0.0;
        for (int r = i + lane; r < m; r += 32) s += v[r] * (double)col[r];
        s = warp_sum(s);
        const double f = 2.0 * s / vv;
        for (int r = i + lane; r < m; r += 32) col[r] = (T)((double)col[r] - f * v[r]);
      }
    }
    for (int r = i + threadIdx.x; r < m; r += blockDim.x) pc[r] = (r == i) ? (T)alpha : T(0);
    __syncthreads();
  }
  const int k = s_k;
  if (threadIdx.x == 0) {
    int t = k;
    for (int j = 0; j < nc; ++j) if (!chosen[j]) perm[t++] = j;
  }
  __syncthreads();
  return k;
}

// T = R11^{-1} R12 from the factored A of blk_pivoted_qr (back substitution,
// one thread per redundant column); T is k x (nc - k), row-major.
template <typename T>
__device__ void blk_id_T(const T* A, int m, const int* perm, int k, int nc, T* Tm) {
  const int nR = nc - k;
  for (int c = threadIdx.x; c < nR; c += blockDim.x) {
    const T* r12 = A + (int64_t)perm[k + c] * m;
    for (int t = k - 1; t >= 0; --t) {
      T s = r12[t];
      for (int u = t + 1; u < k; ++u) s -= A[(int64_t)perm[u] * m + t] * Tm[(int64_t)u * nR + c];
      Tm[(int64_t)t * nR + c] = s / A[(int64_t)perm[t] * m + t];
    }
  }
  __syncthreads();
}

// Rank tolerance of the pivoted QR of a sketch, relative to eps: the sketch's
// skeleton set is chosen at kSketchRankTol * eps so that the interpolation of
// A_{N,c} itself meets eps (a Gaussian sketch's pivots track those of A_{N,c}
// only to a modest factor).
constexpr double kSketchRankTol = 0.1;

// T for given skeletons by least squares on M itself (the sketched ID of
// Section 4.3 keeps only the sketch's choice of skeletons): Householder QR of
// the columns perm[0..k) of C (a copy of M, m x nc, column-major) in that
// order, applied to the other columns -- the first k steps of
// blk_pivoted_qr with the pivots given -- then T = R11^-1 R12 (k x (nc - k)),
// which minimizes every column norm of M_r - M_s T.  Returns the largest
// squared residual column norm (rows k..m-1 of the transformed redundant
// columns), or -1 if a skeleton column vanishes.  v: m doubles; chosen: nc
// ints of scratch.
template <typename T>
__device__ double blk_ls_id(T* C, int m, int nc, const int* perm, int k, int* chosen, double* v, T* Tm) {
  __shared__ double s_alpha, s_vv, s_red[32];
  __shared__ int s_bad;
  for (int j = threadIdx.x; j < nc; j += blockDim.x) chosen[j] = 0;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int i = 0; i < k; ++i) {
    const int piv = perm[i];
    T* pc = C + (int64_t)piv * m;
    if (warp == 0) {
      double acc = 0.0;
      for (int r = i + lane; r < m; r += 32) { const double x = (double)pc[r]; acc += x * x; }
      acc = warp_sum(acc);
      if (lane == 0) {
        if (!(acc > 0.0)) {
          s_bad = 1;
        } else {
          const double x0 = (double)pc[i];
          const double a2 = (x0 >= 0.0) ? -sqrt(acc) : sqrt(acc);
          s_alpha = a2;
          s_vv = acc - x0 * x0 + (x0 - a2) * (x0 - a2);
          chosen[piv] = 1;
        }
      }
    }
    __syncthreads();
    if (s_bad) return -1.0;
    const double alpha = s_alpha, vv = s_vv;
    for (int r = i + threadIdx.x; r < m; r += blockDim.x) v[r] = (double)pc[r] - (r == i ? alpha : 0.0);
    __syncthreads();
    if (vv > 0.0) {
      for (int j = warp; j < nc; j += nwarps) {
        if (chosen[j]) continue;
        T* col = C + (int64_t)j * m;
        double s = 0.0;
        for (int r = i + lane; r < m; r += 32) s += v[r] * (double)col[r];
        s = warp_sum(s);
        const double f = 2.0 * s / vv;
        for (int r = i + lane; r < m; r += 32) col[r] = (T)((double)col[r] - f * v[r]);
      }
    }
    for (int r = i + threadIdx.x; r < m; r += blockDim.x) pc[r] = (r == i) ? (T)alpha : T(0);
    __syncthreads();
  }
  blk_id_T(C, m, perm, k, nc, Tm);
  double e2 = 0.0;
  for (int c = warp; c < nc - k; c += nwarps) {
    const T* col = C + (int64_t)perm[k + c] * m;
    double s = 0.0;
    for (int r = k + lane; r < m; r += 32) { const double x = (double)col[r]; s += x * x; }
    e2 = fmax(e2, warp_sum(s));
  }
  if (lane == 0) s_red[warp] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < nwarps; ++w) mx = fmax(mx, s_red[w]);
    s_red[0] = mx;
  }
  __syncthreads();
  const double r = s_red[0];
  __syncthreads();
  return r;
}

// splitmix64 (Steele, Lea and Flood, 2014): output number c >= 1 of the
// stream seeded with s is the mixing function of the state s + c * gamma.
__device__ __forceinline__ uint64_t smix_at(uint64_t s, uint64_t c) {
  uint64_t z = s + c * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Standard normal number e of the stream seeded with key: Box-Muller (cosine
// branch) of u1 = 1 - U(2e + 1) in (0, 1] and u2 = U(2e + 2), U(c) the top 53
// bits of output c over 2^53.
__device__ __forceinline__ double sketch_normal(uint64_t key, uint64_t e) {
  const double u1 = 1.0 - (double)(smix_at(key, 2 * e + 1) >> 11) * 0x1p-53;
  const double u2 = (double)(smix_at(key, 2 * e + 2) >> 11) * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
// Rank tolerance of the pivoted QR of a sketch with `power` power
// iterations: Y's singular values are A's to the power 2 power + 1.
__device__ __forceinline__ double sketch_rank_tol(double eps, int power) {
  const double t = eps * kSketchRankTol;
  double r = t;
  for (int p = 0; p < power; ++p) r *= t * t;
  return r;
}

// Key of the front whose smallest DOF id is c0 (see SketchStream).
__device__ __forceinline__ uint64_t sketch_key(const SketchStream& ss, int c0) {
  return smix_at(ss.seed, ss.level_base + (uint64_t)c0 + 1);
}

}  // namespace hif
