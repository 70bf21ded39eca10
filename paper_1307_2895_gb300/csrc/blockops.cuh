// Dense block operations executed cooperatively by one thread block on a
// matrix in shared or global memory (row-major, leading dimension ld).
// Every routine ends with __syncthreads().
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hif {

// (i, j), j <= i, of the e-th entry of a lower triangle enumerated by rows.
// The square root is taken in FP32 (exact enough up to e ~ 2^24, corrected
// by the integer steps beyond): on this GPU the FP64 pipe is the scarce one.
__device__ __forceinline__ void tri_decode(int64_t e, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((int64_t)(r + 1) * (r + 2) / 2 <= e) ++r;
  while ((int64_t)r * (r + 1) / 2 > e) --r;
  i = r;
  j = (int)(e - (int64_t)r * (r + 1) / 2);
}

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

// In-place lower Cholesky A = L L^T (right-looking).  Only the lower triangle
// is read; the strict upper triangle is used as scratch (original diagonal).
// tau == 0: a non-positive or non-finite pivot sets bit 0 of status[0] and is
// replaced by 1.  tau > 0 (safeguarded form, used when the block carries FP32
// rounding): a pivot below tau * d0 is rounding noise; it is replaced by
// max(|d|, sqrt(tau) d0), which keeps the factor SPD and bounds the growth of
// the column below it (|l_ij| <= sqrt(d0_i / sqrt(tau))), and counted in
// status[1].  d0 is the pivot's original diagonal entry (or the block's
// largest original diagonal entry when that is not positive); only a block
// without a positive finite diagonal sets bit 0.  d0v, when given, holds the
// original diagonal entries (a diagonal tile of a larger matrix whose
// earlier panels have already been eliminated); the upper triangle is then
// left untouched.
// sgn (tau == 0 only): an indefinite block is factored as A = L D L^T with
// D = diag(sgn), sgn_j = +-1 (Section 5: LDL^T when A is not SPD; 1 x 1
// pivots in order, |D| split into L): a negative pivot d gives sgn_j = -1,
// l_jj = sqrt(-d), the column below divided by -l_jj and the trailing update
// A -= sgn_j l l^T; it is counted in status[4].  Only a zero or non-finite
// pivot sets bit 0.  With every pivot positive the arithmetic is that of the
// Cholesky decomposition exactly.  Returns true (in every thread) if a pivot
// was negative.
template <typename T>
__device__ bool blk_cholesky(T* A, int n, int ld, int* status, T tau = T(0), const T* d0v = nullptr,
                             T* sgn = nullptr) {
  __shared__ T s_piv, s_dmax, s_sgn;
  __shared__ int s_neg;
  if (threadIdx.x == 0) s_neg = 0;
  if (tau > T(0)) {
    if (!d0v)
      for (int j = 1 + threadIdx.x; j < n; j += blockDim.x)
        A[(int64_t)(j - 1) * ld + j] = A[(int64_t)j * ld + j];
    if (threadIdx.x == 0) {
      T dm = T(0);
      for (int j = 0; j < n; ++j) {
        const T d = d0v ? d0v[j] : A[(int64_t)j * ld + j];
        if (d > dm && isfinite((double)d)) dm = d;
      }
      s_dmax = dm;
    }
    __syncthreads();
  }
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T d = A[(int64_t)j * ld + j];
      T s = T(1);
      if (tau > T(0)) {
        T d0 = d0v ? d0v[j] : (j == 0) ? d : A[(int64_t)(j - 1) * ld + j];
        if (!(d0 > T(0)) || !isfinite((double)d0)) d0 = s_dmax;
        if (!(d0 > T(0))) {
          atomicOr(status, 1);
          d = T(1);
        } else if (!(d > tau * d0) || !isfinite((double)d)) {
          atomicAdd(status + 1, 1);
          const T floor_d = dsqrt(tau) * d0;
          d = (isfinite((double)d) && fabs((double)d) > (double)floor_d) ? (T)fabs((double)d) : floor_d;
        }
      } else if (sgn && d < T(0) && isfinite((double)d)) {
        atomicAdd(status + 4, 1);
        s = T(-1);
        d = -d;
        s_neg = 1;
      } else if (!(d > T(0)) || !isfinite((double)d)) {
        atomicOr(status, 1);
        d = T(1);
      }
      d = dsqrt(d);
      A[(int64_t)j * ld + j] = d;
      s_piv = s / d;
      s_sgn = s;
      if (sgn) sgn[j] = s;
    }
    __syncthreads();
    const T r = s_piv, sj = s_sgn;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * ld + j] *= r;
    __syncthreads();
    const int m = n - j - 1;
    const int64_t tot = (int64_t)m * (m + 1) / 2;   // lower triangle of the trailing block only
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      int a, b;
      tri_decode(e, a, b);
      const int i = j + 1 + a, k = j + 1 + b;
      A[(int64_t)i * ld + k] -= (sj * A[(int64_t)i * ld + j]) * A[(int64_t)k * ld + j];
    }
    __syncthreads();
  }
  return s_neg != 0;
}

// A = L U in place (n x n, ld), pivots in order, L unit lower (strictly below
// the diagonal) and U upper (on and above it); the two-sided elimination of
// an unsymmetric block.  A zero or non-finite pivot sets bit 0 of *status and
// is replaced by 1 (the factorization then reports the error).
template <typename T>
__device__ void blk_lu_nopivot(T* A, int n, int ld, int* status) {
  __shared__ T s_rpiv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T d = A[(int64_t)j * ld + j];
      if (d == T(0) || !isfinite((double)d)) {
        atomicOr(status, 1);
        d = T(1);
        A[(int64_t)j * ld + j] = d;
      }
      s_rpiv = T(1) / d;
    }
    __syncthreads();
    const T r = s_rpiv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * ld + j] *= r;
    __syncthreads();
    const int m = n - j - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int i = j + 1 + (int)(e / m), k = j + 1 + (int)(e % m);
      A[(int64_t)i * ld + k] -= A[(int64_t)i * ld + j] * A[(int64_t)j * ld + k];
    }
    __syncthreads();
  }
}

// X = L^{-1} for lower-triangular L (n x n).  X is written in full (zeros
// above the diagonal).  Column-oriented forward substitution on the identity.
template <typename T>
__device__ void blk_tri_inverse(const T* L, int n, int ldl, T* X, int ldx) {
  // reciprocals of the diagonal, each taken once (a division is many FP64
  // instructions, and every lane of a warp pays for it)
  constexpr int kRecip = 256;
  __shared__ T s_rinv[kRecip];
  for (int k = threadIdx.x; k < n && k < kRecip; k += blockDim.x) s_rinv[k] = T(1) / L[(int64_t)k * ldl + k];
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), c = (int)(e % n);
    X[(int64_t)i * ldx + c] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T r = k < kRecip ? s_rinv[k] : T(1) / L[(int64_t)k * ldl + k];
    for (int c = threadIdx.x; c <= k; c += blockDim.x) X[(int64_t)k * ldx + c] *= r;
    __syncthreads();
    const int m = n - k - 1;
    const int64_t tot = (int64_t)m * (k + 1);
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      const int i = k + 1 + (int)(e / (k + 1));
      const int c = (int)(e % (k + 1));
      X[(int64_t)i * ldx + c] -= L[(int64_t)i * ldl + k] * X[(int64_t)k * ldx + c];
    }
    __syncthreads();
  }
}

// C (m x n) = A (m x kk) * Linv^T, Linv lower (n x n, kk == n): C[i][j] = sum_{t<=j} A[i][t] Linv[j][t].
template <typename T>
__device__ void blk_mul_linvT(const T* A, int lda, const T* Linv, int ldl, int m, int n, T* C, int ldc) {
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const T* a = A + (int64_t)i * lda;
    const T* l = Linv + (int64_t)j * ldl;
    T s = T(0);
    for (int t = 0; t <= j; ++t) s += a[t] * l[t];
    C[(int64_t)i * ldc + j] = s;
  }
  __syncthreads();
}

// C (m x m, full symmetric) -= G diag(sgn) G^T, G m x kk (sgn NULL: all +1).
template <typename T>
__device__ void blk_syrk_sub(T* C, int ldc, const T* G, int ldg, int m, int kk, const T* sgn = nullptr) {
  const int64_t tot = (int64_t)m * (m + 1) / 2;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i, j;
    tri_decode(e, i, j);
    const T* gi = G + (int64_t)i * ldg;
    const T* gj = G + (int64_t)j * ldg;
    T s = T(0);
    if (sgn)
      for (int t = 0; t < kk; ++t) s += (gi[t] * sgn[t]) * gj[t];
    else
      for (int t = 0; t < kk; ++t) s += gi[t] * gj[t];
    const T v = C[(int64_t)i * ldc + j] - s;
    C[(int64_t)i * ldc + j] = v;
    C[(int64_t)j * ldc + i] = v;
  }
  __syncthreads();
}

// Columns of G (m x n) times sgn (G <- G diag(sgn)).
template <typename T>
__device__ void blk_scale_cols(T* G, int ldg, int m, int n, const T* sgn) {
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    G[(int64_t)i * ldg + j] *= sgn[j];
  }
  __syncthreads();
}

// Pack the lower triangle of A (n x n, ld) by rows into P.
template <typename T>
__device__ void blk_pack_lower(const T* A, int lda, T* P, int n) {
  const int64_t tot = (int64_t)n * (n + 1) / 2;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i, t;
    tri_decode(e, i, t);
    P[e] = A[(int64_t)i * lda + t];
  }
  __syncthreads();
}

template <typename T>
__device__ void blk_copy(const T* A, int lda, T* B, int ldb, int m, int n) {
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    B[(int64_t)i * ldb + j] = A[(int64_t)i * lda + j];
  }
  __syncthreads();
}

// Copy the lower triangle of A into B and zero B's strict upper triangle.
template <typename T>
__device__ void blk_copy_lower(const T* A, int lda, T* B, int ldb, int n) {
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    B[(int64_t)i * ldb + j] = (j <= i) ? A[(int64_t)i * lda + j] : T(0);
  }
  __syncthreads();
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace hif
