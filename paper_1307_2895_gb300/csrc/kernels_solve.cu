// Stencil operator and CG vector kernels (FP64).  One thread per unknown,
// all right-hand sides per thread; vectors are N x nr row-major (stride ld).
// Reductions: per-block partial sums, then the last block to finish sums the
// partials in block order (deterministic for a fixed grid).
#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"

namespace hif {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = (lane < nw) ? sh[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}

// Partials of nv values per block -> out[0..nv) by the last block.
__device__ void finish_reduce(const double* vals, int nv, double* partials, unsigned* counter,
                              double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  for (int t = 0; t < nv; ++t) {
    const double s = block_sum(vals[t], sh);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * nv + t] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int t = 0; t < nv; ++t) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += partials[(int64_t)b * nv + t];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[t] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

struct Stencil {
  GridInfo g;
  const double* a_stag;
  const double* bnode;
};

__device__ __forceinline__ double sbond(const Stencil& S, int axis, int j0, int j1, int j2) {
  const int n = S.g.n, m = S.g.m;
  if (S.g.dim == 2) {
    if (axis == 0) return S.a_stag[(int64_t)(j1 - 1) * n + j0];
    return S.a_stag[(int64_t)n * m + (int64_t)j1 * m + (j0 - 1)];
  }
  const int64_t blk = (int64_t)n * m * m;
  if (axis == 0) return S.a_stag[((int64_t)(j2 - 1) * m + (j1 - 1)) * n + j0];
  if (axis == 1) return S.a_stag[blk + ((int64_t)(j2 - 1) * n + j1) * m + (j0 - 1)];
  return S.a_stag[2 * blk + ((int64_t)j2 * m + (j1 - 1)) * m + (j0 - 1)];
}

// y = A x for one unknown g, all columns; optionally returns sum_r w_r * (x.y)_r style dots via acc.
template <int MAXR>
__device__ __forceinline__ void stencil_row(const Stencil& S, int64_t gid, const double* x, int ld,
                                            int nr, double* y) {
  const int m = S.g.m, dim = S.g.dim;
  const int j0 = (int)(gid % m) + 1;
  const int j1 = (int)((gid / m) % m) + 1;
  const int j2 = (dim == 3) ? (int)(gid / ((int64_t)m * m)) + 1 : 1;
  const double h2 = S.g.inv_h2;
  double diag = S.bnode[gid];
  for (int r = 0; r < nr; ++r) y[r] = 0.0;
  int jj[3] = {j0, j1, j2};
  int64_t stride[3] = {1, m, (int64_t)m * m};
  for (int ax = 0; ax < dim; ++ax) {
    int lo[3] = {jj[0], jj[1], jj[2]};
    lo[ax] -= 1;
    const double alo = sbond(S, ax, lo[0], lo[1], lo[2]) * h2;
    const double ahi = sbond(S, ax, jj[0], jj[1], jj[2]) * h2;
    diag += alo + ahi;
    if (jj[ax] > 1) {
      const double* xn = x + (gid - stride[ax]) * ld;
      for (int r = 0; r < nr; ++r) y[r] -= alo * xn[r];
    }
    if (jj[ax] < m) {
      const double* xn = x + (gid + stride[ax]) * ld;
      for (int r = 0; r < nr; ++r) y[r] -= ahi * xn[r];
    }
  }
  const double* xs = x + gid * ld;
  for (int r = 0; r < nr; ++r) y[r] += diag * xs[r];
}

constexpr int kMaxR = 32;

// y = A x
__global__ void k_matvec(Stencil S, int64_t N, const double* __restrict__ x, int ldx,
                         double* __restrict__ y, int ldy, int nr) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= N) return;
  double t[kMaxR];
  stencil_row<kMaxR>(S, gid, x, ldx, nr, t);
  for (int r = 0; r < nr; ++r) y[gid * ldy + r] = t[r];
}

// q = A p ; pq_r = p_r . q_r
__global__ void k_mv_dot(Stencil S, int64_t N, const double* __restrict__ p, double* __restrict__ q,
                         int nr, double* partials, unsigned* counter, double* pq) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[kMaxR];
  for (int r = 0; r < nr; ++r) vals[r] = 0.0;
  if (gid < N) {
    double t[kMaxR];
    stencil_row<kMaxR>(S, gid, p, nr, nr, t);
    for (int r = 0; r < nr; ++r) {
      q[gid * nr + r] = t[r];
      vals[r] = t[r] * p[gid * nr + r];
    }
  }
  finish_reduce(vals, nr, partials, counter, pq);
}

// alpha = rz/pq (active columns); x += alpha p; r -= alpha q; rr = r.r
__global__ void k_axpy2(int64_t N, int nr, double* __restrict__ x, double* __restrict__ r,
                        const double* __restrict__ p, const double* __restrict__ q,
                        const double* rz, const double* pq, const int* active, double* alpha_out,
                        double* partials, unsigned* counter, double* rr) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[kMaxR];
  for (int c = 0; c < nr; ++c) {
    const double a = (active[c] && pq[c] != 0.0) ? rz[c] / pq[c] : 0.0;
    if (gid == 0) alpha_out[c] = a;
    double rv = 0.0;
    if (gid < N) {
      const int64_t o = gid * nr + c;
      x[o] += a * p[o];
      rv = r[o] - a * q[o];
      r[o] = rv;
    }
    vals[c] = rv * rv;
  }
  finish_reduce(vals, nr, partials, counter, rr);
}

// rz = r.z ; zq = z.q
__global__ void k_dot2(int64_t N, int nr, const double* __restrict__ r, const double* __restrict__ z,
                       const double* __restrict__ q, double* partials, unsigned* counter, double* out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[2 * kMaxR];
  for (int c = 0; c < nr; ++c) {
    double a = 0.0, b = 0.0;
    if (gid < N) {
      const int64_t o = gid * nr + c;
      a = r[o] * z[o];
      b = z[o] * q[o];
    }
    vals[c] = a;
    vals[nr + c] = b;
  }
  finish_reduce(vals, 2 * nr, partials, counter, out);
}

// beta = -alpha zq / rz_old (flexible / Polak-Ribiere form); p = z + beta p
__global__ void k_update_p(int64_t N, int nr, double* __restrict__ p, const double* __restrict__ z,
                           const double* alpha, const double* rz_old, const double* rzzq,
                           const int* active, int restart) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= N) return;
  for (int c = 0; c < nr; ++c) {
    if (!active[c]) continue;
    const int64_t o = gid * nr + c;
    if (restart || rz_old[c] == 0.0) {
      p[o] = z[o];
    } else {
      const double beta = -alpha[c] * rzzq[nr + c] / rz_old[c];
      p[o] = z[o] + beta * p[o];
    }
  }
}

// out = b - A x (for the true residual), and its squared norms
__global__ void k_residual(Stencil S, int64_t N, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ out, int nr, double* partials, unsigned* counter,
                           double* nrm2) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[kMaxR];
  for (int r = 0; r < nr; ++r) vals[r] = 0.0;
  if (gid < N) {
    double t[kMaxR];
    stencil_row<kMaxR>(S, gid, x, nr, nr, t);
    for (int r = 0; r < nr; ++r) {
      const double v = b[gid * nr + r] - t[r];
      out[gid * nr + r] = v;
      vals[r] = v * v;
    }
  }
  finish_reduce(vals, nr, partials, counter, nrm2);
}

__global__ void k_sqnorm(int64_t N, int nr, const double* __restrict__ v, double* partials,
                         unsigned* counter, double* out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[kMaxR];
  for (int c = 0; c < nr; ++c) {
    const double a = (gid < N) ? v[gid * nr + c] : 0.0;
    vals[c] = a * a;
  }
  finish_reduce(vals, nr, partials, counter, out);
}

// ---- double-double outer iterate -------------------------------------------
// Error-free transformations (Knuth TwoSum, FMA TwoProd) with explicit
// round-to-nearest intrinsics so that no contraction changes them.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = fma(a, b, -p);
}

// r = f - A (xh + xl) in the bond form of the stencil,
//   (A x)_i = sum_e a_e n^2 (x_i - x_j) + b_i x_i  (x_j = 0 on the boundary),
// accumulated in double-double and rounded once; also sum_r |r|^2.
__global__ void k_dd_residual(Stencil S, int64_t N, const double* __restrict__ f,
                              const double* __restrict__ xh, const double* __restrict__ xl,
                              double* __restrict__ rout, int nr, double* partials,
                              unsigned* counter, double* nrm2) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double vals[kMaxR];
  for (int c = 0; c < nr; ++c) vals[c] = 0.0;
  if (gid < N) {
    const int m = S.g.m, dim = S.g.dim;
    const int jj[3] = {(int)(gid % m) + 1, (int)((gid / m) % m) + 1,
                       dim == 3 ? (int)(gid / ((int64_t)m * m)) + 1 : 1};
    const int64_t stride[3] = {1, m, (int64_t)m * m};
    const double n2 = S.g.inv_h2;   // n^2, exact for n <= 2^26
    for (int c = 0; c < nr; ++c) {
      const double xhi = xh[gid * nr + c], xli = xl[gid * nr + c];
      double sh = f[gid * nr + c], sl = 0.0;
      for (int ax = 0; ax < dim; ++ax) {
        for (int side = 0; side < 2; ++side) {
          int lo[3] = {jj[0], jj[1], jj[2]};
          if (side == 0) lo[ax] -= 1;
          const double a = sbond(S, ax, lo[0], lo[1], lo[2]);
          double wh, wl;
          two_prod(a, n2, wh, wl);
          const bool inner = side == 0 ? jj[ax] > 1 : jj[ax] < m;
          double dh, dl;
          if (inner) {
            const int64_t nb = side == 0 ? gid - stride[ax] : gid + stride[ax];
            two_sum(xhi, -xh[nb * nr + c], dh, dl);
            dl += xli - xl[nb * nr + c];
          } else {
            dh = xhi;
            dl = xli;
          }
          double ph, pl;
          two_prod(wh, dh, ph, pl);
          pl += wh * dl + wl * dh;
          double t, e;
          two_sum(sh, -ph, t, e);
          sh = t;
          sl += e - pl;
        }
      }
      {
        double ph, pl;
        two_prod(S.bnode[gid], xhi, ph, pl);
        pl += S.bnode[gid] * xli;
        double t, e;
        two_sum(sh, -ph, t, e);
        sh = t;
        sl += e - pl;
      }
      const double r = sh + sl;
      rout[gid * nr + c] = r;
      vals[c] = r * r;
    }
  }
  finish_reduce(vals, nr, partials, counter, nrm2);
}

// (xh, xl) += d for the active columns
__global__ void k_dd_add(int64_t N, int nr, double* __restrict__ xh, double* __restrict__ xl,
                         const double* __restrict__ d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nr) return;
  double s, err;
  two_sum(xh[e], d[e], s, err);
  err += xl[e];
  double hi, lo;
  two_sum(s, err, hi, lo);
  xh[e] = hi;
  xl[e] = lo;
}

// copies between a strided user layout and the packed N x nr layout, with type conversion
template <typename TI, typename TO>
__global__ void k_convert(int64_t N, int nr, const TI* __restrict__ in, int ldi, TO* __restrict__ out, int ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nr) return;
  const int64_t i = e / nr;
  const int c = (int)(e % nr);
  out[i * ldo + c] = (TO)in[i * ldi + c];
}

// active[c] = (rr[c] > thr2[c])
__global__ void k_set_active(int nr, const double* rr, const double* thr2, int* active) {
  const int c = threadIdx.x;
  if (c < nr) active[c] = rr[c] > thr2[c] ? 1 : 0;
}

// ---------------------------------------------------------------------------
static inline int nblk(int64_t n) { return (int)((n + 255) / 256); }

void launch_matvec(GridInfo g, const double* a_stag, const double* b, const double* x, int ldx,
                   double* y, int ldy, int nr, cudaStream_t st) {
  const int64_t N = (int64_t)g.m * g.m * (g.dim == 3 ? g.m : 1);
  Stencil S{g, a_stag, b};
  k_matvec<<<nblk(N), 256, 0, st>>>(S, N, x, ldx, y, ldy, nr);
}

void launch_mv_dot(GridInfo g, const double* a_stag, const double* b, const double* p, double* q,
                   int nr, double* partials, unsigned* counter, double* pq, cudaStream_t st) {
  const int64_t N = (int64_t)g.m * g.m * (g.dim == 3 ? g.m : 1);
  Stencil S{g, a_stag, b};
  k_mv_dot<<<nblk(N), 256, 0, st>>>(S, N, p, q, nr, partials, counter, pq);
}

void launch_axpy2(int64_t N, int nr, double* x, double* r, const double* p, const double* q,
                  const double* rz, const double* pq, const int* active, double* alpha,
                  double* partials, unsigned* counter, double* rr, cudaStream_t st) {
  k_axpy2<<<nblk(N), 256, 0, st>>>(N, nr, x, r, p, q, rz, pq, active, alpha, partials, counter, rr);
}

void launch_dot2(int64_t N, int nr, const double* r, const double* z, const double* q,
                 double* partials, unsigned* counter, double* out, cudaStream_t st) {
  k_dot2<<<nblk(N), 256, 0, st>>>(N, nr, r, z, q, partials, counter, out);
}

void launch_update_p(int64_t N, int nr, double* p, const double* z, const double* alpha,
                     const double* rz_old, const double* rzzq, const int* active, int restart,
                     cudaStream_t st) {
  k_update_p<<<nblk(N), 256, 0, st>>>(N, nr, p, z, alpha, rz_old, rzzq, active, restart);
}

void launch_residual(GridInfo g, const double* a_stag, const double* bn, const double* rhs,
                     const double* x, double* out, int nr, double* partials, unsigned* counter,
                     double* nrm2, cudaStream_t st) {
  const int64_t N = (int64_t)g.m * g.m * (g.dim == 3 ? g.m : 1);
  Stencil S{g, a_stag, bn};
  k_residual<<<nblk(N), 256, 0, st>>>(S, N, rhs, x, out, nr, partials, counter, nrm2);
}

void launch_sqnorm(int64_t N, int nr, const double* v, double* partials, unsigned* counter,
                   double* out, cudaStream_t st) {
  k_sqnorm<<<nblk(N), 256, 0, st>>>(N, nr, v, partials, counter, out);
}

void launch_dd_residual(GridInfo g, const double* a_stag, const double* bn, const double* f,
                        const double* xh, const double* xl, double* r, int nr, double* partials,
                        unsigned* counter, double* nrm2, cudaStream_t st) {
  const int64_t N = (int64_t)g.m * g.m * (g.dim == 3 ? g.m : 1);
  Stencil S{g, a_stag, bn};
  k_dd_residual<<<nblk(N), 256, 0, st>>>(S, N, f, xh, xl, r, nr, partials, counter, nrm2);
}

void launch_dd_add(int64_t N, int nr, double* xh, double* xl, const double* d, cudaStream_t st) {
  k_dd_add<<<nblk(N * nr), 256, 0, st>>>(N, nr, xh, xl, d);
}

void launch_set_active(int nr, const double* rr, const double* thr2, int* active, cudaStream_t st) {
  k_set_active<<<1, 32, 0, st>>>(nr, rr, thr2, active);
}

template <typename TI, typename TO>
void launch_convert(int64_t N, int nr, const TI* in, int ldi, TO* out, int ldo, cudaStream_t st) {
  k_convert<TI, TO><<<nblk(N * nr), 256, 0, st>>>(N, nr, in, ldi, out, ldo);
}
template void launch_convert<double, double>(int64_t, int, const double*, int, double*, int, cudaStream_t);
template void launch_convert<double, float>(int64_t, int, const double*, int, float*, int, cudaStream_t);
template void launch_convert<float, double>(int64_t, int, const float*, int, double*, int, cudaStream_t);

}  // namespace hif
