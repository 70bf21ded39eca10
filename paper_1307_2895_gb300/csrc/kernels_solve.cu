// Stencil operator and CG vector kernels (FP64).  Vectors are N x nr
// row-major (stride nr unless stated), nr <= 16.  Every kernel runs a fixed
// grid of grid-stride threads that keep their partial sums in registers; a
// reduction ends with a shared-memory tree per block and the last block to
// finish sums the per-block partials in block order, so results do not depend
// on scheduling.  (FP64 arithmetic is the scarce resource on this GPU: the
// cross-thread part of a reduction costs ~255 additions per block, not per
// element.)
#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"

namespace hif {

constexpr int kVecThreads = 256;

// Programmatic dependent launch of the CG vector kernels: a kernel waits for
// its predecessor in the stream to complete (and its writes to be visible)
// before it reads anything, then lets its own successor launch, so that the
// successor's launch overlaps this kernel instead of following it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

static inline int vec_blocks(int64_t n) {
  const int64_t b = (n + kVecThreads - 1) / kVecThreads;
  return (int)(b < kVecBlocksMax ? (b > 0 ? b : 1) : kVecBlocksMax);
}

// In the last block: out[v] = sum over blocks b (in block order within each
// thread's stride, then a fixed tree) of partials[b * nv + v].  Every thread
// takes value v = tid % nv and the blocks b = tid / nv + k * (blockDim / nv),
// so the partials are read with many loads in flight.  nv <= blockDim.x.
__device__ void last_block_sum(const double* partials, int nv, double* shr, double* out) {
  const int tid = threadIdx.x;
  const int lanes = blockDim.x / nv;           // threads per value
  double s = 0.0;
  if (tid < lanes * nv) {
    const int v = tid % nv;
    for (int b = tid / nv; b < (int)gridDim.x; b += lanes) s += partials[(int64_t)b * nv + v];
  }
  __syncthreads();
  shr[tid] = s;
  __syncthreads();
  for (int step = lanes >> 1; step > 0; step >>= 1) {
    if (tid < step * nv) shr[tid] += shr[tid + step * nv];
    __syncthreads();
  }
  if (tid < nv) out[tid] = shr[tid];
}

// Sum acc[0..nv) over the grid into out[0..nv).  Needs nv*blockDim.x doubles
// of dynamic shared memory.
template <int NV>
__device__ void grid_reduce(const double (&acc)[NV], int nv, double* partials, unsigned* counter,
                            double* out) {
  extern __shared__ double shr[];
  __shared__ bool last;
  const int tid = threadIdx.x;
  for (int v = 0; v < nv; ++v) shr[tid * nv + v] = acc[v];
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (tid < s)
      for (int v = 0; v < nv; ++v) shr[tid * nv + v] += shr[(tid + s) * nv + v];
    __syncthreads();
  }
  if (tid < nv) partials[(int64_t)blockIdx.x * nv + tid] = shr[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  last_block_sum(partials, nv, shr, out);
  if (tid == 0) *counter = 0u;
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

// y[0..R) = (A x)_gid for the columns r < nr of x (row stride ld).
template <int R>
__device__ __forceinline__ void stencil_row(const Stencil& S, int64_t gid, const double* x, int ld,
                                            int nr, double (&y)[R]) {
  const int m = S.g.m, dim = S.g.dim;
  const int jj[3] = {(int)(gid % m) + 1, (int)((gid / m) % m) + 1,
                     dim == 3 ? (int)(gid / ((int64_t)m * m)) + 1 : 1};
  const int64_t stride[3] = {1, m, (int64_t)m * m};
  const double h2 = S.g.inv_h2;
  double diag = S.bnode[gid];
#pragma unroll
  for (int r = 0; r < R; ++r) y[r] = 0.0;
  for (int ax = 0; ax < dim; ++ax) {
    int lo[3] = {jj[0], jj[1], jj[2]};
    lo[ax] -= 1;
    const double alo = sbond(S, ax, lo[0], lo[1], lo[2]) * h2;
    const double ahi = sbond(S, ax, jj[0], jj[1], jj[2]) * h2;
    diag += alo + ahi;
    if (jj[ax] > 1) {
      const double* xn = x + (gid - stride[ax]) * ld;
#pragma unroll
      for (int r = 0; r < R; ++r) if (r < nr) y[r] -= alo * xn[r];
    }
    if (jj[ax] < m) {
      const double* xn = x + (gid + stride[ax]) * ld;
#pragma unroll
      for (int r = 0; r < R; ++r) if (r < nr) y[r] -= ahi * xn[r];
    }
  }
  const double* xs = x + gid * ld;
#pragma unroll
  for (int r = 0; r < R; ++r) if (r < nr) y[r] += diag * xs[r];
}

#define GRID_LOOP(gid, N) for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < (N); \
                               gid += (int64_t)gridDim.x * blockDim.x)

// y = A x (strided)
template <int R>
__global__ void k_matvec(Stencil S, int64_t N, const double* __restrict__ x, int ldx,
                         double* __restrict__ y, int ldy, int nr) {
  GRID_LOOP(gid, N) {
    double t[R];
    stencil_row<R>(S, gid, x, ldx, nr, t);
#pragma unroll
    for (int r = 0; r < R; ++r) if (r < nr) y[gid * ldy + r] = t[r];
  }
}

// q = A p ; pq_r = p_r . q_r
template <int R>
__global__ void k_mv_dot(Stencil S, int64_t N, const double* __restrict__ p, double* __restrict__ q,
                         int nr, double* partials, unsigned* counter, double* pq) {
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  GRID_LOOP(gid, N) {
    double t[R];
    stencil_row<R>(S, gid, p, nr, nr, t);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < nr) {
        q[gid * nr + r] = t[r];
        acc[r] = fma(t[r], p[gid * nr + r], acc[r]);
      }
  }
  grid_reduce<R>(acc, nr, partials, counter, pq);
}

// alpha = rz/pq (active columns); x += alpha p; r -= alpha q; rr = r.r
template <int R>
__global__ void k_axpy2(int64_t N, int nr, double* __restrict__ x, double* __restrict__ r,
                        const double* __restrict__ p, const double* __restrict__ q,
                        const double* rz, const double* pq, const int* active, double* alpha_out,
                        double* partials, unsigned* counter, double* rr) {
  double a[R], acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) {
    a[c] = (c < nr && active[c] && pq[c] != 0.0) ? rz[c] / pq[c] : 0.0;
    acc[c] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x < nr) {
    const int c = threadIdx.x;
    alpha_out[c] = (active[c] && pq[c] != 0.0) ? rz[c] / pq[c] : 0.0;
  }
  GRID_LOOP(gid, N) {
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (c < nr) {
        const int64_t o = gid * nr + c;
        x[o] = fma(a[c], p[o], x[o]);
        const double rv = fma(-a[c], q[o], r[o]);
        r[o] = rv;
        acc[c] = fma(rv, rv, acc[c]);
      }
  }
  grid_reduce<R>(acc, nr, partials, counter, rr);
}

// rz = r.z ; zq = z.q   (out = [rz(0..nr) | zq(0..nr)])
template <int R>
__global__ void k_dot2(int64_t N, int nr, const double* __restrict__ r, const double* __restrict__ z,
                       const double* __restrict__ q, double* partials, unsigned* counter, double* out) {
  double acc[2 * R];
#pragma unroll
  for (int c = 0; c < 2 * R; ++c) acc[c] = 0.0;
  GRID_LOOP(gid, N) {
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (c < nr) {
        const int64_t o = gid * nr + c;
        const double zv = z[o];
        acc[c] = fma(r[o], zv, acc[c]);
        acc[R + c] = fma(zv, q[o], acc[R + c]);
      }
  }
  double packed[2 * R];
#pragma unroll
  for (int c = 0; c < 2 * R; ++c) packed[c] = 0.0;
#pragma unroll
  for (int c = 0; c < R; ++c)
    if (c < nr) {
      packed[c] = acc[c];
      packed[nr + c] = acc[R + c];
    }
  grid_reduce<2 * R>(packed, 2 * nr, partials, counter, out);
}

// beta = -alpha zq / rz_old (flexible / Polak-Ribiere form); p = z + beta p
template <int R>
__global__ void k_update_p(int64_t N, int nr, double* __restrict__ p, const double* __restrict__ z,
                           const double* alpha, const double* rz_old, const double* rzzq,
                           const int* active, int restart) {
  double beta[R];
  bool act[R], rs[R];
#pragma unroll
  for (int c = 0; c < R; ++c) {
    act[c] = c < nr && active[c];
    rs[c] = restart || (c < nr && rz_old[c] == 0.0);
    beta[c] = (c < nr && !rs[c]) ? -alpha[c] * rzzq[nr + c] / rz_old[c] : 0.0;
  }
  GRID_LOOP(gid, N) {
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (act[c]) {
        const int64_t o = gid * nr + c;
        p[o] = rs[c] ? z[o] : fma(beta[c], p[o], z[o]);
      }
  }
}

// out = b - A x (FP64) and its squared norms
template <int R>
__global__ void k_residual(Stencil S, int64_t N, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ out, int nr, double* partials, unsigned* counter,
                           double* nrm2) {
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  GRID_LOOP(gid, N) {
    double t[R];
    stencil_row<R>(S, gid, x, nr, nr, t);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < nr) {
        const double v = b[gid * nr + r] - t[r];
        out[gid * nr + r] = v;
        acc[r] = fma(v, v, acc[r]);
      }
  }
  grid_reduce<R>(acc, nr, partials, counter, nrm2);
}

template <int R>
__global__ void k_sqnorm(int64_t N, int nr, const double* __restrict__ v, double* partials,
                         unsigned* counter, double* out) {
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  GRID_LOOP(gid, N) {
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (c < nr) {
        const double a = v[gid * nr + c];
        acc[c] = fma(a, a, acc[c]);
      }
  }
  grid_reduce<R>(acc, nr, partials, counter, out);
}

// ---- element-parallel CG kernels ------------------------------------------
// One thread per (unknown, column) element e = i * R + c of an N x R vector
// (R a power of two, so a grid-stride thread keeps one column); reductions
// sum threads of equal column in a shared-memory tree, then across blocks.
// Returns true in the last block, after out[] is written and visible to the
// whole block (its threads may then act on the sums).
template <int R, int NG>
__device__ bool grid_reduce_cols(const double (&acc)[NG], double* partials, unsigned* counter,
                                 double* out) {
  __shared__ double shr[NG][kVecThreads];
  __shared__ bool last;
  const int tid = threadIdx.x;
#pragma unroll
  for (int g = 0; g < NG; ++g) shr[g][tid] = acc[g];
  __syncthreads();
  for (int s = blockDim.x >> 1; s >= R; s >>= 1) {
    if (tid < s)
#pragma unroll
      for (int g = 0; g < NG; ++g) shr[g][tid] += shr[g][tid + s];
    __syncthreads();
  }
  if (tid < R)
#pragma unroll
    for (int g = 0; g < NG; ++g) partials[((int64_t)blockIdx.x * NG + g) * R + tid] = shr[g][tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  last_block_sum(partials, NG * R, &shr[0][0], out);
  if (tid == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// Stencil weights, computed once per problem: W[i*S + 0] = diagonal,
// W[i*S + 1 + 2*axis + side] = coupling to the neighbour below (side 0) or
// above (side 1) along axis (0 when that neighbour is a boundary node),
// S = 2 dim + 1.
__global__ void k_stencil_weights(Stencil S, int64_t N, double* __restrict__ W) {
  const int m = S.g.m, dim = S.g.dim, ns = 2 * dim + 1;
  const double h2 = S.g.inv_h2;
  GRID_LOOP(gid, N) {
    const int jj[3] = {(int)(gid % m) + 1, (int)((gid / m) % m) + 1,
                       dim == 3 ? (int)(gid / ((int64_t)m * m)) + 1 : 1};
    double diag = S.bnode[gid];
    for (int ax = 0; ax < dim; ++ax) {
      int lo[3] = {jj[0], jj[1], jj[2]};
      lo[ax] -= 1;
      const double alo = sbond(S, ax, lo[0], lo[1], lo[2]) * h2;
      const double ahi = sbond(S, ax, jj[0], jj[1], jj[2]) * h2;
      diag += alo + ahi;
      W[gid * ns + 1 + 2 * ax] = jj[ax] > 1 ? -alo : 0.0;
      W[gid * ns + 2 + 2 * ax] = jj[ax] < m ? -ahi : 0.0;
    }
    W[gid * ns] = diag;
  }
}

// Widening float -> double on the integer pipes (exact for normal numbers,
// zeros, infinities and NaNs; subnormals take the hardware conversion).  On
// this GPU the FP64 pipe is the narrow one, and the CG vector kernels spend
// most of their time on it.
template <typename TZ>
__device__ __forceinline__ double widen(TZ v) { return (double)v; }
template <>
__device__ __forceinline__ double widen<float>(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u && (u & 0x7fffffu)) return (double)v;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
  unsigned long long ex;
  if (e == 0u) ex = 0ull;
  else if (e == 0xffu) ex = 0x7ffull;
  else ex = (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sgn | (ex << 52) | man));
}

// Narrowing double -> TZ; for float, round-to-nearest-even on the integer
// pipes when the result is a normal float (the same value as the hardware
// conversion), the hardware conversion otherwise (zero, subnormal, overflow,
// infinity, NaN).
template <typename TZ>
__device__ __forceinline__ TZ narrow(double v) { return (TZ)v; }
template <>
__device__ __forceinline__ float narrow<float>(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
  if (e < 897u || e > 1150u) return (float)v;          // float exponent outside 1..254
  const unsigned long long man = u & 0xFFFFFFFFFFFFFull;
  unsigned m = (unsigned)(man >> 29);
  const unsigned rem = (unsigned)(man & 0x1FFFFFFFull), half = 0x10000000u;
  if (rem > half || (rem == half && (m & 1u))) ++m;
  unsigned fe = e - 896u;
  if (m == 0x800000u) {                                 // the rounding carried into the exponent
    m = 0u;
    ++fe;
  }
  if (fe >= 255u) return (float)v;                      // rounds to infinity
  return __uint_as_float(((unsigned)(u >> 63) << 31) | (fe << 23) | m);
}

// (A x)[e] for element e = gid * R + c from the weights (boundary neighbours
// have weight +0.0 exactly and are read at the node itself; the test is on
// the bits, off the FP64 pipe)
template <int R, int DIM>
__device__ __forceinline__ double stencil_w(const double* __restrict__ W, int m, int64_t gid, int c,
                                            const double* __restrict__ x) {
  constexpr int ns = 2 * DIM + 1;
  const double* w = W + gid * ns;
  const int64_t stride[3] = {1, m, (int64_t)m * m};
  double y = w[0] * x[gid * R + c];
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const int64_t lo = __double_as_longlong(w[1 + 2 * ax]) != 0 ? gid - stride[ax] : gid;
    const int64_t hi = __double_as_longlong(w[2 + 2 * ax]) != 0 ? gid + stride[ax] : gid;
    y = fma(w[1 + 2 * ax], x[lo * R + c], y);
    y = fma(w[2 + 2 * ax], x[hi * R + c], y);
  }
  return y;
}

// q = A p and pq = p.q per column; with alpha_out, the last block also sets
// alpha = rz / pq on the active columns (0 elsewhere), once per column, so
// that the update kernel divides nothing (FP64 division is a long sequence
// on this GPU's narrow FP64 pipe).
template <int R, int DIM>
__global__ void k_mv_dot_e(const double* __restrict__ W, int m, int64_t N, const double* __restrict__ p,
                           double* __restrict__ q, double* partials, unsigned* counter, double* pq,
                           const double* rz, const int* active, double* alpha_out) {
  pdl_enter();
  double acc[1] = {0.0};
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t eu = e + u * stride;
      v[u] = stencil_w<R, DIM>(W, m, eu / R, (int)(eu % R), p);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      q[e + u * stride] = v[u];
      acc[0] = fma(v[u], p[e + u * stride], acc[0]);
    }
  }
  for (; e < n; e += stride) {
    const double v = stencil_w<R, DIM>(W, m, e / R, (int)(e % R), p);
    q[e] = v;
    acc[0] = fma(v, p[e], acc[0]);
  }
  if (grid_reduce_cols<R, 1>(acc, partials, counter, pq) && alpha_out && threadIdx.x < R) {
    const int c = threadIdx.x;
    alpha_out[c] = (active[c] && pq[c] != 0.0) ? rz[c] / pq[c] : 0.0;
  }
}

// x += alpha p; r -= alpha q (alpha from k_mv_dot_e, 0 on frozen columns);
// rr = r.r; zin = (TZ) r
template <int R, typename TZ>
__global__ void k_axpy2_e(int64_t N, double* __restrict__ x, double* __restrict__ r,
                          const double* __restrict__ p, const double* __restrict__ q, const double* alpha,
                          double* partials, unsigned* counter, double* rr, TZ* __restrict__ zin,
                          const double* thr2, int* active_next, double* ring_rr) {
  pdl_enter();
  const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % R);
  const double a = alpha[c];
  double acc[1] = {0.0};
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    double xv[4], pv[4], qv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xv[u] = x[e + u * stride];
      pv[u] = p[e + u * stride];
      qv[u] = q[e + u * stride];
      rv[u] = r[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[e + u * stride] = fma(a, pv[u], xv[u]);
      const double rn = fma(-a, qv[u], rv[u]);
      r[e + u * stride] = rn;
      zin[e + u * stride] = narrow<TZ>(rn);
      acc[0] = fma(rn, rn, acc[0]);
    }
  }
  for (; e < n; e += stride) {
    x[e] = fma(a, p[e], x[e]);
    const double rv = fma(-a, q[e], r[e]);
    r[e] = rv;
    zin[e] = narrow<TZ>(rv);
    acc[0] = fma(rv, rv, acc[0]);
  }
  // the last block (every block has read active[] by then): the columns still
  // above their threshold, and the sums for the host's ring (mapped memory)
  if (grid_reduce_cols<R, 1>(acc, partials, counter, rr) && threadIdx.x < R) {
    const int cc = threadIdx.x;
    if (active_next) active_next[cc] = rr[cc] > thr2[cc] ? 1 : 0;
    if (ring_rr) {
      ring_rr[cc] = rr[cc];
      __threadfence_system();
    }
  }
}

// out = [r.z | z.q]; the last block also sets beta = -alpha zq / rz_old per
// column (the flexible / Polak-Ribiere form; 0 where rz_old is 0)
template <int R, typename TZ>
__global__ void k_dot2_e(int64_t N, const double* __restrict__ r, const TZ* __restrict__ z,
                         const double* __restrict__ q, double* partials, unsigned* counter, double* out,
                         double* ring_rz, const double* alpha, const double* rz_old, double* beta_out) {
  pdl_enter();
  double acc[2] = {0.0, 0.0};
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    double rv[4], zv[4], qv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rv[u] = r[e + u * stride];
      zv[u] = widen<TZ>(z[e + u * stride]);
      qv[u] = q[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[0] = fma(rv[u], zv[u], acc[0]);
      acc[1] = fma(zv[u], qv[u], acc[1]);
    }
  }
  for (; e < n; e += stride) {
    const double zv = widen<TZ>(z[e]);
    acc[0] = fma(r[e], zv, acc[0]);
    acc[1] = fma(zv, q[e], acc[1]);
  }
  if (grid_reduce_cols<R, 2>(acc, partials, counter, out) && threadIdx.x < R) {
    const int c = threadIdx.x;
    beta_out[c] = rz_old[c] != 0.0 ? -alpha[c] * out[R + c] / rz_old[c] : 0.0;
    if (ring_rz) {
      ring_rz[c] = out[c];   // r.z for the host's breakdown check
      __threadfence_system();
    }
  }
}

// p = z + beta p (beta from k_dot2_e; p = z on a restart)
template <int R, typename TZ>
__global__ void k_update_p_e(int64_t N, double* __restrict__ p, const TZ* __restrict__ z,
                             const double* betav, const double* rz_old, const int* active, int restart) {
  pdl_enter();
  const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % R);
  if (!active[c]) return;
  const bool rs = restart || rz_old[c] == 0.0;
  const double beta = rs ? 0.0 : betav[c];
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    double zv[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zv[u] = widen<TZ>(z[e + u * stride]);
      pv[u] = p[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[e + u * stride] = rs ? zv[u] : fma(beta, pv[u], zv[u]);
  }
  for (; e < n; e += stride) {
    const double zv = widen<TZ>(z[e]);
    p[e] = rs ? zv : fma(beta, p[e], zv);
  }
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
template <int R>
__global__ void k_dd_residual(Stencil S, int64_t N, const double* __restrict__ f,
                              const double* __restrict__ xh, const double* __restrict__ xl,
                              double* __restrict__ rout, int nr, double* partials,
                              unsigned* counter, double* nrm2) {
  double acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = 0.0;
  const int m = S.g.m, dim = S.g.dim;
  const int64_t stride[3] = {1, m, (int64_t)m * m};
  const double n2 = S.g.inv_h2;   // n^2, exact for n <= 2^26
  GRID_LOOP(gid, N) {
    const int jj[3] = {(int)(gid % m) + 1, (int)((gid / m) % m) + 1,
                       dim == 3 ? (int)(gid / ((int64_t)m * m)) + 1 : 1};
    double sh[R], sl[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      sh[c] = c < nr ? f[gid * nr + c] : 0.0;
      sl[c] = 0.0;
    }
    for (int ax = 0; ax < dim; ++ax) {
      for (int side = 0; side < 2; ++side) {
        int lo[3] = {jj[0], jj[1], jj[2]};
        if (side == 0) lo[ax] -= 1;
        const double a = sbond(S, ax, lo[0], lo[1], lo[2]);
        double wh, wl;
        two_prod(a, n2, wh, wl);
        const bool inner = side == 0 ? jj[ax] > 1 : jj[ax] < m;
        const int64_t nb = side == 0 ? gid - stride[ax] : gid + stride[ax];
#pragma unroll
        for (int c = 0; c < R; ++c) {
          if (c >= nr) continue;
          const double xhi = xh[gid * nr + c], xli = xl[gid * nr + c];
          double dh, dl;
          if (inner) {
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
          two_sum(sh[c], -ph, t, e);
          sh[c] = t;
          sl[c] += e - pl;
        }
      }
    }
    const double bv = S.bnode[gid];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      if (c >= nr) continue;
      const double xhi = xh[gid * nr + c], xli = xl[gid * nr + c];
      double ph, pl;
      two_prod(bv, xhi, ph, pl);
      pl += bv * xli;
      double t, e;
      two_sum(sh[c], -ph, t, e);
      const double r = t + (sl[c] + e - pl);
      rout[gid * nr + c] = r;
      acc[c] = fma(r, r, acc[c]);
    }
  }
  grid_reduce<R>(acc, nr, partials, counter, nrm2);
}

// (xh, xl) += d
__global__ void k_dd_add(int64_t N, int nr, double* __restrict__ xh, double* __restrict__ xl,
                         const double* __restrict__ d) {
  GRID_LOOP(e, N * nr) {
    double s, err;
    two_sum(xh[e], d[e], s, err);
    err += xl[e];
    double hi, lo;
    two_sum(s, err, hi, lo);
    xh[e] = hi;
    xl[e] = lo;
  }
}

// copies between a strided user layout and the packed N x nr layout, with type conversion
template <typename TI, typename TO>
__global__ void k_convert(int64_t N, int nr, const TI* __restrict__ in, int ldi, TO* __restrict__ out, int ldo) {
  GRID_LOOP(e, N * nr) {
    const int64_t i = e / nr;
    const int c = (int)(e % nr);
    out[i * ldo + c] = (TO)in[i * ldi + c];
  }
}

// active[c] = (rr[c] > thr2[c])
__global__ void k_set_active(int nr, const double* rr, const double* thr2, int* active) {
  const int c = threadIdx.x;
  if (c < nr) active[c] = rr[c] > thr2[c] ? 1 : 0;
}

// ---------------------------------------------------------------------------
static inline int64_t grid_n(GridInfo g) { return (int64_t)g.m * g.m * (g.dim == 3 ? g.m : 1); }

template <typename K>
static void set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) raise_smem_limit(kern);
}

#define DISPATCH_R(nr, ...)                                     \
  do {                                                          \
    if ((nr) <= 1) { constexpr int R = 1; __VA_ARGS__; }        \
    else if ((nr) <= 2) { constexpr int R = 2; __VA_ARGS__; }   \
    else if ((nr) <= 4) { constexpr int R = 4; __VA_ARGS__; }   \
    else if ((nr) <= 8) { constexpr int R = 8; __VA_ARGS__; }   \
    else { constexpr int R = 16; __VA_ARGS__; }                 \
  } while (0)

void launch_matvec(GridInfo g, const double* a_stag, const double* b, const double* x, int ldx,
                   double* y, int ldy, int nr, cudaStream_t st) {
  const int64_t N = grid_n(g);
  Stencil S{g, a_stag, b};
  for (int r0 = 0; r0 < nr; r0 += 16) {
    const int c = nr - r0 < 16 ? nr - r0 : 16;
    note_launches(1);
    DISPATCH_R(c, k_matvec<R><<<vec_blocks(N), kVecThreads, 0, st>>>(S, N, x + r0, ldx, y + r0, ldy, c));
  }
}

void launch_mv_dot(GridInfo g, const double* a_stag, const double* b, const double* p, double* q,
                   int nr, double* partials, unsigned* counter, double* pq, cudaStream_t st) {
  const int64_t N = grid_n(g);
  Stencil S{g, a_stag, b};
  const size_t smem = sizeof(double) * kVecThreads * nr;
  DISPATCH_R(nr, set_smem(k_mv_dot<R>, smem); note_launches(1);
                  k_mv_dot<R><<<vec_blocks(N), kVecThreads, smem, st>>>(S, N, p, q, nr, partials, counter, pq));
}

void launch_axpy2(int64_t N, int nr, double* x, double* r, const double* p, const double* q,
                  const double* rz, const double* pq, const int* active, double* alpha,
                  double* partials, unsigned* counter, double* rr, cudaStream_t st) {
  const size_t smem = sizeof(double) * kVecThreads * nr;
  DISPATCH_R(nr, set_smem(k_axpy2<R>, smem); note_launches(1);
                  k_axpy2<R><<<vec_blocks(N), kVecThreads, smem, st>>>(N, nr, x, r, p, q, rz, pq, active,
                                                                     alpha, partials, counter, rr));
}

void launch_dot2(int64_t N, int nr, const double* r, const double* z, const double* q,
                 double* partials, unsigned* counter, double* out, cudaStream_t st) {
  const size_t smem = sizeof(double) * kVecThreads * 2 * nr;
  DISPATCH_R(nr, set_smem(k_dot2<R>, smem); note_launches(1);
                  k_dot2<R><<<vec_blocks(N), kVecThreads, smem, st>>>(N, nr, r, z, q, partials, counter, out));
}

void launch_update_p(int64_t N, int nr, double* p, const double* z, const double* alpha,
                     const double* rz_old, const double* rzzq, const int* active, int restart,
                     cudaStream_t st) {
  note_launches(1);
  DISPATCH_R(nr, k_update_p<R><<<vec_blocks(N), kVecThreads, 0, st>>>(N, nr, p, z, alpha, rz_old, rzzq,
                                                                     active, restart));
}

void launch_residual(GridInfo g, const double* a_stag, const double* bn, const double* rhs,
                     const double* x, double* out, int nr, double* partials, unsigned* counter,
                     double* nrm2, cudaStream_t st) {
  const int64_t N = grid_n(g);
  Stencil S{g, a_stag, bn};
  const size_t smem = sizeof(double) * kVecThreads * nr;
  DISPATCH_R(nr, set_smem(k_residual<R>, smem); note_launches(1);
                  k_residual<R><<<vec_blocks(N), kVecThreads, smem, st>>>(S, N, rhs, x, out, nr, partials,
                                                                        counter, nrm2));
}

void launch_sqnorm(int64_t N, int nr, const double* v, double* partials, unsigned* counter,
                   double* out, cudaStream_t st) {
  const size_t smem = sizeof(double) * kVecThreads * nr;
  DISPATCH_R(nr, set_smem(k_sqnorm<R>, smem); note_launches(1);
                  k_sqnorm<R><<<vec_blocks(N), kVecThreads, smem, st>>>(N, nr, v, partials, counter, out));
}

void launch_dd_residual(GridInfo g, const double* a_stag, const double* bn, const double* f,
                        const double* xh, const double* xl, double* r, int nr, double* partials,
                        unsigned* counter, double* nrm2, cudaStream_t st) {
  const int64_t N = grid_n(g);
  Stencil S{g, a_stag, bn};
  const size_t smem = sizeof(double) * kVecThreads * nr;
  DISPATCH_R(nr, set_smem(k_dd_residual<R>, smem); note_launches(1);
                  k_dd_residual<R><<<vec_blocks(N), kVecThreads, smem, st>>>(S, N, f, xh, xl, r, nr, partials,
                                                                           counter, nrm2));
}

void launch_dd_add(int64_t N, int nr, double* xh, double* xl, const double* d, cudaStream_t st) {
  note_launches(1);
  k_dd_add<<<vec_blocks(N * nr), kVecThreads, 0, st>>>(N, nr, xh, xl, d);
}

#define DISPATCH_POW2(R_, ...)                                  \
  do {                                                          \
    switch (R_) {                                               \
      case 1: { constexpr int R = 1; __VA_ARGS__; } break;      \
      case 2: { constexpr int R = 2; __VA_ARGS__; } break;      \
      case 4: { constexpr int R = 4; __VA_ARGS__; } break;      \
      case 8: { constexpr int R = 8; __VA_ARGS__; } break;      \
      default: { constexpr int R = 16; __VA_ARGS__; } break;    \
    }                                                           \
  } while (0)

static inline int elem_blocks(int64_t n) {
  // grid-stride threads; a multiple of every R in {1,..,16} by construction (256 per block)
  return vec_blocks(n);
}

void launch_stencil_weights(GridInfo g, const double* a_stag, const double* b, double* W, cudaStream_t st) {
  const int64_t N = grid_n(g);
  Stencil S{g, a_stag, b};
  note_launches(1);
  k_stencil_weights<<<vec_blocks(N), kVecThreads, 0, st>>>(S, N, W);
}

void launch_mv_dot_e(GridInfo g, const double* W, const double* p, double* q, int R_, double* partials,
                     unsigned* counter, double* pq, cudaStream_t st, const double* rz, const int* active,
                     double* alpha) {
  const int64_t N = grid_n(g);
  note_launches(1);
  if (g.dim == 2)
    DISPATCH_POW2(R_, (launch_pdl(k_mv_dot_e<R, 2>, elem_blocks(N * R), kVecThreads, st, W, g.m, N, p, q,
                                  partials, counter, pq, rz, active, alpha)));
  else
    DISPATCH_POW2(R_, (launch_pdl(k_mv_dot_e<R, 3>, elem_blocks(N * R), kVecThreads, st, W, g.m, N, p, q,
                                  partials, counter, pq, rz, active, alpha)));
}

template <typename TZ>
void launch_axpy2_e(int64_t N, int R_, double* x, double* r, const double* p, const double* q,
                    const double* alpha, double* partials, unsigned* counter, double* rr, TZ* zin, cudaStream_t st,
                    const double* thr2, int* active_next, double* ring_rr) {
  note_launches(1);
  DISPATCH_POW2(R_, launch_pdl(k_axpy2_e<R, TZ>, elem_blocks(N * R), kVecThreads, st, N, x, r, p, q, alpha,
                               partials, counter, rr, zin, thr2, active_next, ring_rr));
}

template <typename TZ>
void launch_dot2_e(int64_t N, int R_, const double* r, const TZ* z, const double* q, double* partials,
                   unsigned* counter, double* out, cudaStream_t st, double* ring_rz, const double* alpha,
                   const double* rz_old, double* beta) {
  note_launches(1);
  DISPATCH_POW2(R_, launch_pdl(k_dot2_e<R, TZ>, elem_blocks(N * R), kVecThreads, st, N, r, z, q, partials,
                               counter, out, ring_rz, alpha, rz_old, beta));
}

template <typename TZ>
void launch_update_p_e(int64_t N, int R_, double* p, const TZ* z, const double* beta, const double* rz_old,
                       const int* active, int restart, cudaStream_t st) {
  note_launches(1);
  DISPATCH_POW2(R_, launch_pdl(k_update_p_e<R, TZ>, elem_blocks(N * R), kVecThreads, st, N, p, z, beta, rz_old,
                               active, restart));
}

template void launch_axpy2_e<double>(int64_t, int, double*, double*, const double*, const double*,
                                     const double*, double*, unsigned*, double*, double*, cudaStream_t,
                                     const double*, int*, double*);
template void launch_axpy2_e<float>(int64_t, int, double*, double*, const double*, const double*,
                                    const double*, double*, unsigned*, double*, float*, cudaStream_t,
                                    const double*, int*, double*);
template void launch_dot2_e<double>(int64_t, int, const double*, const double*, const double*, double*,
                                    unsigned*, double*, cudaStream_t, double*, const double*, const double*,
                                    double*);
template void launch_dot2_e<float>(int64_t, int, const double*, const float*, const double*, double*,
                                   unsigned*, double*, cudaStream_t, double*, const double*, const double*,
                                   double*);
template void launch_update_p_e<double>(int64_t, int, double*, const double*, const double*, const double*,
                                        const int*, int, cudaStream_t);
template void launch_update_p_e<float>(int64_t, int, double*, const float*, const double*, const double*,
                                       const int*, int, cudaStream_t);

void launch_set_active(int nr, const double* rr, const double* thr2, int* active, cudaStream_t st) {
  note_launches(1);
  k_set_active<<<1, 32, 0, st>>>(nr, rr, thr2, active);
}

template <typename TI, typename TO>
void launch_convert(int64_t N, int nr, const TI* in, int ldi, TO* out, int ldo, cudaStream_t st) {
  note_launches(1);
  k_convert<TI, TO><<<vec_blocks(N * nr), kVecThreads, 0, st>>>(N, nr, in, ldi, out, ldo);
}
// ---- flexible GMRES (Arnoldi with classical Gram-Schmidt, twice) ----------
// Basis slabs: V_i = V + i * slab (N x R, FP64), Z_i = Z + i * slab (the
// preconditioner's type).  Each column c is an independent GMRES.

// out[i * R + c] = <V_i(:, c), w(:, c)> for i = blockIdx.y; per-i partials and
// counters, summed by the last block of each i in block order.
template <int R>
__global__ void k_multi_dot(int64_t N, const double* __restrict__ V, int64_t slab, const double* __restrict__ w,
                            double* partials, unsigned* counters, double* out) {
  __shared__ double shr[kVecThreads];
  __shared__ bool last;
  const int i = blockIdx.y;
  const double* v = V + (int64_t)i * slab;
  double acc = 0.0;
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) acc = fma(v[e], w[e], acc);
  const int tid = threadIdx.x;
  shr[tid] = acc;
  __syncthreads();
  for (int s = blockDim.x >> 1; s >= R; s >>= 1) {
    if (tid < s) shr[tid] += shr[tid + s];
    __syncthreads();
  }
  double* part = partials + (int64_t)i * gridDim.x * R;
  if (tid < R) part[(int64_t)blockIdx.x * R + tid] = shr[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(counters + i, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  last_block_sum(part, R, shr, out + (int64_t)i * R);
  if (tid == 0) counters[i] = 0u;
}

// w -= sum_{i < nv} h[i * R + c] V_i(:, c)
template <int R>
__global__ void k_multi_axpy(int64_t N, const double* __restrict__ V, int64_t slab, int nv,
                             const double* __restrict__ h, double* __restrict__ w) {
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int c = (int)(e % R);
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s = fma(h[i * R + c], V[(int64_t)i * slab + e], s);
    w[e] -= s;
  }
}

// v = w / ||w|| per column from nrm2 (a zero column stays zero); hnorm[c] =
// ||w(:, c)|| when hnorm is not null
template <int R>
__global__ void k_normalize(int64_t N, const double* __restrict__ w, const double* __restrict__ nrm2,
                            double* __restrict__ v, double* hnorm) {
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = (int)(e % R);   // fixed per thread: the stride is a multiple of R
  const double nr = sqrt(nrm2[c]);
  const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
  if (hnorm && blockIdx.x == 0 && threadIdx.x < R) hnorm[threadIdx.x] = sqrt(nrm2[threadIdx.x]);
  for (; e < n; e += stride) v[e] = w[e] * inv;
}

// d += sum_{i < nv} y[i * R + c] Z_i(:, c)
template <int R, typename TZ>
__global__ void k_zy_add(int64_t N, const TZ* __restrict__ Z, int64_t slab, int nv, const double* __restrict__ y,
                         double* __restrict__ d) {
  const int64_t n = N * R, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int c = (int)(e % R);
    double s = d[e];
    for (int i = 0; i < nv; ++i) s = fma(y[i * R + c], widen<TZ>(Z[(int64_t)i * slab + e]), s);
    d[e] = s;
  }
}

static inline int gmres_blocks(int64_t n) {
  // a multiple of every R in {1,..,16} (256 threads per block); 2 blocks per SM
  // for the reductions, which run one grid row per basis vector
  const int64_t b = (n + kVecThreads - 1) / kVecThreads;
  return (int)(b < 304 ? (b > 0 ? b : 1) : 304);
}

void launch_multi_dot(int64_t N, int R, const double* V, int64_t slab, int nv, const double* w, double* partials,
                      unsigned* counters, double* out, cudaStream_t st) {
  if (nv <= 0) return;
  note_launches(1);
  DISPATCH_POW2(R, (k_multi_dot<R><<<dim3(gmres_blocks(N * R), nv), kVecThreads, 0, st>>>(N, V, slab, w, partials,
                                                                                         counters, out)));
}

void launch_multi_axpy(int64_t N, int R, const double* V, int64_t slab, int nv, const double* h, double* w,
                       cudaStream_t st) {
  if (nv <= 0) return;
  note_launches(1);
  DISPATCH_POW2(R, (k_multi_axpy<R><<<elem_blocks(N * R), kVecThreads, 0, st>>>(N, V, slab, nv, h, w)));
}

void launch_normalize(int64_t N, int R, const double* w, const double* nrm2, double* v, double* hnorm,
                      cudaStream_t st) {
  note_launches(1);
  DISPATCH_POW2(R, (k_normalize<R><<<elem_blocks(N * R), kVecThreads, 0, st>>>(N, w, nrm2, v, hnorm)));
}

template <typename TZ>
void launch_zy_add(int64_t N, int R, const TZ* Z, int64_t slab, int nv, const double* y, double* d,
                   cudaStream_t st) {
  if (nv <= 0) return;
  note_launches(1);
  DISPATCH_POW2(R, (k_zy_add<R, TZ><<<elem_blocks(N * R), kVecThreads, 0, st>>>(N, Z, slab, nv, y, d)));
}
template void launch_zy_add<double>(int64_t, int, const double*, int64_t, int, const double*, double*, cudaStream_t);
template void launch_zy_add<float>(int64_t, int, const float*, int64_t, int, const double*, double*, cudaStream_t);

template void launch_convert<double, double>(int64_t, int, const double*, int, double*, int, cudaStream_t);
template void launch_convert<double, float>(int64_t, int, const double*, int, float*, int, cudaStream_t);
template void launch_convert<float, double>(int64_t, int, const float*, int, double*, int, cudaStream_t);

}  // namespace hif
