// Apply sweeps of the factorization (Eq. 3.1 / 4.2).  One thread block per
// block of the factor (cell or front) of one level; the right-hand sides are
// processed R at a time.  Vectors: N x nrhs row-major, row stride ldx.
//
// F^-1 = V_0 V_1/2 ... D^-1 ... V_1/2^T V_0^T, per block (p eliminated,
// q its neighbours; fronts carry T, cells do not; A_pp = L D_p L^T with
// D_p = diag(S), all +1 for an SPD block, and G = A_qp L^-T D_p):
//   up   (V^T, then D_p^-1 on p):  [front] x_p -= T^T x_q;  y_p = Linv x_p;
//                                  x_q -= G y_p;  x_p = S y_p
//   down (V):    x_p = Linv^T (x_p - G^T x_q);  [front] x_q -= T x_p
// F = V_0^-T ... D ... V_0^-1:
//   fwd_up   (V^-1):  [front] x_q += T x_p;  x_p = L^T x_p + G^T x_q
//   fwd_down (D_p, then V^-T):  x_p = S x_p;  x_q += G x_p;  x_p = L x_p;
//                               [front] x_p += T^T x_q
// Two-sided (unsymmetric) blocks, A_pp = L U: the same steps with L^-1 and
// G = A_qp U^-1 in the up sweep, U^-T and (L^-1 A_pq)^T in the place of
// Linv and G in the down sweep, U^T in the place of L^T in fwd_up.
// Cells of one level share boundary DOFs, so their x_q updates use atomics,
// or, in the deterministic mode, go to a contribution buffer (one row per
// (cell, q-row) pair) that a second launch sums per DOF in cell order; the
// DOFs of a front belong to it alone.
//
// The F^-1 sweeps read each block of the factor once: when the launch's
// largest block fits, the block's Linv (packed), G and T are first copied to
// shared memory by bulk copies (TMA), then every product is a serial dot per
// (output row, group of right-hand sides), one thread each, with no
// cross-lane reductions.  One launch per level and direction, with
// programmatic dependent launch between them.
#include <atomic>

#include "hif_internal.h"
#include "blockops.cuh"
#include "kernels.h"

namespace hif {

// L2: read through L2 only (rows written by other blocks of the same launch).
template <typename T, int R, bool L2 = false>
__device__ __forceinline__ void gather(T* dst, const T* x, const int* ids, int n, int nr, int ldx) {
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, r = e % R;
    const T* src = x + (int64_t)ids[i] * ldx + r;
    dst[e] = (r < nr) ? (L2 ? __ldcg(src) : *src) : T(0);
  }
}

// ---- TMA bulk staging -------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// The mbarrier of a CTA's bulk copies: initialized once per CTA by thread 0,
// before a __syncthreads() and before any thread polls it.
__device__ __forceinline__ void bulk_init(uint64_t* mbar) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// One thread starts bulk copies (global -> this CTA's shared memory) of the
// listed regions, all completing one phase of the CTA's mbarrier (parity:
// the phase's parity, 0 for the first copy of the CTA, flipped by each later
// one); every thread then waits with a bounded spin.  Regions are 16-byte
// aligned with sizes that are multiples of 16 bytes.  Shared memory the
// block's threads wrote before (an earlier block of the same CTA) is ordered
// before the copies by a proxy fence.  wait() returns false (and sets bit 3
// of *err) if the wait ran out; it then waits once more, bounded, for the
// copies to land.
struct BulkStage {
  uint64_t* mbar;
  uint32_t parity;
  __device__ void start(int nreg, void* const* dst, const void* const* src, const uint32_t* bytes) {
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      uint32_t total = 0;
      for (int k = 0; k < nreg; ++k) total += bytes[k];
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(total)
                   : "memory");
      for (int k = 0; k < nreg; ++k)
        if (bytes[k] > 0)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(dst[k])),
              "l"(src[k]), "r"(bytes[k]), "r"(smem_u32(mbar))
              : "memory");
    }
  }
  __device__ bool try_wait() const {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
  }
  __device__ bool wait(int* err, long polls = 1L << 26) const {
    for (long it = 0; it < polls; ++it)
      if (try_wait()) return true;
    if (err) atomicOr(err, 8);
    for (long it = 0; it < polls; ++it)
      if (try_wait()) break;
    return false;
  }
};

__device__ __forceinline__ int64_t tri(int i) { return (int64_t)i * (i + 1) / 2; }

// Shared-memory plan of one F^-1 sweep block:
// [mbarrier | Linv | G | T | xp | yp | xq] (each region 16-byte aligned).
template <typename T, int R>
struct SweepSmem {
  uint64_t* mbar;
  T *Ls, *Gs, *Ts, *xp, *yp, *xq;
  __device__ SweepSmem(unsigned char* raw, int np, int nq, bool staged, bool front) {
    mbar = reinterpret_cast<uint64_t*>(raw);
    T* p = reinterpret_cast<T*>(raw + 16);
    Ls = Gs = Ts = nullptr;
    if (staged) {
      Ls = p;
      p += packed_size(np);
      Gs = p;
      p += pad4((int64_t)nq * np);
      if (front) {
        Ts = p;
        p += pad4((int64_t)nq * np);
      }
    }
    xp = p;
    p += pad4((int64_t)np * R);
    yp = p;
    p += pad4((int64_t)np * R);
    xq = p;
  }
};

// Columns per thread in the products: each thread owns one output row and a
// group of CG consecutive right-hand sides (register accumulators).
template <int R> struct ColGroup { static constexpr int CG = R < 2 ? R : 2; static constexpr int NG = R / CG; };

// The rotation of a front skeletonized by the SVD on its slots, x_c = [x_q;
// x_p] (R columns): oq / op <- the q / p rows of V^T x_c (transpose) or of
// V x_c; V is (nq + np) x (nq + np), row-major, read from global memory.
// The outputs are distinct from the inputs; the caller synchronizes.
template <typename T, int R>
__device__ void svd_rotate(const T* __restrict__ V, int np, int nq, const T* xq, const T* xp, T* oq, T* op,
                           bool transpose) {
  const int nc = np + nq;
  for (int e = threadIdx.x; e < nc * R; e += blockDim.x) {
    const int j = e / R, r = e % R;
    T acc = T(0);
    if (transpose) {
      for (int t = 0; t < nq; ++t) acc += V[(int64_t)t * nc + j] * xq[t * R + r];
      for (int t = 0; t < np; ++t) acc += V[(int64_t)(nq + t) * nc + j] * xp[t * R + r];
    } else {
      const T* v = V + (int64_t)j * nc;
      for (int t = 0; t < nq; ++t) acc += v[t] * xq[t * R + r];
      for (int t = 0; t < np; ++t) acc += v[nq + t] * xp[t * R + r];
    }
    if (j < nq) oq[j * R + r] = acc;
    else op[(j - nq) * R + r] = acc;
  }
}

template <typename T, int R>
__device__ __forceinline__ void stage_factor(SweepSmem<T, R>& sm, BulkStage& bs, const T*& Linv, const T*& G,
                                             const T*& Tm, int np, int nq, bool front) {
  void* dst[3] = {sm.Ls, sm.Gs, sm.Ts};
  const void* src[3] = {Linv, G, Tm};
  uint32_t bytes[3] = {(uint32_t)(sizeof(T) * packed_size(np)), (uint32_t)(sizeof(T) * pad4((int64_t)nq * np)),
                       front ? (uint32_t)(sizeof(T) * pad4((int64_t)nq * np)) : 0u};
  bs.start(front ? 3 : 2, dst, src, bytes);
  Linv = sm.Ls;
  G = sm.Gs;
  Tm = sm.Ts;
}

__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One block of the up sweep (V^T) by the whole thread block.  wait() runs
// after the block's factor copy has started and before it reads any vector
// row (the previous level's results); it returns false to skip the block.
// L2: vector rows are read through L2 only.
template <typename T, int R, bool L2, typename Wait>
__device__ void sweep_up_block(const ApplyDesc& bd, const int* __restrict__ ipool, const T* __restrict__ fac,
                               T* __restrict__ x, int nr, int ldx, int is_front, int staged, int* err,
                               unsigned char* smem_raw, Wait wait, uint32_t parity = 0,
                               T* __restrict__ contrib = nullptr) {
  constexpr int CG = ColGroup<R>::CG, NG = ColGroup<R>::NG;
  const int np = bd.np, nq = bd.nq;
  if (np == 0) {
    wait();
    return;
  }
  const int* idp = ipool + bd.ids;
  const int* idq = idp + np;
  SweepSmem<T, R> sm(smem_raw, np, nq, staged, is_front);
  BulkStage bs{sm.mbar, parity};
  const T* Linv = fac + bd.Linv;
  const T* G = fac + bd.G;
  const T* Tm = is_front ? fac + bd.T : nullptr;
  if (staged) stage_factor<T, R>(sm, bs, Linv, G, Tm, np, nq, is_front);
  const bool go = wait();
  T* xp = sm.xp;
  T* yp = sm.yp;
  T* xq = sm.xq;
  if (go) {
    gather<T, R, L2>(xp, x, idp, np, nr, ldx);
    if (is_front) gather<T, R, L2>(xq, x, idq, nq, nr, ldx);
  }
  // every thread leaves if one thread's wait for the factor copy ran out
  if (!__syncthreads_and(!staged || bs.wait(err))) return;
  if (!go) return;
  if (is_front && bd.V >= 0) {                   // SVD front: x_c <- V^T x_c
    T* tq = xq + pad4((int64_t)nq * R);
    svd_rotate<T, R>(fac + bd.V, np, nq, xq, xp, tq, yp, true);
    __syncthreads();
    for (int e = threadIdx.x; e < np * R; e += blockDim.x) xp[e] = yp[e];
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x) xq[e] = tq[e];
    __syncthreads();
  } else if (is_front && nq > 0) {               // x_p -= T^T x_q
    for (int e = threadIdx.x; e < np * NG; e += blockDim.x) {
      const int i = e / NG, c0 = (e % NG) * CG;
      T acc[CG] = {};
      for (int s2 = 0; s2 < nq; ++s2) {
        const T t = Tm[(int64_t)s2 * np + i];
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[c] += t * xq[s2 * R + c0 + c];
      }
#pragma unroll
      for (int c = 0; c < CG; ++c) xp[i * R + c0 + c] -= acc[c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < np * NG; e += blockDim.x) {   // y_p = Linv x_p
    const int i = e / NG, c0 = (e % NG) * CG;
    const T* l = Linv + tri(i);
    T acc[CG] = {};
    const T* xv = xp + c0;
#pragma unroll 4
    for (int t = 0; t <= i; ++t) {
      const T lv = l[t];
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[c] += lv * xv[c];
      xv += R;
    }
    const T sg = fac[bd.S + i];                   // the sign of D_p's entry (LDL^T), +1 if SPD
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      yp[i * R + c0 + c] = acc[c];
      if (c0 + c < nr) x[(int64_t)idp[i] * ldx + c0 + c] = sg * acc[c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nq * NG; e += blockDim.x) {   // x_q -= G y_p
    const int s2 = e / NG, c0 = (e % NG) * CG;
    const T* g = G + (int64_t)s2 * np;
    T acc[CG] = {};
    for (int t = 0; t < np; ++t) {
      const T gv = g[t];
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[c] += gv * yp[t * R + c0 + c];
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      if (c0 + c >= nr) continue;
      T* dst = x + (int64_t)idq[s2] * ldx + c0 + c;
      if (is_front) *dst = xq[s2 * R + c0 + c] - acc[c];
      else if (contrib) contrib[(bd.cslot + s2) * R + c0 + c] = acc[c];
      else atomicAdd(dst, -acc[c]);
    }
  }
}

template <typename T, int R>
__global__ void k_apply_up(const ApplyDesc* __restrict__ blocks, const int* __restrict__ ipool,
                           const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx,
                           int is_front, int staged, int* err, T* __restrict__ contrib) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplyDesc bd = blocks[blockIdx.x];
  bulk_init(reinterpret_cast<uint64_t*>(smem_raw));
  __syncthreads();
  sweep_up_block<T, R, false>(
      bd, ipool, fac, x, nr, ldx, is_front, staged, err, smem_raw,
      [] {
        pdl_wait_then_release();
        return true;
      },
      0u, contrib);
}

// One block of the down sweep (V), as sweep_up_block.
template <typename T, int R, bool L2, typename Wait>
__device__ void sweep_down_block(const ApplyDesc& bd, const int* __restrict__ ipool, const T* __restrict__ fac,
                                 T* __restrict__ x, int nr, int ldx, int is_front, int staged, int* err,
                                 unsigned char* smem_raw, Wait wait, uint32_t parity = 0) {
  constexpr int CG = ColGroup<R>::CG, NG = ColGroup<R>::NG;
  const int np = bd.np, nq = bd.nq;
  if (np == 0) {
    wait();
    return;
  }
  const int* idp = ipool + bd.ids;
  const int* idq = idp + np;
  SweepSmem<T, R> sm(smem_raw, np, nq, staged, is_front);
  BulkStage bs{sm.mbar, parity};
  const T* Linv = fac + (bd.Linv2 >= 0 ? bd.Linv2 : bd.Linv);   // two-sided: U^-T
  const T* G = fac + (bd.G2 >= 0 ? bd.G2 : bd.G);               // two-sided: (L^-1 A_pq)^T
  const T* Tm = is_front ? fac + bd.T : nullptr;
  if (staged) stage_factor<T, R>(sm, bs, Linv, G, Tm, np, nq, is_front);
  const bool go = wait();
  T* xp = sm.xp;
  T* zp = sm.yp;
  T* xq = sm.xq;
  const bool svd = is_front && bd.V >= 0;
  if (go) {
    gather<T, R, L2>(xp, x, idp, np, nr, ldx);
    gather<T, R, L2>(xq, x, idq, nq, nr, ldx);
  }
  if (!__syncthreads_and(!staged || bs.wait(err))) return;
  if (!go) return;
  if (nq > 0) {                                  // w = x_p - G^T x_q (in place)
    for (int e = threadIdx.x; e < np * NG; e += blockDim.x) {
      const int i = e / NG, c0 = (e % NG) * CG;
      T acc[CG] = {};
      for (int s2 = 0; s2 < nq; ++s2) {
        const T gv = G[(int64_t)s2 * np + i];
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[c] += gv * xq[s2 * R + c0 + c];
      }
#pragma unroll
      for (int c = 0; c < CG; ++c) xp[i * R + c0 + c] -= acc[c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < np * NG; e += blockDim.x) {   // z = Linv^T w
    const int i = e / NG, c0 = (e % NG) * CG;
    T acc[CG] = {};
    const T* lcol = Linv + tri(i) + i;           // Linv[t][i], row t starts at tri(t)
    const T* xv = xp + i * R + c0;
#pragma unroll 4
    for (int t = i; t < np; ++t) {
      const T lv = *lcol;
      lcol += t + 1;
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[c] += lv * xv[c];
      xv += R;
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      zp[i * R + c0 + c] = acc[c];
      if (!svd && c0 + c < nr) x[(int64_t)idp[i] * ldx + c0 + c] = acc[c];
    }
  }
  if (svd) {                                     // SVD front: x_c <- V x_c
    __syncthreads();
    T* tq = xq + pad4((int64_t)nq * R);
    svd_rotate<T, R>(fac + bd.V, np, nq, xq, zp, tq, xp, false);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x)
      if (e % R < nr) x[(int64_t)idq[e / R] * ldx + e % R] = tq[e];
    for (int e = threadIdx.x; e < np * R; e += blockDim.x)
      if (e % R < nr) x[(int64_t)idp[e / R] * ldx + e % R] = xp[e];
  } else if (is_front && nq > 0) {               // x_q -= T z
    __syncthreads();
    for (int e = threadIdx.x; e < nq * NG; e += blockDim.x) {
      const int s2 = e / NG, c0 = (e % NG) * CG;
      const T* t = Tm + (int64_t)s2 * np;
      T acc[CG] = {};
      for (int c1 = 0; c1 < np; ++c1) {
        const T tv = t[c1];
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[c] += tv * zp[c1 * R + c0 + c];
      }
#pragma unroll
      for (int c = 0; c < CG; ++c)
        if (c0 + c < nr) x[(int64_t)idq[s2] * ldx + c0 + c] = xq[s2 * R + c0 + c] - acc[c];
    }
  }
}

template <typename T, int R>
__global__ void k_apply_down(const ApplyDesc* __restrict__ blocks, const int* __restrict__ ipool,
                             const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx,
                             int is_front, int staged, int* err, T* __restrict__ contrib) {
  (void)contrib;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplyDesc bd = blocks[blockIdx.x];
  bulk_init(reinterpret_cast<uint64_t*>(smem_raw));
  __syncthreads();
  sweep_down_block<T, R, false>(bd, ipool, fac, x, nr, ldx, is_front, staged, err, smem_raw, [] {
    pdl_wait_then_release();
    return true;
  });
}

// The root (a cell without boundary): D^-1 x = Linv^T (Linv x) by one block,
// the up body then the down body, in one launch instead of two.  The down
// body reads Linv from global memory (the up body's staging copy leaves it in
// L2) and the rows the up body wrote (same block, after the barrier).
template <typename T, int R>
__global__ void k_apply_root(const ApplyDesc* __restrict__ blocks, const int* __restrict__ ipool,
                             const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx,
                             int is_front, int staged, int* err, T* __restrict__ contrib) {
  (void)contrib;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplyDesc bd = blocks[0];
  bulk_init(reinterpret_cast<uint64_t*>(smem_raw));
  __syncthreads();
  sweep_up_block<T, R, false>(bd, ipool, fac, x, nr, ldx, 0, staged, err, smem_raw, [] {
    pdl_wait_then_release();
    return true;
  });
  __syncthreads();
  sweep_down_block<T, R, false>(bd, ipool, fac, x, nr, ldx, 0, 0, err, smem_raw, [] { return true; });
}

// ---- check of the bounded wait: a bulk-copy phase that no copy completes
// (the transaction count is announced, nothing is copied), waited for with
// `polls` polls; the wait gives up, sets bit 3 of *err and returns.
__global__ void k_wait_test_bulk(int* err, long polls) {
  __shared__ __align__(16) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(16u)
                 : "memory");
  }
  __syncthreads();
  BulkStage bs{&mbar, 0u};
  bs.wait(err, polls);
}

void launch_wait_test_bulk(int* err, long polls, cudaStream_t st) {
  note_launches(1);
  k_wait_test_bulk<<<1, 32, 0, st>>>(err, polls);
}

// ---- forward operator F (used by the error estimates; not staged) ----------
template <typename T, int R>
__global__ void k_fwd_up(const ApplyDesc* __restrict__ blocks, const int* __restrict__ ipool,
                         const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx, int is_front,
                         int staged, int* err, T* __restrict__ contrib) {
  (void)err;
  (void)contrib;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  (void)staged;
  const ApplyDesc bd = blocks[blockIdx.x];
  const int np = bd.np, nq = bd.nq;
  if (np == 0) return;
  const int* idp = ipool + bd.ids;
  const int* idq = idp + np;
  T* xp = reinterpret_cast<T*>(smem_raw);
  T* xq = xp + pad4((int64_t)np * R);
  T* tq = xq + pad4((int64_t)nq * R);
  const T* Lp = fac + (bd.L2 >= 0 ? bd.L2 : bd.L);     // two-sided: U^T
  const T* G = fac + (bd.G2 >= 0 ? bd.G2 : bd.G);
  gather<T, R>(xp, x, idp, np, nr, ldx);
  gather<T, R>(xq, x, idq, nq, nr, ldx);
  __syncthreads();
  if (is_front && bd.V >= 0) {    // SVD front: x_c <- V^T x_c (Q_c^-1 = Q_c^T)
    T* tp = tq + pad4((int64_t)nq * R);
    svd_rotate<T, R>(fac + bd.V, np, nq, xq, xp, tq, tp, true);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x) {
      xq[e] = tq[e];
      if (e % R < nr) x[(int64_t)idq[e / R] * ldx + e % R] = tq[e];
    }
    for (int e = threadIdx.x; e < np * R; e += blockDim.x) xp[e] = tp[e];
    __syncthreads();
  } else if (is_front && nq > 0) {       // x_q += T x_p
    const T* Tm = fac + bd.T;
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x) {
      const int s2 = e / R, r = e % R;
      T acc = T(0);
      for (int c = 0; c < np; ++c) acc += Tm[(int64_t)s2 * np + c] * xp[c * R + r];
      tq[e] = xq[e] + acc;
      if (r < nr) x[(int64_t)idq[s2] * ldx + r] = tq[e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x) xq[e] = tq[e];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < np * R; e += blockDim.x) {   // x_p = L^T x_p + G^T x_q
    const int i = e / R, r = e % R;
    T acc = T(0);
    for (int t = i; t < np; ++t) acc += Lp[tri(t) + i] * xp[t * R + r];
    for (int s2 = 0; s2 < nq; ++s2) acc += G[(int64_t)s2 * np + i] * xq[s2 * R + r];
    if (r < nr) x[(int64_t)idp[i] * ldx + r] = acc;
  }
}

template <typename T, int R>
__global__ void k_fwd_down(const ApplyDesc* __restrict__ blocks, const int* __restrict__ ipool,
                           const T* __restrict__ fac, T* __restrict__ x, int nr, int ldx, int is_front,
                           int staged, int* err, T* __restrict__ contrib) {
  (void)err;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  (void)staged;
  const ApplyDesc bd = blocks[blockIdx.x];
  const int np = bd.np, nq = bd.nq;
  if (np == 0) return;
  const int* idp = ipool + bd.ids;
  const int* idq = idp + np;
  T* xp = reinterpret_cast<T*>(smem_raw);
  T* xq = xp + pad4((int64_t)np * R);
  T* oq = xq + pad4((int64_t)nq * R);   // SVD fronts: the rotated q rows
  T* tp = oq + pad4((int64_t)nq * R);   // SVD fronts: L x_p before the rotation
  const bool svd = is_front && bd.V >= 0;
  const T* Lp = fac + bd.L;
  const T* G = fac + bd.G;
  gather<T, R>(xp, x, idp, np, nr, ldx);
  if (is_front) gather<T, R>(xq, x, idq, nq, nr, ldx);
  __syncthreads();
  for (int e = threadIdx.x; e < np * R; e += blockDim.x) xp[e] *= fac[bd.S + e / R];   // D_p
  __syncthreads();
  for (int e = threadIdx.x; e < nq * R; e += blockDim.x) {   // x_q += G x_p
    const int s2 = e / R, r = e % R;
    const T* g = G + (int64_t)s2 * np;
    T acc = T(0);
    for (int c = 0; c < np; ++c) acc += g[c] * xp[c * R + r];
    if (is_front) {
      xq[e] += acc;
      if (!svd && r < nr) x[(int64_t)idq[s2] * ldx + r] = xq[e];
    } else if (contrib) {
      contrib[(bd.cslot + s2) * R + r] = acc;
    } else if (r < nr) {
      atomicAdd(x + (int64_t)idq[s2] * ldx + r, acc);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < np * R; e += blockDim.x) {   // x_p = L x_p [+ T^T x_q]
    const int i = e / R, r = e % R;
    const T* l = Lp + tri(i);
    T acc = T(0);
    for (int t = 0; t <= i; ++t) acc += l[t] * xp[t * R + r];
    if (svd) {
      tp[e] = acc;
      continue;
    }
    if (is_front) {
      const T* Tm = fac + bd.T;
      for (int s2 = 0; s2 < nq; ++s2) acc += Tm[(int64_t)s2 * np + i] * xq[s2 * R + r];
    }
    if (r < nr) x[(int64_t)idp[i] * ldx + r] = acc;
  }
  if (svd) {                      // x_c <- V x_c (Q_c^-T = Q_c)
    __syncthreads();
    svd_rotate<T, R>(fac + bd.V, np, nq, xq, tp, oq, xp, false);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * R; e += blockDim.x)
      if (e % R < nr) x[(int64_t)idq[e / R] * ldx + e % R] = oq[e];
    for (int e = threadIdx.x; e < np * R; e += blockDim.x)
      if (e % R < nr) x[(int64_t)idp[e / R] * ldx + e % R] = xp[e];
  }
}

// ---------------------------------------------------------------------------
constexpr size_t kSweepSmemCap = 200 * 1024;
constexpr size_t kStageCap = 96 * 1024;   // stage only when two blocks still fit an SM

template <typename T>
static size_t vec_smem(int R, int max_np, int max_nq) {
  return 16 + sizeof(T) * (size_t)(2 * pad4((int64_t)max_np * R) + 2 * pad4((int64_t)max_nq * R));
}

template <typename T>
static size_t stage_smem(int max_np, int max_nq, int is_front) {
  return sizeof(T) * (size_t)(packed_size(max_np) + (is_front ? 2 : 1) * pad4((int64_t)max_nq * max_np));
}

// The deterministic scatter's second launch: x[dofs[k]] += sign * (sum of
// the DOF's contribution rows in cell order), one thread per (DOF, column).
template <typename T, int R>
__global__ void k_contrib_reduce(const int* __restrict__ ptr, const int* __restrict__ dofs,
                                 const int* __restrict__ slots, int ndof, const T* __restrict__ contrib,
                                 T* __restrict__ x, int nr, int ldx, T sign) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ndof * nr) return;
  const int k = (int)(e / nr), c = (int)(e % nr);
  T s = T(0);
  for (int j = ptr[k]; j < ptr[k + 1]; ++j) s += contrib[(int64_t)slots[j] * R + c];
  x[(int64_t)dofs[k] * ldx + c] += sign * s;
}

template <typename T, int R>
static void launch_sweep_R(int op, const ApplyDesc* blocks, int nblocks, const int* ipool,
                           const T* fac, T* x, int nr, int ldx, int is_front, int max_np,
                           int max_nq, int* err, cudaStream_t st, SweepShape shape, const ContribPlan* cp) {
  const size_t vsm = vec_smem<T>(R, max_np, max_nq);
  const size_t ssm = stage_smem<T>(max_np, max_nq, is_front);
  const bool finv = op <= 1 || op == 4;   // F^-1 sweeps (4: the fused root)
  const int staged = finv && (vsm + ssm <= kStageCap) && shape.staged != 0;
  const size_t smem = vsm + (staged ? ssm : 0);
  void (*fn)(const ApplyDesc*, const int*, const T*, T*, int, int, int, int, int*, T*) = nullptr;
  // cells' x_q updates: to the contribution buffer, then summed per DOF
  T* contrib = (cp && cp->ndof > 0 && !is_front && (op == 0 || op == 3)) ? static_cast<T*>(cp->buf) : nullptr;
  switch (op) {
    case 0: fn = k_apply_up<T, R>; break;
    case 1: fn = k_apply_down<T, R>; break;
    case 2: fn = k_fwd_up<T, R>; break;
    case 3: fn = k_fwd_down<T, R>; break;
    default: fn = k_apply_root<T, R>; break;
  }
  // raise the dynamic shared-memory limit and prefer the largest shared
  // carveout once per kernel (not again while a stream capture records it)
  static std::atomic<bool> attr_set[5] = {false, false, false, false, false};
  if (!attr_set[op]) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemCap);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_set[op] = true;
  }
  // one thread per (row, column group) of the largest product, in warps,
  // so that small blocks leave room for more resident blocks per SM
  constexpr int NG = ColGroup<R>::NG;
  int work = (max_np > max_nq ? max_np : max_nq) * NG;
  int threads = ((work + 31) / 32) * 32;
  threads = threads < 32 ? 32 : (threads > 256 ? 256 : threads);
  if (shape.threads > 0) threads = shape.threads;
  note_launches(contrib ? 2 : 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if (finv) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, fn, blocks, ipool, fac, x, nr, ldx, is_front, staged, err, contrib);
  } else {
    fn<<<nblocks, threads, smem, st>>>(blocks, ipool, fac, x, nr, ldx, is_front, staged, err, contrib);
  }
  if (contrib) {
    const int64_t n = (int64_t)cp->ndof * nr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = finv ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_contrib_reduce<T, R>, cp->ptr, cp->dofs, cp->slots, cp->ndof,
                       (const T*)contrib, x, nr, ldx, op == 0 ? T(-1) : T(1));
  }
}

template <typename T>
int sweep_chunk(int max_np, int max_nq, int nrhs) {
  int R = 32;
  while (R > 1 && (R / 2 >= nrhs || vec_smem<T>(R, max_np, max_nq) > kSweepSmemCap)) R /= 2;
  return R;
}

template <typename T>
void launch_sweep(int op, const ApplyDesc* blocks, int nblocks, const int* ipool, const T* fac,
                  T* x, int nrhs, int ldx, int is_front, int max_np, int max_nq, int* err, cudaStream_t st,
                  SweepShape shape, const ContribPlan* cp) {
  if (nblocks == 0) return;
  const int R = sweep_chunk<T>(max_np, max_nq, nrhs);
  for (int r0 = 0; r0 < nrhs; r0 += R) {
    const int nr = (nrhs - r0) < R ? (nrhs - r0) : R;
    T* xr = x + r0;
    switch (R) {
      case 32: launch_sweep_R<T, 32>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
      case 16: launch_sweep_R<T, 16>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
      case 8: launch_sweep_R<T, 8>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
      case 4: launch_sweep_R<T, 4>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
      case 2: launch_sweep_R<T, 2>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
      default: launch_sweep_R<T, 1>(op, blocks, nblocks, ipool, fac, xr, nr, ldx, is_front, max_np, max_nq, err, st, shape, cp); break;
    }
  }
}

template void launch_sweep<double>(int, const ApplyDesc*, int, const int*, const double*, double*,
                                   int, int, int, int, int, int*, cudaStream_t, SweepShape, const ContribPlan*);
template void launch_sweep<float>(int, const ApplyDesc*, int, const int*, const float*, float*,
                                  int, int, int, int, int, int*, cudaStream_t, SweepShape, const ContribPlan*);

}  // namespace hif
