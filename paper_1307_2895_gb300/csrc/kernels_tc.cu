// Tensor-core (tcgen05, kind::tf32) products of the FP32 tiled elimination
// (Lemma 2.1 on large cells and on the redundant blocks of large fronts):
// the panel solve M <- M D_p^T, the trailing update A_ij -= L_ip L_jp^T and
// the Schur complement U = F_BB - G G^T of the blocked right-looking
// Cholesky in kernels_tiled.cu, whose SIMT versions they replace in the
// mixed-precision mode.
//
// One CTA (512 threads) computes a 128 x 64 block of a product A B^T with
// both operands read k-contiguous ("K-major") through functors:
//   * K is staged in chunks of 32 FP32 values (128 bytes per row) into a
//     two-stage shared-memory ring, written by all threads in the 128-byte
//     swizzled K-major layout that the MMA's shared-memory descriptors read;
//   * one thread issues the chunk's tcgen05.mma (M = 128, N = 64, K = 8 per
//     instruction); each of the chunk's four K = 8 steps accumulates its
//     split products from zero in a tensor-memory accumulator of its own
//     (64 columns; two sets of four, 512 columns, alternate between chunks),
//     and tcgen05.commit signals their completion;
//   * while the next chunk's MMAs run, every warp reads the finished chunk's
//     four partial sums back with tcgen05.ld (warp w owns TMEM lanes
//     32 (w mod 4) ..) and adds them to FP32 registers with round-to-nearest:
//     the tensor core's own accumulation covers the products of 8 values of
//     K only (its adder truncates; measured), the rest is an ordinary FP32
//     sum.  The CTA holds all 512 TMEM columns, so its shared-memory request
//     is above half an SM's: one CTA per SM, and an allocation never waits;
//   * the epilogue transposes the registers through shared memory so that
//     the global read-modify-write of the output is coalesced.
//
// TF32 keeps 10 mantissa bits.  Each operand value is split into `parts`
// TF32 numbers by repeated round-to-nearest: x = x0 + x1 + x2 (+ a remainder
// below 2^-33 |x|), and the products kept are those of order at least 2^-22:
//   parts = 3: x0 y0, x0 y1, x1 y0, x0 y2, x1 y1, x2 y0  (six MMAs; the split
//              keeps 33 bits, about FP32 accuracy)
//   parts = 2: x0 y0, x0 y1, x1 y0                      (three; about 2^-21)
//   parts = 1: x0 y0                                    (plain TF32, 2^-11)
// (the split-operand schemes of Markidis et al., 2018, and Ootomo & Yokota,
// 2022), smallest terms first.  Accumulation is FP32 in tensor memory.
//
// Every wait is bounded by the global timer: after about a second the kernel
// sets bit 5 (32) of status[0], waits once more (bounded) for its MMAs and
// releases its tensor memory before returning.
#include <atomic>
#include <cstdint>

#include "hif_internal.h"
#include "kernels.h"
#include "tile_mma.cuh"

namespace hif {
namespace {

constexpr int kBM = 128;            // output rows per CTA (MMA M)
constexpr int kBN = 64;             // output columns per CTA (MMA N)
constexpr int kChunk = 32;          // FP32 values of K per stage (128 bytes)
constexpr int kThreads = 512;
constexpr int kABytes = kBM * 128;  // one operand part (hi or lo), 128 rows
constexpr int kBBytes = kBN * 128;
constexpr int kStages = 2;
constexpr int kTmemCols = 512;            // 2 x 4 accumulators of 64 columns
// stage: the operand parts A_0 .. A_{parts-1}, then B_0 .. B_{parts-1}
__host__ __device__ constexpr int stage_bytes(int parts) { return parts * (kABytes + kBBytes); }
// + alignment slack + barriers; at least 116 KB: one CTA per SM (TMEM)
__host__ __device__ constexpr int smem_bytes(int parts) {
  return kStages * stage_bytes(parts) + 1088 > 116 * 1024 ? kStages * stage_bytes(parts) + 1088 : 116 * 1024;
}
constexpr uint64_t kWaitNs = 1000000000ull;                     // bound of every wait

// Instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor: 128-byte swizzle, K-major; 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (1),
// descriptor version 1 at bit 46, layout type 2 (128-byte swizzle) at 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Byte offset of element (row r, k) of a 128-byte-swizzled K-major tile of
// FP32 rows of 32 values: the 16-byte chunk index is XORed with r mod 8.
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4) | ((k & 3) << 2)));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the phase of parity `parity`; false after ns
// nanoseconds of the global timer.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > ns) return false;
  return true;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float rna_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// The TF32 parts of v, part i at p0 + i * stride + off: repeated
// round-to-nearest, the last part keeps the remainder.
template <int PARTS>
__device__ __forceinline__ void store_split(uint8_t* p0, int stride, uint32_t off, float v) {
  float x = v;
#pragma unroll
  for (int i = 0; i < PARTS; ++i) {
    const float h = (i + 1 < PARTS) ? rna_tf32(x) : x;
    *reinterpret_cast<float*>(p0 + i * stride + off) = h;
    x -= h;
  }
}

// (A part, B part) products kept for PARTS parts, smallest terms first.
template <int PARTS> struct Pairs;
template <> struct Pairs<1> {
  static constexpr int n = 1;
  __device__ static constexpr int a(int) { return 0; }
  __device__ static constexpr int b(int) { return 0; }
};
template <> struct Pairs<2> {
  static constexpr int n = 3;
  __device__ static constexpr int a(int t) { return t == 1 ? 1 : 0; }   // (0,1) (1,0) (0,0)
  __device__ static constexpr int b(int t) { return t == 0 ? 1 : 0; }
};
template <> struct Pairs<3> {
  static constexpr int n = 6;   // (1,1) (0,2) (2,0) (0,1) (1,0) (0,0)
  __device__ static constexpr int a(int t) { return t == 0 ? 1 : t == 2 ? 2 : t == 4 ? 1 : 0; }
  __device__ static constexpr int b(int t) { return t == 0 ? 1 : t == 1 ? 2 : t == 3 ? 1 : 0; }
};

constexpr int kPerThreadA = kBM * kChunk / kThreads;   // 8
constexpr int kPerThreadB = kBN * kChunk / kThreads;   // 4
constexpr int kAccCols = kBM * kBN / kThreads;         // 16 accumulator values per thread

// Shared state of one CTA: the 1024-aligned stage ring, two chunk barriers,
// the tensor-memory base address and the thread's FP32 accumulators (row
// 32 (warp mod 4) + lane, columns 16 (warp / 4) ..).
template <int PARTS>
struct TcCta {
  static constexpr int kStage = stage_bytes(PARTS);
  uint8_t* ring;
  uint64_t* bars;
  uint32_t tmem;
  int* status;
  bool ok;
  uint64_t wait_ns = kWaitNs;   // bound of the waits for the MMAs
  float acc[kAccCols];

  __device__ void init(uint8_t* raw, int* st) {
    status = st;
    ok = true;
    const uint32_t a = su32(raw);
    ring = raw + (((a + 1023u) & ~1023u) - a);
    bars = reinterpret_cast<uint64_t*>(ring + kStages * kStage);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + kStages);
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
      for (int s = 0; s < kStages; ++s) mbar_init(su32(bars + s));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
#pragma unroll
    for (int i = 0; i < kAccCols; ++i) acc[i] = 0.f;
    fence_before();
    __syncthreads();
    fence_after();
    tmem = *slot;
  }

  __device__ void fail() {
    if (ok) atomicOr(status, 32);
    ok = false;
  }

  // add chunk c (its four partial sums, accumulator set c & 1) to the registers
  __device__ void drain(int c) {
    const uint32_t bar = su32(bars + (c & 1)), par = (uint32_t)((c >> 1) & 1);
    if (!mbar_wait(bar, par, wait_ns)) {
      fail();
      mbar_wait(bar, par, wait_ns);
    }
    fence_after();
    const int warp = threadIdx.x >> 5;
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(4 * kBN * (c & 1) + kAccCols * (warp >> 2));
    float v[kChunk / 8][kAccCols];
#pragma unroll
    for (int j = 0; j < kChunk / 8; ++j) tmem_ld16(base + (uint32_t)(kBN * j), v[j]);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < kChunk / 8; ++j)
#pragma unroll
      for (int i = 0; i < kAccCols; ++i) acc[i] += v[j][i];
    fence_before();
  }

  // acc = sum_{k < K} fa(r, k) fb(q, k).  BKC: fb is read k-fastest across
  // threads (operand stored k-contiguous), else q-fastest.
  template <bool BKC, typename FA, typename FB>
  __device__ __forceinline__ void load_chunk(int K, int k0, FA& fa, FB& fb, float (&va)[kPerThreadA],
                                             float (&vb)[kPerThreadB]) {
#pragma unroll
    for (int i = 0; i < kPerThreadA; ++i) {
      const int e = threadIdx.x + kThreads * i, r = e >> 5, k = k0 + (e & 31);
      va[i] = k < K ? fa(r, k) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < kPerThreadB; ++i) {
      const int e = threadIdx.x + kThreads * i;
      const int q = BKC ? (e >> 5) : (e & 63), k = k0 + (BKC ? (e & 31) : (e >> 6));
      vb[i] = k < K ? fb(q, k) : 0.f;
    }
  }

  // acc = sum_{k < K} fa(r, k) fb(q, k).  BKC: fb is read k-fastest across
  // threads (operand stored k-contiguous), else q-fastest.  The global loads
  // of chunk ch + 1 are issued right after chunk ch's MMAs, so they are in
  // flight while those MMAs run and chunk ch - 1 is drained.
  template <bool BKC, typename FA, typename FB>
  __device__ void product(int K, FA fa, FB fb) {
    const int nch = K > 0 ? (K + kChunk - 1) / kChunk : 1;
    const uint64_t dA = sw128_desc(su32(ring)), dB = sw128_desc(su32(ring) + PARTS * kABytes);
    float va[kPerThreadA], vb[kPerThreadB];
    load_chunk<BKC>(K, 0, fa, fb, va, vb);
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch & 1;
      // stage s was last read by the MMAs of chunk ch - 2, drained (waited
      // for) by every thread in the previous iteration
      uint8_t* st = ring + s * kStage;
#pragma unroll
      for (int i = 0; i < kPerThreadA; ++i) {
        const int e = threadIdx.x + kThreads * i;
        store_split<PARTS>(st, kABytes, sw128_off(e >> 5, e & 31), va[i]);
      }
#pragma unroll
      for (int i = 0; i < kPerThreadB; ++i) {
        const int e = threadIdx.x + kThreads * i;
        const int q = BKC ? (e >> 5) : (e & 63), kk = BKC ? (e & 31) : (e >> 6);
        store_split<PARTS>(st + PARTS * kABytes, kBBytes, sw128_off(q, kk), vb[i]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        fence_after();
        const uint64_t so = (uint64_t)((s * kStage) >> 4);
#pragma unroll
        for (int j = 0; j < kChunk / 8; ++j)          // 8 TF32 values of K = 32 bytes along the row
#pragma unroll
          for (int t = 0; t < Pairs<PARTS>::n; ++t)
            mma_tf32(tmem + (uint32_t)(kBN * (4 * s + j)),
                     dA + so + (uint64_t)((Pairs<PARTS>::a(t) * kABytes + 32 * j) >> 4),
                     dB + so + (uint64_t)((Pairs<PARTS>::b(t) * kBBytes + 32 * j) >> 4), t > 0 ? 1u : 0u);
        mma_commit(su32(bars + s));
      }
      if (ch + 1 < nch) load_chunk<BKC>(K, (ch + 1) * kChunk, fa, fb, va, vb);
      if (ch >= 1) drain(ch - 1);
    }
    drain(nch - 1);
  }

  // epi(r, q, v) for the 128 x 64 block, consecutive lanes on consecutive q
  // (coalesced along output rows).
  template <typename EPI>
  __device__ void epilogue(EPI epi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, grp = warp >> 2;
    // every MMA has completed: the ring is free.  Warp tile 32 x 16.
    float* tr = reinterpret_cast<float*>(ring) + warp * 32 * (kAccCols + 1);
#pragma unroll
    for (int j = 0; j < kAccCols; ++j) tr[lane * (kAccCols + 1) + j] = acc[j];
    __syncwarp();
    const int rr0 = lane >> 4, q = lane & 15;
#pragma unroll 4
    for (int rr = rr0; rr < 32; rr += 2) epi(32 * quarter + rr, kAccCols * grp + q, tr[rr * (kAccCols + 1) + q]);
  }

  __device__ void finish() {
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
};

// Row block `rb` of the rows below panel p: 128-row blocks of F_II from row
// (p + 1) 64 on, then of F_BI.  Returns false when rb is past both.
struct RowBlock {
  float* base;
  int r0, rows;
  bool inII;
};

__device__ __forceinline__ bool row_block(const TCell& c, float* work, int p, int rb, RowBlock& b) {
  const int oI = (p + 1) * TB;
  const int nbI = c.nI > oI ? (c.nI - oI + kBM - 1) / kBM : 0;
  if (rb < nbI) {
    b.base = work + c.FII;
    b.r0 = oI + kBM * rb;
    b.rows = c.nI;
    b.inII = true;
    return true;
  }
  rb -= nbI;
  if (rb >= (c.nB + kBM - 1) / kBM) return false;
  b.base = work + c.FBI;
  b.r0 = kBM * rb;
  b.rows = c.nB;
  b.inII = false;
  return true;
}

// Panel p: rows below the diagonal tile times D_p^T (in place).
template <int PARTS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_trsm(const TDesc* __restrict__ td, int p,
                                                      float* __restrict__ work, int* status) {
  extern __shared__ uint8_t tc_smem[];
  const TCell c = tcell(td[blockIdx.y]);
  if (p >= c.P) return;
  RowBlock b;
  if (!row_block(c, work, p, blockIdx.x, b)) return;
  const int o = p * TB, w = min(TB, c.nI - o), ld = c.nI;
  const float* D = work + c.X + (int64_t)p * TB * TB;
  TcCta<PARTS> cta;
  cta.init(tc_smem, status);
  float* M = b.base;
  const int r0 = b.r0, rows = b.rows;
  cta.template product<true>(
      w, [&](int r, int k) { return r0 + r < rows ? M[(int64_t)(r0 + r) * ld + o + k] : 0.f; },
      [&](int q, int k) { return D[q * TB + k]; });
  cta.epilogue([&](int r, int q, float v) {
    if (r0 + r < rows && q < w) M[(int64_t)(r0 + r) * ld + o + q] = v;
  });
  cta.finish();
}

// Panel p: column tile j = p + 1 + blockIdx.y of the rows below the panel
// (F_II at and below tile j, all of F_BI) minus L_{., p} L_{j, p}^T.
template <int PARTS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_update(const TDesc* __restrict__ td, int p,
                                                        float* __restrict__ work, int* status) {
  extern __shared__ uint8_t tc_smem[];
  const TCell c = tcell(td[blockIdx.z]);
  if (p >= c.P) return;
  const int j = p + 1 + blockIdx.y;
  if (j >= c.P) return;
  RowBlock b;
  if (!row_block(c, work, p, blockIdx.x, b)) return;
  if (b.inII && b.r0 + kBM <= j * TB) return;   // entirely above tile j
  const int o = p * TB, w = min(TB, c.nI - o), ld = c.nI, oc = j * TB;
  const float* FII = work + c.FII;
  TcCta<PARTS> cta;
  cta.init(tc_smem, status);
  float* M = b.base;
  const int r0 = b.r0, rows = b.rows, nI = c.nI;
  const bool inII = b.inII;
  cta.template product<true>(
      w, [&](int r, int k) { return r0 + r < rows ? M[(int64_t)(r0 + r) * ld + o + k] : 0.f; },
      [&](int q, int k) { return oc + q < nI ? FII[(int64_t)(oc + q) * ld + o + k] : 0.f; });
  cta.epilogue([&](int r, int q, float v) {
    const int R = r0 + r, Q = oc + q;
    if (R < rows && Q < nI && (!inII || R >= oc)) M[(int64_t)R * ld + Q] -= v;
  });
  cta.finish();
}

// U -= G G^T for one dense block (G: nB x K row-major with row stride ld, U:
// nB x nB): rows 128 a .. (two row tiles) by column tile bt; tiles strictly
// below the diagonal are mirrored, diagonal tiles written whole.
template <int PARTS>
__device__ __forceinline__ void syrk_block(const float* G, int ld, int K, float* U, int nB, int a, int bt,
                                           int* status, uint8_t* smem) {
  const int r0 = a * kBM, oc = bt * TB;
  TcCta<PARTS> cta;
  cta.init(smem, status);
  cta.template product<true>(
      K, [&](int r, int k) { return r0 + r < nB ? G[(int64_t)(r0 + r) * ld + k] : 0.f; },
      [&](int q, int k) { return oc + q < nB ? G[(int64_t)(oc + q) * ld + k] : 0.f; });
  cta.epilogue([&](int r, int q, float v) {
    const int R = r0 + r, Q = oc + q;
    if (R < nB && Q < nB && R >= oc) {
      const float u = U[(int64_t)R * nB + Q] - v;
      U[(int64_t)R * nB + Q] = u;
      if (R >= oc + TB) U[(int64_t)Q * nB + R] = u;
    }
  });
  cta.finish();
}

// Schur complement of the tiled elimination: U = F_BB - G G^T, G = F_BI.
template <int PARTS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_syrk(const TDesc* __restrict__ td, float* __restrict__ work,
                                                      int* status) {
  extern __shared__ uint8_t tc_smem[];
  const TCell c = tcell(td[blockIdx.z]);
  const int a = blockIdx.x, bt = blockIdx.y;
  if (bt >= c.RB || 2 * a >= c.RB || bt > 2 * a + 1) return;
  syrk_block<PARTS>(work + c.FBI, c.nI, c.nI, work + c.FBB, c.nB, a, bt, status, tc_smem);
}

// The same on nb contiguous blocks: G_b = G + b m k (m x k), U_b = U + b m m.
template <int PARTS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_syrk_flat(const float* __restrict__ G, float* __restrict__ U,
                                                           int m, int k, int* status) {
  extern __shared__ uint8_t tc_smem[];
  const int RB = (m + TB - 1) / TB, a = blockIdx.x, bt = blockIdx.y;
  if (bt >= RB || 2 * a >= RB || bt > 2 * a + 1) return;
  const int64_t b = blockIdx.z;
  syrk_block<PARTS>(G + b * m * k, k, k, U + b * m * m, m, a, bt, status, tc_smem);
}

// ---- check of the bounded wait: a CTA takes its tensor memory and its
// barriers as the Schur update does, issues no MMA, and drains chunk 0 with
// waits of `ns` nanoseconds; the wait gives up (bit 5 of *status), and the
// CTA frees its tensor memory and returns.
__global__ void __launch_bounds__(kThreads, 1) k_wait_test_mma(int* status, uint64_t ns) {
  extern __shared__ uint8_t tc_smem[];
  TcCta<1> cta;
  cta.init(tc_smem, status);
  cta.wait_ns = ns;
  cta.drain(0);
  cta.finish();
}

template <int PARTS>
void set_smem_attr() {
  static std::atomic<bool> done{false};
  if (done) return;
  cudaFuncSetAttribute(k_tc_trsm<PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(PARTS));
  cudaFuncSetAttribute(k_tc_update<PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(PARTS));
  cudaFuncSetAttribute(k_tc_syrk<PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(PARTS));
  cudaFuncSetAttribute(k_tc_syrk_flat<PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(PARTS));
  done = true;
}

int row_blocks(int max_nI, int max_nB, int p) {
  const int oI = (p + 1) * TB;
  return (max_nI > oI ? (max_nI - oI + kBM - 1) / kBM : 0) + (max_nB + kBM - 1) / kBM;
}

template <int PARTS>
long long panel(const TDesc* td, int nsel, int p, int P, int max_nI, int max_nB, float* work, int* status,
                cudaStream_t st) {
  set_smem_attr<PARTS>();
  const int nrb = row_blocks(max_nI, max_nB, p), sm = smem_bytes(PARTS);
  long long nl = 0;
  if (nrb > 0) {
    k_tc_trsm<PARTS><<<dim3(nrb, nsel), kThreads, sm, st>>>(td, p, work, status);
    ++nl;
    if (P - p - 1 > 0) {
      k_tc_update<PARTS><<<dim3(nrb, P - p - 1, nsel), kThreads, sm, st>>>(td, p, work, status);
      ++nl;
    }
  }
  return nl;
}

template <int PARTS>
long long syrk(const TDesc* td, int nsel, int max_nB, float* work, int* status, cudaStream_t st) {
  set_smem_attr<PARTS>();
  const int RB = (max_nB + TB - 1) / TB;
  if (RB == 0) return 0;
  k_tc_syrk<PARTS><<<dim3((RB + 1) / 2, RB, nsel), kThreads, smem_bytes(PARTS), st>>>(td, work, status);
  return 1;
}

template <int PARTS>
void syrk_flat(int nb, int m, int k, const float* G, float* U, int* status, cudaStream_t st) {
  set_smem_attr<PARTS>();
  const int RB = (m + TB - 1) / TB;
  if (nb == 0 || RB == 0) return;
  k_tc_syrk_flat<PARTS><<<dim3((RB + 1) / 2, RB, nb), kThreads, smem_bytes(PARTS), st>>>(G, U, m, k, status);
}

}  // namespace

long long tc_panel(const TDesc* td, int nsel, int p, int P, int max_nI, int max_nB, float* work, int parts,
                   int* status, cudaStream_t st) {
  if (parts >= 3) return panel<3>(td, nsel, p, P, max_nI, max_nB, work, status, st);
  if (parts == 2) return panel<2>(td, nsel, p, P, max_nI, max_nB, work, status, st);
  return panel<1>(td, nsel, p, P, max_nI, max_nB, work, status, st);
}

long long tc_syrk(const TDesc* td, int nsel, int max_nB, float* work, int parts, int* status, cudaStream_t st) {
  if (parts >= 3) return syrk<3>(td, nsel, max_nB, work, status, st);
  if (parts == 2) return syrk<2>(td, nsel, max_nB, work, status, st);
  return syrk<1>(td, nsel, max_nB, work, status, st);
}

void launch_wait_test_mma(int* status, uint64_t ns, cudaStream_t st) {
  static std::atomic<bool> done{false};
  if (!done) {
    cudaFuncSetAttribute(k_wait_test_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(1));
    done = true;
  }
  note_launches(1);
  k_wait_test_mma<<<1, kThreads, smem_bytes(1), st>>>(status, ns);
}

void tc_syrk_flat(int nb, int m, int k, const float* G, float* U, int parts, int* status, cudaStream_t st) {
  if (parts >= 3) return syrk_flat<3>(nb, m, k, G, U, status, st);
  if (parts == 2) return syrk_flat<2>(nb, m, k, G, U, status, st);
  syrk_flat<1>(nb, m, k, G, U, status, st);
}

}  // namespace hif
