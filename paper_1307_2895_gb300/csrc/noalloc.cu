// hif_residual_norms_noalloc: squared residual norms ||f_r - A x_r||^2 of the
// stencil operator without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// check a solution -- code running inside another library's allocator
// callback or memory-managed region (a re-entrant allocation there can
// deadlock or fragment the pool), and callers that must not let an
// allocation synchronize the device in the middle of a stream of work.  They
// pass only their inputs and the output; the reduction scratch lives in a
// fixed device array of this library.
//
// The scratch is a file-scope __device__ array of kScratchDoubles doubles
// (plus a counter): every GPU that loads the library holds it until the
// process exits.  Every call shares it and it keeps the last call's contents;
// the counter is cleared at the start of each call, the partial sums are
// fully overwritten.  Calls that overlap on the GPU (on different streams, or
// from different threads) race on the scratch and give wrong results.
//
// The first call on a device looks up the scratch's device address with
// cudaGetSymbolAddress while that device is current; make that first call
// before any stream capture begins.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/hif.h"
#include "hif_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 304;                 // fixed grid: 2 blocks per SM
constexpr int kNaMaxRhs = 16;                  // columns per call
constexpr int kScratchDoubles = kNaBlocks * kNaMaxRhs;   // 4864 doubles = 38 KB

struct __align__(256) NaScratch {
  double partials[kScratchDoubles];
  unsigned counter;
};
static __device__ __align__(256) NaScratch g_na_scratch;

std::mutex g_na_mutex;
constexpr int kMaxDevices = 64;
NaScratch* g_na_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double na_bond(const double* a_stag, int dim, int n, int m, int axis, int j0,
                                          int j1, int j2) {
  if (dim == 2) {
    if (axis == 0) return a_stag[(int64_t)(j1 - 1) * n + j0];
    return a_stag[(int64_t)n * m + (int64_t)j1 * m + (j0 - 1)];
  }
  const int64_t blk = (int64_t)n * m * m;
  if (axis == 0) return a_stag[((int64_t)(j2 - 1) * m + (j1 - 1)) * n + j0];
  if (axis == 1) return a_stag[blk + ((int64_t)(j2 - 1) * n + j1) * m + (j0 - 1)];
  return a_stag[2 * blk + ((int64_t)j2 * m + (j1 - 1)) * m + (j0 - 1)];
}

__global__ void k_na_clear(NaScratch* s) { s->counter = 0u; }

// Same arithmetic as the solver's FP64 residual kernel (row form of the
// stencil, per-thread FMA accumulation, block tree, last-block sum in block
// order), writing only the norms.
__global__ void k_residual_norms_na(NaScratch* sc, const double* __restrict__ a_stag,
                                    const double* __restrict__ bnode, const double* __restrict__ f,
                                    const double* __restrict__ x, int dim, int n, int nr, int ld,
                                    double* __restrict__ out) {
  __shared__ double shr[kNaThreads * kNaMaxRhs];
  __shared__ bool last;
  const int m = n - 1;
  const int64_t N = (int64_t)m * m * (dim == 3 ? m : 1);
  const double h2 = (double)n * (double)n;
  const int64_t stride[3] = {1, m, (int64_t)m * m};
  double acc[kNaMaxRhs];
  for (int r = 0; r < kNaMaxRhs; ++r) acc[r] = 0.0;
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < N;
       gid += (int64_t)gridDim.x * blockDim.x) {
    const int jj[3] = {(int)(gid % m) + 1, (int)((gid / m) % m) + 1,
                       dim == 3 ? (int)(gid / ((int64_t)m * m)) + 1 : 1};
    double y[kNaMaxRhs];
    for (int r = 0; r < kNaMaxRhs; ++r) y[r] = 0.0;
    double diag = bnode[gid];
    for (int ax = 0; ax < dim; ++ax) {
      int lo[3] = {jj[0], jj[1], jj[2]};
      lo[ax] -= 1;
      const double alo = na_bond(a_stag, dim, n, m, ax, lo[0], lo[1], lo[2]) * h2;
      const double ahi = na_bond(a_stag, dim, n, m, ax, jj[0], jj[1], jj[2]) * h2;
      diag += alo + ahi;
      if (jj[ax] > 1)
        for (int r = 0; r < nr; ++r) y[r] -= alo * x[(gid - stride[ax]) * ld + r];
      if (jj[ax] < m)
        for (int r = 0; r < nr; ++r) y[r] -= ahi * x[(gid + stride[ax]) * ld + r];
    }
    for (int r = 0; r < nr; ++r) {
      const double v = f[gid * ld + r] - (y[r] + diag * x[gid * ld + r]);
      acc[r] = fma(v, v, acc[r]);
    }
  }
  const int tid = threadIdx.x;
  for (int v = 0; v < nr; ++v) shr[tid * nr + v] = acc[v];
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (tid < s)
      for (int v = 0; v < nr; ++v) shr[tid * nr + v] += shr[(tid + s) * nr + v];
    __syncthreads();
  }
  if (tid < nr) sc->partials[(int64_t)blockIdx.x * nr + tid] = shr[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(&sc->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int v = tid; v < nr; v += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += sc->partials[(int64_t)b * nr + v];
    out[v] = s;
  }
  if (tid == 0) sc->counter = 0u;
}

int na_fail(int code, const char* msg) {
  hif::set_last_error(msg);
  return code;
}

// True if the CUDA runtime reports p as device or managed memory.  The query
// allocates nothing; a pointer it cannot classify (host memory, or no device
// at all) is not device memory.
bool na_on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int hif_residual_norms_noalloc(int dim, int n, const double* a_stag, const double* b,
                                          const double* f, const double* x, int nrhs, int ld,
                                          double* rnorm2, void* stream) {
  if (dim != 2 && dim != 3) return na_fail(HIF_ERR_ARG, "dim must be 2 or 3");
  if (n < 4 || n > (1 << 15)) return na_fail(HIF_ERR_ARG, "n out of range");
  if (!a_stag || !b || !f || !x || !rnorm2) return na_fail(HIF_ERR_ARG, "NULL argument");
  if (nrhs < 1 || nrhs > kNaMaxRhs)
    return na_fail(HIF_ERR_ARG, "nrhs must be in 1..16 (the fixed scratch holds 16 columns per call)");
  if (ld < nrhs) return na_fail(HIF_ERR_ARG, "need ld >= nrhs");
  // The kernel dereferences every array directly (nothing is staged here), so
  // host memory is an argument error, not a fault on the device.
  const void* ptrs[5] = {a_stag, b, f, x, rnorm2};
  const char* names[5] = {"a_stag", "b", "f", "x", "rnorm2"};
  for (int i = 0; i < 5; ++i) {
    if (!na_on_device(ptrs[i])) {
      static thread_local char msg[96];
      snprintf(msg, sizeof msg, "%s is not device memory (this entry point stages nothing)", names[i]);
      return na_fail(HIF_ERR_ARG, msg);
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return na_fail(HIF_ERR_CUDA, "no usable current CUDA device");
  NaScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return na_fail(HIF_ERR_CUDA, "cudaGetSymbolAddress of the residual scratch failed");
      }
      g_na_ptr[dev] = static_cast<NaScratch*>(p);
    }
    sc = g_na_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hif::note_launches(2);
  k_na_clear<<<1, 1, 0, st>>>(sc);
  k_residual_norms_na<<<kNaBlocks, kNaThreads, 0, st>>>(sc, a_stag, b, f, x, dim, n, nrhs, ld, rnorm2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(HIF_ERR_CUDA, cudaGetErrorString(e));
  hif::set_last_error("");
  return HIF_OK;
}
