// Host-side internals shared by the library's translation units: the error
// type and status helpers, stream-ordered device buffers and pinned upload
// staging, the per-level sweep descriptors, and the handle.  The C ABI
// (include/hif.h) is implemented in hif_api.cu (handles, statistics,
// structure, rank predictor), hif_factor.cu (hif_factor, Algorithms 3.1 /
// 4.1 / 4.2), hif_apply.cu (F^-1 and F, Eq. 4.2, sweep autotuner) and
// hif_solve.cu (CG / GMRES with F^-1, error estimates).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hif.h"
#include "geometry.h"
#include "hif_internal.h"
#include "host_pool.h"
#include "kernels.h"
#include "symbolic3x.h"


namespace hif {
namespace host {

extern thread_local std::string g_last_error;


struct HifError {
  int code;
  std::string msg;
  HifError(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      throw HifError(e_ == cudaErrorMemoryAllocation ? HIF_ERR_OOM : HIF_ERR_CUDA,        \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                     \
  } while (0)

// Keeps up to 8 GB of freed stream-ordered memory in the current device's
// default pool (see hif_factor.cu).
void keep_pool_memory();

// Stream-ordered device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { swap(o); }
  ~DevBuf() { release(); }
  void swap(DevBuf& o) {
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
    std::swap(st, o.st);
  }
  void alloc(size_t b, cudaStream_t s) {
    release();
    st = s;
    bytes = b;
    if (b == 0) return;
    CU(cudaMallocAsync(&p, b, s));
  }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Pinned host staging of the uploads of one factorization.  A copy from
// pageable memory may wait for the stream to drain before it starts, which
// would stop the host from building the next level while the GPU works;
// from pinned memory it is queued like a kernel.  Chunks of pinned memory
// are taken bump-wise and kept for the next factorization (process-wide
// pool); an arena goes back to the pool only after its stream has been
// synchronized, so no copy still reads it.
class PinnedArena {
 public:
  ~PinnedArena() {
    for (Chunk& c : chunks_) cudaFreeHost(c.p);
  }
  void* take(size_t bytes) {
    bytes = (bytes + 15) & ~size_t(15);
    while (cur_ < chunks_.size() && chunks_[cur_].used + bytes > chunks_[cur_].cap) ++cur_;
    if (cur_ == chunks_.size()) {
      Chunk c;
      c.cap = std::max(bytes, kChunk);
      CU(cudaHostAlloc(reinterpret_cast<void**>(&c.p), c.cap, cudaHostAllocDefault));
      chunks_.push_back(c);
    }
    Chunk& c = chunks_[cur_];
    void* r = c.p + c.used;
    c.used += bytes;
    return r;
  }
  void reset() {
    for (Chunk& c : chunks_) c.used = 0;
    cur_ = 0;
  }

 private:
  static constexpr size_t kChunk = 8u << 20;
  struct Chunk {
    char* p = nullptr;
    size_t cap = 0, used = 0;
  };
  std::vector<Chunk> chunks_;
  size_t cur_ = 0;
};

extern std::mutex g_arena_mu;
extern std::vector<std::unique_ptr<PinnedArena>> g_arenas;
extern thread_local PinnedArena* t_arena;   // the calling thread's factorization, if any

// Scope of one factorization on stream st: uploads from this thread go
// through a pinned arena taken from the pool.
struct ArenaScope {
  std::unique_ptr<PinnedArena> a;
  PinnedArena* prev;
  cudaStream_t st;
  explicit ArenaScope(cudaStream_t s) : prev(t_arena), st(s) {
    {
      std::lock_guard<std::mutex> g(g_arena_mu);
      if (!g_arenas.empty()) {
        a = std::move(g_arenas.back());
        g_arenas.pop_back();
      }
    }
    if (!a) a.reset(new PinnedArena());
    t_arena = a.get();
  }
  ~ArenaScope() {
    t_arena = prev;
    if (cudaStreamSynchronize(st) != cudaSuccess) {   // a failed stream: drop the arena's memory
      cudaGetLastError();
      return;
    }
    a->reset();
    std::lock_guard<std::mutex> g(g_arena_mu);
    g_arenas.push_back(std::move(a));
  }
};

template <typename T>
void upload(DevBuf& d, const std::vector<T>& h, cudaStream_t st) {
  const size_t b = h.size() * sizeof(T);
  d.alloc(b, st);
  if (h.empty()) return;
  if (t_arena && b >= 4096) {
    void* p = t_arena->take(b);
    std::memcpy(p, h.data(), b);
    CU(cudaMemcpyAsync(d.p, p, b, cudaMemcpyHostToDevice, st));
  } else {
    CU(cudaMemcpyAsync(d.p, h.data(), b, cudaMemcpyHostToDevice, st));
  }
}

bool is_device_ptr(const void* p);   // a device or managed allocation

// Apply-side view of one kind of block (cells or fronts) at one level.
struct SweepLevel {
  int nblocks = 0, max_np = 0, max_nq = 0;
  double fac_elems = 0.0;   // factor elements one F^-1 sweep reads (Linv lower, G, T)
  double vec_rows = 0.0;    // vector rows it gathers and writes back (sum of np + nq)
  const ApplyDesc* desc = nullptr;   // device, ApplyDesc[nblocks]
  const int* ipool = nullptr;        // device ids
  DevBuf desc_own, ipool_own;        // owned storage behind desc / ipool when not shared
  DevBuf fac;     // factor pool
  DevBuf fac32;   // float copy (FP32 apply of a double factor, or the root in mixed precision)
  // deterministic scatter of a cell level (ContribPlan): per DOF its rows
  DevBuf cp_ptr, cp_dofs, cp_slots;
  int cp_ndof = 0;
  int64_t cp_rows = 0;   // rows of the contribution buffer the level uses
  // F^-1 with large blocks (nbig > 0): the other blocks' descriptors for the
  // one-block launch, and the large ones (BigBlock) for the many-block one
  int nsmall = 0, small_max_np = 0, small_max_nq = 0;
  DevBuf small_desc;
  int nbig = 0, big_max_np = 0, big_max_nq = 0;
  DevBuf big_desc;
  int64_t big_scr = 0;   // scratch elements of the large blocks
};

// Skeleton structure of one fractional level (for hif_structure).
struct LevelFronts {
  int level = 0;
  std::shared_ptr<const std::vector<HostFront>> fr;
  std::shared_ptr<const std::vector<FrontDesc>> fd;
  std::vector<int> out;     // host copy of the front kernel's outputs
  DevBuf feats;             // rank-predictor features, nf x kFeat floats
};

// Rank-independent structure of level 0 of one grid (cells and the fronts of
// level 1/2 depend only on dim, n and the leaf size): built once, then shared
// read-only by every factorization of that grid.  Its device copies are freed
// with it, when neither the cache nor any handle holds it any more.
struct Level0 {
  Level0() = default;
  Level0(const Level0&) = delete;
  Level0& operator=(const Level0&) = delete;
  ~Level0() {
    void* dev[] = {d_cls0, d_cdesc, d_cipool, d_capply, d_fdesc, d_fip};
    for (void* p : dev)
      if (p) cudaFree(p);
  }
  std::vector<HostCell> cells;
  std::vector<CellDesc> cdesc;
  std::vector<int> cipool;   // host copy of the cells' ids (the deterministic scatter's plan)
  int64_t work_elems = 0, fac_elems = 0;
  int max_nI = 0;
  int cap_max_np = 0, cap_max_nq = 0;
  double cap_fac_elems = 0.0, cap_vec_rows = 0.0;
  std::vector<int> alive1;   // DOFs active after the level-0 elimination
  std::shared_ptr<std::vector<HostFront>> fronts;
  std::shared_ptr<std::vector<FrontDesc>> fdesc;
  int64_t fwork_elems = 0, ffac_elems = 0, fout_elems = 0;
  int max_nc = 0, max_nN = 0;
  int* d_cls0 = nullptr;
  CellDesc* d_cdesc = nullptr;
  int* d_cipool = nullptr;
  ApplyDesc* d_capply = nullptr;
  FrontDesc* d_fdesc = nullptr;
  int* d_fip = nullptr;
};


// Bits of the device status words: a bounded wait ran out (bulk copy into
// shared memory, block-group barrier, tensor-core MMA).
constexpr int kWaitBulk = 8, kWaitGroup = 16, kWaitMma = 32;
void throw_wait_status(int bits);   // throws HIF_ERR_TIMEOUT for the bits set

// Records msg as the calling thread's last error and returns code.
int set_error(int code, const std::string& msg);

// Every entry point that can throw ends its try block with these handlers, so
// that no C++ exception leaves the C ABI: the library's own errors keep their
// status, a failed host allocation is HIF_ERR_OOM and any other host-side
// failure (a thread that cannot start, say) is HIF_ERR_HOST.
#define HIF_CATCH                                                                     \
  catch (const HifError& e) {                                                         \
    return set_error(e.code, e.msg);                                                  \
  }                                                                                   \
  catch (const std::bad_alloc&) {                                                     \
    return set_error(HIF_ERR_OOM, "host allocation failed");                          \
  }                                                                                   \
  catch (const std::exception& e) {                                                   \
    return set_error(HIF_ERR_HOST, std::string("host error: ") + e.what());           \
  }

}  // namespace host
}  // namespace hif

using namespace hif;
using namespace hif::host;

struct hif_handle {
  Geometry G;
  GridInfo gi{};
  int precision = HIF_PREC_FP64;
  int variant = HIF_VARIANT_HIFDE;
  int skip_levels = 0;
  int edge_start = 1;   // HIFDE3X: first level whose edges are skeletonized
  int sketch_power = 0; // power iterations on the randomized ID's sketch
  bool deterministic = false;   // sweeps and root apply without floating-point atomics
  int skel = HIF_SKEL_ID;       // fronts skeletonized by the ID or by the SVD (Section 4.4)
  bool two_sided = false;       // LU elimination, ID of [A_{N,c}; A_{c,N}^T] (the unsymmetric variant)
  double beta[3] = {0.0, 0.0, 0.0};   // two-sided: the convection term beta . grad u
  int64_t big_apply = int64_t(1) << 20;   // F^-1: blocks with np (np + 2 nq) >= this many elements by
                                          // many thread blocks (0: none)
  DevBuf big_scratch;           // their scratch (the largest level's, doubles)
  DevBuf contrib_buf;           // the deterministic scatter's contribution rows (32 doubles each)
  int big_cell = 192;   // cells with at least this many interior DOFs use the tiled elimination
  bool coop_qr = true;  // large fronts: pivoted QR by co-resident block groups
  int tc_split = 3;     // FP32 tiled elimination on the tensor cores: TF32 parts per value (1..3), 0 = SIMT
  bool autotune = true; // time the sweep launch shapes on first use
  int id_mode = HIF_ID_QR;
  int oversample = 10;
  unsigned long long seed = 0;
  double eps = 0.0;
  cudaStream_t st = nullptr;
  cudaStream_t own_stream = nullptr;   // created when the caller passes no stream
  DevBuf a_stag, bnode;
  DevBuf dev_err;   // device status of the apply kernels (bit 3: a bounded wait ran out)
  bool count_sweeps = false;   // while a graph is captured: count sweep bytes and launches, no events
  DevBuf root_scratch;         // the multi-block root apply's y and z (2 |s_L| kRootChunk doubles)
  DevBuf stencil_w; // per-node stencil weights (diagonal and neighbour couplings)
  DevBuf model_bf16; // rank-predictor parameters in BF16 (HIF_ID_LEARNED)
  std::shared_ptr<const Level0> level0;
  std::vector<SweepLevel> cells, fronts;   // levels 0..L-1 (fronts: 2D edges, 3D faces)
  std::vector<SweepLevel> edges;           // levels 0..L-1: hifde3x's edge groups (level l + 2/3)
  SweepLevel root;                         // level L
  std::vector<LevelFronts> finfo;
  int root_size = 0, n_cells = 0, n_fronts = 0, max_rank = 0, near = 0, clamped = 0;
  int sketched = 0, fallback = 0;
  int negative = 0;     // negative pivots (LDL^T of indefinite diagonal blocks)
  double t_fronts_ms = 0.0;
  double t_wall_ms = 0.0, t_wait_ms = 0.0;   // last hif_factor: host wall time, and of it blocked on the device
  long long factor_bytes = 0;
  double factor_flops = 0.0, apply_bytes = 0.0, t_factor_ms = 0.0;
  // optional event timing of the F^-1 sweep launches
  int profile = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double prof_ms = 0.0, prof_bytes = 0.0;
  long long prof_launches = 0;
  // sweep bytes and launches of one replay of the preconditioner graph
  double graph_bytes = 0.0;
  long long graph_launches = 0;
  // ring of per-iteration squared residual norms and r.z (inner CG), written
  // by the last block of the iteration's reductions, so that the host checks
  // an iteration while the next one runs
  double* rr_ring = nullptr;       // mapped pinned memory
  double* rr_ring_dev = nullptr;   // its device address
  cudaEvent_t it_ev[2] = {nullptr, nullptr};
  // inner solver of the refinement steps (HIF_SOLVER_*) and GMRES restart length
  int solver = HIF_SOLVER_AUTO;
  int gmres_m = 50;
  ~hif_handle() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : it_ev)
      if (e) cudaEventDestroy(e);
    if (rr_ring) cudaFreeHost(rr_ring);
  }
};

namespace hif {
namespace host {

// hif_apply.cu
// Separates the large blocks of a level (np (np + 2 nq) >= h->big_apply
// elements, F^-1 only, not in the deterministic mode) from the others; ad:
// the level's descriptors as uploaded to sw.desc.
void split_big(hif_handle* h, SweepLevel& sw, const std::vector<ApplyDesc>& ad, cudaStream_t st);
const float* fac_f32(const SweepLevel& S);   // the factor as the float apply reads it
void demote_factor(hif_handle* h);            // FP32_APPLY: float copy of every block
template <typename T>
void run_apply(hif_handle* h, int mode, T* x, int nrhs);   // F^-1 or F on a packed N x nrhs vector
void resolve_profile(hif_handle* h);          // sum the recorded sweep events
void stage_in(const double* user, int nr, int ld, int64_t N, double* packed, cudaStream_t st, DevBuf& tmp);
void stage_out(const double* packed, int nr, int ld, int64_t N, double* user, cudaStream_t st, DevBuf& tmp);
int check_dev_err(hif_handle* h);             // reads and clears the apply kernels' status

// hif_api.cu: runs task(p) for p < nprob on up to nthreads host threads;
// returns the first failure's status (its message kept) or HIF_OK
int run_batch(int nprob, int nthreads, const std::function<int(int)>& task);

}  // namespace host
}  // namespace hif
