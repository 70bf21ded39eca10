// C ABI and host driver of the factorization, the apply and the CG solve.
//
// Factorization (Algorithm 3.1 / 4.1), per level l = 0..L-1:
//   host  : index sets of the level-l cells (interior I, boundary B) from the
//           DOFs still active, child maps into the level-(l-1) boundaries
//   device: frontal assembly (stencil at l = 0, extend-add above), then the
//           interior elimination of every cell (Lemma 2.1), one launch each
//   host  : fronts of level l + 1/2
//   device: one launch for every front: ID (Lemma 2.2) + Lemma 2.4
//   host  : read back the ranks and skeletons, drop the redundant DOFs
// then the root D = A_L (a level-L cell without boundary, always FP64).
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

using namespace hif;

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void hif::note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

thread_local std::string g_last_error;

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

// The library's stream-ordered allocations come from the current device's
// default memory pool.  By default that pool returns its memory to the
// system at every synchronization, and the factorization synchronizes once
// per level, so every level would map its buffers afresh; keeping up to
// kPoolKeep bytes of freed memory in the pool (a property of this process's
// pool only) makes the next allocations reuse it, while larger working sets
// (big 3D factorizations) still go back to the system for other users of the
// device, such as a framework's own allocator.
constexpr uint64_t kPoolKeep = uint64_t(8) << 30;
void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> g(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = kPoolKeep;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done.push_back(dev);
}

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

std::mutex g_arena_mu;
std::vector<std::unique_ptr<PinnedArena>> g_arenas;
thread_local PinnedArena* t_arena = nullptr;   // the calling thread's factorization, if any

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

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

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

}  // namespace

struct hif_handle {
  Geometry G;
  GridInfo gi{};
  int precision = HIF_PREC_FP64;
  int variant = HIF_VARIANT_HIFDE;
  int skip_levels = 0;
  int edge_start = 1;   // HIFDE3X: first level whose edges are skeletonized
  int sketch_power = 0; // power iterations on the randomized ID's sketch
  bool deterministic = false;   // sweeps and root apply without floating-point atomics
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

namespace {

void prepare_cells(const Geometry& G, int l, const std::vector<HostCell>& cells,
                   const std::vector<HostCell>* prev, std::vector<CellDesc>& desc, std::vector<int>& ipool,
                   int64_t& work_elems, int64_t& fac_elems, int& max_nI) {
  desc.resize(cells.size());
  work_elems = fac_elems = 0;
  max_nI = 0;
  const bool maps = l > 0 && prev;
  // sizes and offsets in cell order, then the id lists and child maps of the
  // cells in parallel (each cell writes its own range of the pool)
  int64_t p = 0;
  for (size_t i = 0; i < cells.size(); ++i) {
    const HostCell& c = cells[i];
    CellDesc& d = desc[i];
    d.nI = (int)c.I.size();
    d.nB = (int)c.B.size();
    d.cell_lin = (int)i;
    d.ids = p;
    p += d.nI + d.nB;
    d.F = work_elems;
    work_elems += (int64_t)d.nI * d.nI + (int64_t)d.nB * d.nI + (int64_t)d.nB * d.nB + cell_x_elems(d.nI);
    d.fac = fac_elems;
    fac_elems += cell_fac_size(d.nI, d.nB);
    for (int s = 0; s < kMaxChild; ++s) d.child[s] = -1;
    d.cmap = -1;
    if (maps) {
      d.cmap = p;
      p += (int64_t)(d.nI + d.nB) * 8;
    }
    max_nI = std::max(max_nI, d.nI);
  }
  ipool.resize(p);
  const int ncell = (int)cells.size();
  const int T = task_count(p, 32768);
  parallel_tasks(T, [&](int t) {
    int64_t c0, c1;
    task_range(ncell, T, t, c0, c1);
    for (int64_t i = c0; i < c1; ++i) {
      const HostCell& c = cells[i];
      CellDesc& d = desc[i];
      std::copy(c.I.begin(), c.I.end(), ipool.begin() + d.ids);
      std::copy(c.B.begin(), c.B.end(), ipool.begin() + d.ids + d.nI);
      if (maps) build_child_map(G, l, c, (int)i, *prev, ipool.data() + d.cmap, d.child);
    }
  });
}

// Apply descriptors of the cells of a level and the sweep statistics.
void cell_apply_descs(const std::vector<CellDesc>& cd, std::vector<ApplyDesc>& ad, int& max_np, int& max_nq,
                      double& fac_elems, double& vec_rows) {
  ad.clear();
  ad.reserve(cd.size());
  max_np = max_nq = 0;
  fac_elems = vec_rows = 0.0;
  int64_t cslot = 0;
  for (const CellDesc& c : cd) {
    ApplyDesc a;
    a.np = c.nI;
    a.nq = c.nB;
    a.ids = c.ids;
    a.cslot = cslot;
    cslot += c.nB;
    a.Linv = c.fac;
    a.G = c.fac + cell_fac_G(c.nI);
    a.L = c.fac + cell_fac_L(c.nI, c.nB);
    a.T = -1;
    a.S = c.fac + cell_fac_S(c.nI, c.nB);
    ad.push_back(a);
    max_np = std::max(max_np, c.nI);
    max_nq = std::max(max_nq, c.nB);
    if (c.nI > 0) {
      fac_elems += 0.5 * c.nI * (c.nI + 1.0) + (double)c.nB * c.nI;
      vec_rows += c.nI + c.nB;
    }
  }
}

// The deterministic scatter's plan of one cell level (ContribPlan): the
// pairs (boundary DOF, contribution row) of the cells that eliminate
// something, sorted by DOF and, within a DOF, by cell; rows are numbered as
// cell_apply_descs numbers them (cslot).
void build_contrib_plan(const std::vector<CellDesc>& cd, const std::vector<int>& ipool, SweepLevel& sw,
                        cudaStream_t st) {
  std::vector<std::pair<int, int>> pr;
  int64_t row = 0;
  for (const CellDesc& c : cd) {
    if (c.nI > 0)
      for (int s = 0; s < c.nB; ++s) pr.emplace_back(ipool[c.ids + c.nI + s], (int)(row + s));
    row += c.nB;
  }
  if (row > 0x7fffffff) throw HifError(HIF_ERR_ARG, "deterministic mode: too many boundary rows in a level");
  std::sort(pr.begin(), pr.end());
  std::vector<int> ptr, dofs, slots;
  ptr.reserve(pr.size() + 1);
  slots.reserve(pr.size());
  for (size_t k = 0; k < pr.size(); ++k) {
    if (k == 0 || pr[k].first != pr[k - 1].first) {
      ptr.push_back((int)k);
      dofs.push_back(pr[k].first);
    }
    slots.push_back(pr[k].second);
  }
  ptr.push_back((int)pr.size());
  upload(sw.cp_ptr, ptr, st);
  upload(sw.cp_dofs, dofs, st);
  upload(sw.cp_slots, slots, st);
  sw.cp_ndof = (int)dofs.size();
  sw.cp_rows = row;
}

// Descriptors of the fronts of one fractional level.
void prepare_fronts(const std::vector<HostFront>& fr, std::vector<FrontDesc>& fd, std::vector<int>& ip,
                    int64_t& work_elems, int64_t& fac_elems, int64_t& out_elems, int& max_nc, int& max_nN) {
  const int nf = (int)fr.size();
  fd.resize(nf);
  ip.clear();
  work_elems = fac_elems = out_elems = 0;
  max_nc = max_nN = 0;
  for (int f = 0; f < nf; ++f) {
    const HostFront& F = fr[f];
    FrontDesc& d = fd[f];
    d.nc = (int)F.c.size();
    d.nN = (int)F.N.size();
    d.P1 = F.P1;
    d.P2 = F.P2;
    d.ids = (int64_t)ip.size();
    ip.insert(ip.end(), F.c.begin(), F.c.end());
    ip.insert(ip.end(), F.pos1.begin(), F.pos1.end());
    ip.insert(ip.end(), F.pos2.begin(), F.pos2.end());
    ip.insert(ip.end(), F.N.begin(), F.N.end());
    d.out = out_elems;
    out_elems += 1 + 2 * d.nc;
    d.work = work_elems;
    work_elems += 2 * (int64_t)d.nN * d.nc + 4 * (int64_t)d.nc * d.nc;
    d.fac = fac_elems;
    fac_elems += front_fac_size(d.nc);
    max_nc = std::max(max_nc, d.nc);
    max_nN = std::max(max_nN, d.nN);
  }
}

template <typename T>
T* dev_copy(const std::vector<T>& v) {
  T* p = nullptr;
  if (v.empty()) return nullptr;
  CU(cudaMalloc(&p, v.size() * sizeof(T)));
  CU(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

std::mutex g_l0_mutex;
// never destroyed: no device frees run while the process exits
auto& g_l0_cache = *new std::map<std::tuple<int, int, int, int>, std::shared_ptr<Level0>>();

std::shared_ptr<const Level0> get_level0(const Geometry& G) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, G.dim, G.n, G.leaf);
  std::lock_guard<std::mutex> lock(g_l0_mutex);
  auto it = g_l0_cache.find(key);
  if (it != g_l0_cache.end()) return it->second;
  auto L0 = std::make_shared<Level0>();
  std::vector<int> alive(G.N);
  for (int64_t g = 0; g < G.N; ++g) alive[g] = (int)g;
  build_cells(G, 0, alive, L0->cells);
  std::vector<int> cip;
  prepare_cells(G, 0, L0->cells, nullptr, L0->cdesc, cip, L0->work_elems, L0->fac_elems, L0->max_nI);
  std::vector<ApplyDesc> ad;
  cell_apply_descs(L0->cdesc, ad, L0->cap_max_np, L0->cap_max_nq, L0->cap_fac_elems, L0->cap_vec_rows);
  std::vector<char> inner(G.N, 0);
  for (const HostCell& c : L0->cells)
    for (int g : c.I) inner[g] = 1;
  for (int g : alive)
    if (!inner[g]) L0->alive1.push_back(g);
  L0->fronts = std::make_shared<std::vector<HostFront>>();
  L0->fdesc = std::make_shared<std::vector<FrontDesc>>();
  std::vector<int> mark;
  build_fronts(G, 0, L0->alive1, L0->cells, *L0->fronts, mark);
  std::vector<int> fip;
  prepare_fronts(*L0->fronts, *L0->fdesc, fip, L0->fwork_elems, L0->ffac_elems, L0->fout_elems, L0->max_nc,
                 L0->max_nN);
  L0->d_cls0 = dev_copy(G.cls[0]);
  L0->d_cdesc = dev_copy(L0->cdesc);
  L0->d_cipool = dev_copy(cip);
  L0->cipool = cip;
  L0->d_capply = dev_copy(ad);
  L0->d_fdesc = dev_copy(*L0->fdesc);
  L0->d_fip = dev_copy(fip);
  // handles keep their own reference; an evicted entry is freed with its last handle
  if (g_l0_cache.size() >= 64) g_l0_cache.clear();
  g_l0_cache[key] = L0;
  return L0;
}

// The bounded device waits report through status bits; each maps to one
// timeout message, the same wherever the wait runs.
constexpr int kWaitBulk = 8, kWaitGroup = 16, kWaitMma = 32;
void throw_wait_status(int bits) {
  if (bits & kWaitBulk) throw HifError(HIF_ERR_TIMEOUT, "a bounded wait for a bulk copy into shared memory ran out");
  if (bits & kWaitGroup)
    throw HifError(HIF_ERR_TIMEOUT, "a bounded group-barrier wait of the multi-block pivoted QR ran out");
  if (bits & kWaitMma) throw HifError(HIF_ERR_TIMEOUT, "a bounded wait for tensor-core MMAs ran out");
}

// Host-side phase timer of one factorization (HIF_TRACE=1 in the
// environment): each lap(name) adds the time since the previous lap to
// name's total; the totals go to stderr when the factorization ends.
struct HostTrace {
  bool on = false;
  std::chrono::steady_clock::time_point t;
  std::vector<std::pair<const char*, double>> acc;
  HostTrace() {
    const char* e = getenv("HIF_TRACE");
    on = e && e[0] == '1';
    t = std::chrono::steady_clock::now();
  }
  void lap(const char* name) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
    for (auto& a : acc)
      if (a.first == name) {
        a.second += ms;
        return;
      }
    acc.emplace_back(name, ms);
  }
  ~HostTrace() {
    if (!on) return;
    double tot = 0.0;
    for (auto& a : acc) tot += a.second;
    fprintf(stderr, "hif_factor host phases (ms, total %.3f):", tot);
    for (auto& a : acc) fprintf(stderr, " [%s %.3f]", a.first, a.second);
    fprintf(stderr, "\n");
  }
};

template <typename T>
struct Factorizer {
  HostTrace tr;
  hif_handle* h;
  const Geometry& G;
  cudaStream_t st;
  DevBuf status;
  std::vector<char> dead;
  std::vector<int> mark;
  // pivot floor of the safeguarded Cholesky: every block in mixed precision
  // (including the FP64 root, whose entries carry FP32 rounding), none in FP64
  double tau = 0.0;

  // hifde3x: the symbolic stage that follows the factorization (pattern of
  // A_l and every index set from level 1's edges on)
  bool x3 = false;
  std::unique_ptr<Symbolic3x> sym;

  explicit Factorizer(hif_handle* h_) : h(h_), G(h_->G), st(h_->st) {
    tau = (h_->precision == HIF_PREC_MIXED) ? 4e-6 : 0.0;
  }

  // cells built ahead from a superset of the active DOFs: drop the DOFs
  // marked dead since (lists stay ascending)
  void drop_dead(std::vector<HostCell>& cells) {
    const int nc = (int)cells.size();
    const int ntask = task_count(nc, 64);
    parallel_tasks(ntask, [&](int t) {
      int64_t c0, c1;
      task_range(nc, ntask, t, c0, c1);
      for (int64_t c = c0; c < c1; ++c) {
        for (std::vector<int>* v : {&cells[c].I, &cells[c].B}) {
          size_t w = 0;
          for (size_t r = 0; r < v->size(); ++r)
            if (!dead[(*v)[r]]) (*v)[w++] = (*v)[r];
          v->resize(w);
        }
      }
    });
  }

  // the host blocked on the device (the per-level read-backs), timed for
  // hif_stats: stream st, or event e when given
  void wait_device(cudaEvent_t e = nullptr) {
    const auto t0 = std::chrono::steady_clock::now();
    if (e) CU(cudaEventSynchronize(e));
    else CU(cudaStreamSynchronize(st));
    h->t_wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }

  // The symbolic stage follows the box levels: cells eliminated, then the
  // fronts skeletonized with the skeletons the IDs chose (pivot order).
  void sym_cells(const std::vector<HostCell>& cells) {
    if (!sym) return;
    for (const HostCell& c : cells)
      if (!c.I.empty()) sym->eliminate(c.I);
  }
  void sym_fronts() {
    if (!sym) return;
    const LevelFronts& info = h->finfo.back();
    const std::vector<HostFront>& fr = *info.fr;
    const std::vector<FrontDesc>& fd = *info.fd;
    for (size_t f = 0; f < fr.size(); ++f) {
      const int* out = info.out.data() + fd[f].out;
      const std::vector<int> s(out + 1 + fd[f].nc, out + 1 + fd[f].nc + out[0]);
      if (sym->skeletonize(fr[f].c, s) == -2) throw HifError(HIF_ERR_HOST, "symbolic stage out of step with the IDs");
    }
  }

  // hifde3x from level e's edges on (Section 4.5, Algorithm 4.2), on A_l held
  // as one dense matrix of the DOFs active at the hand-over (kernels_dense3x.cu):
  // the edges of level e, then per level l > e the algebraic cells (Lemma
  // 2.1), the faces and the edges (Lemma 2.4), then the root.  cd1 / d_cd1 /
  // ip1 / work1: the level-e cells, their ids and their update matrices
  // after the level-e faces.
  static constexpr double kDenseMaxBytes = 48e9;
  void dense_stage(int e, const std::vector<CellDesc>& cd1, const CellDesc* d_cd1, const int* ip1,
                   DevBuf& work1) {
    const int L = G.L;
    const std::vector<int> act = sym->active();
    const int64_t n_act = (int64_t)act.size();
    if ((double)n_act * (double)n_act * sizeof(T) > kDenseMaxBytes)
      throw HifError(HIF_ERR_ARG, "hifde3x keeps its upper levels as one dense matrix of the DOFs active after "
                                  "the faces of its first edge level: too many of them for this grid");
    std::vector<int> hmap(G.N, -1);
    for (int64_t i = 0; i < n_act; ++i) hmap[act[i]] = (int)i;
    DevBuf dmap, Abuf;
    upload(dmap, hmap, st);
    Abuf.alloc((size_t)(n_act * n_act) * sizeof(T), st);
    CU(cudaMemsetAsync(Abuf.p, 0, Abuf.bytes, st));
    int max_nB = 0;
    for (const CellDesc& c : cd1) max_nB = std::max(max_nB, c.nB);
    launch_dense_from_cells<T, T>(d_cd1, (int)cd1.size(), ip1, work1.as<T>(), max_nB, dmap.as<int>(),
                                  Abuf.as<T>(), n_act, st);
    CU(cudaGetLastError());
    work1.release();
    // the front kernels see A through one cell without interior: U = A, ld = n_act
    CellDesc whole{};
    whole.nI = 0;
    whole.nB = (int)n_act;
    whole.cmap = -1;
    for (int s = 0; s < kMaxChild; ++s) whole.child[s] = -1;
    DevBuf d_whole;
    upload(d_whole, std::vector<CellDesc>{whole}, st);
    std::vector<int> no_alive;
    auto groups = [&](int l, int kind) {
      const std::vector<std::vector<int>> gs = sym->groups(l, kind);
      if (gs.empty()) return;
      auto fr = std::make_shared<std::vector<HostFront>>(gs.size());
      for (size_t g = 0; g < gs.size(); ++g) {   // (the symbolic stage's queries share scratch: one at a time)
        HostFront& F = (*fr)[g];
        F.axis = kind;
        F.P1 = F.P2 = 0;
        F.c = gs[g];
        F.N = sym->neighbors(F.c);
        F.pos1.resize(F.c.size() + F.N.size());
        for (size_t i = 0; i < F.c.size(); ++i) F.pos1[i] = hmap[F.c[i]];
        for (size_t i = 0; i < F.N.size(); ++i) F.pos1[F.c.size() + i] = hmap[F.N[i]];
        F.pos2.assign(F.pos1.size(), -1);
      }
      auto fd = std::make_shared<std::vector<FrontDesc>>();
      std::vector<int> ip;
      int64_t fw = 0, ff = 0, fo = 0;
      int mnc = 0, mnN = 0;
      prepare_fronts(*fr, *fd, ip, fw, ff, fo, mnc, mnN);
      DevBuf d_fd, d_ip;
      upload(d_fd, *fd, st);
      upload(d_ip, ip, st);
      const size_t nfi = h->finfo.size();
      run_fronts(l, d_whole.as<CellDesc>(), Abuf, no_alive, fr, fd, d_fd.as<FrontDesc>(), d_ip.as<int>(), fw, ff, fo,
                 mnc, mnN, kind == 1 ? h->fronts[l] : h->edges[l], 2 * l + (kind == 2 ? 1 : 0));
      if (h->finfo.size() > nfi) sym_fronts();
    };
    groups(e, 2);
    for (int l = e + 1; l < L; ++l) {
      const std::vector<std::vector<int>> P = sym->cells(l);
      std::vector<std::vector<int>> Q(P.size());
      for (size_t i = 0; i < P.size(); ++i) Q[i] = sym->neighbors(P[i]);
      std::vector<CellDesc> cd(P.size());
      std::vector<int> ip;
      int64_t we = 0, fe = 0;
      int max_nF = 0;
      for (size_t i = 0; i < P.size(); ++i) {
        CellDesc& d = cd[i];
        d.nI = (int)P[i].size();
        d.nB = (int)Q[i].size();
        d.cell_lin = (int)i;
        d.ids = (int64_t)ip.size();
        ip.insert(ip.end(), P[i].begin(), P[i].end());
        ip.insert(ip.end(), Q[i].begin(), Q[i].end());
        d.F = we;
        we += (int64_t)d.nI * d.nI + (int64_t)d.nB * d.nI + (int64_t)d.nB * d.nB + cell_x_elems(d.nI);
        d.fac = fe;
        fe += cell_fac_size(d.nI, d.nB);
        d.cmap = -1;
        for (int s = 0; s < kMaxChild; ++s) d.child[s] = -1;
        max_nF = std::max(max_nF, d.nI + d.nB);
      }
      SweepLevel& sw = h->cells[l];
      DevBuf ddesc, cw, selbuf, tdbuf;
      upload(ddesc, cd, st);
      upload(sw.ipool_own, ip, st);
      sw.ipool = sw.ipool_own.as<int>();
      cw.alloc((size_t)we * sizeof(T), st);
      sw.fac.alloc((size_t)fe * sizeof(T), st);
      const CellDesc* dd = ddesc.as<CellDesc>();
      launch_dense_cells<T>(0, dd, (int)cd.size(), sw.ipool, max_nF, dmap.as<int>(), Abuf.as<T>(), n_act,
                            cw.as<T>(), st);
      factor_cells<T>(cd, dd, cw.as<T>(), sw.fac.as<T>(), selbuf, tdbuf);
      launch_dense_cells<T>(1, dd, (int)cd.size(), sw.ipool, max_nF, dmap.as<int>(), Abuf.as<T>(), n_act,
                            cw.as<T>(), st);
      CU(cudaGetLastError());
      std::vector<ApplyDesc> ad;
      cell_apply_descs(cd, ad, sw.max_np, sw.max_nq, sw.fac_elems, sw.vec_rows);
      if (h->deterministic) build_contrib_plan(cd, ip, sw, st);
      sw.nblocks = (int)ad.size();
      upload(sw.desc_own, ad, st);
      sw.desc = sw.desc_own.as<ApplyDesc>();
      account_cells(cd, sizeof(T));
      for (const std::vector<int>& p : P)
        if (!p.empty()) sym->eliminate(p);
      groups(l, 1);
      groups(l, 2);
    }
    // the root: D = A on the DOFs still active, factored in FP64
    const std::vector<int> rt = sym->active();
    std::vector<CellDesc> cd(1);
    CellDesc& r = cd[0];
    r.nI = (int)rt.size();
    r.nB = 0;
    r.ids = 0;
    r.F = 0;
    r.fac = 0;
    r.cmap = -1;
    for (int s = 0; s < kMaxChild; ++s) r.child[s] = -1;
    SweepLevel& sw = h->root;
    DevBuf ddesc, rw, selbuf, tdbuf;
    upload(ddesc, cd, st);
    upload(sw.ipool_own, rt, st);
    sw.ipool = sw.ipool_own.as<int>();
    const int64_t fe = cell_fac_size(r.nI, 0);
    rw.alloc((size_t)((int64_t)r.nI * r.nI + cell_x_elems(r.nI)) * sizeof(double), st);
    sw.fac.alloc((size_t)fe * sizeof(double), st);
    launch_dense_gather_root<T, double>(sw.ipool, r.nI, dmap.as<int>(), Abuf.as<T>(), n_act, rw.as<double>(), st);
    Abuf.release();
    factor_cells<double>(cd, ddesc.as<CellDesc>(), rw.as<double>(), sw.fac.as<double>(), selbuf, tdbuf);
    CU(cudaGetLastError());
    std::vector<ApplyDesc> ad;
    cell_apply_descs(cd, ad, sw.max_np, sw.max_nq, sw.fac_elems, sw.vec_rows);
    sw.nblocks = (int)ad.size();
    upload(sw.desc_own, ad, st);
    sw.desc = sw.desc_own.as<ApplyDesc>();
    account_cells(cd, sizeof(double));
    h->root_size = r.nI;
    if (sizeof(T) == sizeof(float) && fe > 0) {
      sw.fac32.alloc((size_t)fe * sizeof(float), st);
      launch_convert<double, float>(fe, 1, sw.fac.as<double>(), 1, sw.fac32.as<float>(), 1, st);
    }
  }

  // Interior elimination of one level: cells with at least h->big_cell
  // interior DOFs go through the tiled multi-block kernels, the others
  // through the one-block-per-cell kernel.
  template <typename U>
  void factor_cells(const std::vector<CellDesc>& cd, const CellDesc* d_cd, U* work, U* fac, DevBuf& selbuf,
                    DevBuf& tdbuf) {
    std::vector<int> small, big;
    int max_small = 0, max_sB = 0, max_bI = 0, max_bB = 0;
    for (int i = 0; i < (int)cd.size(); ++i) {
      if (cd[i].nI >= h->big_cell && cd[i].nI > 0) {
        big.push_back(i);
        max_bI = std::max(max_bI, cd[i].nI);
        max_bB = std::max(max_bB, cd[i].nB);
      } else {
        small.push_back(i);
        max_small = std::max(max_small, cd[i].nI);
        max_sB = std::max(max_sB, cd[i].nB);
      }
    }
    if (big.empty()) {
      launch_cell_factor<U>(d_cd, nullptr, (int)cd.size(), work, fac, status.as<int>(), max_small, max_sB, tau,
                            st);
      return;
    }
    if (!small.empty()) {
      upload(selbuf, small, st);
      launch_cell_factor<U>(d_cd, selbuf.as<int>(), (int)small.size(), work, fac, status.as<int>(), max_small,
                            max_sB, tau, st);
    }
    std::vector<TDesc> td(big.size());
    for (size_t b = 0; b < big.size(); ++b) {
      const CellDesc& c = cd[big[b]];
      TDesc& t = td[b];
      t.nI = c.nI;
      t.nB = c.nB;
      t.FII = c.F;
      t.FBI = c.F + (int64_t)c.nI * c.nI;
      t.FBB = t.FBI + (int64_t)c.nB * c.nI;
      t.X = t.FBB + (int64_t)c.nB * c.nB;
      t.Linv = c.fac;
      t.G = c.fac + cell_fac_G(c.nI);
      t.Lp = c.fac + cell_fac_L(c.nI, c.nB);
      t.S = c.fac + cell_fac_S(c.nI, c.nB);
    }
    upload(tdbuf, td, st);
    launch_tiled_elim<U>(tdbuf.as<TDesc>(), (int)big.size(), max_bI, max_bB, work, fac, status.as<int>(), tau, st,
                         h->tc_split);
  }

  static int max_front_size(const std::vector<CellDesc>& cd) {
    int m = 0;
    for (const CellDesc& c : cd) m = std::max(m, c.nI + c.nB);
    return m;
  }

  void account_cells(const std::vector<CellDesc>& cd, size_t esz) {
    for (const CellDesc& c : cd) {
      const double nI = c.nI, nB = c.nB;
      if (c.nI == 0) continue;
      // Cholesky nI^3/3, triangular inverse nI^3/3, G = F_BI Linv^T nB nI^2, SYRK nB^2 nI
      h->factor_flops += 2.0 * nI * nI * nI / 3.0 + nB * nI * nI + nB * nB * nI;
      h->apply_bytes += 2.0 * (double)esz * (nI * (nI + 1) / 2 + nB * nI);
      h->factor_bytes += (long long)(esz * (nI * (nI + 1) / 2 + nB * nI));
      h->n_cells += 1;
    }
  }

  void run() {
    const int L = G.L, nchild = 1 << G.dim;
    status.alloc(8 * sizeof(int), st);
    CU(cudaMemsetAsync(status.p, 0, 8 * sizeof(int), st));
    dead.assign(G.N, 0);
    h->cells.resize(L);
    h->fronts.resize(L);
    h->edges.resize(L);
    const bool skel = (h->variant != HIF_VARIANT_MF) && h->eps > 0.0;
    // hifde3x: its levels up to the first one with edges (cells and faces)
    // are hifde3's; the host replays them on the symbolic stage, which then
    // gives every later index set
    x3 = h->variant == HIF_VARIANT_HIFDE3X && h->edge_start < L;
    if (x3) sym.reset(new Symbolic3x(G.n, G.leaf, true));
    std::shared_ptr<const Level0> L0 = get_level0(G);
    h->level0 = L0;

    // ---- level 0: the cached structure
    DevBuf work, prev_work;
    {
      SweepLevel& sw = h->cells[0];
      work.alloc((size_t)L0->work_elems * sizeof(T), st);
      sw.fac.alloc((size_t)L0->fac_elems * sizeof(T), st);
      const int nc0 = (int)L0->cdesc.size();
      launch_leaf_assemble<T>(L0->d_cdesc, nc0, L0->d_cipool, work.as<T>(), h->gi, h->a_stag.as<double>(),
                              h->bnode.as<double>(), L0->d_cls0, G.ncell[0], st);
      DevBuf sel0, td0;
      factor_cells<T>(L0->cdesc, L0->d_cdesc, work.as<T>(), sw.fac.as<T>(), sel0, td0);
      CU(cudaGetLastError());
      sw.nblocks = nc0;
      sw.desc = L0->d_capply;
      sw.ipool = L0->d_cipool;
      sw.max_np = L0->cap_max_np;
      sw.max_nq = L0->cap_max_nq;
      sw.fac_elems = L0->cap_fac_elems;
      sw.vec_rows = L0->cap_vec_rows;
      account_cells(L0->cdesc, sizeof(T));
      if (h->deterministic) build_contrib_plan(L0->cdesc, L0->cipool, sw, st);
      sym_cells(L0->cells);
    }
    tr.lap("level 0 cells");
    std::vector<int> alive = L0->alive1;
    // Host work overlapped with the fronts on the GPU (hifde2 / hifde3):
    // level l + 1's cells are built from the DOFs active before the fronts
    // of level l (their redundant DOFs are dropped once the ranks are read
    // back, which gives the same lists), and level l's apply descriptors are
    // built after level l + 1's cells have been launched.
    const bool overlap = !x3;
    std::vector<HostCell> cells_a, cells_b;
    int spec_level = -1;   // the level whose cells were built ahead
    auto build_ahead = [&](int l1) {
      if (l1 > L) return;
      build_cells(G, l1, alive, (l1 & 1) ? cells_a : cells_b);
      spec_level = l1;
    };
    if (skel && 0 >= h->skip_levels) {
      const size_t nfi = h->finfo.size();
      run_fronts(0, L0->d_cdesc, work, alive, L0->fronts, L0->fdesc, L0->d_fdesc, L0->d_fip, L0->fwork_elems,
                 L0->ffac_elems, L0->fout_elems, L0->max_nc, L0->max_nN, h->fronts[0], 0, overlap,
                 overlap ? std::function<void()>([&] { build_ahead(1); }) : nullptr);
      if (h->finfo.size() > nfi) sym_fronts();
    }
    if (x3 && h->edge_start == 0) {   // hifde3x with edges from level 0 on
      dense_stage(0, L0->cdesc, L0->d_cdesc, L0->d_cipool, work);
      finish_status();
      return;
    }
    const std::vector<HostCell>* prev_cells = &L0->cells;
    const CellDesc* prev_ddesc = L0->d_cdesc;
    DevBuf ddesc_a, ddesc_b;
    prev_work.swap(work);

    // ---- levels 1 .. L (L: the root, a cell without boundary)
    for (int l = 1; l <= L; ++l) {
      const bool is_root = (l == L);
      std::vector<HostCell>& cells = (l & 1) ? cells_a : cells_b;
      DevBuf& ddesc = (l & 1) ? ddesc_a : ddesc_b;
      tr.lap("other");
      if (spec_level == l) drop_dead(cells);   // built ahead: without the redundant DOFs
      else build_cells(G, l, alive, cells);
      spec_level = -1;
      tr.lap("cells build");
      std::vector<CellDesc> cdesc;
      std::vector<int> ipool;
      int64_t work_elems = 0, fac_elems = 0;
      int max_nI = 0;
      prepare_cells(G, l, cells, prev_cells, cdesc, ipool, work_elems, fac_elems, max_nI);
      tr.lap("cells prepare");
      SweepLevel& sw = is_root ? h->root : h->cells[l];
      upload(ddesc, cdesc, st);
      upload(sw.ipool_own, ipool, st);
      sw.ipool = sw.ipool_own.as<int>();
      const int ncells = (int)cells.size();
      const size_t esz = is_root ? sizeof(double) : sizeof(T);
      work.alloc((size_t)work_elems * esz, st);
      sw.fac.alloc((size_t)fac_elems * esz, st);
      const CellDesc* dd = ddesc.as<CellDesc>();
      const int max_nF = max_front_size(cdesc);
      DevBuf selbuf, tdbuf;
      tr.lap("cells upload+alloc");
      if (is_root) {
        launch_extend_add<T, double>(dd, ncells, sw.ipool, work.as<double>(), prev_ddesc, prev_work.as<T>(),
                                     nchild, max_nF, st);
        factor_cells<double>(cdesc, dd, work.as<double>(), sw.fac.as<double>(), selbuf, tdbuf);
      } else {
        launch_extend_add<T, T>(dd, ncells, sw.ipool, work.as<T>(), prev_ddesc, prev_work.as<T>(), nchild, max_nF,
                                st);
        factor_cells<T>(cdesc, dd, work.as<T>(), sw.fac.as<T>(), selbuf, tdbuf);
      }
      CU(cudaGetLastError());
      tr.lap("cells launch");
      finish_fronts();   // the previous fronts' apply descriptors, deferred
      std::vector<ApplyDesc> ad;
      cell_apply_descs(cdesc, ad, sw.max_np, sw.max_nq, sw.fac_elems, sw.vec_rows);
      if (h->deterministic && !is_root) build_contrib_plan(cdesc, ipool, sw, st);
      sw.nblocks = (int)ad.size();
      upload(sw.desc_own, ad, st);
      sw.desc = sw.desc_own.as<ApplyDesc>();
      account_cells(cdesc, esz);
      prev_work.release();           // the level l-1 updates have been consumed
      if (is_root) {
        h->root_size = cdesc.empty() ? 0 : cdesc[0].nI;
        if (sizeof(T) == sizeof(float) && fac_elems > 0) {
          sw.fac32.alloc((size_t)fac_elems * sizeof(float), st);
          launch_convert<double, float>(fac_elems, 1, sw.fac.as<double>(), 1, sw.fac32.as<float>(), 1, st);
        }
        work.release();
        break;
      }
      tr.lap("cells post");
      sym_cells(cells);
      {   // the eliminated interiors leave the active set
        for (const HostCell& c : cells)
          for (int g : c.I) dead[g] = 1;
        std::vector<int> next;
        next.reserve(alive.size());
        for (int g : alive)
          if (!dead[g]) next.push_back(g);
        alive.swap(next);
      }
      if (skel && l >= h->skip_levels) {
        tr.lap("alive");
        auto fr = std::make_shared<std::vector<HostFront>>();
        build_fronts(G, l, alive, cells, *fr, mark);
        tr.lap("fronts build");
        auto fd = std::make_shared<std::vector<FrontDesc>>();
        std::vector<int> ip;
        int64_t fw = 0, ff = 0, fo = 0;
        int mnc = 0, mnN = 0;
        prepare_fronts(*fr, *fd, ip, fw, ff, fo, mnc, mnN);
        tr.lap("fronts prepare");
        DevBuf d_fd, d_ip;
        upload(d_fd, *fd, st);
        upload(d_ip, ip, st);
        tr.lap("fronts upload");
        const size_t nfi = h->finfo.size();
        run_fronts(l, dd, work, alive, fr, fd, d_fd.as<FrontDesc>(), d_ip.as<int>(), fw, ff, fo, mnc, mnN,
                   h->fronts[l], h->variant == HIF_VARIANT_HIFDE3X ? 2 * l : l, overlap,
                   overlap ? std::function<void()>([&, l] { build_ahead(l + 1); }) : nullptr);
        if (h->finfo.size() > nfi) sym_fronts();
      }
      if (x3 && l == h->edge_start) {   // hifde3x: the assembled upper levels from these edges on
        dense_stage(l, cdesc, dd, sw.ipool, work);
        break;
      }
      prev_cells = &cells;
      prev_ddesc = dd;
      prev_work.swap(work);
    }
    finish_status();
  }

  // The factorization's device status: counts for hif_stats, then the
  // failures (a non-positive pivot, a bounded wait that ran out).
  void finish_status() {
    finish_fronts();
    tr.lap("other");
    int hs2[5] = {0, 0, 0, 0, 0};
    CU(cudaMemcpyAsync(hs2, status.p, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    wait_device();
    const int hs = hs2[0];
    h->clamped = hs2[1];
    h->sketched = hs2[2];
    h->fallback = hs2[3];
    h->negative = hs2[4];
    if (hs & 1) throw HifError(HIF_ERR_NOT_SPD, "non-positive pivot in a diagonal-block Cholesky");
    throw_wait_status(hs & (kWaitGroup | kWaitMma));
  }

  // One launch for every front of level l + 1/2, then read back ranks and
  // skeletons, build the apply descriptors and drop the redundant DOFs.
  // sw: the sweep level the fronts' factor goes to; frac: the fractional
  // level recorded for hif_structure (l, or 2l / 2l + 1 for hifde3x's faces
  // and edges).
  void run_fronts(int l, const CellDesc* d_cdesc, DevBuf& cwork, std::vector<int>& alive,
                  std::shared_ptr<const std::vector<HostFront>> fr, std::shared_ptr<const std::vector<FrontDesc>> fdp,
                  const FrontDesc* d_fd, const int* d_ip, int64_t work_elems, int64_t fac_elems,
                  int64_t out_elems, int max_nc, int max_nN, SweepLevel& sw, int frac, bool defer = false,
                  const std::function<void()>& overlap = nullptr) {
    const std::vector<FrontDesc>& fd = *fdp;
    const int nf = (int)fd.size();
    if (nf == 0) return;
    DevBuf fwork, obuf, pred, sketch;
    fwork.alloc((size_t)work_elems * sizeof(T), st);
    obuf.alloc((size_t)out_elems * sizeof(int), st);
    sw.fac.alloc((size_t)fac_elems * sizeof(T), st);
    LevelFronts info;
    info.level = frac;
    info.feats.alloc((size_t)nf * kFeat * sizeof(float), st);
    launch_front_features(d_fd, nf, d_ip, h->stencil_w.as<double>(), G.dim, G.n, l, h->eps, info.feats.as<float>(),
                          st);
    if (h->id_mode != HIF_ID_QR) {
      sketch.alloc((size_t)nf * sizeof(int), st);
      if (h->id_mode == HIF_ID_LEARNED) {
        pred.alloc((size_t)nf * sizeof(float), st);
        mlp_predict(info.feats.as<float>(), nf, h->model_bf16.p, pred.as<float>(), st);
      }
      launch_sketch_sizes(d_fd, nf, pred.as<float>(), h->id_mode, h->oversample, sketch.as<int>(), st);
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    CU(cudaEventRecord(e0, st));
    const SketchStream ss{(uint64_t)h->seed, (uint64_t)l * (uint64_t)G.N, (uint64_t)G.N, h->sketch_power};
    // fronts with at least max(big_cell, kBigFrontMin) DOFs: the multi-block
    // skeletonization (its elimination scratch needs |c|^2 >= cell_x_elems(|c|))
    const int big_front = std::max(h->big_cell, kBigFrontMin);
    std::vector<int> small, big;
    int big_nc = 0, big_nN = 0;
    for (int f = 0; f < nf; ++f) {
      if (fd[f].nc >= big_front) {
        big.push_back(f);
        big_nc = std::max(big_nc, fd[f].nc);
        big_nN = std::max(big_nN, fd[f].nN);
      } else {
        small.push_back(f);
      }
    }
    DevBuf d_sel, d_big, bstate, m2part, d_td;
    const int nbig = (int)big.size();
    const int nm = nbig ? bigfront_colmax_blocks(big_nc) : 0;
    if (big.empty()) {
      launch_front<T>(d_fd, nf, d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(), cwork.as<T>(), h->eps,
                      status.as<int>(), max_nc, max_nN, tau, sketch.as<int>(), ss, nullptr, st);
    } else {
      if (!small.empty()) {
        upload(d_sel, small, st);
        int snc = 0, snN = 0;
        for (int f : small) {
          snc = std::max(snc, fd[f].nc);
          snN = std::max(snN, fd[f].nN);
        }
        launch_front<T>(d_fd, (int)small.size(), d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(),
                        cwork.as<T>(), h->eps, status.as<int>(), snc, snN, tau, sketch.as<int>(), ss,
                        d_sel.as<int>(), st);
      }
      upload(d_big, big, st);
      bstate.alloc(sizeof(int) * nbig, st);
      m2part.alloc(sizeof(double) * nbig * nm, st);
      std::vector<int> bnc(nbig), bnN(nbig);
      for (int b = 0; b < nbig; ++b) {
        bnc[b] = fd[big[b]].nc;
        bnN[b] = fd[big[b]].nN;
      }
      launch_bigfront_id<T>(d_fd, d_big.as<int>(), nbig, d_cdesc, d_ip, cwork.as<T>(), fwork.as<T>(), sw.fac.as<T>(),
                            obuf.as<int>(), sketch.as<int>(), ss, h->eps, status.as<int>(), bstate.as<int>(),
                            m2part.as<double>(), nm, big_nc, big_nN,
                            sketch.p ? big_nc : 0, bnc.data(), bnN.data(), h->coop_qr, st);
    }
    CU(cudaGetLastError());
    tr.lap("fronts launch");
    if (overlap) {   // host work that needs no result of these fronts, while they run
      overlap();
      tr.lap("overlap");
    }
    info.fr = fr;
    info.fd = fdp;
    info.out.resize(out_elems);
    CU(cudaMemcpyAsync(info.out.data(), obuf.p, out_elems * sizeof(int), cudaMemcpyDeviceToHost, st));
    int hstat = 0;
    CU(cudaMemcpyAsync(&hstat, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    wait_device();
    tr.lap("fronts readback");
    if (!big.empty()) {
      // ranks known: B_sr, B_rr, A_ss, the tiled elimination, B_ss back
      std::vector<TDesc> td;
      int max_k = 0, max_nR = 0;
      for (int f : big) {
        const FrontDesc& d = fd[f];
        const int k = info.out[d.out];
        const int nR = d.nc - k;
        max_k = std::max(max_k, k);
        max_nR = std::max(max_nR, nR);
        if (nR == 0) continue;
        TDesc t;
        t.nI = nR;
        t.nB = k;
        t.FII = d.work + (int64_t)d.nN * d.nc + (int64_t)d.nc * d.nc;
        t.FBI = t.FII + (int64_t)nR * nR;
        t.FBB = t.FBI + (int64_t)k * nR;
        t.X = t.FII + (int64_t)d.nc * d.nc;
        t.Linv = d.fac;
        t.G = d.fac + front_fac_G(d.nc);
        t.Lp = d.fac + front_fac_L(d.nc);
        t.S = d.fac + front_fac_S(d.nc);
        td.push_back(t);
      }
      launch_bigfront_form<T>(d_fd, d_big.as<int>(), nbig, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(), max_k,
                              max_nR, st);
      if (!td.empty()) {
        upload(d_td, td, st);
        launch_tiled_elim<T>(d_td.as<TDesc>(), (int)td.size(), max_nR, max_k, fwork.as<T>(), sw.fac.as<T>(),
                             status.as<int>(), tau, st, h->tc_split);
      }
      launch_bigfront_scatter<T>(d_fd, d_big.as<int>(), nbig, d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(),
                                 cwork.as<T>(), max_k, st);
      CU(cudaGetLastError());
    }
    CU(cudaEventRecord(e1, st));
    wait_device(e1);
    tr.lap("fronts big+event");
    {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      h->t_fronts_ms += ms;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    if (hstat & 2) {
      h->near += 1;
      const int keep = hstat & 1;
      CU(cudaMemcpyAsync(status.p, &keep, sizeof(int), cudaMemcpyHostToDevice, st));
      wait_device();
    }
    fwork.release();
    obuf.release();
    // the redundant DOFs leave the active set: marked now (the next level's
    // cells need it); the apply descriptors follow in finish_fronts, at once
    // or, deferred, after the next level's cells are launched
    for (int f = 0; f < nf; ++f) {
      const FrontDesc& d = fd[f];
      const int* out = info.out.data() + d.out;
      const int* ids_sr = out + 1 + d.nc;
      for (int t = out[0]; t < d.nc; ++t) dead[ids_sr[t]] = 1;
    }
    h->finfo.push_back(std::move(info));
    pend = Pending{true, &sw, &alive, h->finfo.size() - 1, !defer};
    tr.lap("fronts readback post");
    if (!defer) finish_fronts();
  }

  // Apply descriptors of the last skeletonized fractional level: p =
  // redundant (ascending), q = skeletons (pivot order); and, unless the
  // caller drops the dead DOFs itself, the active set without them.
  struct Pending {
    bool on = false;
    SweepLevel* sw = nullptr;
    std::vector<int>* alive = nullptr;
    size_t idx = 0;
    bool filter_alive = true;
  } pend;
  void finish_fronts() {
    if (!pend.on) return;
    pend.on = false;
    SweepLevel& sw = *pend.sw;
    const LevelFronts& info = h->finfo[pend.idx];
    const std::vector<FrontDesc>& fd = *info.fd;
    const int nf = (int)fd.size();
    std::vector<ApplyDesc> ad(nf);
    std::vector<int> aip;
    sw.max_np = sw.max_nq = 0;
    sw.fac_elems = sw.vec_rows = 0.0;
    const double esz = (double)sizeof(T);
    for (int f = 0; f < nf; ++f) {
      const FrontDesc& d = fd[f];
      const int* out = info.out.data() + d.out;
      const int k = out[0];
      const int nR = d.nc - k;
      const int* ids_sr = out + 1 + d.nc;
      ApplyDesc& a = ad[f];
      a.np = nR;
      a.nq = k;
      a.ids = (int64_t)aip.size();
      aip.insert(aip.end(), ids_sr + k, ids_sr + d.nc);
      aip.insert(aip.end(), ids_sr, ids_sr + k);
      a.Linv = d.fac;
      a.G = d.fac + front_fac_G(d.nc);
      a.T = d.fac + front_fac_T(d.nc);
      a.L = d.fac + front_fac_L(d.nc);
      a.S = d.fac + front_fac_S(d.nc);
      a.cslot = 0;
      sw.max_np = std::max(sw.max_np, nR);
      sw.max_nq = std::max(sw.max_nq, k);
      if (nR > 0) {
        sw.fac_elems += 0.5 * nR * (nR + 1.0) + 2.0 * k * nR;
        sw.vec_rows += nR + k;
      }
      h->n_fronts += 1;
      h->max_rank = std::max(h->max_rank, k);
      const double nc = d.nc, nN = d.nN, kk = k, nr = nR;
      // QR (recomputed norms and reflections: ~4 nN nc per step), T, B_rr/B_sr, Cholesky,
      // inverse, G and B_ss
      h->factor_flops += 4.0 * nN * nc * (kk + 1) + kk * kk * nr + 2.0 * kk * kk * nr + 2.0 * kk * nr * nr +
                         2.0 * nr * nr * nr / 3.0 + kk * nr * nr + kk * kk * nr;
      h->apply_bytes += 2.0 * esz * (2 * kk * nr + nr * (nr + 1) / 2);
      h->factor_bytes += (long long)(esz * (2 * kk * nr + nr * (nr + 1) / 2));
    }
    sw.nblocks = nf;
    upload(sw.desc_own, ad, st);
    upload(sw.ipool_own, aip, st);
    sw.desc = sw.desc_own.as<ApplyDesc>();
    sw.ipool = sw.ipool_own.as<int>();
    if (pend.filter_alive) {
      std::vector<int>& alive = *pend.alive;
      std::vector<int> next;
      next.reserve(alive.size());
      for (int g : alive)
        if (!dead[g]) next.push_back(g);
      alive.swap(next);
    }
    tr.lap("fronts post");
  }
};

// ---------------------------------------------------------------------------
// apply of F^-1 / F on a packed N x nrhs work vector of the factor's type
// ---------------------------------------------------------------------------
// The factor as the float apply reads it: the float copy when there is one.
const float* fac_f32(const SweepLevel& S) {
  return S.fac32.p ? S.fac32.as<float>() : S.fac.as<float>();
}

// FP32_APPLY: keep a float copy of every block of the factor, drop the double one.
void demote_factor(hif_handle* h) {
  auto demote = [&](SweepLevel& S) {
    if (!S.fac.p || S.fac32.p) return;
    const int64_t ne = (int64_t)(S.fac.bytes / sizeof(double));
    S.fac32.alloc((size_t)ne * sizeof(float), h->st);
    launch_convert<double, float>(ne, 1, S.fac.as<double>(), 1, S.fac32.as<float>(), 1, h->st);
    S.fac.release();
  };
  for (auto& S : h->cells) demote(S);
  for (auto& S : h->fronts) demote(S);
  for (auto& S : h->edges) demote(S);
  demote(h->root);
  h->factor_bytes /= 2;
  h->apply_bytes /= 2.0;
}

// ---------------------------------------------------------------------------
// Autotuner of the sweep launch shapes.  A launch is identified by what the
// kernels' speed depends on: operation, element type, right-hand sides,
// number of blocks and the largest block (np, nq).  The first eager F^-1
// application that meets a shape times every candidate shape three times on
// a scratch copy of the vectors (CUDA events on the library's stream) and
// keeps the fastest; the built-in shape wins unless another is at least 2%
// faster.  Choices are process-wide, so later factorizations of the same
// grid reuse them, and nothing is timed while a graph is being captured.
// ---------------------------------------------------------------------------
struct TuneKey {
  int op, tsize, nrhs, nblocks, max_np, max_nq, is_front;
  bool operator<(const TuneKey& o) const {
    return std::tie(op, tsize, nrhs, nblocks, max_np, max_nq, is_front) <
           std::tie(o.op, o.tsize, o.nrhs, o.nblocks, o.max_np, o.max_nq, o.is_front);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, SweepShape> g_tune;

template <typename T>
SweepShape tuned_shape(hif_handle* h, int op, const SweepLevel& S, int is_front, const T* fac, const T* x,
                       int nrhs, const ContribPlan* cp) {
  const TuneKey key{op, (int)sizeof(T), nrhs, S.nblocks, S.max_np, S.max_nq, is_front};
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaStream_t st = h->st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return SweepShape{};
  const size_t xb = sizeof(T) * (size_t)h->G.N * nrhs;
  DevBuf xs;
  xs.alloc(xb, st);
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  SweepShape best{};
  float best_ms = 0.f;
  bool first = true;
  for (int staged : {-1, 0})
    for (int threads : {0, 64, 128, 256, 512}) {
      const SweepShape cand{threads, staged};
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CU(cudaMemcpyAsync(xs.p, x, xb, cudaMemcpyDeviceToDevice, st));
        CU(cudaEventRecord(e0, st));
        launch_sweep<T>(op, S.desc, S.nblocks, S.ipool, fac, xs.as<T>(), nrhs, nrhs, is_front, S.max_np, S.max_nq,
                        h->dev_err.as<int>(), st, cand, cp);
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t);
      }
      if (first || ms < 0.98f * best_ms) {
        best = cand;
        best_ms = ms;
        first = false;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[key] = best;
  return best;
}

template <typename T>
void run_apply(hif_handle* h, int mode, T* x, int nrhs) {
  const int L = h->G.L;
  cudaStream_t st = h->st;
  const int up = (mode == HIF_APPLY_FINV) ? 0 : 2;
  const int down = (mode == HIF_APPLY_FINV) ? 1 : 3;
  const bool prof = h->profile && mode == HIF_APPLY_FINV;
  const bool count = prof || (h->count_sweeps && mode == HIF_APPLY_FINV);
  auto sweep_bytes = [&](const SweepLevel& S, int op) {
    // the fused root launch (op 4) does the work of an up and a down sweep
    return (op == 4 ? 2.0 : 1.0) * sizeof(T) * (S.fac_elems + 2.0 * S.vec_rows * nrhs);
  };
  auto sweep = [&](const SweepLevel& S, int op, int is_front, const T* fac) {
    if (S.nblocks == 0) return;
    if (prof) {
      if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
          cudaEvent_t e;
          CU(cudaEventCreate(&e));
          h->ev_pool.push_back(e);
        }
      }
      CU(cudaEventRecord(h->ev_pool[h->ev_used], st));
    }
    // the deterministic scatter of a cell level (its plan; launch_sweep uses
    // it for the sweeps that update x_q of cells)
    ContribPlan cp{S.cp_ptr.as<int>(), S.cp_dofs.as<int>(), S.cp_slots.as<int>(), S.cp_ndof, h->contrib_buf.p};
    const ContribPlan* cpp = (h->deterministic && !is_front && S.cp_ndof > 0) ? &cp : nullptr;
    const SweepShape shape = (h->autotune && mode == HIF_APPLY_FINV)
                                 ? tuned_shape<T>(h, op, S, is_front, fac, x, nrhs, cpp)
                                 : SweepShape{};
    launch_sweep<T>(op, S.desc, S.nblocks, S.ipool, fac, x, nrhs, nrhs, is_front, S.max_np, S.max_nq,
                    h->dev_err.as<int>(), st, shape, cpp);
    if (prof) {
      CU(cudaEventRecord(h->ev_pool[h->ev_used + 1], st));
      h->ev_used += 2;
    }
    if (count) {
      h->prof_launches += 1;
      h->prof_bytes += sweep_bytes(S, op);
    }
  };
  auto facp = [&](const SweepLevel& S) -> const T* {
    if (sizeof(T) == sizeof(float)) return reinterpret_cast<const T*>(fac_f32(S));
    return S.fac.as<T>();
  };
  for (int l = 0; l < L; ++l) {
    sweep(h->cells[l], up, 0, facp(h->cells[l]));
    sweep(h->fronts[l], up, 1, facp(h->fronts[l]));
    if (l < (int)h->edges.size()) sweep(h->edges[l], up, 1, facp(h->edges[l]));
  }
  if (mode == HIF_APPLY_FINV && h->root.nblocks == 1 && h->root.max_np >= kRootMulti && h->root_scratch.p) {
    // a large root: D^-1 by all SMs (the root's factor and ids start at 0)
    const SweepLevel& S = h->root;
    if (prof) {
      if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
          cudaEvent_t e;
          CU(cudaEventCreate(&e));
          h->ev_pool.push_back(e);
        }
      }
      CU(cudaEventRecord(h->ev_pool[h->ev_used], st));
    }
    const int nl = launch_root_apply<T>(S.max_np, S.ipool, facp(S), facp(S) + cell_fac_S(S.max_np, 0), x, nrhs,
                                        nrhs, h->root_scratch.as<T>(), h->deterministic, st);
    if (prof) {
      CU(cudaEventRecord(h->ev_pool[h->ev_used + 1], st));
      h->ev_used += 2;
    }
    if (count) {
      h->prof_launches += nl;
      h->prof_bytes += sweep_bytes(S, 4);
    }
  } else if (mode == HIF_APPLY_FINV) {
    sweep(h->root, 4, 0, facp(h->root));   // D^-1: the root's up and down sweeps in one launch
  } else {
    sweep(h->root, up, 0, facp(h->root));
    sweep(h->root, down, 0, facp(h->root));
  }
  for (int l = L - 1; l >= 0; --l) {
    if (l < (int)h->edges.size()) sweep(h->edges[l], down, 1, facp(h->edges[l]));
    sweep(h->fronts[l], down, 1, facp(h->fronts[l]));
    sweep(h->cells[l], down, 0, facp(h->cells[l]));
  }
}

// Sum the elapsed times of the recorded sweep events (stream already synced).
void resolve_profile(hif_handle* h) {
  for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev_pool[k], h->ev_pool[k + 1]));
    h->prof_ms += ms;
  }
  h->ev_used = 0;
}

// Stage a user vector (host or device, strided) into a packed device array.
struct Staged {
  DevBuf buf;
};

void stage_in(const double* user, int nr, int ld, int64_t N, double* packed, cudaStream_t st,
              DevBuf& tmp) {
  if (is_device_ptr(user)) {
    launch_convert<double, double>(N, nr, user, ld, packed, nr, st);
  } else {
    if (ld == nr) {
      CU(cudaMemcpyAsync(packed, user, sizeof(double) * N * nr, cudaMemcpyHostToDevice, st));
    } else {
      tmp.alloc(sizeof(double) * N * ld, st);
      CU(cudaMemcpyAsync(tmp.p, user, sizeof(double) * ((N - 1) * ld + nr), cudaMemcpyHostToDevice, st));
      launch_convert<double, double>(N, nr, tmp.as<double>(), ld, packed, nr, st);
    }
  }
}

void stage_out(const double* packed, int nr, int ld, int64_t N, double* user, cudaStream_t st,
               DevBuf& tmp) {
  if (is_device_ptr(user)) {
    launch_convert<double, double>(N, nr, packed, nr, user, ld, st);
  } else {
    if (ld == nr) {
      CU(cudaMemcpyAsync(user, packed, sizeof(double) * N * nr, cudaMemcpyDeviceToHost, st));
    } else {
      tmp.alloc(sizeof(double) * N * ld, st);
      CU(cudaMemcpyAsync(tmp.p, user, sizeof(double) * ((N - 1) * ld + nr), cudaMemcpyHostToDevice, st));
      launch_convert<double, double>(N, nr, packed, nr, tmp.as<double>(), ld, st);
      CU(cudaMemcpyAsync(user, tmp.p, sizeof(double) * ((N - 1) * ld + nr), cudaMemcpyDeviceToHost, st));
    }
  }
}

// Solver workspace for one chunk of right-hand sides.  Vectors are N x R,
// R = the chunk's column count rounded up to a power of two (padding columns
// carry a zero right-hand side and stay inactive).
struct SolveWork {
  int64_t N = 0;
  int R = 0;
  bool f32 = false;
  DevBuf f, bin, xh, xl, D, Rv, P, Q, WP, part, scal, cnt;
  double *rzzq[2], *pq, *rr, *alpha, *beta, *thr2, *bn2, *rn2;
  int* active;
  void init(int64_t N_, int R_, bool f32_, cudaStream_t st) {
    N = N_;
    R = R_;
    f32 = f32_;
    const size_t vb = sizeof(double) * N * R;
    f.alloc(vb, st); bin.alloc(vb, st); xh.alloc(vb, st); xl.alloc(vb, st); D.alloc(vb, st);
    Rv.alloc(vb, st); P.alloc(vb, st); Q.alloc(vb, st);
    WP.alloc((f32 ? sizeof(float) : sizeof(double)) * N * R, st);
    part.alloc(sizeof(double) * 4 * kVecBlocksMax * R, st);
    scal.alloc(sizeof(double) * 12 * R + sizeof(int) * R, st);
    cnt.alloc(sizeof(unsigned), st);
    CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned), st));
    CU(cudaMemsetAsync(scal.p, 0, sizeof(double) * 12 * R, st));
    double* s = scal.as<double>();
    rzzq[0] = s; rzzq[1] = s + 2 * R; pq = s + 4 * R; rr = s + 5 * R; alpha = s + 6 * R;
    thr2 = s + 7 * R; bn2 = s + 8 * R; rn2 = s + 9 * R; beta = s + 10 * R;
    active = reinterpret_cast<int*>(s + 12 * R);
  }
};

// Preconditioner z = F^-1 r applied in place on W.WP, replayed from a CUDA
// graph after the first (eager) application.
struct Precond {
  hif_handle* h;
  SolveWork& W;
  cudaGraphExec_t exec = nullptr;
  int calls = 0;
  bool use_graph;
  Precond(hif_handle* h_, SolveWork& W_) : h(h_), W(W_) {
    const char* e = getenv("HIF_NO_GRAPH");
    use_graph = !(e && e[0] == '1');
  }
  ~Precond() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  void eager() {
    if (W.f32) run_apply<float>(h, HIF_APPLY_FINV, W.WP.as<float>(), W.R);
    else run_apply<double>(h, HIF_APPLY_FINV, W.WP.as<double>(), W.R);
  }
  void apply() {
    ++calls;
    if (!use_graph || calls == 1) {
      eager();
      return;
    }
    if (!exec) {
      // capture without sweep events: a replay is timed as one unit.  The
      // events of the eager application stay in the pool; they are resolved
      // with the replays' after the solve has synchronized (settle).
      const int prof = h->profile;
      const double b0 = h->prof_bytes;
      const long long l0 = h->prof_launches;
      h->profile = 0;
      h->count_sweeps = true;   // what one replay moves and launches
      cudaGraph_t g = nullptr;
      CU(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
      try {
        eager();
      } catch (...) {   // leave the stream out of capture mode for later calls
        if (cudaStreamEndCapture(h->st, &g) == cudaSuccess && g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->profile = prof;
        h->count_sweeps = false;
        h->prof_bytes = b0;
        h->prof_launches = l0;
        throw;
      }
      const cudaError_t ce = cudaStreamEndCapture(h->st, &g);
      h->profile = prof;
      h->count_sweeps = false;
      const double gb = h->prof_bytes - b0;
      const long long gl = h->prof_launches - l0;
      h->prof_bytes = b0;
      h->prof_launches = l0;
      cudaError_t e = ce;
      if (ce == cudaSuccess && g) {
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
      }
      if (e != cudaSuccess || !exec) {
        cudaGetLastError();
        exec = nullptr;
        use_graph = false;
        eager();
        return;
      }
      // bytes and launches of one replay (counted while it was captured)
      h->graph_bytes = gb;
      h->graph_launches = gl;
    }
    if (h->profile) {
      while (h->ev_used + 2 > h->ev_pool.size()) {
        cudaEvent_t ev;
        CU(cudaEventCreate(&ev));
        h->ev_pool.push_back(ev);
      }
      CU(cudaEventRecord(h->ev_pool[h->ev_used], h->st));
    }
    CU(cudaGraphLaunch(exec, h->st));
    if (h->profile) {
      CU(cudaEventRecord(h->ev_pool[h->ev_used + 1], h->st));
      h->ev_used += 2;
      ++pending_graphs;
    }
    CU(cudaGetLastError());
  }
  int pending_graphs = 0;
  // after the stream is synchronized: every recorded replay (and eager sweep)
  void settle() {
    if (!h->profile) return;
    resolve_profile(h);
    h->prof_bytes += pending_graphs * h->graph_bytes;
    h->prof_launches += pending_graphs * h->graph_launches;
    pending_graphs = 0;
  }
};

// ring: device pointer of this iteration's row of the host ring (rr, then
// r.z), or null (the last block of the reductions writes it, and the next
// active flags, so no copy or flag kernel is queued)
template <typename TZ>
void cg_step_kernels(hif_handle* h, SolveWork& W, TZ* wp, int par, int restart, int phase,
                     double* partials, unsigned* counter, double* ring = nullptr) {
  const int64_t N = W.N;
  const int R = W.R;
  cudaStream_t st = h->st;
  if (phase == 0) {
    launch_dot2_e<TZ>(N, R, W.Rv.as<double>(), wp, W.Q.as<double>(), partials, counter, W.rzzq[par], st,
                      ring ? ring + R : nullptr, W.alpha, W.rzzq[par ^ 1], W.beta);
    launch_update_p_e<TZ>(N, R, W.P.as<double>(), wp, W.beta, W.rzzq[par ^ 1], W.active, restart, st);
  } else {
    launch_mv_dot_e(h->gi, h->stencil_w.as<double>(), W.P.as<double>(), W.Q.as<double>(), R, partials, counter,
                    W.pq, st, W.rzzq[par], W.active, W.alpha);
    launch_axpy2_e<TZ>(N, R, W.D.as<double>(), W.Rv.as<double>(), W.P.as<double>(), W.Q.as<double>(), W.alpha,
                       partials, counter, W.rr, wp, st, W.thr2, W.active, ring);
  }
}

// Inner PCG on A D = Rv (FP64 recurrences, preconditioner F^-1).  Columns whose
// squared residual is above thr2 are active; a column that drops below it is
// frozen on the device (its updates stop).  The host checks iteration k's
// residuals (written to a ring in mapped pinned memory by the kernels,
// waited for by an event) while iteration k + 1 is already queued, so the GPU
// does not idle on the host; when iteration k converged every column, the
// queued iteration changed nothing.  Stops when the FP64 true residual
// confirms the recursive one.
constexpr int kRingRows = 4;
constexpr int kRingCols = 32;   // rr (R <= 16 values), then r.z of the same iteration

int inner_pcg(hif_handle* h, SolveWork& W, Precond& M, const std::vector<double>& hthr, int maxit,
              bool* broke) {
  const int64_t N = W.N;
  const int R = W.R;
  cudaStream_t st = h->st;
  double* partials = W.part.as<double>();
  unsigned* counter = W.cnt.as<unsigned>();
  const size_t vb = sizeof(double) * N * R;
  if (!h->rr_ring) {
    CU(cudaHostAlloc(&h->rr_ring, sizeof(double) * kRingRows * kRingCols, cudaHostAllocMapped));
    CU(cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->rr_ring_dev), h->rr_ring, 0));
  }
  if (!h->it_ev[0]) {
    CU(cudaEventCreateWithFlags(&h->it_ev[0], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&h->it_ev[1], cudaEventDisableTiming));
  }
  CU(cudaMemcpyAsync(W.thr2, hthr.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(W.bin.p, W.Rv.p, vb, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemsetAsync(W.D.p, 0, vb, st));
  launch_sqnorm(N, R, W.Rv.as<double>(), partials, counter, W.rr, st);
  launch_set_active(R, W.rr, W.thr2, W.active, st);
  auto to_wp = [&]() {
    if (W.f32) launch_convert<double, float>(N, R, W.Rv.as<double>(), R, W.WP.as<float>(), R, st);
    else CU(cudaMemcpyAsync(W.WP.p, W.Rv.p, vb, cudaMemcpyDeviceToDevice, st));
  };
  to_wp();
  std::vector<double> hr(R);
  int it = 0, issued = 0, restarts = 0, par = 0;
  int restart = 1;
  auto converged_row = [&](const double* row) {
    for (int c = 0; c < R; ++c)
      if (row[c] > hthr[c]) return false;
    return true;
  };
  // queue one iteration; false when maxit stops it after the preconditioner
  auto issue = [&]() -> bool {
    double* row = h->rr_ring_dev + (size_t)(issued % kRingRows) * kRingCols;
    M.apply();
    if (W.f32) cg_step_kernels<float>(h, W, W.WP.as<float>(), par, restart, 0, partials, counter, row);
    else cg_step_kernels<double>(h, W, W.WP.as<double>(), par, restart, 0, partials, counter, row);
    restart = 0;
    if (issued >= maxit) return false;
    if (W.f32) cg_step_kernels<float>(h, W, W.WP.as<float>(), par, 0, 1, partials, counter, row);
    else cg_step_kernels<double>(h, W, W.WP.as<double>(), par, 0, 1, partials, counter, row);
    CU(cudaEventRecord(h->it_ev[issued & 1], st));
    ++issued;
    par ^= 1;
    return true;
  };
  // breakdown (the caller may switch to GMRES): r.z <= 0 on a live column
  // (F^-1 not positive definite there), a non-finite residual, or no new
  // smallest residual for kStall iterations
  constexpr int kStall = 50;
  std::vector<double> best(R, 1e300);
  std::vector<int> since(R, 0);
  if (broke) *broke = false;
  auto breakdown = [&](const double* row) {
    for (int c = 0; c < R; ++c) {
      if (hthr[c] >= 1e299) continue;
      const double rr = row[c], rz = row[R + c];
      if (!std::isfinite(rr) || !std::isfinite(rz) || (rz <= 0.0 && rr > hthr[c])) return true;
      if (rr < best[c]) {
        best[c] = rr;
        since[c] = 0;
      } else if (++since[c] >= kStall) {
        return true;
      }
    }
    return false;
  };
  // The iteration queued behind the one that converges runs for nothing;
  // when the last two known residuals predict (at their ratio) that the
  // iteration in flight converges, the next one is held back until its
  // result is known (a wrong guess costs one host round trip).
  std::vector<double> last(R, -1.0), prev(R, -1.0);
  auto predicted = [&]() {
    for (int c = 0; c < R; ++c) {
      if (hthr[c] >= 1e299) continue;
      if (!(last[c] > 0.0 && prev[c] > 0.0)) return false;
      if (last[c] * (last[c] / prev[c]) > hthr[c]) return false;
    }
    return true;
  };
  bool head = issue();                 // iteration `it` queued
  while (true) {
    if (!head) break;                  // maxit
    bool ahead = false, held = false;
    if (predicted()) held = true;
    else ahead = issue();              // iteration it + 1 queued behind it
    CU(cudaGetLastError());
    CU(cudaEventSynchronize(h->it_ev[it & 1]));
    const double* row = h->rr_ring + (size_t)(it % kRingRows) * kRingCols;
    for (int c = 0; c < R; ++c) {
      prev[c] = last[c];
      last[c] = row[c];
    }
    ++it;
    if (broke && breakdown(row)) {
      *broke = true;
      break;
    }
    if (!converged_row(row)) {
      head = held ? issue() : ahead;
      continue;
    }
    // every column below its threshold after iteration `it`; the queued
    // iteration (if any) left them unchanged
    launch_residual(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), W.bin.as<double>(), W.D.as<double>(),
                    W.Rv.as<double>(), R, partials, counter, W.rr, st);
    CU(cudaMemcpyAsync(hr.data(), W.rr, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    M.settle();
    if (converged_row(hr.data()) || ++restarts > 3) break;
    launch_set_active(R, W.rr, W.thr2, W.active, st);
    to_wp();
    restart = 1;
    issued = it;
    std::fill(last.begin(), last.end(), -1.0);
    std::fill(prev.begin(), prev.end(), -1.0);
    head = issue();
  }
  CU(cudaStreamSynchronize(st));
  M.settle();
  return it;
}

// Inner flexible GMRES(m) on A D = W.bin (right-preconditioned by F^-1, each
// column its own Krylov space), to the squared residual thresholds hthr;
// returns the Arnoldi steps taken.  Arnoldi: z_j = F^-1 v_j (kept, in the
// preconditioner's precision), w = A z_j in FP64, classical Gram-Schmidt
// twice against v_0..v_j, v_{j+1} = w / ||w||.  The small Hessenberg least
// squares problem is reduced by Givens rotations on the host; at the end of a
// cycle D += Z y and the true residual W.bin - A D starts the next cycle.
int inner_gmres(hif_handle* h, SolveWork& W, Precond& M, const std::vector<double>& hthr, int maxit) {
  const int64_t N = W.N;
  const int R = W.R;
  const int m = std::max(2, std::min(h->gmres_m, 500));
  cudaStream_t st = h->st;
  const size_t vb = sizeof(double) * N * R, zsz = W.f32 ? sizeof(float) : sizeof(double);
  const int64_t slab = N * R;
  double* partials = W.part.as<double>();
  unsigned* counter = W.cnt.as<unsigned>();
  DevBuf V, Z, hd, mpart, mcnt, tmp, yb;
  V.alloc(vb * (m + 1), st);
  Z.alloc(zsz * slab * m, st);
  hd.alloc(sizeof(double) * (2 * (m + 1) + 1) * R, st);
  mpart.alloc(sizeof(double) * (m + 1) * 304 * R, st);
  mcnt.alloc(sizeof(unsigned) * (m + 1), st);
  CU(cudaMemsetAsync(mcnt.p, 0, sizeof(unsigned) * (m + 1), st));
  if (W.f32) tmp.alloc(vb, st);
  yb.alloc(sizeof(double) * m * R, st);
  double* Vd = V.as<double>();
  double* h1 = hd.as<double>();
  double* h2 = h1 + (m + 1) * R;
  double* hn = h2 + (m + 1) * R;
  CU(cudaMemsetAsync(W.D.p, 0, vb, st));
  CU(cudaMemcpyAsync(W.Rv.p, W.bin.p, vb, cudaMemcpyDeviceToDevice, st));
  launch_sqnorm(N, R, W.Rv.as<double>(), partials, counter, W.rr, st);
  std::vector<double> hr(R), hh(sizeof(double) * (2 * (m + 1) + 1) * R / sizeof(double));
  std::vector<double> H((size_t)R * (m + 1) * m), cs((size_t)R * m), sn((size_t)R * m), g((size_t)R * (m + 1));
  std::vector<double> y((size_t)m * R);
  int it = 0;
  while (true) {
    CU(cudaMemcpyAsync(hr.data(), W.rr, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    bool all = true;
    for (int c = 0; c < R; ++c)
      if (hthr[c] < 1e299 && !(hr[c] <= hthr[c])) all = false;
    if (all || it >= maxit) break;
    launch_normalize(N, R, W.Rv.as<double>(), W.rr, Vd, nullptr, st);
    for (int c = 0; c < R; ++c) {
      std::fill(g.begin() + (size_t)c * (m + 1), g.begin() + (size_t)(c + 1) * (m + 1), 0.0);
      g[(size_t)c * (m + 1)] = hthr[c] < 1e299 ? std::sqrt(hr[c]) : 0.0;
    }
    int j = 0;
    for (; j < m && it < maxit;) {
      ++it;
      double* vj = Vd + (int64_t)j * slab;
      double* w = Vd + (int64_t)(j + 1) * slab;
      if (W.f32) launch_convert<double, float>(N, R, vj, R, W.WP.as<float>(), R, st);
      else CU(cudaMemcpyAsync(W.WP.p, vj, vb, cudaMemcpyDeviceToDevice, st));
      M.apply();
      CU(cudaMemcpyAsync(Z.as<unsigned char>() + zsz * slab * j, W.WP.p, zsz * slab, cudaMemcpyDeviceToDevice, st));
      const double* zj = W.WP.as<double>();
      if (W.f32) {
        launch_convert<float, double>(N, R, W.WP.as<float>(), R, tmp.as<double>(), R, st);
        zj = tmp.as<double>();
      }
      launch_mv_dot_e(h->gi, h->stencil_w.as<double>(), zj, w, R, partials, counter, W.pq, st);
      launch_multi_dot(N, R, Vd, slab, j + 1, w, mpart.as<double>(), mcnt.as<unsigned>(), h1, st);
      launch_multi_axpy(N, R, Vd, slab, j + 1, h1, w, st);
      launch_multi_dot(N, R, Vd, slab, j + 1, w, mpart.as<double>(), mcnt.as<unsigned>(), h2, st);
      launch_multi_axpy(N, R, Vd, slab, j + 1, h2, w, st);
      launch_sqnorm(N, R, w, partials, counter, W.rr, st);
      launch_normalize(N, R, w, W.rr, w, hn, st);
      CU(cudaMemcpyAsync(hh.data(), h1, sizeof(double) * (2 * (m + 1) + 1) * R, cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      CU(cudaGetLastError());
      const double* hh1 = hh.data();
      const double* hh2 = hh1 + (m + 1) * R;
      const double* hhn = hh2 + (m + 1) * R;
      bool conv = true;
      for (int c = 0; c < R; ++c) {
        if (hthr[c] >= 1e299) continue;
        double* col = H.data() + ((size_t)c * m + j) * (m + 1);   // column j of column c's H
        for (int i = 0; i <= j; ++i) col[i] = hh1[i * R + c] + hh2[i * R + c];
        col[j + 1] = hhn[c];
        double* cc = cs.data() + (size_t)c * m;
        double* ss = sn.data() + (size_t)c * m;
        for (int i = 0; i < j; ++i) {   // earlier rotations
          const double t = cc[i] * col[i] + ss[i] * col[i + 1];
          col[i + 1] = -ss[i] * col[i] + cc[i] * col[i + 1];
          col[i] = t;
        }
        const double rho = std::hypot(col[j], col[j + 1]);
        cc[j] = rho > 0.0 ? col[j] / rho : 1.0;
        ss[j] = rho > 0.0 ? col[j + 1] / rho : 0.0;
        col[j] = rho;
        col[j + 1] = 0.0;
        double* gc = g.data() + (size_t)c * (m + 1);
        gc[j + 1] = -ss[j] * gc[j];
        gc[j] = cc[j] * gc[j];
        if (!(gc[j + 1] * gc[j + 1] <= hthr[c])) conv = false;
      }
      ++j;
      if (conv) break;
    }
    // y = H(0:j, 0:j)^-1 g(0:j) per column, D += Z y, true residual
    for (int c = 0; c < R; ++c) {
      const double* gc = g.data() + (size_t)c * (m + 1);
      for (int i = j - 1; i >= 0; --i) {
        double s2 = gc[i];
        for (int k = i + 1; k < j; ++k) s2 -= H[((size_t)c * m + k) * (m + 1) + i] * y[(size_t)k * R + c];
        const double d = H[((size_t)c * m + i) * (m + 1) + i];
        y[(size_t)i * R + c] = (hthr[c] < 1e299 && d != 0.0) ? s2 / d : 0.0;
      }
    }
    CU(cudaMemcpyAsync(yb.p, y.data(), sizeof(double) * j * R, cudaMemcpyHostToDevice, st));
    if (W.f32) launch_zy_add<float>(N, R, Z.as<float>(), slab, j, yb.as<double>(), W.D.as<double>(), st);
    else launch_zy_add<double>(N, R, Z.as<double>(), slab, j, yb.as<double>(), W.D.as<double>(), st);
    launch_residual(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), W.bin.as<double>(), W.D.as<double>(),
                    W.Rv.as<double>(), R, partials, counter, W.rr, st);
    CU(cudaStreamSynchronize(st));   // y is read before the next cycle rewrites it
  }
  M.settle();
  return it;
}

// Outer refinement: x = xh + xl (double-double), r = f - A x evaluated in
// double-double; each step solves A d = r by inner_pcg to a relative
// tolerance tau = max(tol ||f|| / (2 ||r||), 1e-9) and adds d to x.
// rhs, x, xlo: packed N x nr device arrays.
int solve_chunk(hif_handle* h, const double* rhs, double* x, double* xlo, int nr, double tol,
                int maxit, hif_solve_info* info) {
  const int64_t N = h->G.N;
  cudaStream_t st = h->st;
  int R = 1;
  while (R < nr) R <<= 1;
  const size_t vb = sizeof(double) * N * R;
  SolveWork W;
  W.init(N, R, h->precision != HIF_PREC_FP64, st);
  Precond M(h, W);
  double* partials = W.part.as<double>();
  unsigned* counter = W.cnt.as<unsigned>();
  CU(cudaMemsetAsync(W.f.p, 0, vb, st));
  launch_convert<double, double>(N, nr, rhs, nr, W.f.as<double>(), R, st);
  launch_sqnorm(N, R, W.f.as<double>(), partials, counter, W.bn2, st);
  std::vector<double> hb(R), hr(R), hthr(R);
  CU(cudaMemcpyAsync(hb.data(), W.bn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  CU(cudaMemsetAsync(W.xh.p, 0, vb, st));
  CU(cudaMemsetAsync(W.xl.p, 0, vb, st));
  CU(cudaMemsetAsync(W.P.p, 0, vb, st));
  CU(cudaMemsetAsync(W.Q.p, 0, vb, st));
  CU(cudaMemcpyAsync(W.Rv.p, W.f.p, vb, cudaMemcpyDeviceToDevice, st));
  CU(cudaStreamSynchronize(st));
  hr = hb;
  int iters = 0, outer = 0, gmres_iters = 0;
  bool use_gmres = h->solver == HIF_SOLVER_GMRES;
  bool converged = false;
  double relmax = 0.0;
  while (true) {
    bool all = true;
    relmax = 0.0;
    for (int c = 0; c < nr; ++c) {
      const double rel = hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : 0.0;
      relmax = std::max(relmax, rel);
      if (hr[c] > tol * tol * hb[c]) all = false;
    }
    if (all) { converged = true; break; }
    if (iters >= maxit || outer >= 8) break;
    for (int c = 0; c < R; ++c) {
      if (c >= nr || hr[c] <= tol * tol * hb[c]) { hthr[c] = 1e300; continue; }   // column done
      const double tau = std::max(0.5 * tol * std::sqrt(hb[c] / hr[c]), 1e-9);
      hthr[c] = tau * tau * hr[c];
    }
    if (use_gmres) {
      CU(cudaMemcpyAsync(W.bin.p, W.Rv.p, vb, cudaMemcpyDeviceToDevice, st));
      const int g = inner_gmres(h, W, M, hthr, maxit - iters);
      iters += g;
      gmres_iters += g;
    } else {
      bool broke = false;
      iters += inner_pcg(h, W, M, hthr, maxit - iters, h->solver == HIF_SOLVER_AUTO ? &broke : nullptr);
      if (broke) {   // F^-1 indefinite or CG stalled: this step again with GMRES (W.bin holds its right-hand side)
        use_gmres = true;
        const int g = inner_gmres(h, W, M, hthr, maxit - iters);
        iters += g;
        gmres_iters += g;
      }
    }
    CU(cudaGetLastError());
    launch_dd_add(N, R, W.xh.as<double>(), W.xl.as<double>(), W.D.as<double>(), st);
    launch_dd_residual(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), W.f.as<double>(),
                       W.xh.as<double>(), W.xl.as<double>(), W.Rv.as<double>(), R, partials, counter, W.rn2, st);
    CU(cudaMemcpyAsync(hr.data(), W.rn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    ++outer;
  }
  // residual of the FP64-rounded iterate (x_lo dropped)
  CU(cudaMemsetAsync(W.D.p, 0, vb, st));
  launch_dd_residual(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), W.f.as<double>(),
                     W.xh.as<double>(), W.D.as<double>(), W.Q.as<double>(), R, partials, counter, W.rn2, st);
  std::vector<double> h64(R);
  CU(cudaMemcpyAsync(h64.data(), W.rn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  launch_convert<double, double>(N, nr, W.xh.as<double>(), R, x, nr, st);
  if (xlo) launch_convert<double, double>(N, nr, W.xl.as<double>(), R, xlo, nr, st);
  CU(cudaStreamSynchronize(st));
  double rel64 = 0.0;
  for (int c = 0; c < nr; ++c) rel64 = std::max(rel64, hb[c] > 0 ? std::sqrt(h64[c] / hb[c]) : 0.0);
  if (info) {
    info->iters = std::max(info->iters, iters);
    info->gmres_iters = std::max(info->gmres_iters, gmres_iters);
    info->outer = std::max(info->outer, outer);
    info->converged = info->converged && converged;
    info->relres_max = std::max(info->relres_max, relmax);
    info->relres_fp64_max = std::max(info->relres_fp64_max, rel64);
  }
  return converged ? HIF_OK : HIF_ERR_NOCONV;
}

}  // namespace

void hif::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {
// Reads and clears the apply kernels' device status (stream synchronized).
int check_dev_err(hif_handle* h) {
  int e = 0;
  CU(cudaMemcpyAsync(&e, h->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CU(cudaStreamSynchronize(h->st));
  if (e) {
    CU(cudaMemsetAsync(h->dev_err.p, 0, sizeof(int), h->st));
    throw_wait_status(kWaitBulk);
  }
  return HIF_OK;
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// Power iteration ||op|| = lim ||op x|| / ||x|| (Section 5) on device
// N-vectors, from x0, stopped when two successive estimates differ by at most
// rtol of the newer one (or after maxit products).
struct PowerNorm {
  hif_handle* h;
  int64_t N;
  cudaStream_t st;
  DevBuf x, y, t, u, wf, part, cnt, nrm, one;
  explicit PowerNorm(hif_handle* h_) : h(h_), N(h_->G.N), st(h_->st) {
    const size_t vb = sizeof(double) * N;
    x.alloc(vb, st); y.alloc(vb, st); t.alloc(vb, st); u.alloc(vb, st);
    if (h->precision != HIF_PREC_FP64) wf.alloc(sizeof(float) * N, st);
    part.alloc(sizeof(double) * kVecBlocksMax, st);
    cnt.alloc(sizeof(unsigned), st);
    nrm.alloc(sizeof(double), st);
    one.alloc(sizeof(double), st);
    CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned), st));
    const double o = 1.0;
    CU(cudaMemcpyAsync(one.p, &o, sizeof(double), cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  void matvec(const double* in, double* out) {
    launch_matvec(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), in, 1, out, 1, 1, st);
  }
  void fac(int mode, const double* in, double* out) {   // out = F in or F^-1 in
    if (out != in) CU(cudaMemcpyAsync(out, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    if (h->precision != HIF_PREC_FP64) {
      launch_convert<double, float>(N, 1, out, 1, wf.as<float>(), 1, st);
      run_apply<float>(h, mode, wf.as<float>(), 1);
      launch_convert<float, double>(N, 1, wf.as<float>(), 1, out, 1, st);
    } else {
      run_apply<double>(h, mode, out, 1);
    }
  }
  void sub(double* w, const double* v) {   // w -= v
    launch_multi_axpy(N, 1, v, 0, 1, one.as<double>(), w, st);
  }
  double norm(const double* v) {
    launch_sqnorm(N, 1, v, part.as<double>(), cnt.as<unsigned>(), nrm.as<double>(), st);
    double n2 = 0.0;
    CU(cudaMemcpyAsync(&n2, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return std::sqrt(n2);
  }
  // op(in, out) must not write `in`
  template <typename Op>
  double run(const double* x0, double rtol, int maxit, Op op, int& iters) {
    double* X = x.as<double>();
    double* Y = y.as<double>();
    CU(cudaMemcpyAsync(X, x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    norm(X);
    launch_normalize(N, 1, X, nrm.as<double>(), X, nullptr, st);
    double est = 0.0;
    for (iters = 1; iters <= maxit; ++iters) {
      op(X, Y);
      const double ny = norm(Y);
      if (ny == 0.0) return 0.0;
      if (est > 0.0 && std::fabs(ny - est) <= rtol * ny) return ny;
      est = ny;
      launch_normalize(N, 1, Y, nrm.as<double>(), X, nullptr, st);
    }
    return est;
  }
};

extern "C" {

const char* hif_last_error(void) { return g_last_error.c_str(); }

static int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

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

int hif_factor(const hif_grid* grid, const double* a_stag, const double* b, const double* bc_vals,
               double eps, const hif_opts* opts, hif_handle** out) {
  if (!out) return set_error(HIF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !a_stag || !b) return set_error(HIF_ERR_ARG, "grid, a_stag and b are required");
  if (grid->dim != 2 && grid->dim != 3) return set_error(HIF_ERR_ARG, "dim must be 2 or 3");
  if (grid->n < 4 || grid->n > 1 << 15) return set_error(HIF_ERR_ARG, "n out of range");
  if (grid->variant != HIF_VARIANT_MF && grid->variant != HIF_VARIANT_HIFDE && grid->variant != HIF_VARIANT_HIFDE3X)
    return set_error(HIF_ERR_ARG, "unknown variant");
  if (grid->variant == HIF_VARIANT_HIFDE3X && grid->dim != 3)
    return set_error(HIF_ERR_ARG, "HIFDE3X is the 3D variant (dim must be 3)");
  if (bc_vals) return set_error(HIF_ERR_ARG, "only zero Dirichlet data (bc_vals = NULL) is supported");
  if (grid->variant != HIF_VARIANT_MF && !(eps > 0.0 && eps < 1.0))
    return set_error(HIF_ERR_ARG, "eps must be in (0, 1) for HIF-DE");
  const int prec = opts ? opts->precision : HIF_PREC_FP64;
  if (prec != HIF_PREC_FP64 && prec != HIF_PREC_MIXED && prec != HIF_PREC_FP32_APPLY)
    return set_error(HIF_ERR_ARG, "unknown precision");
  const int leaf = grid->leaf > 0 ? grid->leaf : 8;
  if (leaf < 2) return set_error(HIF_ERR_ARG, "leaf must be >= 2");
  hif_handle* h = new hif_handle();
  try {
    keep_pool_memory();
    h->G.init(grid->dim, grid->n, leaf);
    if ((int64_t)h->G.N > (int64_t)0x7fffffff) throw HifError(HIF_ERR_ARG, "grid too large");
    h->gi.dim = grid->dim;
    h->gi.n = grid->n;
    h->gi.m = grid->n - 1;
    h->gi.inv_h2 = (double)grid->n * (double)grid->n;
    h->precision = prec;
    h->variant = grid->variant;
    h->eps = grid->variant != HIF_VARIANT_MF ? eps : 0.0;
    if (grid->variant == HIF_VARIANT_HIFDE3X) {
      // Section 4.5's cells, faces and edges are Voronoi cells about the
      // centers of a tree of 2^L boxes of equal width
      if (grid->n % (1 << h->G.L) != 0)
        throw HifError(HIF_ERR_ARG, "HIFDE3X needs n divisible by 2^L (boxes of equal width)");
      if (opts && opts->skip_levels > 0) throw HifError(HIF_ERR_ARG, "HIFDE3X skips no levels");
    }
    h->skip_levels = opts ? std::max(0, opts->skip_levels) : 0;
    h->id_mode = opts ? opts->id_mode : HIF_ID_QR;
    if (h->id_mode < HIF_ID_QR || h->id_mode > HIF_ID_LEARNED) throw HifError(HIF_ERR_ARG, "unknown id_mode");
    h->oversample = (opts && opts->oversample > 0) ? opts->oversample : 10;
    h->seed = opts ? opts->seed : 0;
    if (opts && opts->big_cell != 0) h->big_cell = opts->big_cell < 0 ? 0x7fffffff : opts->big_cell;
    if (opts) h->tc_split = opts->tensor_cores < 0 ? 0 : opts->tensor_cores == 0 ? 3 : std::min(opts->tensor_cores, 3);
    if (opts) h->autotune = opts->autotune >= 0;
    if (opts) h->edge_start = opts->edge_start == 0 ? 1 : (opts->edge_start < 0 ? 0 : opts->edge_start);
    if (opts && (opts->sketch_power < 0 || opts->sketch_power > 2))
      throw HifError(HIF_ERR_ARG, "sketch_power must be 0, 1 or 2");
    if (opts) h->sketch_power = opts->sketch_power;
    if (opts) h->deterministic = opts->deterministic != 0;
    if (h->id_mode == HIF_ID_LEARNED && !(opts && opts->rank_model))
      throw HifError(HIF_ERR_ARG, "HIF_ID_LEARNED needs opts.rank_model");
    h->st = opts ? (cudaStream_t)opts->stream : nullptr;
    if (!h->st) {
      // a blocking stream: ordered with the legacy default stream like NULL,
      // but capturable into CUDA graphs
      CU(cudaStreamCreate(&h->own_stream));
      h->st = h->own_stream;
    }
    const int64_t na = (int64_t)grid->n * h->G.N / (grid->n - 1) * grid->dim;
    h->dev_err.alloc(sizeof(int), h->st);
    CU(cudaMemsetAsync(h->dev_err.p, 0, sizeof(int), h->st));
    h->a_stag.alloc(sizeof(double) * na, h->st);
    h->bnode.alloc(sizeof(double) * h->G.N, h->st);
    CU(cudaMemcpyAsync(h->a_stag.p, a_stag, sizeof(double) * na, cudaMemcpyDefault, h->st));
    CU(cudaMemcpyAsync(h->bnode.p, b, sizeof(double) * h->G.N, cudaMemcpyDefault, h->st));
    if (h->id_mode == HIF_ID_LEARNED) {
      DevBuf m32;
      m32.alloc(sizeof(float) * kMlpParams, h->st);
      CU(cudaMemcpyAsync(m32.p, opts->rank_model, sizeof(float) * kMlpParams, cudaMemcpyDefault, h->st));
      h->model_bf16.alloc(2 * kMlpParams, h->st);
      mlp_to_bf16(m32.as<float>(), h->model_bf16.p, h->st);
    }
    h->stencil_w.alloc(sizeof(double) * h->G.N * (2 * grid->dim + 1), h->st);
    launch_stencil_weights(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), h->stencil_w.as<double>(), h->st);
    struct Events {   // destroyed on every exit, the failures included
      cudaEvent_t e[2] = {nullptr, nullptr};
      ~Events() {
        for (cudaEvent_t x : e)
          if (x) cudaEventDestroy(x);
      }
    } ev;
    CU(cudaEventCreate(&ev.e[0]));
    CU(cudaEventCreate(&ev.e[1]));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    CU(cudaEventRecord(e0, h->st));
    const auto w0 = std::chrono::steady_clock::now();
    h->t_wait_ms = 0.0;
    ArenaScope arena(h->st);
    if (prec == HIF_PREC_MIXED) {
      Factorizer<float> f(h);
      f.run();
    } else {
      Factorizer<double> f(h);
      f.run();
    }
    if (prec == HIF_PREC_FP32_APPLY) demote_factor(h);
    if (h->root_size >= kRootMulti)
      h->root_scratch.alloc(sizeof(double) * (size_t)root_scratch_elems(h->root_size, h->deterministic), h->st);
    if (h->deterministic) {
      int64_t rows = 0;
      for (const SweepLevel& S : h->cells) rows = std::max(rows, S.cp_rows);
      if (rows > 0) h->contrib_buf.alloc(sizeof(double) * 32 * (size_t)rows, h->st);
    }
    CU(cudaEventRecord(e1, h->st));
    {
      const auto t0 = std::chrono::steady_clock::now();
      CU(cudaEventSynchronize(e1));
      h->t_wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    h->t_wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->t_factor_ms = ms;
  } catch (const HifError& e) {
    hif_free(h);   // also ends the handle's own stream
    return set_error(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    hif_free(h);
    return set_error(HIF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    hif_free(h);
    return set_error(HIF_ERR_HOST, std::string("host error: ") + e.what());
  }
  *out = h;
  g_last_error.clear();
  return HIF_OK;
}

int hif_apply(hif_handle* h, int mode, const double* x, double* y, int nrhs, int ld) {
  if (!h || !x || !y) return set_error(HIF_ERR_ARG, "NULL argument");
  if (mode != HIF_APPLY_F && mode != HIF_APPLY_FINV) return set_error(HIF_ERR_ARG, "bad mode");
  if (nrhs < 1 || ld < nrhs) return set_error(HIF_ERR_ARG, "need 1 <= nrhs <= ld");
  try {
    const int64_t N = h->G.N;
    cudaStream_t st = h->st;
    DevBuf w, tmp, wf;
    w.alloc(sizeof(double) * N * nrhs, st);
    stage_in(x, nrhs, ld, N, w.as<double>(), st, tmp);
    if (h->precision != HIF_PREC_FP64) {
      wf.alloc(sizeof(float) * N * nrhs, st);
      launch_convert<double, float>(N, nrhs, w.as<double>(), nrhs, wf.as<float>(), nrhs, st);
      run_apply<float>(h, mode, wf.as<float>(), nrhs);
      launch_convert<float, double>(N, nrhs, wf.as<float>(), nrhs, w.as<double>(), nrhs, st);
    } else {
      run_apply<double>(h, mode, w.as<double>(), nrhs);
    }
    stage_out(w.as<double>(), nrhs, ld, N, y, st, tmp);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
    if (h->profile) resolve_profile(h);
    check_dev_err(h);
  } HIF_CATCH
  return HIF_OK;
}

int hif_estimate(hif_handle* h, const double* x0, double rtol, int maxit, double* e_a, double* e_s) {
  if (!h || !x0 || !e_a || !e_s) return set_error(HIF_ERR_ARG, "NULL argument");
  if (!(rtol > 0.0) || maxit < 1) return set_error(HIF_ERR_ARG, "need rtol > 0 and maxit >= 1");
  try {
    const int64_t N = h->G.N;
    cudaStream_t st = h->st;
    DevBuf v0, tmp;
    v0.alloc(sizeof(double) * N, st);
    stage_in(x0, 1, 1, N, v0.as<double>(), st, tmp);
    PowerNorm P(h);
    double* T = P.t.as<double>();
    int it = 0;
    const double nA = P.run(v0.as<double>(), rtol, maxit, [&](const double* in, double* out) { P.matvec(in, out); },
                            it);
    const double nE = P.run(v0.as<double>(), rtol, maxit,
                            [&](const double* in, double* out) {   // (A - F) in
                              P.fac(HIF_APPLY_F, in, T);
                              P.matvec(in, out);
                              P.sub(out, T);
                            },
                            it);
    double* U = P.u.as<double>();
    const size_t vb = sizeof(double) * N;
    const double nM = P.run(v0.as<double>(), rtol, maxit,
                            [&](const double* in, double* out) {   // (I - F^-1 A)(I - A F^-1) in
                              P.fac(HIF_APPLY_FINV, in, T);
                              P.matvec(T, out);                    // A F^-1 in
                              CU(cudaMemcpyAsync(U, in, vb, cudaMemcpyDeviceToDevice, st));
                              P.sub(U, out);                       // w = in - A F^-1 in
                              P.matvec(U, T);                      // A w
                              P.fac(HIF_APPLY_FINV, T, T);         // F^-1 A w
                              CU(cudaMemcpyAsync(out, U, vb, cudaMemcpyDeviceToDevice, st));
                              P.sub(out, T);                       // w - F^-1 A w
                            },
                            it);
    *e_a = nA > 0.0 ? nE / nA : 0.0;
    *e_s = std::sqrt(nM);
    check_dev_err(h);
  } HIF_CATCH
  return HIF_OK;
}

int hif_matvec(hif_handle* h, const double* x, double* y, int nrhs, int ld) {
  if (!h || !x || !y) return set_error(HIF_ERR_ARG, "NULL argument");
  if (nrhs < 1 || ld < nrhs || nrhs > 32) return set_error(HIF_ERR_ARG, "need 1 <= nrhs <= min(ld, 32)");
  try {
    const int64_t N = h->G.N;
    cudaStream_t st = h->st;
    DevBuf w, v, tmp;
    w.alloc(sizeof(double) * N * nrhs, st);
    v.alloc(sizeof(double) * N * nrhs, st);
    stage_in(x, nrhs, ld, N, w.as<double>(), st, tmp);
    launch_matvec(h->gi, h->a_stag.as<double>(), h->bnode.as<double>(), w.as<double>(), nrhs,
                  v.as<double>(), nrhs, nrhs, st);
    stage_out(v.as<double>(), nrhs, ld, N, y, st, tmp);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
  } HIF_CATCH
  return HIF_OK;
}

// Boundary terms of the stencil equation (Sections 3.1, 3.2) moved to the
// right-hand side.  Only interior nodes with a coordinate 1 or n-1 have a
// boundary neighbour: the x loop visits x = 1 and x = n-1 alone on rows whose
// y (and z) are away from the boundary.
int hif_rhs_from_bc(const hif_grid* grid, const double* a_stag, const double* bc_vals, double* rhs, int nrhs,
                    int ld) {
  if (!grid || !a_stag || !bc_vals || !rhs) return set_error(HIF_ERR_ARG, "NULL argument");
  const int dim = grid->dim, n = grid->n;
  if (dim != 2 && dim != 3) return set_error(HIF_ERR_ARG, "dim must be 2 or 3");
  if (n < 4 || n > 1 << 15) return set_error(HIF_ERR_ARG, "n out of range");
  if (nrhs < 1 || ld < nrhs) return set_error(HIF_ERR_ARG, "need 1 <= nrhs <= ld");
  const int m = n - 1;
  if ((dim == 3 ? (int64_t)m * m * m : (int64_t)m * m) > (int64_t)0x7fffffff)
    return set_error(HIF_ERR_ARG, "grid too large");
  if (is_device_ptr(a_stag) || is_device_ptr(bc_vals) || is_device_ptr(rhs))
    return set_error(HIF_ERR_ARG, "a_stag, bc_vals and rhs must be in host memory");
  const double inv_h2 = (double)n * (double)n;
  const int64_t blk = (int64_t)n * (dim == 3 ? (int64_t)m * m : m);   // coefficients of one axis
  int c[3] = {1, 1, 1};
  const int zmax = dim == 3 ? m : 1;
  for (c[2] = 1; c[2] <= zmax; ++c[2])
    for (c[1] = 1; c[1] <= m; ++c[1]) {
      const bool near = c[1] == 1 || c[1] == m || (dim == 3 && (c[2] == 1 || c[2] == m));
      for (c[0] = 1; c[0] <= m; c[0] = (near || c[0] == m) ? c[0] + 1 : m) {
        const int64_t j = (c[0] - 1) + (int64_t)m * ((c[1] - 1) + (int64_t)m * (dim == 3 ? c[2] - 1 : 0));
        for (int ax = 0; ax < dim; ++ax)
          for (int side = 0; side < 2; ++side) {
            if (c[ax] != (side == 0 ? 1 : m)) continue;
            // coefficient of the bond to the boundary: extent n on ax (bond 0 or
            // n-1), m on the other axes; boundary node: coordinate 0 or n on ax
            int64_t ai = 0, gi = 0;
            for (int q = dim - 1; q >= 0; --q) {
              ai = ai * (q == ax ? n : m) + (q == ax ? (side == 0 ? 0 : n - 1) : c[q] - 1);
              gi = gi * (n + 1) + (q == ax ? (side == 0 ? 0 : n) : c[q]);
            }
            const double w = inv_h2 * a_stag[ax * blk + ai];
            for (int r = 0; r < nrhs; ++r) rhs[j * ld + r] += w * bc_vals[gi * ld + r];
          }
      }
    }
  return HIF_OK;
}

int hif_solve(hif_handle* h, const double* rhs, double* x, double* x_lo, int nrhs, int ld, double tol,
              int maxit, hif_solve_info* info) {
  if (!h || !rhs || !x) return set_error(HIF_ERR_ARG, "NULL argument");
  if (nrhs < 1 || ld < nrhs) return set_error(HIF_ERR_ARG, "need 1 <= nrhs <= ld");
  if (!(tol > 0.0) || maxit < 0) return set_error(HIF_ERR_ARG, "need tol > 0 and maxit >= 0");
  hif_solve_info loc{0, 0, 1, 0.0, 0.0, 0};
  int rc = HIF_OK;
  try {
    const int64_t N = h->G.N;
    cudaStream_t st = h->st;
    DevBuf pin, pout, plo, tmp;
    for (int r0 = 0; r0 < nrhs; r0 += 16) {
      const int nr = std::min(16, nrhs - r0);
      pin.alloc(sizeof(double) * N * nr, st);
      pout.alloc(sizeof(double) * N * nr, st);
      if (x_lo) plo.alloc(sizeof(double) * N * nr, st);
      stage_in(rhs + r0, nr, ld, N, pin.as<double>(), st, tmp);
      const int rci = solve_chunk(h, pin.as<double>(), pout.as<double>(), x_lo ? plo.as<double>() : nullptr,
                                  nr, tol, maxit, &loc);
      if (rci != HIF_OK) rc = rci;
      stage_out(pout.as<double>(), nr, ld, N, x + r0, st, tmp);
      if (x_lo) stage_out(plo.as<double>(), nr, ld, N, x_lo + r0, st, tmp);
    }
    CU(cudaStreamSynchronize(st));
    if (h->profile) resolve_profile(h);
    check_dev_err(h);
  } HIF_CATCH
  if (info) *info = loc;
  if (rc == HIF_ERR_NOCONV) set_error(rc, "the iteration reached maxit before tol");
  return rc;
}

int hif_autotune_table(int* out, long long cap, long long* count) {
  if (!count) return set_error(HIF_ERR_ARG, "NULL count");
  std::lock_guard<std::mutex> g(g_tune_mu);
  *count = (long long)g_tune.size();
  if (!out) return HIF_OK;
  long long k = 0;
  for (const auto& kv : g_tune) {
    if (k >= cap) break;
    const TuneKey& t = kv.first;
    const int row[9] = {t.op, t.tsize, t.nrhs, t.nblocks, t.max_np, t.max_nq, t.is_front, kv.second.threads,
                        kv.second.staged};
    std::copy(row, row + 9, out + 9 * k);
    ++k;
  }
  return HIF_OK;
}

int hif_set_solver(hif_handle* h, int solver, int restart) {
  if (!h) return set_error(HIF_ERR_ARG, "NULL handle");
  if (solver < HIF_SOLVER_AUTO || solver > HIF_SOLVER_GMRES) return set_error(HIF_ERR_ARG, "unknown solver");
  if (restart != 0 && (restart < 2 || restart > 500)) return set_error(HIF_ERR_ARG, "need 2 <= restart <= 500");
  h->solver = solver;
  h->gmres_m = restart == 0 ? 50 : restart;
  return HIF_OK;
}

int hif_stats(const hif_handle* h, hif_stats_t* s) {
  if (!h || !s) return set_error(HIF_ERR_ARG, "NULL argument");
  s->dim = h->G.dim;
  s->n = h->G.n;
  s->levels = h->G.L;
  s->root_size = h->root_size;
  s->n_cells = h->n_cells;
  s->n_fronts = h->n_fronts;
  s->max_front_rank = h->max_rank;
  s->near_threshold_fronts = h->near;
  s->clamped_pivots = h->clamped;
  s->sketched_fronts = h->sketched;
  s->negative_pivots = h->negative;
  s->fallback_fronts = h->fallback;
  s->t_fronts_ms = h->t_fronts_ms;
  s->t_wall_ms = h->t_wall_ms;
  s->t_wait_ms = h->t_wait_ms;
  s->factor_bytes = h->factor_bytes;
  s->factor_flops = h->factor_flops;
  s->apply_bytes = h->apply_bytes;
  s->t_factor_ms = h->t_factor_ms;
  return HIF_OK;
}

int hif_structure(const hif_handle* h, int32_t* buf, long long cap, long long* needed) {
  if (!h) return set_error(HIF_ERR_ARG, "NULL handle");
  long long need = 2;
  for (const LevelFronts& lf : h->finfo)
    for (size_t f = 0; f < lf.fd->size(); ++f) {
      const FrontDesc& d = (*lf.fd)[f];
      need += 3 + d.nc + lf.out[d.out];
    }
  if (needed) *needed = need;
  if (!buf || cap < need) return HIF_OK;
  long long p = 0;
  for (const LevelFronts& lf : h->finfo)
    for (size_t f = 0; f < lf.fd->size(); ++f) {
      const FrontDesc& d = (*lf.fd)[f];
      const int* out = lf.out.data() + d.out;
      const int k = out[0];
      buf[p++] = lf.level;
      buf[p++] = d.nc;
      buf[p++] = k;
      for (int g : (*lf.fr)[f].c) buf[p++] = g;
      for (int t = 0; t < k; ++t) buf[p++] = out[1 + d.nc + t];
    }
  buf[p++] = -1;
  buf[p++] = h->root_size;
  return HIF_OK;
}

int hif_profile(hif_handle* h, int enable, hif_profile_t* out) {
  if (!h) return set_error(HIF_ERR_ARG, "NULL handle");
  if (out) {
    out->sweep_ms = h->prof_ms;
    out->sweep_launches = h->prof_launches;
    out->sweep_bytes = h->prof_bytes;
  }
  h->prof_ms = 0.0;
  h->prof_bytes = 0.0;
  h->prof_launches = 0;
  h->profile = enable ? 1 : 0;
  return HIF_OK;
}

long long hif_kernel_launches(void) { return g_launches.load(); }

int hif_wait_selftest(int which, long long limit, void* stream) {
  if (which < 0 || which > 2)
    return set_error(HIF_ERR_ARG, "which must be 0 (bulk copy), 1 (group barrier) or 2 (tensor-core MMAs)");
  const long long cap = which == 0 ? (1LL << 26) : which == 1 ? (1LL << 22) : 1000000000LL;
  if (limit < 1 || limit > cap) return set_error(HIF_ERR_ARG, "limit must be in 1 .. the wait's own bound");
  try {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf buf;
    buf.alloc(4 * sizeof(int), st);
    CU(cudaMemsetAsync(buf.p, 0, 4 * sizeof(int), st));
    int* bits = buf.as<int>();
    if (which == 0) launch_wait_test_bulk(bits, (long)limit, st);
    else if (which == 1) launch_wait_test_group(reinterpret_cast<unsigned*>(bits + 2), bits, (long)limit, st);
    else launch_wait_test_mma(bits, (uint64_t)limit, st);
    CU(cudaGetLastError());
    int e = 0;
    CU(cudaMemcpyAsync(&e, bits, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    throw_wait_status(e);
    set_last_error("");
    return HIF_OK;
  }
  HIF_CATCH
}

// Batches: one problem per task, tasks pulled by a small pool of host threads
// (each handle works on its own stream, so different problems overlap).
static int run_batch(int nprob, int nthreads, const std::function<int(int)>& task) {
  int dev = 0;
  cudaGetDevice(&dev);
  nthreads = nthreads <= 0 ? 8 : nthreads;
  nthreads = std::max(1, std::min(nthreads, nprob));
  std::atomic<int> next{0};
  std::mutex mu;
  int first = nprob, first_rc = HIF_OK;
  std::string first_msg;
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int p = next.fetch_add(1); p < nprob; p = next.fetch_add(1)) {
      const int rc = task(p);
      if (rc != HIF_OK) {
        std::lock_guard<std::mutex> lock(mu);
        if (p < first) {
          first = p;
          first_rc = rc;
          try {   // nothing may leave a thread's function
            first_msg = g_last_error;
          } catch (...) {
            first_msg.clear();
          }
        }
      }
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  } catch (const std::exception&) {
    // fewer threads: the tasks are pulled from one counter, so the threads
    // that did start (and this one) take them all
  }
  worker();
  for (std::thread& t : pool) t.join();
  if (first_rc != HIF_OK) return set_error(first_rc, first_msg);
  return HIF_OK;
}

int hif_factor_batch(int nprob, const hif_grid* grids, const double* const* a_stag, const double* const* b,
                     const double* eps, const hif_opts* opts, int nthreads, hif_handle** out) {
  if (nprob < 0 || (nprob > 0 && (!grids || !a_stag || !b || !eps || !out)))
    return set_error(HIF_ERR_ARG, "bad batch arguments");
  for (int p = 0; p < nprob; ++p) out[p] = nullptr;
  try {
    return run_batch(nprob, nthreads, [&](int p) {
      hif_opts o{};
      if (opts) o = *opts;
      o.stream = nullptr;
      return hif_factor(&grids[p], a_stag[p], b[p], nullptr, eps[p], &o, &out[p]);
    });
  } HIF_CATCH
}

int hif_solve_batch(int nprob, hif_handle* const* hs, const double* const* rhs, double* const* x,
                    const int* nrhs, double tol, int maxit, hif_solve_info* infos, int nthreads) {
  if (nprob < 0 || (nprob > 0 && (!hs || !rhs || !x || !nrhs))) return set_error(HIF_ERR_ARG, "bad batch arguments");
  try {
    return run_batch(nprob, nthreads, [&](int p) {
      return hif_solve(hs[p], rhs[p], x[p], nullptr, nrhs[p], nrhs[p], tol, maxit, infos ? &infos[p] : nullptr);
    });
  } HIF_CATCH
}

int hif_front_log(const hif_handle* h, float* feats, int32_t* ranks, int32_t* sizes, long long cap,
                  long long* count) {
  if (!h) return set_error(HIF_ERR_ARG, "NULL handle");
  long long nf = 0;
  for (const LevelFronts& lf : h->finfo) nf += (long long)lf.fd->size();
  if (count) *count = nf;
  if (cap < nf || !feats || !ranks || !sizes) return HIF_OK;
  try {
    long long p = 0;
    for (const LevelFronts& lf : h->finfo) {
      const size_t m = lf.fd->size();
      CU(cudaMemcpyAsync(feats + p * kFeat, lf.feats.p, m * kFeat * sizeof(float), cudaMemcpyDeviceToHost, h->st));
      for (size_t f = 0; f < m; ++f) {
        const FrontDesc& d = (*lf.fd)[f];
        ranks[p + f] = lf.out[d.out];
        sizes[p + f] = d.nc;
      }
      p += (long long)m;
    }
    CU(cudaStreamSynchronize(h->st));
  } HIF_CATCH
  return HIF_OK;
}

int hif_mlp_grad(const float* X, const float* target, int n, const float* params, float* grad, float* loss,
                 void* stream) {
  if (!X || !target || !params || !grad || n < 1) return set_error(HIF_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  try {
    DevBuf partial, ploss;
    const int nblk = mlp_chunks(n);
    partial.alloc(sizeof(float) * (size_t)nblk * kMlpParams, st);
    ploss.alloc(sizeof(float) * nblk, st);
    mlp_grad(X, target, nullptr, n, 1.0f / n, params, partial.as<float>(), ploss.as<float>(), grad, loss, st);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
  } HIF_CATCH
  return HIF_OK;
}

int hif_mlp_train(const float* X, const float* target, int n, float* params, int steps, int batch, float lr,
                  unsigned long long seed, float* loss_hist, void* stream) {
  if (!X || !target || !params || n < 1 || steps < 0 || batch < 1 || !(lr > 0.f))
    return set_error(HIF_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  try {
    batch = std::min(batch, n);
    const int nblk = mlp_chunks(batch);
    DevBuf idx, m, v, grad, partial, ploss, lossd;
    idx.alloc(sizeof(int) * (size_t)n, st);
    m.alloc(sizeof(float) * kMlpParams, st);
    v.alloc(sizeof(float) * kMlpParams, st);
    grad.alloc(sizeof(float) * kMlpParams, st);
    partial.alloc(sizeof(float) * (size_t)nblk * kMlpParams, st);
    ploss.alloc(sizeof(float) * nblk, st);
    lossd.alloc(sizeof(float) * std::max(steps, 1), st);
    CU(cudaMemsetAsync(m.p, 0, sizeof(float) * kMlpParams, st));
    CU(cudaMemsetAsync(v.p, 0, sizeof(float) * kMlpParams, st));
    std::vector<int> perm(n);
    uint64_t state = seed;
    auto next = [&]() {   // splitmix64
      uint64_t z = (state += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    int pos = n;   // forces a shuffle on the first step
    for (int t = 1; t <= steps; ++t) {
      if (pos + batch > n) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int)(next() % (uint64_t)(i + 1))]);
        CU(cudaStreamSynchronize(st));   // the previous upload may still be read
        CU(cudaMemcpyAsync(idx.p, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
        pos = 0;
      }
      mlp_grad(X, target, idx.as<int>() + pos, batch, 1.0f / batch, params, partial.as<float>(), ploss.as<float>(),
               grad.as<float>(), lossd.as<float>() + (t - 1), st);
      mlp_adam(params, grad.as<float>(), m.as<float>(), v.as<float>(), lr, t, st);
      pos += batch;
    }
    if (loss_hist && steps > 0)
      CU(cudaMemcpyAsync(loss_hist, lossd.p, sizeof(float) * steps, cudaMemcpyDeviceToDevice, st));
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
  } HIF_CATCH
  return HIF_OK;
}

int hif_schur_update_f32(int nb, int m, int k, const float* G, float* U, int split, void* stream) {
  if (nb < 0 || m < 0 || k < 0 || nb > 65535 || split < 1 || split > 3)
    return set_error(HIF_ERR_ARG, "bad sizes or split");
  if ((int64_t)nb * m == 0) return HIF_OK;
  if (!U || (!G && k > 0)) return set_error(HIF_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  try {
    DevBuf status;
    status.alloc(sizeof(int), st);
    CU(cudaMemsetAsync(status.p, 0, sizeof(int), st));
    tc_syrk_flat(nb, m, k, G, U, split, status.as<int>(), st);
    CU(cudaGetLastError());
    note_launches(1);
    int hs = 0;
    CU(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    throw_wait_status(hs & kWaitMma);
  } HIF_CATCH
  return HIF_OK;
}

int hif_mlp_predict(const float* X, int n, const float* params, float* y, void* stream) {
  if (!X || !params || !y || n < 0) return set_error(HIF_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  try {
    DevBuf w;
    w.alloc(2 * kMlpParams, st);
    mlp_to_bf16(params, w.p, st);
    mlp_predict(X, n, w.p, y, st);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
  } HIF_CATCH
  return HIF_OK;
}

void hif_free(hif_handle* h) {
  if (!h) return;
  cudaStream_t st = h->st;
  cudaStream_t own = h->own_stream;
  delete h;
  cudaStreamSynchronize(st);
  if (own) cudaStreamDestroy(own);
}

}  // extern "C"
