// hif_factor and hif_factor_batch: the host driver of the factorization.
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
#include <map>

#include "hif_host.h"

namespace hif {
namespace host {

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

std::mutex g_arena_mu;
std::vector<std::unique_ptr<PinnedArena>> g_arenas;
thread_local PinnedArena* t_arena = nullptr;   // the calling thread's factorization, if any

void throw_wait_status(int bits) {
  if (bits & kWaitBulk) throw HifError(HIF_ERR_TIMEOUT, "a bounded wait for a bulk copy into shared memory ran out");
  if (bits & kWaitGroup)
    throw HifError(HIF_ERR_TIMEOUT, "a bounded group-barrier wait of the multi-block pivoted QR ran out");
  if (bits & kWaitMma) throw HifError(HIF_ERR_TIMEOUT, "a bounded wait for tensor-core MMAs ran out");
}

}  // namespace host
}  // namespace hif

namespace {

void prepare_cells(const Geometry& G, int l, const std::vector<HostCell>& cells,
                   const std::vector<HostCell>* prev, std::vector<CellDesc>& desc, std::vector<int>& ipool,
                   int64_t& work_elems, int64_t& fac_elems, int& max_nI, bool two_sided = false) {
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
    if (two_sided) {   // F_IB and its scratch; the second factor set
      d.FIB = work_elems;
      work_elems += cell_work2_size(d.nI, d.nB);
      d.fac2 = fac_elems;
      fac_elems += cell_fac2_size(d.nI, d.nB);
    }
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
    if (c.fac2 >= 0) {   // two-sided
      a.Linv2 = c.fac2;
      a.G2 = c.fac2 + packed_size(c.nI);
      a.L2 = a.G2 + pad4((int64_t)c.nB * c.nI);
    }
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
                    int64_t& work_elems, int64_t& fac_elems, int64_t& out_elems, int& max_nc, int& max_nN,
                    bool two_sided = false) {
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
    // two-sided: the stacked 2|N| x |c| block, A_cc and six |c|^2 scratch blocks
    work_elems += two_sided ? 2 * (int64_t)d.nN * d.nc + 7 * (int64_t)d.nc * d.nc
                            : 2 * (int64_t)d.nN * d.nc + 4 * (int64_t)d.nc * d.nc;
    d.fac = fac_elems;
    fac_elems += front_fac_size(d.nc);
    if (two_sided) {
      d.fac2 = fac_elems;
      fac_elems += front_fac2_size(d.nc);
    }
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
auto& g_l0_cache = *new std::map<std::tuple<int, int, int, int, int>, std::shared_ptr<Level0>>();

std::shared_ptr<const Level0> get_level0(const Geometry& G, bool two_sided) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, G.dim, G.n, G.leaf, two_sided ? 1 : 0);
  std::lock_guard<std::mutex> lock(g_l0_mutex);
  auto it = g_l0_cache.find(key);
  if (it != g_l0_cache.end()) return it->second;
  auto L0 = std::make_shared<Level0>();
  std::vector<int> alive(G.N);
  for (int64_t g = 0; g < G.N; ++g) alive[g] = (int)g;
  build_cells(G, 0, alive, L0->cells);
  std::vector<int> cip;
  prepare_cells(G, 0, L0->cells, nullptr, L0->cdesc, cip, L0->work_elems, L0->fac_elems, L0->max_nI, two_sided);
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
                 L0->max_nN, two_sided);
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
      split_big(h, sw, ad, st);
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
    if (h->two_sided) {   // every cell by the one-block LU kernel
      launch_cell_lu<U>(d_cd, nullptr, (int)cd.size(), work, fac, status.as<int>(), st);
      return;
    }
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
    std::shared_ptr<const Level0> L0 = get_level0(G, h->two_sided);
    h->level0 = L0;

    // ---- level 0: the cached structure
    DevBuf work, prev_work;
    {
      SweepLevel& sw = h->cells[0];
      work.alloc((size_t)L0->work_elems * sizeof(T), st);
      sw.fac.alloc((size_t)L0->fac_elems * sizeof(T), st);
      const int nc0 = (int)L0->cdesc.size();
      launch_leaf_assemble<T>(L0->d_cdesc, nc0, L0->d_cipool, work.as<T>(), h->gi, h->a_stag.as<double>(),
                              h->bnode.as<double>(), L0->d_cls0, G.ncell[0], h->two_sided ? h->beta : nullptr, st);
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
      prepare_cells(G, l, cells, prev_cells, cdesc, ipool, work_elems, fac_elems, max_nI, h->two_sided);
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
      if (!is_root) split_big(h, sw, ad, st);
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
        prepare_fronts(*fr, *fd, ip, fw, ff, fo, mnc, mnN, h->two_sided);
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
    DevBuf d_ccell, d_cptr, d_clist;
    if (h->skel == HIF_SKEL_SVD || h->two_sided) big.clear();   // every front by a one-block kernel
    const int nbig = (int)big.size();
    const int nm = nbig ? bigfront_colmax_blocks(big_nc) : 0;
    if (h->two_sided) {
      launch_front_lu<T>(d_fd, nf, d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(), cwork.as<T>(),
                         h->eps, status.as<int>(), max_nc, max_nN, st);
    } else if (h->skel == HIF_SKEL_SVD) {
      // the fronts' SVDs from the update matrices as they stand, then each
      // bordering cell's update matrix rotated by its fronts
      std::map<int, std::vector<int>> by_cell;   // cell -> (front, side) pairs
      for (int f = 0; f < nf; ++f) {
        const HostFront& F = (*fr)[f];
        for (int t = 0; t < fd[f].nc; ++t)
          if (F.pos1[t] < 0 || F.pos2[t] < 0)
            throw HifError(HIF_ERR_ARG, "HIF_SKEL_SVD: a front without two bordering cells");
        by_cell[fd[f].P1].insert(by_cell[fd[f].P1].end(), {f, 1});
        by_cell[fd[f].P2].insert(by_cell[fd[f].P2].end(), {f, 2});
      }
      std::vector<int> ccell, cptr{0}, clist;
      for (const auto& kv : by_cell) {
        ccell.push_back(kv.first);
        clist.insert(clist.end(), kv.second.begin(), kv.second.end());
        cptr.push_back((int)(clist.size() / 2));
      }
      upload(d_ccell, ccell, st);
      upload(d_cptr, cptr, st);
      upload(d_clist, clist, st);
      launch_front_svd<T>(d_fd, nf, d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(), cwork.as<T>(),
                          h->eps, status.as<int>(), max_nc, tau, st);
      launch_svd_rotate<T>(d_ccell.as<int>(), d_cptr.as<int>(), d_clist.as<int>(), (int)ccell.size(), d_fd,
                           d_cdesc, d_ip, obuf.as<int>(), fwork.as<T>(), sw.fac.as<T>(), cwork.as<T>(), max_nc, st);
    } else if (big.empty()) {
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
      const bool rot = h->skel == HIF_SKEL_SVD && k > 0 && nR > 0;   // the SVD's rotation V (T's slot)
      a.V = rot ? a.T : -1;
      if (d.fac2 >= 0) {   // two-sided
        a.Linv2 = d.fac2;
        a.G2 = d.fac2 + packed_size(d.nc);
        a.L2 = a.G2 + pad4((int64_t)d.nc * d.nc);
      }
      sw.max_np = std::max(sw.max_np, nR);
      sw.max_nq = std::max(sw.max_nq, k);
      if (nR > 0) {
        sw.fac_elems += 0.5 * nR * (nR + 1.0) + (rot ? 1.0 * k * nR + (double)d.nc * d.nc : 2.0 * k * nR);
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
    split_big(h, sw, ad, st);
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

}  // namespace

extern "C" {

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
    if (opts && opts->big_apply != 0) h->big_apply = opts->big_apply < 0 ? 0 : opts->big_apply;
    h->two_sided = opts && opts->two_sided != 0;
    if (h->two_sided) {
      if (grid->variant == HIF_VARIANT_HIFDE3X) throw HifError(HIF_ERR_ARG, "two_sided: not with HIFDE3X");
      if (prec == HIF_PREC_MIXED) throw HifError(HIF_ERR_ARG, "two_sided: FP64 or FP32_APPLY precision only");
      if ((opts->id_mode != HIF_ID_QR) || opts->skel != HIF_SKEL_ID)
        throw HifError(HIF_ERR_ARG, "two_sided: the pivoted-QR ID only");
      for (int a = 0; a < 3; ++a) {
        const double bv = a < grid->dim ? opts->beta[a] : 0.0;
        if (!std::isfinite(bv)) throw HifError(HIF_ERR_ARG, "two_sided: beta must be finite");
        h->beta[a] = bv;
      }
      h->big_cell = 0x7fffffff;   // one-block kernels everywhere
      h->big_apply = 0;
    } else if (opts && (opts->beta[0] != 0.0 || opts->beta[1] != 0.0 || opts->beta[2] != 0.0)) {
      throw HifError(HIF_ERR_ARG, "beta (a convection term) needs two_sided");
    }
    h->skel = opts ? opts->skel : HIF_SKEL_ID;
    if (h->skel != HIF_SKEL_ID && h->skel != HIF_SKEL_SVD) throw HifError(HIF_ERR_ARG, "unknown skel");
    if (h->skel == HIF_SKEL_SVD) {
      if (grid->variant == HIF_VARIANT_HIFDE3X)
        throw HifError(HIF_ERR_ARG, "HIF_SKEL_SVD: not with HIFDE3X (the rotated DOFs have no single position)");
      if (prec == HIF_PREC_MIXED) throw HifError(HIF_ERR_ARG, "HIF_SKEL_SVD: FP64 or FP32_APPLY precision only");
      if (h->id_mode != HIF_ID_QR) throw HifError(HIF_ERR_ARG, "HIF_SKEL_SVD excludes the randomized ID");
    }
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
    if (h->root_size >= kRootMulti && !h->two_sided)   // (two-sided: the one-block root sweep)
      h->root_scratch.alloc(sizeof(double) * (size_t)root_scratch_elems(h->root_size, h->deterministic), h->st);
    {   // scratch of the levels' large blocks (F^-1 by many thread blocks)
      int64_t big = 0;
      for (auto* v : {&h->cells, &h->fronts, &h->edges})
        for (const SweepLevel& S : *v) big = std::max(big, S.big_scr);
      if (big > 0) h->big_scratch.alloc(sizeof(double) * (size_t)big, h->st);
    }
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

}  // extern "C"
