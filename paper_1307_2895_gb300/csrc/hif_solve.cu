// Krylov drivers with F^-1 as the preconditioner (CG with a double-double
// iterate and residual, flexible GMRES), the power-iteration error
// estimates of Section 5, and hif_solve / hif_solve_batch / hif_estimate /
// hif_matvec / hif_set_solver.
#include "hif_host.h"

namespace {

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
      const long long k0 = hif_kernel_launches();
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
      graph_kernels = hif_kernel_launches() - k0;   // the kernels one replay runs
      note_launches(-graph_kernels);                 // recorded, not run, by the capture
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
    note_launches(graph_kernels);   // the launch counter counts every kernel a replay runs
    if (h->profile) {
      CU(cudaEventRecord(h->ev_pool[h->ev_used + 1], h->st));
      h->ev_used += 2;
      ++pending_graphs;
    }
    CU(cudaGetLastError());
  }
  int pending_graphs = 0;
  long long graph_kernels = 0;
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

int hif_estimate(hif_handle* h, const double* x0, double rtol, int maxit, double* e_a, double* e_s) {
  if (!h || !x0 || !e_a || !e_s) return set_error(HIF_ERR_ARG, "NULL argument");
  if (h->beta[0] != 0.0 || h->beta[1] != 0.0 || h->beta[2] != 0.0)
    return set_error(HIF_ERR_ARG, "hif_estimate: the stencil products here have no convection term (beta != 0)");
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
  if (h->beta[0] != 0.0 || h->beta[1] != 0.0 || h->beta[2] != 0.0)
    return set_error(HIF_ERR_ARG, "hif_matvec: the stencil products here have no convection term (beta != 0)");
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
int hif_solve(hif_handle* h, const double* rhs, double* x, double* x_lo, int nrhs, int ld, double tol,
              int maxit, hif_solve_info* info) {
  if (!h || !rhs || !x) return set_error(HIF_ERR_ARG, "NULL argument");
  if (h->beta[0] != 0.0 || h->beta[1] != 0.0 || h->beta[2] != 0.0)
    return set_error(HIF_ERR_ARG, "hif_solve: the stencil products here have no convection term (beta != 0)");
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

int hif_set_solver(hif_handle* h, int solver, int restart) {
  if (!h) return set_error(HIF_ERR_ARG, "NULL handle");
  if (solver < HIF_SOLVER_AUTO || solver > HIF_SOLVER_GMRES) return set_error(HIF_ERR_ARG, "unknown solver");
  if (restart != 0 && (restart < 2 || restart > 500)) return set_error(HIF_ERR_ARG, "need 2 <= restart <= 500");
  h->solver = solver;
  h->gmres_m = restart == 0 ? 50 : restart;
  return HIF_OK;
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

}  // extern "C"
