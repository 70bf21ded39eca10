// F^-1 and F (Eq. 4.2) on packed vectors: the level-by-level sweep launches,
// the sweep autotuner, the FP32 copy of the factor, and hif_apply /
// hif_profile / hif_autotune_table.
#include "hif_host.h"

namespace hif {
namespace host {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// apply of F^-1 / F on a packed N x nrhs work vector of the factor's type
// ---------------------------------------------------------------------------
void split_big(hif_handle* h, SweepLevel& sw, const std::vector<ApplyDesc>& ad, cudaStream_t st) {
  sw.nbig = sw.nsmall = 0;
  sw.big_scr = 0;
  if (h->big_apply <= 0 || h->deterministic) return;
  std::vector<ApplyDesc> small;
  std::vector<BigBlock> big;
  int snp = 0, snq = 0, bnp = 0, bnq = 0;
  int64_t scr = 0;
  for (const ApplyDesc& a : ad) {
    const int64_t elems = (int64_t)a.np * ((int64_t)a.np + 2 * (int64_t)a.nq);
    if (a.np > 0 && a.V < 0 && elems >= h->big_apply) {   // (SVD fronts: one block each)
      big.push_back(BigBlock{a, scr});
      scr += 2 * (int64_t)a.np * kBigChunk;
      bnp = std::max(bnp, a.np);
      bnq = std::max(bnq, a.nq);
    } else {
      small.push_back(a);
      snp = std::max(snp, a.np);
      snq = std::max(snq, a.nq);
    }
  }
  if (big.empty()) return;
  upload(sw.small_desc, small, st);
  upload(sw.big_desc, big, st);
  sw.nsmall = (int)small.size();
  sw.small_max_np = snp;
  sw.small_max_nq = snq;
  sw.nbig = (int)big.size();
  sw.big_max_np = bnp;
  sw.big_max_nq = bnq;
  sw.big_scr = scr;
}

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

// The launch's blocks: desc[0..nblocks) with ids in ipool, largest np / nq.
struct SweepBlocks {
  const ApplyDesc* desc;
  int nblocks;
  const int* ipool;
  int max_np, max_nq;
};

template <typename T>
SweepShape tuned_shape(hif_handle* h, int op, const SweepBlocks& S, int is_front, const T* fac, const T* x,
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
    // F^-1 with large blocks: those by the many-block kernels, the others as usual
    const bool big = (op == 0 || op == 1) && S.nbig > 0 && h->big_scratch.p;
    const SweepBlocks B = big ? SweepBlocks{S.small_desc.as<ApplyDesc>(), S.nsmall, S.ipool, S.small_max_np,
                                            S.small_max_nq}
                              : SweepBlocks{S.desc, S.nblocks, S.ipool, S.max_np, S.max_nq};
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
    if (B.nblocks > 0) {
      const SweepShape shape = (h->autotune && mode == HIF_APPLY_FINV)
                                   ? tuned_shape<T>(h, op, B, is_front, fac, x, nrhs, cpp)
                                   : SweepShape{};
      launch_sweep<T>(op, B.desc, B.nblocks, B.ipool, fac, x, nrhs, nrhs, is_front, B.max_np, B.max_nq,
                      h->dev_err.as<int>(), st, shape, cpp);
    }
    int nl_big = 0;
    if (big)
      nl_big = launch_big_sweep<T>(op, S.big_desc.as<BigBlock>(), S.nbig, S.big_max_np, S.big_max_nq, is_front,
                                   S.ipool, fac, x, nrhs, nrhs, h->big_scratch.as<T>(), S.big_scr, st);
    if (prof) {
      CU(cudaEventRecord(h->ev_pool[h->ev_used + 1], st));
      h->ev_used += 2;
    }
    if (count) {
      h->prof_launches += (B.nblocks > 0 ? 1 : 0) + nl_big;
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


template void run_apply<float>(hif_handle*, int, float*, int);
template void run_apply<double>(hif_handle*, int, double*, int);

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

}  // namespace host
}  // namespace hif

extern "C" {

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


}  // extern "C"
