// C ABI: errors, handle release, statistics and structure, boundary data,
// the bounded-wait self-test and the rank-predictor (MLP) entry points.  The
// factorization, the apply and the solvers are in hif_factor.cu,
// hif_apply.cu and hif_solve.cu.
#include "hif_host.h"

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void hif::note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }


namespace hif {
namespace host {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int run_batch(int nprob, int nthreads, const std::function<int(int)>& task) {
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

}  // namespace host
}  // namespace hif

void hif::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

extern "C" {
long long hif_kernel_launches(void) { return g_launches.load(); }


const char* hif_last_error(void) { return g_last_error.c_str(); }

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
